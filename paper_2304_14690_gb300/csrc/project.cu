// Per-call kernels of the pressure-correction sub-step and the pc_project / pc_solve_poisson
// entry points (§2.3; Eqs. 4, 18-20).
//
//  prep        u~ = u* + dt f~ (Eq. 20 right-hand side combined into one transferred field);
//              mixed precision keeps u~ as an unevaluated FP32 pair (hi, lo)
//  transfer    U_face = sum_k W_k u~_k (WLS value rows); FP64, or FP32 with compensated
//              products and sums (TwoProduct by fma, TwoSum; Dekker 1971, Knuth) in mixed mode
//  divergence  s = D_h U / (beta dt), with the sums of s and s^2 for the compatibility mean
//  residual    r = s - mean - L_h p in FP64 (refinement sweeps of the mixed solve)
//  gauge       p -= mean(p) (or p at the corner cell) when the problem is singular
//  gradient    g = sum_k D_k p_k at every node, then Eq. 4 at fluid nodes and Eqs. 18-19 at
//              boundary/virtual nodes
//  check       max |D_h (U - beta dt G_h p)| (only when statistics are requested)
#include <cmath>
#include <cstdio>
#include <cstring>

#include "pc_internal.cuh"

namespace pc {

pc_status solve_fp32_grid(Plan *p, int src_mode, const void *s, int dst_mode, double *pout,
                          cudaStream_t st);
pc_status solve_fp64_grid(Plan *p, const double *s, double *pout, cudaStream_t st);

enum { SRC_F32_ = 0, SRC_F64_ = 1 };
enum { DST_F64_SET_ = 1, DST_F64_ADD_ = 2 };

// ----------------------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
// Block-wide sum added atomically to *dst (blockDim.x a multiple of 32, <= 1024).
__device__ void block_sum_add(double v, double *dst) {
  __shared__ double sh[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) atomicAdd(dst, v);
  }
}
__device__ void block_max_update(double v, double *dst) {
  __shared__ double sh[32];
  v = warp_max(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    v = warp_max(v);
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)__double_as_longlong(v));
  }
}

// ----------------------------------------------------------------------------- prep
template <typename VT>
__device__ __forceinline__ double ld(const VT *p, long long i) { return (double)p[i]; }

// u~ = u* + dt f~; FP64 copy (fp64 path) or (hi, lo) FP32 pair (mixed). Also max |u*|.
template <typename VT>
__global__ void prep_kernel(long long count, const VT *u, const VT *f, double dt, double *ut64,
                            float *uhi, float *ulo, DevStats *stats) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (i < count) {
    double v = ld(u, i);
    m = fabs(v);
    if (f) v = fma(dt, ld(f, i), v);
    if (ut64) ut64[i] = v;
    if (uhi) {
      float hi = (float)v;
      uhi[i] = hi;
      ulo[i] = (float)(v - (double)hi);
    }
  }
  block_max_update(m, &stats->max_u);
}

// ----------------------------------------------------------------------------- transfer
__global__ void transfer64_kernel(long long rows, int K, const int32_t *__restrict__ col,
                                  const double *__restrict__ w, const double *__restrict__ u,
                                  double *__restrict__ U) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) {
    long long at = (long long)k * rows + r;
    acc = fma(w[at], u[col[at]], acc);
  }
  U[r] = acc;
}

// Compensated dot product in FP32 arithmetic: (whi + wlo) . (uhi + ulo) accumulated as an
// unevaluated pair; products by TwoProduct (fma), sums by TwoSum.
struct DF { float hi, lo; };
__device__ __forceinline__ void df_acc(DF &s, float whi, float wlo, float uhi, float ulo) {
  float p = whi * uhi;
  float e = fmaf(whi, uhi, -p);
  e = fmaf(whi, ulo, e);
  e = fmaf(wlo, uhi, e);
  float t = s.hi + p;
  float z = t - s.hi;
  float err = (s.hi - (t - z)) + (p - z);
  s.hi = t;
  s.lo += err + e;
}

__global__ void transfer_mixed_kernel(long long rows, int K, const int32_t *__restrict__ col,
                                      const float *__restrict__ whi, const float *__restrict__ wlo,
                                      const float *__restrict__ uhi, const float *__restrict__ ulo,
                                      double *__restrict__ U) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  DF s{0.f, 0.f};
  for (int k = 0; k < K; ++k) {
    long long at = (long long)k * rows + r;
    int c = col[at];
    df_acc(s, whi[at], wlo[at], uhi[c], ulo[c]);
  }
  U[r] = (double)s.hi + (double)s.lo;
}

// ----------------------------------------------------------------------------- grid geometry
struct GridDev {
  int dim;
  int n[3];
  int nf[3];          // faces along each axis (n or n+1)
  int periodic[3];
  int lo_kind[3], hi_kind[3];   // 0 Neumann, 1 Dirichlet (ghost sign), ignored when periodic
  double inv_h[3], inv_h2[3];
};

__device__ __forceinline__ void unflat(const GridDev &g, long long c, int *i) {
  for (int a = g.dim - 1; a >= 0; --a) { i[a] = (int)(c % g.n[a]); c /= g.n[a]; }
}
// Linear index of face (i with i[axis] replaced by fi) in the face array of `axis`.
__device__ __forceinline__ long long face_index(const GridDev &g, int axis, const int *i, int fi) {
  long long f = 0;
  for (int a = 0; a < g.dim; ++a) {
    int extent = (a == axis) ? g.nf[a] : g.n[a];
    int v = (a == axis) ? fi : i[a];
    f = f * extent + v;
  }
  return f;
}
__device__ __forceinline__ long long cell_index(const GridDev &g, const int *i) {
  long long c = 0;
  for (int a = 0; a < g.dim; ++a) c = c * g.n[a] + i[a];
  return c;
}

// s = D_h U / (beta dt), plus sum(s), sum(s^2).
__global__ void divergence_kernel(GridDev g, long long ncells, const double *U0, const double *U1,
                                  const double *U2, double inv_bdt, double *s, DevStats *stats) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (c < ncells) {
    int i[3];
    unflat(g, c, i);
    const double *U[3] = {U0, U1, U2};
    double acc = 0.0;
    for (int a = 0; a < g.dim; ++a) {
      int hi = i[a] + 1;
      if (g.periodic[a] && hi == g.n[a]) hi = 0;
      double d = U[a][face_index(g, a, i, hi)] - U[a][face_index(g, a, i, i[a])];
      acc += d * g.inv_h[a];
    }
    v = acc * inv_bdt;
    s[c] = v;
  }
  block_sum_add(v, &stats->sum_s);
  block_sum_add(v * v, &stats->sum_s2);
}

__global__ void sum_kernel(long long count, const double *x, double *sum, double *sum2) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = (c < count) ? x[c] : 0.0;
  block_sum_add(v, sum);
  if (sum2) block_sum_add(v * v, sum2);
}

// L_h p at cell i (ghost rules: Neumann p_ghost = p_edge, Dirichlet -p_edge, periodic wrap).
__device__ __forceinline__ double lap_at(const GridDev &g, const double *p, const int *i, double pc) {
  double acc = 0.0;
  int j[3] = {i[0], i[1], i[2]};
  for (int a = 0; a < g.dim; ++a) {
    double pl, pr;
    if (i[a] > 0) { j[a] = i[a] - 1; pl = p[cell_index(g, j)]; }
    else if (g.periodic[a]) { j[a] = g.n[a] - 1; pl = p[cell_index(g, j)]; }
    else pl = g.lo_kind[a] ? -pc : pc;
    if (i[a] < g.n[a] - 1) { j[a] = i[a] + 1; pr = p[cell_index(g, j)]; }
    else if (g.periodic[a]) { j[a] = 0; pr = p[cell_index(g, j)]; }
    else pr = g.hi_kind[a] ? -pc : pc;
    j[a] = i[a];
    acc = fma((pl + pr) - 2.0 * pc, g.inv_h2[a], acc);
  }
  return acc;
}

// r = s - mean(s) - L_h p in FP64, stored as FP32 for the next FP32 solve; adds ||r||^2.
__global__ void residual_kernel(GridDev g, long long ncells, const double *s, const double *p,
                                int singular, float *r, DevStats *stats, double *res2) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (c < ncells) {
    int i[3] = {0, 0, 0};
    unflat(g, c, i);
    double pc = p[c];
    double mean = singular ? stats->sum_s / (double)ncells : 0.0;
    v = (s[c] - mean) - lap_at(g, p, i, pc);
    if (r) r[c] = (float)v;
  }
  block_sum_add(v * v, res2);
}

__global__ void gauge_sum_kernel(long long ncells, const double *p, DevStats *stats) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = (c < ncells) ? p[c] : 0.0;
  if (c == 0) stats->corner_p = v;
  block_sum_add(v, &stats->sum_p);
}

// p -= shift (gauge), and the (hi, lo) FP32 split of p for the compensated gradient.
__global__ void finalize_p_kernel(long long ncells, double *p, int gauge_mode, const DevStats *stats,
                                  float *phi, float *plo) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  double shift = 0.0;
  if (gauge_mode == 1) shift = stats->sum_p / (double)ncells;
  else if (gauge_mode == 2) shift = stats->corner_p;
  double v = p[c] - shift;
  p[c] = v;
  if (phi) {
    float hi = (float)v;
    phi[c] = hi;
    plo[c] = (float)(v - (double)hi);
  }
}

// ----------------------------------------------------------------------------- gradient
template <typename VT>
__device__ __forceinline__ void store_v(VT *p, long long i, double v) { p[i] = (VT)v; }

template <typename VT, int DIM>
__global__ void gradient64_kernel(long long N, int K, const int32_t *__restrict__ col,
                                  const double *__restrict__ D, const double *__restrict__ p,
                                  const uint8_t *__restrict__ type, const VT *__restrict__ u,
                                  double dt, double beta, VT *__restrict__ uo, VT *__restrict__ fo) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double g[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) g[a] = 0.0;
  for (int k = 0; k < K; ++k) {
    double pv = p[col[(long long)k * N + i]];
#pragma unroll
    for (int a = 0; a < DIM; ++a) g[a] = fma(D[((long long)a * K + k) * N + i], pv, g[a]);
  }
  const bool ib = type[i] != PC_NODE_FLUID;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double us = (double)u[(long long)a * N + i];
    if (ib) {
      store_v(uo, (long long)a * N + i, 0.0);
      if (fo) store_v(fo, (long long)a * N + i, -us / dt + beta * g[a]);
    } else {
      store_v(uo, (long long)a * N + i, us - beta * dt * g[a]);
      if (fo) store_v(fo, (long long)a * N + i, 0.0);
    }
  }
}

template <typename VT, int DIM>
__global__ void gradient_mixed_kernel(long long N, int K, const int32_t *__restrict__ col,
                                      const float *__restrict__ Dhi, const float *__restrict__ Dlo,
                                      const float *__restrict__ phi, const float *__restrict__ plo,
                                      const uint8_t *__restrict__ type, const VT *__restrict__ u,
                                      double dt, double beta, VT *__restrict__ uo, VT *__restrict__ fo) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  DF g[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) g[a] = DF{0.f, 0.f};
  for (int k = 0; k < K; ++k) {
    int c = col[(long long)k * N + i];
    float ph = phi[c], pl = plo[c];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      long long at = ((long long)a * K + k) * N + i;
      df_acc(g[a], Dhi[at], Dlo[at], ph, pl);
    }
  }
  const bool ib = type[i] != PC_NODE_FLUID;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double ga = (double)g[a].hi + (double)g[a].lo;
    double us = (double)u[(long long)a * N + i];
    if (ib) {
      store_v(uo, (long long)a * N + i, 0.0);
      if (fo) store_v(fo, (long long)a * N + i, -us / dt + beta * ga);
    } else {
      store_v(uo, (long long)a * N + i, us - beta * dt * ga);
      if (fo) store_v(fo, (long long)a * N + i, 0.0);
    }
  }
}

// ----------------------------------------------------------------------------- check
// max over cells of |D_h (U - beta dt G_h p)|; wall faces carry no flux and no gradient.
__global__ void div_check_kernel(GridDev g, long long ncells, const double *U0, const double *U1,
                                 const double *U2, const double *p, double bdt, DevStats *stats) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (c < ncells) {
    int i[3] = {0, 0, 0};
    unflat(g, c, i);
    const double *U[3] = {U0, U1, U2};
    double pc = p[c];
    double acc = 0.0;
    int j[3] = {i[0], i[1], i[2]};
    for (int a = 0; a < g.dim; ++a) {
      // gradient on the low and high faces of the cell
      double pl, pr;
      if (i[a] > 0) { j[a] = i[a] - 1; pl = p[cell_index(g, j)]; }
      else if (g.periodic[a]) { j[a] = g.n[a] - 1; pl = p[cell_index(g, j)]; }
      else pl = g.lo_kind[a] ? -pc : pc;
      if (i[a] < g.n[a] - 1) { j[a] = i[a] + 1; pr = p[cell_index(g, j)]; }
      else if (g.periodic[a]) { j[a] = 0; pr = p[cell_index(g, j)]; }
      else pr = g.hi_kind[a] ? -pc : pc;
      j[a] = i[a];
      int hi = i[a] + 1;
      if (g.periodic[a] && hi == g.n[a]) hi = 0;
      double Ulo = U[a][face_index(g, a, i, i[a])] - bdt * (pc - pl) * g.inv_h[a];
      double Uhi = U[a][face_index(g, a, i, hi)] - bdt * (pr - pc) * g.inv_h[a];
      acc += (Uhi - Ulo) * g.inv_h[a];
    }
    v = fabs(acc);
  }
  block_max_update(v, &stats->max_div);
}

// ----------------------------------------------------------------------------- host
static GridDev grid_dev(const Plan *p) {
  GridDev g{};
  g.dim = p->dim;
  for (int a = 0; a < 3; ++a) {
    if (a < p->dim) {
      const AxisInfo &ax = p->ax[a];
      g.n[a] = ax.n;
      g.nf[a] = ax.nfaces;
      g.periodic[a] = ax.periodic;
      g.lo_kind[a] = ax.bc_lo == PC_BC_DIRICHLET;
      g.hi_kind[a] = ax.bc_hi == PC_BC_DIRICHLET;
      g.inv_h[a] = 1.0 / ax.h;
      g.inv_h2[a] = 1.0 / (ax.h * ax.h);
    } else {
      g.n[a] = 1;
      g.nf[a] = 1;
    }
  }
  return g;
}

static bool is_device_ptr(const void *ptr) {
  if (!ptr) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Grid-level solve: s64 (device) -> p (device, FP64), gauge applied; fills dstats fields.
static pc_status solve_grid(Plan *p, const double *s64, double *pout, bool want_final_residual,
                            cudaStream_t st) {
  const long long nc = p->ncells;
  const int T = 256;
  GridDev g = grid_dev(p);
  if (p->precision == PC_PREC_FP64) {
    PC_TRY(solve_fp64_grid(p, s64, pout, st));
    prof_mark(p, st, 3);
  } else {
    int sweeps = (p->precision == PC_PREC_MIXED) ? p->refine_iters : 0;
    PC_TRY(solve_fp32_grid(p, SRC_F64_, s64, DST_F64_SET_, pout, st));
    prof_mark(p, st, 3);
    for (int it = 0; it < sweeps; ++it) {
      float *r32 = reinterpret_cast<float *>(p->work64);   // work64 is free in mixed mode
      residual_kernel<<<grid_for(nc, T), T, 0, st>>>(g, nc, s64, pout, p->singular, r32, p->dstats,
                                                     &p->dstats->res2[it]);
      count_launch(p);
      prof_mark(p, st, 4);
      PC_TRY(solve_fp32_grid(p, SRC_F32_, r32, DST_F64_ADD_, pout, st));
      prof_mark(p, st, 3);
    }
  }
  if (want_final_residual) {
    int it = (p->precision == PC_PREC_MIXED) ? p->refine_iters : 0;
    residual_kernel<<<grid_for(nc, T), T, 0, st>>>(g, nc, s64, pout, p->singular, nullptr, p->dstats,
                                                   &p->dstats->res2[it]);
    count_launch(p);
    prof_mark(p, st, 7);
  }
  // gauge (singular problems), then the FP32 split of p for the mixed gradient
  int gmode = p->singular ? (p->gauge == 1 ? 2 : 1) : 0;
  if (gmode) {
    gauge_sum_kernel<<<grid_for(nc, T), T, 0, st>>>(nc, pout, p->dstats);
    count_launch(p);
  }
  bool mixed = p->precision != PC_PREC_FP64;
  if (gmode || mixed) {
    finalize_p_kernel<<<grid_for(nc, T), T, 0, st>>>(nc, pout, gmode, p->dstats, mixed ? p->phi : nullptr,
                                                     mixed ? p->plo : nullptr);
    count_launch(p);
  }
  prof_mark(p, st, 5);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

static pc_status fill_stats(Plan *p, pc_stats *stats, cudaStream_t st) {
  DevStats ds;
  PC_CUDA_TRY(cudaMemcpyAsync(&ds, p->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, st));
  PC_CUDA_TRY(cudaStreamSynchronize(st));
  memset(stats, 0, sizeof(*stats));
  const double nc = (double)p->ncells;
  stats->removed_mean = p->singular ? ds.sum_s / nc : 0.0;
  stats->source_norm = std::sqrt(fmax(ds.sum_s2, 0.0));
  int its = (p->precision == PC_PREC_MIXED) ? p->refine_iters : 0;
  for (int i = 0; i <= its && i < 9; ++i) stats->residual_norm[i] = std::sqrt(fmax(ds.res2[i], 0.0));
  stats->refine_iters_done = its;
  stats->max_div_after = ds.max_div;
  stats->max_abs_u_star = ds.max_u;
  int gmode = p->singular ? (p->gauge == 1 ? 2 : 1) : 0;
  stats->gauge_shift = gmode == 1 ? ds.sum_p / nc : (gmode == 2 ? ds.corner_p : 0.0);
  return PC_OK;
}

static pc_status project_impl(Plan *p, double dt, const void *u_star, const void *f_in, double *p_out,
                              void *u_out, void *f_out, pc_stats *stats, cudaStream_t st) {
  const int d = p->dim;
  const long long N = p->N, nc = p->ncells;
  const size_t vsz = p->vdtype == PC_DTYPE_F64 ? 8 : 4;
  const size_t vbytes = (size_t)d * N * vsz;
  // host pointers are staged through plan buffers
  const bool hu = !is_device_ptr(u_star), hf = !is_device_ptr(f_in), hp = !is_device_ptr(p_out),
             huo = !is_device_ptr(u_out), hfo = !is_device_ptr(f_out);
  const void *du = u_star, *df = f_in;
  double *dp = p_out;
  void *duo = u_out, *dfo = f_out;
  if (hu) { PC_CUDA_TRY(cudaMemcpyAsync(p->stage_u, u_star, vbytes, cudaMemcpyHostToDevice, st)); du = p->stage_u; }
  if (f_in && hf) { PC_CUDA_TRY(cudaMemcpyAsync(p->stage_f, f_in, vbytes, cudaMemcpyHostToDevice, st)); df = p->stage_f; }
  if (hp) dp = p->stage_p;
  if (huo) duo = p->stage_uo;
  if (f_out && hfo) dfo = p->stage_fo;

  prof_begin(p, st);
  PC_CUDA_TRY(cudaMemsetAsync(p->dstats, 0, sizeof(DevStats), st));
  const int T = 256;
  const bool mixed = p->precision != PC_PREC_FP64;
  const long long cnt = (long long)d * N;
  if (p->vdtype == PC_DTYPE_F64)
    prep_kernel<double><<<grid_for(cnt, T), T, 0, st>>>(cnt, (const double *)du, (const double *)df, dt,
                                                         mixed ? nullptr : p->ut64, mixed ? p->uhi : nullptr,
                                                         mixed ? p->ulo : nullptr, p->dstats);
  else
    prep_kernel<float><<<grid_for(cnt, T), T, 0, st>>>(cnt, (const float *)du, (const float *)df, dt,
                                                        mixed ? nullptr : p->ut64, mixed ? p->uhi : nullptr,
                                                        mixed ? p->ulo : nullptr, p->dstats);
  count_launch(p);
  prof_mark(p, st, 0);
  for (int a = 0; a < d; ++a) {
    long long rows = p->nface_total[a];
    if (mixed)
      transfer_mixed_kernel<<<grid_for(rows, T), T, 0, st>>>(rows, p->K, p->fcol[a], p->fwhi[a], p->fwlo[a],
                                                             p->uhi + (long long)a * N, p->ulo + (long long)a * N,
                                                             p->U64[a]);
    else
      transfer64_kernel<<<grid_for(rows, T), T, 0, st>>>(rows, p->K, p->fcol[a], p->fw64[a],
                                                         p->ut64 + (long long)a * N, p->U64[a]);
    count_launch(p);
  }
  prof_mark(p, st, 1);
  GridDev g = grid_dev(p);
  divergence_kernel<<<grid_for(nc, T), T, 0, st>>>(g, nc, p->U64[0], p->U64[1], p->U64[2], 1.0 / (p->beta * dt),
                                                   p->s64, p->dstats);
  count_launch(p);
  prof_mark(p, st, 2);
  PC_CUDA_TRY(cudaGetLastError());
  PC_TRY(solve_grid(p, p->s64, dp, stats != nullptr, st));
  const void *ug = du;
  if (p->vdtype == PC_DTYPE_F64) {
    if (mixed) {
      if (d == 2) gradient_mixed_kernel<double, 2><<<grid_for(N, T), T, 0, st>>>(N, p->Kg, p->ncol, p->nDhi, p->nDlo, p->phi, p->plo, p->ntype, (const double *)ug, dt, p->beta, (double *)duo, (double *)dfo);
      else gradient_mixed_kernel<double, 3><<<grid_for(N, T), T, 0, st>>>(N, p->Kg, p->ncol, p->nDhi, p->nDlo, p->phi, p->plo, p->ntype, (const double *)ug, dt, p->beta, (double *)duo, (double *)dfo);
    } else {
      if (d == 2) gradient64_kernel<double, 2><<<grid_for(N, T), T, 0, st>>>(N, p->Kg, p->ncol, p->nD64, dp, p->ntype, (const double *)ug, dt, p->beta, (double *)duo, (double *)dfo);
      else gradient64_kernel<double, 3><<<grid_for(N, T), T, 0, st>>>(N, p->Kg, p->ncol, p->nD64, dp, p->ntype, (const double *)ug, dt, p->beta, (double *)duo, (double *)dfo);
    }
  } else {
    if (mixed) {
      if (d == 2) gradient_mixed_kernel<float, 2><<<grid_for(N, T), T, 0, st>>>(N, p->Kg, p->ncol, p->nDhi, p->nDlo, p->phi, p->plo, p->ntype, (const float *)ug, dt, p->beta, (float *)duo, (float *)dfo);
      else gradient_mixed_kernel<float, 3><<<grid_for(N, T), T, 0, st>>>(N, p->Kg, p->ncol, p->nDhi, p->nDlo, p->phi, p->plo, p->ntype, (const float *)ug, dt, p->beta, (float *)duo, (float *)dfo);
    } else {
      if (d == 2) gradient64_kernel<float, 2><<<grid_for(N, T), T, 0, st>>>(N, p->Kg, p->ncol, p->nD64, dp, p->ntype, (const float *)ug, dt, p->beta, (float *)duo, (float *)dfo);
      else gradient64_kernel<float, 3><<<grid_for(N, T), T, 0, st>>>(N, p->Kg, p->ncol, p->nD64, dp, p->ntype, (const float *)ug, dt, p->beta, (float *)duo, (float *)dfo);
    }
  }
  count_launch(p);
  prof_mark(p, st, 6);
  if (stats) {
    div_check_kernel<<<grid_for(nc, T), T, 0, st>>>(g, nc, p->U64[0], p->U64[1], p->U64[2], dp, p->beta * dt,
                                                    p->dstats);
    count_launch(p);
    prof_mark(p, st, 7);
  }
  PC_CUDA_TRY(cudaGetLastError());
  if (hp) PC_CUDA_TRY(cudaMemcpyAsync(p_out, dp, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (huo) PC_CUDA_TRY(cudaMemcpyAsync(u_out, duo, vbytes, cudaMemcpyDeviceToHost, st));
  if (f_out && hfo) PC_CUDA_TRY(cudaMemcpyAsync(f_out, dfo, vbytes, cudaMemcpyDeviceToHost, st));
  if (stats) PC_TRY(fill_stats(p, stats, st));
  if (hp || huo || (f_out && hfo)) PC_CUDA_TRY(cudaStreamSynchronize(st));
  return PC_OK;
}

static pc_status solve_impl(Plan *p, const double *s, double *p_out, pc_stats *stats, cudaStream_t st) {
  const long long nc = p->ncells;
  const bool hs = !is_device_ptr(s), hp = !is_device_ptr(p_out);
  const double *ds = s;
  double *dp = p_out;
  if (hs) { PC_CUDA_TRY(cudaMemcpyAsync(p->stage_s, s, nc * sizeof(double), cudaMemcpyHostToDevice, st)); ds = p->stage_s; }
  if (hp) dp = p->stage_p;
  prof_begin(p, st);
  PC_CUDA_TRY(cudaMemsetAsync(p->dstats, 0, sizeof(DevStats), st));
  sum_kernel<<<grid_for(nc, 256), 256, 0, st>>>(nc, ds, &p->dstats->sum_s, &p->dstats->sum_s2);
  count_launch(p);
  prof_mark(p, st, 2);
  PC_TRY(solve_grid(p, ds, dp, stats != nullptr, st));
  if (hp) PC_CUDA_TRY(cudaMemcpyAsync(p_out, dp, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (stats) PC_TRY(fill_stats(p, stats, st));
  if (hp) PC_CUDA_TRY(cudaStreamSynchronize(st));
  return PC_OK;
}

}  // namespace pc

extern "C" pc_status pc_project(pc_plan *plan, double dt, const void *u_star, const void *f_ib_in,
                                double *p_out, void *u_out, void *f_ib_out, pc_stats *stats,
                                void *cuda_stream) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  if (!u_star || !p_out || !u_out) return pc::fail(PC_ERR_INVALID_ARG, "u_star, p_out and u_out are required");
  if (!(dt > 0.0) || !std::isfinite(dt)) return pc::fail(PC_ERR_INVALID_ARG, "dt must be positive and finite");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) {
    if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device %d", p->device);
  }
  return pc::project_impl(p, dt, u_star, f_ib_in, p_out, u_out, f_ib_out, stats, (cudaStream_t)cuda_stream);
}

extern "C" pc_status pc_solve_poisson(pc_plan *plan, const double *s, double *p_out, pc_stats *stats,
                                      void *cuda_stream) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p || !s || !p_out) return pc::fail(PC_ERR_INVALID_ARG, "plan, s and p_out are required");
  if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device %d", p->device);
  return pc::solve_impl(p, s, p_out, stats, (cudaStream_t)cuda_stream);
}

extern "C" pc_status pc_project_batch(int count, pc_plan *const *plans, const pc_project_args *args,
                                      void *cuda_stream) {
  if (count < 0 || (count > 0 && (!plans || !args))) return pc::fail(PC_ERR_INVALID_ARG, "bad batch arguments");
  for (int i = 0; i < count; ++i) {
    pc_status s = pc_project(plans[i], args[i].dt, args[i].u_star, args[i].f_ib_in, args[i].p_out,
                             args[i].u_out, args[i].f_ib_out, nullptr, cuda_stream);
    if (s != PC_OK) return s;
  }
  return PC_OK;
}
