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
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <vector>

#include "numeric.cuh"
#include "pc_internal.cuh"

namespace pc {

enum { SRC_F32_ = 0, SRC_F64_ = 1 };
enum { DST_F64_SET_ = 1, DST_F64_ADD_ = 2, DST_PAIR_SET_ = 3, DST_PAIR_ADD_ = 4 };

// ----------------------------------------------------------------------------- block context
// Kernels address their block through a VBlock: the hardware block in a single-problem launch,
// or the problem-local block of a batched launch (one launch for many problems, batch.cu).
struct VBlock {
  unsigned x, y, z, nx, ny, nz;
};
__device__ __forceinline__ VBlock hw_block() {
  return VBlock{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z};
}

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
// Deterministic grid-wide sum: every block writes its partial (fixed shuffle tree), the last
// block to finish sums all partials in block order and writes *dst, then resets the counter.
// Results are bitwise reproducible, unlike concurrent floating-point atomics. Inside a block the
// sum runs in double-float FP32 arithmetic (TwoSum; Knuth) on the exact FP32 split of each
// value, so the FP64 pipe sees one add per block instead of a shuffle tree per thread; the
// relative error stays below about 2^-44 of the sum of magnitudes.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}
__device__ __forceinline__ void df_add(float &hi, float &lo, float bhi, float blo) {
  float s, e;
  two_sum(hi, bhi, s, e);
  e += lo + blo;
  hi = s + e;
  lo = e - (hi - s);
}
__device__ __forceinline__ void warp_sum_df(float &hi, float &lo) {
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
    df_add(hi, lo, h2, l2);
  }
}
__device__ bool grid_sum(double v, double *partials, unsigned int *counter, double *dst, const VBlock &vb) {
  __shared__ float2 sh[32];
  __shared__ bool last;
  const unsigned nblk = vb.nx * vb.ny * vb.nz;
  const unsigned bid = vb.x + vb.nx * (vb.y + vb.ny * vb.z);
  float hi, lo;
  split_f64(v, hi, lo);
  warp_sum_df(hi, lo);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = make_float2(hi, lo);
  __syncthreads();
  if (wid == 0) {
    const float2 w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : make_float2(0.f, 0.f);
    hi = w.x;
    lo = w.y;
    warp_sum_df(hi, lo);
    if (lane == 0) {
      partials[bid] = f2d_bits(hi) + f2d_bits(lo);
      __threadfence();
      last = atomicAdd(counter, 1u) == nblk - 1;
    }
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // The whole last block sums the partials: thread t takes partials t, t + blockDim, ... in
  // order, then a fixed shuffle tree and the warp totals in warp order (deterministic).
  __shared__ double shw[32];
  double t = 0.0;
  for (unsigned b = threadIdx.x; b < nblk; b += blockDim.x) t += __ldcg(partials + b);
  t = warp_sum(t);
  if (lane == 0) shw[wid] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += shw[w];
    *dst = tot;
    *counter = 0u;
    return true;
  }
  return false;
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

__device__ __forceinline__ double as_f64(double v) { return v; }
__device__ __forceinline__ double as_f64(float v) { return f2d_bits(v); }

// u~ = u* + dt f~; FP64 copy (FP64 path, SPLIT = false) or (hi, lo) FP32 pair (mixed). Compile-
// time variants keep the common case (no force, no statistics) free of FP64 arithmetic.
// Element kernels over a flat array: each thread takes kFlatPerThread elements, 256 apart.
constexpr int kFlatThreads = 256;
constexpr int kFlatPerThread = 4;
constexpr int kFlatPerBlock = kFlatThreads * kFlatPerThread;

template <typename VT, bool HAS_F, bool STATS, bool SPLIT>
__device__ __forceinline__ void prep_kernel_body(unsigned b, long long count, const VT *__restrict__ u, const VT *__restrict__ f, double dt,
                            double *__restrict__ ut64, float2 *__restrict__ u2, DevStats *stats) {
  double m = 0.0;
#pragma unroll
  for (int k = 0; k < kFlatPerThread; ++k) {
    const long long i = (long long)b * kFlatPerBlock + k * kFlatThreads + threadIdx.x;
    if (i < count) {
      const VT ui = u[i];
      if (STATS) m = fmax(m, fabs(as_f64(ui)));
      if (HAS_F) {
        double v = fma(dt, as_f64(f[i]), as_f64(ui));
        if (SPLIT) u2[i] = as_pair(v);
        else ut64[i] = v;
      } else {
        if (SPLIT) u2[i] = as_pair(ui);
        else ut64[i] = as_f64(ui);
      }
    }
  }
  if (STATS) block_max_update(m, &stats->max_u);
}
template <typename VT, bool HAS_F, bool STATS, bool SPLIT>
__global__ void prep_kernel(long long count, const VT *__restrict__ u, const VT *__restrict__ f, double dt,
                            double *__restrict__ ut64, float2 *__restrict__ u2, DevStats *stats) {
  pdl_enter();
  prep_kernel_body<VT, HAS_F, STATS, SPLIT>(blockIdx.x, count, u, f, dt, ut64, u2, stats);
}

template <typename VT>
static void launch_prep(bool has_f, bool stats, bool split, long long cnt, const VT *u, const VT *f, double dt,
                        double *ut64, float2 *u2, DevStats *ds, cudaStream_t st) {
  const int T = kFlatThreads;
  const int G = grid_for(cnt, kFlatPerBlock);
#define PC_PREP(F, S, P) launch_pdl(prep_kernel<VT, F, S, P>, G, T, 0, st, cnt, u, f, dt, ut64, u2, ds)
  if (has_f) {
    if (stats) { if (split) PC_PREP(true, true, true); else PC_PREP(true, true, false); }
    else { if (split) PC_PREP(true, false, true); else PC_PREP(true, false, false); }
  } else {
    if (stats) { if (split) PC_PREP(false, true, true); else PC_PREP(false, true, false); }
    else { if (split) PC_PREP(false, false, true); else PC_PREP(false, false, false); }
  }
#undef PC_PREP
}

// ----------------------------------------------------------------------------- transfer
// Value row r of the face array (rows faces, neighbour-rank-major weights) applied to u~.
__device__ __forceinline__ double transfer64_row(int r, int rows, int K, const int32_t *__restrict__ col,
                                                 const double *__restrict__ w, const double *__restrict__ u) {
  double acc = 0.0;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const long long at = (long long)k * rows + r;
    acc = fma(__ldcs(w + at), __ldg(u + __ldcs(col + at)), acc);
  }
  return acc;
}
__global__ void transfer64_kernel(int rows, int K, const int32_t *__restrict__ col,
                                  const double *__restrict__ w, const double *__restrict__ u,
                                  double *__restrict__ U) {
  pdl_enter();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  U[r] = transfer64_row(r, rows, K, col, w, u);
}


// KC > 0: the neighbour count is a compile-time constant and the loop is unrolled, so all
// index and weight loads are in flight before the dependent gathers (memory-level parallelism).
// The gathered node value as an FP32 (hi, lo) pair, here the pairs of u~ that prep wrote.
struct PairSrc {
  const float2 *p;
  __device__ __forceinline__ float2 operator()(int c) const { return __ldg(p + c); }
};

template <int KC, typename Src>
__device__ __forceinline__ double transfer_mixed_row(int r, int rows, int Kr, const int32_t *__restrict__ col,
                                                     const float2 *__restrict__ w2, Src src) {
  const int K = KC > 0 ? KC : Kr;
  DF s{0.f, 0.f};
  if (KC > 0) {
    int c[KC > 0 ? KC : 1];
    float2 w[KC > 0 ? KC : 1];
#pragma unroll
    for (int k = 0; k < K; ++k) {   // read once: streamed past the caches that hold the gathered values
      c[k] = __ldcs(col + (long long)k * rows + r);
      w[k] = __ldcs(w2 + (long long)k * rows + r);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) df_acc(s, w[k], src(c[k]));
  } else {
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const long long at = (long long)k * rows + r;
      df_acc(s, __ldcs(w2 + at), src(__ldcs(col + at)));
    }
  }
  return df_value(s);
}
template <int KC, typename Src>
__device__ __forceinline__ void transfer_mixed_kernel_body(const VBlock &vb, int rows, int Kr, const int32_t *__restrict__ col,
                                      const float2 *__restrict__ w2, Src src,
                                      double *__restrict__ U) {
  int r = vb.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  U[r] = transfer_mixed_row<KC>(r, rows, Kr, col, w2, src);
}
template <int KC, typename Src>
__global__ void transfer_mixed_kernel(int rows, int Kr, const int32_t *__restrict__ col,
                                      const float2 *__restrict__ w2, Src src, double *__restrict__ U) {
  pdl_enter();
  transfer_mixed_kernel_body<KC>(hw_block(), rows, Kr, col, w2, src, U);
}

// ----------------------------------------------------------------------------- grid geometry
// Cell kernels view the grid as g.rows rows of the last axis. A block of 256 threads covers
// 2^tw_bits positions of the last axis times 2^th_bits thread rows, and every thread walks
// g.cr consecutive rows, so the fixed cost of a block (problem lookup, reductions) is spread
// over 256 * cr cells. The launch is one-dimensional: block b is tile (b % gx, b / gx). The
// kernels are templated on the dimension and unroll their axis loops, so the small index
// arrays stay in registers.

// Column of this thread and its first row in block b.
__device__ __forceinline__ void tile_pos(const GridDev &g, unsigned b, int &x, int &row0) {
  const int t = threadIdx.x;
  const int by = (int)(b / (unsigned)g.gx);
  const int bx = (int)b - by * g.gx;
  x = (bx << g.tw_bits) + (t & ((1 << g.tw_bits) - 1));
  row0 = ((by << g.th_bits) + (t >> g.tw_bits)) * g.cr;
}
// Multi-index of cell (row, x).
template <int DIM>
__device__ __forceinline__ void cell_at(const GridDev &g, int row, int x, int *i) {
  if (DIM == 2) { i[0] = row; i[1] = x; i[2] = 0; return; }
  const int i0 = row / g.n[1];
  i[0] = i0; i[1] = row - i0 * g.n[1]; i[2] = x;
}
__device__ __forceinline__ int cell_index(const GridDev &g, const int *i) {
  return i[0] * g.cs[0] + i[1] * g.cs[1] + i[2] * g.cs[2];
}
// Linear index of face fi along `axis` with the other coordinates of cell i.
__device__ __forceinline__ int face_index(const GridDev &g, int axis, const int *i, int fi) {
  int f = 0;
#pragma unroll
  for (int b = 0; b < 3; ++b) f += ((b == axis) ? fi : i[b]) * g.fs[axis][b];
  return f;
}
__device__ __forceinline__ VBlock tile_block(const GridDev &g, unsigned b) {
  return VBlock{b, 0u, 0u, (unsigned)g.nblk, 1u, 1u};
}

// ----------------------------------------------------------------------------- double-float
// Unevaluated FP32 pairs (hi + lo, struct DF above) with error-free transformations (Knuth's TwoSum, Dekker's
// product through fma); the _rn intrinsics keep the compiler from contracting them.
__device__ __forceinline__ DF df_of(double v) {
  DF r;
  split_f64(v, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float z = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return DF{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float h = __fadd_rn(p, e);
  return DF{h, __fsub_rn(e, __fsub_rn(h, p))};
}

// ----------------------------------------------------------------------------- divergence
// s = D_h U / (beta dt) (FP64; as an FP32 pair in double-float arithmetic on the mixed path),
// its FP32 copy; want_sums 1: sum(s) and the mean, 2: also sum(s^2) (statistics).
template <int DIM>
__device__ __forceinline__ void divergence_body(unsigned b, const GridDev &g, const double *U0, const double *U1,
                                                const double *U2, double inv_bdt, double *s, float2 *s2, float *s32,
                                                DevStats *stats, double *partials, unsigned int *counter,
                                                int want_sums, double inv_ncells) {
  int x, row0;
  tile_pos(g, b, x, row0);
  const double *U[3] = {U0, U1, U2};
  double c[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) c[a] = g.inv_h[a] * inv_bdt;
  double sum = 0.0, sum2 = 0.0;
  if (s2 && x < g.n[DIM - 1]) {
    // mixed path: the source is kept as an FP32 pair, so it is formed in double-float arithmetic
    // (FP32 operations with error-free transformations, about 48 bits) from the FP64 faces: the
    // FP64 pipe runs at a small fraction of the FP32 rate on this GPU
    DF cd[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) cd[a] = df_of(c[a]);
    DF sd{0.0f, 0.0f}, sd2{0.0f, 0.0f};
    const int rend = min(row0 + g.cr, g.rows);
    for (int row = row0; row < rend; ++row) {
      int i[3];
      cell_at<DIM>(g, row, x, i);
      DF v{0.0f, 0.0f};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        int hi = i[a] + 1;
        if (g.periodic[a] && hi == g.n[a]) hi = 0;
        const DF d = df_sub(df_of(U[a][face_index(g, a, i, hi)]), df_of(U[a][face_index(g, a, i, i[a])]));
        v = (a == 0) ? df_mul(d, cd[0]) : df_add(v, df_mul(d, cd[a]));
      }
      const int ci = cell_index(g, i);
      if (g.mask && !g.mask[ci]) v = DF{0.0f, 0.0f};   // outside the flow domain (RHS mask)
      s2[ci] = make_float2(v.hi, v.lo);
      if (s32) s32[ci] = v.hi;   // FP32 copy read by the first FP32 transform pass
      if (want_sums) sd = df_add(sd, v);
      if (want_sums > 1) sd2 = df_add(sd2, df_mul(v, v));
    }
    sum = f2d_bits(sd.hi) + f2d_bits(sd.lo);
    sum2 = f2d_bits(sd2.hi) + f2d_bits(sd2.lo);
  } else if (x < g.n[DIM - 1]) {
    const int rend = min(row0 + g.cr, g.rows);
    for (int row = row0; row < rend; ++row) {
      int i[3];
      cell_at<DIM>(g, row, x, i);
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        int hi = i[a] + 1;
        if (g.periodic[a] && hi == g.n[a]) hi = 0;
        const double d = U[a][face_index(g, a, i, hi)] - U[a][face_index(g, a, i, i[a])];
        v = (a == 0) ? d * c[0] : fma(d, c[a], v);
      }
      const int ci = cell_index(g, i);
      if (g.mask && !g.mask[ci]) v = 0.0;   // outside the flow domain (RHS mask)
      if (s2) s2[ci] = as_pair(v);     // the refinement keeps s as a (hi, lo) pair
      else s[ci] = v;
      if (s32) s32[ci] = d2f_rz_bits(v);   // FP32 copy read by the first FP32 transform pass
      if (want_sums) sum += v;
      if (want_sums > 1) sum2 = fma(v, v, sum2);
    }
  }
  if (want_sums) {
    const VBlock vb = tile_block(g, b);
    if (grid_sum(sum, partials, counter, &stats->sum_s, vb)) stats->mean_s = stats->sum_s * inv_ncells;
    if (want_sums > 1) grid_sum(sum2, partials + g.nblk, counter + 1, &stats->sum_s2, vb);
  }
}

template <int DIM>
__global__ void divergence_kernel(GridDev g, const double *U0, const double *U1, const double *U2,
                                  double inv_bdt, double *s, float2 *s2, float *s32, DevStats *stats,
                                  double *partials, unsigned int *counter, int want_sums, double inv_ncells) {
  pdl_enter();
  divergence_body<DIM>(blockIdx.x, g, U0, U1, U2, inv_bdt, s, s2, s32, stats, partials, counter, want_sums,
                       inv_ncells);
}

// Direct divergence (PC_DIV_WLS_DIRECT): s = (1/(beta dt)) sum_a sum_k D_a,k u~_a,k at every
// cell centre from the cell derivative rows ([K][cells] columns, [dim][K][cells] weights), one
// cell per thread, FP64 (u~ in ut64) or compensated FP32 (pairs of weights and u~). Zero outside
// the RHS mask; the same outputs and sums as the face divergence.
template <int DIM, bool MIXED>
__global__ void direct_div_kernel(int nc, int K, const int32_t *__restrict__ col, const double *__restrict__ D,
                                  const float2 *__restrict__ D2, const double *__restrict__ ut64,
                                  const float2 *__restrict__ u2, int N, double inv_bdt, const uint8_t *__restrict__ mask,
                                  double *s, float2 *s2, float *s32, DevStats *stats, double *partials,
                                  unsigned int *counter, int want_sums, double inv_ncells) {
  pdl_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (c < nc) {
    if (MIXED) {
      DF acc{0.f, 0.f};
      for (int k = 0; k < K; ++k) {
        const int j = __ldcs(col + (long long)k * nc + c);
#pragma unroll
        for (int a = 0; a < DIM; ++a)
          df_acc(acc, __ldcs(D2 + ((long long)a * K + k) * nc + c), __ldg(u2 + (long long)a * N + j));
      }
      v = df_value(acc) * inv_bdt;
    } else {
      double acc = 0.0;
      for (int k = 0; k < K; ++k) {
        const int j = __ldcs(col + (long long)k * nc + c);
#pragma unroll
        for (int a = 0; a < DIM; ++a)
          acc = fma(__ldcs(D + ((long long)a * K + k) * nc + c), __ldg(ut64 + (long long)a * N + j), acc);
      }
      v = acc * inv_bdt;
    }
    if (mask && !mask[c]) v = 0.0;
    if (s2) s2[c] = as_pair(v);
    else s[c] = v;
    if (s32) s32[c] = d2f_rz_bits(v);
  }
  if (want_sums) {
    const VBlock vb = hw_block();
    if (grid_sum(v, partials, counter, &stats->sum_s, vb)) stats->mean_s = stats->sum_s * inv_ncells;
    if (want_sums > 1) grid_sum(v * v, partials + gridDim.x, counter + 1, &stats->sum_s2, vb);
  }
}

// ----------------------------------------------------------------------------- flat kernels
// Weights of the mean of a vertex grid with N-N axes: the DCT-I basis is orthogonal in the
// trapezoid inner product (weight 1/2 at both end vertices of each such axis), so the part of
// the source outside the range of the operator (the compatibility constant) and the constant
// part of a solution are means in those weights. dim = 0: unit weights (cell grids).
struct TrapWeights {
  int dim;
  int n[3];      // points per axis (C order, last axis fastest)
  int trap[3];   // 1: N-N vertex axis
  double total;  // sum of the weights
};
__device__ __forceinline__ double trap_weight(const TrapWeights &w, long long c) {
  double wt = 1.0;
#pragma unroll
  for (int a = 2; a >= 0; --a) {   // constant indices: the weights stay in registers
    if (a >= w.dim) continue;
    const long long q = c / w.n[a];
    const int i = (int)(c - q * w.n[a]);
    c = q;
    if (w.trap[a] && (i == 0 || i == w.n[a] - 1)) wt *= 0.5;
  }
  return wt;
}

// Sum (weighted, see TrapWeights) and sum of squares of a cell array (the source of
// pc_solve_poisson), and its mean.
__device__ __forceinline__ void sum_kernel_body(unsigned b, unsigned nblk, long long count, const double *x,
                                                DevStats *stats, double *partials, unsigned int *counter,
                                                const TrapWeights &w) {
  double v1 = 0.0, v2 = 0.0;
#pragma unroll
  for (int k = 0; k < kFlatPerThread; ++k) {
    const long long c = (long long)b * kFlatPerBlock + k * kFlatThreads + threadIdx.x;
    if (c < count) {
      const double v = x[c];
      v1 += w.dim ? trap_weight(w, c) * v : v;
      v2 = fma(v, v, v2);
    }
  }
  const VBlock vb{b, 0u, 0u, nblk, 1u, 1u};
  if (grid_sum(v1, partials, counter, &stats->sum_s, vb))
    stats->mean_s = stats->sum_s / (w.dim ? w.total : (double)count);
  grid_sum(v2, partials + nblk, counter + 1, &stats->sum_s2, vb);
}

__global__ void sum_kernel(long long count, const double *x, DevStats *stats, double *partials,
                           unsigned int *counter, TrapWeights w) {
  pdl_enter();
  sum_kernel_body(blockIdx.x, gridDim.x, count, x, stats, partials, counter, w);
}

// ----------------------------------------------------------------------------- residual
// The two neighbours of cell c along axis a (ghost rules at the domain boundary: Neumann
// p_ghost = p_edge, Dirichlet -p_edge, periodic wrap).
__device__ __forceinline__ void neighbours(const GridDev &g, const double *p, const int *i, int c,
                                           int a, double pc, double &pl, double &pr) {
  const int st = g.cs[a];
  if (i[a] > 0) pl = p[c - st];
  else if (g.periodic[a]) pl = p[c + (g.n[a] - 1) * st];
  else pl = g.lo_kind[a] ? -pc : pc;
  if (i[a] < g.n[a] - 1) pr = p[c + st];
  else if (g.periodic[a]) pr = p[c - (g.n[a] - 1) * st];
  else pr = g.hi_kind[a] ? -pc : pc;
}

// A stored value as a double-float pair: FP64 values are split exactly as split_f64 does,
// pairs are taken as they are.
__device__ __forceinline__ DF to_df(double v) { return df_of(v); }
__device__ __forceinline__ DF to_df(float2 v) { return DF{v.x, v.y}; }
__device__ __forceinline__ DF df_neg_(DF a) { return DF{-a.hi, -a.lo}; }
// Ghost value beyond a non-periodic end (GridDev lo_kind / hi_kind): from the edge value dc, or
// the value at inner (the next point inward, which the end mirrors on a vertex grid).
template <typename PV>
__device__ __forceinline__ DF ghost_df(int kind, DF dc, const PV *__restrict__ p, int inner) {
  if (kind == 0) return dc;
  if (kind == 1) return df_neg_(dc);
  if (kind == 2) return to_df(p[inner]);
  return DF{0.0f, 0.0f};
}

// r = s - mean(s) - L_h p, evaluated in double-float arithmetic (about 48 significant bits:
// the FP64 pipe of this GPU runs at 1/64 of the FP32 rate) and stored as FP32 for the next
// FP32 solve; optionally ||r||^2. The refinement converges to the solution of this residual,
// so its ~2^-44 relative rounding bounds the attainable accuracy far below the 1e-10 target.
// SV, PV: storage of s and p, double or a float2 (hi, lo) pair (the refinement keeps both as
// pairs; FP64 arrays come from pc_solve_poisson and from the statistics of FP64 plans).
// Refinement step of a residual launch: k sweeps are done before it. With rule set (the
// stopping rule is on), the launch does nothing once a residual before it ended the refinement
// (refine_stopped_before, checked by the kernel: rule 1 by the single-problem kernel, rule 2 by a
// caller that already did), and otherwise records the max norm of r_k (and, for k = 0, of s)
// for the rule; tol: the rule's tolerance.
struct RefineStep {
  int k, rule;
  float tol;
  int chunk;   // single-problem launches: consecutive blocks per CTA (0 or 1: one)
};

// Refinement runs under the stopping rule (MIXED with refine_tol > 0 and sweeps allowed): every
// residual records its max norm, the kernels of a sweep that the rule ended exit at once, and
// every solve writes p in FP64 since any of them may be the last.
constexpr int kLateChunk = 8;
static bool refine_adaptive(const Plan *p) {
  return p->precision == PC_PREC_MIXED && p->refine_tol > 0.0 && p->refine_iters > 0;
}

// Block-wide maximum of non-negative v merged into *dst with one atomic maximum of its bits (the
// order of the blocks does not matter, so the result is reproducible).
__device__ __forceinline__ void block_max_bits(float v, float *dst) {
  __shared__ float sh[32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) atomicMax(reinterpret_cast<unsigned *>(dst), __float_as_uint(v));
  }
}

template <int DIM, bool SINGULAR, bool WRITE_R, bool NORM, typename SV, typename PV>
__device__ __forceinline__ void residual_body(unsigned b, const GridDev &g, const SV *__restrict__ s,
                                              const PV *__restrict__ p, float *__restrict__ r,
                                              DevStats *stats, double *res2, double *partials,
                                              unsigned int *counter, RefineStep rs, float &rmx_acc,
                                              float &smx_acc) {
  int x, row0;
  tile_pos(g, b, x, row0);
  double nrm = 0.0;
  float rmx = 0.0f, smx = 0.0f;
  if (x < g.n[DIM - 1]) {
    DF mean{0.0f, 0.0f};
    if (SINGULAR) mean = df_of(stats->mean_s);
    const int rend = min(row0 + g.cr, g.rows);
    for (int row = row0; row < rend; ++row) {
      int i[3];
      cell_at<DIM>(g, row, x, i);
      const int c = cell_index(g, i);
      const DF dc = to_df(p[c]);
      DF acc{0.0f, 0.0f};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        // neighbours with the ghost rules: Neumann p_ghost = p_edge, Dirichlet -p_edge (cell
        // grids), the next value inward (Neumann about a vertex), 0 (Dirichlet vertex), periodic wrap
        const int st = g.cs[a];
        DF pl, pr;
        if (i[a] > 0) pl = to_df(p[c - st]);
        else if (g.periodic[a]) pl = to_df(p[c + (g.n[a] - 1) * st]);
        else pl = ghost_df(g.lo_kind[a], dc, p, c + st);
        if (i[a] < g.n[a] - 1) pr = to_df(p[c + st]);
        else if (g.periodic[a]) pr = to_df(p[c - (g.n[a] - 1) * st]);
        else pr = ghost_df(g.hi_kind[a], dc, p, c - st);
        // the differences first: pl - dc and pr - dc cancel before any rounding of the sum
        // (forming pl + pr first raised the refinement floor: p 9.4e-13 from the FP64 path on
        // the channel instead of 1.5e-14)
        const DF t = df_add(df_sub(pl, dc), df_sub(pr, dc));
        acc = df_add(acc, df_mul(t, DF{g.ih2_hi[a], g.ih2_lo[a]}));
      }
      DF sc = to_df(s[c]);
      if (rs.rule && rs.k == 0) smx = fmaxf(smx, fabsf(sc.hi));
      if (SINGULAR) sc = df_sub(sc, mean);
      const DF v = df_sub(sc, acc);
      if (WRITE_R) r[c] = v.hi;
      if (rs.rule) rmx = fmaxf(rmx, fabsf(v.hi));
      if (NORM) {
        const double vd = f2d_bits(v.hi) + f2d_bits(v.lo);
        nrm = fma(vd, vd, nrm);
      }
    }
  }
  rmx_acc = fmaxf(rmx_acc, rmx);
  smx_acc = fmaxf(smx_acc, smx);
  if (NORM) grid_sum(nrm, partials, counter, res2, tile_block(g, b));
}
// The rule's max norms of a CTA's blocks, merged once per CTA (a maximum is exact and
// order-independent, so the grouping of blocks does not change it).
__device__ __forceinline__ void residual_record(const RefineStep &rs, float rmx, float smx, DevStats *stats) {
  if (!rs.rule) return;
  block_max_bits(rmx, &stats->rmax[rs.k]);
  if (rs.k == 0) block_max_bits(smx, &stats->smax);
}
// CTA b evaluates blocks b * rs.chunk, ... of the grid's decomposition (the residual per cell,
// its max norm and its L2 partial per block do not depend on how blocks are grouped).
template <int DIM, bool SINGULAR, bool WRITE_R, bool NORM, typename SV, typename PV>
__global__ void residual_kernel(GridDev g, const SV *__restrict__ s, const PV *__restrict__ p,
                                float *__restrict__ r, DevStats *stats, double *res2,
                                double *partials, unsigned int *counter, RefineStep rs) {
  pdl_enter();
  if (rs.rule == 1 && refine_stopped_before(stats, rs.k, rs.tol)) return;   // the refinement already ended
  const int c = rs.chunk > 1 ? rs.chunk : 1;
  const int b0 = blockIdx.x * c, b1 = min(b0 + c, g.nblk);
  float rmx = 0.0f, smx = 0.0f;
  for (int b = b0; b < b1; ++b)
    residual_body<DIM, SINGULAR, WRITE_R, NORM, SV, PV>(b, g, s, p, r, stats, res2, partials, counter, rs, rmx, smx);
  residual_record(rs, rmx, smx, stats);
}

// ----------------------------------------------------------------------------- gauge
// Sum of p (weighted, see TrapWeights; and the corner value); the reducing block stores the
// gauge constant.
__device__ __forceinline__ void gauge_sum_body(unsigned b, unsigned nblk, long long ncells, const double *p,
                                               DevStats *stats, double *partials, unsigned int *counter,
                                               int gauge_mode, const TrapWeights &w) {
  DF acc{0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < kFlatPerThread; ++k) {
    const long long c = (long long)b * kFlatPerBlock + k * kFlatThreads + threadIdx.x;
    if (c < ncells) {
      double v = p[c];
      if (c == 0) stats->corner_p = v;
      if (w.dim) v *= trap_weight(w, c);   // a power of two: exact
      acc = df_add(acc, df_of(v));
    }
  }
  if (grid_sum(f2d_bits(acc.hi) + f2d_bits(acc.lo), partials, counter, &stats->sum_p, VBlock{b, 0u, 0u, nblk, 1u, 1u}))
    stats->shift = (gauge_mode == 1) ? stats->sum_p / (w.dim ? w.total : (double)ncells) : p[0];
}

__global__ void gauge_sum_kernel(long long ncells, const double *p, DevStats *stats, double *partials,
                                 unsigned int *counter, int gauge_mode, TrapWeights w) {
  pdl_enter();
  gauge_sum_body(blockIdx.x, gridDim.x, ncells, p, stats, partials, counter, gauge_mode, w);
}

// p -= shift (gauge), and the (hi, lo) FP32 split of p for the compensated gradient.
template <bool GAUGE, bool SPLIT>
__device__ __forceinline__ void finalize_p_body(unsigned b, int ncells, double *__restrict__ p,
                                                const DevStats *stats, float2 *__restrict__ p2) {
  double shift = 0.0;
  if (GAUGE) shift = stats->shift;
#pragma unroll
  for (int k = 0; k < kFlatPerThread; ++k) {
    const long long c = (long long)b * kFlatPerBlock + k * kFlatThreads + threadIdx.x;
    if (c < ncells) {
      double v = p[c];
      if (GAUGE) {
        v -= shift;
        p[c] = v;
      }
      if (SPLIT) p2[c] = as_pair(v);
    }
  }
}
template <bool GAUGE, bool SPLIT>
__global__ void finalize_p_kernel(int ncells, double *__restrict__ p, const DevStats *stats,
                                  float2 *__restrict__ p2) {
  pdl_enter();
  finalize_p_body<GAUGE, SPLIT>(blockIdx.x, ncells, p, stats, p2);
}

// ----------------------------------------------------------------------------- gradient
template <typename VT>
__device__ __forceinline__ void store_v(VT *p, long long i, double v) { p[i] = (VT)v; }

// WLS gradient of p at node i (derivative rows over the 3^d cell block).
template <int DIM>
__device__ __forceinline__ void grad64_at(int i, int N, int K, const int32_t *__restrict__ col,
                                          const double *__restrict__ D, const double *__restrict__ p, double *g) {
#pragma unroll
  for (int a = 0; a < DIM; ++a) g[a] = 0.0;
#pragma unroll 3
  for (int k = 0; k < K; ++k) {
    double pv = __ldg(p + __ldcs(col + (long long)k * N + i));
#pragma unroll
    for (int a = 0; a < DIM; ++a) g[a] = fma(__ldcs(D + ((long long)a * K + k) * N + i), pv, g[a]);
  }
}

template <typename VT, int DIM>
__global__ void gradient64_kernel(int N, int K, const int32_t *__restrict__ col,
                                  const double *__restrict__ D, const double *__restrict__ p,
                                  const uint8_t *__restrict__ type, const VT *__restrict__ u,
                                  double inv_dt, double dt, double beta, VT *__restrict__ uo,
                                  VT *__restrict__ fo, int b0) {
  pdl_enter();
  int i = (blockIdx.x + b0) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double g[DIM];
  grad64_at<DIM>(i, N, K, col, D, p, g);
  const bool ib = type[i] != PC_NODE_FLUID;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double us = (double)u[(long long)a * N + i];
    if (ib) {
      store_v(uo, (long long)a * N + i, 0.0);
      if (fo) store_v(fo, (long long)a * N + i, -us * inv_dt + beta * g[a]);
    } else {
      store_v(uo, (long long)a * N + i, us - beta * dt * g[a]);
      if (fo) store_v(fo, (long long)a * N + i, 0.0);
    }
  }
}

// Compensated WLS gradient of the split pressure at node i.
template <int DIM>
__device__ __forceinline__ void grad_mixed_at(int i, int N, const int32_t *__restrict__ col,
                                              const float2 *__restrict__ D2, const float2 *__restrict__ p2, double *gout) {
  constexpr int KB = (DIM == 2) ? 9 : 27;   // the 3^d gradient block
  DF g[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) g[a] = DF{0.f, 0.f};
  int c[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) c[k] = __ldcs(col + (long long)k * N + i);   // rows: read once, streamed
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const float2 pv = __ldg(p2 + c[k]);
#pragma unroll
    for (int a = 0; a < DIM; ++a) df_acc(g[a], __ldcs(D2 + ((long long)a * KB + k) * N + i), pv);
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) gout[a] = df_value(g[a]);
}

template <typename VT, int DIM>
__device__ __forceinline__ void gradient_mixed_kernel_body(const VBlock &vb, int N, int K, const int32_t *__restrict__ col,
                                      const float2 *__restrict__ D2, const float2 *__restrict__ p2,
                                      const uint8_t *__restrict__ type, const VT *__restrict__ u,
                                      double inv_dt, double dt, double beta, VT *__restrict__ uo,
                                      VT *__restrict__ fo) {
  int i = vb.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  (void)K;
  double g[DIM];
  grad_mixed_at<DIM>(i, N, col, D2, p2, g);
  const bool ib = type[i] != PC_NODE_FLUID;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double ga = g[a];
    double us = (double)u[(long long)a * N + i];
    if (ib) {
      store_v(uo, (long long)a * N + i, 0.0);
      if (fo) store_v(fo, (long long)a * N + i, -us * inv_dt + beta * ga);
    } else {
      store_v(uo, (long long)a * N + i, us - beta * dt * ga);
      if (fo) store_v(fo, (long long)a * N + i, 0.0);
    }
  }
}
template <typename VT, int DIM>
__global__ void gradient_mixed_kernel(int N, int K, const int32_t *__restrict__ col,
                                      const float2 *__restrict__ D2, const float2 *__restrict__ p2,
                                      const uint8_t *__restrict__ type, const VT *__restrict__ u,
                                      double inv_dt, double dt, double beta, VT *__restrict__ uo,
                                      VT *__restrict__ fo, int b0) {
  pdl_enter();
  VBlock vb = hw_block();
  vb.x += (unsigned)b0;
  gradient_mixed_kernel_body<VT, DIM>(vb, N, K, col, D2, p2, type, u, inv_dt, dt, beta, uo, fo);
}

// ----------------------------------------------------------------------------- check
// max over cells of |D_h (U - beta dt G_h p)|; wall faces carry no flux and no gradient. Cells
// outside the RHS mask are skipped.
template <int DIM>
__global__ void div_check_kernel(GridDev g, const double *U0, const double *U1,
                                 const double *U2, const double *p, double bdt, DevStats *stats) {
  pdl_enter();
  int x, row0;
  tile_pos(g, blockIdx.x, x, row0);
  const double *U[3] = {U0, U1, U2};
  double v = 0.0;
  if (x < g.n[DIM - 1]) {
    const int rend = min(row0 + g.cr, g.rows);
    for (int row = row0; row < rend; ++row) {
      int i[3];
      cell_at<DIM>(g, row, x, i);
      const int c = cell_index(g, i);
      if (g.mask && !g.mask[c]) continue;   // the source was zeroed there on purpose
      const double pc = p[c];
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        // gradient on the low and high faces of the cell
        double pl, pr;
        neighbours(g, p, i, c, a, pc, pl, pr);
        int hi = i[a] + 1;
        if (g.periodic[a] && hi == g.n[a]) hi = 0;
        const double Ulo = U[a][face_index(g, a, i, i[a])] - bdt * (pc - pl) * g.inv_h[a];
        const double Uhi = U[a][face_index(g, a, i, hi)] - bdt * (pr - pc) * g.inv_h[a];
        acc += (Uhi - Ulo) * g.inv_h[a];
      }
      v = fmax(v, fabs(acc));
    }
  }
  block_max_update(v, &stats->max_div);
}

// ----------------------------------------------------------------------------- IB-force iteration
// Kernels of pc_project_ib (§2.3). After the first pass only the force at the boundary and
// virtual nodes changes, so a pass updates u~ at those nodes, recomputes the fluxes of the
// faces whose value row reaches one of them (idx lists built once per plan), and evaluates the
// gradient and the new force (Eq. 19) at those nodes alone; the gradient at the fluid nodes is
// taken once, after the last pass. Every value is computed by the same per-row and per-node
// arithmetic as the full pass, so the iterates equal those of repeated pc_project calls.
//
// Face flags: flag[r] = 1 when row r of this face array gathers a boundary/virtual node.
__global__ void ib_face_flags_kernel(int rows, int K, const int32_t *__restrict__ col,
                                     const uint8_t *__restrict__ type, uint8_t *__restrict__ flag) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  uint8_t f = 0;
  for (int k = 0; k < K; ++k) f |= (uint8_t)(__ldg(type + __ldg(col + (long long)k * rows + r)) != PC_NODE_FLUID);
  flag[r] = f;
}

// Compact force [dim][nib] from a full [dim][N] array (nullptr: zero).
template <typename VT>
__global__ void ib_gather_kernel(int nib, int N, int dim, const int32_t *__restrict__ idx,
                                 const VT *__restrict__ f, VT *__restrict__ fc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nib) return;
  const int i = __ldg(idx + j);
  for (int a = 0; a < dim; ++a) fc[(long long)a * nib + j] = f ? f[(long long)a * N + i] : (VT)0;
}

// u~ = u* + dt f~ at the boundary/virtual nodes from the current iterate fc (the arithmetic of
// the full prep with a force), which is also saved as the previous iterate fo for the stopping
// rule before the pass overwrites fc with the new force.
template <typename VT, bool SPLIT>
__global__ void ib_prep_kernel(int nib, int N, int dim, const int32_t *__restrict__ idx,
                               const VT *__restrict__ u, const VT *__restrict__ fc, VT *__restrict__ fo,
                               double dt, double *__restrict__ ut64, float2 *__restrict__ u2) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nib) return;
  const int i = __ldg(idx + j);
  for (int a = 0; a < dim; ++a) {
    const long long at = (long long)a * N + i;
    const VT f = fc[(long long)a * nib + j];
    fo[(long long)a * nib + j] = f;
    const double v = fma(dt, as_f64(f), as_f64(u[at]));
    if (SPLIT) u2[at] = as_pair(v);
    else ut64[at] = v;
  }
}

// Fluxes of the listed faces only.
__global__ void ib_transfer64_kernel(int nl, const int32_t *__restrict__ list, int rows, int K,
                                     const int32_t *__restrict__ col, const double *__restrict__ w,
                                     const double *__restrict__ u, double *__restrict__ U) {
  pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const int r = __ldg(list + t);
  U[r] = transfer64_row(r, rows, K, col, w, u);
}
template <int KC>
__global__ void ib_transfer_mixed_kernel(int nl, const int32_t *__restrict__ list, int rows, int Kr,
                                         const int32_t *__restrict__ col, const float2 *__restrict__ w2,
                                         PairSrc src, double *__restrict__ U) {
  pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nl) return;
  const int r = __ldg(list + t);
  U[r] = transfer_mixed_row<KC>(r, rows, Kr, col, w2, src);
}

// New force at the boundary/virtual nodes (Eq. 19), compact [dim][nib].
template <typename VT, int DIM, bool MIXED>
__global__ void ib_force_kernel(int nib, const int32_t *__restrict__ idx, int N, int K,
                                const int32_t *__restrict__ col, const double *__restrict__ D,
                                const float2 *__restrict__ D2, const double *__restrict__ p,
                                const float2 *__restrict__ p2, const VT *__restrict__ u, double inv_dt,
                                double beta, VT *__restrict__ fc) {
  pdl_enter();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nib) return;
  const int i = __ldg(idx + j);
  double g[DIM];
  if (MIXED) grad_mixed_at<DIM>(i, N, col, D2, p2, g);
  else grad64_at<DIM>(i, N, K, col, D, p, g);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const double us = (double)u[(long long)a * N + i];
    store_v(fc, (long long)a * nib + j, -us * inv_dt + beta * g[a]);
  }
}

// Sums over the boundary/virtual nodes of |f_new - f_old|^2 and |f_old|^2 (deterministic: a
// fixed grid of kIbBlocks blocks, grid-stride, then the last-block reduction). The thread that
// completes the second sum applies the stopping rule of §2.3 to the means, records the pass in
// ctl and, inside the loop graph (COND), sets the condition of the while node: another pass
// unless converged or max_iters passes are done.
constexpr int kIbBlocks = 32;
template <typename VT, bool COND>
__global__ void ib_change_kernel(int nib, int dim, const VT *__restrict__ fn, const VT *__restrict__ fo,
                                 DevStats *stats, double *partials, unsigned int *counter, IbCtl *ctl,
                                 double tol, int max_iters, cudaGraphConditionalHandle cond) {
  pdl_enter();
  double d = 0.0, o = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nib; j += gridDim.x * blockDim.x)
    for (int a = 0; a < dim; ++a) {
      const double n = as_f64(fn[(long long)a * nib + j]), f = as_f64(fo[(long long)a * nib + j]);
      d = fma(n - f, n - f, d);
      o = fma(f, f, o);
    }
  const VBlock vb = hw_block();
  grid_sum(d, partials, counter, &stats->ib_diff, vb);
  if (grid_sum(o, partials + gridDim.x, counter + 1, &stats->ib_prev, vb)) {
    // every block has passed the first sum, whose total was stored before its last block
    // entered the second one (store, fence, counter) and is read past L1 here
    const double diff = __ldcg(&stats->ib_diff) / (double)nib;
    const double prev = stats->ib_prev / (double)nib;
    const int it = ctl->it;
    if (it < kIbMaxIters) {
      ctl->hist[2 * it] = diff;
      ctl->hist[2 * it + 1] = prev;
    }
    const bool conv = prev == 0.0 ? diff == 0.0 : diff <= tol * prev;
    ctl->it = it + 1;
    ctl->conv = conv ? 1 : 0;
    ctl->diff = diff;
    ctl->prev = prev;
    if (COND) cudaGraphSetConditional(cond, (!conv && it + 1 < max_iters) ? 1u : 0u);
  }
}

// Safety bound of the loop graph, independent of the stopping rule: it runs after the rule in
// every execution of the while body and clears the condition once 1 + (body executions) passes
// are done, so the loop ends after max_iters passes even if the rule's reduction never decided.
__global__ void ib_guard_kernel(IbCtl *ctl, int max_iters, cudaGraphConditionalHandle cond) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int n = ++ctl->body;
    if (n + 1 >= max_iters) cudaGraphSetConditional(cond, 0u);
  }
}

// ----------------------------------------------------------------------------- vertex grids
// A vertex grid is solved on its unknowns with the vertex transforms (DCT-I, DST-I, the
// quarter-wave bases; fft.cuh). The gradient of a pass reads p on the whole lattice, where a
// Dirichlet boundary vertex holds its known value 0.
struct VertexGrid {
  int dim;
  int nv[3];                        // unknowns per axis
  int j0[3], nf[3];                 // lattice index of the first unknown, lattice vertices
};
// Both kernels run on a grid whose x covers the last axis and whose y (and z) are the indices of
// the other axes, so no thread divides to find its position.
__device__ __forceinline__ void grid_position(int dim, int *idx) {
  if (dim == 3) {
    idx[2] = blockIdx.x * blockDim.x + threadIdx.x;
    idx[1] = blockIdx.y;
    idx[0] = blockIdx.z;
  } else {
    idx[1] = blockIdx.x * blockDim.x + threadIdx.x;
    idx[0] = blockIdx.y;
    idx[2] = 0;
  }
}
// p at the unknowns (pv) -> p on the lattice in FP64 (pl) and as FP32 (hi, lo) pairs (pl2) for
// the compensated gradient; Dirichlet boundary vertices are exactly 0.
__global__ void vertex_embed_kernel(VertexGrid V, const double *__restrict__ pv, double *__restrict__ pl,
                                    float2 *__restrict__ pl2) {
  pdl_enter();
  int idx[3];
  grid_position(V.dim, idx);
  if ((V.dim == 3 ? idx[2] : idx[1]) >= (V.dim == 3 ? V.nf[2] : V.nf[1])) return;
  int u = 0, l = 0;
  bool unknown = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= V.dim) continue;
    l = l * V.nf[a] + idx[a];
    const int ua = idx[a] - V.j0[a];
    if (ua < 0 || ua >= V.nv[a]) unknown = false;   // a Dirichlet boundary vertex
    u = u * V.nv[a] + (ua < 0 ? 0 : ua);
  }
  const double v = unknown ? pv[u] : 0.0;
  if (pl) pl[l] = v;
  if (pl2) pl2[l] = as_pair(v);
}
// Launch shape: x over the last axis, y and z over the others.
static dim3 vertex_grid_dims(int dim, const int *shape, int threads) {
  return dim3((unsigned)((shape[dim - 1] + threads - 1) / threads), (unsigned)shape[dim - 2],
              dim == 3 ? (unsigned)shape[0] : 1u);
}

static GridDev grid_dev(const Plan *p);

static VertexGrid vertex_grid(const Plan *p) {
  VertexGrid V{};
  V.dim = p->dim;
  for (int a = 0; a < 3; ++a) {
    V.nv[a] = p->nv[a];
    V.j0[a] = p->vj0[a];
    V.nf[a] = p->nf[a];
  }
  return V;
}

// Mean weights of a plan: trapezoid weights on the N-N axes of a vertex grid, else unit.
static TrapWeights trap_weights(const Plan *p) {
  TrapWeights w{};
  if (!p->vertex) return w;
  double total = 1.0;
  bool any = false;
  for (int a = 0; a < p->dim; ++a) {
    w.n[a] = p->ax[a].n;
    w.trap[a] = p->ax[a].kind == KIND_VNN;
    any |= w.trap[a] != 0;
    total *= w.trap[a] ? (double)(w.n[a] - 1) : (double)w.n[a];
  }
  if (!any) return TrapWeights{};
  w.dim = p->dim;
  w.total = total;
  return w;
}
static double mean_weight_total(const Plan *p) {
  const TrapWeights w = trap_weights(p);
  return w.dim ? w.total : (double)p->ncells;
}


// ----------------------------------------------------------------------------- batched kernels
// One launch per pipeline stage for a whole batch of problems. seg[p] is the first block of
// problem p in the launch (seg[count] = total blocks); each problem keeps exactly the block
// decomposition of its single-problem launch, so sums and results are bitwise the same.
__device__ __forceinline__ int batch_problem_of(const int *seg, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(seg + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ VBlock flat_block(int local, int nblocks) {
  return VBlock{(unsigned)local, 0u, 0u, (unsigned)nblocks, 1u, 1u};
}

__global__ void batch_zero_stats(const BatchProblem *__restrict__ P) {
  pdl_enter();
  unsigned *w = reinterpret_cast<unsigned *>(P[blockIdx.x].ds);
  for (int k = threadIdx.x; k < (int)(sizeof(DevStats) / 4); k += blockDim.x) w[k] = 0u;
}

template <typename VT>
__global__ void batch_prep(const BatchProblem *__restrict__ P, const int *__restrict__ seg, int count) {
  pdl_enter();
  const int pi = batch_problem_of(seg, count, blockIdx.x);
  const BatchProblem &q = P[pi];
  const unsigned lb = blockIdx.x - seg[pi];
  const long long cnt = (long long)q.dim * q.N;
  if (q.f) prep_kernel_body<VT, true, false, true>(lb, cnt, (const VT *)q.u, (const VT *)q.f, q.dt, nullptr, q.u2, nullptr);
  else prep_kernel_body<VT, false, false, true>(lb, cnt, (const VT *)q.u, nullptr, q.dt, nullptr, q.u2, nullptr);
}

template <int KC>
__global__ void batch_transfer(const BatchProblem *__restrict__ P, const int *__restrict__ seg, int count, int a) {
  pdl_enter();
  const int pi = batch_problem_of(seg, count, blockIdx.x);
  const BatchProblem &q = P[pi];
  const VBlock vb = flat_block(blockIdx.x - seg[pi], seg[pi + 1] - seg[pi]);
  transfer_mixed_kernel_body<KC>(vb, q.frows[a], q.K, q.fcol[a], q.fw2[a], PairSrc{q.u2 + (long long)a * q.N},
                                 q.U64[a]);
}

// Cell and residual stages of a group (one dimension per group: DIM is a template parameter).
// The problem's grid description is copied into shared memory first: its fields are then
// shared-memory operands, as a kernel parameter's are constant-bank operands in the single call.
__device__ __forceinline__ const GridDev &stage_grid(const GridDev &src) {
  __shared__ __align__(16) GridDev gs;
  const unsigned *a = reinterpret_cast<const unsigned *>(&src);
  unsigned *b = reinterpret_cast<unsigned *>(&gs);
  for (int w = threadIdx.x; w < (int)(sizeof(GridDev) / 4); w += blockDim.x) b[w] = __ldg(a + w);
  __syncthreads();
  return gs;
}
template <int DIM>
__global__ void batch_divergence(const BatchProblem *__restrict__ P, const int *__restrict__ seg, int count) {
  pdl_enter();
  const int pi = batch_problem_of(seg, count, blockIdx.x);
  const BatchProblem &q = P[pi];
  const unsigned lb = blockIdx.x - seg[pi];
  const GridDev &g = stage_grid(q.g);
  divergence_body<DIM>(lb, g, q.U64[0], q.U64[1], q.U64[2], q.inv_bdt, nullptr, reinterpret_cast<float2 *>(q.s64),
                       q.s32, q.ds, q.partials, q.counters, q.singular, q.inv_ncells);
}

// Residual k of every problem (k sweeps done). Problems under the stopping rule (tol > 0)
// record the max norm of r_k and skip the launch once the rule ended their refinement. A CTA
// evaluates kResidualChunk consecutive blocks of its problem's single-call decomposition (the
// residual per cell and its max norm do not depend on how blocks are grouped), so a skipped
// launch costs a quarter of the CTAs.
constexpr int kResidualChunk = 4;
template <int DIM>
__global__ void batch_residual(const BatchProblem *__restrict__ P, const int *__restrict__ seg, int count, int k) {
  pdl_enter();
  const int pi = batch_problem_of(seg, count, blockIdx.x);
  const BatchProblem &q = P[pi];
  const float2 *s2 = reinterpret_cast<const float2 *>(q.s64);
  const bool rule = q.tol > 0.0f;
  if (rule && refine_stopped_before(q.ds, k, q.tol)) return;
  const RefineStep rs{k, rule ? 2 : 0, q.tol, 1};
  const int b0 = (int)(blockIdx.x - seg[pi]) * kResidualChunk;
  const int b1 = min(b0 + kResidualChunk, q.g.nblk);
  float rmx = 0.0f, smx = 0.0f;
  for (int b = b0; b < b1; ++b) {
    if (q.singular) residual_body<DIM, true, true, false>(b, q.g, s2, q.p2, q.r32, q.ds, nullptr, q.partials, q.counters, rs, rmx, smx);
    else residual_body<DIM, false, true, false>(b, q.g, s2, q.p2, q.r32, q.ds, nullptr, q.partials, q.counters, rs, rmx, smx);
  }
  residual_record(rs, rmx, smx, q.ds);
}

__global__ void batch_gauge_sum(const BatchProblem *__restrict__ P, const int *__restrict__ seg, int count) {
  pdl_enter();
  const int pi = batch_problem_of(seg, count, blockIdx.x);
  const BatchProblem &q = P[pi];
  gauge_sum_body(blockIdx.x - seg[pi], seg[pi + 1] - seg[pi], q.ncells, q.p, q.ds, q.partials, q.counters, q.gmode,
                 TrapWeights{});
}

__global__ void batch_finalize(const BatchProblem *__restrict__ P, const int *__restrict__ seg, int count) {
  pdl_enter();
  const int pi = batch_problem_of(seg, count, blockIdx.x);
  const BatchProblem &q = P[pi];
  const unsigned lb = blockIdx.x - seg[pi];
  if (q.gmode) finalize_p_body<true, true>(lb, q.ncells, q.p, q.ds, q.p2);
}

template <typename VT, int DIM>
__global__ void batch_gradient(const BatchProblem *__restrict__ P, const int *__restrict__ seg, int count) {
  pdl_enter();
  const int pi = batch_problem_of(seg, count, blockIdx.x);
  const BatchProblem &q = P[pi];
  const VBlock vb = flat_block(blockIdx.x - seg[pi], seg[pi + 1] - seg[pi]);
  gradient_mixed_kernel_body<VT, DIM>(vb, q.N, q.Kg, q.ncol, q.nD2, q.p2, q.ntype, (const VT *)q.u, q.inv_dt,
                                      q.dt, q.beta, (VT *)q.uo, (VT *)q.fo);
}

// Launchers used by the batch executor (batch.cu).
void batch_launch(int stage, int variant, const BatchProblem *P, const int *seg, int count, int total_blocks,
                  int extra, cudaStream_t st) {
  if (total_blocks <= 0) return;
  const int T = 256;
  switch (stage) {
    case BATCH_ZERO: launch_pdl(batch_zero_stats, count, 64, 0, st, P); break;
    case BATCH_PREP:
      if (variant == PC_DTYPE_F64) launch_pdl(batch_prep<double>, total_blocks, T, 0, st, P, seg, count);
      else launch_pdl(batch_prep<float>, total_blocks, T, 0, st, P, seg, count);
      break;
    case BATCH_TRANSFER:
      if (variant == 12) launch_pdl(batch_transfer<12>, total_blocks, T, 0, st, P, seg, count, extra);
      else if (variant == 27) launch_pdl(batch_transfer<27>, total_blocks, T, 0, st, P, seg, count, extra);
      else launch_pdl(batch_transfer<0>, total_blocks, T, 0, st, P, seg, count, extra);
      break;
    case BATCH_DIVERGENCE:   // variant: the group's dimension
      if (variant == 3) launch_pdl(batch_divergence<3>, total_blocks, T, 0, st, P, seg, count);
      else launch_pdl(batch_divergence<2>, total_blocks, T, 0, st, P, seg, count);
      break;
    case BATCH_RESIDUAL:
      if (variant == 3) launch_pdl(batch_residual<3>, total_blocks, T, 0, st, P, seg, count, extra);
      else launch_pdl(batch_residual<2>, total_blocks, T, 0, st, P, seg, count, extra);
      break;
    case BATCH_GAUGE_SUM: launch_pdl(batch_gauge_sum, total_blocks, T, 0, st, P, seg, count); break;
    case BATCH_FINALIZE: launch_pdl(batch_finalize, total_blocks, T, 0, st, P, seg, count); break;
    case BATCH_GRADIENT:
      if (variant == 2 * 10 + PC_DTYPE_F64) launch_pdl(batch_gradient<double, 2>, total_blocks, T, 0, st, P, seg, count);
      else if (variant == 3 * 10 + PC_DTYPE_F64) launch_pdl(batch_gradient<double, 3>, total_blocks, T, 0, st, P, seg, count);
      else if (variant == 2 * 10 + PC_DTYPE_F32) launch_pdl(batch_gradient<float, 2>, total_blocks, T, 0, st, P, seg, count);
      else launch_pdl(batch_gradient<float, 3>, total_blocks, T, 0, st, P, seg, count);
      break;
  }
}

// Block counts of each stage for one problem (identical to the single-problem launches).
void batch_block_counts(const Plan *p, int *nb) {
  const long long N = p->N, nc = p->ncells;
  const GridDev g = grid_dev(p);
  nb[BATCH_ZERO] = 1;
  nb[BATCH_PREP] = grid_for((long long)p->dim * N, kFlatPerBlock);
  for (int a = 0; a < 3; ++a) nb[BATCH_TRANSFER + a] = a < p->dim ? grid_for(p->nface_total[a], 256) : 0;
  nb[BATCH_DIVERGENCE] = g.nblk;
  nb[BATCH_RESIDUAL] = (g.nblk + kResidualChunk - 1) / kResidualChunk;
  nb[BATCH_GAUGE_SUM] = p->singular ? grid_for(nc, kFlatPerBlock) : 0;
  nb[BATCH_FINALIZE] = p->singular ? grid_for(nc, kFlatPerBlock) : 0;   // else split by the last pass
  nb[BATCH_GRADIENT] = grid_for(N, 256);
}

void batch_problem_fill(const Plan *p, const pc_project_args &a, BatchProblem &q) {
  memset(&q, 0, sizeof(q));
  q.g = grid_dev(p);
  q.dim = p->dim; q.vdtype = p->vdtype; q.N = (int)p->N; q.ncells = (int)p->ncells; q.K = p->K; q.Kg = p->Kg;
  q.singular = p->singular;
  q.gmode = p->singular ? (p->gauge == 1 ? 2 : 1) : 0;
  q.kmax = p->precision == PC_PREC_MIXED ? p->refine_iters : 0;
  q.tol = refine_adaptive(p) ? (float)p->refine_tol : 0.0f;
  q.u = a.u_star; q.f = a.f_ib_in; q.uo = a.u_out; q.fo = a.f_ib_out; q.p = a.p_out;
  q.dt = a.dt; q.inv_dt = 1.0 / a.dt; q.beta = p->beta; q.inv_bdt = 1.0 / (p->beta * a.dt);
  q.inv_ncells = 1.0 / (double)p->ncells;
  q.u2 = p->u2;
  for (int k = 0; k < 3; ++k) {
    q.fcol[k] = p->fcol[k]; q.fw2[k] = p->fw2[k]; q.U64[k] = p->U64[k];
    q.frows[k] = (int)p->nface_total[k];
  }
  q.s64 = p->s64;
  q.s32 = reinterpret_cast<float *>(p->work64);
  q.r32 = reinterpret_cast<float *>(p->work64);
  q.p2 = p->p2; q.ncol = p->ncol; q.nD2 = p->nD2; q.ntype = p->ntype;
  q.ds = p->dstats; q.partials = p->partials; q.counters = p->counters;
}

// ----------------------------------------------------------------------------- host
static GridDev grid_dev(const Plan *p) {
  GridDev g{};
  g.dim = p->dim;
  g.mask = (p->rhs_mask_on && !p->vertex) ? p->rhs_mask : nullptr;   // vertex plans mask their unknowns
  for (int a = 0; a < 3; ++a) {
    if (a < p->dim) {
      const AxisInfo &ax = p->ax[a];
      g.n[a] = ax.n;
      g.nf[a] = ax.nfaces;
      g.periodic[a] = ax.periodic;
      switch (ax.kind) {   // vertex grids: 2 mirror about the end vertex, 3 the known zero
        case KIND_VNN: g.lo_kind[a] = 2; g.hi_kind[a] = 2; break;
        case KIND_VDD: g.lo_kind[a] = 3; g.hi_kind[a] = 3; break;
        case KIND_VND: g.lo_kind[a] = 2; g.hi_kind[a] = 3; break;
        case KIND_VDN: g.lo_kind[a] = 3; g.hi_kind[a] = 2; break;
        default:
          g.lo_kind[a] = ax.bc_lo == PC_BC_DIRICHLET;
          g.hi_kind[a] = ax.bc_hi == PC_BC_DIRICHLET;
      }
      g.inv_h[a] = 1.0 / ax.h;
      g.inv_h2[a] = 1.0 / (ax.h * ax.h);
      g.ih2_hi[a] = (float)g.inv_h2[a];
      g.ih2_lo[a] = (float)(g.inv_h2[a] - (double)g.ih2_hi[a]);
    } else {
      g.n[a] = 1;
      g.nf[a] = 1;
    }
  }
  // strides (C order, last axis of the problem fastest; unused padded axes have stride 0)
  int st = 1;
  for (int a = p->dim - 1; a >= 0; --a) { g.cs[a] = st; st *= g.n[a]; }
  for (int a = p->dim; a < 3; ++a) g.cs[a] = 0;
  for (int ax = 0; ax < p->dim; ++ax) {
    int fst = 1;
    for (int b = p->dim - 1; b >= 0; --b) {
      g.fs[ax][b] = fst;
      fst *= (b == ax) ? g.nf[b] : g.n[b];
    }
    for (int b = p->dim; b < 3; ++b) g.fs[ax][b] = 0;
  }
  // cell tiles: 2^tw_bits positions of the last axis (32..256) x 2^th_bits thread rows, cr = 4
  // rows per thread. The tiling depends on the grid only (not on how full the GPU is), so a
  // problem has the same blocks, and the same reduction order, alone and in a batch.
  const int nl = g.n[p->dim - 1];
  g.rows = (int)(p->ncells / nl);
  g.tw_bits = 5;
  while ((1 << g.tw_bits) < nl && g.tw_bits < 8) ++g.tw_bits;
  g.th_bits = 8 - g.tw_bits;
  g.gx = (nl + (1 << g.tw_bits) - 1) >> g.tw_bits;
  auto nblk_for = [&](int cr) {
    const long long rpb = (long long)cr << g.th_bits;
    return (long long)g.gx * ((g.rows + rpb - 1) / rpb);
  };
  g.cr = 4;
  g.nblk = (int)nblk_for(g.cr);
  return g;
}

// The same tiling with cr rows per thread. A launch whose results do not depend on its blocks
// (no grid sums: a divergence without sums) may take more, smaller blocks when it runs alone; a
// batch keeps four rows per thread.
static GridDev with_rows_per_thread(GridDev g, int cr) {
  const long long rpb = (long long)cr << g.th_bits;
  g.cr = cr;
  g.nblk = (int)((long long)g.gx * ((g.rows + rpb - 1) / rpb));
  return g;
}
constexpr int kSingleRows = 2;   // rows per thread of the sum-free single-problem divergence

// Launch shape covering every cell: x over the last axis, y/z over the others.


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
template <typename SV, typename PV>
static void launch_residual(bool singular, bool write_r, bool norm, cudaStream_t st, const GridDev &g0,
                            const SV *s, const PV *p, float *r, DevStats *ds, double *res2, double *partials,
                            unsigned int *counters, RefineStep rs = RefineStep{0, 0, 0.0f, 1}) {
  // four rows per thread, the grid's own tiling: on the 256x128x128 box it took 0.194 ms for
  // three residuals against 0.290 ms with two rows per thread (the channel is unchanged)
  const GridDev g = g0;
  const int grid = (g.nblk + (rs.chunk > 1 ? rs.chunk : 1) - 1) / (rs.chunk > 1 ? rs.chunk : 1);
#define PC_RES(S, W, N)                                                                                       \
  do {                                                                                                        \
    if (g.dim == 2)                                                                                           \
      launch_pdl(residual_kernel<2, S, W, N, SV, PV>, grid, 256, 0, st, g, s, p, r, ds, res2, partials, counters, rs); \
    else                                                                                                      \
      launch_pdl(residual_kernel<3, S, W, N, SV, PV>, grid, 256, 0, st, g, s, p, r, ds, res2, partials, counters, rs); \
  } while (0)
  if (singular) {
    if (write_r) { if (norm) PC_RES(true, true, true); else PC_RES(true, true, false); }
    else PC_RES(true, false, true);
  } else {
    if (write_r) { if (norm) PC_RES(false, true, true); else PC_RES(false, true, false); }
    else PC_RES(false, false, true);
  }
#undef PC_RES
}

// s2 (nullable): the source as (hi, lo) pairs (projections); otherwise s64 in FP64
// (pc_solve_poisson). FP32 solves keep the refinement iterate in p->p2 as (hi, lo) pairs, read
// by the residual and the gradient; the last solve also writes p in FP64 to pout.
// Gauge of the solved p: 0 none, 1 zero mean (trapezoid-weighted on the N-N axes of a vertex
// grid: no constant part in the DCT-I expansion), 2 zero first point. Problems with a zero mode
// take the plan's gauge: the refinement cannot correct the constant that FP32 rounding leaves
// (L_h of a constant is zero).
static int gauge_mode(const Plan *p) {
  if (!p->singular) return 0;
  return p->gauge == 1 ? 2 : 1;
}

static pc_status solve_grid(Plan *p, const double *s64, double *pout, bool want_final_residual,
                            cudaStream_t st, const float *s32 = nullptr, const float2 *s2 = nullptr) {
  const long long nc = p->ncells;
  const int T = kFlatThreads;
  GridDev g = grid_dev(p);
  if (p->precision == PC_PREC_FP64) {
    PC_TRY(solve_fp64_grid(p, s64, pout, st));
    prof_mark(p, st, 3);
  } else {
    const int sweeps = (p->precision == PC_PREC_MIXED) ? p->refine_iters : 0;
    const bool adaptive = refine_adaptive(p);
    const float tol = adaptive ? (float)p->refine_tol : 0.0f;
    // residual k (after k sweeps) and the solve of sweep j run only while the rule has not
    // ended the refinement at an earlier residual
    // Under the rule, sweeps beyond the second (which the rule has ended on every workload
    // measured) run with kLateChunk tiles or blocks per CTA: few CTAs, so skipping them is cheap
    auto chunk = [&](int j) { return (adaptive && j > 2) ? kLateChunk : 1; };
    auto step = [&](int k) { return RefineStep{k, adaptive ? 1 : 0, tol, chunk(k)}; };
    auto gate = [&](int j) { return adaptive ? RefineGate{p->dstats, j, tol} : RefineGate{nullptr, 0, 0.0f}; };
    const bool norm = want_final_residual;
    double *first_out = (sweeps == 0 || adaptive) ? pout : nullptr;
    if (s32) PC_TRY(solve_fp32_grid(p, SRC_F32_, s32, DST_PAIR_SET_, p->p2, st, first_out));
    else PC_TRY(solve_fp32_grid(p, SRC_F64_, s64, DST_PAIR_SET_, p->p2, st, first_out));
    prof_mark(p, st, 3);
    for (int it = 0; it < sweeps; ++it) {
      float *r32 = reinterpret_cast<float *>(p->work64);   // work64 is free in mixed mode
      if (s2)
        launch_residual(p->singular, true, norm, st, g, s2, (const float2 *)p->p2, r32, p->dstats,
                        &p->dstats->res2[it], p->partials, p->counters, step(it));
      else
        launch_residual(p->singular, true, norm, st, g, s64, (const float2 *)p->p2, r32, p->dstats,
                        &p->dstats->res2[it], p->partials, p->counters, step(it));
      count_launch(p);
      prof_mark(p, st, 4);
      PC_TRY(solve_fp32_grid(p, SRC_F32_, r32, DST_PAIR_ADD_, p->p2, st,
                             (adaptive || it == sweeps - 1) ? pout : nullptr, gate(it + 1), chunk(it + 1)));
      prof_mark(p, st, 3);
    }
    // the residual after the last allowed sweep (statistics, and the rule's verdict on them)
    if (sweeps > 0 && want_final_residual) {
      if (s2)
        launch_residual(p->singular, false, true, st, g, s2, (const float2 *)p->p2, (float *)nullptr, p->dstats,
                        &p->dstats->res2[sweeps], p->partials, p->counters, step(sweeps));
      else
        launch_residual(p->singular, false, true, st, g, s64, (const float2 *)p->p2, (float *)nullptr, p->dstats,
                        &p->dstats->res2[sweeps], p->partials, p->counters, step(sweeps));
      count_launch(p);
      prof_mark(p, st, 7);
    }
  }
  // the residual of an FP64 or unrefined FP32 solve (statistics; the residual of L_h: FD solves only)
  const bool refined = p->precision == PC_PREC_MIXED && p->refine_iters > 0;
  if (want_final_residual && p->eigen == PC_EIG_FD && !refined) {
    if (p->precision == PC_PREC_FP64)
      launch_residual(p->singular, false, true, st, g, s64, (const double *)pout, (float *)nullptr, p->dstats,
                      &p->dstats->res2[0], p->partials, p->counters);
    else if (s2)
      launch_residual(p->singular, false, true, st, g, s2, (const float2 *)p->p2, (float *)nullptr, p->dstats,
                      &p->dstats->res2[0], p->partials, p->counters);
    else
      launch_residual(p->singular, false, true, st, g, s64, (const float2 *)p->p2, (float *)nullptr, p->dstats,
                      &p->dstats->res2[0], p->partials, p->counters);
    count_launch(p);
    prof_mark(p, st, 7);
  }
  // gauge, then the FP32 split of p for the mixed gradient
  const int gmode = gauge_mode(p);
  if (gmode) {
    launch_pdl(gauge_sum_kernel, grid_for(nc, kFlatPerBlock), T, 0, st, nc, pout, p->dstats, p->partials, p->counters,
               gmode, trap_weights(p));
    count_launch(p);
  }
  bool mixed = p->precision != PC_PREC_FP64;
  if (gmode) {   // a vertex plan splits p on the lattice afterwards (vertex_embed_kernel)
    const int G = grid_for(nc, kFlatPerBlock);
    if (mixed && !p->vertex) launch_pdl(finalize_p_kernel<true, true>, G, T, 0, st, (int)nc, pout, p->dstats, p->p2);
    else launch_pdl(finalize_p_kernel<true, false>, G, T, 0, st, (int)nc, pout, p->dstats, nullptr);
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
  const double nc = mean_weight_total(p);   // cells, or the trapezoid weights of a vertex grid
  const bool zero_mode = p->singular;
  stats->removed_mean = zero_mode ? ds.sum_s / nc : 0.0;
  stats->source_norm = std::sqrt(fmax(ds.sum_s2, 0.0));
  const bool adaptive = refine_adaptive(p);
  int its = (p->precision == PC_PREC_MIXED) ? p->refine_iters : 0;
  bool conv = true;
  if (adaptive) {   // the device's decisions, replayed on the stored max norms
    conv = false;
    for (int k = 0; k <= its; ++k)
      if (refine_stop_at(ds.rmax, ds.smax, k, (float)p->refine_tol)) {
        its = k;
        conv = true;
        break;
      }
  }
  for (int i = 0; i <= its && i < 9; ++i) stats->residual_norm[i] = std::sqrt(fmax(ds.res2[i], 0.0));
  stats->refine_iters_done = its;
  stats->refine_converged = conv ? 1 : 0;
  stats->max_div_after = ds.max_div;
  stats->max_abs_u_star = ds.max_u;
  const int gmode = gauge_mode(p);
  stats->gauge_shift = gmode == 1 ? ds.sum_p / nc : (gmode == 2 ? ds.corner_p : 0.0);
  // a NaN or infinity anywhere in u~ reaches the source sums (the maxima above skip NaN)
  if (!std::isfinite(ds.sum_s) || !std::isfinite(ds.sum_s2))
    return fail(PC_ERR_INVALID_ARG, "non-finite source: u_star, f_ib_in or dt hold a NaN or infinity");
  if (!conv)
    return fail(PC_ERR_NOT_CONVERGED, "refinement: max |r| / max |s| = %.3g after %d sweeps (tolerance %.3g)",
                (double)ds.rmax[its] / fmax((double)ds.smax, 1e-300), its, p->refine_tol);
  return PC_OK;
}

// Gradient and correction at every node (Eq. 4 at fluid nodes, Eqs. 18-19 at boundary/virtual
// nodes) from the solved pressure: p2 pairs (mixed) or the FP64 p in dp.
// Blocks [b0, b0 + nb) of the node grid (nb < 0: all from b0).
static void launch_gradient(Plan *p, cudaStream_t st, const double *dp, const void *ug, double dt, void *duo,
                            void *dfo, int b0 = 0, int nb = -1) {
  const int T = 256;
  const long long N = p->N;
  const int d = p->dim;
  const bool mixed = p->precision != PC_PREC_FP64;
  const int G = nb < 0 ? grid_for(N, T) - b0 : nb;
  if (G <= 0) return;
  if (p->vdtype == PC_DTYPE_F64) {
    if (mixed) {
      if (d == 2) launch_pdl(gradient_mixed_kernel<double, 2>, G, T, 0, st, (int)N, p->Kg, p->ncol, p->nD2, p->p2, p->ntype, (const double *)ug, 1.0 / dt, dt, p->beta, (double *)duo, (double *)dfo, b0);
      else launch_pdl(gradient_mixed_kernel<double, 3>, G, T, 0, st, (int)N, p->Kg, p->ncol, p->nD2, p->p2, p->ntype, (const double *)ug, 1.0 / dt, dt, p->beta, (double *)duo, (double *)dfo, b0);
    } else {
      if (d == 2) launch_pdl(gradient64_kernel<double, 2>, G, T, 0, st, (int)N, p->Kg, p->ncol, p->nD64, dp, p->ntype, (const double *)ug, 1.0 / dt, dt, p->beta, (double *)duo, (double *)dfo, b0);
      else launch_pdl(gradient64_kernel<double, 3>, G, T, 0, st, (int)N, p->Kg, p->ncol, p->nD64, dp, p->ntype, (const double *)ug, 1.0 / dt, dt, p->beta, (double *)duo, (double *)dfo, b0);
    }
  } else {
    if (mixed) {
      if (d == 2) launch_pdl(gradient_mixed_kernel<float, 2>, G, T, 0, st, (int)N, p->Kg, p->ncol, p->nD2, p->p2, p->ntype, (const float *)ug, 1.0 / dt, dt, p->beta, (float *)duo, (float *)dfo, b0);
      else launch_pdl(gradient_mixed_kernel<float, 3>, G, T, 0, st, (int)N, p->Kg, p->ncol, p->nD2, p->p2, p->ntype, (const float *)ug, 1.0 / dt, dt, p->beta, (float *)duo, (float *)dfo, b0);
    } else {
      if (d == 2) launch_pdl(gradient64_kernel<float, 2>, G, T, 0, st, (int)N, p->Kg, p->ncol, p->nD64, dp, p->ntype, (const float *)ug, 1.0 / dt, dt, p->beta, (float *)duo, (float *)dfo, b0);
      else launch_pdl(gradient64_kernel<float, 3>, G, T, 0, st, (int)N, p->Kg, p->ncol, p->nD64, dp, p->ntype, (const float *)ug, 1.0 / dt, dt, p->beta, (float *)duo, (float *)dfo, b0);
    }
  }
}

// Source of the direct-divergence mode into the same buffers as the face divergence.
static void launch_direct_div(Plan *p, cudaStream_t st, double inv_bdt, int want_sums) {
  const bool mixed = p->precision != PC_PREC_FP64;
  const int nc = (int)p->ncells, T = 256, G = grid_for(nc, T);
  const GridDev g = grid_dev(p);
  double *s = mixed ? nullptr : p->s64;
  float2 *s2 = mixed ? reinterpret_cast<float2 *>(p->s64) : nullptr;
  float *s32 = mixed ? reinterpret_cast<float *>(p->work64) : nullptr;
  const double inc = 1.0 / (double)nc;
  if (p->dim == 2) {
    if (mixed) launch_pdl(direct_div_kernel<2, true>, G, T, 0, st, nc, p->K, p->ccol, p->cD64, p->cD2, p->ut64, p->u2, (int)p->N, inv_bdt, g.mask, s, s2, s32, p->dstats, p->partials, p->counters, want_sums, inc);
    else launch_pdl(direct_div_kernel<2, false>, G, T, 0, st, nc, p->K, p->ccol, p->cD64, p->cD2, p->ut64, p->u2, (int)p->N, inv_bdt, g.mask, s, s2, s32, p->dstats, p->partials, p->counters, want_sums, inc);
  } else {
    if (mixed) launch_pdl(direct_div_kernel<3, true>, G, T, 0, st, nc, p->K, p->ccol, p->cD64, p->cD2, p->ut64, p->u2, (int)p->N, inv_bdt, g.mask, s, s2, s32, p->dstats, p->partials, p->counters, want_sums, inc);
    else launch_pdl(direct_div_kernel<3, false>, G, T, 0, st, nc, p->K, p->ccol, p->cD64, p->cD2, p->ut64, p->u2, (int)p->N, inv_bdt, g.mask, s, s2, s32, p->dstats, p->partials, p->counters, want_sums, inc);
  }
}

// The source and solve of a pass on a vertex-grid plan: the direct divergence at the vertex
// unknowns (FP64, into s64), the solve on the unknowns (dp), and p on the whole lattice
// (work64 in FP64, p2 as pairs in mixed and FP32 plans), which the gradient reads.
static pc_status vertex_pass_solve(Plan *p, cudaStream_t st, double inv_bdt, double *dp, bool want_stats) {
  const long long nc = p->ncells, npt = p->npts;
  const bool mixed = p->precision != PC_PREC_FP64;
  const int T = 256, G = grid_for(npt, T);
  const uint8_t *mask = p->rhs_mask_on ? p->rhs_mask : nullptr;
  double *sv = p->s64;
  if (p->dim == 2) {
    if (mixed) launch_pdl(direct_div_kernel<2, true>, G, T, 0, st, (int)npt, p->K, p->ccol, p->cD64, p->cD2, p->ut64, p->u2, (int)p->N, inv_bdt, mask, sv, (float2 *)nullptr, (float *)nullptr, p->dstats, p->partials, p->counters, 0, 0.0);
    else launch_pdl(direct_div_kernel<2, false>, G, T, 0, st, (int)npt, p->K, p->ccol, p->cD64, p->cD2, p->ut64, p->u2, (int)p->N, inv_bdt, mask, sv, (float2 *)nullptr, (float *)nullptr, p->dstats, p->partials, p->counters, 0, 0.0);
  } else {
    if (mixed) launch_pdl(direct_div_kernel<3, true>, G, T, 0, st, (int)npt, p->K, p->ccol, p->cD64, p->cD2, p->ut64, p->u2, (int)p->N, inv_bdt, mask, sv, (float2 *)nullptr, (float *)nullptr, p->dstats, p->partials, p->counters, 0, 0.0);
    else launch_pdl(direct_div_kernel<3, false>, G, T, 0, st, (int)npt, p->K, p->ccol, p->cD64, p->cD2, p->ut64, p->u2, (int)p->N, inv_bdt, mask, sv, (float2 *)nullptr, (float *)nullptr, p->dstats, p->partials, p->counters, 0, 0.0);
  }
  count_launch(p);
  // the source sums: the (weighted) mean the residual removes on zero-mode problems, and the
  // statistics
  if (want_stats || p->singular) {
    launch_pdl(sum_kernel, grid_for(nc, kFlatPerBlock), kFlatThreads, 0, st, nc, (const double *)p->s64, p->dstats,
               p->partials, p->counters, trap_weights(p));
    count_launch(p);
  }
  prof_mark(p, st, 2);
  PC_TRY(solve_grid(p, p->s64, dp, want_stats, st));
  const VertexGrid V = vertex_grid(p);
  launch_pdl(vertex_embed_kernel, vertex_grid_dims(p->dim, V.nf, T), T, 0, st, V, (const double *)dp, p->work64,
             mixed ? reinterpret_cast<float2 *>(p->p2) : (float2 *)nullptr);
  count_launch(p);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

static pc_status project_impl(Plan *p, double dt, const void *u_star, const void *f_in, double *p_out,
                              void *u_out, void *f_out, pc_stats *stats, cudaStream_t st,
                              bool all_device = false) {
  const int d = p->dim;
  const long long N = p->N, nc = p->ncells;
  const size_t vsz = p->vdtype == PC_DTYPE_F64 ? 8 : 4;
  const size_t vbytes = (size_t)d * N * vsz;
  // host pointers are staged through plan buffers
  const bool hu = !all_device && !is_device_ptr(u_star), hf = !all_device && !is_device_ptr(f_in),
             hp = !all_device && !is_device_ptr(p_out), huo = !all_device && !is_device_ptr(u_out),
             hfo = !all_device && !is_device_ptr(f_out);
  const void *du = u_star, *df = f_in;
  double *dp = p_out;
  void *duo = u_out, *dfo = f_out;
  if ((hu || (f_in && hf) || huo || (f_out && hfo)) && !p->stage_u) PC_TRY(plan_node_staging(p));
  if (hu) { PC_CUDA_TRY(cudaMemcpyAsync(p->stage_u, u_star, vbytes, cudaMemcpyHostToDevice, st)); du = p->stage_u; }
  if (f_in && hf) { PC_CUDA_TRY(cudaMemcpyAsync(p->stage_f, f_in, vbytes, cudaMemcpyHostToDevice, st)); df = p->stage_f; }
  if (hp) dp = p->stage_p;
  const long long np_out = p->vertex ? p->nvtot : nc;   // pressure values returned
  if (huo) duo = p->stage_uo;
  if (f_out && hfo) dfo = p->stage_fo;

  prof_begin(p, st);
  PC_CUDA_TRY(cudaMemsetAsync(p->dstats, 0, sizeof(DevStats), st));
  const int T = 256;
  const bool mixed = p->precision != PC_PREC_FP64;
  const long long cnt = (long long)d * N;
  if (p->vdtype == PC_DTYPE_F64)
    launch_prep<double>(df != nullptr, stats != nullptr, mixed, cnt, (const double *)du, (const double *)df, dt,
                        p->ut64, p->u2, p->dstats, st);
  else
    launch_prep<float>(df != nullptr, stats != nullptr, mixed, cnt, (const float *)du, (const float *)df, dt,
                       p->ut64, p->u2, p->dstats, st);
  count_launch(p);
  prof_mark(p, st, 0);
  if (p->vertex) {
    PC_TRY(vertex_pass_solve(p, st, 1.0 / (p->beta * dt), dp, stats != nullptr));
  } else if (p->divmode == PC_DIV_WLS_DIRECT) {
    launch_direct_div(p, st, 1.0 / (p->beta * dt), stats ? 2 : (p->singular ? 1 : 0));
    count_launch(p);
    prof_mark(p, st, 2);
  }
  for (int a = 0; a < d && p->divmode == PC_DIV_FACES; ++a) {
    const long long rows = p->nface_total[a];
    const int G = grid_for(rows, T);
    if (mixed) {
      const PairSrc src{p->u2 + (long long)a * N};
      if (p->K == 12) launch_pdl(transfer_mixed_kernel<12, PairSrc>, G, T, 0, st, (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
      else if (p->K == 27) launch_pdl(transfer_mixed_kernel<27, PairSrc>, G, T, 0, st, (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
      else launch_pdl(transfer_mixed_kernel<0, PairSrc>, G, T, 0, st, (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
    } else {
      launch_pdl(transfer64_kernel, G, T, 0, st, (int)rows, p->K, p->fcol[a], p->fw64[a],
                 p->ut64 + (long long)a * N, p->U64[a]);
    }
    count_launch(p);
  }
  GridDev g = grid_dev(p);
  if (p->divmode == PC_DIV_FACES) {
    prof_mark(p, st, 1);
    auto divk = (d == 2) ? divergence_kernel<2> : divergence_kernel<3>;
    const int sums = stats ? 2 : (p->singular ? 1 : 0);
    const GridDev gd = sums ? g : with_rows_per_thread(g, kSingleRows);
    launch_pdl(divk, gd.nblk, 256, 0, st, gd, p->U64[0], p->U64[1], p->U64[2], 1.0 / (p->beta * dt),
               mixed ? nullptr : p->s64, mixed ? reinterpret_cast<float2 *>(p->s64) : nullptr,
               mixed ? reinterpret_cast<float *>(p->work64) : nullptr, p->dstats, p->partials, p->counters,
               sums, 1.0 / (double)nc);
    count_launch(p);
    prof_mark(p, st, 2);
  }
  PC_CUDA_TRY(cudaGetLastError());
  if (!p->vertex)
    PC_TRY(solve_grid(p, p->s64, dp, stats != nullptr, st,
                      mixed ? reinterpret_cast<const float *>(p->work64) : nullptr,
                      mixed ? reinterpret_cast<const float2 *>(p->s64) : nullptr));
  const double *gp = p->vertex ? p->work64 : dp;   // the pressure the gradient reads (FP64 plans)
  // Host results: the pressure is final here, so its copy runs on the plan's copy stream while
  // the gradient computes; the gradient runs in two halves and the first half's u and f are
  // copied while the second half computes (copy engines and kernels overlap).
  const bool host_out = hp || huo || (f_out && hfo);
  if (host_out && !p->copy_st) {
    PC_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking));
    for (int e = 0; e < 3; ++e) PC_CUDA_TRY(cudaEventCreateWithFlags(&p->copy_ev[e], cudaEventDisableTiming));
  }
  if (hp) {
    PC_CUDA_TRY(cudaEventRecord(p->copy_ev[0], st));
    PC_CUDA_TRY(cudaStreamWaitEvent(p->copy_st, p->copy_ev[0], 0));
    PC_CUDA_TRY(cudaMemcpyAsync(p_out, dp, np_out * sizeof(double), cudaMemcpyDeviceToHost, p->copy_st));
  }
  const int gblocks = grid_for(N, 256);
  const bool split = (huo || (f_out && hfo)) && gblocks >= 2;
  const int b1 = gblocks / 2;
  const long long n1 = split ? std::min(N, (long long)b1 * 256) : 0;   // nodes of the first half
  auto copy_nodes = [&](long long i0, long long i1, cudaStream_t cs) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < d && e == cudaSuccess && i1 > i0; ++a) {
      const size_t off = ((size_t)a * N + i0) * vsz, len = (size_t)(i1 - i0) * vsz;
      if (huo) e = cudaMemcpyAsync((char *)u_out + off, (const char *)duo + off, len, cudaMemcpyDeviceToHost, cs);
      if (e == cudaSuccess && f_out && hfo)
        e = cudaMemcpyAsync((char *)f_out + off, (const char *)dfo + off, len, cudaMemcpyDeviceToHost, cs);
    }
    return e;
  };
  if (split) {
    launch_gradient(p, st, gp, du, dt, duo, dfo, 0, b1);
    count_launch(p);
    PC_CUDA_TRY(cudaEventRecord(p->copy_ev[1], st));
    PC_CUDA_TRY(cudaStreamWaitEvent(p->copy_st, p->copy_ev[1], 0));
    PC_CUDA_TRY(copy_nodes(0, n1, p->copy_st));
    launch_gradient(p, st, gp, du, dt, duo, dfo, b1, -1);
  } else {
    launch_gradient(p, st, gp, du, dt, duo, dfo);
  }
  count_launch(p);
  prof_mark(p, st, 6);
  if (stats && p->divmode == PC_DIV_FACES) {   // no face fluxes in the direct mode
    auto chk = (d == 2) ? div_check_kernel<2> : div_check_kernel<3>;
    launch_pdl(chk, g.nblk, 256, 0, st, g, p->U64[0], p->U64[1], p->U64[2], dp, p->beta * dt, p->dstats);
    count_launch(p);
    prof_mark(p, st, 7);
  }
  PC_CUDA_TRY(cudaGetLastError());
  if (split) PC_CUDA_TRY(copy_nodes(n1, N, st));
  else PC_CUDA_TRY(copy_nodes(0, N, st));
  if (host_out) {   // join the copy stream
    PC_CUDA_TRY(cudaEventRecord(p->copy_ev[2], p->copy_st));
    PC_CUDA_TRY(cudaStreamWaitEvent(st, p->copy_ev[2], 0));
  }
  if (stats) PC_TRY(fill_stats(p, stats, st));
  if (hp || huo || (f_out && hfo)) PC_CUDA_TRY(cudaStreamSynchronize(st));
  return PC_OK;
}

// Grid-level solve of device arrays with a caller-built plan description (no staging, no
// statistics): source sums, transform solve, gauge. Used by the allocation-free entry point.
pc_status solve_grid_device(Plan *p, const double *s, double *pout, cudaStream_t st) {
  const long long nc = p->ncells;
  launch_pdl(sum_kernel, grid_for(nc, kFlatPerBlock), kFlatThreads, 0, st, nc, s, p->dstats, p->partials, p->counters,
             TrapWeights{});
  count_launch(p);
  PC_CUDA_TRY(cudaGetLastError());
  return solve_grid(p, s, pout, false, st);
}

// pc_solve_poisson on a vertex-grid plan: the solve on the unknowns, with the trapezoid-weighted
// mean on N-N axes.
static pc_status vertex_solve(Plan *p, const double *s, double *p_out, pc_stats *stats, cudaStream_t st,
                              bool all_device = false) {
  const long long nc = p->ncells;
  const bool hs = !all_device && !is_device_ptr(s), hp = !all_device && !is_device_ptr(p_out);
  const double *ds = s;
  double *dp = p_out;
  if (hs) {
    PC_CUDA_TRY(cudaMemcpyAsync(p->stage_s, s, nc * sizeof(double), cudaMemcpyHostToDevice, st));
    ds = p->stage_s;
  }
  if (hp) dp = p->stage_p;
  prof_begin(p, st);
  PC_CUDA_TRY(cudaMemsetAsync(p->dstats, 0, sizeof(DevStats), st));
  launch_pdl(sum_kernel, grid_for(nc, kFlatPerBlock), kFlatThreads, 0, st, nc, ds, p->dstats, p->partials,
             p->counters, trap_weights(p));
  count_launch(p);
  prof_mark(p, st, 2);
  PC_TRY(solve_grid(p, ds, dp, stats != nullptr, st));
  PC_CUDA_TRY(cudaGetLastError());
  if (hp) PC_CUDA_TRY(cudaMemcpyAsync(p_out, dp, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (stats) PC_TRY(fill_stats(p, stats, st));
  if (hp) PC_CUDA_TRY(cudaStreamSynchronize(st));
  return PC_OK;
}

static pc_status solve_impl(Plan *p, const double *s, double *p_out, pc_stats *stats, cudaStream_t st,
                            bool all_device = false) {
  const long long nc = p->ncells;
  const bool hs = !all_device && !is_device_ptr(s), hp = !all_device && !is_device_ptr(p_out);
  const double *ds = s;
  double *dp = p_out;
  if (hs) { PC_CUDA_TRY(cudaMemcpyAsync(p->stage_s, s, nc * sizeof(double), cudaMemcpyHostToDevice, st)); ds = p->stage_s; }
  if (hp) dp = p->stage_p;
  prof_begin(p, st);
  PC_CUDA_TRY(cudaMemsetAsync(p->dstats, 0, sizeof(DevStats), st));
  launch_pdl(sum_kernel, grid_for(nc, kFlatPerBlock), kFlatThreads, 0, st, nc, ds, p->dstats, p->partials, p->counters,
             TrapWeights{});
  count_launch(p);
  prof_mark(p, st, 2);
  PC_TRY(solve_grid(p, ds, dp, stats != nullptr, st));
  if (hp) PC_CUDA_TRY(cudaMemcpyAsync(p_out, dp, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (stats) PC_TRY(fill_stats(p, stats, st));
  if (hp) PC_CUDA_TRY(cudaStreamSynchronize(st));
  return PC_OK;
}

static bool graph_cached(const Plan *p, double dt, const void *u, const void *f, const double *po,
                         const void *uo, const void *fo) {
  for (int i = 0; i < kGraphCache; ++i) {
    const GraphEntry &c = p->graphs[i];
    if (c.exec && c.kind == 0 && c.u == u && c.f == f && c.p == po && c.uo == uo && c.fo == fo && c.dt == dt &&
        c.prof == p->prof)
      return true;
  }
  return false;
}

// A cached CUDA graph of one call: looked up by `match`, else captured once on the plan's private
// stream by `capture` (which records the argument set in the entry), then replayed with one
// launch on the caller's stream. pc_project and pc_solve_poisson with device arrays use it.
template <typename Match, typename Capture>
static pc_status run_graph(Plan *p, cudaStream_t st, Match match, Capture capture) {
  GraphEntry *e = nullptr;
  for (int i = 0; i < kGraphCache; ++i)
    if (p->graphs[i].exec && p->graphs[i].prof == p->prof && match(p->graphs[i])) {
      e = &p->graphs[i];
      break;
    }
  if (!e) {
    e = &p->graphs[0];
    for (int i = 1; i < kGraphCache; ++i)
      if (p->graphs[i].stamp < e->stamp) e = &p->graphs[i];
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    e->exec = nullptr;
    e->graph = nullptr;
    PC_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    p->capturing = true;
    // event-record nodes at the phase boundaries only in a profiled graph: they are full
    // dependencies and would cut the programmatic overlap between the kernels around them
    p->cap_events = p->prof;
    p->cap_n = 0;
    const long long l0 = p->launches;
    pc_status s = capture(*e, p->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &g);
    p->capturing = false;
    e->launches = p->launches - l0;
    p->launches = l0;
    if (s != PC_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return s != PC_OK ? s : fail(PC_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(ce));
    }
    cudaError_t ie = cudaGraphInstantiate(&e->exec, g, 0ULL);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(g);
      e->exec = nullptr;
      return fail(PC_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
    }
    e->graph = g;
    // map the event-record nodes back to the phase boundaries they were captured for
    size_t nn = 0;
    PC_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    PC_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
    e->nev = p->cap_n;
    for (int i = 0; i < e->nev; ++i) e->evnode[i] = nullptr;
    for (size_t k = 0; k < nn; ++k) {
      cudaGraphNodeType ty;
      PC_CUDA_TRY(cudaGraphNodeGetType(nodes[k], &ty));
      if (ty != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev;
      PC_CUDA_TRY(cudaGraphEventRecordNodeGetEvent(nodes[k], &ev));
      for (int i = 0; i < e->nev; ++i)
        if (p->cap_ev[i] == ev) e->evnode[i] = nodes[k];
    }
    for (int i = 0; i + 1 < e->nev; ++i) e->tag[i] = p->cap_tag[i];
    e->prof = p->prof;
  }
  e->stamp = ++p->graph_clock;
  if (p->prof && p->slots && p->slots_used < kProfSlots) {
    ProfSlot *slot = &p->slots[p->slots_used++];
    slot->n = 0;
    bool ok = true;
    for (int i = 0; i < e->nev && ok; ++i)
      ok = e->evnode[i] && cudaGraphExecEventRecordNodeSetEvent(e->exec, e->evnode[i], slot->ev[i]) == cudaSuccess;
    if (ok) {
      slot->n = e->nev;
      for (int i = 0; i + 1 < e->nev; ++i) slot->tag[i] = e->tag[i];
    }
  }
  PC_CUDA_TRY(cudaGraphLaunch(e->exec, st));
  p->launches += e->launches;
  return PC_OK;
}

// pc_project through a cached CUDA graph, one per argument set (pointers and dt).
static pc_status project_graph(Plan *p, double dt, const void *u_star, const void *f_in, double *p_out,
                               void *u_out, void *f_out, cudaStream_t st) {
  return run_graph(
      p, st,
      [&](const GraphEntry &c) {
        return c.kind == 0 && c.u == u_star && c.f == f_in && c.p == p_out && c.uo == u_out && c.fo == f_out &&
               c.dt == dt;
      },
      [&](GraphEntry &e, cudaStream_t cs) {
        pc_status s = project_impl(p, dt, u_star, f_in, p_out, u_out, f_out, nullptr, cs, true);
        e.kind = 0; e.u = u_star; e.f = f_in; e.p = p_out; e.uo = u_out; e.fo = f_out; e.dt = dt;
        return s;
      });
}

// pc_solve_poisson with device arrays through a cached CUDA graph, one per (s, p_out).
static pc_status solve_graph(Plan *p, const double *s, double *p_out, cudaStream_t st) {
  return run_graph(
      p, st, [&](const GraphEntry &c) { return c.kind == 1 && c.u == s && c.p == p_out; },
      [&](GraphEntry &e, cudaStream_t cs) {
        pc_status r = p->vertex ? vertex_solve(p, s, p_out, nullptr, cs, true) : solve_impl(p, s, p_out, nullptr, cs, true);
        e.kind = 1; e.u = s; e.f = nullptr; e.p = p_out; e.uo = nullptr; e.fo = nullptr; e.dt = 0.0;
        return r;
      });
}

// ----------------------------------------------------------------------------- IB-force iteration
// Tables of the iteration, built on the first pc_project_ib call of a plan instance (one setup
// synchronisation): the boundary/virtual node list, the faces each axis must refresh after the
// first pass (ascending face order), and the two compact force iterates.
static pc_status ib_tables(Plan *p, cudaStream_t st) {
  if (p->nib >= 0) return PC_OK;
  const long long N = p->N;
  const int d = p->dim;
  std::vector<uint8_t> type((size_t)N);
  PC_CUDA_TRY(cudaMemcpyAsync(type.data(), p->ntype, (size_t)N, cudaMemcpyDeviceToHost, st));
  PC_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int32_t> idx;
  for (long long i = 0; i < N; ++i)
    if (type[(size_t)i] != PC_NODE_FLUID) idx.push_back((int32_t)i);
  std::vector<int32_t> faces[3];
  if (!idx.empty() && p->divmode == PC_DIV_FACES) {
    long long maxrows = 0;
    for (int a = 0; a < d; ++a) maxrows = p->nface_total[a] > maxrows ? p->nface_total[a] : maxrows;
    uint8_t *flag = nullptr;
    PC_CUDA_TRY(cudaMalloc(&flag, (size_t)maxrows));
    std::vector<uint8_t> hf((size_t)maxrows);
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < d && e == cudaSuccess; ++a) {
      const long long rows = p->nface_total[a];
      ib_face_flags_kernel<<<grid_for(rows, 256), 256, 0, st>>>((int)rows, p->K, p->fcol[a], p->ntype, flag);
      e = cudaMemcpyAsync(hf.data(), flag, (size_t)rows, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      for (long long r = 0; r < rows && e == cudaSuccess; ++r)
        if (hf[(size_t)r]) faces[a].push_back((int32_t)r);
    }
    cudaFree(flag);
    if (e != cudaSuccess) return fail(PC_ERR_CUDA, "IB face tables: %s", cudaGetErrorString(e));
  }
  const long long nib = (long long)idx.size();
  const size_t vsz = p->vdtype == PC_DTYPE_F64 ? 8 : 4;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t ints = (size_t)nib;
  for (int a = 0; a < d; ++a) ints += faces[a].size();
  const size_t fbytes = up((size_t)d * nib * vsz);
  const size_t total = up(ints * 4) + 2 * fbytes + up(sizeof(IbCtl)) + 256;
  char *base = nullptr;
  PC_TRY(plan_alloc(p, (void **)&base, total));
  p->ib_ctl = reinterpret_cast<IbCtl *>(base + up(ints * 4) + 2 * fbytes);
  int32_t *ip = reinterpret_cast<int32_t *>(base);
  p->ib_idx = ip;
  if (nib) PC_CUDA_TRY(cudaMemcpyAsync(ip, idx.data(), (size_t)nib * 4, cudaMemcpyHostToDevice, st));
  ip += nib;
  for (int a = 0; a < d; ++a) {
    p->ib_face[a] = ip;
    p->nib_face[a] = (int64_t)faces[a].size();
    if (!faces[a].empty())
      PC_CUDA_TRY(cudaMemcpyAsync(ip, faces[a].data(), faces[a].size() * 4, cudaMemcpyHostToDevice, st));
    ip += faces[a].size();
  }
  p->ib_f[0] = base + up(ints * 4);
  p->ib_f[1] = base + up(ints * 4) + fbytes;
  PC_CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors die here
  p->nib = nib;
  return PC_OK;
}

template <typename VT>
static void ib_launch_force(Plan *p, cudaStream_t st, const double *dp, const VT *u, double dt, VT *fc) {
  const int T = 256;
  const int G = grid_for(p->nib, T);
  const bool mixed = p->precision != PC_PREC_FP64;
  const int nib = (int)p->nib, N = (int)p->N;
  if (p->dim == 2) {
    if (mixed) launch_pdl(ib_force_kernel<VT, 2, true>, G, T, 0, st, nib, p->ib_idx, N, p->Kg, p->ncol, p->nD64, p->nD2, dp, p->p2, u, 1.0 / dt, p->beta, fc);
    else launch_pdl(ib_force_kernel<VT, 2, false>, G, T, 0, st, nib, p->ib_idx, N, p->Kg, p->ncol, p->nD64, p->nD2, dp, p->p2, u, 1.0 / dt, p->beta, fc);
  } else {
    if (mixed) launch_pdl(ib_force_kernel<VT, 3, true>, G, T, 0, st, nib, p->ib_idx, N, p->Kg, p->ncol, p->nD64, p->nD2, dp, p->p2, u, 1.0 / dt, p->beta, fc);
    else launch_pdl(ib_force_kernel<VT, 3, false>, G, T, 0, st, nib, p->ib_idx, N, p->Kg, p->ncol, p->nD64, p->nD2, dp, p->p2, u, 1.0 / dt, p->beta, fc);
  }
}

// One pass of the iteration: u~ (all nodes on the first pass, then the IB nodes), fluxes (all
// faces on the first pass, then the listed faces), source, solve, the new force at the IB nodes
// (ib_f[1], after the current one has been saved in ib_f[0]) and the stopping rule. With cond
// != 0 the rule also sets the while condition of the loop graph.
template <typename VT>
static pc_status ib_pass(Plan *p, bool first, double dt, const VT *du, double *dp, double tol, int max_iters,
                         bool use_cond, cudaGraphConditionalHandle cond, cudaStream_t st) {
  const int d = p->dim;
  const long long N = p->N, nc = p->ncells;
  const bool mixed = p->precision != PC_PREC_FP64;
  const int T = 256;
  const int nib = (int)p->nib;
  VT *fo = static_cast<VT *>(p->ib_f[0]), *fc = static_cast<VT *>(p->ib_f[1]);
  prof_begin(p, st);
  PC_CUDA_TRY(cudaMemsetAsync(p->dstats, 0, sizeof(DevStats), st));
  if (first) {
    launch_prep<VT>(false, false, mixed, (long long)d * N, du, nullptr, dt, p->ut64, p->u2, p->dstats, st);
    count_launch(p);
  }
  if (nib) {
    if (mixed) launch_pdl(ib_prep_kernel<VT, true>, grid_for(nib, T), T, 0, st, nib, (int)N, d, p->ib_idx, du, (const VT *)fc, fo, dt, p->ut64, p->u2);
    else launch_pdl(ib_prep_kernel<VT, false>, grid_for(nib, T), T, 0, st, nib, (int)N, d, p->ib_idx, du, (const VT *)fc, fo, dt, p->ut64, p->u2);
    count_launch(p);
  }
  prof_mark(p, st, 0);
  if (p->vertex) {                           // the whole source again, solve and restriction
    PC_TRY(vertex_pass_solve(p, st, 1.0 / (p->beta * dt), dp, false));
  } else if (p->divmode == PC_DIV_WLS_DIRECT) {   // the whole source again: no face lists in this mode
    launch_direct_div(p, st, 1.0 / (p->beta * dt), p->singular ? 1 : 0);
    count_launch(p);
    prof_mark(p, st, 2);
  }
  for (int a = 0; a < d && p->divmode == PC_DIV_FACES; ++a) {
    const long long rows = p->nface_total[a];
    const long long nl = first ? rows : p->nib_face[a];
    if (nl == 0) continue;
    const int G = grid_for(nl, T);
    if (mixed) {
      const PairSrc src{p->u2 + (long long)a * N};
      if (first) {
        if (p->K == 12) launch_pdl(transfer_mixed_kernel<12, PairSrc>, G, T, 0, st, (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
        else if (p->K == 27) launch_pdl(transfer_mixed_kernel<27, PairSrc>, G, T, 0, st, (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
        else launch_pdl(transfer_mixed_kernel<0, PairSrc>, G, T, 0, st, (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
      } else {
        if (p->K == 12) launch_pdl(ib_transfer_mixed_kernel<12>, G, T, 0, st, (int)nl, p->ib_face[a], (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
        else if (p->K == 27) launch_pdl(ib_transfer_mixed_kernel<27>, G, T, 0, st, (int)nl, p->ib_face[a], (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
        else launch_pdl(ib_transfer_mixed_kernel<0>, G, T, 0, st, (int)nl, p->ib_face[a], (int)rows, p->K, p->fcol[a], p->fw2[a], src, p->U64[a]);
      }
    } else {
      if (first) launch_pdl(transfer64_kernel, G, T, 0, st, (int)rows, p->K, p->fcol[a], p->fw64[a], p->ut64 + (long long)a * N, p->U64[a]);
      else launch_pdl(ib_transfer64_kernel, G, T, 0, st, (int)nl, p->ib_face[a], (int)rows, p->K, p->fcol[a], p->fw64[a], p->ut64 + (long long)a * N, p->U64[a]);
    }
    count_launch(p);
  }
  if (p->divmode == PC_DIV_FACES) {
    prof_mark(p, st, 1);
    GridDev g = grid_dev(p);
    auto divk = (d == 2) ? divergence_kernel<2> : divergence_kernel<3>;
    const GridDev gd = p->singular ? g : with_rows_per_thread(g, kSingleRows);
    launch_pdl(divk, gd.nblk, 256, 0, st, gd, p->U64[0], p->U64[1], p->U64[2], 1.0 / (p->beta * dt),
               mixed ? nullptr : p->s64, mixed ? reinterpret_cast<float2 *>(p->s64) : nullptr,
               mixed ? reinterpret_cast<float *>(p->work64) : nullptr, p->dstats, p->partials, p->counters,
               p->singular ? 1 : 0, 1.0 / (double)nc);
    count_launch(p);
    prof_mark(p, st, 2);
  }
  PC_CUDA_TRY(cudaGetLastError());
  if (!p->vertex)
    PC_TRY(solve_grid(p, p->s64, dp, false, st, mixed ? reinterpret_cast<const float *>(p->work64) : nullptr,
                      mixed ? reinterpret_cast<const float2 *>(p->s64) : nullptr));
  if (nib) {
    ib_launch_force<VT>(p, st, p->vertex ? p->work64 : dp, du, dt, fc);
    count_launch(p);
    prof_mark(p, st, 6);
    const int G = grid_for(nib, T) < kIbBlocks ? grid_for(nib, T) : kIbBlocks;
    if (use_cond)
      launch_pdl(ib_change_kernel<VT, true>, G, T, 0, st, nib, d, (const VT *)fc, (const VT *)fo, p->dstats, p->partials, p->counters, p->ib_ctl, tol, max_iters, cond);
    else
      launch_pdl(ib_change_kernel<VT, false>, G, T, 0, st, nib, d, (const VT *)fc, (const VT *)fo, p->dstats, p->partials, p->counters, p->ib_ctl, tol, max_iters, cond);
    count_launch(p);
    prof_mark(p, st, 7);
  }
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

// Start of a time step: pass counter cleared, the initial force (IB entries of f_init, or zero)
// as the current iterate.
template <typename VT>
static pc_status ib_start(Plan *p, const VT *f_init, cudaStream_t st) {
  PC_CUDA_TRY(cudaMemsetAsync(p->ib_ctl, 0, offsetof(IbCtl, hist), st));
  ib_gather_kernel<VT><<<grid_for(p->nib, 256), 256, 0, st>>>((int)p->nib, (int)p->N, p->dim, p->ib_idx, f_init,
                                                              static_cast<VT *>(p->ib_f[1]));
  count_launch(p);
  return PC_OK;
}

void ib_drop_graph(Plan *p) {
  if (p->ib_graph.exec) cudaGraphExecDestroy(p->ib_graph.exec);
  if (p->ib_graph.graph) cudaGraphDestroy(p->ib_graph.graph);
  p->ib_graph = IbGraph{};
}

// The whole time step as one CUDA graph: start, first pass, a while node whose body is one later
// pass (its condition set on the device by the stopping rule), then the gradient and Eq. 4 at
// every node. Captured once per argument set on the plan's private streams with plain launches
// (no programmatic edges in the conditional body) and no profiler events.
template <typename VT>
static pc_status ib_capture(Plan *p, double dt, const VT *du, const VT *f_init, double tol, int max_iters,
                            double *dp, VT *duo, VT *dfo) {
  ib_drop_graph(p);
  if (!p->ib_body_stream) PC_CUDA_TRY(cudaStreamCreateWithFlags(&p->ib_body_stream, cudaStreamNonBlocking));
  cudaStream_t cs = p->cap_stream, bs = p->ib_body_stream;
  const bool prof = p->prof;
  p->prof = false;
  p->cur = nullptr;
  tl_plain_launch = true;
  const long long l0 = p->launches;
  long long l1 = 0, l2 = 0, l3 = 0;
  pc_status s = PC_OK;
  cudaGraph_t g = nullptr, body_done = nullptr;
  cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t node = nullptr;
    cudaGraphNodeParams cp = {};
    if (s == PC_OK) {
      ce = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, nullptr, nullptr, nullptr);
      if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&h, cg, 0u, cudaGraphCondAssignDefault);
      if (ce != cudaSuccess) s = fail(PC_ERR_CUDA, "IB loop graph: %s", cudaGetErrorString(ce));
    }
    if (s == PC_OK) s = ib_start<VT>(p, f_init, cs);
    if (s == PC_OK) s = ib_pass<VT>(p, true, dt, du, dp, tol, max_iters, true, h, cs);
    l1 = p->launches;
    if (s == PC_OK) {
      ce = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, &edges, &ndeps);
      if (ce == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ce = cudaGraphAddNode(&node, cg, deps, edges, ndeps, &cp);
      }
      if (ce == cudaSuccess) ce = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
      if (ce == cudaSuccess)
        ce = cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal);
      if (ce != cudaSuccess) s = fail(PC_ERR_CUDA, "IB loop graph: %s", cudaGetErrorString(ce));
      else {
        s = ib_pass<VT>(p, false, dt, du, dp, tol, max_iters, true, h, bs);
        if (s == PC_OK) {
          ib_guard_kernel<<<1, 32, 0, bs>>>(p->ib_ctl, max_iters, h);
          count_launch(p);
          if (cudaGetLastError() != cudaSuccess) s = fail(PC_ERR_CUDA, "IB loop guard launch failed");
        }
        ce = cudaStreamEndCapture(bs, &body_done);
        if (s == PC_OK && ce != cudaSuccess) s = fail(PC_ERR_CUDA, "IB loop body capture: %s", cudaGetErrorString(ce));
      }
    }
    l2 = p->launches;
    if (s == PC_OK) {
      launch_gradient(p, cs, p->vertex ? p->work64 : dp, du, dt, duo, dfo);
      count_launch(p);
      if (cudaGetLastError() != cudaSuccess) s = fail(PC_ERR_CUDA, "IB loop graph: gradient launch failed");
    }
    l3 = p->launches;
    ce = cudaStreamEndCapture(cs, &g);
    if (s == PC_OK && ce != cudaSuccess) s = fail(PC_ERR_CUDA, "IB loop capture: %s", cudaGetErrorString(ce));
  } else {
    s = fail(PC_ERR_CUDA, "IB loop capture: %s", cudaGetErrorString(ce));
  }
  tl_plain_launch = false;
  p->prof = prof;
  p->launches = l0;
  if (s != PC_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  cudaGraphExec_t ex = nullptr;
  ce = cudaGraphInstantiate(&ex, g, 0ULL);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(PC_ERR_CUDA, "IB loop graph instantiation: %s", cudaGetErrorString(ce));
  }
  IbGraph &e = p->ib_graph;
  e.graph = g; e.exec = ex;
  e.u = du; e.f = f_init; e.p = dp; e.uo = duo; e.fo = dfo; e.dt = dt; e.tol = tol; e.max_iters = max_iters;
  e.l_first = l1 - l0; e.l_body = l2 - l1; e.l_final = l3 - l2;
  return PC_OK;
}

template <typename VT>
static pc_status project_ib_impl(Plan *p, double dt, const VT *du, const VT *f_init, double tol, int max_iters,
                                 double *dp, VT *duo, VT *dfo, double *history, pc_ib_result *res,
                                 cudaStream_t st) {
  PC_TRY(ib_tables(p, st));
  IbCtl h;
  memset(&h, 0, offsetof(IbCtl, hist));
  if (p->nib == 0) {
    // no boundary/virtual nodes: one pass with zero force, nothing to iterate
    PC_TRY(ib_pass<VT>(p, true, dt, du, dp, tol, max_iters, false, 0, st));
    h.it = 1;
    h.conv = 1;
    h.hist[0] = h.hist[1] = 0.0;
    launch_gradient(p, st, p->vertex ? p->work64 : dp, du, dt, duo, dfo);
    count_launch(p);
    PC_CUDA_TRY(cudaGetLastError());
  } else if (p->graphs_on) {
    IbGraph &e = p->ib_graph;
    if (!(e.exec && e.u == du && e.f == f_init && e.p == dp && e.uo == duo && e.fo == dfo && e.dt == dt &&
          e.tol == tol && e.max_iters == max_iters))
      PC_TRY(ib_capture<VT>(p, dt, du, f_init, tol, max_iters, dp, duo, dfo));
    PC_CUDA_TRY(cudaGraphLaunch(e.exec, st));
    PC_CUDA_TRY(cudaMemcpyAsync(&h, p->ib_ctl, offsetof(IbCtl, hist) + 2 * sizeof(double) * max_iters,
                                cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    p->launches += e.l_first + (long long)(h.it - 1) * e.l_body + e.l_final;
  } else {
    // the same passes driven from the host: the pass counter and the decision are read back
    // after every pass
    PC_TRY(ib_start<VT>(p, f_init, st));
    for (int it = 0;; ++it) {
      PC_TRY(ib_pass<VT>(p, it == 0, dt, du, dp, tol, max_iters, false, 0, st));
      PC_CUDA_TRY(cudaMemcpyAsync(&h, p->ib_ctl, offsetof(IbCtl, hist), cudaMemcpyDeviceToHost, st));
      PC_CUDA_TRY(cudaStreamSynchronize(st));
      if (h.conv || h.it >= max_iters) break;
    }
    launch_gradient(p, st, p->vertex ? p->work64 : dp, du, dt, duo, dfo);
    count_launch(p);
    PC_CUDA_TRY(cudaGetLastError());
    PC_CUDA_TRY(cudaMemcpyAsync(&h, p->ib_ctl, offsetof(IbCtl, hist) + 2 * sizeof(double) * max_iters,
                                cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (history)
    for (int k = 0; k < h.it; ++k) { history[2 * k] = h.hist[2 * k]; history[2 * k + 1] = h.hist[2 * k + 1]; }
  if (res) {
    res->iterations = h.it;
    res->converged = h.conv;
    res->diff = h.it ? h.hist[2 * (h.it - 1)] : 0.0;
    res->prev = h.it ? h.hist[2 * (h.it - 1) + 1] : 0.0;
  }
  for (int k = 0; k < 2 * h.it; ++k)
    if (!std::isfinite(h.hist[k]))
      return fail(PC_ERR_NOT_CONVERGED, "the IB force is not finite after pass %d (diverged, or non-finite input)",
                  k / 2 + 1);
  return PC_OK;
}

}  // namespace pc

extern "C" pc_status pc_project(pc_plan *plan, double dt, const void *u_star, const void *f_ib_in,
                                double *p_out, void *u_out, void *f_ib_out, pc_stats *stats,
                                void *cuda_stream) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  if (p->grid_only) return pc::fail(PC_ERR_INVALID_ARG, "a grid-only plan has no nodes: use pc_solve_poisson");
  if (!u_star || !p_out || !u_out) return pc::fail(PC_ERR_INVALID_ARG, "u_star, p_out and u_out are required");
  if (!(dt > 0.0) || !std::isfinite(dt)) return pc::fail(PC_ERR_INVALID_ARG, "dt must be positive and finite");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) {
    if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device %d", p->device);
  }
  if (p->graphs_on && !stats &&
      (pc::graph_cached(p, dt, u_star, f_ib_in, p_out, u_out, f_ib_out) ||
       (pc::is_device_ptr(u_star) && pc::is_device_ptr(f_ib_in) && pc::is_device_ptr(p_out) &&
        pc::is_device_ptr(u_out) && pc::is_device_ptr(f_ib_out))))
    return pc::project_graph(p, dt, u_star, f_ib_in, p_out, u_out, f_ib_out, (cudaStream_t)cuda_stream);
  return pc::project_impl(p, dt, u_star, f_ib_in, p_out, u_out, f_ib_out, stats, (cudaStream_t)cuda_stream);
}

extern "C" pc_status pc_solve_poisson(pc_plan *plan, const double *s, double *p_out, pc_stats *stats,
                                      void *cuda_stream) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p || !s || !p_out) return pc::fail(PC_ERR_INVALID_ARG, "plan, s and p_out are required");
  if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device %d", p->device);
  // device arrays without statistics: one launch of a graph cached per (s, p_out)
  if (p->graphs_on && !stats && pc::is_device_ptr(s) && pc::is_device_ptr(p_out))
    return pc::solve_graph(p, s, p_out, (cudaStream_t)cuda_stream);
  if (p->vertex) return pc::vertex_solve(p, s, p_out, stats, (cudaStream_t)cuda_stream);
  return pc::solve_impl(p, s, p_out, stats, (cudaStream_t)cuda_stream);
}

extern "C" pc_status pc_project_ib(pc_plan *plan, double dt, const void *u_star, const void *f_ib_init,
                                   double tol, int max_iters, double *p_out, void *u_out, void *f_ib_out,
                                   double *history, pc_ib_result *result, void *cuda_stream) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  if (p->grid_only) return pc::fail(PC_ERR_INVALID_ARG, "a grid-only plan has no nodes");
  if (!u_star || !p_out || !u_out) return pc::fail(PC_ERR_INVALID_ARG, "u_star, p_out and u_out are required");
  if (!(dt > 0.0) || !std::isfinite(dt)) return pc::fail(PC_ERR_INVALID_ARG, "dt must be positive and finite");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return pc::fail(PC_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (max_iters < 1 || max_iters > pc::kIbMaxIters)
    return pc::fail(PC_ERR_INVALID_ARG, "max_iters must be in [1, %d]", pc::kIbMaxIters);
  if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device %d", p->device);
  if (!pc::is_device_ptr(u_star) || (f_ib_init && !pc::is_device_ptr(f_ib_init)) || !pc::is_device_ptr(p_out) ||
      !pc::is_device_ptr(u_out) || (f_ib_out && !pc::is_device_ptr(f_ib_out)))
    return pc::fail(PC_ERR_INVALID_ARG, "pc_project_ib takes device pointers only");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return pc::fail(PC_ERR_INVALID_ARG, "pc_project_ib waits on the host between passes and cannot be captured");
  if (p->vdtype == PC_DTYPE_F64)
    return pc::project_ib_impl<double>(p, dt, (const double *)u_star, (const double *)f_ib_init, tol, max_iters,
                                       p_out, (double *)u_out, (double *)f_ib_out, history, result, st);
  return pc::project_ib_impl<float>(p, dt, (const float *)u_star, (const float *)f_ib_init, tol, max_iters, p_out,
                                    (float *)u_out, (float *)f_ib_out, history, result, st);
}

extern "C" pc_status pc_plan_set_rhs_mask(pc_plan *plan, const uint8_t *mask, void *cuda_stream) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  if (p->grid_only) return pc::fail(PC_ERR_INVALID_ARG, "a grid-only plan has no projection to mask");
  if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device %d", p->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!mask) {
    if (p->rhs_mask_on) {
      p->rhs_mask_on = false;
      pc::plan_drop_graphs(p);
    }
    return PC_OK;
  }
  // one byte per pressure point: the cells, or the unknowns of a vertex grid
  const size_t nm = (size_t)(p->npts > 0 ? p->npts : p->ncells);
  if (!p->rhs_mask) PC_TRY(pc::plan_alloc(p, (void **)&p->rhs_mask, nm));
  PC_CUDA_TRY(cudaMemcpyAsync(p->rhs_mask, mask, nm, cudaMemcpyDefault, st));
  PC_CUDA_TRY(cudaStreamSynchronize(st));
  if (!p->rhs_mask_on) {
    p->rhs_mask_on = true;
    pc::plan_drop_graphs(p);   // captured launches hold the grid description without the mask
  }
  return PC_OK;
}
