// Transform-based Poisson solve on the pressure grid (§2.3, three-step algorithm):
//   1. forward 1D transforms along each axis in turn,
//   2. division by the sum of the 1D eigenvalues of the central-difference Laplacian,
//   3. backward 1D transforms.
// One kernel launch per axis pass. The contiguous (last) axis is processed in row tiles, the
// other axes in column tiles of W adjacent lines so that every global access is coalesced
// without a transpose. The division is fused into the pass of axis 0, which does its forward
// transform, the division and its inverse transform on the tile while it sits in shared memory.
// 2D: [fwd ax1] -> [fwd ax0, divide, inv ax0] -> [inv ax1]; 3D adds ax1 passes around the middle.
//
// Mixed precision: the transforms run in FP32; the iterate p is kept in FP64 and corrected by
// sweeps p += solve32(s - L_h p) whose residual is formed in FP64 (iterative refinement).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fft.cuh"
#include "numeric.cuh"
#include "passes.cuh"
#include "pc_internal.cuh"

namespace pc {

// Source element gi in the pass precision (FP64 sources enter FP32 passes truncated to 24 bits,
// by integer operations; the refinement corrects what that drops).
__device__ __forceinline__ float to_real(double v, float *) { return d2f_rz_bits(v); }
__device__ __forceinline__ double to_real(double v, double *) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f2d_bits(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }

template <typename Real>
__device__ __forceinline__ Real load_src(const PassArgs<Real> &A, int gi) {
  if (A.src_mode == SRC_F32) return (Real)__ldg(static_cast<const float *>(A.src) + gi);
  if (A.src_mode == SRC_F64) return to_real(__ldg(static_cast<const double *>(A.src) + gi), (Real *)nullptr);
  return static_cast<const Real *>(A.src)[gi];
}

constexpr int kLoadsPerThread = 2 * kSlotsPerThread;   // n / tpl <= 8

// One axis pass over a tile of lines: [forward transform] [eigenvalue division] [inverse].
// Dynamic shared memory: L*M complex slots, then per line the eigenvalue sum of the other
// axes, the line's base cell index (-1 for lines past a ragged end) and its zero-mode flag.
// Threads beyond L * tpl (a batched launch sized for a larger tile) take part in the barriers
// only.
template <typename Real>
__device__ __forceinline__ void axis_pass_body(const PassArgs<Real> &A, const int tile, unsigned char *smem_raw) {
  using T = typename Cplx<Real>::T;
  T *buf = reinterpret_cast<T *>(smem_raw);
  Real *lamo = reinterpret_cast<Real *>(buf + A.L * A.M);
  int *lbase = reinterpret_cast<int *>(lamo + A.L);
  int *lzero = lbase + A.L;
  const int t = threadIdx.x;
  const bool active = t < (A.L << A.tpl_bits);
  TileGeom g;
  g.L = A.L;
  g.M = A.M;
  g.tpl = 1 << A.tpl_bits;
  if (A.col) { g.es = A.L; g.ls = 1; g.line = t & (A.L - 1); g.lane = t >> A.lbits; }
  else { g.es = 1; g.ls = A.M; g.line = t >> A.tpl_bits; g.lane = t & (g.tpl - 1); }
  if (!active) { g.line = 0; g.lane = 1 << 24; }   // every position loop is empty
  const int n = A.n;

  if (t < A.L) {
    int base, valid;
    if (A.col) {
      int o = tile / A.tiles_per_outer;
      int f = (tile - o * A.tiles_per_outer) * A.L + t;
      valid = f < A.inner;
      base = o * n * A.stride + f;
    } else {
      int line = tile * A.L + t;
      valid = line < A.lines;
      base = line * n;
    }
    lbase[t] = valid ? base : -1;
    if (A.do_div && valid) {
      int rem = base, idx[3] = {0, 0, 0};
      for (int b = A.dim - 1; b >= 0; --b) { idx[b] = rem % A.shape[b]; rem /= A.shape[b]; }
      Real lo = 0;
      int zero = 1;
      for (int b = 0; b < A.dim; ++b) {
        if (b == A.axis) continue;
        lo += A.lam[b][idx[b]];
        zero &= idx[b] == 0;
      }
      lamo[t] = lo;
      lzero[t] = zero;
    }
  }
  __syncthreads();
  const int line = g.line;
  const int base = lbase[line];
  const bool valid = active && base >= 0;
  const int stride = A.stride;
  const bool fft_inv_dir = !(A.kind == KIND_ND || A.kind == KIND_DN);

  // All global loads of a thread are issued before any is used (memory-level parallelism).
  Real xin[kLoadsPerThread];
#pragma unroll
  for (int b = 0; b < kLoadsPerThread; ++b) {
    const int j = g.lane + b * g.tpl;
    xin[b] = (valid && j < n) ? load_src(A, base + j * stride) : (Real)0;
  }
  if (A.do_fwd) {
    // F1: scatter the real line into the complex slots (Makhoul / DCT-IV ordering).
#pragma unroll
    for (int b = 0; b < kLoadsPerThread; ++b) {
      const int j = g.lane + b * g.tpl;
      if (j < n) {
        int q, comp;
        bool neg;
        fwd_slot_of(A.kind, n, j, q, comp, neg);
        reinterpret_cast<Real *>(&slot(buf, g, line, q))[comp] = neg ? -xin[b] : xin[b];
      }
    }
    __syncthreads();
    pretwiddle(buf, g, A.kind, A.tw);
    fft_lines(buf, g, A.st, A.nst, A.tw, false);
    fwd_post(buf, g, A.kind, n, A.tw);
  } else {
#pragma unroll
    for (int b = 0; b < kLoadsPerThread; ++b) {
      const int j = g.lane + b * g.tpl;
      if (j < n) realref(buf, g, line, j) = xin[b];
    }
    __syncthreads();
  }

  if (A.do_div) {
    // p^ = s^ / (lambda_axis(j) + sum of the other axes' eigenvalues); zero mode -> 0.
    if (valid) {
      const Real lo = lamo[line];
      const bool z = A.singular && lzero[line];
      const Real *la = A.lam[A.axis];
      for (int j = g.lane; j < n; j += g.tpl) {
        Real &v = realref(buf, g, line, j);
        v = (z && j == 0) ? (Real)0 : v / (__ldg(la + j) + lo);
      }
    }
    __syncthreads();
  }

  if (A.do_inv) {
    inv_pre(buf, g, A.kind, n, A.tw);
    fft_lines(buf, g, A.st, A.nst, A.tw, fft_inv_dir);
    inv_post_twiddle(buf, g, A.kind, A.tw);
    if (!valid) return;
    double old[kLoadsPerThread];
    if (A.dst_mode == DST_F64_ADD) {
#pragma unroll
      for (int b = 0; b < kLoadsPerThread; ++b) {
        const int i = g.lane + b * g.tpl;
        old[b] = (i < n) ? static_cast<const double *>(A.dst)[base + i * stride] : 0.0;
      }
    }
#pragma unroll
    for (int b = 0; b < kLoadsPerThread; ++b) {
      const int i = g.lane + b * g.tpl;
      if (i >= n) continue;
      int j;
      bool neg;
      inv_src_of(A.kind, n, i, j, neg);
      Real x = realref(buf, g, line, j) * (neg ? -A.out_scale : A.out_scale);
      int gi = base + i * stride;
      if (A.dst_mode == DST_WORK) static_cast<Real *>(A.dst)[gi] = x;
      else if (A.dst_mode == DST_F64_SET) static_cast<double *>(A.dst)[gi] = to_f64(x);
      else static_cast<double *>(A.dst)[gi] = old[b] + to_f64(x);
    }
  } else {
    if (!valid) return;
#pragma unroll
    for (int b = 0; b < kLoadsPerThread; ++b) {
      const int j = g.lane + b * g.tpl;
      if (j < n) static_cast<Real *>(A.dst)[base + j * stride] = realref(buf, g, line, j);
    }
  }
}

template <typename Real>
__global__ void __launch_bounds__(1024) axis_pass(PassArgs<Real> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  axis_pass_body<Real>(A, blockIdx.x, smem_raw);
}

// Batched pass: CTA b processes tile items[b].y of the pass described by args[items[b].x] (one
// launch for every problem of a batch; each problem keeps its own tile shape).
template <typename Real>
__global__ void __launch_bounds__(1024) axis_pass_batched(const PassArgs<Real> *__restrict__ args,
                                                          const int2 *__restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) PassArgs<Real> A;
  const int2 it = items[blockIdx.x];
  {
    const unsigned *src = reinterpret_cast<const unsigned *>(args + it.x);
    unsigned *dst = reinterpret_cast<unsigned *>(&A);
    for (int w = threadIdx.x; w < (int)(sizeof(PassArgs<Real>) / 4); w += blockDim.x) dst[w] = __ldg(src + w);
  }
  __syncthreads();
  axis_pass_body<Real>(A, it.y, smem_raw);
}

// ----------------------------------------------------------------------------- host side

static void radix_plan(int M, int *radix, int &nr) {
  nr = 0;
  int m = M;
  while (m % 4 == 0) { radix[nr++] = 4; m /= 4; }
  while (m % 2 == 0) { radix[nr++] = 2; m /= 2; }
  while (m % 3 == 0) { radix[nr++] = 3; m /= 3; }
  while (m % 5 == 0) { radix[nr++] = 5; m /= 5; }
}

static int ilog2(int v) {
  int b = 0;
  while ((1 << b) < v) ++b;
  return b;
}

bool axis_length_supported(int n) {
  if (n < 2 || (n & 1)) return false;
  int m = n / 2;
  for (int r : {2, 3, 5}) while (m % r == 0) m /= r;
  return m == 1 && n / 2 <= 2048;
}

pc_status build_axis_tables(Plan *p) {
  for (int a = 0; a < p->dim; ++a) {
    AxisInfo &ax = p->ax[a];
    const int n = ax.n, M = n / 2;
    ax.M = M;
    radix_plan(M, ax.radix, ax.nradix);
    std::vector<double2> tw(tw_total(M));
    auto put = [&](int off, int k, double ang) { tw[off + k] = make_double2(std::cos(ang), std::sin(ang)); };
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < M; ++k) put(0, k, -2.0 * pi * k / M);
    for (int k = 0; k <= M; ++k) put(tw_rdft(M), k, -2.0 * pi * k / n);
    for (int k = 0; k <= M; ++k) put(tw_quarter(M), k, -pi * k / (2.0 * n));
    for (int k = 0; k < M; ++k) put(tw_dct4pre(M), k, -pi * (4.0 * k + 1.0) / (4.0 * n));
    for (int k = 0; k < M; ++k) put(tw_dct4post(M), k, -pi * k / (double)n);
    std::vector<float2> tw32(tw.size());
    for (size_t i = 0; i < tw.size(); ++i) tw32[i] = make_float2((float)tw[i].x, (float)tw[i].y);
    // eigenvalues per spectral index, -(4/h^2) sin^2(theta/2) with the angle of each basis
    std::vector<double> lam(n);
    std::vector<float> lam32(n);
    const double c = -4.0 / (ax.h * ax.h);
    for (int m = 0; m < n; ++m) {
      double th;  // sin argument
      switch (ax.kind) {
        case KIND_PP: {
          int w = (m == 0) ? 0 : (m == 1 ? n / 2 : m / 2);
          th = pi * w / n;
          break;
        }
        case KIND_NN: th = pi * m / (2.0 * n); break;
        case KIND_DD: th = pi * (m + 1.0) / (2.0 * n); break;
        default: th = pi * (2.0 * m + 1.0) / (4.0 * n); break;
      }
      double s = std::sin(th);
      lam[m] = c * s * s;
      lam32[m] = (float)lam[m];
    }
    PC_TRY(plan_alloc(p, (void **)&ax.tw64, tw.size() * sizeof(double2)));
    PC_TRY(plan_alloc(p, (void **)&ax.tw32, tw32.size() * sizeof(float2)));
    PC_TRY(plan_alloc(p, (void **)&ax.lam64, n * sizeof(double)));
    PC_TRY(plan_alloc(p, (void **)&ax.lam32, n * sizeof(float)));
    PC_CUDA_TRY(cudaMemcpy(ax.tw64, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice));
    PC_CUDA_TRY(cudaMemcpy(ax.tw32, tw32.data(), tw32.size() * sizeof(float2), cudaMemcpyHostToDevice));
    PC_CUDA_TRY(cudaMemcpy(ax.lam64, lam.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    PC_CUDA_TRY(cudaMemcpy(ax.lam32, lam32.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  }
  return PC_OK;
}

template <typename Real>
pc_status build_pass(const Plan *p, const PassSpec &ps, PassArgs<Real> &A, long long &tiles, int &threads,
                     size_t &smem, int batch_threads) {
  using T = typename Cplx<Real>::T;
  const int axis = ps.axis;
  const bool fwd = ps.fwd, div = ps.div, inv = ps.inv;
  const int src_mode = ps.src_mode, dst_mode = ps.dst_mode;
  const void *src = ps.src;
  void *dst = ps.dst;
  const AxisInfo &ax = p->ax[axis];
  memset(&A, 0, sizeof(A));
  A.axis = axis;
  A.kind = ax.kind;
  A.n = ax.n;
  A.M = ax.M;
  A.nst = ax.nradix;
  {
    int Ns = 1;
    for (int i = 0; i < ax.nradix; ++i) {
      StageInfo &si = A.st[i];
      si.R = ax.radix[i];
      si.Ns = Ns;
      si.stride_m = ax.M / (Ns * si.R);
      si.shift = ((Ns & (Ns - 1)) == 0) ? ilog2(Ns) : -1;
      si.magic = (unsigned)(((1ULL << 32) + Ns - 1) / Ns);
      Ns *= si.R;
    }
  }
  A.tw = (const T *)(sizeof(Real) == 8 ? (const void *)ax.tw64 : (const void *)ax.tw32);
  A.dim = p->dim;
  int stride = 1;
  for (int b = 0; b < p->dim; ++b) A.shape[b] = (int)p->n[b];
  for (int b = axis + 1; b < p->dim; ++b) stride *= (int)p->n[b];
  A.stride = stride;
  const int last = p->dim - 1;
  A.col = axis != last;
  const int M = ax.M;
  // threads per line: a power of two >= M/4 (bounds the registers held across barriers)
  const int tpl = 1 << ilog2((M + kSlotsPerThread - 1) / kSlotsPerThread);
  const int max_lines = 1024 / tpl;
  const int budget = 4096;          // complex slots per tile
  const int want_ctas = 152;        // at least one CTA per SM on both dies
  int L;
  if (A.col) {
    // 32-byte row segments when the grid allows it, fewer lines when CTAs would be too few
    L = (sizeof(Real) == 8) ? 4 : 8;
    while (L * 2 <= 32 && L * 2 * M <= budget && L * 2 <= max_lines) L *= 2;
    long long outer = p->ncells / ((long long)stride * ax.n);
    if (batch_threads > 0) L = 32;   // a batch fills its CTAs from many problems
    while (L > 1 && batch_threads <= 0 && outer * ((stride + L - 1) / L) < want_ctas) L /= 2;
    while (L > 1 && batch_threads > 0 && L * tpl > batch_threads) L /= 2;
    while (L > 1 && (L * M > budget || L > max_lines)) L /= 2;
    if (L > stride) L = 1 << (ilog2(stride + 1) - 1);
    A.inner = stride;
    A.tiles_per_outer = (stride + L - 1) / L;
    tiles = outer * A.tiles_per_outer;
  } else {
    long long lines = p->ncells / ax.n;
    L = budget / M;
    if (L < 1) L = 1;
    L = 1 << (ilog2(L + 1) - 1);
    while (L > max_lines) L /= 2;
    while (L > 1 && batch_threads <= 0 && (lines + L - 1) / L < want_ctas) L /= 2;
    while (L > 1 && batch_threads > 0 && L * tpl > batch_threads) L /= 2;
    A.lines = (int)lines;
    tiles = (lines + L - 1) / L;
  }
  A.L = L;
  A.lbits = ilog2(L);
  A.tpl_bits = ilog2(tpl);
  A.do_fwd = fwd;
  A.do_div = div;
  A.do_inv = inv;
  for (int b = 0; b < p->dim; ++b)
    A.lam[b] = (const Real *)(sizeof(Real) == 8 ? (const void *)p->ax[b].lam64 : (const void *)p->ax[b].lam32);
  A.singular = p->singular;
  A.src_mode = src_mode;
  A.src = src;
  A.dst_mode = dst_mode;
  A.dst = dst;
  A.out_scale = (Real)inv_scale(ax.kind, ax.n);
  threads = L * tpl;
  if (threads > 1024 || L * M > 2 * budget)
    return fail(PC_ERR_UNSUPPORTED, "axis %d: tile of %d x %d too large", axis, L, M);
  smem = (size_t)L * M * sizeof(T) + (size_t)L * (sizeof(Real) + 2 * sizeof(int));
  return PC_OK;
}

template pc_status build_pass<float>(const Plan *, const PassSpec &, PassArgs<float> &, long long &, int &, size_t &, int);
template pc_status build_pass<double>(const Plan *, const PassSpec &, PassArgs<double> &, long long &, int &, size_t &, int);

template <typename Real>
static pc_status launch_pass(Plan *p, const PassSpec &ps, cudaStream_t st) {
  PassArgs<Real> A;
  long long tiles;
  int threads;
  size_t smem;
  PC_TRY(build_pass<Real>(p, ps, A, tiles, threads, smem, 0));
  axis_pass<Real><<<(unsigned)tiles, threads, smem, st>>>(A);
  count_launch(p);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

template <typename Real>
pc_status launch_batched_pass(const PassArgs<Real> *dargs, const int2 *ditems, int nitems, int threads,
                              size_t smem, cudaStream_t st) {
  if (nitems <= 0) return PC_OK;
  axis_pass_batched<Real><<<(unsigned)nitems, threads, smem, st>>>(dargs, ditems);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}
template pc_status launch_batched_pass<float>(const PassArgs<float> *, const int2 *, int, int, size_t, cudaStream_t);
template pc_status launch_batched_pass<double>(const PassArgs<double> *, const int2 *, int, int, size_t, cudaStream_t);

// Kernel attributes set once per device, before any stream capture.
pc_status prepare_kernels() {
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  return PC_OK;
}

std::vector<PassSpec> solve_pass_specs(const Plan *p, bool fp32, int src_mode, const void *src,
                                       int dst_mode, void *dst) {
  std::vector<PassSpec> v;
  void *work = fp32 ? (void *)p->work32 : (void *)p->work64;
  const int d = p->dim;
  int cur_mode = src_mode;
  const void *cur = src;
  for (int a = d - 1; a >= 1; --a) {     // forward passes: last axis down to axis 1
    v.push_back(PassSpec{a, true, false, false, cur_mode, cur, DST_WORK, work});
    cur_mode = SRC_WORK;
    cur = work;
  }
  v.push_back(PassSpec{0, true, true, true, cur_mode, cur, DST_WORK, work});   // axis 0 with the division
  for (int a = 1; a < d; ++a) {         // inverse passes: axis 1 up to the last axis
    const bool final_pass = (a == d - 1);
    v.push_back(PassSpec{a, false, false, true, SRC_WORK, work, final_pass ? dst_mode : DST_WORK,
                         final_pass ? dst : work});
  }
  return v;
}

// Full solve with Real precision: src (cells, src_mode) -> dst (dst_mode).
template <typename Real>
static pc_status solve_real(Plan *p, int src_mode, const void *src, int dst_mode, void *dst,
                            cudaStream_t st) {
  if (p->dim < 2) return fail(PC_ERR_UNSUPPORTED, "dim 1");
  for (const PassSpec &ps : solve_pass_specs(p, sizeof(Real) == 4, src_mode, src, dst_mode, dst))
    PC_TRY(launch_pass<Real>(p, ps, st));
  return PC_OK;
}

pc_status solve_fp64_grid(Plan *p, const double *s, double *pout, cudaStream_t st) {
  return solve_real<double>(p, SRC_F64, s, DST_F64_SET, pout, st);
}

pc_status solve_fp32_grid(Plan *p, int src_mode, const void *s, int dst_mode, double *pout,
                          cudaStream_t st) {
  return solve_real<float>(p, src_mode, s, dst_mode, pout, st);
}

}  // namespace pc
