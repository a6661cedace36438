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

// One axis pass over a tile of lines: [forward transform] [eigenvalue division] [inverse].
// Dynamic shared memory: two buffers of L*M complex slots (the FFT ping-pongs between them),
// then per line the eigenvalue sum of the other axes, the line's base cell index (-1 for lines
// past a ragged end) and its zero-mode flag. Threads beyond L * tpl (a batched launch sized for
// a larger tile) take part in the barriers only. Steps and barriers:
//   forward:  load line -> scatter to slots | FFT stages | post-process -> global (forward-only)
//             or -> real coefficients in the other buffer with the division fused |
//   inverse:  (inverse-only: load coefficients -> other buffer |) pre-process -> slots |
//             FFT stages | normalise and store.
template <typename Real, int EMAX>
__device__ __forceinline__ void axis_pass_body(const PassArgs<Real> &A, const int tile, unsigned char *smem_raw) {
  using T = typename Cplx<Real>::T;
  T *buf0 = reinterpret_cast<T *>(smem_raw);
  T *buf1 = buf0 + A.L * A.M;
  Real *lamo = reinterpret_cast<Real *>(buf1 + A.L * A.M);
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
  const bool dct4 = A.kind == KIND_ND || A.kind == KIND_DN;

  // All global loads of a thread are issued before any is used (memory-level parallelism).
  Real xin[2 * EMAX];
#pragma unroll
  for (int b = 0; b < 2 * EMAX; ++b) {
    const int j = g.lane + b * g.tpl;
    xin[b] = (valid && j < n) ? load_src(A, base + j * stride) : (Real)0;
  }
  T *res;        // buffer with the latest slots
  T *coef;       // buffer with the real coefficients for the inverse
  if (A.do_fwd) {
    // F1: scatter the real line into the complex slots (Makhoul / DCT-IV ordering).
#pragma unroll
    for (int b = 0; b < 2 * EMAX; ++b) {
      const int j = g.lane + b * g.tpl;
      if (j < n) {
        int q, comp;
        bool neg;
        fwd_slot_of(A.kind, n, j, q, comp, neg);
        reinterpret_cast<Real *>(&slot(buf0, g, line, q))[comp] = neg ? -xin[b] : xin[b];
      }
    }
    __syncthreads();
    res = fft_run<T, EMAX, false>(buf0, buf1, g, A.st, A.nst, A.tw, dct4 ? A.tw + tw_dct4pre(A.M) : nullptr);
    if (!A.do_inv) {
      // forward-only pass: the coefficients go straight to global memory (DST_WORK)
      if (valid) {
        Real *dst = static_cast<Real *>(A.dst);
        fwd_post(res, g, A.kind, n, A.tw, [&](int pos, Real X) { dst[base + pos * stride] = X; });
      }
      return;
    }
    coef = (res == buf0) ? buf1 : buf0;
    if (valid) {
      // p^ = s^ / (lambda_axis(j) + sum of the other axes' eigenvalues); zero mode -> 0
      const Real lo = lamo[line];
      const bool z = A.singular && lzero[line];
      const Real *la = A.lam[A.axis];
      const bool dv = A.do_div;
      fwd_post(res, g, A.kind, n, A.tw, [&](int pos, Real X) {
        if (dv) X = (z && pos == 0) ? (Real)0 : X / (__ldg(la + pos) + lo);
        realref(coef, g, line, pos) = X;
      });
    }
    __syncthreads();
  } else {
    // inverse-only pass: the coefficients are staged in shared memory first
    coef = buf1;
    res = buf0;
#pragma unroll
    for (int b = 0; b < 2 * EMAX; ++b) {
      const int j = g.lane + b * g.tpl;
      if (j < n) realref(coef, g, line, j) = xin[b];
    }
    __syncthreads();
  }
  if (!A.do_inv) return;
  // I1: coefficients -> slots (into the buffer the forward FFT result came from)
  T *slots = (coef == buf0) ? buf1 : buf0;
  if (valid) inv_pre(slots, g, A.kind, n, A.tw, [&](int i) -> Real { return realref(coef, g, line, i); });
  __syncthreads();
  if (dct4) res = fft_run<T, EMAX, false>(slots, coef, g, A.st, A.nst, A.tw, nullptr);
  else res = fft_run<T, EMAX, true>(slots, coef, g, A.st, A.nst, A.tw, nullptr);
  if (!valid) return;
  // I3: normalise and store, in chunks of 8 outputs (the old values of an accumulating store
  // are loaded together)
  const Real scale = A.out_scale;
  constexpr int kChunk = 8;
#pragma unroll
  for (int c0 = 0; c0 < 2 * EMAX; c0 += kChunk) {
    Real x[kChunk];
    // previous value of an accumulating store: an FP64 value or a (hi, lo) pair, 8 bytes either way
    unsigned long long old[kChunk];
    const bool acc = A.dst_mode == DST_F64_ADD || A.dst_mode == DST_PAIR_ADD;
#pragma unroll
    for (int b = 0; b < kChunk; ++b) {
      const int i = g.lane + (c0 + b) * g.tpl;
      x[b] = (i < n) ? inv_out(res, g, A.kind, n, A.tw, i) * scale : (Real)0;
      old[b] = (acc && i < n) ? static_cast<const unsigned long long *>(A.dst)[base + i * stride] : 0ULL;
    }
#pragma unroll
    for (int b = 0; b < kChunk; ++b) {
      const int i = g.lane + (c0 + b) * g.tpl;
      if (i >= n) continue;
      const int gi = base + i * stride;
      if (A.dst_mode == DST_WORK) {
        static_cast<Real *>(A.dst)[gi] = x[b];
      } else if (A.dst_mode == DST_PAIR_SET || A.dst_mode == DST_PAIR_ADD) {
        // FP32 passes only: the pair (hi, lo) += x with Knuth's TwoSum, renormalised
        float hi = (float)x[b], lo = 0.0f;
        if (A.dst_mode == DST_PAIR_ADD) {
          const float a = __uint_as_float((unsigned)old[b]), alo = __uint_as_float((unsigned)(old[b] >> 32));
          const float bb = hi;
          const float s1 = __fadd_rn(a, bb), z = __fsub_rn(s1, a);
          const float e = __fadd_rn(__fadd_rn(__fsub_rn(a, __fsub_rn(s1, z)), __fsub_rn(bb, z)), alo);
          hi = __fadd_rn(s1, e);
          lo = __fsub_rn(e, __fsub_rn(hi, s1));
        }
        static_cast<float2 *>(A.dst)[gi] = make_float2(hi, lo);
        if (A.f64) A.f64[gi] = f2d_bits(hi) + f2d_bits(lo);
      } else {
        static_cast<double *>(A.dst)[gi] =
            (A.dst_mode == DST_F64_SET) ? to_f64(x[b]) : __longlong_as_double((long long)old[b]) + to_f64(x[b]);
      }
    }
  }
}

template <typename Real, int EMAX>
__global__ void __launch_bounds__(kMaxPassThreads) axis_pass(PassArgs<Real> A) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  axis_pass_body<Real, EMAX>(A, blockIdx.x, smem_raw);
}

// Batched pass: CTA b processes tile items[b].y of the pass described by args[items[b].x] (one
// launch for every problem of a batch; each problem keeps its own tile shape).
template <typename Real, int EMAX>
__global__ void __launch_bounds__(kMaxPassThreads) axis_pass_batched(const PassArgs<Real> *__restrict__ args,
                                                                     const int2 *__restrict__ items) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) PassArgs<Real> A;
  const int2 it = items[blockIdx.x];
  {
    const unsigned *src = reinterpret_cast<const unsigned *>(args + it.x);
    unsigned *dst = reinterpret_cast<unsigned *>(&A);
    for (int w = threadIdx.x; w < (int)(sizeof(PassArgs<Real>) / 4); w += blockDim.x) dst[w] = __ldg(src + w);
  }
  __syncthreads();
  axis_pass_body<Real, EMAX>(A, it.y, smem_raw);
}

// ----------------------------------------------------------------------------- host side

// Radix schedule of a length-M FFT with at most E slots per thread: the largest power-of-two
// radices up to min(E, 16) first, then the factors 3 and 5.
static void radix_plan(int M, int E, int *radix, int &nr) {
  nr = 0;
  int m = M;
  int rmax = E < 16 ? E : 16;
  if (rmax < 2) rmax = 2;
  for (int r = rmax; r >= 2; r >>= 1)
    while (m % r == 0) { radix[nr++] = r; m /= r; }
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
    // eigenvalues per spectral index with the angle theta of each basis vector (th = theta/2):
    // central finite differences -(4/h^2) sin^2(theta/2), pseudo-spectral -(theta/h)^2
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
      lam[m] = p->eigen == PC_EIG_SPECTRAL ? -(2.0 * th / ax.h) * (2.0 * th / ax.h) : c * s * s;
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
  const int M = ax.M;
  // threads per line: a power of two with at most E slots per thread; the kernel instance is
  // the smallest power of two >= M / tpl
  const int E = (sizeof(Real) == 8) ? ax.slots64 : ax.slots32;
  const int tpl = 1 << ilog2((M + E - 1) / E);
  const int emax = 1 << ilog2((M + tpl - 1) / tpl);
  A.emax = emax;
  {
    int radix[kMaxRadices], nr;
    radix_plan(M, emax, radix, nr);
    A.nst = nr;
    int Ns = 1;
    for (int i = 0; i < nr; ++i) {
      StageInfo &si = A.st[i];
      si.R = radix[i];
      si.Ns = Ns;
      si.stride_m = M / (Ns * si.R);
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
  const int max_threads = batch_threads > 0 ? batch_threads : 256;
  const int max_lines = max_threads / tpl > 0 ? max_threads / tpl : 1;
  const int budget = 8192;          // complex slots per tile (two buffers: 2 x 64 KB in FP32)
  const int want_ctas = 2 * 152;    // two CTAs per SM on both dies
  int L;
  if (A.col) {
    // 32-byte row segments when the grid allows it, fewer lines when CTAs would be too few
    L = 32;
    while (L > 1 && (L * M > budget || L > max_lines)) L /= 2;
    long long outer = p->ncells / ((long long)stride * ax.n);
    const int Lmin = (sizeof(Real) == 8) ? 4 : 8;
    while (L > Lmin && batch_threads <= 0 && outer * ((stride + L - 1) / L) < want_ctas) L /= 2;
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
  A.f64 = ps.f64;
  threads = L * tpl;
  if (threads > kMaxPassThreads || L * M > budget)
    return fail(PC_ERR_UNSUPPORTED, "axis %d: tile of %d x %d too large", axis, L, M);
  if (batch_threads > 0 && emax > kBatchPassEmax)
    return fail(PC_ERR_UNSUPPORTED, "axis %d: %d slots per thread exceed the batched kernel", axis, emax);
  smem = 2 * (size_t)L * M * sizeof(T) + (size_t)L * (sizeof(Real) + 2 * sizeof(int));
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
  switch (A.emax) {
    case 1: case 2: launch_pdl(axis_pass<Real, 2>, (unsigned)tiles, threads, smem, st, A); break;
    case 4: launch_pdl(axis_pass<Real, 4>, (unsigned)tiles, threads, smem, st, A); break;
    case 8: launch_pdl(axis_pass<Real, 8>, (unsigned)tiles, threads, smem, st, A); break;
    case 16: launch_pdl(axis_pass<Real, 16>, (unsigned)tiles, threads, smem, st, A); break;
    default: return fail(PC_ERR_UNSUPPORTED, "no transform kernel for %d slots per thread", A.emax);
  }
  count_launch(p);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

template <typename Real>
pc_status launch_batched_pass(const PassArgs<Real> *dargs, const int2 *ditems, int nitems, int threads,
                              size_t smem, int emax, cudaStream_t st) {
  if (nitems <= 0) return PC_OK;
  switch (emax) {
    case 1: case 2: launch_pdl(axis_pass_batched<Real, 2>, (unsigned)nitems, threads, smem, st, dargs, ditems); break;
    case 4: launch_pdl(axis_pass_batched<Real, 4>, (unsigned)nitems, threads, smem, st, dargs, ditems); break;
    case 8: launch_pdl(axis_pass_batched<Real, 8>, (unsigned)nitems, threads, smem, st, dargs, ditems); break;
    case 16: launch_pdl(axis_pass_batched<Real, 16>, (unsigned)nitems, threads, smem, st, dargs, ditems); break;
    default: return fail(PC_ERR_UNSUPPORTED, "no batched transform kernel for %d slots per thread", emax);
  }
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}
template pc_status launch_batched_pass<float>(const PassArgs<float> *, const int2 *, int, int, size_t, int, cudaStream_t);
template pc_status launch_batched_pass<double>(const PassArgs<double> *, const int2 *, int, int, size_t, int, cudaStream_t);

// Kernel attributes set once per device, before any stream capture.
pc_status prepare_kernels() {
  const int lim = 200 * 1024;
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return PC_OK;
}

std::vector<PassSpec> solve_pass_specs(const Plan *p, bool fp32, int src_mode, const void *src,
                                       int dst_mode, void *dst, double *f64) {
  std::vector<PassSpec> v;
  void *work = fp32 ? (void *)p->work32 : (void *)p->work64;
  const int d = p->dim;
  int cur_mode = src_mode;
  const void *cur = src;
  for (int a = d - 1; a >= 1; --a) {     // forward passes: last axis down to axis 1
    v.push_back(PassSpec{a, true, false, false, cur_mode, cur, DST_WORK, work, nullptr});
    cur_mode = SRC_WORK;
    cur = work;
  }
  v.push_back(PassSpec{0, true, true, true, cur_mode, cur, DST_WORK, work, nullptr});   // axis 0, division
  for (int a = 1; a < d; ++a) {         // inverse passes: axis 1 up to the last axis
    const bool final_pass = (a == d - 1);
    v.push_back(PassSpec{a, false, false, true, SRC_WORK, work, final_pass ? dst_mode : DST_WORK,
                         final_pass ? dst : work, final_pass ? f64 : nullptr});
  }
  return v;
}

// Full solve with Real precision: src (cells, src_mode) -> dst (dst_mode).
template <typename Real>
static pc_status solve_real(Plan *p, int src_mode, const void *src, int dst_mode, void *dst,
                            cudaStream_t st, double *f64 = nullptr) {
  if (p->dim < 2) return fail(PC_ERR_UNSUPPORTED, "dim 1");
  for (const PassSpec &ps : solve_pass_specs(p, sizeof(Real) == 4, src_mode, src, dst_mode, dst, f64))
    PC_TRY(launch_pass<Real>(p, ps, st));
  return PC_OK;
}

pc_status solve_fp64_grid(Plan *p, const double *s, double *pout, cudaStream_t st) {
  return solve_real<double>(p, SRC_F64, s, DST_F64_SET, pout, st);
}

pc_status solve_fp32_grid(Plan *p, int src_mode, const void *s, int dst_mode, void *dst,
                          cudaStream_t st, double *f64) {
  return solve_real<float>(p, src_mode, s, dst_mode, dst, st, f64);
}

}  // namespace pc
