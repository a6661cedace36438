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
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lean_pass.cuh"

namespace pc {

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

// A complex FFT length the passes take: 2^a 3^b 5^c, at most 2048.
static bool fft_length_supported(int M) {
  if (M < 2 || M > 2048) return false;
  int m = M;
  for (int r : {2, 3, 5}) while (m % r == 0) m /= r;
  return m == 1;
}

bool axis_length_supported(int n) { return n >= 2 && (n & 1) == 0 && fft_length_supported(n / 2); }

int fft_length_of(int kind, int n) {
  if (kind == KIND_VNN) return n - 1;   // DCT-I of m + 1 unknowns: real DFT of length 2m
  if (kind == KIND_VDD) return n + 1;   // DST-I of m - 1 unknowns: real DFT of length 2m
  return n / 2;
}

bool vertex_axis_supported(int kind, int m) {
  if (kind == KIND_VNN || kind == KIND_VDD) return fft_length_supported(m);
  return axis_length_supported(m);   // P-P and the quarter-wave pairs: length m, m even
}

pc_status build_axis_tables(Plan *p) {
  for (int a = 0; a < p->dim; ++a) {
    AxisInfo &ax = p->ax[a];
    const int n = ax.n, M = fft_length_of(ax.kind, n);
    const int nt = 2 * M;   // length of the real transform the FFT serves (n for cell kinds)
    ax.M = M;
    std::vector<double2> tw(tw_total(M));
    auto put = [&](int off, int k, double ang) { tw[off + k] = make_double2(std::cos(ang), std::sin(ang)); };
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < M; ++k) put(0, k, -2.0 * pi * k / M);
    for (int k = 0; k <= M; ++k) put(tw_rdft(M), k, -2.0 * pi * k / nt);
    for (int k = 0; k <= M; ++k) put(tw_quarter(M), k, -pi * k / (2.0 * nt));
    for (int k = 0; k < M; ++k) put(tw_dct4pre(M), k, -pi * (4.0 * k + 1.0) / (4.0 * nt));
    for (int k = 0; k < M; ++k) put(tw_dct4post(M), k, -pi * k / (double)nt);
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
        // vertex grids: M cells on DCT-I / DST-I axes, basis cos(pi k j/M) and sin(pi (k+1) j/M)
        // for coefficient k; n cells on quarter-wave axes, theta = pi (k + 1/2)/n
        case KIND_VNN: th = pi * m / (2.0 * M); break;
        case KIND_VDD: th = pi * (m + 1.0) / (2.0 * M); break;
        default: th = pi * (2.0 * m + 1.0) / (4.0 * n); break;   // ND, DN, VND, VDN
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
  // slots per thread; 0 and 1 (FP32 only): variant 0 or 1 of the lean pass of the length
  // (lean_pass.cuh) where it has one, else 4
  int E = (sizeof(Real) == 8) ? ax.slots64 : ax.slots32;
  // the lean passes move row tiles in 16-byte accesses (16-byte aligned arrays), store forward
  // coefficients as FP32 work and read inverse-only coefficients in FP32
  auto al16 = [](const void *q) { return ((uintptr_t)q & 15) == 0; };
  const bool row = axis == p->dim - 1;
  const bool lean_io = (!fwd || inv || dst_mode == DST_WORK) && (fwd || src_mode != SRC_F64) &&
                       (!row || (al16(src) && al16(dst) && al16(ps.f64)));
  const bool lean = sizeof(Real) == 4 && E <= 1 && pass_family(ax.kind) <= 2 && lean::length_ok(M) && lean_io;
  const int lv = E == 1 ? 1 : 0;
  if (E <= 1) E = 4;
  // threads per line: a power of two with at most E slots per thread; the kernel instance is
  // the smallest power of two >= M / tpl. A line must fit one CTA: longer lines take more
  // slots per thread (up to 16)
  while (E < 16 && (M + E - 1) / E > kMaxPassThreads) E *= 2;
  const int tpl = 1 << ilog2((M + E - 1) / E);
  const int emax = 1 << ilog2((M + tpl - 1) / tpl);
  A.emax = emax;
  if (!lean) {
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
  A.out_scale = (Real)inv_scale(ax.M);
  A.f64 = ps.f64;
  A.gate = ps.gate;
  A.chunk = ps.chunk > 1 ? ps.chunk : 1;
  if (lean) {
    // compile-time tile: L lines of T = M / E threads each, 256 threads
    const int L = lean::lines_of(M, lv);
    if (A.col) {
      const long long outer = p->ncells / ((long long)stride * ax.n);
      A.inner = stride;
      A.tiles_per_outer = (stride + L - 1) / L;
      tiles = outer * A.tiles_per_outer;
    } else {
      const long long lines = p->ncells / ax.n;
      A.lines = (int)lines;
      tiles = (lines + L - 1) / L;
    }
    A.L = L;
    A.lean = lean::lean_id(M, pass_family(ax.kind));
    threads = lean::kThreads;
    A.ntiles = (int)tiles;
    smem = lean::smem_of(M, lv);
    return PC_OK;
  }
  const int max_threads = batch_threads > 0 ? batch_threads : 256;
  const int max_lines = max_threads / tpl > 0 ? max_threads / tpl : 1;
  const int budget = 8192;          // complex slots per tile (two buffers: 2 x 64 KB in FP32)
  // CTAs per SM the tile size aims for (part of the plan's schedule; 152 SMs on both dies)
  const int want_ctas = ((sizeof(Real) == 8) ? ax.ctas64 : ax.ctas32) * 152;
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
  threads = L * tpl;
  A.ntiles = (int)tiles;
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
  tiles = (tiles + A.chunk - 1) / A.chunk;   // CTAs
  if constexpr (sizeof(Real) == 4) {
    if (A.lean) {
      PC_TRY(launch_lean(A.lean, A, nullptr, nullptr, (unsigned)tiles, threads, smem, st));
      count_launch(p);
      return PC_OK;
    }
    // FP32 passes: the instance of the axis's transform family (one translation unit each)
    switch (pass_family(A.kind)) {
      case 0: PC_TRY(launch_pass_f32_family0(A, tiles, threads, smem, st)); break;
      case 1: PC_TRY(launch_pass_f32_family1(A, tiles, threads, smem, st)); break;
      case 2: PC_TRY(launch_pass_f32_family2(A, tiles, threads, smem, st)); break;
      default: PC_TRY(launch_pass_vertex_f32(A, tiles, threads, smem, st)); break;
    }
  } else {
    if (pass_family(A.kind) >= 3) PC_TRY(launch_pass_vertex_f64(A, tiles, threads, smem, st));
    else PC_TRY((launch_axis_pass_spec<Real, -1, false>(A, tiles, threads, smem, st)));
  }
  count_launch(p);
  return PC_OK;
}

// Kernel attributes set once per device, before any stream capture.
pc_status prepare_kernels() {
  const int lim = 200 * 1024;
  PC_TRY(prepare_pass_f32_family0(lim));
  PC_TRY(prepare_pass_f32_family1(lim));
  PC_TRY(prepare_pass_f32_family2(lim));
  PC_TRY(prepare_pass_vertex(lim));
  PC_TRY(prepare_batched_f32(lim));
  PC_TRY(prepare_lean(lim));
  PC_TRY((prepare_axis_pass_spec<double, -1, false>(lim)));
  return PC_OK;
}

std::vector<PassSpec> solve_pass_specs(const Plan *p, bool fp32, int src_mode, const void *src,
                                       int dst_mode, void *dst, double *f64, RefineGate gate, int chunk) {
  std::vector<PassSpec> v;
  void *work = fp32 ? (void *)p->work32 : (void *)p->work64;
  const int d = p->dim;
  int cur_mode = src_mode;
  const void *cur = src;
  for (int a = d - 1; a >= 1; --a) {     // forward passes: last axis down to axis 1
    v.push_back(PassSpec{a, true, false, false, cur_mode, cur, DST_WORK, work, nullptr, gate, chunk});
    cur_mode = SRC_WORK;
    cur = work;
  }
  v.push_back(PassSpec{0, true, true, true, cur_mode, cur, DST_WORK, work, nullptr, gate, chunk});   // axis 0, division
  for (int a = 1; a < d; ++a) {         // inverse passes: axis 1 up to the last axis
    const bool final_pass = (a == d - 1);
    v.push_back(PassSpec{a, false, false, true, SRC_WORK, work, final_pass ? dst_mode : DST_WORK,
                         final_pass ? dst : work, final_pass ? f64 : nullptr, gate, chunk});
  }
  return v;
}

// Full solve with Real precision: src (cells, src_mode) -> dst (dst_mode).
template <typename Real>
static pc_status solve_real(Plan *p, int src_mode, const void *src, int dst_mode, void *dst,
                            cudaStream_t st, double *f64 = nullptr, RefineGate gate = RefineGate{nullptr, 0, 0.0f},
                            int chunk = 1) {
  if (p->dim < 2) return fail(PC_ERR_UNSUPPORTED, "dim 1");
  for (const PassSpec &ps : solve_pass_specs(p, sizeof(Real) == 4, src_mode, src, dst_mode, dst, f64, gate, chunk))
    PC_TRY(launch_pass<Real>(p, ps, st));
  return PC_OK;
}

pc_status solve_fp64_grid(Plan *p, const double *s, double *pout, cudaStream_t st) {
  return solve_real<double>(p, SRC_F64, s, DST_F64_SET, pout, st);
}

pc_status solve_fp32_grid(Plan *p, int src_mode, const void *s, int dst_mode, void *dst,
                          cudaStream_t st, double *f64, RefineGate gate, int chunk) {
  return solve_real<float>(p, src_mode, s, dst_mode, dst, st, f64, gate, chunk);
}

}  // namespace pc
