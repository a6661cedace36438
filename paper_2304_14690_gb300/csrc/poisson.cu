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
#include "pc_internal.cuh"

namespace pc {

enum SrcMode { SRC_F32 = 0, SRC_F64 = 1, SRC_WORK = 2 };
enum DstMode { DST_WORK = 0, DST_F64_SET = 1, DST_F64_ADD = 2 };

template <typename Real>
struct PassArgs {
  using T = typename Cplx<Real>::T;
  int axis, kind, n, M, nradix;
  int radix[kMaxRadices];
  const T *tw;
  int dim;
  int shape[3];
  long long stride;     // element stride along the axis
  long long inner;      // column tiles: number of line positions f (= stride)
  long long lines;      // row tiles: number of lines
  int L;                // lines per tile
  int col;              // 1: column tile
  int tiles_per_outer;  // column tiles: ceil(inner / L)
  int do_fwd, do_div, do_inv;
  const Real *lam[3];
  int singular;
  int src_mode;
  const void *src;
  int dst_mode;
  void *dst;
  Real out_scale;       // normalisation of the inverse (2/n)
};

template <typename Real>
__device__ __forceinline__ long long line_base(const PassArgs<Real> &A, int tile, int l, bool &valid) {
  if (A.col) {
    long long o = tile / A.tiles_per_outer;
    long long f = (long long)(tile % A.tiles_per_outer) * A.L + l;
    valid = f < A.inner;
    return o * (long long)A.n * A.stride + f;
  }
  long long line = (long long)tile * A.L + l;
  valid = line < A.lines;
  return line * A.n;
}

template <typename Real>
__device__ __forceinline__ Real load_src(const PassArgs<Real> &A, long long gi) {
  if (A.src_mode == SRC_F32) return (Real)static_cast<const float *>(A.src)[gi];
  if (A.src_mode == SRC_F64) return (Real)static_cast<const double *>(A.src)[gi];
  return static_cast<const Real *>(A.src)[gi];
}

template <typename Real>
__global__ void __launch_bounds__(1024) axis_pass(PassArgs<Real> A) {
  using T = typename Cplx<Real>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);
  TileGeom g;
  g.L = A.L;
  g.M = A.M;
  if (A.col) { g.es = A.L; g.ls = 1; g.line_fastest = true; }
  else { g.es = 1; g.ls = A.M; g.line_fastest = false; }
  const int tile = blockIdx.x;
  const int n = A.n;
  const int items = A.L * n;
  const bool fft_inv_dir = !(A.kind == KIND_ND || A.kind == KIND_DN);

  if (A.do_fwd) {
    // F1: scatter the real line into the complex slots (Makhoul / DCT-IV ordering).
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
      int line, j;
      decode(g, t, n, line, j);
      bool valid;
      long long base = line_base(A, tile, line, valid);
      Real x = valid ? load_src(A, base + (long long)j * A.stride) : (Real)0;
      int q, comp;
      float sgn;
      fwd_slot_of(A.kind, n, j, q, comp, sgn);
      reinterpret_cast<Real *>(&slot(buf, g, line, q))[comp] = (Real)sgn * x;
    }
    __syncthreads();
    pretwiddle(buf, g, A.kind, A.tw);
    fft_lines(buf, g, A.radix, A.nradix, A.tw, false);
    fwd_post(buf, g, A.kind, n, A.tw);
  } else {
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
      int line, j;
      decode(g, t, n, line, j);
      bool valid;
      long long base = line_base(A, tile, line, valid);
      realref(buf, g, line, j) = valid ? load_src(A, base + (long long)j * A.stride) : (Real)0;
    }
    __syncthreads();
  }

  if (A.do_div) {
    // p^ = s^ / (lambda_axis(j) + sum of the other axes' eigenvalues); zero mode -> 0.
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
      int line, j;
      decode(g, t, n, line, j);
      bool valid;
      long long base = line_base(A, tile, line, valid);
      if (!valid) continue;
      long long rem = base;   // cell index of element j = 0 of the line
      int idx[3] = {0, 0, 0};
      for (int b = A.dim - 1; b >= 0; --b) {
        idx[b] = (int)(rem % A.shape[b]);
        rem /= A.shape[b];
      }
      idx[A.axis] = j;
      Real lam = 0;
      bool zero = true;
      for (int b = 0; b < A.dim; ++b) {
        lam += A.lam[b][idx[b]];
        zero = zero && idx[b] == 0;
      }
      Real &v = realref(buf, g, line, j);
      v = (A.singular && zero) ? (Real)0 : v / lam;
    }
    __syncthreads();
  }

  if (A.do_inv) {
    inv_pre(buf, g, A.kind, n, A.tw);
    fft_lines(buf, g, A.radix, A.nradix, A.tw, fft_inv_dir);
    inv_post_twiddle(buf, g, A.kind, A.tw);
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
      int line, i;
      decode(g, t, n, line, i);
      bool valid;
      long long base = line_base(A, tile, line, valid);
      if (!valid) continue;
      int j;
      float sgn;
      inv_src_of(A.kind, n, i, j, sgn);
      Real x = realref(buf, g, line, j) * ((Real)sgn * A.out_scale);
      long long gi = base + (long long)i * A.stride;
      if (A.dst_mode == DST_WORK) static_cast<Real *>(A.dst)[gi] = x;
      else if (A.dst_mode == DST_F64_SET) static_cast<double *>(A.dst)[gi] = (double)x;
      else static_cast<double *>(A.dst)[gi] += (double)x;
    }
  } else {
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
      int line, j;
      decode(g, t, n, line, j);
      bool valid;
      long long base = line_base(A, tile, line, valid);
      if (!valid) continue;
      static_cast<Real *>(A.dst)[base + (long long)j * A.stride] = realref(buf, g, line, j);
    }
  }
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
static pc_status launch_pass(Plan *p, int axis, bool fwd, bool div, bool inv, int src_mode,
                             const void *src, int dst_mode, void *dst, cudaStream_t st) {
  using T = typename Cplx<Real>::T;
  const AxisInfo &ax = p->ax[axis];
  PassArgs<Real> A;
  memset(&A, 0, sizeof(A));
  A.axis = axis;
  A.kind = ax.kind;
  A.n = ax.n;
  A.M = ax.M;
  A.nradix = ax.nradix;
  for (int i = 0; i < ax.nradix; ++i) A.radix[i] = ax.radix[i];
  A.tw = (const T *)(sizeof(Real) == 8 ? (const void *)ax.tw64 : (const void *)ax.tw32);
  A.dim = p->dim;
  long long stride = 1;
  for (int b = 0; b < p->dim; ++b) A.shape[b] = (int)p->n[b];
  for (int b = axis + 1; b < p->dim; ++b) stride *= p->n[b];
  A.stride = stride;
  const int last = p->dim - 1;
  A.col = axis != last;
  const int M = ax.M;
  // Tile size: up to 4096 complex slots; column tiles need >= 32 bytes per row segment.
  const int budget = 4096;
  long long tiles;
  if (A.col) {
    int W = (int)(sizeof(Real) == 8 ? 4 : 8);
    while (W * 2 * M <= budget && W < 32) W *= 2;
    while (W > 1 && W * M > budget) W /= 2;
    if (W > stride) W = (int)stride;
    A.L = W;
    A.inner = stride;
    A.tiles_per_outer = (int)((stride + W - 1) / W);
    long long outer = p->ncells / (stride * ax.n);
    tiles = outer * A.tiles_per_outer;
  } else {
    long long lines = p->ncells / ax.n;
    int L = budget / M;
    if (L < 1) L = 1;
    // keep several CTAs per SM when the grid is small
    while (L > 1 && (lines + L - 1) / L < 4 * 152) L /= 2;
    A.L = L;
    A.lines = lines;
    tiles = (lines + L - 1) / L;
  }
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
  int slots = A.L * M;
  int threads = ((slots / kSlotsPerThread + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  if (threads > 1024) threads = 1024;
  // pairs of the real-DFT wrappers: L*(M/2+1) <= threads*(kSlotsPerThread/2+1) needs L <= threads
  if (threads * kSlotsPerThread < slots || A.L > threads)
    return fail(PC_ERR_UNSUPPORTED, "axis %d: tile of %d slots too large", axis, slots);
  size_t smem = (size_t)slots * sizeof(T);
  static bool attr_set[2] = {false, false};
  if (!attr_set[sizeof(Real) == 8]) {
    PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set[sizeof(Real) == 8] = true;
  }
  axis_pass<Real><<<(unsigned)tiles, threads, smem, st>>>(A);
  count_launch(p);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

// Full solve with Real precision: src (cells, src_mode) -> dst (dst_mode).
template <typename Real>
static pc_status solve_real(Plan *p, int src_mode, const void *src, int dst_mode, void *dst,
                            cudaStream_t st) {
  Real *work = (Real *)(sizeof(Real) == 8 ? (void *)p->work64 : (void *)p->work32);
  const int d = p->dim;
  if (d == 1) return fail(PC_ERR_UNSUPPORTED, "dim 1");
  // forward passes: last axis down to 1
  int cur_mode = src_mode;
  const void *cur = src;
  for (int a = d - 1; a >= 1; --a) {
    PC_TRY(launch_pass<Real>(p, a, true, false, false, cur_mode, cur, DST_WORK, work, st));
    cur_mode = SRC_WORK;
    cur = work;
  }
  // axis 0: forward, divide, inverse
  bool last_pass = (d == 1);
  (void)last_pass;
  PC_TRY(launch_pass<Real>(p, 0, true, true, true, cur_mode, cur, DST_WORK, work, st));
  // inverse passes: axis 1 .. last; the last one writes the destination
  for (int a = 1; a < d; ++a) {
    bool final_pass = (a == d - 1);
    PC_TRY(launch_pass<Real>(p, a, false, false, true, SRC_WORK, work,
                             final_pass ? dst_mode : DST_WORK, final_pass ? dst : (void *)work, st));
  }
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
