// Device code of the transform passes (§2.3 three-step solve): one axis pass over a tile of
// lines in shared memory (axis_pass_body), run by the single-problem kernel and by the batched
// kernel of pc_project_batch. The single-problem kernel is specialised on the transform family
// of the axis (KC: 0 real DFT, 1 DCT-II/DST-II, 2 DCT-IV/DST-IV) and on a power-of-two line
// length (no radix-3/5 stages), so an instance holds the code of one family only; the batched
// kernel dispatches each tile to the body of its family and length class. The arithmetic of a
// line is the same in every instance (the specialisation only removes branches), so single and
// batched results stay bitwise equal.
#pragma once

#include "fft.cuh"
#include "numeric.cuh"
#include "passes.cuh"
#include "pc_internal.cuh"

namespace pc {

// Transform kind of a pass: fixed by the family where the family has one member, else read
// (KC = -1: any cell-grid kind).
template <int KC>
__device__ __forceinline__ int pass_kind(int k) {
  if (KC == 0) return KIND_PP;
  if (KC == 1) return k == KIND_DD ? KIND_DD : KIND_NN;
  if (KC == 2) return k == KIND_DN ? KIND_DN : KIND_ND;
  if (KC == 3) return k == KIND_VDD ? KIND_VDD : KIND_VNN;
  if (KC == 4) return k == KIND_VDN ? KIND_VDN : KIND_VND;
  __builtin_assume(k >= KIND_PP && k <= KIND_DN);
  return k;
}

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

// I3: store the n outputs of this thread's line, in chunks of 8 (the old values of an
// accumulating store are loaded together). get(s, i) is output i, the s-th of this thread.
template <typename Real, int EMAX, typename Get>
__device__ __forceinline__ void store_line(const PassArgs<Real> &A, const TileGeom &g, int base, int n, Get get) {
  const int stride = A.stride;
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
      x[b] = (i < n) ? get(c0 + b, i) : (Real)0;
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

// One axis pass over a tile of lines: [forward transform] [eigenvalue division] [inverse].
// Dynamic shared memory: two buffers of L*M complex slots (the FFT ping-pongs between them),
// then per line the eigenvalue sum of the other axes, the line's base cell index (-1 for lines
// past a ragged end) and its zero-mode flag. Threads beyond L * tpl (a batched launch sized for
// a larger tile) take part in the barriers only. Steps and barriers:
//   forward:  load line -> scatter to slots | FFT stages | post-process -> global (forward-only)
//             or -> real coefficients in the other buffer with the division fused |
//   inverse:  (inverse-only: load coefficients -> other buffer |) pre-process -> slots |
//             FFT stages | normalise and store.
// The quarter-wave vertex kinds (family 4) run the cell grid's DCT-II/DST-II pair in the other
// order: analysis through its inverse (stage | pre-process | FFT | coefficients, divided, kept
// in registers |), synthesis through its forward (scatter | FFT | post-process -> other buffer
// | store).
template <typename Real, int EMAX, int KC = -1, bool POW2 = false>
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
      // the line's index along each axis (loops over constant indices: registers, no local array)
      int rem = base, idx[3] = {0, 0, 0};
#pragma unroll
      for (int b = 2; b >= 0; --b)
        if (b < A.dim) { idx[b] = rem % A.shape[b]; rem /= A.shape[b]; }
      Real lo = 0;
      int zero = 1;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (b >= A.dim || b == A.axis) continue;
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
  const int kind = pass_kind<KC>(A.kind);
  const bool dct4 = kind == KIND_ND || kind == KIND_DN;

  // All global loads of a thread are issued before any is used (memory-level parallelism).
  Real xin[2 * EMAX];
#pragma unroll
  for (int b = 0; b < 2 * EMAX; ++b) {
    const int j = g.lane + b * g.tpl;
    xin[b] = (valid && j < n) ? load_src(A, base + j * stride) : (Real)0;
  }

  if constexpr (KC == 4) {
    const int bk = (kind == KIND_VDN) ? KIND_DD : KIND_NN;   // the cell grid's pair, reversed
    if (A.do_fwd) {
      // analysis: the DCT-III / DST-III of the line (the cell grid's inverse), times 1/M
#pragma unroll
      for (int b = 0; b < 2 * EMAX; ++b) {
        const int j = g.lane + b * g.tpl;
        if (j < n) realref(buf1, g, line, j) = xin[b];
      }
      __syncthreads();
      if (valid) inv_pre(buf0, g, bk, n, A.tw, [&](int i) -> Real { return realref(buf1, g, line, i); });
      __syncthreads();
      T *res = fft_run<T, EMAX, true, POW2>(buf0, buf1, g, A.st, A.nst, A.tw, nullptr);
      const Real lo = A.do_div ? lamo[line] : (Real)0;
      const bool z = A.do_div && A.singular && lzero[line];
      const Real *la = A.lam[A.axis];
#pragma unroll
      for (int b = 0; b < 2 * EMAX; ++b) {
        const int i = g.lane + b * g.tpl;
        Real c = (valid && i < n) ? inv_out(res, g, bk, n, A.tw, i) * A.out_scale : (Real)0;
        if (A.do_div && valid && i < n) c = (z && i == 0) ? (Real)0 : c / (__ldg(la + i) + lo);
        xin[b] = c;
      }
      if (!A.do_inv) {
        // forward-only pass: the coefficients go to global memory (DST_WORK)
        if (valid) store_line<Real, EMAX>(A, g, base, n, [&](int s, int) -> Real { return s < 2 * EMAX ? xin[s] : (Real)0; });
        return;
      }
      __syncthreads();   // every thread has read the FFT result: both buffers are free
    }
    // synthesis: the DCT-II / DST-II of the coefficients in xin (the cell grid's forward)
#pragma unroll
    for (int b = 0; b < 2 * EMAX; ++b) {
      const int i = g.lane + b * g.tpl;
      if (i < n) {
        int q, comp;
        bool neg;
        fwd_slot_of(bk, n, i, q, comp, neg);
        reinterpret_cast<Real *>(&slot(buf0, g, line, q))[comp] = neg ? -xin[b] : xin[b];
      }
    }
    __syncthreads();
    T *res = fft_run<T, EMAX, false, POW2>(buf0, buf1, g, A.st, A.nst, A.tw, nullptr);
    T *outb = (res == buf0) ? buf1 : buf0;
    if (valid) fwd_post(res, g, bk, n, A.tw, [&](int pos, Real X) { realref(outb, g, line, pos) = X; });
    __syncthreads();
    if (valid) store_line<Real, EMAX>(A, g, base, n, [&](int, int i) -> Real { return realref(outb, g, line, i); });
    return;
  } else {
    T *res;        // buffer with the latest slots
    T *coef;       // buffer with the real coefficients for the inverse
    if (A.do_fwd) {
      // F1: scatter the real line into the complex slots (Makhoul / DCT-IV ordering; the even or
      // odd extension of a vertex DCT-I / DST-I line)
      if (kind == KIND_VNN || kind == KIND_VDD) {
#pragma unroll
        for (int b = 0; b < 2 * EMAX; ++b) {
          const int j = g.lane + b * g.tpl;
          if (j < n) ext_scatter(buf0, g, line, kind, j, xin[b]);
        }
        if (kind == KIND_VDD && g.lane == 0) {   // the zeros of the odd extension
          realref(buf0, g, line, 0) = (Real)0;
          realref(buf0, g, line, g.M) = (Real)0;
        }
      } else {
#pragma unroll
        for (int b = 0; b < 2 * EMAX; ++b) {
          const int j = g.lane + b * g.tpl;
          if (j < n) {
            int q, comp;
            bool neg;
            fwd_slot_of(kind, n, j, q, comp, neg);
            reinterpret_cast<Real *>(&slot(buf0, g, line, q))[comp] = neg ? -xin[b] : xin[b];
          }
        }
      }
      __syncthreads();
      res = fft_run<T, EMAX, false, POW2>(buf0, buf1, g, A.st, A.nst, A.tw, dct4 ? A.tw + tw_dct4pre(A.M) : nullptr);
      if (!A.do_inv) {
        // forward-only pass: the coefficients go straight to global memory (DST_WORK)
        if (valid) {
          Real *dst = static_cast<Real *>(A.dst);
          fwd_post(res, g, kind, n, A.tw, [&](int pos, Real X) { dst[base + pos * stride] = X; });
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
        fwd_post(res, g, kind, n, A.tw, [&](int pos, Real X) {
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
    if (valid) inv_pre(slots, g, kind, n, A.tw, [&](int i) -> Real { return realref(coef, g, line, i); });
    __syncthreads();
    if (dct4) res = fft_run<T, EMAX, false, POW2>(slots, coef, g, A.st, A.nst, A.tw, nullptr);
    else res = fft_run<T, EMAX, true, POW2>(slots, coef, g, A.st, A.nst, A.tw, nullptr);
    if (!valid) return;
    // I3: normalise and store
    const Real scale = A.out_scale;
    store_line<Real, EMAX>(A, g, base, n, [&](int, int i) -> Real { return inv_out(res, g, kind, n, A.tw, i) * scale; });
  }
}

// Single-problem pass: CTA b transforms tiles b * A.chunk, ... (A.chunk consecutive tiles).
template <typename Real, int EMAX, int KC, bool POW2>
__global__ void __launch_bounds__(kMaxPassThreads) axis_pass(PassArgs<Real> A) {
  pdl_enter();
  if (A.gate.st && refine_stopped_before(A.gate.st, A.gate.j, A.gate.tol)) return;   // refinement already ended
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t0 = blockIdx.x * A.chunk, t1 = min(t0 + A.chunk, A.ntiles);
  for (int t = t0; t < t1; ++t) {
    if (t > t0) __syncthreads();   // the previous tile no longer reads the buffers
    axis_pass_body<Real, EMAX, KC, POW2>(A, t, smem_raw);
  }
}

// Batched pass: one launch covers every problem of a batch whatever its transform family, line
// length and dimension. CTA b transforms tiles items[b].y, items[b].y + 1, ... (items[b].z of
// them) of the pass args[items[b].x]: consecutive tiles of one problem, so the pass arguments are
// read once per CTA and a pass that does nothing (a refinement sweep the stopping rule already
// ended) costs one CTA per chunk. The work list is sorted by family and length, so the CTAs
// resident at one time run the same code, and each tile runs the body of its (family,
// power-of-two length) class, the same code as the single-problem instance: batched and single
// results are bitwise equal.
template <typename Real, int EMAX>
__global__ void __launch_bounds__(kBatchedThreads, EMAX <= 4 ? 4 : (EMAX == 8 ? 3 : 2)) axis_pass_batched(const PassArgs<Real> *__restrict__ args,
                                                                        const int4 *__restrict__ items) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) PassArgs<Real> A;
  const int4 it = items[blockIdx.x];
  {
    const unsigned *src = reinterpret_cast<const unsigned *>(args + it.x);
    unsigned *dst = reinterpret_cast<unsigned *>(&A);
    for (int w = threadIdx.x; w < (int)(sizeof(PassArgs<Real>) / 4); w += blockDim.x) dst[w] = __ldg(src + w);
  }
  __syncthreads();
  // the gate is checked before the tile loads here (inside the body it would cost this kernel
  // spills: six bodies share its register budget)
  if (A.gate.st && refine_stopped_before(A.gate.st, A.gate.j, A.gate.tol)) return;
  const int cls = pass_family(A.kind) * 2 + (((A.M & (A.M - 1)) == 0) ? 1 : 0);
  for (int t = it.y; t < it.y + it.z; ++t) {
    if (t > it.y) __syncthreads();   // the previous tile no longer reads the buffers
    switch (cls) {
      case 0: axis_pass_body<Real, EMAX, 0, false>(A, t, smem_raw); break;
      case 1: axis_pass_body<Real, EMAX, 0, true>(A, t, smem_raw); break;
      case 2: axis_pass_body<Real, EMAX, 1, false>(A, t, smem_raw); break;
      case 3: axis_pass_body<Real, EMAX, 1, true>(A, t, smem_raw); break;
      case 4: axis_pass_body<Real, EMAX, 2, false>(A, t, smem_raw); break;
      default: axis_pass_body<Real, EMAX, 2, true>(A, t, smem_raw); break;
    }
  }
}

template <typename Real>
pc_status launch_batched(const PassArgs<Real> *dargs, const int4 *ditems, int nitems, int threads, size_t smem,
                         int emax, cudaStream_t st) {
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

template <typename Real>
pc_status prepare_batched(int lim) {
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<Real, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<Real, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<Real, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_batched<Real, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return PC_OK;
}

// Launch of the single-problem pass kernel of family KC on a pass of A.emax slots per thread,
// and the shared-memory attribute of its instances (set once per device).
template <typename Real, int KC, bool POW2>
pc_status launch_axis_pass_spec(const PassArgs<Real> &A, long long tiles, int threads, size_t smem, cudaStream_t st) {
  switch (A.emax) {
    case 1: case 2: launch_pdl(axis_pass<Real, 2, KC, POW2>, (unsigned)tiles, threads, smem, st, A); break;
    case 4: launch_pdl(axis_pass<Real, 4, KC, POW2>, (unsigned)tiles, threads, smem, st, A); break;
    case 8: launch_pdl(axis_pass<Real, 8, KC, POW2>, (unsigned)tiles, threads, smem, st, A); break;
    case 16: launch_pdl(axis_pass<Real, 16, KC, POW2>, (unsigned)tiles, threads, smem, st, A); break;
    default: return fail(PC_ERR_UNSUPPORTED, "no transform kernel for %d slots per thread", A.emax);
  }
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}
template <typename Real, int KC, bool POW2>
pc_status prepare_axis_pass_spec(int lim) {
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<Real, 2, KC, POW2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<Real, 4, KC, POW2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<Real, 8, KC, POW2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass<Real, 16, KC, POW2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return PC_OK;
}

}  // namespace pc
