// Device code of the transform passes (§2.3 three-step solve): one axis pass over a tile of
// lines in shared memory (axis_pass_body), run by the single-problem kernel and by the
// persistent kernel of pc_project_batch. The single-problem kernel is specialised on the
// transform family of the axis (KC: 0 real DFT, 1 DCT-II/DST-II, 2 DCT-IV/DST-IV) and on a
// power-of-two line length (no radix-3/5 stages), so an instance holds the code of one family
// only; the persistent kernel takes every family and length at run time (KC = -1) and stages
// its next tile with TMA bulk copies. The arithmetic of a line is the same in every instance
// (the specialisation only removes branches), so single and batched results stay bitwise equal.
#pragma once

#include "fft.cuh"
#include "numeric.cuh"
#include "passes.cuh"
#include "pc_internal.cuh"

namespace pc {

// Transform kind of a pass: fixed by the family where the family has one member, else read.
template <int KC>
__device__ __forceinline__ int pass_kind(int k) {
  if (KC == 0) return KIND_PP;
  if (KC == 1) return k == KIND_DD ? KIND_DD : KIND_NN;
  if (KC == 2) return k == KIND_DN ? KIND_DN : KIND_ND;
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

// One axis pass over a tile of lines: [forward transform] [eigenvalue division] [inverse].
// Dynamic shared memory: two buffers of L*M complex slots (the FFT ping-pongs between them),
// then per line the eigenvalue sum of the other axes, the line's base cell index (-1 for lines
// past a ragged end) and its zero-mode flag. Threads beyond L * tpl (a batched launch sized for
// a larger tile) take part in the barriers only. Steps and barriers:
//   forward:  load line -> scatter to slots | FFT stages | post-process -> global (forward-only)
//             or -> real coefficients in the other buffer with the division fused |
//   inverse:  (inverse-only: load coefficients -> other buffer |) pre-process -> slots |
//             FFT stages | normalise and store.
// No-op hook of axis_pass_body.
struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// stg (nullable): the tile's input already staged in shared memory by the caller (row tiles:
// line l at stg[l n + j]; column tiles: position j at stg[j L + l]), read instead of global
// memory. after_load() is called by every thread once the tile's input has been consumed (after
// the barrier that follows the scatter into the FFT buffers), when stg may be refilled.
template <typename Real, int EMAX, int KC = -1, bool POW2 = false, typename Hook = NoHook>
__device__ __forceinline__ void axis_pass_body(const PassArgs<Real> &A, const int tile, unsigned char *smem_raw,
                                               const Real *stg = nullptr, Hook after_load = Hook()) {
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
  const int kind = pass_kind<KC>(A.kind);
  const bool dct4 = kind == KIND_ND || kind == KIND_DN;

  // All global loads of a thread are issued before any is used (memory-level parallelism).
  Real xin[2 * EMAX];
  if (stg) {
    const Real *sl = A.col ? stg + line : stg + line * n;
    const int sst = A.col ? A.L : 1;
#pragma unroll
    for (int b = 0; b < 2 * EMAX; ++b) {
      const int j = g.lane + b * g.tpl;
      xin[b] = (valid && j < n) ? sl[j * sst] : (Real)0;
    }
  } else {
#pragma unroll
    for (int b = 0; b < 2 * EMAX; ++b) {
      const int j = g.lane + b * g.tpl;
      xin[b] = (valid && j < n) ? load_src(A, base + j * stride) : (Real)0;
    }
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
        fwd_slot_of(kind, n, j, q, comp, neg);
        reinterpret_cast<Real *>(&slot(buf0, g, line, q))[comp] = neg ? -xin[b] : xin[b];
      }
    }
    __syncthreads();
    after_load();
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
    after_load();
  }
  if (!A.do_inv) return;
  // I1: coefficients -> slots (into the buffer the forward FFT result came from)
  T *slots = (coef == buf0) ? buf1 : buf0;
  if (valid) inv_pre(slots, g, kind, n, A.tw, [&](int i) -> Real { return realref(coef, g, line, i); });
  __syncthreads();
  if (dct4) res = fft_run<T, EMAX, false, POW2>(slots, coef, g, A.st, A.nst, A.tw, nullptr);
  else res = fft_run<T, EMAX, true, POW2>(slots, coef, g, A.st, A.nst, A.tw, nullptr);
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
      x[b] = (i < n) ? inv_out(res, g, kind, n, A.tw, i) * scale : (Real)0;
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

template <typename Real, int EMAX, int KC, bool POW2>
__global__ void __launch_bounds__(kMaxPassThreads) axis_pass(PassArgs<Real> A) {
  pdl_enter();
  if (A.gate.st && refine_stopped_before(A.gate.st, A.gate.j, A.gate.tol)) return;   // refinement already ended
  extern __shared__ __align__(16) unsigned char smem_raw[];
  axis_pass_body<Real, EMAX, KC, POW2>(A, blockIdx.x, smem_raw);
}

// ----------------------------------------------------------------------------- tile staging
// The persistent pass stages the next tile's input into shared memory with TMA bulk copies
// (cp.async.bulk, completion counted in bytes on an mbarrier) while the current tile is being
// transformed, so the global-memory latency of the loads is off the critical path. Waits on the
// mbarrier are bounded: a copy that never lands sets FLAG_TIMEOUT in the problem's status word
// and the CTA returns (after a second bounded wait for its copies in flight).
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Whether the pass *G (in global memory) belongs to a refinement sweep that the stopping rule
// already ended: every thread reading it gets the same answer.
template <typename Real>
__device__ __forceinline__ bool gate_closed(const PassArgs<Real> *G) {
  const DevStats *st =
      reinterpret_cast<const DevStats *>(__ldg(reinterpret_cast<const unsigned long long *>(&G->gate.st)));
  return st && refine_stopped_before(st, __ldg(&G->gate.j), __ldg(&G->gate.tol));
}

// Warp 0 of the CTA: stage the input of tile t of pass *G into stg, if the pass reads 4-byte
// elements whose tile rows start on 16-byte boundaries (row tiles: n % 4 == 0; column tiles:
// stride and lines per tile multiples of 4) and its problem is not skipped. Returns (uniformly
// over the warp) whether a copy was issued; its bytes complete the current phase of bar.
template <typename Real>
__device__ __noinline__ bool stage_tile(const PassArgs<Real> *G, int t, Real *stg, unsigned long long *bar) {
  if (sizeof(Real) != 4) return false;
  const int src_mode = __ldg(&G->src_mode);
  const char *src = reinterpret_cast<const char *>(__ldg(reinterpret_cast<const unsigned long long *>(&G->src)));
  if (src_mode == SRC_F64 || (reinterpret_cast<unsigned long long>(src) & 15)) return false;
  const int n = __ldg(&G->n), L = __ldg(&G->L), col = __ldg(&G->col), stride = __ldg(&G->stride);
  const int lane = threadIdx.x & 31;
  if (col) {
    if ((stride & 3) || (L & 3)) return false;
    const int tpo = __ldg(&G->tiles_per_outer), inner = __ldg(&G->inner);
    const int o = t / tpo;
    const int f0 = (t - o * tpo) * L;
    const int lv = min(L, inner - f0);
    const long long base = (long long)o * n * stride + f0;
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(bar, (unsigned)(n * lv * 4));
    }
    __syncwarp();
    for (int j = lane; j < n; j += 32)
      bulk_g2s(stg + (long long)j * L, src + 4 * (base + (long long)j * stride), (unsigned)(lv * 4), bar);
  } else {
    if (n & 3) return false;
    const int lines = __ldg(&G->lines);
    const int line0 = t * L;
    const int lc = min(L, lines - line0);
    const long long bytes = (long long)lc * n * 4;
    const char *from = src + 4 * ((long long)line0 * n);
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(bar, (unsigned)bytes);
    }
    __syncwarp();
    constexpr long long kChunk = 4096;
    for (long long c = (long long)lane * kChunk; c < bytes; c += 32 * kChunk)
      bulk_g2s(reinterpret_cast<char *>(stg) + c, from + c, (unsigned)min(kChunk, bytes - c), bar);
  }
  return true;
}

// Persistent batched pass: a grid of at most (resident CTAs per SM) x (SMs) CTAs walks the work
// list, CTA b taking items b, b + gridDim.x, ...; item (a, t) is tile t of the pass args[a]. One
// launch covers every problem of a batch whatever its transform family, line length and
// dimension; the work list is sorted by family and length, so the CTAs resident at one time run
// the same code, one body per (family, power-of-two length) as in the single-problem kernel.
// Each tile is transformed exactly as by the single-problem kernel. Dynamic shared memory: the
// gate table (gate_bytes), the staging buffer (stage_bytes), then the body's buffers.
// Gated launches (refinement sweeps under the stopping rule): the items' pass arguments are
// args[a0, a0 + nargs); each CTA first evaluates every one's gate into the table, one byte per
// pass, so an item is checked with one shared-memory read (passes beyond the table's bytes are
// checked in global memory).
template <typename Real, int EMAX>
__global__ void __launch_bounds__(kPersistentThreads, 3) axis_pass_persistent(const PassArgs<Real> *__restrict__ args,
                                                                        const int2 *__restrict__ items, int nitems,
                                                                        int stage_bytes, int gate_bytes, int a0,
                                                                        int nargs, int gated) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) PassArgs<Real> A;
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int s_staged, s_ok;
  unsigned char *gates = smem_raw;
  Real *stg = reinterpret_cast<Real *>(smem_raw + gate_bytes);   // 16-byte aligned: the bulk copies' rule
  unsigned char *body_smem = smem_raw + gate_bytes + stage_bytes;
  const bool use_stage = stage_bytes > 0;
  if (gated)
    for (int a = threadIdx.x; a < nargs && a < gate_bytes; a += blockDim.x) gates[a] = gate_closed(args + a0 + a) ? 1 : 0;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    s_staged = 0;
  }
  __syncthreads();
  auto closed = [&](int ai) -> bool {
    if (!gated) return false;
    const int g = ai - a0;
    return (g >= 0 && g < gate_bytes && g < nargs) ? gates[g] != 0 : gate_closed(args + ai);
  };
  if (use_stage && threadIdx.x < 32 && (int)blockIdx.x < nitems) {
    const int2 w0 = items[blockIdx.x];
    const bool st = !closed(w0.x) && stage_tile(args + w0.x, w0.y, stg, &bar);
    if (threadIdx.x == 0) s_staged = st ? 1 : 0;
  }
  unsigned phase = 0;
  int cur = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];
    // an item of a problem whose refinement already stopped is passed over without a barrier:
    // every thread reads the same flag (set by an earlier kernel), and such an item is never
    // staged, so the staging state carries over to the next item unchanged
    if (closed(w.x)) continue;
    __syncthreads();   // the previous tile no longer reads A or the buffers; s_staged is set
    if (w.x != cur) {
      const unsigned *src = reinterpret_cast<const unsigned *>(args + w.x);
      unsigned *dst = reinterpret_cast<unsigned *>(&A);
      for (int k = threadIdx.x; k < (int)(sizeof(PassArgs<Real>) / 4); k += blockDim.x) dst[k] = __ldg(src + k);
      cur = w.x;
    }
    const bool staged = s_staged != 0;
    if (staged && threadIdx.x == 0) {
      bool ok = mbar_wait_bounded(&bar, phase);
      if (!ok) mbar_wait_bounded(&bar, phase);   // copies still in flight: a second bounded wait
      s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (staged) {
      if (!s_ok) {
        if (threadIdx.x == 0 && A.err) atomicOr(A.err, (unsigned)FLAG_TIMEOUT);
        return;
      }
      if (threadIdx.x != 0) mbar_wait_bounded(&bar, phase);   // completed: returns at once
      phase ^= 1u;
    }
    const int next = it + gridDim.x;
    auto after_load = [&]() {
      if (use_stage && threadIdx.x < 32) {
        const bool st = next < nitems && !closed(items[next].x) && stage_tile(args + items[next].x, items[next].y, stg, &bar);
        if (threadIdx.x == 0) s_staged = st ? 1 : 0;
      }
    };
    // the body of the item's transform family and length class (registers are allocated for
    // the largest of the six, not for a body that holds every family at once)
    const Real *in = staged ? stg : nullptr;
    switch (pass_family(A.kind) * 2 + (((A.M & (A.M - 1)) == 0) ? 1 : 0)) {
      case 0: axis_pass_body<Real, EMAX, 0, false>(A, w.y, body_smem, in, after_load); break;
      case 1: axis_pass_body<Real, EMAX, 0, true>(A, w.y, body_smem, in, after_load); break;
      case 2: axis_pass_body<Real, EMAX, 1, false>(A, w.y, body_smem, in, after_load); break;
      case 3: axis_pass_body<Real, EMAX, 1, true>(A, w.y, body_smem, in, after_load); break;
      case 4: axis_pass_body<Real, EMAX, 2, false>(A, w.y, body_smem, in, after_load); break;
      default: axis_pass_body<Real, EMAX, 2, true>(A, w.y, body_smem, in, after_load); break;
    }
  }
}

template <typename Real>
pc_status launch_persistent(const PassArgs<Real> *dargs, const int2 *ditems, int nitems, int grid, int threads,
                            size_t smem, int stage_bytes, int gate_bytes, int a0, int nargs, int gated, int emax,
                            cudaStream_t st) {
  if (nitems <= 0) return PC_OK;
  const size_t sm = smem + (size_t)stage_bytes + (size_t)gate_bytes;
#define PC_PERS(E)                                                                                                  \
  launch_pdl(axis_pass_persistent<Real, E>, (unsigned)grid, threads, sm, st, dargs, ditems, nitems, stage_bytes, \
             gate_bytes, a0, nargs, gated)
  switch (emax) {
    case 1: case 2: PC_PERS(2); break;
    case 4: PC_PERS(4); break;
    case 8: PC_PERS(8); break;
    case 16: PC_PERS(16); break;
    default: return fail(PC_ERR_UNSUPPORTED, "no persistent transform kernel for %d slots per thread", emax);
  }
#undef PC_PERS
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

// Resident CTAs per SM of the persistent instance for emax slots, threads and smem bytes.
template <typename Real>
int persistent_ctas_per_sm(int emax, int threads, size_t smem) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (emax) {
    case 1: case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, axis_pass_persistent<Real, 2>, threads, smem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, axis_pass_persistent<Real, 4>, threads, smem); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, axis_pass_persistent<Real, 8>, threads, smem); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, axis_pass_persistent<Real, 16>, threads, smem); break;
    default: break;
  }
  if (e != cudaSuccess) { cudaGetLastError(); return 1; }
  return n > 0 ? n : 1;
}

template <typename Real>
pc_status prepare_persistent(int lim) {
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_persistent<Real, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_persistent<Real, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_persistent<Real, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  PC_CUDA_TRY(cudaFuncSetAttribute(axis_pass_persistent<Real, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
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
