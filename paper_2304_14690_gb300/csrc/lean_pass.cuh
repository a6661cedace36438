// Compile-time FP32 transform passes (§2.3 three-step solve) for the cell-grid transform families
// (real DFT, DCT-II/DST-II, DCT-IV/DST-IV) at the line lengths n = 2M the workloads use
// (M in {16, 32, 48, 64, 96, 128, 192, 256, 384, 512}).
//
// The general passes (axis_pass.cuh) take the line length, the radix schedule and the tile
// shape at run time; their index arithmetic, predication and twiddle addressing cost about 130
// thread instructions per cell and pass. Here every one of these is a compile-time constant:
//   - a tile is L lines x M complex slots in shared memory, slot-major with the line index fast
//     (slot q of line l at q * LP + l, LP = L + 1), so the FFT's accesses (every thread of a
//     half-warp on another line, the same slot) are conflict-free whatever the slot pattern;
//   - each line is served by T = M / E threads holding E complex values in registers; the FFT
//     is a Stockham autosort whose stages (radix 16, 8, 4, 2 and a final 3) each read E slots,
//     twiddle, run the small DFTs in registers and write E slots (two barriers, one buffer).
//     Two schedules per length: variant 0 with the most slots per thread (fewest instructions)
//     and variant 1 with fewer (more warps for small grids);
//   - the inverse transform runs the same forward FFT on conjugated slots (conj(FFT(conj Z))
//     is the inverse DFT), so a length has one FFT body, out of line and shared by a pass's
//     forward and inverse halves;
//   - in a pass that divides (forward, division, inverse), each thread post-processes a pair of
//     slots (k, M - k; DCT-IV: k, M - 1 - k) into four coefficients, divides them and
//     pre-processes the same pair for the inverse in registers, with no barrier in between;
//   - global memory moves in quads of four consecutive cells (16-byte accesses on row tiles,
//     four coalesced scalar accesses across lines on column tiles); forward-only passes store
//     each pair's coefficients, and inverse-only passes load them, straight from global memory.
// The thread-to-slot maps of the real-to-real wrappers follow fft.cuh (Makhoul's reordering;
// DCT-IV through a half-length FFT with pre- and post-twiddles).
#pragma once

#include "axis_pass.cuh"

namespace pc {
namespace lean {

constexpr int kThreads = 256;   // CTA size of every lean pass

// Two variants per length: v = 0, large slot counts E (few threads per line, radix-16/8 stages:
// the fewest instructions per cell, for grids that fill the GPU); v = 1, smaller E (more threads
// per line and more warps, for single grids too small to hide latency with v = 0). T = M / E
// threads per line, L = 256 / T lines per tile.
__host__ __device__ constexpr int slots_of(int M, int v = 0) {
  return v == 0 ? (M == 16 ? 4 : M == 32 ? 8 : M == 48 ? 12 : M == 64 ? 8 : M == 96 ? 24 : M == 128 ? 16
                  : M == 192 ? 24 : M == 256 ? 16 : M == 384 ? 24 : M == 512 ? 32 : 0)
                : (M == 16 ? 4 : M == 32 ? 4 : M == 48 ? 12 : M == 64 ? 4 : M == 96 ? 12 : M == 128 ? 8
                  : M == 192 ? 12 : M == 256 ? 4 : M == 384 ? 12 : M == 512 ? 8 : 0);
}
__host__ __device__ constexpr bool length_ok(int M) { return slots_of(M) > 0; }
__host__ __device__ constexpr int lines_of(int M, int v = 0) { return kThreads / (M / slots_of(M, v)); }
// Shared memory of one tile: slots, then per line its eigenvalue sum, base cell and zero flag.
__host__ __device__ constexpr int smem_of(int M, int v = 0) {
  return M * (lines_of(M, v) + 1) * 8 + lines_of(M, v) * 12;
}
// Register class of a length: 0 for E <= 16 in both variants (kernel bounded at 64
// registers), 1 above.
__host__ __device__ constexpr int reg_class(int M) { return slots_of(M) > 16 ? 1 : 0; }

// Radix of stage s (0 after the last stage). The factor 3 is always last, so every span
// before it is a power of two.
__host__ __device__ constexpr int radix_of(int M, int v, int s) {
  return v == 0 ? (M == 16 ? (s < 2 ? 4 : 0)
                 : M == 32 ? (s == 0 ? 8 : s == 1 ? 4 : 0)
                 : M == 48 ? (s < 2 ? 4 : s == 2 ? 3 : 0)
                 : M == 64 ? (s < 2 ? 8 : 0)
                 : M == 96 ? (s == 0 ? 8 : s == 1 ? 4 : s == 2 ? 3 : 0)
                 : M == 128 ? (s == 0 ? 16 : s == 1 ? 8 : 0)
                 : M == 192 ? (s < 2 ? 8 : s == 2 ? 3 : 0)
                 : M == 256 ? (s < 2 ? 16 : 0)
                 : M == 384 ? (s < 2 ? 8 : s == 2 ? 2 : s == 3 ? 3 : 0)
                 : M == 512 ? (s < 2 ? 16 : s == 2 ? 2 : 0) : 0)
                : (M == 16 ? (s < 2 ? 4 : 0)
                 : M == 32 ? (s < 2 ? 4 : s == 2 ? 2 : 0)
                 : M == 48 ? (s < 2 ? 4 : s == 2 ? 3 : 0)
                 : M == 64 ? (s < 3 ? 4 : 0)
                 : M == 96 ? (s < 2 ? 4 : s == 2 ? 2 : s == 3 ? 3 : 0)
                 : M == 128 ? (s < 2 ? 8 : s == 2 ? 2 : 0)
                 : M == 192 ? (s < 3 ? 4 : s == 3 ? 3 : 0)
                 : M == 256 ? (s < 4 ? 4 : 0)
                 : M == 384 ? (s < 3 ? 4 : s == 3 ? 2 : s == 4 ? 3 : 0)
                 : M == 512 ? (s < 3 ? 8 : 0) : 0);
}
// Span Ns of stage s: the product of the radices before it.
__host__ __device__ constexpr int span_of(int M, int v, int s) {
  return s == 0 ? 1 : span_of(M, v, s - 1) * radix_of(M, v, s - 1);
}

// Every schedule: the radices multiply to M, each divides E, and T = M / E is a power of two.
__host__ __device__ constexpr bool schedule_ok(int M, int v) {
  int prod = 1;
  for (int s = 0; radix_of(M, v, s) > 0; ++s) {
    if (slots_of(M, v) % radix_of(M, v, s) != 0) return false;
    if (radix_of(M, v, s) == 3 && radix_of(M, v, s + 1) != 0) return false;
    prod *= radix_of(M, v, s);
  }
  const int T = M / slots_of(M, v);
  return prod == M && (T & (T - 1)) == 0 && T <= kThreads;
}
static_assert(schedule_ok(16, 0) && schedule_ok(32, 0) && schedule_ok(48, 0) && schedule_ok(64, 0) &&
              schedule_ok(96, 0) && schedule_ok(128, 0) && schedule_ok(192, 0) && schedule_ok(256, 0) &&
              schedule_ok(384, 0) && schedule_ok(512, 0), "lean schedules, variant 0");
static_assert(schedule_ok(16, 1) && schedule_ok(32, 1) && schedule_ok(48, 1) && schedule_ok(64, 1) &&
              schedule_ok(96, 1) && schedule_ok(128, 1) && schedule_ok(192, 1) && schedule_ok(256, 1) &&
              schedule_ok(384, 1) && schedule_ok(512, 1), "lean schedules, variant 1");

template <int M_, int V_ = 0>
struct Geo {
  static constexpr int M = M_;
  static constexpr int E = slots_of(M, V_);
  static constexpr int T = M / E;
  static constexpr int L = kThreads / T;
  static constexpr int NT = L * T;   // threads of the CTA
  static constexpr int LP = L + 1;
  static constexpr int N = 2 * M;   // real line length
};

// e^{-2 pi i/3}: cos = -1/2, sin = -sqrt(3)/2
__device__ __forceinline__ void dft3(float2 &a0, float2 &a1, float2 &a2) {
  const float c = 0.86602540378443864676f;
  const float2 s = make_float2(a1.x + a2.x, a1.y + a2.y);
  const float2 d = make_float2(a1.x - a2.x, a1.y - a2.y);
  const float2 t = make_float2(a0.x - 0.5f * s.x, a0.y - 0.5f * s.y);
  a0 = make_float2(a0.x + s.x, a0.y + s.y);
  // y1 = t - i c d, y2 = t + i c d
  a1 = make_float2(t.x + c * d.y, t.y - c * d.x);
  a2 = make_float2(t.x - c * d.y, t.y + c * d.x);
}

template <int R>
__device__ __forceinline__ void dft_r(float2 *v) {
  if constexpr (R == 3) dft3(v[0], v[1], v[2]);
  else small_dft<float2, R, false>(v, nullptr, 0);
}

// Stage s of the forward FFT on every line of the tile: thread (line l, lane u) runs the
// butterflies j = u + T b, b < E / R. Butterfly j reads slots j + r M/R, multiplies them by
// w_{Ns R}^{r (j mod Ns)}, runs a radix-R DFT and writes slot (j / Ns) Ns R + (j mod Ns) + r Ns.
// pre (stage 0 only, nullable): a factor per input slot (the DCT-IV pre-twiddle).
template <int M, int V, int S>
__device__ __forceinline__ void stage(float2 *buf, int u, int l, const float2 *__restrict__ tw,
                                      const float2 *__restrict__ pre) {
  using G = Geo<M, V>;
  constexpr int R = radix_of(M, V, S), NS = span_of(M, V, S);
  constexpr int E = G::E, T = G::T, LP = G::LP, NB = E / R, MR = M / R;
  float2 v[E];
  const float2 *rd = buf + u * LP + l;
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      v[b * R + r] = rd[(T * b + r * MR) * LP];
      if (pre) v[b * R + r] = cmul(v[b * R + r], __ldg(pre + u + T * b + r * MR));
    }
  // k = j mod NS and q = j / NS of butterfly j = u + T b (NS and T are powers of two, u < T)
  int kb, qb;
  if constexpr (NS <= T) { kb = u & (NS - 1); qb = u / NS; }
  else { kb = u; qb = 0; }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if constexpr (NS > 1) {
      constexpr int stw = M / (NS * R);
      const int k = (NS <= T) ? kb : kb + T * (b % (NS > T ? NS / T : 1));
      const int kk = k * stw;   // twiddle of input r: w_M^{r k stw}
#pragma unroll
      for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], __ldg(tw + r * kk));
    }
    dft_r<R>(v + b * R);
  }
  __syncthreads();
  float2 *wr = buf + l;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    int k, q;
    if constexpr (NS <= T) { k = kb; q = qb + (T / NS) * b; }
    else { k = kb + T * (b % (NS / T)); q = b / (NS / T); }
#pragma unroll
    for (int r = 0; r < R; ++r) wr[(q * NS * R + k + r * NS) * LP] = v[b * R + r];
  }
  __syncthreads();
}

// The forward FFT of every line of the tile (stages S, S + 1, ...); natural order in the slots.
template <int M, int V, int S>
__device__ __forceinline__ void fft(float2 *buf, int u, int l, const float2 *__restrict__ tw,
                                    const float2 *__restrict__ pre) {
  if constexpr (radix_of(M, V, S) > 0) {
    stage<M, V, S>(buf, u, l, tw, S == 0 ? pre : nullptr);
    fft<M, V, S + 1>(buf, u, l, tw, nullptr);
  }
}
// Out of line, so that a pass's forward and inverse halves share one copy of the stages (the
// unrolled stages are large, and instruction fetch is the first stall of these passes).
template <int M, int V>
__device__ __noinline__ void fft_all(float2 *buf, int u, int l, const float2 *__restrict__ tw,
                                     const float2 *__restrict__ pre) {
  fft<M, V, 0>(buf, u, l, tw, pre);
}

// Natural coefficient index -> position in the pass's coefficient layout (DST-II reversed).
template <int FAM>
__device__ __forceinline__ int coef_pos(int kind, int n, int i) {
  return (FAM == 1 && kind == KIND_DD) ? n - 1 - i : i;
}

// The four coefficient positions of pair k (k in [0, M/2)) in the order fwd_pair and inv_pair
// use: family 0 the packed real DFT [X0, X_{n/2}, Re X1, Im X1, ...] (k = 0: X0, X_{n/2} and
// the self-paired V_{M/2}); family 1 X_k, X_{n-k}, X_{M-k}, X_{M+k} (k = 0: X_0, X_M, X_{M/2},
// X_{n-M/2}), DST-II reversed; family 2 X_2q, X_{n-1-2q} for q = k and q = M - 1 - k.
template <int M, int FAM>
__device__ __forceinline__ void pair_positions(int k, int kind, int (&pos)[4]) {
  constexpr int n = 2 * M;
  if constexpr (FAM == 2) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = h == 0 ? k : M - 1 - k;
      pos[2 * h] = 2 * q;
      pos[2 * h + 1] = n - 1 - 2 * q;
    }
  } else if constexpr (FAM == 0) {
    if (k == 0) { pos[0] = 0; pos[1] = 1; pos[2] = M; pos[3] = M + 1; }
    else { pos[0] = 2 * k; pos[1] = 2 * k + 1; pos[2] = 2 * (M - k); pos[3] = 2 * (M - k) + 1; }
  } else {
    const int i0 = (k == 0) ? 0 : k, i1 = (k == 0) ? M : n - k, i2 = (k == 0) ? M / 2 : M - k,
              i3 = (k == 0) ? n - M / 2 : M + k;
    pos[0] = coef_pos<FAM>(kind, n, i0);
    pos[1] = coef_pos<FAM>(kind, n, i1);
    pos[2] = coef_pos<FAM>(kind, n, i2);
    pos[3] = coef_pos<FAM>(kind, n, i3);
  }
}

// Forward post-processing of pair k (k in [0, M/2)) of line l: the four coefficients it
// yields, as (position, value). Family 0: real DFT in packed order [X0, X_{n/2}, Re X1, Im X1,
// ...]; family 1: DCT-II (DST-II reversed); family 2: DCT-IV / DST-IV of slots k and M - 1 - k.
template <int M, int V, int FAM>
__device__ __forceinline__ void fwd_pair(const float2 *buf, int l, int k, int kind, const float2 *__restrict__ tw,
                                         int (&pos)[4], float (&val)[4]) {
  constexpr int LP = Geo<M, V>::LP;
  pair_positions<M, FAM>(k, kind, pos);
  if constexpr (FAM == 2) {
    const float2 *tp = tw + tw_dct4post(M);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = h == 0 ? k : M - 1 - k;
      const float2 y = cmul(buf[q * LP + l], __ldg(tp + q));
      val[2 * h] = y.x;
      val[2 * h + 1] = (kind == KIND_ND) ? -y.y : y.y;
    }
    return;
  }
  const float2 *wq = tw + tw_quarter(M);
  float2 Vk, Vm;   // V_k and V_{M-k} of the real DFT of the (reordered) line
  if (k == 0) {
    const float2 z0 = buf[l], zh = buf[(M / 2) * LP + l];
    const float V0 = z0.x + z0.y, VM = z0.x - z0.y;
    Vm = make_float2(zh.x, -zh.y);   // V_{M/2} = conj Z_{M/2}
    if constexpr (FAM == 0) {
      val[0] = V0;
      val[1] = VM;
      val[2] = Vm.x;
      val[3] = Vm.y;
    } else {
      const float2 th = cmul(Vm, __ldg(wq + M / 2));
      val[0] = V0;
      val[1] = __ldg(wq + M).x * VM;
      val[2] = th.x;
      val[3] = -th.y;
    }
    return;
  }
  const float2 zk = buf[k * LP + l], zm = buf[(M - k) * LP + l];
  // V_k = E + w^k O, V_{M-k} = conj(E - w^k O); E = (Z_k + conj Z_{M-k})/2, O = -i (Z_k - conj Z_{M-k})/2
  const float2 Eh = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
  const float2 O = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
  const float2 Ow = cmul(O, __ldg(tw + tw_rdft(M) + k));
  Vk = make_float2(Eh.x + Ow.x, Eh.y + Ow.y);
  Vm = make_float2(Eh.x - Ow.x, Ow.y - Eh.y);
  if constexpr (FAM == 0) {
    val[0] = Vk.x;
    val[1] = Vk.y;
    val[2] = Vm.x;
    val[3] = Vm.y;
  } else {
    // t = e^{-i pi k/(2n)} V_k: X_k = Re t, X_{n-k} = -Im t
    const float2 tk = cmul(Vk, __ldg(wq + k)), tm = cmul(Vm, __ldg(wq + M - k));
    val[0] = tk.x;
    val[1] = -tk.y;
    val[2] = tm.x;
    val[3] = -tm.y;
  }
}

// Inverse pre-processing of pair k of line l from its four coefficients (the positions
// fwd_pair gives, in the same order): writes the conjugated slots the forward FFT then
// inverts (family 2: the slots themselves, DCT-IV being its own inverse up to 2/n).
template <int M, int V, int FAM>
__device__ __forceinline__ void inv_pair(float2 *buf, int l, int k, int kind, const float2 *__restrict__ tw,
                                         const float (&val)[4]) {
  constexpr int LP = Geo<M, V>::LP;
  if constexpr (FAM == 2) {
    const float2 *t4 = tw + tw_dct4pre(M);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = h == 0 ? k : M - 1 - k;
      const float x0 = val[2 * h], x1 = val[2 * h + 1];   // X_2q, X_{n-1-2q}
      const float2 z = (kind == KIND_ND) ? make_float2(x0, x1) : make_float2(x1, x0);
      buf[q * LP + l] = cmul(z, __ldg(t4 + q));
    }
    return;
  }
  const float2 *wq = tw + tw_quarter(M);
  if (k == 0) {
    float a, b;
    float2 xh;   // the self-paired coefficient V_{M/2}
    if constexpr (FAM == 0) {
      a = val[0];
      b = val[1];
      xh = make_float2(val[2], val[3]);
    } else {
      const float2 wM = __ldg(wq + M);
      a = val[0];
      b = val[1] * wM.x - val[1] * wM.y;                      // Re V_M, V_M = (X_M - i X_M) conj(wq_M)
      xh = cmulc(make_float2(val[2], -val[3]), __ldg(wq + M / 2));
    }
    buf[l] = make_float2(0.5f * (a + b), -0.5f * (a - b));  // conj Z_0
    buf[(M / 2) * LP + l] = xh;                               // conj Z_{M/2} = V_{M/2}
    return;
  }
  float2 xk, xm;   // V_k, V_{M-k}
  if constexpr (FAM == 0) {
    xk = make_float2(val[0], val[1]);
    xm = make_float2(val[2], val[3]);
  } else {
    // V_i = (X_i - i X_{n-i}) e^{+i pi i/(2n)}
    xk = cmulc(make_float2(val[0], -val[1]), __ldg(wq + k));
    xm = cmulc(make_float2(val[2], -val[3]), __ldg(wq + M - k));
  }
  // Z_k = E + i O, Z_{M-k} = conj(E - i O); E = (V_k + conj V_{M-k})/2, O = (V_k - conj V_{M-k}) conj(w^k)/2
  const float2 Eh = make_float2(0.5f * (xk.x + xm.x), 0.5f * (xk.y - xm.y));
  const float2 D = make_float2(0.5f * (xk.x - xm.x), 0.5f * (xk.y + xm.y));
  const float2 O = cmulc(D, __ldg(tw + tw_rdft(M) + k));
  buf[k * LP + l] = make_float2(Eh.x - O.y, -(Eh.y + O.x));        // conj(E + i O)
  buf[(M - k) * LP + l] = make_float2(Eh.x + O.y, Eh.y - O.x);     // E - i O
}

// ----------------------------------------------------------------------------- global I/O
// A thread moves its line's values in quads of four consecutive positions 4 qd .. 4 qd + 3
// (one 16-byte access on row tiles, four coalesced scalar accesses on column tiles) and its
// coefficients in the pairs of pair_positions. Where a line lives: `gb` its first cell and
// `gs` the element stride along it (1 on row tiles).
struct LineRef {
  int gb, gs;
  bool valid;
};

// Load the quad at position 4 qd of a line from A.src (FP64 sources truncated to FP32).
template <bool COL>
__device__ __forceinline__ float4 load_quad(const PassArgs<float> &A, const LineRef &lr, int qd) {
  if (!lr.valid) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const int g = lr.gb + 4 * qd * lr.gs;
  if (A.src_mode == SRC_F64) {
    const double *s = static_cast<const double *>(A.src);
    if constexpr (COL) {
      return make_float4(d2f_rz_bits(__ldg(s + g)), d2f_rz_bits(__ldg(s + g + lr.gs)),
                         d2f_rz_bits(__ldg(s + g + 2 * lr.gs)), d2f_rz_bits(__ldg(s + g + 3 * lr.gs)));
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2 *>(s + g));
      const double2 b = __ldg(reinterpret_cast<const double2 *>(s + g + 2));
      return make_float4(d2f_rz_bits(a.x), d2f_rz_bits(a.y), d2f_rz_bits(b.x), d2f_rz_bits(b.y));
    }
  }
  const float *s = static_cast<const float *>(A.src);
  if constexpr (COL) return make_float4(s[g], s[g + lr.gs], s[g + 2 * lr.gs], s[g + 3 * lr.gs]);
  else return *reinterpret_cast<const float4 *>(s + g);
}

// Forward scatter of the quad at position 4 qd into the slots of line l: input x_j at real
// position j of the slots (real DFT); at Makhoul's position j/2 (j even) or n - 1 - j/2 (j odd),
// times (-1)^j for DST-II, so that positions 4qd and 4qd + 2 share slot qd and positions
// 4qd + 1 and 4qd + 3 slot M - 1 - qd; or DCT-IV's z_q = (x_2q, x_{n-1-2q}), swapped for DST-IV.
template <int M, int V, int FAM>
__device__ __forceinline__ void scatter_quad(float2 *buf, int l, int qd, int kind, float4 x) {
  constexpr int LP = Geo<M, V>::LP;
  float *re = reinterpret_cast<float *>(buf);
  if constexpr (FAM == 0) {
    buf[(2 * qd) * LP + l] = make_float2(x.x, x.y);
    buf[(2 * qd + 1) * LP + l] = make_float2(x.z, x.w);
  } else if constexpr (FAM == 1) {
    const float sg = (kind == KIND_DD) ? -1.0f : 1.0f;   // DST-II: (-1)^j x_j
    buf[qd * LP + l] = make_float2(x.x, x.z);
    buf[(M - 1 - qd) * LP + l] = make_float2(sg * x.w, sg * x.y);
  } else {
    // z_q = (x_2q, x_{n-1-2q}) (DCT-IV), swapped (DST-IV)
    const int c = (kind == KIND_ND) ? 0 : 1;
    re[2 * ((2 * qd) * LP + l) + c] = x.x;
    re[2 * ((2 * qd + 1) * LP + l) + c] = x.z;
    re[2 * ((M - 1 - 2 * qd) * LP + l) + (c ^ 1)] = x.y;
    re[2 * ((M - 2 - 2 * qd) * LP + l) + (c ^ 1)] = x.w;
  }
}

// Outputs 4 qd .. 4 qd + 3 of a line after the final FFT (before the 1/M normalisation): the
// conjugated slots of the inverse real DFT / DCT-III / DST-III, or DCT-IV / DST-IV post-twiddled.
template <int M, int V, int FAM>
__device__ __forceinline__ float4 gather_quad(const float2 *buf, int l, int qd, int kind, const float2 *__restrict__ tw) {
  constexpr int LP = Geo<M, V>::LP;
  if constexpr (FAM == 0) {
    const float2 a = buf[(2 * qd) * LP + l], b = buf[(2 * qd + 1) * LP + l];
    return make_float4(a.x, -a.y, b.x, -b.y);
  } else if constexpr (FAM == 1) {
    const float2 zq = buf[qd * LP + l], zm = buf[(M - 1 - qd) * LP + l];
    if (kind == KIND_DD) return make_float4(zq.x, zm.y, -zq.y, -zm.x);
    return make_float4(zq.x, -zm.y, -zq.y, zm.x);
  } else {
    const float2 *tp = tw + tw_dct4post(M);
    const int qa = 2 * qd, qb = M - 1 - 2 * qd, qc = 2 * qd + 1, qe = M - 2 - 2 * qd;
    const float2 ya = cmul(buf[qa * LP + l], __ldg(tp + qa)), yb = cmul(buf[qb * LP + l], __ldg(tp + qb));
    const float2 yc = cmul(buf[qc * LP + l], __ldg(tp + qc)), ye = cmul(buf[qe * LP + l], __ldg(tp + qe));
    const float sg = (kind == KIND_ND) ? -1.0f : 1.0f;
    return make_float4(ya.x, sg * yb.y, yc.x, sg * ye.y);
  }
}

// Store the quad at position 4 qd of a line into A.dst by A.dst_mode (op: the old pairs of an
// accumulating store, load_old_pairs).
template <bool COL>
__device__ __forceinline__ void store_quad(const PassArgs<float> &A, const LineRef &lr, int qd, float4 x,
                                           const float4 (&op)[2]) {
  if (!lr.valid) return;
  const int g = lr.gb + 4 * qd * lr.gs;
  const int mode = A.dst_mode;
  if (mode == DST_WORK) {
    float *d = static_cast<float *>(A.dst);
    if constexpr (COL) {
      d[g] = x.x; d[g + lr.gs] = x.y; d[g + 2 * lr.gs] = x.z; d[g + 3 * lr.gs] = x.w;
    } else {
      *reinterpret_cast<float4 *>(d + g) = x;
    }
    return;
  }
  const float xv[4] = {x.x, x.y, x.z, x.w};
  if (mode == DST_PAIR_SET || mode == DST_PAIR_ADD) {
    // the FP32 pair (hi, lo) of the refinement iterate += x with Knuth's TwoSum, renormalised
    float2 *d = static_cast<float2 *>(A.dst);
    const float2 old[4] = {make_float2(op[0].x, op[0].y), make_float2(op[0].z, op[0].w),
                           make_float2(op[1].x, op[1].y), make_float2(op[1].z, op[1].w)};
    float2 r[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float hi = xv[c], lo = 0.0f;
      if (mode == DST_PAIR_ADD) {
        const float a = old[c].x, alo = old[c].y, bb = hi;
        const float s1 = __fadd_rn(a, bb), z = __fsub_rn(s1, a);
        const float e = __fadd_rn(__fadd_rn(__fsub_rn(a, __fsub_rn(s1, z)), __fsub_rn(bb, z)), alo);
        hi = __fadd_rn(s1, e);
        lo = __fsub_rn(e, __fsub_rn(hi, s1));
      }
      r[c] = make_float2(hi, lo);
    }
    if constexpr (COL) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        d[g + c * lr.gs] = r[c];
        if (A.f64) A.f64[g + c * lr.gs] = f2d_bits(r[c].x) + f2d_bits(r[c].y);
      }
    } else {
      *reinterpret_cast<float4 *>(d + g) = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
      *reinterpret_cast<float4 *>(d + g + 2) = make_float4(r[2].x, r[2].y, r[3].x, r[3].y);
      if (A.f64) {
        double2 *f = reinterpret_cast<double2 *>(A.f64 + g);
        f[0] = make_double2(f2d_bits(r[0].x) + f2d_bits(r[0].y), f2d_bits(r[1].x) + f2d_bits(r[1].y));
        f[1] = make_double2(f2d_bits(r[2].x) + f2d_bits(r[2].y), f2d_bits(r[3].x) + f2d_bits(r[3].y));
      }
    }
    return;
  }
  // FP64 destination (set or accumulate): not on the projection's path
  double *d = static_cast<double *>(A.dst);
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    const int gi = g + c * lr.gs;
    d[gi] = (mode == DST_F64_SET) ? f2d_bits(xv[c]) : d[gi] + f2d_bits(xv[c]);
  }
}

// Coefficients of pair k at positions pos (pair_positions) of a line: stored to A.dst
// (forward-only passes, DST_WORK) or loaded from A.src (inverse-only passes, FP32). Row tiles
// move the position pairs that are adjacent (families 0 and 2) as 8-byte accesses.
template <int FAM, bool COL>
__device__ __forceinline__ void store_pair(const PassArgs<float> &A, const LineRef &lr, const int (&pos)[4],
                                           const float (&val)[4]) {
  if (!lr.valid) return;
  float *d = static_cast<float *>(A.dst);
  if constexpr (!COL && FAM == 0) {   // (pos0, pos0 + 1), (pos2, pos2 + 1)
    *reinterpret_cast<float2 *>(d + lr.gb + pos[0]) = make_float2(val[0], val[1]);
    *reinterpret_cast<float2 *>(d + lr.gb + pos[2]) = make_float2(val[2], val[3]);
  } else if constexpr (!COL && FAM == 2) {   // (2k, 2k + 1) = pos 0, 3; (n-2-2k, n-1-2k) = pos 2, 1
    *reinterpret_cast<float2 *>(d + lr.gb + pos[0]) = make_float2(val[0], val[3]);
    *reinterpret_cast<float2 *>(d + lr.gb + pos[2]) = make_float2(val[2], val[1]);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) d[lr.gb + pos[c] * lr.gs] = val[c];
  }
}
template <int FAM, bool COL>
__device__ __forceinline__ void load_pair(const PassArgs<float> &A, const LineRef &lr, const int (&pos)[4],
                                          float (&val)[4]) {
  if (!lr.valid) {
    val[0] = val[1] = val[2] = val[3] = 0.0f;
    return;
  }
  const float *s = static_cast<const float *>(A.src);
  if constexpr (!COL && FAM == 0) {
    const float2 a = *reinterpret_cast<const float2 *>(s + lr.gb + pos[0]);
    const float2 b = *reinterpret_cast<const float2 *>(s + lr.gb + pos[2]);
    val[0] = a.x; val[1] = a.y; val[2] = b.x; val[3] = b.y;
  } else if constexpr (!COL && FAM == 2) {
    const float2 a = *reinterpret_cast<const float2 *>(s + lr.gb + pos[0]);
    const float2 b = *reinterpret_cast<const float2 *>(s + lr.gb + pos[2]);
    val[0] = a.x; val[3] = a.y; val[2] = b.x; val[1] = b.y;
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) val[c] = s[lr.gb + pos[c] * lr.gs];
  }
}

// Old pairs of an accumulating store (DST_PAIR_ADD) at the quad at position 4 qd.
template <bool COL>
__device__ __forceinline__ void load_old_pairs(const PassArgs<float> &A, const LineRef &lr, int qd, float4 (&o)[2]) {
  o[0] = o[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (!lr.valid || A.dst_mode != DST_PAIR_ADD) return;
  const float2 *d = static_cast<const float2 *>(A.dst);
  const int g = lr.gb + 4 * qd * lr.gs;
  if constexpr (COL) {
    const float2 a = d[g], b = d[g + lr.gs], c = d[g + 2 * lr.gs], e = d[g + 3 * lr.gs];
    o[0] = make_float4(a.x, a.y, b.x, b.y);
    o[1] = make_float4(c.x, c.y, e.x, e.y);
  } else {
    o[0] = *reinterpret_cast<const float4 *>(d + g);
    o[1] = *reinterpret_cast<const float4 *>(d + g + 2);
  }
}

// One pass over tile `tile`: [forward transform] [division] [inverse transform] as A asks
// (a division always sits between a forward and an inverse transform). The FFT maps threads
// line-fast; the quads and pairs map them line-fast on column tiles (coalesced across lines)
// and position-fast on row tiles (coalesced along the line). Out of line: one function per
// length, variant, family and layout keeps the compile time linear in their number.
template <int M, int V, int FAM, bool COL>
__device__ __noinline__ void body_layout(const PassArgs<float> &A, int tile, float2 *buf, const float *lamo,
                                         const int *lbase, const int *lzero) {
  using G = Geo<M, V>;
  constexpr int E = G::E, T = G::T, L = G::L, n = G::N, NQ = E / 2;
  const int t = threadIdx.x;
  const int l = t % L, u = t / L;                     // FFT map
  const int pl = COL ? l : t / T, pu = COL ? u : t % T;   // quad and pair map
  const int kind = pass_kind<FAM>(A.kind);
  const float2 *tw = A.tw;
  LineRef lr;
  if constexpr (COL) {
    lr.gb = lbase[pl];
    lr.valid = lr.gb >= 0;
    lr.gs = A.stride;
  } else {
    const int line = tile * L + pl;
    lr.valid = line < A.lines;
    lr.gb = line * n;
    lr.gs = 1;
  }

  if (A.do_fwd) {
    float4 xq[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) xq[i] = load_quad<COL>(A, lr, pu + T * i);
#pragma unroll
    for (int i = 0; i < NQ; ++i) scatter_quad<M, V, FAM>(buf, pl, pu + T * i, kind, xq[i]);
    __syncthreads();
    fft_all<M, V>(buf, u, l, tw, FAM == 2 ? tw + tw_dct4pre(M) : nullptr);
    if (!A.do_inv) {
      // forward-only pass: the coefficients of each pair straight to global memory
#pragma unroll
      for (int i = 0; i < NQ; ++i) {
        int pos[4];
        float val[4];
        fwd_pair<M, V, FAM>(buf, pl, pu + T * i, kind, tw, pos, val);
        store_pair<FAM, COL>(A, lr, pos, val);
      }
      return;
    }
    // forward post-processing, division, inverse pre-processing: per pair, in registers (a
    // pair's slots are read and rewritten by the same thread)
    const bool dv = A.do_div;
    const float lo = dv ? lamo[pl] : 0.0f;
    const bool zm = dv && A.singular && lzero[pl];
    const float *la = A.lam[A.axis];
#pragma unroll 1
    for (int i = 0; i < NQ; ++i) {
      const int k = pu + T * i;
      int pos[4];
      float val[4];
      fwd_pair<M, V, FAM>(buf, pl, k, kind, tw, pos, val);
      if (dv) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          val[c] = (zm && pos[c] == 0) ? 0.0f : __fdividef(val[c], __ldg(la + pos[c]) + lo);
      }
      inv_pair<M, V, FAM>(buf, pl, k, kind, tw, val);
    }
    __syncthreads();
  } else {
    // inverse-only pass: each pair's coefficients from global memory, pre-processed into its
    // slots; two pairs per iteration (their loads issued together)
#pragma unroll 1
    for (int i = 0; i < NQ; i += 2) {
      float val[2][4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int pos[4];
        pair_positions<M, FAM>(pu + T * (i + h), kind, pos);
        load_pair<FAM, COL>(A, lr, pos, val[h]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) inv_pair<M, V, FAM>(buf, pl, pu + T * (i + h), kind, tw, val[h]);
    }
    __syncthreads();
  }
  fft_all<M, V>(buf, u, l, tw, nullptr);
  const float scale = A.out_scale;
  // outputs, two quads at a time (the old values of an accumulating store loaded first)
#pragma unroll 1
  for (int i = 0; i < NQ; i += 2) {
    float4 o[2][2];
    load_old_pairs<COL>(A, lr, pu + T * i, o[0]);
    load_old_pairs<COL>(A, lr, pu + T * (i + 1), o[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int qd = pu + T * (i + h);
      float4 x = gather_quad<M, V, FAM>(buf, pl, qd, kind, tw);
      x = make_float4(x.x * scale, x.y * scale, x.z * scale, x.w * scale);
      store_quad<COL>(A, lr, qd, x, o[h]);
    }
  }
}

// One tile of a lean pass: per-line set-up (base cell, eigenvalue sum of the other axes, zero
// mode flag), then the pass in the tile's layout.
template <int M, int V, int FAM>
__device__ __forceinline__ void body(const PassArgs<float> &A, int tile, unsigned char *smem_raw) {
  using G = Geo<M, V>;
  constexpr int L = G::L;
  float2 *buf = reinterpret_cast<float2 *>(smem_raw);
  float *lamo = reinterpret_cast<float *>(buf + M * G::LP);
  int *lbase = reinterpret_cast<int *>(lamo + L);
  int *lzero = lbase + L;
  const int t = threadIdx.x;
  const int n = G::N;
  if (t < L) {
    int base, valid;
    if (A.col) {
      const int o = tile / A.tiles_per_outer;
      const int f = (tile - o * A.tiles_per_outer) * L + t;
      valid = f < A.inner;
      base = o * n * A.stride + f;
    } else {
      const int line = tile * L + t;
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
      float lo = 0.0f;
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
  if (A.col) body_layout<M, V, FAM, true>(A, tile, buf, lamo, lbase, lzero);
  else body_layout<M, V, FAM, false>(A, tile, buf, lamo, lbase, lzero);
}

// The variant of the pass, told by its tile's line count (the same for both variants of the
// lengths that have one only).
template <int M, int FAM>
__device__ __forceinline__ void body_v(const PassArgs<float> &A, int tile, unsigned char *smem) {
  if constexpr (slots_of(M, 0) == slots_of(M, 1)) {
    body<M, 0, FAM>(A, tile, smem);
  } else {
    if (A.L == Geo<M, 0>::L) body<M, 0, FAM>(A, tile, smem);
    else body<M, 1, FAM>(A, tile, smem);
  }
}

// The lean pass kernel of register class RC (lengths with E <= 16 slots per thread, or above)
// and transform family FAM. items == nullptr: a single-problem pass A1, CTA b transforming tiles
// b * chunk, ...; else a batched pass, CTA b transforming tiles items[b].y .. items[b].y +
// items[b].z - 1 of args[items[b].x]. Both copy their arguments to shared memory and run the
// same body, so a batched problem's results are bitwise those of its single call.
template <int RC, int FAM>
__global__ void __launch_bounds__(kThreads, RC == 0 ? 4 : 2)
    lean_kernel(PassArgs<float> A1, const PassArgs<float> *__restrict__ args, const int4 *__restrict__ items) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) PassArgs<float> A;
  int t0, t1;
  {
    const unsigned *src;
    if (items) {
      const int4 it = items[blockIdx.x];
      src = reinterpret_cast<const unsigned *>(args + it.x);
      t0 = it.y;
      t1 = it.y + it.z;
    } else {
      src = reinterpret_cast<const unsigned *>(&A1);
      t0 = blockIdx.x * A1.chunk;
      t1 = min(t0 + A1.chunk, A1.ntiles);
    }
    unsigned *dst = reinterpret_cast<unsigned *>(&A);
    for (int w = threadIdx.x; w < (int)(sizeof(PassArgs<float>) / 4); w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  if (A.gate.st && refine_stopped_before(A.gate.st, A.gate.j, A.gate.tol)) return;   // refinement already ended
  for (int t = t0; t < t1; ++t) {
    if (t > t0) __syncthreads();   // the previous tile no longer reads the buffer
    if constexpr (RC == 0) {
      switch (A.M) {
        case 16: body_v<16, FAM>(A, t, smem_raw); break;
        case 32: body_v<32, FAM>(A, t, smem_raw); break;
        case 48: body_v<48, FAM>(A, t, smem_raw); break;
        case 64: body_v<64, FAM>(A, t, smem_raw); break;
        case 128: body_v<128, FAM>(A, t, smem_raw); break;
        default: body_v<256, FAM>(A, t, smem_raw); break;
      }
    } else {
      switch (A.M) {
        case 96: body_v<96, FAM>(A, t, smem_raw); break;
        case 192: body_v<192, FAM>(A, t, smem_raw); break;
        case 384: body_v<384, FAM>(A, t, smem_raw); break;
        default: body_v<512, FAM>(A, t, smem_raw); break;
      }
    }
  }
}

// Kernel id of a lean pass: 1 + 3 * register class + family (0: a general pass).
__host__ __device__ constexpr int lean_id(int M, int fam) { return 1 + 3 * reg_class(M) + fam; }

template <int RC, int FAM>
pc_status launch_kernel(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems, unsigned grid,
                        int threads, size_t smem, cudaStream_t st) {
  if (grid == 0) return PC_OK;
  launch_pdl(lean_kernel<RC, FAM>, grid, threads, smem, st, A, dargs, ditems);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

}  // namespace lean
}  // namespace pc
