// Compile-time FP32 transform passes (§2.3 three-step solve) for the cell-grid transform families
// (real DFT, DCT-II/DST-II, DCT-IV/DST-IV) at the line lengths n = 2M the workloads use
// (M in {16, 32, 48, 64, 96, 128, 192, 256, 384, 512}).
//
// The general passes (axis_pass.cuh) take the line length, the radix schedule and the tile
// shape at run time; their index arithmetic, predication and twiddle addressing cost about 130
// thread instructions per cell and pass. Here every one of these is a compile-time constant:
//   - a tile is L lines x M complex slots in shared memory, slot-major with the line index fast
//     (slot q of line l at q * LP + l, LP = L + 1), so the FFT's accesses (every thread of a
//     half-warp on another line, the same slot) are conflict-free whatever the slot pattern,
//     and position-fast accesses of one line (row loads and stores) are too (LP odd);
//   - each line is served by T = M / E threads holding E complex values in registers; the FFT
//     is a Stockham autosort whose stages (radix 16, 8, 4, 2 and a final 3) each read E slots,
//     twiddle, run the small DFTs in registers and write E slots (two barriers, one buffer);
//   - the inverse transform runs the same forward FFT on conjugated slots (conj(FFT(conj Z))
//     is the inverse DFT), so a length has one FFT body;
//   - in a pass that divides (forward, division, inverse), each thread post-processes a pair of
//     slots (k, M - k) into four coefficients, divides them and pre-processes the same pair for
//     the inverse in registers, with no barrier in between.
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
template <int M, int V, int S = 0>
__device__ __forceinline__ void fft(float2 *buf, int u, int l, const float2 *__restrict__ tw,
                                    const float2 *__restrict__ pre) {
  if constexpr (radix_of(M, V, S) > 0) {
    stage<M, V, S>(buf, u, l, tw, S == 0 ? pre : nullptr);
    fft<M, V, S + 1>(buf, u, l, tw, nullptr);
  }
}

// Real position p of line l in the buffer (slot p / 2, real part for even p).
template <int M, int V>
__device__ __forceinline__ float &re_at(float2 *buf, int l, int p) {
  return reinterpret_cast<float *>(buf)[2 * ((p >> 1) * Geo<M, V>::LP + l) + (p & 1)];
}

// Where input x_j of a forward transform goes among the real positions of the slots (the
// complex slot q holds positions 2q, 2q + 1), and its sign.
template <int FAM>
__device__ __forceinline__ int fwd_pos(int kind, int n, int j, bool &neg) {
  neg = false;
  if constexpr (FAM == 0) return j;
  if constexpr (FAM == 1) {
    neg = (kind == KIND_DD) && (j & 1);                 // DST-II: (-1)^j x_j
    return (j & 1) ? n - 1 - (j >> 1) : (j >> 1);       // Makhoul's reordering
  }
  // DCT-IV: z_q = (x_2q, x_{n-1-2q}); DST-IV swaps the two
  if (kind == KIND_ND) return (j & 1) ? n - j : j;
  return (j & 1) ? n - 1 - j : j + 1;
}

// Natural coefficient index -> position in the pass's coefficient layout (DST-II reversed).
template <int FAM>
__device__ __forceinline__ int coef_pos(int kind, int n, int i) {
  return (FAM == 1 && kind == KIND_DD) ? n - 1 - i : i;
}

// The four coefficient positions of pair k (k in [0, M/2)) in the order fwd_pair and inv_pair
// use: family 0 the packed real DFT [X0, X_{n/2}, Re X1, Im X1, ...] (k = 0: X0, X_{n/2} and
// the self-paired V_{M/2}); family 1 X_k, X_{n-k}, X_{M-k}, X_{M+k} (k = 0: X_0, X_M, X_{M/2},
// X_{n-M/2}), DST-II reversed; family 2 X_2q, X_{n-1-2q} for q = k and q = k + M/2.
template <int M, int FAM>
__device__ __forceinline__ void pair_positions(int k, int kind, int (&pos)[4]) {
  constexpr int n = 2 * M;
  if constexpr (FAM == 2) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = k + h * (M / 2);
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
// ...]; family 1: DCT-II (DST-II reversed); family 2: DCT-IV / DST-IV of slots k and k + M/2.
template <int M, int V, int FAM>
__device__ __forceinline__ void fwd_pair(const float2 *buf, int l, int k, int kind, const float2 *__restrict__ tw,
                                         int (&pos)[4], float (&val)[4]) {
  constexpr int LP = Geo<M, V>::LP;
  pair_positions<M, FAM>(k, kind, pos);
  if constexpr (FAM == 2) {
    const float2 *tp = tw + tw_dct4post(M);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = k + h * (M / 2);
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
      const int q = k + h * (M / 2);
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

// Output i of a line after the final FFT (before the 1/M normalisation).
template <int M, int V, int FAM>
__device__ __forceinline__ float inv_value(const float2 *buf, int l, int i, int kind, const float2 *__restrict__ tw) {
  constexpr int LP = Geo<M, V>::LP, n = 2 * M;
  if constexpr (FAM == 0) {
    const float2 z = buf[(i >> 1) * LP + l];
    return (i & 1) ? -z.y : z.x;
  } else if constexpr (FAM == 1) {
    const int j = (i & 1) ? n - 1 - (i >> 1) : (i >> 1);
    const float2 z = buf[(j >> 1) * LP + l];
    const float v = (j & 1) ? -z.y : z.x;
    return (kind == KIND_DD && (i & 1)) ? -v : v;
  } else {
    const int q = (i & 1) ? ((n - 1 - i) >> 1) : (i >> 1);
    const float2 y = cmul(buf[q * LP + l], __ldg(tw + tw_dct4post(M) + q));
    if ((i & 1) == 0) return y.x;
    return (kind == KIND_ND) ? -y.y : y.y;
  }
}

// Global element i (i < 2E) of this thread in a load or store phase of tile `tile`: its line,
// position along the line, global index and validity. Row tiles are one contiguous run of
// L lines (consecutive threads on consecutive cells); column tiles put the line index fast
// (consecutive threads on adjacent lines, one global row segment per position).
template <int M, int V, bool COL>
struct ElemMap {
  using G = Geo<M, V>;
  int t, l, u, rowbase, rowend, stride;
  const int *lbase;
  __device__ __forceinline__ void at(int i, int &line, int &pos, int &gi, bool &valid) const {
    if constexpr (COL) {
      line = l;
      pos = u + G::T * i;
      const int b = lbase[l];
      valid = b >= 0;
      gi = b + pos * stride;
    } else {
      const int e = t + G::NT * i;
      line = e / G::N;
      pos = e - line * G::N;
      gi = rowbase + e;
      valid = gi < rowend;
    }
  }
};

// Load phase: elements c0 .. c0 + CH - 1 of this thread, from A.src by A.src_mode, handed to
// put(line, pos, value) once all of the chunk's loads are issued. CH divides the 2E elements.
template <int M, int V>
__host__ __device__ constexpr int load_chunk_of() { return (2 * slots_of(M, V)) % 16 == 0 ? 16 : 8; }
template <int M, int V, bool COL, typename Put>
__device__ __forceinline__ void load_chunk(const PassArgs<float> &A, const ElemMap<M, V, COL> &em, int c0, Put put) {
  constexpr int kChunk = load_chunk_of<M, V>();
  float x[kChunk];
  if (A.src_mode == SRC_F64) {
    const double *src = static_cast<const double *>(A.src);
#pragma unroll
    for (int b = 0; b < kChunk; ++b) {
      int line, pos, gi;
      bool valid;
      em.at(c0 + b, line, pos, gi, valid);
      x[b] = valid ? d2f_rz_bits(__ldg(src + gi)) : 0.0f;
    }
  } else {
    const float *src = static_cast<const float *>(A.src);
#pragma unroll
    for (int b = 0; b < kChunk; ++b) {
      int line, pos, gi;
      bool valid;
      em.at(c0 + b, line, pos, gi, valid);
      x[b] = valid ? src[gi] : 0.0f;
    }
  }
#pragma unroll
  for (int b = 0; b < kChunk; ++b) {
    int line, pos, gi;
    bool valid;
    em.at(c0 + b, line, pos, gi, valid);
    put(line, pos, x[b]);
  }
}

// Store phase: every element of the tile through get(line, pos) into A.dst by A.dst_mode, in
// chunks (the old values of an accumulating store are loaded together).
template <int M, int V, bool COL, typename Get>
__device__ __forceinline__ void store_phase(const PassArgs<float> &A, const ElemMap<M, V, COL> &em, Get get) {
  constexpr int NE = 2 * Geo<M, V>::E, kC = NE < 8 ? NE : 8;
  const int mode = A.dst_mode;
#pragma unroll 1
  for (int c0 = 0; c0 < NE; c0 += kC) {
    float x[kC];
#pragma unroll
    for (int b = 0; b < kC; ++b) {
      int line, pos, gi;
      bool valid;
      em.at(c0 + b, line, pos, gi, valid);
      x[b] = get(line, pos);
    }
    if (mode == DST_WORK) {
      float *dst = static_cast<float *>(A.dst);
#pragma unroll
      for (int b = 0; b < kC; ++b) {
        int line, pos, gi;
        bool valid;
        em.at(c0 + b, line, pos, gi, valid);
        if (valid) dst[gi] = x[b];
      }
    } else if (mode == DST_PAIR_SET || mode == DST_PAIR_ADD) {
      // the FP32 pair (hi, lo) of the refinement iterate += x with Knuth's TwoSum, renormalised
      float2 *dst = static_cast<float2 *>(A.dst);
      float2 old[kC];
#pragma unroll
      for (int b = 0; b < kC; ++b) {
        int line, pos, gi;
        bool valid;
        em.at(c0 + b, line, pos, gi, valid);
        old[b] = (mode == DST_PAIR_ADD && valid) ? dst[gi] : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int b = 0; b < kC; ++b) {
        int line, pos, gi;
        bool valid;
        em.at(c0 + b, line, pos, gi, valid);
        float hi = x[b], lo = 0.0f;
        if (mode == DST_PAIR_ADD) {
          const float a = old[b].x, alo = old[b].y, bb = hi;
          const float s1 = __fadd_rn(a, bb), z = __fsub_rn(s1, a);
          const float e = __fadd_rn(__fadd_rn(__fsub_rn(a, __fsub_rn(s1, z)), __fsub_rn(bb, z)), alo);
          hi = __fadd_rn(s1, e);
          lo = __fsub_rn(e, __fsub_rn(hi, s1));
        }
        if (valid) {
          dst[gi] = make_float2(hi, lo);
          if (A.f64) A.f64[gi] = f2d_bits(hi) + f2d_bits(lo);
        }
      }
    } else {
      // FP64 destination (set or accumulate): not on the projection's path
      double *dst = static_cast<double *>(A.dst);
#pragma unroll 1
      for (int b = 0; b < kC; ++b) {
        int line, pos, gi;
        bool valid;
        em.at(c0 + b, line, pos, gi, valid);
        if (valid) dst[gi] = (mode == DST_F64_SET) ? f2d_bits(x[b]) : dst[gi] + f2d_bits(x[b]);
      }
    }
  }
}

// One pass over tile `tile`: [forward transform] [division] [inverse transform] as A asks
// (a division always sits between a forward and an inverse transform). Out of line: one
// function per length, family and layout keeps the compile time linear in their number.
template <int M, int V, int FAM, bool COL>
__device__ __noinline__ void body_layout(const PassArgs<float> &A, int tile, float2 *buf, const float *lamo,
                                         const int *lbase, const int *lzero) {
  using G = Geo<M, V>;
  constexpr int E = G::E, T = G::T, L = G::L, n = G::N, NE = 2 * E;
  const int t = threadIdx.x;
  const int l = t % L, u = t / L;   // FFT and pair map: line fast
  const int kind = pass_kind<FAM>(A.kind);
  const float2 *tw = A.tw;
  ElemMap<M, V, COL> em;
  em.t = t; em.l = l; em.u = u; em.stride = A.stride; em.lbase = lbase;
  em.rowbase = tile * (L * n);
  em.rowend = A.lines * n;

  if (A.do_fwd) {
    // load (a chunk's loads issued together), scatter into the slots
#pragma unroll 1
    for (int c0 = 0; c0 < NE; c0 += load_chunk_of<M, V>())
      load_chunk<M, V, COL>(A, em, c0, [&](int line, int pos, float x) {
        bool neg;
        const int p = fwd_pos<FAM>(kind, n, pos, neg);
        re_at<M, V>(buf, line, p) = neg ? -x : x;
      });
    __syncthreads();
    fft<M, V>(buf, u, l, tw, FAM == 2 ? tw + tw_dct4pre(M) : nullptr);
    if (!A.do_inv) {
      // forward-only pass: coefficients -> their positions in the buffer -> global
      float val[E / 2][4];
#pragma unroll
      for (int i = 0; i < E / 2; ++i) {
        int pos[4];
        fwd_pair<M, V, FAM>(buf, l, u + T * i, kind, tw, pos, val[i]);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < E / 2; ++i) {
        int pos[4];
        pair_positions<M, FAM>(u + T * i, kind, pos);
#pragma unroll
        for (int c = 0; c < 4; ++c) re_at<M, V>(buf, l, pos[c]) = val[i][c];
      }
      __syncthreads();
      store_phase<M, V, COL>(A, em, [&](int line, int p) { return re_at<M, V>(buf, line, p); });
      return;
    }
    // forward post-processing, division, inverse pre-processing: per pair, in registers
    const float lo = A.do_div ? lamo[l] : 0.0f;
    const bool zm = A.do_div && A.singular && lzero[l];
    const float *la = A.lam[A.axis];
    const bool dv = A.do_div;
#pragma unroll 1
    for (int i = 0; i < E / 2; ++i) {
      const int k = u + T * i;
      int pos[4];
      float val[4];
      fwd_pair<M, V, FAM>(buf, l, k, kind, tw, pos, val);
      if (dv) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          val[c] = (zm && pos[c] == 0) ? 0.0f : __fdividef(val[c], __ldg(la + pos[c]) + lo);
      }
      inv_pair<M, V, FAM>(buf, l, k, kind, tw, val);
    }
    __syncthreads();
  } else {
    // inverse-only pass: coefficients -> buffer positions, then the pairs' pre-processing
#pragma unroll 1
    for (int c0 = 0; c0 < NE; c0 += load_chunk_of<M, V>())
      load_chunk<M, V, COL>(A, em, c0, [&](int line, int pos, float x) { re_at<M, V>(buf, line, pos) = x; });
    __syncthreads();
    float val[E / 2][4];
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
      int pos[4];
      pair_positions<M, FAM>(u + T * i, kind, pos);
#pragma unroll
      for (int c = 0; c < 4; ++c) val[i][c] = re_at<M, V>(buf, l, pos[c]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < E / 2; ++i) inv_pair<M, V, FAM>(buf, l, u + T * i, kind, tw, val[i]);
    __syncthreads();
  }
  fft<M, V>(buf, u, l, tw, nullptr);
  const float scale = A.out_scale;
  store_phase<M, V, COL>(A, em, [&](int line, int p) { return inv_value<M, V, FAM>(buf, line, p, kind, tw) * scale; });
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
