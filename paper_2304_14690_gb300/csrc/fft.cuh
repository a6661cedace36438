// Shared-memory transforms for the Poisson solve (§2.3 three-step algorithm).
//
// A CTA holds a tile of L lines of one axis in shared memory as complex slots: line l,
// slot q at buf[l*ls + q*es] (row tiles: es = 1, ls = M; column tiles: es = L, ls = 1).
// Every thread works on one line of the tile: column tiles map consecutive threads to
// consecutive lines (coalesced global access across adjacent lines), row tiles map them to
// consecutive positions of one line. A thread covers the positions lane, lane + tpl, ... of its
// line, tpl = threads per line (a power of two, >= M/2), so all index arithmetic is shifts,
// masks and one multiply-high per FFT stage.
//
// Every real-to-real transform of length n (n even) runs through one complex FFT of length
// M = n/2:
//   periodic    real DFT, packed output [X0, X_{n/2}, Re X1, Im X1, Re X2, ...]
//   Neu-Neu     DCT-II forward / DCT-III inverse (Makhoul's reordering + real DFT)
//   Dir-Dir     DST-II / DST-III (DCT-II of the sign-alternated line, reversed)
//   Neu-Dir     DCT-IV (self-inverse up to 2/n), half-length complex FFT with pre/post twiddles
//   Dir-Neu     DST-IV (DCT-IV of the reversed line with alternating output signs)
// The FFT is a mixed-radix (2,3,4,5) Stockham autosort done in place: every stage reads its
// butterfly inputs into registers, synchronises, and writes the outputs.
#pragma once

#include <cuda_runtime.h>
#include "pc_internal.cuh"

namespace pc {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename T> __device__ __forceinline__ T cmk(decltype(T::x) a, decltype(T::x) b) {
  T r; r.x = a; r.y = b; return r;
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return cmk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return cmk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  return cmk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ T cmulc(T a, T b) {
  return cmk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ T cconj(T a) { return cmk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ T cscale(T a, decltype(T::x) s) { return cmk<T>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename T> __device__ __forceinline__ T cmul_mi(T a) { return cmk<T>(a.y, -a.x); }
template <typename T> __device__ __forceinline__ T cmul_pi(T a) { return cmk<T>(-a.y, a.x); }
template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Thread-to-tile map: this thread's line and its first position; tpl threads per line.
struct TileGeom {
  int L;     // lines in the tile
  int M;     // complex slots per line
  int ls;    // slot stride between lines
  int es;    // slot stride along a line
  int line;  // line of this thread
  int lane;  // first position of this thread on its line
  int tpl;   // threads per line (position stride)
};

// Work items a thread keeps in registers across a barrier are bounded by tpl >= M/2: every
// FFT stage is one butterfly per thread.
constexpr int kSlotsPerThread = 2;

// One FFT stage: radix R, current span Ns, twiddle stride M/(Ns R). j / Ns is a shift when Ns
// is a power of two, else a multiply-high by magic = ceil(2^32/Ns) (exact for j < 2^16).
struct StageInfo {
  int R, Ns, stride_m, shift;   // shift < 0: use magic
  unsigned magic;
};

// Table offsets inside one axis twiddle buffer (see AxisInfo).
__host__ __device__ inline int tw_rdft(int M) { return M; }            // e^{-2 pi i k/n}, k=0..M
__host__ __device__ inline int tw_quarter(int M) { return 2 * M + 1; }  // e^{-i pi k/(2n)}, k=0..M
__host__ __device__ inline int tw_dct4pre(int M) { return 3 * M + 2; }  // e^{-i pi (4p+1)/(4n)}, p<M
__host__ __device__ inline int tw_dct4post(int M) { return 4 * M + 2; } // e^{-i pi q/n}, q<M
__host__ __device__ inline int tw_total(int M) { return 5 * M + 2; }

template <typename T>
__device__ __forceinline__ T &slot(T *buf, const TileGeom &g, int line, int q) {
  return buf[line * g.ls + q * g.es];
}
template <typename T>
__device__ __forceinline__ decltype(T::x) &realref(T *buf, const TileGeom &g, int line, int j) {
  using R = decltype(T::x);
  return reinterpret_cast<R *>(buf)[2 * (line * g.ls + (j >> 1) * g.es) + (j & 1)];
}

// Small DFT of radix R on v[0..R-1] (forward sign -1, inverse +1). Radix 3 and 5 take their
// roots of unity from the length-M FFT table (M divisible by R).
template <typename T, int R>
__device__ __forceinline__ void small_dft(T *v, const T *tw, int M, bool inv) {
  if (R == 2) {
    T a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  } else if (R == 4) {
    T a0 = v[0], a1 = v[1], a2 = v[2], a3 = v[3];
    T s02 = cadd(a0, a2), d02 = csub(a0, a2);
    T s13 = cadd(a1, a3), d13 = csub(a1, a3);
    T rot = inv ? cmul_pi(d13) : cmul_mi(d13);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, rot);
    v[3] = csub(d02, rot);
  } else {
    T in[R];
#pragma unroll
    for (int r = 0; r < R; ++r) in[r] = v[r];
    const int step = M / R;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      T acc = in[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        T w = ldg(&tw[((q * r) % R) * step]);
        acc = cadd(acc, inv ? cmulc(in[r], w) : cmul(in[r], w));
      }
      v[q] = acc;
    }
  }
}

// One Stockham stage of radix R over every line of the tile (all threads of the CTA).
template <typename T, int R, int MAXB>
__device__ void fft_stage(T *buf, const TileGeom &g, const StageInfo &s, const T *tw, bool inv) {
  const int NBl = g.M / R;
  T v[MAXB][R];
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    int j = g.lane + b * g.tpl;
    if (j < NBl) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = slot(buf, g, g.line, j + r * NBl);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    int j = g.lane + b * g.tpl;
    if (j < NBl) {
      int q = s.shift >= 0 ? (j >> s.shift) : (int)__umulhi((unsigned)j, s.magic);
      int k = j - q * s.Ns;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        T w = ldg(&tw[r * k * s.stride_m]);
        v[b][r] = inv ? cmulc(v[b][r], w) : cmul(v[b][r], w);
      }
      small_dft<T, R>(v[b], tw, g.M, inv);
      int base = q * s.Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) slot(buf, g, g.line, base + r * s.Ns) = v[b][r];
    }
  }
  __syncthreads();
}

// Complex FFT of length g.M on every line (unnormalised).
template <typename T>
__device__ void fft_lines(T *buf, const TileGeom &g, const StageInfo *st, int nst, const T *tw,
                          bool inv) {
  for (int s = 0; s < nst; ++s) {
    const StageInfo si = st[s];
    if (si.R == 4) fft_stage<T, 4, 1>(buf, g, si, tw, inv);
    else if (si.R == 2) fft_stage<T, 2, 1>(buf, g, si, tw, inv);
    else if (si.R == 3) fft_stage<T, 3, 1>(buf, g, si, tw, inv);
    else fft_stage<T, 5, 1>(buf, g, si, tw, inv);
  }
}

// ----------------------------------------------------------------------------- forward
// Where real input x_j goes among the complex slots before the FFT (F1): slot, component
// (0 real, 1 imaginary) and sign.
__device__ __forceinline__ void fwd_slot_of(int kind, int n, int j, int &q, int &comp, bool &neg) {
  neg = false;
  if (kind == KIND_PP) { q = j >> 1; comp = j & 1; return; }
  if (kind == KIND_NN || kind == KIND_DD) {
    int v = (j & 1) ? (n - 1 - (j >> 1)) : (j >> 1);   // Makhoul reorder
    q = v >> 1; comp = v & 1;
    neg = (kind == KIND_DD) && (j & 1);                 // (-1)^j
    return;
  }
  // DCT-IV / DST-IV: z_p = (a + i b) with (a, b) = (x_2p, x_{n-1-2p}) or swapped for DST-IV
  bool even = (j & 1) == 0;
  q = even ? (j >> 1) : ((n - 1 - j) >> 1);
  comp = even ? 0 : 1;
  if (kind == KIND_DN) comp ^= 1;
}

// F2: slot-local pre-twiddle (DCT-IV / DST-IV only).
template <typename T>
__device__ void pretwiddle(T *buf, const TileGeom &g, int kind, const T *tw) {
  if (kind != KIND_ND && kind != KIND_DN) return;
  const T *t4 = tw + tw_dct4pre(g.M);
  for (int q = g.lane; q < g.M; q += g.tpl) {
    T &z = slot(buf, g, g.line, q);
    z = cmul(z, ldg(&t4[q]));
  }
  __syncthreads();
}

// F4: FFT output -> real spectral coefficients in natural order (in place, via registers).
template <typename T>
__device__ void fwd_post(T *buf, const TileGeom &g, int kind, int n, const T *tw) {
  using R = decltype(T::x);
  const int M = g.M;
  const int line = g.line;
  if (kind == KIND_ND || kind == KIND_DN) {
    // y_q = e^{-i pi q/n} Z_q; X_2q = Re y_q; X_{n-1-2q} = -Im y_q (DCT-IV), +Im y_q (DST-IV)
    const T *tp = tw + tw_dct4post(M);
    constexpr int MAXI = kSlotsPerThread;
    T y[MAXI];
#pragma unroll
    for (int b = 0; b < MAXI; ++b) {
      int q = g.lane + b * g.tpl;
      if (q < M) y[b] = cmul(slot(buf, g, line, q), ldg(&tp[q]));
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXI; ++b) {
      int q = g.lane + b * g.tpl;
      if (q < M) {
        realref(buf, g, line, 2 * q) = y[b].x;
        realref(buf, g, line, n - 1 - 2 * q) = (kind == KIND_ND) ? -y[b].y : y[b].y;
      }
    }
    __syncthreads();
    return;
  }
  // Real DFT of the (reordered) line from the half-length FFT: pairs (k, M-k), k <= M/2.
  const int P = M / 2 + 1;
  const T *w1 = tw + tw_rdft(M);
  if (kind == KIND_PP) {
    for (int k = g.lane; k < P; k += g.tpl) {
      if (k == 0) {
        T z = slot(buf, g, line, 0);
        slot(buf, g, line, 0) = cmk<T>(z.x + z.y, z.x - z.y);
        continue;
      }
      int km = M - k;
      T zk = slot(buf, g, line, k), zm = slot(buf, g, line, km);
      // X_k = E + w^k O,  E = (Zk + conj Zm)/2,  O = -i (Zk - conj Zm)/2
      T E = cscale(cadd(zk, cconj(zm)), (R)0.5), O = cscale(cmul_mi(csub(zk, cconj(zm))), (R)0.5);
      T Xk = cadd(E, cmul(O, ldg(&w1[k])));
      if (km != k) {
        T E2 = cscale(cadd(zm, cconj(zk)), (R)0.5), O2 = cscale(cmul_mi(csub(zm, cconj(zk))), (R)0.5);
        slot(buf, g, line, km) = cadd(E2, cmul(O2, ldg(&w1[km])));
      }
      slot(buf, g, line, k) = Xk;
    }
    __syncthreads();
    return;
  }
  // DCT-II (and DST-II by reversal): V = real DFT of v; t_k = e^{-i pi k/(2n)} V_k;
  // X_k = Re t_k, X_{n-k} = -Im t_k.
  const T *wq = tw + tw_quarter(M);
  constexpr int MAXP = kSlotsPerThread / 2 + 1;
  R out[MAXP][4];
  int pos[MAXP][4];
#pragma unroll
  for (int b = 0; b < MAXP; ++b) {
    int k = g.lane + b * g.tpl;
#pragma unroll
    for (int c = 0; c < 4; ++c) pos[b][c] = -1;
    if (k < P) {
      if (k == 0) {
        T z = slot(buf, g, line, 0);
        R V0 = z.x + z.y, VM = z.x - z.y;
        T tM = cscale(ldg(&wq[M]), VM);
        out[b][0] = V0; pos[b][0] = 0;
        out[b][1] = tM.x; pos[b][1] = M;
      } else {
        int km = M - k;
        T zk = slot(buf, g, line, k), zm = slot(buf, g, line, km);
        T E = cscale(cadd(zk, cconj(zm)), (R)0.5), O = cscale(cmul_mi(csub(zk, cconj(zm))), (R)0.5);
        T Vk = cadd(E, cmul(O, ldg(&w1[k])));
        T tk = cmul(Vk, ldg(&wq[k]));
        out[b][0] = tk.x; pos[b][0] = k;
        out[b][1] = -tk.y; pos[b][1] = n - k;
        if (km != k) {
          T E2 = cscale(cadd(zm, cconj(zk)), (R)0.5), O2 = cscale(cmul_mi(csub(zm, cconj(zk))), (R)0.5);
          T Vm = cadd(E2, cmul(O2, ldg(&w1[km])));
          T tm = cmul(Vm, ldg(&wq[km]));
          out[b][2] = tm.x; pos[b][2] = km;
          out[b][3] = -tm.y; pos[b][3] = n - km;
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < MAXP; ++b) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (pos[b][c] >= 0) {
        int i = pos[b][c];
        if (kind == KIND_DD) i = n - 1 - i;
        realref(buf, g, line, i) = out[b][c];
      }
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------- inverse
// I1: real spectral coefficients (natural order, in place) -> complex slots for the inverse FFT.
template <typename T>
__device__ void inv_pre(T *buf, const TileGeom &g, int kind, int n, const T *tw) {
  using R = decltype(T::x);
  const int M = g.M;
  const int line = g.line;
  if (kind == KIND_ND || kind == KIND_DN) {
    // The inverse of DCT-IV/DST-IV is the same transform times 2/n: same pre-processing.
    constexpr int MAXI = kSlotsPerThread;
    R a[MAXI], bb[MAXI];
#pragma unroll
    for (int b = 0; b < MAXI; ++b) {
      int q = g.lane + b * g.tpl;
      if (q < M) {
        R x0 = realref(buf, g, line, 2 * q), x1 = realref(buf, g, line, n - 1 - 2 * q);
        a[b] = (kind == KIND_ND) ? x0 : x1;
        bb[b] = (kind == KIND_ND) ? x1 : x0;
      }
    }
    __syncthreads();
    const T *t4 = tw + tw_dct4pre(M);
#pragma unroll
    for (int b = 0; b < MAXI; ++b) {
      int q = g.lane + b * g.tpl;
      if (q < M) slot(buf, g, line, q) = cmul(cmk<T>(a[b], bb[b]), ldg(&t4[q]));
    }
    __syncthreads();
    return;
  }
  const int P = M / 2 + 1;
  const T *w1 = tw + tw_rdft(M);
  if (kind == KIND_PP) {
    for (int k = g.lane; k < P; k += g.tpl) {
      if (k == 0) {
        T z = slot(buf, g, line, 0);   // (X_0, X_M), both real
        R E = (R)0.5 * (z.x + z.y), O = (R)0.5 * (z.x - z.y);
        slot(buf, g, line, 0) = cmk<T>(E, O);   // Z_0 = E + i O
        continue;
      }
      int km = M - k;
      T xk = slot(buf, g, line, k), xm = slot(buf, g, line, km);
      // Z_k = E + i O, E = (X_k + conj X_{M-k})/2, O = (X_k - conj X_{M-k}) conj(w^k)/2
      T E = cscale(cadd(xk, cconj(xm)), (R)0.5);
      T O = cscale(cmulc(csub(xk, cconj(xm)), ldg(&w1[k])), (R)0.5);
      T Zk = cadd(E, cmul_pi(O));
      if (km != k) {
        T E2 = cscale(cadd(xm, cconj(xk)), (R)0.5);
        T O2 = cscale(cmulc(csub(xm, cconj(xk)), ldg(&w1[km])), (R)0.5);
        slot(buf, g, line, km) = cadd(E2, cmul_pi(O2));
      }
      slot(buf, g, line, k) = Zk;
    }
    __syncthreads();
    return;
  }
  // DCT-III (DST-III through the reversal Y_i = X_{n-1-i}):
  // V_k = e^{+i pi k/(2n)} (X_k - i X_{n-k}) with X_n = 0, then the inverse real DFT wrapper.
  const T *wq = tw + tw_quarter(M);
  constexpr int MAXP = kSlotsPerThread / 2 + 1;
  T zo[MAXP][2];
#pragma unroll
  for (int b = 0; b < MAXP; ++b) {
    int k = g.lane + b * g.tpl;
    if (k < P) {
      auto X = [&](int i) -> R {
        if (i >= n) return (R)0;
        return realref(buf, g, line, kind == KIND_DD ? n - 1 - i : i);
      };
      auto V = [&](int i) -> T { return cmulc(cmk<T>(X(i), -X(n - i)), ldg(&wq[i])); };
      if (k == 0) {
        R V0 = X(0);
        R VM = V(M).x;   // real: sqrt(2) X_M
        zo[b][0] = cmk<T>((R)0.5 * (V0 + VM), (R)0.5 * (V0 - VM));
      } else {
        int km = M - k;
        T vk = V(k), vm = V(km);
        T E = cscale(cadd(vk, cconj(vm)), (R)0.5);
        T O = cscale(cmulc(csub(vk, cconj(vm)), ldg(&w1[k])), (R)0.5);
        zo[b][0] = cadd(E, cmul_pi(O));
        if (km != k) {
          T E2 = cscale(cadd(vm, cconj(vk)), (R)0.5);
          T O2 = cscale(cmulc(csub(vm, cconj(vk)), ldg(&w1[km])), (R)0.5);
          zo[b][1] = cadd(E2, cmul_pi(O2));
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < MAXP; ++b) {
    int k = g.lane + b * g.tpl;
    if (k < P) {
      slot(buf, g, line, k) = zo[b][0];
      int km = M - k;
      if (k != 0 && km != k) slot(buf, g, line, km) = zo[b][1];
    }
  }
  __syncthreads();
}

// I3 (part 1): slot-local post twiddle for DCT-IV / DST-IV before the gather.
template <typename T>
__device__ void inv_post_twiddle(T *buf, const TileGeom &g, int kind, const T *tw) {
  if (kind != KIND_ND && kind != KIND_DN) return;
  const T *tp = tw + tw_dct4post(g.M);
  for (int q = g.lane; q < g.M; q += g.tpl) {
    T &z = slot(buf, g, g.line, q);
    z = cmul(z, ldg(&tp[q]));
  }
  __syncthreads();
}

// I3 (part 2): where output x_i is read from after the inverse FFT, with sign; the caller
// multiplies by inv_scale(kind, n).
__device__ __forceinline__ void inv_src_of(int kind, int n, int i, int &j, bool &neg) {
  neg = false;
  if (kind == KIND_PP) { j = i; return; }
  if (kind == KIND_NN || kind == KIND_DD) {
    j = (i & 1) ? (n - 1 - (i >> 1)) : (i >> 1);
    neg = (kind == KIND_DD) && (i & 1);
    return;
  }
  // DCT-IV / DST-IV: x_2q = Re y_q, x_{n-1-2q} = -+Im y_q  (real index 2q / 2q+1 of slot q)
  if ((i & 1) == 0) { j = i; return; }
  int q = (n - 1 - i) >> 1;
  j = 2 * q + 1;
  neg = (kind == KIND_ND);
}

// Normalisation of every inverse: 1/M of the half-length inverse FFT for the real DFT and
// DCT-III/DST-III wrappers, 2/n for DCT-IV/DST-IV; both equal 2/n.
__host__ __device__ inline double inv_scale(int, int n) { return 2.0 / n; }

}  // namespace pc
