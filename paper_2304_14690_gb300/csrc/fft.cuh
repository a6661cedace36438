// Shared-memory transforms for the Poisson solve (§2.3 three-step algorithm).
//
// A CTA holds a tile of L lines of one axis in shared memory as complex slots: line l,
// slot q at buf[l*ls + q*es] (row tiles: es = 1, ls = M; column tiles: es = L, ls = 1).
// Column tiles map consecutive threads to consecutive lines (coalesced global access across
// adjacent lines), row tiles map them to consecutive positions of one line. A thread covers the
// positions lane, lane + tpl, ... of its line, tpl = threads per line (a power of two) with at
// most EMAX slots per thread, so all index arithmetic is shifts, masks and one multiply-high
// per FFT stage.
//
// Every real-to-real transform of length n (n even) runs through one complex FFT of length
// M = n/2:
//   periodic    real DFT, packed output [X0, X_{n/2}, Re X1, Im X1, Re X2, ...]
//   Neu-Neu     DCT-II forward / DCT-III inverse (Makhoul's reordering + real DFT)
//   Dir-Dir     DST-II / DST-III (DCT-II of the sign-alternated line, reversed)
//   Neu-Dir     DCT-IV (self-inverse up to 2/n), half-length complex FFT with pre/post twiddles
//   Dir-Neu     DST-IV (DCT-IV of the reversed line with alternating output signs)
// The vertex (regular) grid of §2.3 has its own transforms, on lines of unknowns at the lattice
// vertices (m cells along the axis):
//   Neu-Neu     DCT-I of the m+1 unknowns: the real DFT of length 2m of their even extension,
//               formed in shared memory (M = m); the spectrum is real, X_k = Re V_k
//   Dir-Dir     DST-I of the m-1 unknowns: the real DFT of their odd extension (M = m); the
//               spectrum is imaginary, X_{k-1} = -Im V_k
//   Neu-Dir     quarter-wave cosine basis cos(pi (k + 1/2) j/m): its analysis is the DCT-III
//               and its synthesis the DCT-II of length m, the cell grid's Neu-Neu pair run in
//               the other order (M = m/2)
//   Dir-Neu     quarter-wave sine basis, likewise the cell grid's Dir-Dir pair in the other order
// The FFT is a mixed-radix Stockham autosort (radices 16, 8, 4, 2, 3, 5) between two shared
// buffers: every stage reads its butterflies' inputs from one buffer into registers and writes
// the outputs to the other, one barrier per stage. The radix-8 and radix-16 butterflies run in
// registers (2 x 4 and 4 x 4 decompositions).
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

// ----------------------------------------------------------------------------- butterflies
// Forward transforms use the kernel e^{-2 pi i/R}, inverse ones its conjugate.
template <typename T, bool INV> __device__ __forceinline__ T rot4(T a) { return INV ? cmul_pi(a) : cmul_mi(a); }

template <typename T, bool INV>
__device__ __forceinline__ void dft4(T &a0, T &a1, T &a2, T &a3) {
  const T s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const T s13 = cadd(a1, a3), d13 = rot4<T, INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// e^{-+2 pi i e/16} for the exponents the radix-8 and radix-16 butterflies use (cosines and
// sines of multiples of pi/8).
template <typename T, bool INV>
__device__ __forceinline__ T w16(int e) {
  using R = decltype(T::x);
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, r2 = (R)0.70710678118654752440;
  R re, im;
  switch (e) {
    case 1: re = c1; im = -s1; break;
    case 2: re = r2; im = -r2; break;
    case 3: re = s1; im = -c1; break;
    case 4: re = 0; im = -1; break;
    case 6: re = -r2; im = -r2; break;
    case 9: re = -c1; im = s1; break;
    default: re = 1; im = 0; break;
  }
  return cmk<T>(re, INV ? -im : im);
}

// Small DFT of radix R on v[0..R-1], outputs in natural order. Radix 3 and 5 take their roots of
// unity from the length-M FFT table (M divisible by R).
template <typename T, int R, bool INV>
__device__ __forceinline__ void small_dft(T *v, const T *tw, int M) {
  if (R == 2) {
    const T a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (R == 4) {
    dft4<T, INV>(v[0], v[1], v[2], v[3]);
  } else if (R == 8) {
    // X_{2m} = DFT4(x_k + x_{k+4}), X_{2m+1} = DFT4((x_k - x_{k+4}) w8^k)
    T u[4], d[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      u[k] = cadd(v[k], v[k + 4]);
      d[k] = csub(v[k], v[k + 4]);
    }
    d[1] = cmul(d[1], w16<T, INV>(2));
    d[2] = rot4<T, INV>(d[2]);
    d[3] = cmul(d[3], w16<T, INV>(6));
    dft4<T, INV>(u[0], u[1], u[2], u[3]);
    dft4<T, INV>(d[0], d[1], d[2], d[3]);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      v[2 * m] = u[m];
      v[2 * m + 1] = d[m];
    }
  } else if (R == 16) {
    // input k = k1 + 4 k2, output j = j2 + 4 j1: DFT4 over k2, twiddle w16^(j2 k1), DFT4 over k1
    T y[4][4];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      y[k1][0] = v[k1];
      y[k1][1] = v[k1 + 4];
      y[k1][2] = v[k1 + 8];
      y[k1][3] = v[k1 + 12];
      dft4<T, INV>(y[k1][0], y[k1][1], y[k1][2], y[k1][3]);
    }
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) {
#pragma unroll
      for (int j2 = 1; j2 < 4; ++j2) {
        if (j2 * k1 == 4) y[k1][j2] = rot4<T, INV>(y[k1][j2]);
        else y[k1][j2] = cmul(y[k1][j2], w16<T, INV>(j2 * k1));
      }
    }
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) {
      dft4<T, INV>(y[0][j2], y[1][j2], y[2][j2], y[3][j2]);
#pragma unroll
      for (int j1 = 0; j1 < 4; ++j1) v[j2 + 4 * j1] = y[j1][j2];
    }
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
        const T w = ldg(&tw[((q * r) % R) * step]);
        acc = cadd(acc, INV ? cmulc(in[r], w) : cmul(in[r], w));
      }
      v[q] = acc;
    }
  }
}

// One Stockham stage of radix R from src to dst over every line of the tile. A thread does up to
// MAXB butterflies (j = lane, lane + tpl, ...). pre (nullable): a slot-wise factor applied to the
// inputs (the DCT-IV pre-twiddle, folded into the first stage).
template <typename T, int R, int MAXB, bool INV>
__device__ __forceinline__ void fft_stage(const T *src, T *dst, const TileGeom &g, const StageInfo &s,
                                          const T *tw, const T *pre) {
  const int NBl = g.M / R;
  const int base = g.line * g.ls;
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    const int j = g.lane + b * g.tpl;
    if (j < NBl) {
      T v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int q = j + r * NBl;
        v[r] = src[base + q * g.es];
        if (pre) v[r] = cmul(v[r], ldg(&pre[q]));
      }
      const int qd = s.shift >= 0 ? (j >> s.shift) : (int)__umulhi((unsigned)j, s.magic);
      const int k = j - qd * s.Ns;
      if (s.Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const T w = ldg(&tw[r * k * s.stride_m]);
          v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
        }
      }
      small_dft<T, R, INV>(v, tw, g.M);
      const int ob = qd * s.Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[base + (ob + r * s.Ns) * g.es] = v[r];
    }
  }
  __syncthreads();
}

constexpr int cdiv_c(int a, int b) { return (a + b - 1) / b; }

// Complex FFT of length g.M on every line (unnormalised), ping-ponging between a and b; returns
// the buffer that holds the result. Every thread of the CTA calls it (barriers). POW2: M is a
// power of two, so the radix-3 and radix-5 stages are not compiled into the caller.
template <typename T, int EMAX, bool INV, bool POW2 = false>
__device__ T *fft_run(T *a, T *b, const TileGeom &g, const StageInfo *st, int nst, const T *tw, const T *pre) {
  for (int s = 0; s < nst; ++s) {
    const StageInfo si = st[s];
    const T *p0 = (s == 0) ? pre : nullptr;
    // power-of-two radices above EMAX never occur (radix schedule), so they are not compiled
    switch (si.R) {
      case 16:
        if constexpr (EMAX >= 16) fft_stage<T, 16, cdiv_c(EMAX, 16), INV>(a, b, g, si, tw, p0);
        break;
      case 8:
        if constexpr (EMAX >= 8) fft_stage<T, 8, cdiv_c(EMAX, 8), INV>(a, b, g, si, tw, p0);
        break;
      case 4:
        if constexpr (EMAX >= 4) fft_stage<T, 4, cdiv_c(EMAX, 4), INV>(a, b, g, si, tw, p0);
        break;
      case 2: fft_stage<T, 2, cdiv_c(EMAX, 2), INV>(a, b, g, si, tw, p0); break;
      case 3:
        if constexpr (!POW2) fft_stage<T, 3, cdiv_c(EMAX, 3), INV>(a, b, g, si, tw, p0);
        break;
      default:
        if constexpr (!POW2) fft_stage<T, 5, cdiv_c(EMAX, 5), INV>(a, b, g, si, tw, p0);
        break;
    }
    T *t = a;
    a = b;
    b = t;
  }
  return a;
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

// F1 of the vertex DCT-I / DST-I: input x_j (unknown j of the line) enters the real line of
// length 2M at its own position and at the mirrored one (even extension for DCT-I, odd for DST-I,
// whose unknown j is vertex j + 1). The caller writes the two zeros of the odd extension.
template <typename T>
__device__ __forceinline__ void ext_scatter(T *buf, const TileGeom &g, int line, int kind, int j,
                                            decltype(T::x) x) {
  const int M = g.M;
  const int r = (kind == KIND_VDD) ? j + 1 : j;
  realref(buf, g, line, r) = x;
  if (r > 0 && r < M) realref(buf, g, line, 2 * M - r) = (kind == KIND_VDD) ? -x : x;
}

// F4: FFT output (slots of buf) -> real spectral coefficients in natural order, handed to
// emit(position, value). A thread reads only the slots of its own outputs.
template <typename T, typename Emit>
__device__ __forceinline__ void fwd_post(const T *buf, const TileGeom &g, int kind, int n, const T *tw, Emit emit) {
  using R = decltype(T::x);
  const int M = g.M;
  const int base = g.line * g.ls;
  auto at = [&](int q) { return buf[base + q * g.es]; };
  if (kind == KIND_ND || kind == KIND_DN) {
    // y_q = e^{-i pi q/n} Z_q; X_2q = Re y_q; X_{n-1-2q} = -Im y_q (DCT-IV), +Im y_q (DST-IV)
    const T *tp = tw + tw_dct4post(M);
    for (int q = g.lane; q < M; q += g.tpl) {
      const T y = cmul(at(q), ldg(&tp[q]));
      emit(2 * q, y.x);
      emit(n - 1 - 2 * q, (kind == KIND_ND) ? -y.y : y.y);
    }
    return;
  }
  // Real DFT of the (reordered) line from the half-length FFT: pairs (k, M-k), k <= M/2.
  const int P = M / 2 + 1;
  const T *w1 = tw + tw_rdft(M);
  const T *wq = tw + tw_quarter(M);
  const bool dd = kind == KIND_DD;
  for (int k = g.lane; k < P; k += g.tpl) {
    if (k == 0) {
      const T z = at(0);
      const R V0 = z.x + z.y, VM = z.x - z.y;
      if (kind == KIND_PP) {
        emit(0, V0);
        emit(1, VM);
      } else if (kind == KIND_VNN) {
        emit(0, V0);
        emit(M, VM);
      } else if (kind == KIND_VDD) {
        // V_0 = V_M = 0 for an odd extension: no coefficient
      } else {
        const T tM = cscale(ldg(&wq[M]), VM);
        emit(dd ? n - 1 : 0, V0);
        emit(dd ? n - 1 - M : M, tM.x);
      }
      continue;
    }
    const int km = M - k;
    const T zk = at(k), zm = at(km);
    // V_k = E + w^k O,  E = (Zk + conj Zm)/2,  O = -i (Zk - conj Zm)/2
    const T E = cscale(cadd(zk, cconj(zm)), (R)0.5), O = cscale(cmul_mi(csub(zk, cconj(zm))), (R)0.5);
    const T Vk = cadd(E, cmul(O, ldg(&w1[k])));
    T Vm = Vk;
    if (km != k) {
      const T E2 = cscale(cadd(zm, cconj(zk)), (R)0.5), O2 = cscale(cmul_mi(csub(zm, cconj(zk))), (R)0.5);
      Vm = cadd(E2, cmul(O2, ldg(&w1[km])));
    }
    if (kind == KIND_PP) {
      emit(2 * k, Vk.x);
      emit(2 * k + 1, Vk.y);
      if (km != k) {
        emit(2 * km, Vm.x);
        emit(2 * km + 1, Vm.y);
      }
    } else if (kind == KIND_VNN) {
      // even extension: V_k real, the DCT-I coefficient k
      emit(k, Vk.x);
      if (km != k) emit(km, Vm.x);
    } else if (kind == KIND_VDD) {
      // odd extension: V_k = -i X, the DST-I coefficient of sin(pi k j/M) stored at k - 1
      emit(k - 1, -Vk.y);
      if (km != k) emit(km - 1, -Vm.y);
    } else {
      // DCT-II (DST-II by reversal): t_k = e^{-i pi k/(2n)} V_k; X_k = Re t_k, X_{n-k} = -Im t_k
      const T tk = cmul(Vk, ldg(&wq[k]));
      emit(dd ? n - 1 - k : k, tk.x);
      emit(dd ? k - 1 : n - k, -tk.y);
      if (km != k) {
        const T tm = cmul(Vm, ldg(&wq[km]));
        emit(dd ? n - 1 - km : km, tm.x);
        emit(dd ? km - 1 : n - km, -tm.y);
      }
    }
  }
}

// ----------------------------------------------------------------------------- inverse
// I1: real spectral coefficients (natural order, read through fetch(i)) -> complex slots of
// buf for the inverse FFT. A thread writes the slots of its own pairs; the caller puts a barrier
// after it.
template <typename T, typename Fetch>
__device__ __forceinline__ void inv_pre(T *buf, const TileGeom &g, int kind, int n, const T *tw, Fetch fetch) {
  using R = decltype(T::x);
  const int M = g.M;
  const int base = g.line * g.ls;
  auto put = [&](int q, T v) { buf[base + q * g.es] = v; };
  if (kind == KIND_ND || kind == KIND_DN) {
    // The inverse of DCT-IV/DST-IV is the same transform times 2/n: same pre-processing.
    const T *t4 = tw + tw_dct4pre(M);
    for (int q = g.lane; q < M; q += g.tpl) {
      const R x0 = fetch(2 * q), x1 = fetch(n - 1 - 2 * q);
      const T z = (kind == KIND_ND) ? cmk<T>(x0, x1) : cmk<T>(x1, x0);
      put(q, cmul(z, ldg(&t4[q])));
    }
    return;
  }
  const int P = M / 2 + 1;
  const T *w1 = tw + tw_rdft(M);
  const T *wq = tw + tw_quarter(M);
  const bool dd = kind == KIND_DD;
  // coefficient i of the line (reversed for DST-III); X_n = 0
  auto X = [&](int i) -> R {
    if (i >= n) return (R)0;
    return fetch(dd ? n - 1 - i : i);
  };
  // DCT-III: V_k = e^{+i pi k/(2n)} (X_k - i X_{n-k})
  auto V = [&](int i) -> T { return cmulc(cmk<T>(X(i), -X(n - i)), ldg(&wq[i])); };
  for (int k = g.lane; k < P; k += g.tpl) {
    if (k == 0) {
      R a, b;
      if (kind == KIND_PP) {
        a = fetch(0);   // X_0
        b = fetch(1);   // X_M
      } else if (kind == KIND_VNN) {
        a = fetch(0);
        b = fetch(M);
      } else if (kind == KIND_VDD) {
        a = (R)0;
        b = (R)0;
      } else {
        a = X(0);
        b = V(M).x;     // real: sqrt(2) X_M
      }
      put(0, cmk<T>((R)0.5 * (a + b), (R)0.5 * (a - b)));
      continue;
    }
    const int km = M - k;
    T xk, xm;
    if (kind == KIND_PP) {
      xk = cmk<T>(fetch(2 * k), fetch(2 * k + 1));
      xm = cmk<T>(fetch(2 * km), fetch(2 * km + 1));
    } else if (kind == KIND_VNN) {   // the real, even spectrum of the even extension
      xk = cmk<T>(fetch(k), (R)0);
      xm = cmk<T>(fetch(km), (R)0);
    } else if (kind == KIND_VDD) {   // the imaginary, odd spectrum of the odd extension
      xk = cmk<T>((R)0, -fetch(k - 1));
      xm = cmk<T>((R)0, -fetch(km - 1));
    } else {
      xk = V(k);
      xm = V(km);
    }
    // Z_k = E + i O, E = (X_k + conj X_{M-k})/2, O = (X_k - conj X_{M-k}) conj(w^k)/2
    const T E = cscale(cadd(xk, cconj(xm)), (R)0.5);
    const T O = cscale(cmulc(csub(xk, cconj(xm)), ldg(&w1[k])), (R)0.5);
    put(k, cadd(E, cmul_pi(O)));
    if (km != k) {
      const T E2 = cscale(cadd(xm, cconj(xk)), (R)0.5);
      const T O2 = cscale(cmulc(csub(xm, cconj(xk)), ldg(&w1[km])), (R)0.5);
      put(km, cadd(E2, cmul_pi(O2)));
    }
  }
}

// I3: output x_i (before the 2/n normalisation) from the inverse FFT result in buf.
template <typename T>
__device__ __forceinline__ decltype(T::x) inv_out(const T *buf, const TileGeom &g, int kind, int n, const T *tw,
                                                  int i) {
  const int base = g.line * g.ls;
  if (kind == KIND_PP || kind == KIND_VNN || kind == KIND_VDD) {
    const int r = (kind == KIND_VDD) ? i + 1 : i;   // position in the (extended) real line
    const T z = buf[base + (r >> 1) * g.es];
    return (r & 1) ? z.y : z.x;
  }
  if (kind == KIND_NN || kind == KIND_DD) {
    const int j = (i & 1) ? (n - 1 - (i >> 1)) : (i >> 1);
    const T z = buf[base + (j >> 1) * g.es];
    const auto v = (j & 1) ? z.y : z.x;
    return (kind == KIND_DD && (i & 1)) ? -v : v;
  }
  // DCT-IV / DST-IV: y_q = e^{-i pi q/n} Z_q; x_2q = Re y_q, x_{n-1-2q} = -+Im y_q
  const int q = (i & 1) ? ((n - 1 - i) >> 1) : (i >> 1);
  const T y = cmul(buf[base + q * g.es], ldg(tw + tw_dct4post(g.M) + q));
  if ((i & 1) == 0) return y.x;
  return (kind == KIND_ND) ? -y.y : y.y;
}

// Normalisation of every inverse: 1/M of the half-length inverse FFT for the real DFT and
// DCT-III/DST-III wrappers, 2/n = 1/M for DCT-IV/DST-IV; 1/M too for the vertex transforms (the
// real DFT of the length-2M extension, and the quarter-wave pairs of length 2M).
__host__ __device__ inline double inv_scale(int M) { return 1.0 / M; }

}  // namespace pc
