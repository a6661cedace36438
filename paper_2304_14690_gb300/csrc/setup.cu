// Plan-time setup on the GPU, FP64 (§2.2): linked-list neighbour search and the WLS rows.
//
// Neighbours: the K nearest points of a query in the order (squared distance, index), with
//   delta_a = x_point - x_query, minimum image on periodic axes (one IEEE subtraction and at
//   most one wrap by L = n h), d2 = ((d0*d0) + d1*d1) + d2*d2 evaluated left to right with
//   correctly rounded multiplies and adds (no fused multiply-add), so that every exact
//   implementation of the same rule selects the same set.
// The search visits a window of buckets of radius R around the query's bucket and accepts
// when the K-th distance is strictly below the distance from the query to the window's edge;
// otherwise R grows. Nodes are bucketed by a counting sort (histogram, scan, scatter).
//
// WLS rows (Eqs. 13-17, f-unknown basis Eq. 16): support radius hs = factor * r_K * c_d with
// c_2 = sqrt(pi/K), c_3 = (4 pi/(3K))^(1/3); Gaussian weight exp(-eps r^2/hs^2) (Eq. 17);
// offsets scaled by hs; C = sum w q q^T (Eq. 14) factored by Cholesky; row i of C^-1 A is
// w_k (C^-1 e_i) . q_k because C is symmetric.
#include <cmath>
#include <cstdio>
#include <vector>

#include "pc_internal.cuh"

namespace pc {

struct KnnCtx {
  int dim;
  int nb[3];
  double lo[3], cs[3], L[3], halfL[3];
  int periodic[3];
  // node points (cells == 0)
  const int *start;    // [nbuckets + 1]
  const int *sorted;   // node indices, grouped by bucket
  const double *xyz;   // [dim][N]
  long long N;
  int cells;           // 1: the points are grid points (bucket == point): lo + (i + off) h
  double h[3];
  double off[3];       // 0.5 for cell centres, 0 for vertices
};

__device__ __forceinline__ double min_image(double d, int periodic, double L, double halfL) {
  if (periodic) {
    if (d > halfL) d = __dsub_rn(d, L);
    else if (d < -halfL) d = __dadd_rn(d, L);
  }
  return d;
}

__device__ __forceinline__ double cell_centre(const KnnCtx &c, int a, int i) {
  return __dadd_rn(c.lo[a], __dmul_rn((double)i + c.off[a], c.h[a]));
}

__device__ __forceinline__ double point_coord(const KnnCtx &c, int a, long long id) {
  if (c.cells) {
    long long rem = id;
    int idx[3];
    for (int b = c.dim - 1; b >= 0; --b) { idx[b] = (int)(rem % c.nb[b]); rem /= c.nb[b]; }
    return cell_centre(c, a, idx[a]);
  }
  return c.xyz[(long long)a * c.N + id];
}

// Insert (d2, id) into the ascending list (d2, id) of at most K entries.
__device__ __forceinline__ void topk_insert(double *bd, int *bi, int &cnt, int K, double d2, int id) {
  if (cnt == K && (d2 > bd[K - 1] || (d2 == bd[K - 1] && id > bi[K - 1]))) return;
  int pos = (cnt < K) ? cnt : K - 1;
  while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > id))) {
    bd[pos] = bd[pos - 1];
    bi[pos] = bi[pos - 1];
    --pos;
  }
  bd[pos] = d2;
  bi[pos] = id;
  if (cnt < K) ++cnt;
}

// Exact K nearest points of query q. Returns false when fewer than K points exist.
__device__ bool knn_query(const KnnCtx &c, const double *q, int K, double *bd, int *bi) {
  int b0[3] = {0, 0, 0};
  for (int a = 0; a < c.dim; ++a) {
    double t = floor((q[a] - c.lo[a]) / c.cs[a]);
    int b = (int)fmax(0.0, fmin(t, (double)(c.nb[a] - 1)));
    b0[a] = b;
  }
  for (int R = 1;; ++R) {
    int lo_b[3] = {0, 0, 0}, cnt_b[3] = {1, 1, 1};
    bool covered[3] = {true, true, true};
    for (int a = 0; a < c.dim; ++a) {
      if (c.periodic[a]) {
        if (2 * R + 1 >= c.nb[a]) { lo_b[a] = 0; cnt_b[a] = c.nb[a]; covered[a] = true; }
        else { lo_b[a] = b0[a] - R; cnt_b[a] = 2 * R + 1; covered[a] = false; }
      } else {
        int l = max(b0[a] - R, 0), hgh = min(b0[a] + R, c.nb[a] - 1);
        lo_b[a] = l; cnt_b[a] = hgh - l + 1;
        covered[a] = (l == 0 && hgh == c.nb[a] - 1);
      }
    }
    int cnt = 0;
    long long total = (long long)cnt_b[0] * cnt_b[1] * cnt_b[2];
    for (long long w = 0; w < total; ++w) {
      long long rem = w;
      long long flat = 0;
      int bb[3];   // window visited in C order (last axis fastest)
      for (int a = c.dim - 1; a >= 0; --a) {
        int off = (int)(rem % cnt_b[a]);
        rem /= cnt_b[a];
        int v = lo_b[a] + off;
        if (c.periodic[a]) { v %= c.nb[a]; if (v < 0) v += c.nb[a]; }
        bb[a] = v;
      }
      for (int a = 0; a < c.dim; ++a) flat = flat * c.nb[a] + bb[a];
      if (c.cells) {
        double d2 = 0.0;
        for (int a = 0; a < c.dim; ++a) {
          double dd = min_image(__dsub_rn(cell_centre(c, a, bb[a]), q[a]), c.periodic[a], c.L[a], c.halfL[a]);
          d2 = (a == 0) ? __dmul_rn(dd, dd) : __dadd_rn(d2, __dmul_rn(dd, dd));
        }
        topk_insert(bd, bi, cnt, K, d2, (int)flat);
      } else {
        for (int s = c.start[flat]; s < c.start[flat + 1]; ++s) {
          int id = c.sorted[s];
          double d2 = 0.0;
          for (int a = 0; a < c.dim; ++a) {
            double dd = min_image(__dsub_rn(c.xyz[(long long)a * c.N + id], q[a]), c.periodic[a], c.L[a], c.halfL[a]);
            d2 = (a == 0) ? __dmul_rn(dd, dd) : __dadd_rn(d2, __dmul_rn(dd, dd));
          }
          topk_insert(bd, bi, cnt, K, d2, id);
        }
      }
    }
    double guard = INFINITY;
    bool all_cov = true;
    for (int a = 0; a < c.dim; ++a) {
      if (covered[a]) continue;
      all_cov = false;
      double lo_edge = c.lo[a] + (b0[a] - R) * c.cs[a];
      double hi_edge = c.lo[a] + (b0[a] + R + 1) * c.cs[a];
      if (c.periodic[a] || b0[a] - R > 0) guard = fmin(guard, q[a] - lo_edge);
      if (c.periodic[a] || b0[a] + R + 1 < c.nb[a]) guard = fmin(guard, hi_edge - q[a]);
    }
    if (cnt == K && (all_cov || bd[K - 1] < guard * guard * (1.0 - 1e-12))) return true;
    if (all_cov) return false;
  }
}

// Basis of Eq. 16 (2D) or the complete 3D quadratic, in scaled offsets.
template <int DIM>
__device__ __forceinline__ void wls_basis(const double *xi, double *q) {
  if (DIM == 2) {
    q[0] = 1.0; q[1] = xi[0]; q[2] = xi[1];
    q[3] = 0.5 * xi[0] * xi[0]; q[4] = xi[0] * xi[1]; q[5] = 0.5 * xi[1] * xi[1];
  } else {
    q[0] = 1.0; q[1] = xi[0]; q[2] = xi[1]; q[3] = xi[2];
    q[4] = 0.5 * xi[0] * xi[0]; q[5] = xi[0] * xi[1]; q[6] = xi[0] * xi[2];
    q[7] = 0.5 * xi[1] * xi[1]; q[8] = xi[1] * xi[2]; q[9] = 0.5 * xi[2] * xi[2];
  }
}

struct WlsParams {
  int K;
  double eps, support_factor, c_dim;
  int nrows_out;      // 1 (value row) or DIM (derivative rows)
  int first_row;      // 0 or 1
  int lap_row;        // 1: one more row after them, the Laplacian (sum of the pure second-derivative rows)
};

// Given the neighbours of query q, write nrows_out rows (weights per neighbour) into w_out
// (w_out[r*K + k]). Returns false when C is not positive definite.
template <int DIM>
__device__ bool wls_rows(const KnnCtx &c, const double *q, const int *bi, const double *bd,
                         const WlsParams &P, double *w_out) {
  constexpr int m = (DIM == 2) ? 6 : 10;
  const int K = P.K;
  double r2max = bd[0];
  for (int k = 1; k < K; ++k) r2max = fmax(r2max, bd[k]);
  const double rK = sqrt(r2max);   // farthest stencil point (the K-th of a K-nearest stencil)
  const double hs = P.support_factor * (rK * P.c_dim);
  const double hs2 = hs * hs;
  double C[m][m];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) C[i][j] = 0.0;
  double xi_all[kMaxK][DIM];
  double w_all[kMaxK];
  for (int k = 0; k < K; ++k) {
    double xi[DIM];
    for (int a = 0; a < DIM; ++a) {
      double dd = min_image(__dsub_rn(point_coord(c, a, bi[k]), q[a]), c.periodic[a], c.L[a], c.halfL[a]);
      xi[a] = dd / hs;
      xi_all[k][a] = xi[a];
    }
    double w = (bd[k] <= hs2) ? exp(-P.eps * bd[k] / hs2) : 0.0;
    w_all[k] = w;
    double qv[m];
    wls_basis<DIM>(xi, qv);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= i; ++j) C[i][j] += w * qv[i] * qv[j];
  }
  // Cholesky C = L L^T (lower triangle in place)
  for (int j = 0; j < m; ++j) {
    double s = C[j][j];
    for (int k = 0; k < j; ++k) s -= C[j][k] * C[j][k];
    if (!(s > 1e-14 * C[0][0])) return false;
    double d = sqrt(s);
    C[j][j] = d;
    for (int i = j + 1; i < m; ++i) {
      double t = C[i][j];
      for (int k = 0; k < j; ++k) t -= C[i][k] * C[j][k];
      C[i][j] = t / d;
    }
  }
  // basis indices of the pure second derivatives (the 1/2 factors of the basis make their rows
  // the derivatives themselves)
  const int p0 = (DIM == 2) ? 3 : 4, p1 = (DIM == 2) ? 5 : 7, p2 = (DIM == 2) ? -1 : 9;
  for (int r = 0; r < P.nrows_out + (P.lap_row ? 1 : 0); ++r) {
    const bool lap = r == P.nrows_out;
    const int e = lap ? -1 : P.first_row + r;
    double y[m];
    // L z = rhs ; L^T y = z  (rhs: the unit vector e, or the sum of the pure second-derivative ones)
    for (int i = 0; i < m; ++i) {
      double t = lap ? ((i == p0 || i == p1 || i == p2) ? 1.0 : 0.0) : ((i == e) ? 1.0 : 0.0);
      for (int k = 0; k < i; ++k) t -= C[i][k] * y[k];
      y[i] = t / C[i][i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < m; ++k) t -= C[k][i] * y[k];
      y[i] = t / C[i][i];
    }
    const double scale = lap ? 1.0 / (hs * hs) : ((e == 0) ? 1.0 : 1.0 / hs);
    for (int k = 0; k < K; ++k) {
      double qv[m];
      wls_basis<DIM>(xi_all[k], qv);
      double dot = 0.0;
      for (int i = 0; i < m; ++i) dot += y[i] * qv[i];
      w_out[r * K + k] = w_all[k] * dot * scale;
    }
  }
  return true;
}

// Failure record: flags[0] ORs the kinds; flags[1..2] hold the smallest (query set, row) key
// so the host can name the first query that failed (set 0..2: faces of that axis, 3: nodes, 4: cells).
__device__ __forceinline__ void record_failure(unsigned int *flags, unsigned int kind, int set, long long row) {
  atomicOr(flags, kind);
  unsigned long long key = ((unsigned long long)set << 48) | (unsigned long long)row;
  atomicMin(reinterpret_cast<unsigned long long *>(flags + 2), key);
}

// FP64 weight (FP64 plans) and/or its FP32 (hi, lo) pair (mixed and FP32 plans).
__device__ __forceinline__ void split_store(double v, double *w64, float2 *w2, long long at) {
  if (w64) w64[at] = v;
  if (w2) {
    float hi = (float)v;
    w2[at] = make_float2(hi, (float)(v - (double)hi));
  }
}

// Value rows of the faces normal to `axis`.
template <int DIM>
__global__ void face_rows_kernel(KnnCtx c, WlsParams P, int axis, int nf_axis, int bc_lo_wall,
                                 int bc_hi_wall, int n_axis, long long rows, const double *glo,
                                 const double *gh, const int *gshape, int32_t *col, double *w64,
                                 float2 *w2, unsigned int *flags) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  // face multi-index (C order of the face array)
  int idx[3];
  long long rem = r;
  for (int a = DIM - 1; a >= 0; --a) {
    int extent = (a == axis) ? nf_axis : gshape[a];
    idx[a] = (int)(rem % extent);
    rem /= extent;
  }
  const int K = P.K;
  bool wall = (idx[axis] == 0 && bc_lo_wall) || (idx[axis] == n_axis && bc_hi_wall);
  if (wall) {
    for (int k = 0; k < K; ++k) {
      col[(long long)k * rows + r] = 0;
      split_store(0.0, w64, w2, (long long)k * rows + r);
    }
    return;
  }
  double q[3];
  for (int a = 0; a < DIM; ++a) {
    q[a] = (a == axis) ? __dadd_rn(glo[a], __dmul_rn((double)idx[a], gh[a]))
                       : __dadd_rn(glo[a], __dmul_rn((double)idx[a] + 0.5, gh[a]));
  }
  double bd[kMaxK];
  int bi[kMaxK];
  double w[kMaxK];
  bool ok = knn_query(c, q, K, bd, bi);
  if (!ok) record_failure(flags, FLAG_KNN_SHORT, axis, r);
  else if (!wls_rows<DIM>(c, q, bi, bd, P, w)) { ok = false; record_failure(flags, FLAG_WLS_SINGULAR, axis, r); }
  if (!ok) {
    for (int k = 0; k < K; ++k) { bi[k] = 0; w[k] = 0.0; }
  }
  for (int k = 0; k < K; ++k) {
    col[(long long)k * rows + r] = bi[k];
    split_store(w[k], w64, w2, (long long)k * rows + r);
  }
}

// Derivative rows of every pressure point over its K nearest nodes (the direct divergence of
// the source at the pressure points, §2.3): weights [DIM][K][points]. The points are
// lo + (i + off) h over the index box gshape: the cell centres (off = 1/2) or the vertex
// unknowns (off = index of the first unknown).
template <int DIM>
__global__ void cell_rows_kernel(KnnCtx c, WlsParams P, long long rows, const double *glo, const double *gh,
                                 const int *gshape, const double *goff, int32_t *col, double *w64, float2 *w2,
                                 unsigned int *flags) {
  long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  int idx[3];
  long long rem = r;
  for (int a = DIM - 1; a >= 0; --a) {
    idx[a] = (int)(rem % gshape[a]);
    rem /= gshape[a];
  }
  const int K = P.K;
  double q[3];
  for (int a = 0; a < DIM; ++a) q[a] = __dadd_rn(glo[a], __dmul_rn((double)idx[a] + goff[a], gh[a]));
  double bd[kMaxK];
  int bi[kMaxK];
  double w[DIM * kMaxK];
  bool ok = knn_query(c, q, K, bd, bi);
  if (!ok) record_failure(flags, FLAG_KNN_SHORT, 4, r);
  else if (!wls_rows<DIM>(c, q, bi, bd, P, w)) { ok = false; record_failure(flags, FLAG_WLS_SINGULAR, 4, r); }
  if (!ok) {
    for (int k = 0; k < K; ++k) bi[k] = 0;
    for (int k = 0; k < DIM * K; ++k) w[k] = 0.0;
  }
  for (int k = 0; k < K; ++k) {
    col[(long long)k * rows + r] = bi[k];
    for (int a = 0; a < DIM; ++a) split_store(w[a * K + k], w64, w2, ((long long)a * K + k) * rows + r);
  }
}

// Derivative rows of every node over the 3^DIM block of pressure points around it: along each
// axis the cell holding the node (on a vertex lattice: the nearest vertex) and its two
// neighbours, shifted inward at a non-periodic wall, wrapped on a periodic axis; listed in C
// order of the block offsets. Three distinct points per axis determine a quadratic exactly,
// which a K-nearest choice next to a 3D wall does not guarantee.
template <int DIM>
__global__ void node_rows_kernel(KnnCtx c, WlsParams P, const double *xyz, long long N,
                                 int32_t *col, double *D64, float2 *D2, unsigned int *flags) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  constexpr int KB = (DIM == 2) ? 9 : 27;
  double q[3];
  for (int a = 0; a < DIM; ++a) q[a] = xyz[(long long)a * N + i];
  int cells[3][3];
  for (int a = 0; a < DIM; ++a) {
    const double x = (q[a] - c.lo[a]) / c.h[a];
    const double t = c.off[a] == 0.0 ? floor(x + 0.5) : floor(x);
    int ci;
    if (c.periodic[a]) {
      ci = (int)t % c.nb[a];
      if (ci < 0) ci += c.nb[a];
    } else {
      ci = (int)fmax(0.0, fmin(t, (double)(c.nb[a] - 1)));
    }
    int st = ci - 1;
    if (!c.periodic[a]) st = max(0, min(st, c.nb[a] - 3));
    for (int o = 0; o < 3; ++o) {
      int v = st + o;
      if (c.periodic[a]) { v %= c.nb[a]; if (v < 0) v += c.nb[a]; }
      cells[a][o] = v;
    }
  }
  double bd[KB];
  int bi[KB];
  double w[DIM * KB];
  for (int k = 0; k < KB; ++k) {
    int rem = k, idx[3];
    for (int a = DIM - 1; a >= 0; --a) { idx[a] = cells[a][rem % 3]; rem /= 3; }
    long long flat = 0;
    double d2 = 0.0;
    for (int a = 0; a < DIM; ++a) {
      flat = flat * c.nb[a] + idx[a];
      double dd = min_image(__dsub_rn(cell_centre(c, a, idx[a]), q[a]), c.periodic[a], c.L[a], c.halfL[a]);
      d2 = (a == 0) ? __dmul_rn(dd, dd) : __dadd_rn(d2, __dmul_rn(dd, dd));
    }
    bd[k] = d2;
    bi[k] = (int)flat;
  }
  WlsParams PB = P;
  PB.K = KB;
  bool ok = wls_rows<DIM>(c, q, bi, bd, PB, w);
  if (!ok) {
    record_failure(flags, FLAG_WLS_SINGULAR, 3, i);
    for (int k = 0; k < DIM * KB; ++k) w[k] = 0.0;
  }
  for (int k = 0; k < KB; ++k) col[(long long)k * N + i] = bi[k];
  for (int a = 0; a < DIM; ++a)
    for (int k = 0; k < KB; ++k)
      split_store(w[a * KB + k], D64, D2, ((long long)a * KB + k) * N + i);
}

// ----------------------------------------------------------------------------- bucket sort
__global__ void bucket_count_kernel(const double *xyz, long long N, KnnCtx c, int *bid, int *count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  long long flat = 0;
  for (int a = 0; a < c.dim; ++a) {
    double t = floor((xyz[(long long)a * N + i] - c.lo[a]) / c.cs[a]);
    int b = (int)fmax(0.0, fmin(t, (double)(c.nb[a] - 1)));
    flat = flat * c.nb[a] + b;
  }
  bid[i] = (int)flat;
  atomicAdd(&count[flat], 1);
}

// Exclusive scan, three phases: per-block scan, scan of block sums, add.
__global__ void scan_block_kernel(const int *in, int *out, int *block_sums, long long n) {
  __shared__ int s[1024];
  long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  int v = (i < n) ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int t = (threadIdx.x >= (unsigned)off) ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == 1023) block_sums[blockIdx.x] = s[1023];
}

__global__ void scan_sums_kernel(int *sums, int nblocks) {
  // single thread: the number of blocks is small (<= a few thousand)
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  for (int b = 0; b < nblocks; ++b) { int v = sums[b]; sums[b] = acc; acc += v; }
  sums[nblocks] = acc;
}

__global__ void scan_add_kernel(int *out, const int *sums, long long n) {
  long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
}

__global__ void scatter_kernel(const int *bid, long long N, const int *start, int *cursor, int *sorted) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int b = bid[i];
  int pos = atomicAdd(&cursor[b], 1);
  sorted[start[b] + pos] = (int)i;
}

// Nodes sorted into a bucket grid over the box (about 4 nodes per bucket on average), for the
// K-nearest queries: fills nc (with the box and the bucket arrays) and owns the scratch.
struct NodeBuckets {
  int *bid = nullptr, *count = nullptr, *start = nullptr, *sums = nullptr, *sorted = nullptr;
  void release() {
    cudaFree(bid); cudaFree(count); cudaFree(start); cudaFree(sums); cudaFree(sorted);
    bid = count = start = sums = sorted = nullptr;
  }
};

static pc_status bucket_nodes(int d, const double *lo, const double *L, const int *periodic, const double *h,
                              const double *xyz, long long N, cudaStream_t st, KnnCtx &nc, NodeBuckets &b) {
  nc = KnnCtx{};
  nc.dim = d;
  double vol = 1.0;
  for (int a = 0; a < d; ++a) vol *= L[a];
  double cs = std::pow(4.0 * vol / (double)N, 1.0 / d);
  long long nbt = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < d) {
      int nb = (int)std::floor(L[a] / cs);
      if (nb < 1) nb = 1;
      if (nb > 4096) nb = 4096;
      nc.nb[a] = nb;
      nc.cs[a] = L[a] / nb;
      nc.lo[a] = lo[a];
      nc.L[a] = L[a];
      nc.halfL[a] = 0.5 * nc.L[a];
      nc.periodic[a] = periodic[a];
      nc.h[a] = h[a];
      nbt *= nb;
    } else {
      nc.nb[a] = 1;
      nc.cs[a] = 1.0;
    }
  }
  nc.xyz = xyz;
  nc.N = N;
  nc.cells = 0;
  long long nblk = (nbt + 1 + 1023) / 1024;   // scan covers nbt + 1 entries
  if (cudaMalloc(&b.bid, N * sizeof(int)) != cudaSuccess || cudaMalloc(&b.count, (nbt + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b.start, (nbt + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b.sums, (nblk + 1) * sizeof(int)) != cudaSuccess || cudaMalloc(&b.sorted, N * sizeof(int)) != cudaSuccess) {
    b.release();
    return fail(PC_ERR_OUT_OF_MEMORY, "setup scratch allocation failed");
  }
  cudaMemsetAsync(b.count, 0, (nbt + 1) * sizeof(int), st);
  bucket_count_kernel<<<grid_for(N, 256), 256, 0, st>>>(xyz, N, nc, b.bid, b.count);
  scan_block_kernel<<<(unsigned)nblk, 1024, 0, st>>>(b.count, b.start, b.sums, nbt + 1);
  scan_sums_kernel<<<1, 32, 0, st>>>(b.sums, (int)nblk);
  scan_add_kernel<<<(unsigned)nblk, 1024, 0, st>>>(b.start, b.sums, nbt + 1);
  cudaMemsetAsync(b.count, 0, (nbt + 1) * sizeof(int), st);
  scatter_kernel<<<grid_for(N, 256), 256, 0, st>>>(b.bid, N, b.start, b.count, b.sorted);
  nc.start = b.start;
  nc.sorted = b.sorted;
  return PC_OK;
}

pc_status build_rows(Plan *p, const double *xyz, cudaStream_t st) {
  const int d = p->dim;
  const long long N = p->N;
  KnnCtx nc{};
  NodeBuckets nb{};
  unsigned int *flags = nullptr;
  auto cleanup = [&]() {
    nb.release();
    cudaFree(flags);
  };
  {
    double L[3], lo[3], h[3];
    int per[3];
    for (int a = 0; a < 3; ++a) {
      L[a] = a < d ? p->ax[a].L : 1.0;
      lo[a] = p->lo[a];
      h[a] = p->h[a];
      per[a] = a < d ? (int)p->ax[a].periodic : 0;
    }
    pc_status bs = bucket_nodes(d, lo, L, per, h, xyz, N, st, nc, nb);
    if (bs != PC_OK) return bs;
  }
  if (cudaMalloc(&flags, 4 * sizeof(unsigned)) != cudaSuccess) {
    cleanup();
    return fail(PC_ERR_OUT_OF_MEMORY, "setup scratch allocation failed");
  }
  cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned), st);
  cudaMemsetAsync(flags + 2, 0xff, 2 * sizeof(unsigned), st);

  WlsParams P{};
  P.K = p->K;
  P.eps = p->eps;
  P.support_factor = p->support_factor;
  const double pi = 3.14159265358979323846;
  P.c_dim = (d == 2) ? std::sqrt(pi / p->K) : std::pow(4.0 * pi / (3.0 * p->K), 1.0 / 3.0);
  const bool mixed = p->precision != PC_PREC_FP64;

  double *glo = nullptr, *gh = nullptr, *goff = nullptr;
  int *gshape = nullptr;
  if (cudaMalloc(&glo, 3 * sizeof(double)) != cudaSuccess || cudaMalloc(&gh, 3 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&goff, 3 * sizeof(double)) != cudaSuccess || cudaMalloc(&gshape, 3 * sizeof(int)) != cudaSuccess) {
    cudaFree(glo); cudaFree(gh); cudaFree(goff);
    cleanup();
    return fail(PC_ERR_OUT_OF_MEMORY, "setup scratch allocation failed");
  }
  // the index box of the pressure points: cells, or the unknowns of a vertex grid (which has no
  // face rows, so the face kernels never see the vertex box)
  int hshape[3] = {(int)p->n[0], (int)p->n[1], (int)p->n[2]};
  double hoff[3] = {0.5, 0.5, 0.5};
  if (p->vertex)
    for (int a = 0; a < 3; ++a) {
      hshape[a] = p->nv[a];
      hoff[a] = (double)p->vj0[a];
    }
  cudaMemcpyAsync(glo, p->lo, 3 * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(gh, p->h, 3 * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(goff, hoff, 3 * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(gshape, hshape, 3 * sizeof(int), cudaMemcpyHostToDevice, st);

  P.nrows_out = 1;
  P.first_row = 0;
  for (int a = 0; a < d; ++a) {
    const AxisInfo &ax = p->ax[a];
    long long rows = p->nface_total[a];
    if (rows == 0) continue;   // a vertex grid has no faces
    int lo_wall = (!ax.periodic && ax.bc_lo == PC_BC_NEUMANN_WALL);
    int hi_wall = (!ax.periodic && ax.bc_hi == PC_BC_NEUMANN_WALL);
    if (d == 2)
      face_rows_kernel<2><<<grid_for(rows, 128), 128, 0, st>>>(nc, P, a, ax.nfaces, lo_wall, hi_wall, ax.n, rows, glo, gh,
                                                               gshape, p->fcol[a], p->fw64[a], mixed ? p->fw2[a] : nullptr, flags);
    else
      face_rows_kernel<3><<<grid_for(rows, 128), 128, 0, st>>>(nc, P, a, ax.nfaces, lo_wall, hi_wall, ax.n, rows, glo, gh,
                                                               gshape, p->fcol[a], p->fw64[a], mixed ? p->fw2[a] : nullptr, flags);
  }
  if (p->divmode == PC_DIV_WLS_DIRECT) {
    WlsParams Pc = P;
    Pc.nrows_out = d;
    Pc.first_row = 1;
    if (d == 2)
      cell_rows_kernel<2><<<grid_for(p->npts, 128), 128, 0, st>>>(nc, Pc, p->npts, glo, gh, gshape, goff, p->ccol,
                                                                  p->cD64, mixed ? p->cD2 : nullptr, flags);
    else
      cell_rows_kernel<3><<<grid_for(p->npts, 128), 128, 0, st>>>(nc, Pc, p->npts, glo, gh, gshape, goff, p->ccol,
                                                                  p->cD64, mixed ? p->cD2 : nullptr, flags);
  }
  // pressure points (cell centres, or the vertex lattice with its Dirichlet boundary vertices)
  // as points: bucket == point
  KnnCtx cc{};
  cc.dim = d;
  for (int a = 0; a < 3; ++a) {
    cc.nb[a] = (a < d) ? (p->vertex ? p->nf[a] : (int)p->n[a]) : 1;
    cc.cs[a] = (a < d) ? p->h[a] : 1.0;
    cc.lo[a] = p->lo[a];
    cc.h[a] = p->h[a];
    cc.off[a] = p->vertex ? 0.0 : 0.5;
    cc.L[a] = (double)p->n[a] * p->h[a];
    cc.halfL[a] = 0.5 * cc.L[a];
    cc.periodic[a] = (a < d) ? p->ax[a].periodic : 0;
  }
  cc.cells = 1;
  P.nrows_out = d;
  P.first_row = 1;
  P.c_dim = (d == 2) ? std::sqrt(pi / 9.0) : std::pow(4.0 * pi / (3.0 * 27.0), 1.0 / 3.0);
  if (d == 2)
    node_rows_kernel<2><<<grid_for(N, 128), 128, 0, st>>>(cc, P, xyz, N, p->ncol, p->nD64, mixed ? p->nD2 : nullptr, flags);
  else
    node_rows_kernel<3><<<grid_for(N, 128), 128, 0, st>>>(cc, P, xyz, N, p->ncol, p->nD64, mixed ? p->nD2 : nullptr, flags);
  cudaError_t e = cudaGetLastError();
  unsigned int hf[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  cudaFree(glo);
  cudaFree(gh);
  cudaFree(goff);
  cudaFree(gshape);
  if (e != cudaSuccess) return fail(PC_ERR_CUDA, "setup kernels failed: %s", cudaGetErrorString(e));
  if (hf[0] & (FLAG_WLS_SINGULAR | FLAG_KNN_SHORT)) {
    unsigned long long key = ((unsigned long long)hf[3] << 32) | hf[2];
    int set = (int)(key >> 48);
    long long row = (long long)(key & ((1ULL << 48) - 1));
    return fail(PC_ERR_WLS_SINGULAR, "WLS setup failed (%s%s); first failing query: %s %lld",
                (hf[0] & FLAG_KNN_SHORT) ? "fewer than K neighbours " : "",
                (hf[0] & FLAG_WLS_SINGULAR) ? "normal matrix not positive definite" : "",
                set < 3 ? (set == 0 ? "face row, axis 0," : (set == 1 ? "face row, axis 1," : "face row, axis 2,"))
                        : (set == 4 ? "cell row" : "node"),
                row);
  }
  return PC_OK;
}


// Rows of the meshless momentum operators (§2.2 at the nodes): for every node, its K nearest
// nodes (itself included, at distance 0), the first-derivative rows and the Laplacian row.
template <int DIM>
__global__ void momentum_rows_kernel(KnnCtx c, WlsParams P, const double *xyz, long long N, int32_t *col,
                                     double *w64, float2 *w2, unsigned int *flags) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int K = P.K;
  double q[3];
  for (int a = 0; a < DIM; ++a) q[a] = xyz[(long long)a * N + i];
  double bd[kMaxK];
  int bi[kMaxK];
  double w[(DIM + 1) * kMaxK];
  bool ok = knn_query(c, q, K, bd, bi);
  if (!ok) record_failure(flags, FLAG_KNN_SHORT, 5, i);
  else if (!wls_rows<DIM>(c, q, bi, bd, P, w)) { ok = false; record_failure(flags, FLAG_WLS_SINGULAR, 5, i); }
  if (!ok) {
    for (int k = 0; k < K; ++k) bi[k] = (int)i;
    for (int k = 0; k < (DIM + 1) * K; ++k) w[k] = 0.0;
  }
  for (int k = 0; k < K; ++k) {
    col[(long long)k * N + i] = bi[k];
    for (int r = 0; r <= DIM; ++r) split_store(w[r * K + k], w64, w2, ((long long)r * K + k) * N + i);
  }
}

pc_status build_momentum_rows(const Plan *p, const double *xyz, int K, int32_t *col, double *w64, float2 *w2,
                              cudaStream_t st) {
  const int d = p->dim;
  const long long N = p->N;
  KnnCtx nc{};
  NodeBuckets nb{};
  unsigned int *flags = nullptr;
  {
    double lo[3], h[3];
    for (int a = 0; a < 3; ++a) { lo[a] = p->lo[a]; h[a] = p->h[a]; }
    pc_status bs = bucket_nodes(d, lo, p->phys_L, p->phys_periodic, h, xyz, N, st, nc, nb);
    if (bs != PC_OK) return bs;
  }
  if (cudaMalloc(&flags, 4 * sizeof(unsigned)) != cudaSuccess) {
    nb.release();
    return fail(PC_ERR_OUT_OF_MEMORY, "setup scratch allocation failed");
  }
  cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned), st);
  cudaMemsetAsync(flags + 2, 0xff, 2 * sizeof(unsigned), st);
  WlsParams P{};
  P.K = K;
  P.eps = p->eps;
  P.support_factor = p->support_factor;
  const double pi = 3.14159265358979323846;
  P.c_dim = (d == 2) ? std::sqrt(pi / K) : std::pow(4.0 * pi / (3.0 * K), 1.0 / 3.0);
  P.first_row = 1;
  P.nrows_out = d;
  P.lap_row = 1;
  if (d == 2) momentum_rows_kernel<2><<<grid_for(N, 128), 128, 0, st>>>(nc, P, xyz, N, col, w64, w2, flags);
  else momentum_rows_kernel<3><<<grid_for(N, 128), 128, 0, st>>>(nc, P, xyz, N, col, w64, w2, flags);
  cudaError_t e = cudaGetLastError();
  unsigned int hf[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  nb.release();
  cudaFree(flags);
  if (e != cudaSuccess) return fail(PC_ERR_CUDA, "momentum row setup failed: %s", cudaGetErrorString(e));
  if (hf[0] & (FLAG_WLS_SINGULAR | FLAG_KNN_SHORT)) {
    unsigned long long key = ((unsigned long long)hf[3] << 32) | hf[2];
    return fail(PC_ERR_WLS_SINGULAR, "momentum rows: WLS setup failed at node %lld",
                (long long)(key & ((1ULL << 48) - 1)));
  }
  return PC_OK;
}

}  // namespace pc
