// The first fractional step around the pressure correction: the second-order Adams-Bashforth
// predictor of Eq. 3 (§2.1) on the node cloud, with the meshless operators of §2.2.
//
//   u* = u^n + (3/2) dt R^n - (1/2) dt R^{n-1},   R = -u . grad u + nu lap u + F,
//
// where R^{n-1} also carries -grad p^{n-1}. The gradient and Laplacian at a node come from the
// WLS rows over its K nearest nodes (build_momentum_rows). grad p^{n-1} at a fluid node is the
// gradient the last correction applied: u^n = u*^{n-1} - beta dt grad p^{n-1} (Eq. 18), so it is
// (u*^{n-1} - u^n) / (beta dt), from the u* this object kept. The first step (no R^{n-1}) is
// forward Euler. Boundary points take the prescribed velocity, virtual points zero (§2.3).
//
// One kernel per step, one node per thread: an HBM-bound gather of K columns, (d + 1) K weights
// and the K neighbour velocities, FP64 (FP64 plans) or compensated FP32 pairs (mixed and FP32
// plans, as in the transfer kernels).
#include <cmath>
#include <cstdio>

#include "numeric.cuh"
#include "pc.h"
#include "pc_internal.cuh"

struct pc_momentum {
  pc::Plan *plan = nullptr;
  int K = 0;
  double nu = 0.0, F[3] = {0.0, 0.0, 0.0};
  bool mixed = false;
  int32_t *col = nullptr;       // [K][N]
  double *w64 = nullptr;        // [dim + 1][K][N]: d/dx_0 .. d/dx_{d-1}, Laplacian (FP64 plans)
  float2 *w2 = nullptr;         //   the same as (hi, lo) pairs (mixed and FP32 plans)
  double *R_prev = nullptr;     // [dim][N] R^{n-1} without its pressure term
  double *us_prev = nullptr;    // [dim][N] u*^{n-1} as the correction received it
  int steps = 0;
  double dt = 0.0;
};

namespace pc {
namespace {

bool device_ptr(const void *ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename VT>
__device__ __forceinline__ double vload(const VT *p, long long i) { return (double)p[i]; }

// KC > 0: the neighbour count is a compile-time constant, the loop is unrolled and every column
// and weight load is issued before the dependent gathers (as in the transfer kernels).
template <typename VT, int DIM, bool MIXED, int KC>
__global__ void ab2_predict_kernel(int N, int Kr, const int32_t *__restrict__ col, const double *__restrict__ W,
                                   const float2 *__restrict__ W2, const uint8_t *__restrict__ type,
                                   const VT *__restrict__ u, const VT *__restrict__ ub, double dt, double inv_bdt,
                                   double nu, double F0, double F1, double F2, int first, double *R_prev,
                                   double *us_prev, VT *__restrict__ us) {
  const int K = KC > 0 ? KC : Kr;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint8_t t = type[i];
  if (t != PC_NODE_FLUID) {   // boundary points: prescribed velocity; virtual points: 0
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const long long at = (long long)a * N + i;
      const VT v = (t == PC_NODE_BOUNDARY && ub) ? ub[at] : (VT)0;
      us[at] = v;
      us_prev[at] = (double)v;
      R_prev[at] = 0.0;
    }
    return;
  }
  // acc[a][r]: row r (d/dx_r for r < DIM, the Laplacian for r = DIM) applied to u_a
  double g[DIM][DIM + 1];
  if (MIXED) {
    DF acc[DIM][DIM + 1];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int r = 0; r <= DIM; ++r) acc[a][r] = DF{0.f, 0.f};
#pragma unroll (KC > 0 ? KC : 4)
    for (int k = 0; k < K; ++k) {
      const int j = __ldcs(col + (long long)k * N + i);
      float2 w[DIM + 1];
#pragma unroll
      for (int r = 0; r <= DIM; ++r) w[r] = __ldcs(W2 + ((long long)r * K + k) * N + i);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const float2 ua = as_pair(u[(long long)a * N + j]);
#pragma unroll
        for (int r = 0; r <= DIM; ++r) df_acc(acc[a][r], w[r], ua);
      }
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int r = 0; r <= DIM; ++r) g[a][r] = df_value(acc[a][r]);
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int r = 0; r <= DIM; ++r) g[a][r] = 0.0;
#pragma unroll (KC > 0 ? KC : 4)
    for (int k = 0; k < K; ++k) {
      const int j = __ldcs(col + (long long)k * N + i);
      double w[DIM + 1];
#pragma unroll
      for (int r = 0; r <= DIM; ++r) w[r] = __ldcs(W + ((long long)r * K + k) * N + i);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double ua = vload(u, (long long)a * N + j);
#pragma unroll
        for (int r = 0; r <= DIM; ++r) g[a][r] = fma(w[r], ua, g[a][r]);
      }
    }
  }
  double ui[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) ui[a] = vload(u, (long long)a * N + i);
  const double F[3] = {F0, F1, F2};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double adv = 0.0;
#pragma unroll
    for (int b = 0; b < DIM; ++b) adv = fma(ui[b], g[a][b], adv);
    const double R = -adv + nu * g[a][DIM] + F[a];
    const long long at = (long long)a * N + i;
    double Rold = R, gp = 0.0;
    if (!first) {
      Rold = R_prev[at];
      gp = (us_prev[at] - ui[a]) * inv_bdt;
    }
    const VT v = (VT)(ui[a] + dt * (1.5 * R - 0.5 * (Rold - gp)));
    us[at] = v;
    us_prev[at] = (double)v;
    R_prev[at] = R;
  }
}

template <typename VT>
void launch_predict(pc_momentum *m, double dt, const void *u, const void *ub, void *us, cudaStream_t st) {
  const Plan *p = m->plan;
  const int N = (int)p->N, T = 256, G = grid_for(N, T);
  const double inv_bdt = 1.0 / (p->beta * dt);
  const int first = m->steps == 0;
  const VT *uu = static_cast<const VT *>(u), *bb = static_cast<const VT *>(ub);
  VT *oo = static_cast<VT *>(us);
#define PC_PREDICT(D, MX, KC)                                                                                   \
  ab2_predict_kernel<VT, D, MX, KC><<<G, T, 0, st>>>(N, m->K, m->col, m->w64, m->w2, p->ntype, uu, bb, dt, inv_bdt, \
                                                     m->nu, m->F[0], m->F[1], m->F[2], first, m->R_prev, m->us_prev, oo)
  if (p->dim == 2) {
    if (m->K == 12) {
      if (m->mixed) PC_PREDICT(2, true, 12);
      else PC_PREDICT(2, false, 12);
    } else {
      if (m->mixed) PC_PREDICT(2, true, 0);
      else PC_PREDICT(2, false, 0);
    }
  } else {
    if (m->K == 27) {
      if (m->mixed) PC_PREDICT(3, true, 27);
      else PC_PREDICT(3, false, 27);
    } else {
      if (m->mixed) PC_PREDICT(3, true, 0);
      else PC_PREDICT(3, false, 0);
    }
  }
#undef PC_PREDICT
}

void release(pc_momentum *m) {
  cudaFree(m->col);
  cudaFree(m->w64);
  cudaFree(m->w2);
  cudaFree(m->R_prev);
  cudaFree(m->us_prev);
  delete m;
}

}  // namespace
}  // namespace pc

extern "C" pc_status pc_momentum_create(pc_plan *plan, const double *node_xyz, int knn, double nu,
                                        const double *body_force, void *cuda_stream, pc_momentum **out) {
  using namespace pc;
  Plan *p = reinterpret_cast<Plan *>(plan);
  if (!p || !node_xyz || !out) return fail(PC_ERR_INVALID_ARG, "plan, node_xyz and out are required");
  *out = nullptr;
  if (p->grid_only) return fail(PC_ERR_INVALID_ARG, "a grid-only plan has no nodes");
  const int d = p->dim, kmin = d == 2 ? 6 : 10;
  if (knn < kmin || knn > kMaxK || knn > p->N) return fail(PC_ERR_INVALID_ARG, "knn must be in [%d, %d] and <= N", kmin, kMaxK);
  if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(PC_ERR_INVALID_ARG, "nu must be finite and >= 0");
  if (body_force)
    for (int a = 0; a < d; ++a)
      if (!std::isfinite(body_force[a])) return fail(PC_ERR_INVALID_ARG, "body_force must be finite");
  if (cudaSetDevice(p->device) != cudaSuccess) return fail(PC_ERR_CUDA, "cannot select device %d", p->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  pc_momentum *m = new pc_momentum();
  m->plan = p;
  m->K = knn;
  m->nu = nu;
  for (int a = 0; a < d; ++a) m->F[a] = body_force ? body_force[a] : 0.0;
  m->mixed = p->precision != PC_PREC_FP64;
  const long long N = p->N, K = knn;
  const size_t nw = (size_t)(d + 1) * K * N;
  bool ok = cudaMalloc(&m->col, K * N * sizeof(int32_t)) == cudaSuccess &&
            cudaMalloc(&m->R_prev, (size_t)d * N * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&m->us_prev, (size_t)d * N * sizeof(double)) == cudaSuccess &&
            (m->mixed ? cudaMalloc(&m->w2, nw * sizeof(float2)) : cudaMalloc(&m->w64, nw * sizeof(double))) == cudaSuccess;
  double *xyz = nullptr;
  const bool host = !device_ptr(node_xyz);
  if (ok && host) ok = cudaMalloc(&xyz, (size_t)d * N * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFree(xyz);
    release(m);
    return fail(PC_ERR_OUT_OF_MEMORY, "momentum buffers: device allocation failed");
  }
  if (host && cudaMemcpyAsync(xyz, node_xyz, (size_t)d * N * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaFree(xyz);
    release(m);
    return fail(PC_ERR_CUDA, "copy of node coordinates failed");
  }
  pc_status s = build_momentum_rows(p, host ? xyz : node_xyz, knn, m->col, m->w64, m->w2, st);
  cudaFree(xyz);
  if (s != PC_OK) {
    release(m);
    return s;
  }
  *out = m;
  return PC_OK;
}

extern "C" pc_status pc_momentum_predict(pc_momentum *m, double dt, const void *u_n, const void *u_boundary,
                                         void *u_star, void *cuda_stream) {
  using namespace pc;
  if (!m || !u_n || !u_star) return fail(PC_ERR_INVALID_ARG, "momentum, u_n and u_star are required");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(PC_ERR_INVALID_ARG, "dt must be positive and finite");
  if (m->steps > 0 && dt != m->dt)
    return fail(PC_ERR_INVALID_ARG, "dt changed within an AB2 run (%g, was %g): call pc_momentum_reset", dt, m->dt);
  const Plan *p = m->plan;
  if (cudaSetDevice(p->device) != cudaSuccess) return fail(PC_ERR_CUDA, "cannot select device %d", p->device);
  if (!device_ptr(u_n) || !device_ptr(u_star) || (u_boundary && !device_ptr(u_boundary)))
    return fail(PC_ERR_INVALID_ARG, "pc_momentum_predict takes device pointers only");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (p->vdtype == PC_DTYPE_F64) launch_predict<double>(m, dt, u_n, u_boundary, u_star, st);
  else launch_predict<float>(m, dt, u_n, u_boundary, u_star, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PC_ERR_CUDA, "predictor launch failed: %s", cudaGetErrorString(e));
  m->steps++;
  m->dt = dt;
  return PC_OK;
}

extern "C" pc_status pc_momentum_reset(pc_momentum *m) {
  if (!m) return pc::fail(PC_ERR_INVALID_ARG, "momentum is NULL");
  m->steps = 0;
  return PC_OK;
}

extern "C" pc_status pc_momentum_destroy(pc_momentum *m) {
  if (!m) return PC_OK;
  cudaSetDevice(m->plan->device);
  pc::release(m);
  return PC_OK;
}
