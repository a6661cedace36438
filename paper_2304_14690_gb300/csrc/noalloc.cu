// Allocation-free Poisson solve: pc_solve_poisson_static.
//
// Some callers cannot allocate device memory at the point where they need a solve: code that
// runs under a custom allocator or a memory pool that owns every byte of the device, code inside
// a host callback or a library hook where cudaMalloc would synchronise the device or is simply
// forbidden, and embedded deployments that size device memory once at start-up. For them this
// entry point solves L_h p = s in FP64 with the same transform passes as pc_solve_poisson, but
// takes its whole workspace (transform buffer, twiddle and eigenvalue tables, reduction scratch)
// from one file-scope __device__ array of fixed size instead of a plan. The array exists on every
// device that loads the library, from load until exit.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fft.cuh"
#include "pc_internal.cuh"

namespace pc {

// Largest grid the static workspace holds (cells), and the workspace itself (doubles).
constexpr long long kStaticMaxCells = 1LL << 19;
constexpr long long kStaticDoubles = 1LL << 20;   // 8 MiB
static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
static void *g_static_ptr[kMaxDevices] = {nullptr};
static std::mutex g_static_mutex;

// Device address of the workspace on the current device; the first call per device resolves it
// with cudaGetSymbolAddress, zeroes it and sets the kernels' shared-memory limits.
static pc_status static_scratch(double **out) {
  int dev = -1;
  PC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PC_ERR_UNSUPPORTED, "device id %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(PC_ERR_CUDA, "cudaGetSymbolAddress of the static workspace failed: %s", cudaGetErrorString(e));
    PC_CUDA_TRY(cudaMemset(ptr, 0, sizeof(double) * kStaticDoubles));
    PC_TRY(prepare_kernels());
    g_static_ptr[dev] = ptr;
  }
  *out = static_cast<double *>(g_static_ptr[dev]);
  return PC_OK;
}

// Twiddle and eigenvalue tables of one axis, computed on the device (sincospi of rational
// multiples of pi), in the layout of AxisInfo.
__global__ void static_axis_tables(int n, int M, int kind, double h, double2 *tw, double *lam) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ntw = tw_total(M);
  if (t >= ntw + n) return;
  if (t < ntw) {
    double x;
    if (t < M) x = -2.0 * t / M;
    else if (t < tw_quarter(M)) x = -2.0 * (t - M) / n;
    else if (t < tw_dct4pre(M)) x = -(double)(t - tw_quarter(M)) / (2.0 * n);
    else if (t < tw_dct4post(M)) x = -(4.0 * (t - tw_dct4pre(M)) + 1.0) / (4.0 * n);
    else x = -(double)(t - tw_dct4post(M)) / n;
    double sv, cv;
    sincospi(x, &sv, &cv);
    tw[t] = make_double2(cv, sv);
    return;
  }
  const int m = t - ntw;
  double x;
  switch (kind) {
    case KIND_PP: {
      int w = (m == 0) ? 0 : (m == 1 ? n / 2 : m / 2);
      x = (double)w / n;
      break;
    }
    case KIND_NN: x = m / (2.0 * n); break;
    case KIND_DD: x = (m + 1.0) / (2.0 * n); break;
    default: x = (2.0 * m + 1.0) / (4.0 * n); break;
  }
  const double sv = sinpi(x);
  lam[m] = (-4.0 / (h * h)) * sv * sv;
}

bool axis_length_supported(int n);

}  // namespace pc

extern "C" pc_status pc_solve_poisson_static(int dim, const int64_t *n, const double *h, const int *bc_lo,
                                             const int *bc_hi, int gauge, const double *s, double *p_out,
                                             void *cuda_stream) {
  using namespace pc;
  if (dim != 2 && dim != 3) return fail(PC_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (!n || !h || !bc_lo || !bc_hi || !s || !p_out) return fail(PC_ERR_INVALID_ARG, "NULL argument");
  if (gauge != 0 && gauge != 1) return fail(PC_ERR_INVALID_ARG, "gauge must be 0 or 1");
  long long ncells = 1;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 4 || n[a] > 4096 || !axis_length_supported((int)n[a]))
      return fail(PC_ERR_UNSUPPORTED, "n[%d] = %lld: cells per axis must be even, >= 4, with n/2 = 2^a 3^b 5^c",
                  a, (long long)n[a]);
    if (!(h[a] > 0) || !std::isfinite(h[a])) return fail(PC_ERR_INVALID_ARG, "h[%d] invalid", a);
    if (bc_lo[a] < 0 || bc_lo[a] > 3 || bc_hi[a] < 0 || bc_hi[a] > 3)
      return fail(PC_ERR_INVALID_ARG, "bad boundary kind on axis %d", a);
    if ((bc_lo[a] == PC_BC_PERIODIC) != (bc_hi[a] == PC_BC_PERIODIC))
      return fail(PC_ERR_INVALID_ARG, "periodic must pair with periodic (axis %d)", a);
    ncells *= n[a];
  }
  if (ncells > kStaticMaxCells)
    return fail(PC_ERR_BUDGET, "grid of %lld cells exceeds the static workspace limit of %lld cells",
                ncells, kStaticMaxCells);
  int cur = -1;
  PC_CUDA_TRY(cudaGetDevice(&cur));
  for (const void *ptr : {(const void *)s, (const void *)p_out}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
        !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return fail(PC_ERR_INVALID_ARG, "s and p_out must be device pointers");
    }
    // the kernels run on the current device with its copy of the workspace
    if (at.type == cudaMemoryTypeDevice && at.device != cur)
      return fail(PC_ERR_INVALID_ARG, "s and p_out live on device %d, the current device is %d", at.device, cur);
  }
  double *ws = nullptr;
  PC_TRY(static_scratch(&ws));
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // A plan description on the stack whose every device buffer lies in the static workspace.
  Plan pl;
  pl.dim = dim;
  pl.precision = PC_PREC_FP64;
  pl.gauge = gauge;
  pl.ncells = ncells;
  pl.singular = true;
  long long off = 0;
  pl.work64 = ws + off;
  off += ncells;
  for (int a = 0; a < 3; ++a) {
    pl.n[a] = a < dim ? n[a] : 1;
    pl.h[a] = a < dim ? h[a] : 1.0;
    pl.bc_lo[a] = a < dim ? bc_lo[a] : 0;
    pl.bc_hi[a] = a < dim ? bc_hi[a] : 0;
  }
  for (int a = 0; a < dim; ++a) {
    AxisInfo &ax = pl.ax[a];
    ax.n = (int)n[a];
    ax.M = ax.n / 2;
    ax.h = h[a];
    ax.L = (double)n[a] * h[a];
    ax.periodic = bc_lo[a] == PC_BC_PERIODIC;
    ax.nfaces = ax.periodic ? ax.n : ax.n + 1;
    ax.bc_lo = bc_lo[a];
    ax.bc_hi = bc_hi[a];
    const bool nlo = bc_lo[a] != PC_BC_DIRICHLET, nhi = bc_hi[a] != PC_BC_DIRICHLET;
    ax.kind = ax.periodic ? KIND_PP : (nlo && nhi) ? KIND_NN : (!nlo && !nhi) ? KIND_DD : (nlo ? KIND_ND : KIND_DN);
    if (!nlo || !nhi) pl.singular = false;
    ax.tw64 = reinterpret_cast<double2 *>(ws + off);
    off += 2LL * tw_total(ax.M);
    ax.lam64 = ws + off;
    off += ax.n;
  }
  off = (off + 31) & ~31LL;
  pl.dstats = reinterpret_cast<DevStats *>(ws + off);
  off += (sizeof(DevStats) + 7) / 8 + 32;
  const long long last = pl.n[dim - 1];
  const long long cells_launch = ((last + 255) / 256) * (ncells / last);
  const long long flat_launch = (ncells + 255) / 256;
  pl.partials = ws + off;
  off += 2 * (cells_launch > flat_launch ? cells_launch : flat_launch) + 64;
  pl.counters = reinterpret_cast<unsigned int *>(ws + off);
  off += 8;
  if (off > kStaticDoubles)
    return fail(PC_ERR_BUDGET, "grid needs %lld workspace doubles, the static workspace has %lld", off,
                kStaticDoubles);

  for (int a = 0; a < dim; ++a) {
    const AxisInfo &ax = pl.ax[a];
    const int total = tw_total(ax.M) + ax.n;
    static_axis_tables<<<(total + 255) / 256, 256, 0, st>>>(ax.n, ax.M, ax.kind, ax.h, ax.tw64, ax.lam64);
  }
  // Statistics and the reduction counters start at zero on every call: a completed reduction
  // leaves its counter at zero, but a call cut short (a failed launch) may not have.
  PC_CUDA_TRY(cudaMemsetAsync(pl.dstats, 0, sizeof(DevStats), st));
  PC_CUDA_TRY(cudaMemsetAsync(pl.counters, 0, 8 * sizeof(double), st));
  PC_CUDA_TRY(cudaGetLastError());
  return solve_grid_device(&pl, s, p_out, st);
}
