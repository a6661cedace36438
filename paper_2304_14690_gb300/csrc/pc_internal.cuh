// Internal definitions of libpc: plan layout, error plumbing, small device helpers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pc.h"

namespace pc {

// Transform kind of one axis, from its boundary pair (§2.3: the transform follows the grid
// type and the boundary conditions).
// Transform kind of an axis: its boundary pair on the cell grid (0-4), or on the vertex grid
// (5-8; a vertex P-P axis is KIND_PP): DCT-I, DST-I and the two quarter-wave bases.
enum AxisKind { KIND_PP = 0, KIND_NN = 1, KIND_DD = 2, KIND_ND = 3, KIND_DN = 4,
                KIND_VNN = 5, KIND_VDD = 6, KIND_VND = 7, KIND_VDN = 8 };

constexpr int kMaxRadices = 24;
constexpr int kMaxK = 32;
// Largest row count (cells, faces per axis, nodes) the kernels index with 32-bit row numbers.
constexpr long long kMaxRows = (1LL << 31) - (1LL << 16);
constexpr int kMaxRefine = 8;

// Device-side status word values (written by kernels, read at the next sync point).
enum DeviceFlag { FLAG_WLS_SINGULAR = 1, FLAG_KNN_SHORT = 2, FLAG_NONFINITE = 4 };

struct AxisInfo {
  int kind = 0;
  int n = 0;        // pressure points along the axis: cells, or vertex unknowns
  int M = 0;        // complex FFT length: n/2 (cell kinds, quarter-wave vertex kinds), the
                    // vertex cells m for DCT-I (n = m + 1) and DST-I (n = m - 1)
  // Slots per thread of the transform passes along this axis, per precision (powers of two):
  // they fix the threads per line and the radix schedule (see build_pass), chosen when the
  // plan is built and shared by single and batched calls.
  // slots32 = 0: the lean FP32 pass of the length where it has one (lean_pass.cuh), else 4
  int slots32 = 0, slots64 = 2;
  int ctas32 = 2, ctas64 = 2;    // CTAs per SM the single-problem passes aim for (tile lines)
  double h = 0.0;
  double L = 0.0;   // n * h
  bool periodic = false;
  int nfaces = 0;   // faces normal to this axis along it (n or n+1)
  int bc_lo = 0, bc_hi = 0;
  // Twiddle tables, one buffer per precision: [0,M) e^{-2 pi i k/M}; [M, 2M+1) post/pre
  // twiddle of the real-to-real wrapper (kind dependent); [2M+1, 3M+1) DCT-IV pre twiddle.
  double2 *tw64 = nullptr;
  float2 *tw32 = nullptr;
  double *lam64 = nullptr;   // eigenvalue per spectral index (n entries)
  float *lam32 = nullptr;
};

// Per-call device statistics (mirrors pc_stats fields filled on the device).
struct DevStats {
  double sum_s;            // sum of the source over cells
  double sum_s2;           // sum of squares
  double res2[kMaxRefine + 1];
  double sum_p;            // sum of p before the gauge
  double corner_p;
  double max_div;
  double max_u;
  double mean_s;           // sum_s / ncells, written by the reducing block
  double shift;            // gauge constant, written by the reducing block
  double ib_diff;          // IB-force iteration: sum over IB nodes of |f_new - f_old|^2
  double ib_prev;          //   and of |f_old|^2
  unsigned int flags;
  unsigned int pad;
  // stopping rule of the refinement (MIXED with refine_tol > 0): max norms of the residual after
  // k sweeps and of the source, FP32, reduced with order-independent atomic maxima of their bits
  float rmax[kMaxRefine + 1];
  float smax;
};

// The refinement's stopping rule on the stored max norms: residual k (after k sweeps) ends the
// refinement when ||r_k|| <= tol ||s||, or, from k = 2, when ||r_k|| > 16 (||r_1|| / ||r_0||)
// ||r_{k-1}||: the residual no longer falls at the rate of a sweep, it has reached the rounding
// floor of its own evaluation. FP32 operations in a fixed order (no fused multiply-add is
// possible), so the device kernels and the host report take the same decision.
__host__ __device__ inline bool refine_stop_at(const float *rmax, float smax, int k, float tol) {
  const float rk = rmax[k];
  if (rk <= tol * smax) return true;
  if (k >= 2 && rmax[0] > 0.0f) {
    const float rho = rmax[1] / rmax[0];
    const float bound = (16.0f * rho) * rmax[k - 1];
    if (rk > bound) return true;
  }
  return false;
}
#ifdef __CUDACC__
// On the device: whether a residual before sweep j already ended the refinement (the kernels of
// sweep j, its solve and its residual, then do nothing). Read past L1: written by earlier kernels.
// The same operations as refine_stop_at applied to k = 0, 1, ..., j - 1. Every norm is loaded
// up front (one round trip to L2, not one per residual), and the loops are unrolled over
// constant indices so the values stay in registers (no local memory in the kernels calling it).
__device__ __forceinline__ bool refine_stopped_before(const DevStats *st, int j, float tol) {
  if (j <= 0) return false;
  float r[kMaxRefine + 1];
#pragma unroll
  for (int k = 0; k <= kMaxRefine; ++k) r[k] = (k < j) ? __ldcg(&st->rmax[k]) : 0.0f;
  const float bound_tol = tol * __ldcg(&st->smax);
  bool stop = false;
#pragma unroll
  for (int k = 0; k <= kMaxRefine; ++k) {
    if (k < j) {
      if (r[k] <= bound_tol) stop = true;
      if (k >= 2 && r[0] > 0.0f) {
        const float rho = r[1] / r[0];
        const float bound = (16.0f * rho) * r[k - 1];
        if (r[k] > bound) stop = true;
      }
    }
  }
  return stop;
}
#endif

// A pass or residual of refinement sweep j under the stopping rule: it does nothing once
// refine_stopped_before(st, j, tol). st == nullptr: no rule.
struct RefineGate {
  const DevStats *st;
  int j;
  float tol;
};

// Per-call event record of the optional profiler: segment i (between events i and i+1) belongs
// to phase tag[i].
constexpr int kProfEvents = 48;
constexpr int kProfSlots = 256;
struct ProfSlot {
  cudaEvent_t ev[kProfEvents];
  int tag[kProfEvents];
  int n = 0;
};

// One instantiated CUDA graph of a pc_project call, keyed by its arguments. Its event-record
// nodes (phase boundaries) are re-pointed to a profiler slot's events when profiling is on.
constexpr int kGraphCache = 4;
struct GraphEntry {
  const void *u = nullptr, *f = nullptr;
  void *p = nullptr, *uo = nullptr, *fo = nullptr;
  double dt = 0.0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nev = 0;
  cudaGraphNode_t evnode[kProfEvents];
  int tag[kProfEvents];
  long long launches = 0;
  unsigned long long stamp = 0;
  bool prof = false;      // captured with the profiler's event-record nodes
  int kind = 0;           // 0: pc_project (all the keys above); 1: pc_solve_poisson (u = s, p)
};

// IB-force iteration (pc_project_ib): the device-side state of one time step's loop, written by
// the last block of each pass's stopping-rule reduction, and the instantiated CUDA graph that
// runs the whole loop (a while-conditional node around the later passes).
constexpr int kIbMaxIters = 1000;
struct IbCtl {
  int it;                      // passes done
  int conv;                    // stopping rule met by the last pass
  int body;                    // executions of the loop graph's body (safety bound)
  int pad;
  double diff, prev;           // last pass: mean |f_new - f_old|^2 and mean |f_old|^2 (IB nodes)
  double hist[2 * kIbMaxIters];
};
struct IbGraph {
  const void *u = nullptr, *f = nullptr;
  void *p = nullptr, *uo = nullptr, *fo = nullptr;
  double dt = 0.0, tol = 0.0;
  int max_iters = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long l_first = 0, l_body = 0, l_final = 0;   // kernels per segment (launch counts)
};

struct Plan {
  int device = 0;
  int dim = 2;
  int64_t n[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, h[3] = {1, 1, 1};
  int bc_lo[3] = {0, 0, 0}, bc_hi[3] = {0, 0, 0};
  int64_t N = 0;
  int K = 12;                  // neighbours of a face (transfer) stencil
  int Kg = 9;                  // cells of a node (gradient) stencil: 3^dim
  double eps = 6.3, support_factor = 3.0, beta = 1.5;
  int precision = PC_PREC_FP64;
  int refine_iters = 2;        // MIXED: largest number of refinement sweeps
  double refine_tol = 0.0;     // MIXED: stopping rule tolerance (<= 0: refine_iters sweeps, no rule)
  int gauge = 0;
  int vdtype = PC_DTYPE_F64;
  bool singular = false;

  AxisInfo ax[3];
  int64_t ncells = 0;
  int64_t nface_total[3] = {0, 0, 0};

  // WLS rows, neighbour-rank major: entry k of row r at k*rows + r.
  int32_t *fcol[3] = {nullptr, nullptr, nullptr};
  double *fw64[3] = {nullptr, nullptr, nullptr};
  float2 *fw2[3] = {nullptr, nullptr, nullptr};   // (hi, lo) FP32 split of fw64 (mixed)
  int32_t *ncol = nullptr;     // [Kg][N] cell linear index
  double *nD64 = nullptr;      // [dim][Kg][N]
  float2 *nD2 = nullptr;       // (hi, lo) FP32 split of nD64 (mixed)
  uint8_t *ntype = nullptr;    // [N]

  // Workspace (allocated once; pc_project allocates nothing).
  double *U64[3] = {nullptr, nullptr, nullptr};  // face fluxes
  double *s64 = nullptr;       // source
  double *p64 = nullptr;       // pressure (refined iterate)
  double *work64 = nullptr;    // FP64 transform workspace (cells)
  float *work32 = nullptr;     // FP32 transform workspace (cells)
  float2 *p2 = nullptr;                   // split pressure for the compensated gradient
  float2 *u2 = nullptr;                   // split u~ = u* + dt f for the compensated transfer
  double *ut64 = nullptr;                 // u~ in FP64 (FP64 path)
  DevStats *dstats = nullptr;
  double *partials = nullptr;      // per-block partial sums of the deterministic reductions
  unsigned int *counters = nullptr;  // completion counters of those reductions (kept at zero)
  // Staging for host pointers passed to pc_project.
  void *stage_u = nullptr, *stage_f = nullptr, *stage_uo = nullptr, *stage_fo = nullptr;
  // copy stream and events of the host-array path (results copied back while kernels run)
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev[3] = {nullptr, nullptr, nullptr};
  double *stage_p = nullptr, *stage_s = nullptr;
  // IB-force iteration (pc_project_ib), built on its first call: the boundary/virtual nodes,
  // per axis the faces whose value row reaches one of them (the only fluxes that change after
  // the first pass), and two compact force iterates [dim][nib] of velocity_dtype.
  int64_t nib = -1;
  int32_t *ib_idx = nullptr;
  int32_t *ib_face[3] = {nullptr, nullptr, nullptr};
  int64_t nib_face[3] = {0, 0, 0};
  void *ib_f[2] = {nullptr, nullptr};   // [0] previous iterate, [1] current/new iterate
  IbCtl *ib_ctl = nullptr;
  cudaStream_t ib_body_stream = nullptr;
  IbGraph ib_graph;
  size_t bytes = 0;
  void *allocs[64];
  int nallocs = 0;
  // Clones (pc_plan_clone): a clone borrows the rows, node types and axis tables of its root
  // and owns its workspace; a root with live clones is not destroyed.
  struct Plan *root = nullptr;
  int clones = 0;
  // CUDA graphs of pc_project (on by default for device pointers without statistics)
  bool graphs_on = true;
  int eigen = PC_EIG_FD;       // pc_eigenvalues of the transform solve
  uint8_t *rhs_mask = nullptr; // pc_plan_set_rhs_mask: plan copy of the mask (cells)
  int divmode = PC_DIV_FACES;  // pc_divergence
  // grid-only plans (pc_grid_plan_create): no nodes, only the grid solve. A vertex grid is
  // solved as the periodic cell grid of its symmetric extension, held by the plan's axes.
  bool grid_only = false;
  bool vertex = false;
  bool problem_singular = true;  // the vertex problem (not its extension) has a zero mode
  int vkind[3] = {0, 0, 0};      // per axis: 0 P-P, 1 N-N, 2 D-D, 3 N-D, 4 D-N
  int vn[3] = {1, 1, 1};         // cells of the vertex grid per axis
  int nv[3] = {1, 1, 1};         // unknowns per axis
  long long nvtot = 0;
  int vj0[3] = {0, 0, 0};        // lattice index of the first unknown per axis
  int nf[3] = {1, 1, 1};         // lattice vertices per axis (n periodic, else n + 1)
  long long nftot = 0;
  long long npts = 0;            // pressure points with direct-divergence rows (cells or unknowns)
  double phys_L[3] = {1.0, 1.0, 1.0};   // the physical box (a vertex plan's axes hold the extension)
  int phys_periodic[3] = {0, 0, 0};
  int32_t *ccol = nullptr;     // direct divergence: [K][cells] node index
  double *cD64 = nullptr;      //   [dim][K][cells] derivative-row weights (FP64 plans)
  float2 *cD2 = nullptr;       //   (hi, lo) pairs (mixed and FP32 plans)
  bool rhs_mask_on = false;
  cudaStream_t cap_stream = nullptr;
  GraphEntry graphs[kGraphCache];
  unsigned long long graph_clock = 0;
  bool capturing = false;
  bool cap_events = false;     // the capture records the phase boundaries as event nodes
  cudaEvent_t cap_ev[kProfEvents];
  int cap_tag[kProfEvents];
  int cap_n = 0;
  bool cap_ev_made = false;
  // profiler (off by default)
  bool prof = false;
  ProfSlot *slots = nullptr;
  int slots_used = 0;
  ProfSlot *cur = nullptr;
  long long launches = 0;
};

// Profiler hooks (no-ops unless enabled): begin a call record, close the running segment as
// phase `tag`, count kernel launches.
void prof_begin(Plan *p, cudaStream_t st);
void ib_drop_graph(Plan *p);   // the IB loop graph of a plan (project.cu)
void prof_mark(Plan *p, cudaStream_t st, int tag);
inline void count_launch(Plan *p, int n = 1) { p->launches += n; }

// ----------------------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
pc_status fail(pc_status st, const char *fmt, ...);

#define PC_CUDA_TRY(expr)                                                                    \
  do {                                                                                       \
    cudaError_t _e = (expr);                                                                 \
    if (_e != cudaSuccess)                                                                   \
      return ::pc::fail(PC_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                        __FILE__, __LINE__);                                                 \
  } while (0)

#define PC_TRY(expr)                       \
  do {                                     \
    pc_status _s = (expr);                 \
    if (_s != PC_OK) return _s;            \
  } while (0)

pc_status plan_alloc(Plan *p, void **ptr, size_t bytes);
// Staging buffers of the node arrays for calls with host pointers, allocated on the first such
// call (device-pointer callers never pay for them).
pc_status plan_node_staging(Plan *p);

// ----------------------------------------------------------------------------- launches
inline int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (1LL << 30)) b = 1LL << 30;
  return (int)b;
}

// Transform solves of a grid (poisson.cu): FP64 s -> p, and one FP32 solve whose source and
// destination modes are those of passes.cuh (FP32 or FP64 source; FP64 set or accumulate).
pc_status solve_fp64_grid(Plan *p, const double *s, double *pout, cudaStream_t st);
// chunk: consecutive tiles per CTA (refinement sweeps that the stopping rule usually ends before
// they start are launched with few CTAs, so a skipped sweep costs little)
pc_status solve_fp32_grid(Plan *p, int src_mode, const void *s, int dst_mode, void *dst,
                          cudaStream_t st, double *f64 = nullptr, RefineGate gate = RefineGate{nullptr, 0, 0.0f},
                          int chunk = 1);
// Drops the plan's captured CUDA graphs and batch executables (after a schedule change).
void plan_drop_graphs(Plan *p);
// ----------------------------------------------------------------------------- batches
// Stages of the batched pipeline (one launch per stage for all problems of a batch).
enum BatchStage {
  BATCH_ZERO = 0, BATCH_PREP = 1, BATCH_TRANSFER = 2 /* +axis */, BATCH_DIVERGENCE = 5, BATCH_RESIDUAL = 6,
  BATCH_GAUGE_SUM = 7, BATCH_FINALIZE = 8, BATCH_GRADIENT = 9, BATCH_STAGES = 10
};

// Cell-grid geometry and strides shared by the per-cell kernels (project.cu).
struct GridDev {
  int dim;
  int n[3];           // cells per axis, padded: n3[0..2] with the last axis fastest
  int nf[3];          // faces along each axis (n or n+1)
  int cs[3];          // cell strides
  int fs[3][3];       // fs[a][b]: stride of axis b in the face array of axis a
  int periodic[3];
  // ghost rule at each end, ignored when periodic: 0 Neumann (ghost = edge value), 1 Dirichlet
  // (ghost = -edge value; cell grids), 2 Neumann about a vertex (ghost = the next value inward),
  // 3 Dirichlet vertex (ghost = 0; vertex grids)
  int lo_kind[3], hi_kind[3];
  double inv_h[3], inv_h2[3];
  float ih2_hi[3], ih2_lo[3];   // inv_h2 as an FP32 pair (double-float residual)
  // cell tiles of the cell kernels (project.cu): rows of the last axis, tile width 2^tw_bits,
  // 2^th_bits thread rows of cr rows each, gx tiles along the last axis, nblk blocks
  int rows, tw_bits, th_bits, cr, gx, nblk;
  const uint8_t *mask;          // RHS mask per cell (nonzero = flow domain), nullptr = none
};

// Per-problem parameters of a batched launch (device array, one entry per problem).
struct BatchProblem {
  GridDev g;
  int dim, vdtype, N, ncells, K, Kg, singular, gmode;
  int kmax;            // refinement sweeps at most; under the stopping rule when tol > 0
  float tol;           // the rule's tolerance (<= 0: a fixed sweep count)
  const void *u, *f;
  void *uo, *fo;
  double *p;
  double dt, inv_dt, beta, inv_bdt, inv_ncells;
  float2 *u2;
  const int32_t *fcol[3];
  const float2 *fw2[3];
  double *U64[3];
  int frows[3];
  double *s64;
  float *s32, *r32;
  float2 *p2;
  const int32_t *ncol;
  const float2 *nD2;
  const uint8_t *ntype;
  DevStats *ds;
  double *partials;
  unsigned int *counters;
};

void batch_launch(int stage, int variant, const BatchProblem *P, const int *seg, int count, int total_blocks,
                  int extra, cudaStream_t st);
void batch_block_counts(const Plan *p, int *nb);
void batch_problem_fill(const Plan *p, const pc_project_args &a, BatchProblem &q);
void batch_forget_plan(const Plan *p);

// Solve of device arrays for a plan description built by the caller (project.cu).
pc_status solve_grid_device(Plan *p, const double *s, double *pout, cudaStream_t st);
pc_status prepare_kernels();
// Setup (setup.cu).
pc_status build_rows(Plan *p, const double *xyz_dev, cudaStream_t st);
// Momentum rows at every node over its K nearest nodes: columns [K][N]; first-derivative rows
// and the Laplacian row [dim + 1][K][N], FP64 (w64) and/or FP32 pairs (w2).
pc_status build_momentum_rows(const Plan *p, const double *xyz_dev, int K, int32_t *col, double *w64, float2 *w2,
                              cudaStream_t st);
// Axis tables (poisson.cu).
pc_status build_axis_tables(Plan *p);


// ----------------------------------------------------------------------------- launches
// Programmatic dependent launch: every kernel of the projection path first waits for the
// kernel before it to complete (griddepcontrol.wait: its writes are visible after the wait),
// then lets the next kernel of the stream be scheduled. The next kernel's CTAs can thus be
// resident and waiting when this one ends, which hides the launch gap between dependent
// kernels (also inside CUDA graphs, where the edges become programmatic). Without the launch
// attribute the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Set while a graph whose edges must stay plain is captured (the bodies of conditional nodes):
// launch_pdl then launches without the programmatic attribute.
inline thread_local bool tl_plain_launch = false;

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = tl_plain_launch ? 0 : 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);   // errors surface through cudaGetLastError
}

}  // namespace pc
