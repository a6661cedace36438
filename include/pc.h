/*
 * pc.h - C ABI of the GB300 pressure-correction library (libpc.so).
 *
 * The library performs the pressure-correction sub-step of Fang's hybrid projection method
 * (arXiv 2304.14690, §2.3): weighted-least-squares (WLS) transfer of the provisional velocity
 * u* from an irregular node cloud to the faces of a uniform staggered pressure grid, the
 * divergence source of the modified pressure Poisson equation (Eq. 20) with the immersed-
 * boundary force, a transform-based Poisson solve (§2.3: forward 1D transforms per axis,
 * division by summed eigenvalues, inverse transforms), and the WLS pressure gradient back at
 * the nodes with the velocity correction and IB-force update (Eqs. 18-19).
 *
 * Conventions shared by every entry point
 *  - Grid: dim (2 or 3) axes, n[a] cells of spacing h[a] from lo[a]; cell centre
 *    lo + (i + 1/2) h. Cell arrays are C order (last axis contiguous), one value per cell.
 *  - Nodes: structure of arrays, [dim][num_nodes] (component a of node k at a*num_nodes + k).
 *  - Pointers: every array argument of pc_project / pc_solve_poisson may be a device pointer
 *    or a host pointer (pinned host memory is fastest); the library detects which. Host
 *    arrays are copied through plan-owned device buffers on the given stream. The caller
 *    owns all arrays; the library never keeps a pointer past the call that received it.
 *  - Streams: cuda_stream is a cudaStream_t (NULL = legacy default stream). A plan may be
 *    used by one stream at a time. pc_project and pc_solve_poisson allocate nothing and do
 *    not synchronize, unless host pointers or a stats struct are passed (both need a sync).
 *  - Errors: every entry point returns a pc_status; nothing aborts or traps. The message of
 *    the last failure on the calling thread is pc_last_error_message().
 */
#ifndef PC_H
#define PC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PC_OK = 0,
  PC_ERR_INVALID_ARG = 1,   /* malformed descriptor or argument */
  PC_ERR_UNSUPPORTED = 2,   /* valid but not supported (e.g. an odd cell count on a transform axis) */
  PC_ERR_WLS_SINGULAR = 3,  /* a WLS normal matrix C (Eq. 14) is not positive definite */
  PC_ERR_OUT_OF_MEMORY = 4, /* a device allocation failed */
  PC_ERR_BUDGET = 5,        /* the plan would exceed the caller's device-memory budget */
  PC_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  PC_ERR_NOT_CONVERGED = 7, /* refinement did not reach the requested residual */
  PC_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up */
} pc_status;

/* Boundary kind of one domain face (§2.1 Eqs. 7-8, §2.3, §3.3). */
typedef enum {
  PC_BC_PERIODIC = 0,        /* must pair with PERIODIC on the same axis */
  PC_BC_NEUMANN_WALL = 1,    /* homogeneous Neumann; the face flux is zero (§3.3 workaround) */
  PC_BC_NEUMANN_INFLOW = 2,  /* homogeneous Neumann (Eq. 7); the face keeps its transferred flux */
  PC_BC_DIRICHLET = 3        /* homogeneous Dirichlet p = 0 on the face; transferred flux */
} pc_bc;

typedef enum {
  PC_PREC_FP64 = 0,   /* every step in FP64 */
  PC_PREC_MIXED = 1,  /* compensated FP32 gathers, FP32 transforms, refinement with a residual
                         in double-float arithmetic (~48 significant bits) against the FP64
                         iterate */
  PC_PREC_FP32 = 2    /* as MIXED with no refinement (reports the unrefined FP32 error) */
} pc_precision;

typedef enum { PC_DTYPE_F64 = 0, PC_DTYPE_F32 = 1 } pc_dtype;

/* Eigenvalues of the transform solve (§2.3 allows both with the same transforms). With the
 * angle theta of a basis vector (2 pi k/n periodic, pi k/n N-N, pi (k+1)/n D-D, pi (k+1/2)/n
 * N-D and D-N): central finite differences -(2/h)^2 sin^2(theta/2), the exact inverse of the
 * 2d+1-point Laplacian; pseudo-spectral -(theta/h)^2, the continuous eigenvalue of the function
 * the basis vector samples. */
typedef enum { PC_EIG_FD = 0, PC_EIG_SPECTRAL = 1 } pc_eigenvalues;

/* Where the source of the PPE comes from. PC_DIV_FACES: WLS value rows transfer u~ to the MAC
 * faces and s is their compact divergence D_h U / (beta dt), so the corrected face flux is
 * divergence-free to rounding. PC_DIV_WLS_DIRECT: s = sum_a sum_k D_a,k u~_a,k / (beta dt) with
 * WLS derivative rows at every cell centre over its K nearest nodes (the paper's evaluation of
 * the right-hand side at the pressure points, §2.3); no face fluxes are formed, so max_div_after
 * of pc_stats is not computed (0). The plan then holds K (index) + dim*K (weights) entries more
 * per cell; pc_project_ib recomputes the whole source on every pass and pc_project_batch runs
 * such plans one by one. */
typedef enum { PC_DIV_FACES = 0, PC_DIV_WLS_DIRECT = 1 } pc_divergence;

/* Node kinds of the double discretization (§2.3, Fig. 1). */
typedef enum { PC_NODE_FLUID = 0, PC_NODE_BOUNDARY = 1, PC_NODE_VIRTUAL = 2 } pc_node_type;

/* Obstacle metadata (circle in 2D, sphere in 3D). Used for validation and reports only:
 * the caller classifies nodes itself (node_type). */
typedef struct {
  int shape; /* 0 = circle/sphere */
  double centre[3];
  double radius;
} pc_obstacle;

/* Pressure points: the cell centres of the grid (the staggered grid of §2.3) or its vertices (the
 * regular grid of §2.3 and §3.2; unknowns per axis and boundary pair at pc_grid_plan_create). */
typedef enum { PC_GRID_CELLS = 0, PC_GRID_VERTICES = 1 } pc_grid_type;

typedef struct {
  int dim;                  /* 2 or 3 */
  int64_t n[3];             /* cells per axis; n[a] even on every axis (transform length) */
  double lo[3];             /* lower corner */
  double h[3];              /* spacing; the domain length is n[a]*h[a] */
  int bc_lo[3], bc_hi[3];   /* pc_bc per axis end */
  int64_t num_nodes;        /* N */
  const double *node_xyz;   /* [dim][N] node coordinates (device or host); nodes on a periodic
                               axis must lie in [lo, lo + n h), on other axes inside the box */
  const uint8_t *node_type; /* [N] pc_node_type (device or host) */
  int num_obstacles;
  const pc_obstacle *obstacles; /* host, may be NULL */
  int knn;                  /* neighbours per WLS stencil K (>= 6 in 2D, >= 10 in 3D; <= 32) */
  double wls_eps;           /* Gaussian weight constant eps of Eq. 17 (paper: 6.3) */
  double support_factor;    /* support radius / local spacing (paper: 3, §2.2) */
  double beta;              /* AB2 pressure factor 3/2 of Eq. 4 */
  int precision;            /* pc_precision */
  int refine_iters;         /* MIXED: largest number of refinement sweeps (0..8; see refine_tol) */
  int gauge;                /* 0: mean(p) = 0; 1: p at the corner cell = 0 (§3.1). Applies only
                               when no face is Dirichlet (the solution is then defined up to
                               a constant) */
  int velocity_dtype;       /* pc_dtype of u_star, f_ib_in, u_out, f_ib_out */
  int eigenvalues;          /* pc_eigenvalues. PC_EIG_SPECTRAL needs precision FP64 or FP32
                               (PC_ERR_UNSUPPORTED with MIXED: the refinement residual applies
                               the compact L_h, which is the inverse of the FD eigenvalues only);
                               its solve is not the inverse of L_h, so max_div_after and the
                               residual norms of pc_stats do not apply (reported as 0 residuals) */
  int divergence;           /* pc_divergence */
  int grid_type;            /* pc_grid_type. PC_GRID_VERTICES needs PC_DIV_WLS_DIRECT (a vertex grid
                               has no faces; PC_ERR_UNSUPPORTED otherwise): the source is the WLS
                               divergence at the vertex unknowns, the node gradient uses the 3^d
                               block of lattice vertices around each node (Dirichlet boundary
                               vertices with value 0), and p_out, the RHS mask and the rows of
                               pc_plan_rows(dim + 1) are in the unknowns' layout. The transform
                               limits per axis are those of pc_grid_plan_create's vertex grids */
  double refine_tol;        /* MIXED: stopping rule of the refinement, decided on the device after
                               each residual r_k = s - mean - L_h p_k (k sweeps done), on max
                               norms: stop when ||r_k|| <= refine_tol ||s|| (converged); or when
                               k >= 2 and ||r_k|| > 16 (||r_1|| / ||r_0||) ||r_{k-1}||: the residual
                               no longer falls at the rate of a sweep, it has reached the rounding
                               floor of its own evaluation (about 1e-12 to 1e-10 of ||s|| on 256^2
                               to 4096 x 1024 grids) and the iterate's error is then below the
                               previous one's by about that rate (converged at the floor); or after
                               refine_iters sweeps. Sweeps past the stop are still launched and
                               exit at once, so graphs and batches keep one shape. The verdict is
                               reported with statistics (pc_stats.refine_converged; a call whose
                               sweeps ran out returns PC_ERR_NOT_CONVERGED); without statistics the
                               call does not wait and reports nothing.
                               refine_tol <= 0: exactly refine_iters sweeps, no rule */
} pc_problem_desc;

/* Per-call diagnostics (optional). Filling it synchronizes the stream, and a NaN or infinity that
 * reached the source (through u_star, f_ib_in or dt) is then reported as PC_ERR_INVALID_ARG, with
 * the statistics filled. Without stats nothing is checked. */
typedef struct {
  double removed_mean;      /* mean of the source dropped by the compatibility projection */
  double source_norm;       /* ||s||_2 over cells */
  double residual_norm[9];  /* ||s - mean - L_h p||_2 after the first solve and each sweep */
  int refine_iters_done;
  double max_div_after;     /* max |D_h (U - beta dt G_h p)| over cells (faces corrected) */
  double max_abs_u_star;    /* velocity scale */
  double gauge_shift;       /* constant subtracted from p by the gauge */
  int refine_converged;     /* MIXED with refine_tol > 0: the stopping rule was met (1) or the
                               sweeps ran out (0; the call then returns PC_ERR_NOT_CONVERGED with
                               every output and statistic written) */
} pc_stats;

typedef struct pc_plan pc_plan;

/* Build a plan: neighbour search (§2.2 linked-list search), the WLS rows C^-1 A (§2.2
 * Eqs. 13-17, f-unknown basis of Eq. 16) for every flux-carrying face (value row over the K
 * nearest nodes) and every node (derivative rows over the 3^dim block of cell centres around
 * it, shifted inward at walls, wrapped on periodic axes), eigenvalue and twiddle tables, and
 * the whole workspace of pc_project. The coefficients depend only on positions and are
 * computed once (§2.2, last paragraph). Runs on `device` on `cuda_stream` and returns when
 * done. hbm_budget_bytes = 0 means no budget. Limits: at most 2^31 - 2^16 cells, faces normal to
 * any axis, and nodes (the kernels number rows in 32 bits and offset into the row arrays in 64
 * bits); larger problems return PC_ERR_UNSUPPORTED before any device call. */
pc_status pc_plan_create(const pc_problem_desc *desc, int device, size_t hbm_budget_bytes,
                         void *cuda_stream, pc_plan **out_plan);

/* One pressure-correction pass (one iteration of the IB-force loop of §2.3 with a given
 * force):
 *   u~ = u* + dt f~_in          (right-hand side of Eq. 20 is (1/(beta dt)) div u~)
 *   U  = WLS value rows (u~)    on faces; wall faces 0
 *   s  = D_h U / (beta dt);     L_h p = s (mean of s dropped when singular)
 *   g  = WLS derivative rows (p) at nodes
 *   fluid node:            u_out = u* - beta dt g,  f~_out = 0                   (Eq. 4)
 *   boundary/virtual node: f~_out = -(u*)/dt + beta g, u_out = 0               (Eqs. 18-19)
 * u_star, f_ib_in (nullable = zero), u_out, f_ib_out (nullable): [dim][N] of velocity_dtype.
 * p_out: cells, FP64. Returns without waiting for the GPU unless host pointers or stats. */
pc_status pc_project(pc_plan *plan, double dt, const void *u_star, const void *f_ib_in,
                     double *p_out, void *u_out, void *f_ib_out, pc_stats *stats,
                     void *cuda_stream);

/* The IB-force iteration of §2.3: the modified PPE (Eq. 20) and the force update (Eq. 19) are
 * repeated, each pass with the force of the previous one, until the mean over boundary/virtual
 * nodes of |f_new - f_old|^2 is <= tol times the mean of |f_old|^2 (a zero previous force stops
 * only with zero change), or max_iters passes (>= 1). The paper's tolerance is 1e-3.
 *   f_ib_init  force of the first pass ([dim][N] of velocity_dtype, nullable = zero: the first
 *              iteration of a time step); only its boundary/virtual entries are used, the force
 *              lives at those points
 *   p_out, u_out, f_ib_out   as pc_project, from the last pass (f_ib_out nullable)
 *   history    nullable HOST buffer of 2*max_iters doubles: (mean |df|^2, mean |f_old|^2) per pass
 *   result     nullable: passes run, whether the rule was met, and the last pair
 * Each pass after the first updates u~ only at the boundary/virtual nodes, recomputes only the
 * fluxes of the faces whose WLS value row reaches one of them, solves, and evaluates the gradient
 * at those nodes alone (§2.3); the gradient at the fluid nodes and Eq. 4 follow the last pass.
 * The iterates are bitwise those of repeated pc_project calls fed with the previous force.
 * The stopping rule is evaluated on the device. With CUDA graphs on (pc_set_graphs, the default)
 * the whole time step is one graph launch: a while-conditional node repeats the later passes
 * until the device-side rule stops it (captured once per argument set, dt, tol and max_iters);
 * with graphs off the host reads the decision after every pass. Either way the call returns when
 * the step is done (one stream synchronisation per call, reading the pass count and history).
 * Device pointers only, max_iters in [1, 1000] (PC_ERR_INVALID_ARG otherwise); not capturable
 * (PC_ERR_INVALID_ARG on a capturing stream). The first call on a plan builds the node and face
 * lists (one allocation: about 4 bytes per listed node or face, two force iterates, 16 KB of
 * loop state). */
/* A non-finite stopping sum in any pass (a diverging iteration, or a NaN or infinity in the
 * input) returns PC_ERR_NOT_CONVERGED after result and history are filled. */
typedef struct {
  int iterations;
  int converged;
  double diff;   /* last pass: mean over boundary/virtual nodes of |f_new - f_old|^2 */
  double prev;   /* and of |f_old|^2 */
} pc_ib_result;

pc_status pc_project_ib(pc_plan *plan, double dt, const void *u_star, const void *f_ib_init,
                        double tol, int max_iters, double *p_out, void *u_out, void *f_ib_out,
                        double *history, pc_ib_result *result, void *cuda_stream);

typedef struct {
  double dt;
  const void *u_star;
  const void *f_ib_in;
  double *p_out;
  void *u_out;
  void *f_ib_out;
} pc_project_args;

/* count independent projections (each plan with its own arguments, each plan at most once) on
 * one stream; the results are bitwise those of count separate pc_project calls. Device pointers
 * only. Plans in MIXED or FP32 precision are grouped (by dimension, velocity type, neighbour
 * count and refinement sweeps) and each stage of the pipeline runs as one kernel launch over all
 * problems of a group; the launch sequence is captured into a CUDA graph when a batch
 * composition (plans and argument pointers) is first seen, which also allocates its small work
 * tables, and replayed afterwards (8 compositions are cached). FP64 plans run one by one. */
pc_status pc_project_batch(int count, pc_plan *const *plans, const pc_project_args *args,
                           void *cuda_stream);

/* Batch executor for batches that change from call to call (continuous batching in a request
 * loop): the same grouping and one-launch-per-stage kernels as pc_project_batch, with the same
 * bitwise results, but nothing is captured, cached or allocated per call. The executor owns
 * `slots` table slots of `table_bytes` each (0 = 16 MiB), each a pinned host buffer with a
 * device copy: a launch fills the next slot on the host, copies it with one asynchronous
 * transfer on `cuda_stream` and launches the stage kernels behind it; it waits on the host only
 * when the slot it reuses still belongs to a batch that has not finished. A plan must not be in
 * two batches that may run at the same time (they share the plan's workspace). Errors:
 * PC_ERR_BUDGET when a batch's tables exceed table_bytes; as pc_project_batch otherwise.
 * Launches on one executor are serialised by a lock; destroy waits for its pending batches. */
typedef struct pc_batcher pc_batcher;
pc_status pc_batcher_create(int device, size_t table_bytes, int slots, pc_batcher **out);
pc_status pc_batcher_launch(pc_batcher *batcher, int count, pc_plan *const *plans,
                            const pc_project_args *args, void *cuda_stream);
pc_status pc_batcher_destroy(pc_batcher *batcher);

/* RHS mask (§3.5, lid-driven polar cavity: the source is turned to zero at pressure points
 * outside the flow domain, where part of the solid moves). mask: [cells] uint8 in C order
 * (device or host), nonzero = inside the flow domain. Projections of this plan instance
 * (pc_project, pc_project_ib, the batched calls) then set s = 0 at masked-out cells before the
 * compatibility step and the solve; after the correction the face divergence vanishes inside
 * the mask and equals beta dt times the dropped source outside it, so max_div_after of pc_stats
 * is taken over the cells inside. The mask is copied into plan memory (1 byte per cell,
 * allocated on the first call; the call waits for the copy). NULL clears it. Switching between
 * masked and unmasked drops the plan's captured CUDA graphs; changing the mask's content does
 * not need to. pc_solve_poisson takes its source as given (no mask). A clone starts unmasked.
 * On a vertex-grid plan the mask has one byte per vertex unknown (C order of the unknowns). */
pc_status pc_plan_set_rhs_mask(pc_plan *plan, const uint8_t *mask, void *cuda_stream);

/* Grid-only plans: the Poisson solve of §2.3 without nodes, on the cell centres of the grid
 * (PC_GRID_CELLS, as in every pc_plan_create plan) or on its vertices (PC_GRID_VERTICES: the
 * "regular" grid of §2.3, used for the results of §3.2). On a vertex grid with n cells per axis
 * the unknowns of an axis are, per boundary pair (lo-hi): P-P vertices 0..n-1; N-N 0..n (mirror
 * ghosts p_{-1} = p_1, p_{n+1} = p_{n-1}); D-D 1..n-1 (p_0 = p_n = 0); N-D 0..n-1 (p_n = 0);
 * D-N 1..n (p_0 = 0). The eigenbases are DCT-I (N-N), DST-I (D-D), the real DFT (P-P) and the
 * quarter-wave cosine/sine bases cos(pi (k + 1/2) j/n), sin(pi (k + 1/2) j/n) (N-D, D-N). The
 * solve runs on the unknowns with one transform pass per axis as on the cell grid: DCT-I and
 * DST-I through the real DFT of length 2n of the line extended evenly or oddly in shared memory
 * (n must be 2^a 3^b 5^c <= 2048), the quarter-wave pairs as the DCT-III / DST-III analysis and
 * DCT-II / DST-II synthesis of length n, and P-P as on the cell grid (n even, n/2 2^a 3^b 5^c
 * <= 2048 for both). When every axis is P-P or N-N the constant mode is dropped (on N-N axes it
 * is the trapezoid-weighted mean) and reported in removed_mean, and the solution has no
 * constant part (trapezoid-weighted mean zero); the corner gauge zeroes the first unknown
 * instead. Only pc_solve_poisson, the schedule, profiling and
 * pc_destroy apply to a grid-only plan; the node entry points and pc_plan_clone return
 * PC_ERR_INVALID_ARG.
 * pc_grid_plan_create reads desc during the call only; the plan belongs to the caller until
 * pc_destroy. Errors: PC_ERR_INVALID_ARG for a malformed descriptor (dim, n[a] outside
 * [4, 4096], h, boundary kinds, precision, refine_iters, gauge, eigenvalues, grid_type);
 * PC_ERR_UNSUPPORTED for a solve length the transforms do not cover or pseudo-spectral
 * eigenvalues with the MIXED refinement; PC_ERR_CUDA when the device is unavailable;
 * PC_ERR_OUT_OF_MEMORY. cuda_stream orders the setup copies (NULL: the default stream). */
typedef struct {
  int dim;                  /* 2 or 3 */
  int64_t n[3];             /* cells per axis */
  double h[3];              /* spacing */
  int bc_lo[3], bc_hi[3];   /* pc_bc per axis end */
  int grid_type;            /* pc_grid_type */
  int precision;            /* pc_precision */
  int refine_iters;         /* MIXED: largest number of refinement sweeps */
  int gauge;                /* 0 mean, 1 corner (used when the problem has a zero mode) */
  int eigenvalues;          /* pc_eigenvalues */
  double refine_tol;        /* MIXED: stopping rule, as pc_problem_desc.refine_tol */
} pc_grid_desc;
pc_status pc_grid_plan_create(const pc_grid_desc *desc, int device, void *cuda_stream, pc_plan **out_plan);

/* The grid-level Poisson solve alone (§2.3 three-step algorithm): L_h p = s, cells in FP64,
 * with the plan's precision, refinement and gauge. */
pc_status pc_solve_poisson(pc_plan *plan, const double *s, double *p_out, pc_stats *stats,
                           void *cuda_stream);
/* (On a vertex-grid plan s and p_out have the unknowns' shape, C order. The statistics are those
 * of the solve on the unknowns: source_norm and the residual norms are plain L2 norms over them,
 * removed_mean is the dropped zero-mode coefficient (the trapezoid-weighted mean of s; 0 when an
 * axis has a Dirichlet end) and gauge_shift the constant the gauge took from p.) */

/* Allocation-free grid-level Poisson solve (the paper has no counterpart: this is a service of
 * the library, not a step of the method). Solves L_h p = s in FP64 with the same transform
 * passes as pc_solve_poisson, for a grid given by dim, n[dim], h[dim], bc_lo/bc_hi[dim] (pc_bc)
 * and gauge (0 mean, 1 corner; used when no face is Dirichlet), without a plan.
 *
 * It is for callers that cannot call cudaMalloc when they need a solve: code running under a
 * memory pool or custom allocator that owns all device memory, code inside host callbacks or
 * library hooks where an allocation would synchronise the device or is not permitted, and
 * deployments that fix their device memory at start-up. It allocates nothing: its workspace is
 * one file-scope device array of 8 MiB that every GPU loading the library holds until exit.
 *  - Limit: at most 524288 cells (e.g. 1024 x 512); larger grids return PC_ERR_BUDGET.
 *  - s and p_out are device pointers (C order, one FP64 value per cell); host pointers are
 *    rejected with PC_ERR_INVALID_ARG.
 *  - s and p_out must be device memory of the current device (or managed memory);
 *    PC_ERR_INVALID_ARG otherwise.
 *  - The first call on a device looks up the array's device address, zeroes it and sets kernel
 *    attributes; make that first call before any stream capture. The address is cached per
 *    device: after cudaDeviceReset the cache is stale, so do not use this entry point again in
 *    that process.
 *  - All calls share the one array and it keeps the last call's contents: calls that overlap on
 *    the GPU (different streams, or different host threads) race and corrupt each other. */
pc_status pc_solve_poisson_static(int dim, const int64_t *n, const double *h, const int *bc_lo,
                                  const int *bc_hi, int gauge, const double *s, double *p_out,
                                  void *cuda_stream);

/* WLS rows of a plan, for inspection and tests. which = 0..dim-1: value rows of the faces
 * normal to that axis (rows = faces in C order of that face array); which = dim: derivative
 * rows of the nodes (rows = nodes, weights [dim][rows][K]); which = dim+1 (PC_DIV_WLS_DIRECT
 * plans only): derivative rows of the cell centres (rows = cells in C order, columns node
 * indices, weights [dim][rows][K]). On a vertex-grid plan there are no face rows, the rows of
 * dim+1 are those of the vertex unknowns (C order of the unknowns), and the node rows' columns
 * are linear indices of the vertex lattice (n per periodic axis, n + 1 otherwise, Dirichlet
 * boundary vertices included). col_out: [rows][K] int32 (node
 * index for faces, cell linear index for nodes), w_out: FP64 host buffers. rows_out gets the
 * row count; pass NULL buffers to query it. FP64 plans return the FP64 weights; MIXED and FP32
 * plans keep only the FP32 (hi, lo) pairs after setup (the FP64 weights are setup temporaries)
 * and return hi + lo, within 2^-46 of the FP64 weight. */
pc_status pc_plan_rows(const pc_plan *plan, int which, int64_t *rows_out, int32_t *col_out,
                       double *w_out);

/* Optional per-phase timing with CUDA events recorded on the call's stream (for profiling and
 * roofline reports; leave it off in production and under stream capture). Phases:
 * 0 prep (u~ = u* + dt f~), 1 transfer (faces), 2 divergence, 3 transform passes (all solves),
 * 4 FP64 residuals, 5 gauge, 6 gradient and correction, 7 statistics. pc_profile_read waits for
 * the recorded events, returns the milliseconds summed over the calls made since the last read
 * (at most 256 calls are kept), the number of calls, and the number of kernels libpc launched
 * in them; it then resets the counters. */
typedef struct {
  double phase_ms[8];
  int calls;
  long long kernel_launches;
} pc_profile;

pc_status pc_profile_enable(pc_plan *plan, int on);
pc_status pc_profile_read(pc_plan *plan, pc_profile *out);

/* CUDA graphs (on by default): a pc_project call with device pointers and no stats is
 * captured once per distinct (pointers, dt) into a CUDA graph on a plan-private stream and then
 * replayed with a single launch on the caller's stream (up to 4 argument sets are cached per
 * plan). A pc_solve_poisson call with device arrays and no stats is captured the same way per
 * (s, p_out). Results are identical with graphs on or off. */
pc_status pc_set_graphs(pc_plan *plan, int on);

/* Schedule of the transform passes (§2.3 three-step solve). Every pass along `axis` gives each
 * thread at most `slots` complex slots of a line (2, 4, 8 or 16): this fixes the threads per
 * line and the radix schedule of the FFT (largest power-of-two radices up to min(slots, 16),
 * then 3 and 5). `precision` selects the FP64 passes (PC_PREC_FP64) or the FP32 passes (the
 * other two). A schedule is part of the plan: single and batched calls use it alike, and changing
 * it drops the plan's captured CUDA graphs. Results change only by rounding between schedules.
 * FP32 passes also take slots = 0 and 1: the compile-time pass of the axis's line length, where
 * the length has one (cell-grid transforms, n = 2M with M in {16, 32, 48, 64, 96, 128, 192, 256,
 * 384, 512}; its slots per thread are fixed by M: variant 0 with the most slots per thread and
 * the fewest instructions, variant 1 with fewer slots and more threads per line, for grids too
 * small to hide latency with variant 0), else 4 slots.
 * Errors: PC_ERR_INVALID_ARG for a bad axis or slot count; a schedule whose tile does not fit the
 * kernels fails at the next call with PC_ERR_UNSUPPORTED. Defaults: 0 (FP32), 2 (FP64). */
pc_status pc_plan_set_transform_slots(pc_plan *plan, int axis, pc_precision precision, int slots);
pc_status pc_plan_get_transform_slots(const pc_plan *plan, int axis, pc_precision precision,
                                      int *slots_out);

/* Tile size of the single-problem passes along `axis`: the number of lines per CTA is halved
 * until the pass has at least ctas_per_sm x 152 CTAs (1, 2, 4 or 8; default 2). Part of the
 * schedule like the slots: it drops the plan's graphs, leaves batched calls (whose tiles fill a
 * fixed CTA) alone, and does not change results (each line is transformed the same way in any
 * tile). Errors: PC_ERR_INVALID_ARG for a bad axis or count. */
pc_status pc_plan_set_transform_ctas(pc_plan *plan, int axis, pc_precision precision, int ctas_per_sm);
pc_status pc_plan_get_transform_ctas(const pc_plan *plan, int axis, pc_precision precision, int *ctas_out);

/* Autotuner: times the plan's own transform solve (FP64 for FP64 plans, FP32 otherwise) on
 * `cuda_stream` for every slot count and every CTA target of every axis in turn (coordinate
 * descent, two rounds),
 * keeps the fastest schedule and returns its milliseconds per solve in *best_ms_out
 * (nullable). It synchronises the stream, overwrites the plan's workspace, and must not run
 * during a stream capture or while a call of the plan is in flight. */
pc_status pc_plan_autotune(pc_plan *plan, void *cuda_stream, double *best_ms_out);

/* Device bytes held by the plan. */
pc_status pc_plan_bytes(const pc_plan *plan, size_t *bytes_out);

/* A second workspace for a plan: the clone shares the plan's WLS rows, node types and transform
 * tables (read-only) and owns its own workspace (face fluxes, cell arrays, node copies,
 * statistics, CUDA graphs), so the plan and its clones can run projections at the same time
 * (on different streams, or in one batch) with identical results. Cloning a clone clones its
 * root. A clone costs the workspace only (about 60 bytes per cell plus 8 * dim bytes per node in
 * mixed precision, against the rows' 12 K bytes per face and (4 + 8 dim) 3^dim per node). The
 * transform schedule is copied at cloning time. The root must outlive its clones: pc_destroy of
 * a plan with live clones fails with PC_ERR_INVALID_ARG. */
pc_status pc_plan_clone(pc_plan *plan, void *cuda_stream, pc_plan **out_plan);

pc_status pc_destroy(pc_plan *plan);

/* The first fractional step around the correction: the second-order Adams-Bashforth predictor
 * of Eq. 3 (§2.1) on the plan's nodes,
 *   u* = u^n + (3/2) dt R^n - (1/2) dt R^{n-1},   R = -u . grad u + nu lap u + F,
 * with R^{n-1} carrying -grad p^{n-1}. Gradient and Laplacian at a node are WLS rows (§2.2)
 * over its knn nearest nodes (itself included), with the plan's weight constant and support
 * factor. grad p^{n-1} at a fluid node is recovered from the last correction, u^n = u*^{n-1} -
 * beta dt grad p^{n-1} (Eq. 18), so a run alternates pc_momentum_predict and a correction of its
 * u* (pc_project or pc_project_ib with the same dt) whose u_out is the next u_n. The first step
 * after create or reset is forward Euler. Boundary points get the prescribed velocity
 * (u_boundary, NULL: zero), virtual points zero.
 * pc_momentum_create: node_xyz [dim][N] (device or host, the coordinates the plan was built
 * from), knn in [6, 32] (2D) or [10, 32] (3D) and <= N, nu >= 0, body_force [dim] host or NULL
 * (zero). The plan must outlive the object. Errors: PC_ERR_INVALID_ARG, PC_ERR_WLS_SINGULAR
 * (a node's normal matrix), PC_ERR_OUT_OF_MEMORY, PC_ERR_CUDA.
 * pc_momentum_predict: u_n, u_boundary and u_star [dim][N] in the plan's velocity dtype, device
 * pointers only (PC_ERR_INVALID_ARG otherwise); dt must not change between resets
 * (PC_ERR_INVALID_ARG). Asynchronous on cuda_stream. FP64 arithmetic in FP64 plans,
 * compensated FP32 pairs otherwise. */
typedef struct pc_momentum pc_momentum;
pc_status pc_momentum_create(pc_plan *plan, const double *node_xyz, int knn, double nu, const double *body_force,
                             void *cuda_stream, pc_momentum **out);
pc_status pc_momentum_predict(pc_momentum *m, double dt, const void *u_n, const void *u_boundary, void *u_star,
                              void *cuda_stream);
pc_status pc_momentum_reset(pc_momentum *m);
pc_status pc_momentum_destroy(pc_momentum *m);

const char *pc_status_string(pc_status status);
const char *pc_last_error_message(void); /* thread-local; "" when none */

#ifdef __cplusplus
}
#endif
#endif /* PC_H */
