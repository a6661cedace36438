// Plan lifetime, validation and error reporting of libpc.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "pc_internal.cuh"

namespace pc {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

pc_status fail(pc_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

pc_status plan_alloc(Plan *p, void **ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  if (p->nallocs >= (int)(sizeof(p->allocs) / sizeof(p->allocs[0])))
    return fail(PC_ERR_OUT_OF_MEMORY, "too many plan allocations");
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(PC_ERR_OUT_OF_MEMORY, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  p->allocs[p->nallocs++] = *ptr;
  p->bytes += bytes;
  return PC_OK;
}

// Frees one plan allocation before the plan's end (setup temporaries).
pc_status plan_node_staging(Plan *p) {
  const size_t vb = (size_t)p->dim * p->N * (p->vdtype == PC_DTYPE_F64 ? 8 : 4);
  if (plan_alloc(p, &p->stage_u, vb) != PC_OK || plan_alloc(p, &p->stage_f, vb) != PC_OK ||
      plan_alloc(p, &p->stage_uo, vb) != PC_OK || plan_alloc(p, &p->stage_fo, vb) != PC_OK)
    return PC_ERR_OUT_OF_MEMORY;
  return PC_OK;
}

static void plan_free(Plan *p, void *ptr, size_t bytes) {
  for (int i = 0; i < p->nallocs; ++i)
    if (p->allocs[i] == ptr) {
      cudaFree(ptr);
      p->allocs[i] = p->allocs[--p->nallocs];
      p->bytes -= bytes;
      return;
    }
}

bool axis_length_supported(int n);
bool vertex_axis_supported(int kind, int m);
pc_status prepare_kernels();

void prof_begin(Plan *p, cudaStream_t st) {
  if (p->capturing) {   // phase boundaries become event-record nodes of a profiled graph
    if (!p->cap_events) return;
    p->cap_n = 1;
    cudaEventRecordWithFlags(p->cap_ev[0], st, cudaEventRecordExternal);
    return;
  }
  if (!p->prof || !p->slots) { p->cur = nullptr; return; }
  if (p->slots_used >= kProfSlots) { p->cur = nullptr; return; }
  p->cur = &p->slots[p->slots_used++];
  p->cur->n = 1;
  cudaEventRecord(p->cur->ev[0], st);
}

void prof_mark(Plan *p, cudaStream_t st, int tag) {
  if (p->capturing) {
    if (!p->cap_events || p->cap_n >= kProfEvents) return;
    p->cap_tag[p->cap_n - 1] = tag;
    cudaEventRecordWithFlags(p->cap_ev[p->cap_n], st, cudaEventRecordExternal);
    p->cap_n++;
    return;
  }
  ProfSlot *s = p->cur;
  if (!s || s->n >= kProfEvents) return;
  s->tag[s->n - 1] = tag;
  cudaEventRecord(s->ev[s->n], st);
  s->n++;
}

void plan_drop_graphs(Plan *p) {
  batch_forget_plan(p);
  ib_drop_graph(p);
  for (int i = 0; i < kGraphCache; ++i) {
    if (p->graphs[i].exec) cudaGraphExecDestroy(p->graphs[i].exec);
    if (p->graphs[i].graph) cudaGraphDestroy(p->graphs[i].graph);
    p->graphs[i] = GraphEntry{};
  }
}

static void destroy_plan(Plan *p) {
  if (!p) return;
  batch_forget_plan(p);
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  if (p->slots) {
    for (int i = 0; i < kProfSlots; ++i)
      for (int e = 0; e < kProfEvents; ++e) cudaEventDestroy(p->slots[i].ev[e]);
    delete[] p->slots;
  }
  plan_drop_graphs(p);
  if (p->cap_ev_made)
    for (int e = 0; e < kProfEvents; ++e) cudaEventDestroy(p->cap_ev[e]);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->copy_st) cudaStreamDestroy(p->copy_st);
  for (int e = 0; e < 3; ++e)
    if (p->copy_ev[e]) cudaEventDestroy(p->copy_ev[e]);
  if (p->ib_body_stream) cudaStreamDestroy(p->ib_body_stream);
  for (int i = 0; i < p->nallocs; ++i) cudaFree(p->allocs[i]);
  if (cur >= 0) cudaSetDevice(cur);
  delete p;
}

static int axis_kind(int lo, int hi) {
  if (lo == PC_BC_PERIODIC) return KIND_PP;
  bool nlo = lo != PC_BC_DIRICHLET, nhi = hi != PC_BC_DIRICHLET;
  if (nlo && nhi) return KIND_NN;
  if (!nlo && !nhi) return KIND_DD;
  return nlo ? KIND_ND : KIND_DN;
}

__global__ void check_nodes_kernel(const double *xyz, const uint8_t *type, long long N, int dim,
                                   double lo0, double lo1, double lo2, double L0, double L1, double L2,
                                   int per0, int per1, int per2, unsigned int *bad) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double lo[3] = {lo0, lo1, lo2}, L[3] = {L0, L1, L2};
  const int per[3] = {per0, per1, per2};
  for (int a = 0; a < dim; ++a) {
    double x = xyz[(long long)a * N + i];
    bool ok = isfinite(x) && x >= lo[a] && (per[a] ? x < lo[a] + L[a] : x <= lo[a] + L[a]);
    if (!ok) atomicOr(bad, 1u);
  }
  if (type[i] > PC_NODE_VIRTUAL) atomicOr(bad, 2u);
}

static bool host_ptr(const void *ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
}

// Two partial sums per block of the largest reduction launch (cell grid or flat grid).
// Sizes of a vertex-grid axis of n cells and boundary pair kind: the unknowns, the lattice
// index of the first unknown and the lattice vertices.
static void vertex_axis(int kind, int n, int &nunk, int &j0, int &nlat) {
  nunk = kind == KIND_NN ? n + 1 : (kind == KIND_DD ? n - 1 : n);
  j0 = (kind == KIND_DD || kind == KIND_DN) ? 1 : 0;
  nlat = kind == KIND_PP ? n : n + 1;
}
// Transform kind of a vertex-grid axis with boundary pair kind.
static int vertex_kind(int kind) {
  switch (kind) {
    case KIND_NN: return KIND_VNN;
    case KIND_DD: return KIND_VDD;
    case KIND_ND: return KIND_VND;
    case KIND_DN: return KIND_VDN;
    default: return KIND_PP;
  }
}

static size_t partial_slots(const Plan *p) {
  const long long last = p->n[p->dim - 1];
  const long long cells_launch = ((last + 255) / 256) * (p->ncells / last);
  const long long flat_launch = (p->ncells + 255) / 256;
  return (size_t)(2 * (cells_launch > flat_launch ? cells_launch : flat_launch) + 64);
}

// Per-call workspace of a plan (one projection at a time per workspace): face fluxes, cell
// arrays, node copies, statistics and reduction scratch, and the capture stream and events of
// its CUDA graphs.
static pc_status alloc_workspace(Plan *p, cudaStream_t st) {
  const bool mixed = p->precision != PC_PREC_FP64;
  const long long N = p->N, nc = p->ncells;
  // a vertex pass also holds p on the whole lattice for the gradient, in work64 (FP64) and p2
  const long long nl = (p->vertex && p->nftot > nc) ? p->nftot : nc;
  const int dd = p->dim;
  for (int a = 0; a < dd; ++a)
    if (plan_alloc(p, (void **)&p->U64[a], p->nface_total[a] * 8) != PC_OK) return PC_ERR_OUT_OF_MEMORY;
  if (plan_alloc(p, (void **)&p->s64, nc * 8) != PC_OK || plan_alloc(p, (void **)&p->work64, nl * 8) != PC_OK ||
      plan_alloc(p, (void **)&p->work32, nc * 4) != PC_OK ||
      plan_alloc(p, (void **)&p->dstats, sizeof(DevStats)) != PC_OK ||
      plan_alloc(p, (void **)&p->partials, partial_slots(p) * sizeof(double)) != PC_OK ||
      plan_alloc(p, (void **)&p->counters, 16 * sizeof(unsigned int)) != PC_OK ||
      plan_alloc(p, (void **)&p->stage_p, nc * 8) != PC_OK || plan_alloc(p, (void **)&p->stage_s, nc * 8) != PC_OK)
    return PC_ERR_OUT_OF_MEMORY;
  if (mixed) {
    if (plan_alloc(p, (void **)&p->p2, nl * 8) != PC_OK || plan_alloc(p, (void **)&p->u2, dd * N * 8) != PC_OK)
      return PC_ERR_OUT_OF_MEMORY;
  } else {
    if (plan_alloc(p, (void **)&p->ut64, dd * N * 8) != PC_OK) return PC_ERR_OUT_OF_MEMORY;
  }
  if (cudaMemsetAsync(p->counters, 0, 16 * sizeof(unsigned int), st) != cudaSuccess)
    return fail(PC_ERR_CUDA, "counter reset failed");
  if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(PC_ERR_CUDA, "stream creation failed");
  for (int e = 0; e < kProfEvents; ++e)
    if (cudaEventCreate(&p->cap_ev[e]) != cudaSuccess) return fail(PC_ERR_CUDA, "event creation failed");
  p->cap_ev_made = true;
  return PC_OK;
}

// A vertex plan's pressure grid is its lattice of unknowns, with the vertex transform kinds
// (set after the node rows have been built on the physical grid).
static void vertex_switch_axes(Plan *p) {
  for (int a = 0; a < p->dim; ++a) {
    AxisInfo &ax = p->ax[a];
    ax.n = p->nv[a];
    ax.kind = vertex_kind(p->vkind[a]);
    ax.nfaces = ax.n;
    p->n[a] = ax.n;
    p->nface_total[a] = 0;
  }
}

static pc_status create(const pc_problem_desc *d, int device, size_t budget, cudaStream_t st, Plan **out) {
  if (!d || !out) return fail(PC_ERR_INVALID_ARG, "desc and out_plan are required");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(PC_ERR_INVALID_ARG, "dim must be 2 or 3");
  const int m = d->dim == 2 ? 6 : 10;
  if (d->knn < m || d->knn > kMaxK) return fail(PC_ERR_INVALID_ARG, "knn must be in [%d, %d]", m, kMaxK);
  if (d->num_nodes < d->knn) return fail(PC_ERR_INVALID_ARG, "fewer nodes than knn");
  if (!d->node_xyz || !d->node_type) return fail(PC_ERR_INVALID_ARG, "node_xyz and node_type are required");
  if (!(d->wls_eps > 0) || !(d->support_factor > 0) || !(d->beta > 0))
    return fail(PC_ERR_INVALID_ARG, "wls_eps, support_factor and beta must be positive");
  if (d->precision < PC_PREC_FP64 || d->precision > PC_PREC_FP32) return fail(PC_ERR_INVALID_ARG, "bad precision");
  if (d->refine_iters < 0 || d->refine_iters > kMaxRefine) return fail(PC_ERR_INVALID_ARG, "refine_iters in [0, %d]", kMaxRefine);
  if (d->gauge != 0 && d->gauge != 1) return fail(PC_ERR_INVALID_ARG, "gauge must be 0 or 1");
  if (d->velocity_dtype != PC_DTYPE_F64 && d->velocity_dtype != PC_DTYPE_F32)
    return fail(PC_ERR_INVALID_ARG, "bad velocity_dtype");
  if (d->divergence != PC_DIV_FACES && d->divergence != PC_DIV_WLS_DIRECT)
    return fail(PC_ERR_INVALID_ARG, "divergence must be PC_DIV_FACES or PC_DIV_WLS_DIRECT");
  if (d->eigenvalues != PC_EIG_FD && d->eigenvalues != PC_EIG_SPECTRAL)
    return fail(PC_ERR_INVALID_ARG, "eigenvalues must be PC_EIG_FD or PC_EIG_SPECTRAL");
  if (d->eigenvalues == PC_EIG_SPECTRAL && d->precision == PC_PREC_MIXED)
    return fail(PC_ERR_UNSUPPORTED, "pseudo-spectral eigenvalues need precision FP64 or FP32 (the mixed "
                                    "refinement residual is that of the finite-difference operator)");
  if (d->grid_type != PC_GRID_CELLS && d->grid_type != PC_GRID_VERTICES)
    return fail(PC_ERR_INVALID_ARG, "grid_type must be PC_GRID_CELLS or PC_GRID_VERTICES");
  const bool vert = d->grid_type == PC_GRID_VERTICES;
  if (vert && d->divergence != PC_DIV_WLS_DIRECT)
    return fail(PC_ERR_UNSUPPORTED, "a vertex pressure grid has no faces: it needs PC_DIV_WLS_DIRECT");
  long long ncells = 1, nvtot = 1, nftot = 1;
  int vk[3] = {0, 0, 0}, nint[3] = {1, 1, 1}, nv[3] = {1, 1, 1}, vj0[3] = {0, 0, 0}, nf[3] = {1, 1, 1};
  for (int a = 0; a < d->dim; ++a) {
    if (d->n[a] < 4 || d->n[a] > 4096) return fail(PC_ERR_INVALID_ARG, "n[%d] must be in [4, 4096]", a);
    if (!(d->h[a] > 0) || !std::isfinite(d->h[a]) || !std::isfinite(d->lo[a]))
      return fail(PC_ERR_INVALID_ARG, "h[%d]/lo[%d] invalid", a, a);
    if (d->bc_lo[a] < 0 || d->bc_lo[a] > 3 || d->bc_hi[a] < 0 || d->bc_hi[a] > 3)
      return fail(PC_ERR_INVALID_ARG, "bad boundary kind on axis %d", a);
    if ((d->bc_lo[a] == PC_BC_PERIODIC) != (d->bc_hi[a] == PC_BC_PERIODIC))
      return fail(PC_ERR_INVALID_ARG, "periodic must pair with periodic (axis %d)", a);
    vk[a] = axis_kind(d->bc_lo[a], d->bc_hi[a]);
    if (vert) {
      vertex_axis(vk[a], (int)d->n[a], nv[a], vj0[a], nf[a]);
      nint[a] = nv[a];
      if (!vertex_axis_supported(vertex_kind(vk[a]), (int)d->n[a]))
        return fail(PC_ERR_UNSUPPORTED, "vertex axis %d of %d cells: N-N and D-D axes need 2^a 3^b 5^c <= 2048 "
                    "cells, the others an even count with half of it 2^a 3^b 5^c <= 2048", a, (int)d->n[a]);
    } else {
      nint[a] = nv[a] = nf[a] = (int)d->n[a];
      if (!axis_length_supported(nint[a]))
        return fail(PC_ERR_UNSUPPORTED, "axis %d: the solve length %d must be even with half of it 2^a 3^b 5^c <= 2048",
                    a, nint[a]);
    }
    ncells *= nint[a];
    nvtot *= nv[a];
    nftot *= nf[a];
  }
  // The kernels number rows (cells, faces, nodes, pressure points) with 32-bit indices and form
  // every offset into the row arrays ([K][rows], [dim][3^dim][N]) in 64 bits; a thread index
  // runs at most one block past the last row, so each row count stays below kMaxRows.
  if (ncells > kMaxRows) return fail(PC_ERR_UNSUPPORTED, "grid of %lld cells: at most %lld", ncells, kMaxRows);
  if (d->num_nodes > kMaxRows)
    return fail(PC_ERR_UNSUPPORTED, "%lld nodes: at most %lld", (long long)d->num_nodes, kMaxRows);
  for (int a = 0; a < d->dim && !vert; ++a) {
    const long long faces = ncells / nint[a] * (nint[a] + 1);
    if (faces > kMaxRows) return fail(PC_ERR_UNSUPPORTED, "%lld faces normal to axis %d: at most %lld", faces, a, kMaxRows);
  }
  if (vert && (nftot > kMaxRows || nvtot > kMaxRows))
    return fail(PC_ERR_UNSUPPORTED, "vertex lattice of %lld points: at most %lld", nftot, kMaxRows);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(PC_ERR_CUDA, "device %d not available", device);
  }
  if (cudaSetDevice(device) != cudaSuccess) return fail(PC_ERR_CUDA, "cannot select device %d", device);

  Plan *p = new Plan();
  p->device = device;
  p->dim = d->dim;
  p->N = d->num_nodes;
  p->K = d->knn;
  p->Kg = d->dim == 2 ? 9 : 27;
  p->eps = d->wls_eps;
  p->support_factor = d->support_factor;
  p->beta = d->beta;
  p->precision = d->precision;
  p->refine_iters = d->refine_iters;
  p->refine_tol = std::isfinite(d->refine_tol) ? d->refine_tol : 0.0;
  p->gauge = d->gauge;
  p->vdtype = d->velocity_dtype;
  p->eigen = d->eigenvalues;
  p->divmode = d->divergence;
  p->ncells = ncells;
  p->singular = true;
  p->vertex = vert;
  p->nvtot = nvtot;
  p->nftot = nftot;
  p->npts = vert ? nvtot : ncells;
  for (int a = 0; a < 3; ++a) {
    p->vkind[a] = vk[a];
    p->vn[a] = a < d->dim ? (int)d->n[a] : 1;
    p->nv[a] = nv[a];
    p->vj0[a] = vj0[a];
    p->nf[a] = nf[a];
  }
  for (int a = 0; a < 3; ++a) {
    p->n[a] = a < d->dim ? d->n[a] : 1;
    p->lo[a] = a < d->dim ? d->lo[a] : 0.0;
    p->h[a] = a < d->dim ? d->h[a] : 1.0;
    p->bc_lo[a] = a < d->dim ? d->bc_lo[a] : 0;
    p->bc_hi[a] = a < d->dim ? d->bc_hi[a] : 0;
  }
  for (int a = 0; a < d->dim; ++a) {
    AxisInfo &ax = p->ax[a];
    ax.n = (int)d->n[a];
    ax.h = d->h[a];
    ax.L = (double)d->n[a] * d->h[a];
    ax.periodic = d->bc_lo[a] == PC_BC_PERIODIC;
    ax.nfaces = ax.periodic ? ax.n : ax.n + 1;
    ax.bc_lo = d->bc_lo[a];
    ax.bc_hi = d->bc_hi[a];
    ax.kind = axis_kind(d->bc_lo[a], d->bc_hi[a]);
    if (d->bc_lo[a] == PC_BC_DIRICHLET || d->bc_hi[a] == PC_BC_DIRICHLET) p->singular = false;
  }
  p->problem_singular = p->singular;
  for (int a = 0; a < d->dim; ++a) {
    p->phys_L[a] = p->ax[a].L;
    p->phys_periodic[a] = p->ax[a].periodic;
  }
  for (int a = 0; a < d->dim; ++a) {
    long long rows = 1;
    for (int b = 0; b < d->dim; ++b) rows *= (b == a) ? p->ax[b].nfaces : p->ax[b].n;
    p->nface_total[a] = vert ? 0 : rows;   // a vertex grid has no faces
  }
  auto bail = [&](pc_status s) { destroy_plan(p); return s; };

  // Memory plan (all of it up front: pc_project allocates nothing).
  const bool mixed = p->precision != PC_PREC_FP64;
  const long long N = p->N, K = p->K, nc = ncells;
  const int dd = p->dim;
  size_t need = 0;
  // weights: FP64 in FP64 plans, FP32 (hi, lo) pairs in mixed and FP32 plans (8 bytes either way)
  for (int a = 0; a < dd; ++a) need += (size_t)p->nface_total[a] * (K * (4 + 8) + 8);
  const long long Kg = p->Kg;
  need += (size_t)N * Kg * (4 + dd * 8) + N;
  need += (size_t)nc * (8 + 8 + 4 + (mixed ? 8 : 0) + 8 + 8);
  if (vert && nftot > nc) need += (size_t)(nftot - nc) * (mixed ? 16 : 8);   // lattice copies of p
  need += (size_t)dd * N * 8;
  need += (size_t)dd * N * 8;                             // node coordinates (setup only)
  if (p->divmode == PC_DIV_WLS_DIRECT) need += (size_t)p->npts * K * (4 + dd * 8);   // point rows
  if (budget && need > budget)
    return bail(fail(PC_ERR_BUDGET, "plan needs %zu bytes, budget is %zu", need, budget));

  // read-only rows (shared with clones)
  for (int a = 0; a < dd; ++a) {
    long long rows = p->nface_total[a];
    if (plan_alloc(p, (void **)&p->fcol[a], rows * K * 4) != PC_OK ||
        (!mixed && plan_alloc(p, (void **)&p->fw64[a], rows * K * 8) != PC_OK))
      return bail(PC_ERR_OUT_OF_MEMORY);
    if (mixed && plan_alloc(p, (void **)&p->fw2[a], rows * K * 8) != PC_OK) return bail(PC_ERR_OUT_OF_MEMORY);
  }
  if (plan_alloc(p, (void **)&p->ncol, N * Kg * 4) != PC_OK ||
      (!mixed && plan_alloc(p, (void **)&p->nD64, dd * N * Kg * 8) != PC_OK) ||
      (mixed && plan_alloc(p, (void **)&p->nD2, dd * N * Kg * 8) != PC_OK) ||
      plan_alloc(p, (void **)&p->ntype, N) != PC_OK)
    return bail(PC_ERR_OUT_OF_MEMORY);
  const long long np = p->npts;
  if (p->divmode == PC_DIV_WLS_DIRECT &&
      (plan_alloc(p, (void **)&p->ccol, np * K * 4) != PC_OK ||
       (!mixed && plan_alloc(p, (void **)&p->cD64, dd * np * K * 8) != PC_OK) ||
       (mixed && plan_alloc(p, (void **)&p->cD2, dd * np * K * 8) != PC_OK)))
    return bail(PC_ERR_OUT_OF_MEMORY);
  {
    pc_status ws = alloc_workspace(p, st);
    if (ws != PC_OK) return bail(ws);
  }
  // node coordinates and types on the device
  double *xyz_dev = nullptr;
  if (plan_alloc(p, (void **)&xyz_dev, dd * N * 8) != PC_OK) return bail(PC_ERR_OUT_OF_MEMORY);
  cudaMemcpyKind k1 = host_ptr(d->node_xyz) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaMemcpyKind k2 = host_ptr(d->node_type) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (cudaMemcpyAsync(xyz_dev, d->node_xyz, dd * N * 8, k1, st) != cudaSuccess ||
      cudaMemcpyAsync(p->ntype, d->node_type, N, k2, st) != cudaSuccess)
    return bail(fail(PC_ERR_CUDA, "copy of node arrays failed"));
  {
    unsigned int *bad = reinterpret_cast<unsigned int *>(p->dstats);
    cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
    check_nodes_kernel<<<grid_for(N, 256), 256, 0, st>>>(xyz_dev, p->ntype, N, dd, p->lo[0], p->lo[1], p->lo[2],
                                                         p->ax[0].L, p->ax[1].L, dd > 2 ? p->ax[2].L : 1.0,
                                                         p->ax[0].periodic, p->ax[1].periodic,
                                                         dd > 2 ? (int)p->ax[2].periodic : 0, bad);
    unsigned int hb = 0;
    if (cudaMemcpyAsync(&hb, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return bail(fail(PC_ERR_CUDA, "node validation failed: %s", cudaGetErrorString(cudaGetLastError())));
    if (hb & 1u) return bail(fail(PC_ERR_INVALID_ARG, "a node lies outside the domain or is not finite"));
    if (hb & 2u) return bail(fail(PC_ERR_INVALID_ARG, "node_type values must be 0, 1 or 2"));
  }
  if (prepare_kernels() != PC_OK) return bail(PC_ERR_CUDA);
  // rows on the physical grid, then (vertex plans) the transform axes of the unknowns
  pc_status s = build_rows(p, xyz_dev, st);
  if (s != PC_OK) return bail(s);
  if (vert) vertex_switch_axes(p);
  s = build_axis_tables(p);
  if (s != PC_OK) return bail(s);
  cudaStreamSynchronize(st);
  plan_free(p, xyz_dev, (size_t)dd * N * 8);
  *out = p;
  return PC_OK;
}


// Grid-only plan: the transform tables and the cell workspace, no nodes. A vertex grid is
// solved on its unknowns (n + 1 on N-N axes, n - 1 on D-D axes, n otherwise) with the vertex
// transforms.
static pc_status create_grid(const pc_grid_desc *d, int device, cudaStream_t st, Plan **out) {
  if (!d || !out) return fail(PC_ERR_INVALID_ARG, "desc and out_plan are required");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(PC_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (d->grid_type != PC_GRID_CELLS && d->grid_type != PC_GRID_VERTICES) return fail(PC_ERR_INVALID_ARG, "bad grid_type");
  if (d->precision < PC_PREC_FP64 || d->precision > PC_PREC_FP32) return fail(PC_ERR_INVALID_ARG, "bad precision");
  if (d->refine_iters < 0 || d->refine_iters > kMaxRefine) return fail(PC_ERR_INVALID_ARG, "refine_iters in [0, %d]", kMaxRefine);
  if (d->gauge != 0 && d->gauge != 1) return fail(PC_ERR_INVALID_ARG, "gauge must be 0 or 1");
  if (d->eigenvalues != PC_EIG_FD && d->eigenvalues != PC_EIG_SPECTRAL)
    return fail(PC_ERR_INVALID_ARG, "eigenvalues must be PC_EIG_FD or PC_EIG_SPECTRAL");
  if (d->eigenvalues == PC_EIG_SPECTRAL && d->precision == PC_PREC_MIXED)
    return fail(PC_ERR_UNSUPPORTED, "pseudo-spectral eigenvalues need precision FP64 or FP32");
  const bool vert = d->grid_type == PC_GRID_VERTICES;
  long long ncells = 1, nvtot = 1;
  int nint[3] = {1, 1, 1}, nv[3] = {1, 1, 1}, vk[3] = {0, 0, 0};
  bool psing = true;
  for (int a = 0; a < d->dim; ++a) {
    if (d->n[a] < 4 || d->n[a] > 4096) return fail(PC_ERR_INVALID_ARG, "n[%d] must be in [4, 4096]", a);
    if (!(d->h[a] > 0) || !std::isfinite(d->h[a])) return fail(PC_ERR_INVALID_ARG, "h[%d] invalid", a);
    if (d->bc_lo[a] < 0 || d->bc_lo[a] > 3 || d->bc_hi[a] < 0 || d->bc_hi[a] > 3)
      return fail(PC_ERR_INVALID_ARG, "bad boundary kind on axis %d", a);
    if ((d->bc_lo[a] == PC_BC_PERIODIC) != (d->bc_hi[a] == PC_BC_PERIODIC))
      return fail(PC_ERR_INVALID_ARG, "periodic must pair with periodic (axis %d)", a);
    if (d->bc_lo[a] == PC_BC_DIRICHLET || d->bc_hi[a] == PC_BC_DIRICHLET) psing = false;
    const int n = (int)d->n[a];
    vk[a] = axis_kind(d->bc_lo[a], d->bc_hi[a]);
    if (vert) {
      int j0, nlat;
      vertex_axis(vk[a], n, nv[a], j0, nlat);
      nint[a] = nv[a];
      if (!vertex_axis_supported(vertex_kind(vk[a]), n))
        return fail(PC_ERR_UNSUPPORTED, "vertex axis %d of %d cells: N-N and D-D axes need 2^a 3^b 5^c <= 2048 "
                    "cells, the others an even count with half of it 2^a 3^b 5^c <= 2048", a, n);
    } else {
      nint[a] = nv[a] = n;
      if (!axis_length_supported(nint[a]))
        return fail(PC_ERR_UNSUPPORTED, "axis %d: the solve length %d must be even with half of it 2^a 3^b 5^c <= 2048",
                    a, nint[a]);
    }
    ncells *= nint[a];
    nvtot *= nv[a];
  }
  if (ncells > kMaxRows) return fail(PC_ERR_UNSUPPORTED, "grid of %lld cells: at most %lld", ncells, kMaxRows);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(PC_ERR_CUDA, "device %d not available", device);
  }
  if (cudaSetDevice(device) != cudaSuccess) return fail(PC_ERR_CUDA, "cannot select device %d", device);

  Plan *p = new Plan();
  p->device = device;
  p->grid_only = true;
  p->vertex = vert;
  p->dim = d->dim;
  p->N = 0;
  p->Kg = d->dim == 2 ? 9 : 27;
  p->precision = d->precision;
  p->refine_iters = d->refine_iters;
  p->refine_tol = std::isfinite(d->refine_tol) ? d->refine_tol : 0.0;
  p->gauge = d->gauge;
  p->vdtype = PC_DTYPE_F64;
  p->eigen = d->eigenvalues;
  p->ncells = ncells;
  p->problem_singular = psing;
  p->singular = psing;
  p->nvtot = nvtot;
  for (int a = 0; a < 3; ++a) {
    const bool on = a < d->dim;
    p->n[a] = on ? nint[a] : 1;
    p->lo[a] = 0.0;
    p->h[a] = on ? d->h[a] : 1.0;
    p->bc_lo[a] = on ? d->bc_lo[a] : 0;
    p->bc_hi[a] = on ? d->bc_hi[a] : 0;
    p->vkind[a] = vk[a];
    p->vn[a] = on ? (int)d->n[a] : 1;
    p->nv[a] = nv[a];
    if (on && vert) {
      int nunk;
      vertex_axis(vk[a], (int)d->n[a], nunk, p->vj0[a], p->nf[a]);
    }
  }
  p->nftot = 1;
  for (int a = 0; a < d->dim; ++a) p->nftot *= p->nf[a];
  for (int a = 0; a < d->dim; ++a) {
    AxisInfo &ax = p->ax[a];
    ax.n = nint[a];
    ax.h = d->h[a];
    ax.L = (double)nint[a] * d->h[a];
    ax.bc_lo = p->bc_lo[a];
    ax.bc_hi = p->bc_hi[a];
    ax.periodic = ax.bc_lo == PC_BC_PERIODIC;
    ax.nfaces = ax.periodic ? ax.n : ax.n + 1;
    ax.kind = vert ? vertex_kind(vk[a]) : axis_kind(ax.bc_lo, ax.bc_hi);
    p->nface_total[a] = 0;   // no faces: the plan has no transfer
  }
  auto bail = [&](pc_status s) { destroy_plan(p); return s; };
  pc_status s = alloc_workspace(p, st);
  if (s != PC_OK) return bail(s);
  if (prepare_kernels() != PC_OK) return bail(PC_ERR_CUDA);
  s = build_axis_tables(p);
  if (s != PC_OK) return bail(s);
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(PC_ERR_CUDA, "grid plan setup failed"));
  *out = p;
  return PC_OK;
}

}  // namespace pc

extern "C" pc_status pc_grid_plan_create(const pc_grid_desc *desc, int device, void *cuda_stream, pc_plan **out_plan) {
  if (!out_plan) return pc::fail(PC_ERR_INVALID_ARG, "out_plan is required");
  pc::Plan *p = nullptr;
  pc_status s = pc::create_grid(desc, device, (cudaStream_t)cuda_stream, &p);
  if (s == PC_OK) *out_plan = reinterpret_cast<pc_plan *>(p);
  return s;
}

extern "C" pc_status pc_plan_create(const pc_problem_desc *desc, int device, size_t hbm_budget_bytes,
                                    void *cuda_stream, pc_plan **out_plan) {
  pc::Plan *p = nullptr;
  pc_status s = pc::create(desc, device, hbm_budget_bytes, (cudaStream_t)cuda_stream, &p);
  if (s == PC_OK) *out_plan = reinterpret_cast<pc_plan *>(p);
  return s;
}

extern "C" pc_status pc_destroy(pc_plan *plan) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return PC_OK;
  if (p->clones > 0) return pc::fail(PC_ERR_INVALID_ARG, "the plan has %d live clones: destroy them first", p->clones);
  if (p->root) p->root->clones--;
  pc::destroy_plan(p);
  return PC_OK;
}

extern "C" pc_status pc_plan_clone(pc_plan *plan, void *cuda_stream, pc_plan **out_plan) {
  using namespace pc;
  Plan *src = reinterpret_cast<Plan *>(plan);
  if (!src || !out_plan) return fail(PC_ERR_INVALID_ARG, "plan and out_plan are required");
  if (src->grid_only) return fail(PC_ERR_INVALID_ARG, "grid-only plans are not cloned");
  *out_plan = nullptr;
  Plan *root = src->root ? src->root : src;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cudaSetDevice(root->device) != cudaSuccess) return fail(PC_ERR_CUDA, "cannot select device %d", root->device);
  Plan *p = new Plan();
  p->device = root->device;
  p->dim = root->dim;
  for (int a = 0; a < 3; ++a) {
    p->n[a] = root->n[a]; p->lo[a] = root->lo[a]; p->h[a] = root->h[a];
    p->bc_lo[a] = root->bc_lo[a]; p->bc_hi[a] = root->bc_hi[a];
    p->ax[a] = root->ax[a];                       // tables borrowed; schedule copied
    p->nface_total[a] = root->nface_total[a];
    p->fcol[a] = root->fcol[a]; p->fw64[a] = root->fw64[a]; p->fw2[a] = root->fw2[a];
  }
  p->N = root->N; p->K = root->K; p->Kg = root->Kg;
  p->eps = root->eps; p->support_factor = root->support_factor; p->beta = root->beta;
  p->precision = root->precision; p->refine_iters = root->refine_iters; p->refine_tol = root->refine_tol;
  p->gauge = root->gauge;
  p->vdtype = root->vdtype; p->singular = root->singular; p->ncells = root->ncells;
  p->eigen = root->eigen;
  p->divmode = root->divmode; p->ccol = root->ccol; p->cD64 = root->cD64; p->cD2 = root->cD2;
  p->ncol = root->ncol; p->nD64 = root->nD64; p->nD2 = root->nD2; p->ntype = root->ntype;
  p->graphs_on = root->graphs_on;
  p->vertex = root->vertex; p->problem_singular = root->problem_singular;
  p->nvtot = root->nvtot; p->nftot = root->nftot; p->npts = root->npts;
  for (int a = 0; a < 3; ++a) { p->phys_L[a] = root->phys_L[a]; p->phys_periodic[a] = root->phys_periodic[a]; }
  for (int a = 0; a < 3; ++a) {
    p->vkind[a] = root->vkind[a]; p->vn[a] = root->vn[a]; p->nv[a] = root->nv[a];
    p->vj0[a] = root->vj0[a]; p->nf[a] = root->nf[a];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  pc_status s = alloc_workspace(p, st);
  if (s == PC_OK && cudaStreamSynchronize(st) != cudaSuccess) s = fail(PC_ERR_CUDA, "clone setup failed");
  if (s != PC_OK) {
    destroy_plan(p);
    if (cur >= 0) cudaSetDevice(cur);
    return s;
  }
  p->root = root;
  root->clones++;
  if (cur >= 0) cudaSetDevice(cur);
  *out_plan = reinterpret_cast<pc_plan *>(p);
  return PC_OK;
}

extern "C" pc_status pc_profile_enable(pc_plan *plan, int on) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device");
  if (on && !p->slots) {
    p->slots = new pc::ProfSlot[pc::kProfSlots];
    for (int i = 0; i < pc::kProfSlots; ++i)
      for (int e = 0; e < pc::kProfEvents; ++e)
        if (cudaEventCreate(&p->slots[i].ev[e]) != cudaSuccess)
          return pc::fail(PC_ERR_CUDA, "cudaEventCreate failed");
  }
  p->prof = on != 0;
  p->slots_used = 0;
  p->launches = 0;
  return PC_OK;
}

extern "C" pc_status pc_profile_read(pc_plan *plan, pc_profile *out) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p || !out) return pc::fail(PC_ERR_INVALID_ARG, "plan and out are required");
  memset(out, 0, sizeof(*out));
  if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device");
  for (int i = 0; i < p->slots_used; ++i) {
    pc::ProfSlot &s = p->slots[i];
    if (s.n < 2) continue;
    PC_CUDA_TRY(cudaEventSynchronize(s.ev[s.n - 1]));
    for (int e = 0; e + 1 < s.n; ++e) {
      float ms = 0.f;
      PC_CUDA_TRY(cudaEventElapsedTime(&ms, s.ev[e], s.ev[e + 1]));
      int t = s.tag[e];
      if (t >= 0 && t < 8) out->phase_ms[t] += ms;
    }
    out->calls++;
  }
  out->kernel_launches = p->launches;
  p->slots_used = 0;
  p->launches = 0;
  return PC_OK;
}

extern "C" pc_status pc_set_graphs(pc_plan *plan, int on) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  p->graphs_on = on != 0;
  return PC_OK;
}

extern "C" pc_status pc_plan_bytes(const pc_plan *plan, size_t *bytes_out) {
  const pc::Plan *p = reinterpret_cast<const pc::Plan *>(plan);
  if (!p || !bytes_out) return pc::fail(PC_ERR_INVALID_ARG, "plan and bytes_out are required");
  *bytes_out = p->bytes;
  return PC_OK;
}

extern "C" pc_status pc_plan_rows(const pc_plan *plan, int which, int64_t *rows_out, int32_t *col_out,
                                  double *w_out) {
  const pc::Plan *p = reinterpret_cast<const pc::Plan *>(plan);
  if (!p || !rows_out) return pc::fail(PC_ERR_INVALID_ARG, "plan and rows_out are required");
  if (p->grid_only) return pc::fail(PC_ERR_INVALID_ARG, "a grid-only plan has no WLS rows");
  if (which < 0 || which > p->dim + 1) return pc::fail(PC_ERR_INVALID_ARG, "which must be in [0, dim + 1]");
  if (which == p->dim + 1 && p->divmode != PC_DIV_WLS_DIRECT)
    return pc::fail(PC_ERR_INVALID_ARG, "cell rows exist only in PC_DIV_WLS_DIRECT plans");
  if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cannot select device");
  const bool face = which < p->dim, cell = which == p->dim + 1;
  const long long K = (face || cell) ? p->K : p->Kg;
  long long rows = face ? p->nface_total[which] : (cell ? p->npts : p->N);
  *rows_out = rows;
  if (!col_out && !w_out) return PC_OK;
  // stored neighbour-rank major on the device; returned row major
  std::vector<int32_t> c(rows * K);
  std::vector<double> w((face ? 1 : p->dim) * rows * K);
  const int32_t *dc = face ? p->fcol[which] : (cell ? p->ccol : p->ncol);
  const double *dw = face ? p->fw64[which] : (cell ? p->cD64 : p->nD64);
  PC_CUDA_TRY(cudaMemcpy(c.data(), dc, c.size() * 4, cudaMemcpyDeviceToHost));
  if (dw) {
    PC_CUDA_TRY(cudaMemcpy(w.data(), dw, w.size() * 8, cudaMemcpyDeviceToHost));
  } else {
    // MIXED / FP32 plans keep the weights as FP32 (hi, lo) pairs only
    const float2 *d2 = face ? p->fw2[which] : (cell ? p->cD2 : p->nD2);
    std::vector<float2> w2(w.size());
    PC_CUDA_TRY(cudaMemcpy(w2.data(), d2, w2.size() * sizeof(float2), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < w.size(); ++i) w[i] = (double)w2[i].x + (double)w2[i].y;
  }
  const long long nw = face ? 1 : p->dim;
  for (long long r = 0; r < rows; ++r)
    for (long long k = 0; k < K; ++k) {
      if (col_out) col_out[r * K + k] = c[k * rows + r];
      if (w_out)
        for (long long a = 0; a < nw; ++a) w_out[(a * rows + r) * K + k] = w[(a * K + k) * rows + r];
    }
  return PC_OK;
}

extern "C" const char *pc_status_string(pc_status s) {
  switch (s) {
    case PC_OK: return "ok";
    case PC_ERR_INVALID_ARG: return "invalid argument";
    case PC_ERR_UNSUPPORTED: return "unsupported";
    case PC_ERR_WLS_SINGULAR: return "singular WLS system";
    case PC_ERR_OUT_OF_MEMORY: return "out of device memory";
    case PC_ERR_BUDGET: return "device-memory budget exceeded";
    case PC_ERR_CUDA: return "CUDA error";
    case PC_ERR_NOT_CONVERGED: return "refinement not converged";
    case PC_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

extern "C" const char *pc_last_error_message(void) { return pc::g_err; }
