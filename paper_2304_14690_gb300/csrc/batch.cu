// pc_project_batch: many independent projections with one launch per pipeline stage.
//
// Problems of a batch are grouped by (dimension, velocity type, neighbour count, refinement
// settings) among plans in mixed or FP32 precision. For each group every per-cell and per-node
// stage of the pipeline (prep, transfer per axis, divergence, residuals, gauge, split, gradient)
// is ONE kernel launch over all problems of the group: a segment table maps each block to its
// problem and problem-local block. Each transform pass is ONE launch over the problems of every
// group, 2D and 3D, all transform families and line lengths together: each CTA takes one item
// of a work list of (pass arguments, tile) items. The whole sequence is captured once per
// batch composition into a CUDA graph and replayed. Each problem keeps the block decomposition
// of its single-problem launches and each line is transformed as in a single call, so batch
// results are bitwise those of separate pc_project calls. Plans in FP64 precision, and plans
// with the direct WLS divergence, run one by one through pc_project.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "passes.cuh"
#include "pc_internal.cuh"

namespace pc {

namespace {

constexpr int kBatchThreads = 256;   // CTA size of the batched transform passes
constexpr int kBatchChunk = 4;       // tiles of one problem per CTA of a batched pass

// One launch of a batched transform pass: its items in the work list, over every problem of the
// batch that has this pass (any family, line length and dimension).
struct PassLaunch {
  int items_off = 0;
  int nitems = 0;
  int emax = 1;          // largest slots per thread among the items' passes (kernel instance)
  size_t smem = 0;       // the pass body's shared memory (the largest item's)
  int lean = 0;          // 0: general passes; else the lean kernel id (lean_pass.cuh)
  int pass = 0;          // the pass of the solve: launches of one pass run side by side
};

// Auxiliary streams and events that run the launches of one batched pass side by side (they
// transform disjoint problems), joined back into the caller's stream before the next pass. In a
// captured graph they become parallel branches.
constexpr int kForkWays = 6;
struct Fork {
  cudaStream_t aux[kForkWays] = {};
  cudaEvent_t fork = nullptr, join[kForkWays] = {};
};

pc_status fork_create(Fork &f) {
  for (int i = 0; i < kForkWays; ++i) {
    PC_CUDA_TRY(cudaStreamCreateWithFlags(&f.aux[i], cudaStreamNonBlocking));
    PC_CUDA_TRY(cudaEventCreateWithFlags(&f.join[i], cudaEventDisableTiming));
  }
  PC_CUDA_TRY(cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming));
  return PC_OK;
}

void fork_destroy(Fork &f) {
  for (int i = 0; i < kForkWays; ++i) {
    if (f.aux[i]) cudaStreamDestroy(f.aux[i]);
    if (f.join[i]) cudaEventDestroy(f.join[i]);
    f.aux[i] = nullptr;
    f.join[i] = nullptr;
  }
  if (f.fork) cudaEventDestroy(f.fork);
  f.fork = nullptr;
}

// Problems that share the templated per-stage kernels (dimension, velocity type, neighbour
// count) and the refinement settings.
struct Group {
  std::vector<int> members;
  int dim = 2, vdtype = 0, K = 12, sweeps = 0;
  bool adaptive = false;   // refinement with the device-side stopping rule (refine_tol > 0)
  int total[BATCH_STAGES] = {0};
  BatchProblem *dP = nullptr;
  int *dseg = nullptr;                  // BATCH_STAGES x (n + 1)
  bool any_singular = false;
};

// Table space of one batch in a pinned host buffer and its device copy (the batch executor):
// tables are appended at 256-byte boundaries and copied with one asynchronous transfer.
struct Arena {
  char *host = nullptr;
  char *dev = nullptr;
  size_t cap = 0, used = 0;
};

struct Exec {
  Arena *arena = nullptr;               // set: tables go to the arena, no allocation
  std::vector<Plan *> plans;
  std::vector<pc_project_args> args;
  std::vector<Group> groups;
  std::vector<int> singles;             // problems run through pc_project
  PassArgs<float> *dargs = nullptr;     // transform passes of every problem and solve
  int4 *ditems = nullptr;               // work list: (args index, first tile, tiles, 0)
  std::vector<std::vector<PassLaunch>> passes;   // [solve][pass]
  cudaStream_t cap = nullptr;
  Fork own;                             // streams of the side-by-side pass launches (cached executors)
  Fork *fork = nullptr;                 // the streams used: own, or the batch executor's
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void *> allocs;
  unsigned long long stamp = 0;
  int device = 0;
};

std::mutex g_mutex;
std::vector<Exec *> g_cache;
unsigned long long g_clock = 0;
constexpr size_t kMaxExecs = 8;

void free_exec(Exec *e) {
  if (!e) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(e->device);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  if (e->cap) cudaStreamDestroy(e->cap);
  fork_destroy(e->own);
  for (void *a : e->allocs) cudaFree(a);
  if (cur >= 0) cudaSetDevice(cur);
  delete e;
}

bool same_args(const pc_project_args &a, const pc_project_args &b) {
  return a.dt == b.dt && a.u_star == b.u_star && a.f_ib_in == b.f_ib_in && a.p_out == b.p_out &&
         a.u_out == b.u_out && a.f_ib_out == b.f_ib_out;
}

template <typename T>
pc_status upload(Exec *e, T **dptr, const std::vector<T> &host) {
  size_t bytes = std::max<size_t>(host.size() * sizeof(T), 16);
  if (e->arena) {
    Arena &a = *e->arena;
    const size_t off = (a.used + 255) & ~(size_t)255;
    if (off + bytes > a.cap)
      return fail(PC_ERR_BUDGET, "batch tables need more than the executor's %zu bytes per batch", a.cap);
    if (!host.empty()) memcpy(a.host + off, host.data(), host.size() * sizeof(T));
    *dptr = reinterpret_cast<T *>(a.dev + off);
    a.used = off + bytes;
    return PC_OK;
  }
  if (cudaMalloc(reinterpret_cast<void **>(dptr), bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(PC_ERR_OUT_OF_MEMORY, "batch table allocation of %zu bytes failed", bytes);
  }
  e->allocs.push_back(*dptr);
  if (!host.empty()) PC_CUDA_TRY(cudaMemcpy(*dptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PC_OK;
}

bool batchable(const Plan *p) {
  return (p->precision == PC_PREC_MIXED || p->precision == PC_PREC_FP32) && p->divmode == PC_DIV_FACES;
}

// Per-problem tables of one group: problem descriptions and the block segments of each stage.
pc_status build_group(Exec *e, Group &g) {
  const int n = (int)g.members.size();
  std::vector<BatchProblem> hp(n);
  std::vector<int> seg((size_t)BATCH_STAGES * (n + 1), 0);
  for (int i = 0; i < n; ++i) {
    const Plan *p = e->plans[g.members[i]];
    batch_problem_fill(p, e->args[g.members[i]], hp[i]);
    g.any_singular = g.any_singular || p->singular;
    int nb[BATCH_STAGES];
    batch_block_counts(p, nb);
    for (int s = 0; s < BATCH_STAGES; ++s) seg[(size_t)s * (n + 1) + i + 1] = seg[(size_t)s * (n + 1) + i] + nb[s];
  }
  for (int s = 0; s < BATCH_STAGES; ++s) g.total[s] = seg[(size_t)s * (n + 1) + n];
  PC_TRY(upload(e, &g.dP, hp));
  PC_TRY(upload(e, &g.dseg, seg));
  return PC_OK;
}

// The transform passes of every problem of every group: pass k of solve j of all problems that
// have it is one launch, its items sorted by transform family, power-of-two length
// and line length so the CTAs resident together run the same code.
pc_status build_passes(Exec *e) {
  int jmax = -1;
  for (const Group &g : e->groups) jmax = std::max(jmax, g.sweeps);
  std::vector<PassArgs<float>> args;
  std::vector<int4> items;
  for (int j = 0; j <= jmax; ++j) {
    // pass specs of solve j of every problem that runs it
    std::vector<std::pair<const Plan *, std::vector<PassSpec>>> specs;
    size_t npass = 0;
    for (const Group &g : e->groups) {
      if (g.sweeps < j) continue;
      for (int m : g.members) {
        Plan *p = e->plans[m];
        const void *src = reinterpret_cast<const float *>(p->work64);
        // the iterate is kept in p2 as (hi, lo) pairs; the last solve also writes p in FP64 (as
        // single calls do), and with the stopping rule every solve does (any may be the last)
        // and the sweeps' passes skip once the rule stopped
        double *f64 = (j == g.sweeps || g.adaptive) ? e->args[m].p_out : nullptr;
        const RefineGate gate = (g.adaptive && j > 0) ? RefineGate{p->dstats, j, (float)p->refine_tol}
                                                       : RefineGate{nullptr, 0, 0.0f};
        specs.emplace_back(p, solve_pass_specs(p, true, SRC_F32, src, j == 0 ? DST_PAIR_SET : DST_PAIR_ADD, p->p2,
                                               f64, gate));
        npass = std::max(npass, specs.back().second.size());
      }
    }
    std::vector<PassLaunch> launches;
    for (size_t k = 0; k < npass; ++k) {
      struct Entry { long long key; int ai; long long tiles; };
      // one launch per kernel: the general passes, and the lean passes of each lean kernel
      std::vector<Entry> list[7];
      PassLaunch pl[7];
      for (const auto &ps : specs) {
        if (k >= ps.second.size()) continue;
        PassArgs<float> A;
        long long tiles;
        int threads;
        size_t smem;
        PC_TRY(build_pass<float>(ps.first, ps.second[k], A, tiles, threads, smem, kBatchThreads));
        const bool pow2 = (A.M & (A.M - 1)) == 0;
        const long long key = ((long long)pass_family(A.kind) * 2 + (pow2 ? 0 : 1)) * 65536 + (65535 - A.M);
        const int c = A.lean;
        list[c].push_back(Entry{key, (int)args.size(), tiles});
        args.push_back(A);
        pl[c].smem = std::max(pl[c].smem, smem);
        pl[c].emax = std::max(pl[c].emax, A.emax);
        pl[c].lean = c;
        pl[c].pass = (int)k;
      }
      for (int c = 0; c < 7; ++c) {
        if (list[c].empty()) continue;
        std::stable_sort(list[c].begin(), list[c].end(), [](const Entry &a, const Entry &b) { return a.key < b.key; });
        pl[c].items_off = (int)items.size();
        // consecutive tiles of a problem per CTA: kBatchChunk small tiles of the general passes,
        // one (larger) tile of the lean passes
        // (sweeps from the third on, which the stopping rule usually skips: 8 tiles per CTA)
        const int chunk = c == 0 ? kBatchChunk : (j >= 3 ? 8 : 1);
        for (const Entry &en : list[c])
          for (long long t = 0; t < en.tiles; t += chunk)
            items.push_back(make_int4(en.ai, (int)t, (int)std::min<long long>(chunk, en.tiles - t), 0));
        pl[c].nitems = (int)items.size() - pl[c].items_off;
        launches.push_back(pl[c]);
      }
    }
    e->passes.push_back(launches);
  }
  PC_TRY(upload(e, &e->dargs, args));
  PC_TRY(upload(e, &e->ditems, items));
  return PC_OK;
}

// The whole batch on one stream: the per-group stages, and one launch per transform
// pass for every group. prof (nullable): a plan whose profiler records the phase boundaries
// (direct launches only, not under capture), with the phase tags of pc_profile_read.
pc_status record_exec(Exec *e, cudaStream_t st, Plan *prof = nullptr) {
  long long launches = 0;
  auto mark = [&](int tag) { if (prof) prof_mark(prof, st, tag); };
  auto segs = [](const Group &g, int s) { return g.dseg + (size_t)s * (g.members.size() + 1); };
  if (prof) prof_begin(prof, st);
  for (const Group &g : e->groups) {
    const int n = (int)g.members.size();
    batch_launch(BATCH_ZERO, 0, g.dP, nullptr, n, n, 0, st);
    batch_launch(BATCH_PREP, g.vdtype, g.dP, segs(g, BATCH_PREP), n, g.total[BATCH_PREP], 0, st);
    launches += 2;
  }
  mark(0);
  for (const Group &g : e->groups)
    for (int a = 0; a < g.dim; ++a) {
      const int n = (int)g.members.size();
      batch_launch(BATCH_TRANSFER, g.K, g.dP, segs(g, BATCH_TRANSFER + a), n, g.total[BATCH_TRANSFER + a], a, st);
      ++launches;
    }
  mark(1);
  for (const Group &g : e->groups) {
    const int n = (int)g.members.size();
    batch_launch(BATCH_DIVERGENCE, g.dim, g.dP, segs(g, BATCH_DIVERGENCE), n, g.total[BATCH_DIVERGENCE], 0, st);
    ++launches;
  }
  mark(2);
  for (size_t j = 0; j < e->passes.size(); ++j) {
    if (j > 0) {
      for (const Group &g : e->groups) {
        if (g.sweeps < (int)j) continue;
        const int n = (int)g.members.size();
        batch_launch(BATCH_RESIDUAL, g.dim, g.dP, segs(g, BATCH_RESIDUAL), n, g.total[BATCH_RESIDUAL], (int)j - 1, st);
        ++launches;
      }
      mark(4);
    }
    // the launches of one pass (one per kernel) side by side, then joined
    const std::vector<PassLaunch> &pv = e->passes[j];
    for (size_t a = 0; a < pv.size();) {
      size_t b = a + 1;
      while (b < pv.size() && pv[b].pass == pv[a].pass) ++b;
      const int ways = (int)(b - a);
      const bool side = e->fork && ways > 1 && ways <= kForkWays + 1;
      if (side) PC_CUDA_TRY(cudaEventRecord(e->fork->fork, st));
      for (size_t i = a; i < b; ++i) {
        const PassLaunch &pl = pv[i];
        cudaStream_t ls = st;
        if (side && i > a) {
          ls = e->fork->aux[i - a - 1];
          PC_CUDA_TRY(cudaStreamWaitEvent(ls, e->fork->fork, 0));
        }
        if (pl.lean) {
          PassArgs<float> none;
          memset(&none, 0, sizeof(none));
          PC_TRY(launch_lean(pl.lean, none, e->dargs, e->ditems + pl.items_off, (unsigned)pl.nitems, kBatchThreads, pl.smem, ls));
        } else {
          PC_TRY(launch_batched_f32(e->dargs, e->ditems + pl.items_off, pl.nitems, kBatchThreads, pl.smem, pl.emax, ls));
        }
        if (side && i > a) PC_CUDA_TRY(cudaEventRecord(e->fork->join[i - a - 1], ls));
        ++launches;
      }
      if (side)
        for (size_t i = a + 1; i < b; ++i) PC_CUDA_TRY(cudaStreamWaitEvent(st, e->fork->join[i - a - 1], 0));
      a = b;
    }
    mark(3);
  }
  for (const Group &g : e->groups) {
    const int n = (int)g.members.size();
    if (g.any_singular) {
      batch_launch(BATCH_GAUGE_SUM, 0, g.dP, segs(g, BATCH_GAUGE_SUM), n, g.total[BATCH_GAUGE_SUM], 0, st);
      ++launches;
    }
    batch_launch(BATCH_FINALIZE, 0, g.dP, segs(g, BATCH_FINALIZE), n, g.total[BATCH_FINALIZE], 0, st);
    ++launches;
  }
  mark(5);
  for (const Group &g : e->groups) {
    const int n = (int)g.members.size();
    batch_launch(BATCH_GRADIENT, g.dim * 10 + g.vdtype, g.dP, segs(g, BATCH_GRADIENT), n, g.total[BATCH_GRADIENT], 0,
                 st);
    ++launches;
  }
  mark(6);
  if (prof) count_launch(prof, launches);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

// Groups of the batch and their device tables (no capture).
pc_status build_groups(Exec *e) {
  const int count = (int)e->plans.size();
  for (int i = 0; i < count; ++i) {
    Plan *p = e->plans[i];
    if (!batchable(p)) { e->singles.push_back(i); continue; }
    const int sweeps = p->precision == PC_PREC_MIXED ? p->refine_iters : 0;
    const bool adaptive = p->precision == PC_PREC_MIXED && p->refine_tol > 0.0 && sweeps > 0;
    const int K = (p->K == 12 || p->K == 27) ? p->K : 0;
    Group *g = nullptr;
    for (Group &c : e->groups)
      if (c.dim == p->dim && c.vdtype == p->vdtype && c.K == K && c.sweeps == sweeps && c.adaptive == adaptive) g = &c;
    if (!g) {
      e->groups.emplace_back();
      g = &e->groups.back();
      g->dim = p->dim; g->vdtype = p->vdtype; g->K = K; g->sweeps = sweeps; g->adaptive = adaptive;
    }
    g->members.push_back(i);
  }
  for (Group &g : e->groups) PC_TRY(build_group(e, g));
  if (!e->groups.empty()) PC_TRY(build_passes(e));
  return PC_OK;
}

pc_status build_exec(Exec *e) {
  PC_TRY(build_groups(e));
  PC_CUDA_TRY(cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking));
  PC_TRY(fork_create(e->own));
  e->fork = &e->own;
  if (!e->groups.empty()) {
    PC_CUDA_TRY(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
    pc_status s = record_exec(e, e->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->cap, &graph);
    if (s != PC_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return s != PC_OK ? s : fail(PC_ERR_CUDA, "batch capture failed: %s", cudaGetErrorString(ce));
    }
    e->graph = graph;
    PC_CUDA_TRY(cudaGraphInstantiate(&e->exec, graph, 0ULL));
  }
  return PC_OK;
}

}  // namespace

void batch_forget_plan(const Plan *p) {
  std::lock_guard<std::mutex> lock(g_mutex);
  for (size_t i = 0; i < g_cache.size();) {
    Exec *e = g_cache[i];
    if (std::find(e->plans.begin(), e->plans.end(), p) != e->plans.end()) {
      free_exec(e);
      g_cache.erase(g_cache.begin() + i);
    } else {
      ++i;
    }
  }
}

}  // namespace pc

namespace pc {
namespace {

// Checks shared by pc_project_batch and pc_batcher_launch; returns the batch's device.
pc_status validate_batch(int count, pc_plan *const *plans, const pc_project_args *args, int &device) {
  if (count < 0 || (count > 0 && (!plans || !args))) return fail(PC_ERR_INVALID_ARG, "bad batch arguments");
  device = -1;
  for (int i = 0; i < count; ++i) {
    const Plan *p = reinterpret_cast<const Plan *>(plans[i]);
    if (!p) return fail(PC_ERR_INVALID_ARG, "plan %d is NULL", i);
    if (p->grid_only) return fail(PC_ERR_INVALID_ARG, "plan %d is a grid-only plan: it has no nodes to project", i);
    if (!args[i].u_star || !args[i].p_out || !args[i].u_out || !(args[i].dt > 0.0))
      return fail(PC_ERR_INVALID_ARG, "batch entry %d: u_star, p_out, u_out and dt > 0 are required", i);
    if (device < 0) device = p->device;
    if (p->device != device) return fail(PC_ERR_INVALID_ARG, "all plans of a batch must be on one device");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(PC_ERR_INVALID_ARG, "a plan appears twice in one batch");
    for (const void *ptr : {args[i].u_star, args[i].f_ib_in, (const void *)args[i].p_out, (const void *)args[i].u_out,
                            (const void *)args[i].f_ib_out}) {
      if (!ptr) continue;
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
          !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(PC_ERR_INVALID_ARG, "batch entry %d: batched projections take device pointers only", i);
      }
    }
  }
  return PC_OK;
}

pc_status run_singles(const Exec &e, pc_plan *const *plans, const pc_project_args *args, void *stream) {
  for (int i : e.singles) {
    pc_status s = pc_project(plans[i], args[i].dt, args[i].u_star, args[i].f_ib_in, args[i].p_out, args[i].u_out,
                             args[i].f_ib_out, nullptr, stream);
    if (s != PC_OK) return s;
  }
  return PC_OK;
}

// One table slot of the batch executor: pinned host staging, its device copy, and the event
// recorded after the last batch that used it.
struct Slot {
  Arena arena;
  cudaEvent_t done = nullptr;
  bool pending = false;
};

}  // namespace

struct Batcher {
  int device = 0;
  Fork fork;
  std::vector<Slot> slots;
  size_t next = 0;
  std::mutex m;
};

}  // namespace pc

extern "C" pc_status pc_project_batch(int count, pc_plan *const *plans, const pc_project_args *args,
                                      void *cuda_stream) {
  using namespace pc;
  int device = -1;
  PC_TRY(validate_batch(count, plans, args, device));
  if (count == 0) return PC_OK;
  if (cudaSetDevice(device) != cudaSuccess) return fail(PC_ERR_CUDA, "cannot select device %d", device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Exec *e = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    for (Exec *c : g_cache) {
      if ((int)c->plans.size() != count) continue;
      bool same = true;
      for (int i = 0; i < count && same; ++i)
        same = c->plans[i] == reinterpret_cast<Plan *>(plans[i]) && same_args(c->args[i], args[i]);
      if (same) { e = c; break; }
    }
    if (!e) {
      e = new Exec();
      e->device = device;
      for (int i = 0; i < count; ++i) {
        e->plans.push_back(reinterpret_cast<Plan *>(plans[i]));
        e->args.push_back(args[i]);
      }
      pc_status s = build_exec(e);
      if (s != PC_OK) {
        free_exec(e);
        return s;
      }
      if (g_cache.size() >= kMaxExecs) {
        auto old = std::min_element(g_cache.begin(), g_cache.end(),
                                    [](const Exec *a, const Exec *b) { return a->stamp < b->stamp; });
        free_exec(*old);
        g_cache.erase(old);
      }
      g_cache.push_back(e);
    }
    e->stamp = ++g_clock;
  }
  // a batch whose plans include a profiled one runs its stages directly and records their
  // boundaries into the first such plan's profiler (pc_profile_read)
  Plan *prof = nullptr;
  for (int i = 0; i < count && !prof; ++i)
    if (reinterpret_cast<Plan *>(plans[i])->prof) prof = reinterpret_cast<Plan *>(plans[i]);
  if (prof && !e->groups.empty()) {
    PC_TRY(record_exec(e, st, prof));
  } else if (e->exec) {
    PC_CUDA_TRY(cudaGraphLaunch(e->exec, st));
  }
  return run_singles(*e, plans, args, cuda_stream);
}

extern "C" pc_status pc_batcher_create(int device, size_t table_bytes, int slots, pc_batcher **out) {
  using namespace pc;
  if (!out || slots < 1 || slots > 64) return fail(PC_ERR_INVALID_ARG, "out is required and slots must be in [1, 64]");
  *out = nullptr;
  if (table_bytes == 0) table_bytes = (size_t)16 << 20;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cudaSetDevice(device) != cudaSuccess) return fail(PC_ERR_CUDA, "cannot select device %d", device);
  Batcher *b = new Batcher();
  b->device = device;
  b->slots.resize(slots);
  pc_status s = fork_create(b->fork);
  for (Slot &sl : b->slots) {
    if (s != PC_OK) break;
    sl.arena.cap = table_bytes;
    if (cudaMallocHost(reinterpret_cast<void **>(&sl.arena.host), table_bytes) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&sl.arena.dev), table_bytes) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      s = fail(PC_ERR_OUT_OF_MEMORY, "batch executor: %d slots of %zu bytes", slots, table_bytes);
      break;
    }
  }
  if (cur >= 0) cudaSetDevice(cur);
  if (s != PC_OK) {
    pc_batcher_destroy(reinterpret_cast<pc_batcher *>(b));
    return s;
  }
  *out = reinterpret_cast<pc_batcher *>(b);
  return PC_OK;
}

extern "C" pc_status pc_batcher_launch(pc_batcher *batcher, int count, pc_plan *const *plans,
                                       const pc_project_args *args, void *cuda_stream) {
  using namespace pc;
  Batcher *b = reinterpret_cast<Batcher *>(batcher);
  if (!b) return fail(PC_ERR_INVALID_ARG, "batcher is NULL");
  int device = -1;
  PC_TRY(validate_batch(count, plans, args, device));
  if (count == 0) return PC_OK;
  if (device != b->device) return fail(PC_ERR_INVALID_ARG, "plans are on device %d, the executor on %d", device, b->device);
  std::lock_guard<std::mutex> lock(b->m);
  if (cudaSetDevice(device) != cudaSuccess) return fail(PC_ERR_CUDA, "cannot select device %d", device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Slot &sl = b->slots[b->next % b->slots.size()];
  b->next++;
  if (sl.pending) PC_CUDA_TRY(cudaEventSynchronize(sl.done));   // its previous batch still reads it
  sl.pending = false;
  Exec e;
  e.arena = &sl.arena;
  e.arena->used = 0;
  e.device = device;
  e.fork = &b->fork;
  for (int i = 0; i < count; ++i) {
    e.plans.push_back(reinterpret_cast<Plan *>(plans[i]));
    e.args.push_back(args[i]);
  }
  PC_TRY(build_groups(&e));
  if (e.arena->used > 0)
    PC_CUDA_TRY(cudaMemcpyAsync(sl.arena.dev, sl.arena.host, e.arena->used, cudaMemcpyHostToDevice, st));
  Plan *prof = nullptr;
  for (int i = 0; i < count && !prof; ++i)
    if (reinterpret_cast<Plan *>(plans[i])->prof) prof = reinterpret_cast<Plan *>(plans[i]);
  if (!e.groups.empty()) PC_TRY(record_exec(&e, st, prof));
  PC_CUDA_TRY(cudaEventRecord(sl.done, st));
  sl.pending = true;
  return run_singles(e, plans, args, cuda_stream);
}

extern "C" pc_status pc_batcher_destroy(pc_batcher *batcher) {
  using namespace pc;
  Batcher *b = reinterpret_cast<Batcher *>(batcher);
  if (!b) return PC_OK;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  for (Slot &sl : b->slots) {
    if (sl.pending) cudaEventSynchronize(sl.done);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.arena.dev) cudaFree(sl.arena.dev);
    if (sl.arena.host) cudaFreeHost(sl.arena.host);
  }
  fork_destroy(b->fork);
  if (cur >= 0) cudaSetDevice(cur);
  delete b;
  return PC_OK;
}
