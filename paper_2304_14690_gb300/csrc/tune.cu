// Schedule of the transform passes: slots per thread along each axis, set explicitly or chosen by
// timing the plan's own solve (coordinate descent over the axes). The slots fix the threads per
// line and the radix schedule of every pass along the axis (build_pass, poisson.cu); single and
// batched calls of a plan use the same schedule, so their results stay bitwise equal.
#include <cuda_runtime.h>

#include "passes.cuh"
#include "pc.h"
#include "pc_internal.cuh"

namespace pc {

// 0 and 1 (FP32 only): variant 0 or 1 of the lean pass of the axis length where it has one
// (lean_pass.cuh), else 4
static bool valid_slots(int s, bool fp64) { return s == 2 || s == 4 || s == 8 || s == 16 || (s <= 1 && s >= 0 && !fp64); }

static int &slots_ref(Plan *p, int axis, bool fp64) {
  return fp64 ? p->ax[axis].slots64 : p->ax[axis].slots32;
}
static int &ctas_ref(Plan *p, int axis, bool fp64) {
  return fp64 ? p->ax[axis].ctas64 : p->ax[axis].ctas32;
}
static bool valid_ctas(int c) { return c == 1 || c == 2 || c == 4 || c == 8; }

// One solve of the plan's transform precision from s64 into the staging buffer.
static pc_status run_solve(Plan *p, bool fp64, cudaStream_t st) {
  if (fp64) return solve_fp64_grid(p, p->s64, p->stage_p, st);
  return solve_fp32_grid(p, SRC_F64, p->s64, DST_F64_SET, p->stage_p, st);
}

// Milliseconds per solve: two warm-up solves, then the best of three rounds of reps solves.
static pc_status time_solve(Plan *p, bool fp64, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps,
                            float &ms) {
  for (int w = 0; w < 2; ++w) PC_TRY(run_solve(p, fp64, st));
  ms = 1e30f;
  for (int round = 0; round < 3; ++round) {
    PC_CUDA_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) PC_TRY(run_solve(p, fp64, st));
    PC_CUDA_TRY(cudaEventRecord(e1, st));
    PC_CUDA_TRY(cudaEventSynchronize(e1));
    float t = 0.0f;
    PC_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
    if (t / reps < ms) ms = t / reps;
  }
  return PC_OK;
}

static pc_status autotune(Plan *p, cudaStream_t st, double *best_out) {
  const bool fp64 = p->precision == PC_PREC_FP64;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PC_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(PC_ERR_CUDA, "cudaEventCreate failed");
  }
  pc_status status = PC_OK;
  float best = 0.0f;
  const int reps = p->ncells > (1 << 22) ? 3 : (p->ncells > (1 << 18) ? 10 : 30);
  if (cudaMemsetAsync(p->s64, 0, p->ncells * sizeof(double), st) != cudaSuccess)
    status = fail(PC_ERR_CUDA, "cudaMemsetAsync failed");
  if (status == PC_OK) status = time_solve(p, fp64, st, e0, e1, reps, best);
  for (int round = 0; round < 2 && status == PC_OK; ++round) {
    bool changed = false;
    for (int a = 0; a < p->dim && status == PC_OK; ++a) {
      // the two knobs of the axis in turn: slots per thread, then CTAs per SM
      for (int knob = 0; knob < 2; ++knob) {
        int &s = knob == 0 ? slots_ref(p, a, fp64) : ctas_ref(p, a, fp64);
        for (int cand : {0, 1, 2, 4, 8, 16}) {
          if (cand == s || (knob == 0 ? !valid_slots(cand, fp64) : !valid_ctas(cand))) continue;
          const int keep = s;
          s = cand;
          float t = 0.0f;
          const pc_status r = time_solve(p, fp64, st, e0, e1, reps, t);
          if (r != PC_OK) {
            // a schedule the kernels cannot run (a tile too large): not a candidate
            cudaGetLastError();
            s = keep;
            continue;
          }
          if (t < 0.98f * best) {
            best = t;
            changed = true;
          } else {
            s = keep;
          }
        }
      }
    }
    if (!changed) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan_drop_graphs(p);
  if (best_out) *best_out = best;
  return status;
}

}  // namespace pc

extern "C" pc_status pc_plan_set_transform_slots(pc_plan *plan, int axis, pc_precision precision, int slots) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  if (axis < 0 || axis >= p->dim) return pc::fail(PC_ERR_INVALID_ARG, "axis %d out of range", axis);
  if (!pc::valid_slots(slots, precision == PC_PREC_FP64))
    return pc::fail(PC_ERR_INVALID_ARG, "slots must be 2, 4, 8 or 16, or 0 or 1 for FP32 (got %d)", slots);
  pc::slots_ref(p, axis, precision == PC_PREC_FP64) = slots;
  pc::plan_drop_graphs(p);
  return PC_OK;
}

extern "C" pc_status pc_plan_get_transform_slots(const pc_plan *plan, int axis, pc_precision precision,
                                                 int *slots_out) {
  pc::Plan *p = const_cast<pc::Plan *>(reinterpret_cast<const pc::Plan *>(plan));
  if (!p || !slots_out) return pc::fail(PC_ERR_INVALID_ARG, "plan and slots_out are required");
  if (axis < 0 || axis >= p->dim) return pc::fail(PC_ERR_INVALID_ARG, "axis %d out of range", axis);
  *slots_out = pc::slots_ref(p, axis, precision == PC_PREC_FP64);
  return PC_OK;
}

extern "C" pc_status pc_plan_set_transform_ctas(pc_plan *plan, int axis, pc_precision precision, int ctas_per_sm) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  if (axis < 0 || axis >= p->dim) return pc::fail(PC_ERR_INVALID_ARG, "axis %d out of range", axis);
  if (!pc::valid_ctas(ctas_per_sm)) return pc::fail(PC_ERR_INVALID_ARG, "ctas_per_sm must be 1, 2, 4 or 8 (got %d)", ctas_per_sm);
  pc::ctas_ref(p, axis, precision == PC_PREC_FP64) = ctas_per_sm;
  pc::plan_drop_graphs(p);
  return PC_OK;
}

extern "C" pc_status pc_plan_get_transform_ctas(const pc_plan *plan, int axis, pc_precision precision,
                                                int *ctas_out) {
  pc::Plan *p = const_cast<pc::Plan *>(reinterpret_cast<const pc::Plan *>(plan));
  if (!p || !ctas_out) return pc::fail(PC_ERR_INVALID_ARG, "plan and ctas_out are required");
  if (axis < 0 || axis >= p->dim) return pc::fail(PC_ERR_INVALID_ARG, "axis %d out of range", axis);
  *ctas_out = pc::ctas_ref(p, axis, precision == PC_PREC_FP64);
  return PC_OK;
}

extern "C" pc_status pc_plan_autotune(pc_plan *plan, void *cuda_stream, double *best_ms_out) {
  pc::Plan *p = reinterpret_cast<pc::Plan *>(plan);
  if (!p) return pc::fail(PC_ERR_INVALID_ARG, "plan is NULL");
  int cur = -1;
  cudaGetDevice(&cur);
  if (cudaSetDevice(p->device) != cudaSuccess) return pc::fail(PC_ERR_CUDA, "cudaSetDevice(%d) failed", p->device);
  const pc_status s = pc::autotune(p, (cudaStream_t)cuda_stream, best_ms_out);
  if (cur >= 0) cudaSetDevice(cur);
  return s;
}
