// FP32 persistent batched transform pass (every family, length and dimension in one launch per
// pass), in its own translation unit so the build stays parallel.
#include "axis_pass.cuh"

namespace pc {

pc_status launch_persistent_f32(const PassArgs<float> *dargs, const int2 *ditems, int nitems, int grid, int threads,
                                size_t smem, int stage_bytes, int gate_bytes, int a0, int nargs, int gated, int emax,
                                cudaStream_t st) {
  return launch_persistent<float>(dargs, ditems, nitems, grid, threads, smem, stage_bytes, gate_bytes, a0, nargs, gated,
                                  emax, st);
}

int persistent_f32_ctas_per_sm(int emax, int threads, size_t smem) {
  return persistent_ctas_per_sm<float>(emax, threads, smem);
}

pc_status prepare_persistent_f32(int lim) { return prepare_persistent<float>(lim); }

}  // namespace pc
