// FP32 batched transform pass (every family, length and dimension in one launch per pass), in
// its own translation unit so the build stays parallel.
#include "axis_pass.cuh"

namespace pc {

pc_status launch_batched_f32(const PassArgs<float> *dargs, const int4 *ditems, int nitems, int threads, size_t smem,
                             int emax, cudaStream_t st) {
  return launch_batched<float>(dargs, ditems, nitems, threads, smem, emax, st);
}

pc_status prepare_batched_f32(int lim) { return prepare_batched<float>(lim); }

}  // namespace pc
