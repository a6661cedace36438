// FP32 transform passes (single-problem and batched) of family 0: real DFT (periodic axes). One translation unit per
// family keeps the build parallel.
#include "axis_pass.cuh"

namespace pc {

pc_status launch_pass_f32_family0(const PassArgs<float> &A, long long tiles, int threads, size_t smem,
                                    cudaStream_t st) {
  if ((A.M & (A.M - 1)) == 0) return launch_axis_pass_spec<float, 0, true>(A, tiles, threads, smem, st);
  return launch_axis_pass_spec<float, 0, false>(A, tiles, threads, smem, st);
}

pc_status launch_batched_f32_family0(const PassArgs<float> *dargs, const int2 *ditems, int nitems, int threads,
                                     size_t smem, int emax, bool pow2, cudaStream_t st) {
  if (pow2) return launch_batched_spec<float, 0, true>(dargs, ditems, nitems, threads, smem, emax, st);
  return launch_batched_spec<float, 0, false>(dargs, ditems, nitems, threads, smem, emax, st);
}

pc_status prepare_pass_f32_family0(int lim) {
  PC_TRY((prepare_axis_pass_spec<float, 0, true>(lim)));
  PC_TRY((prepare_axis_pass_spec<float, 0, false>(lim)));
  PC_TRY((prepare_batched_spec<float, 0, true>(lim)));
  return prepare_batched_spec<float, 0, false>(lim);
}

}  // namespace pc
