// FP32 transform passes (single-problem) of family 2: DCT-IV / DST-IV (Neumann-Dirichlet, Dirichlet-Neumann axes). One translation unit per
// family keeps the build parallel.
#include "axis_pass.cuh"

namespace pc {

pc_status launch_pass_f32_family2(const PassArgs<float> &A, long long tiles, int threads, size_t smem,
                                    cudaStream_t st) {
  if ((A.M & (A.M - 1)) == 0) return launch_axis_pass_spec<float, 2, true>(A, tiles, threads, smem, st);
  return launch_axis_pass_spec<float, 2, false>(A, tiles, threads, smem, st);
}

pc_status prepare_pass_f32_family2(int lim) {
  PC_TRY((prepare_axis_pass_spec<float, 2, true>(lim)));
  return prepare_axis_pass_spec<float, 2, false>(lim);
}

}  // namespace pc
