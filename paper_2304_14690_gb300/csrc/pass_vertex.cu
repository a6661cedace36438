// Transform passes along vertex-grid axes (§2.3 regular grid): family 3 (DCT-I of the N-N
// unknowns, DST-I of the D-D unknowns, through the real DFT of their even or odd extension) and
// family 4 (the quarter-wave bases of N-D and D-N axes, through the cell grid's DCT-II/DST-II
// pair in the other order), in FP32 and FP64, in their own translation unit.
#include "axis_pass.cuh"

namespace pc {

pc_status launch_pass_vertex_f32(const PassArgs<float> &A, long long tiles, int threads, size_t smem,
                                 cudaStream_t st) {
  const bool pow2 = (A.M & (A.M - 1)) == 0;
  if (pass_family(A.kind) == 3)
    return pow2 ? launch_axis_pass_spec<float, 3, true>(A, tiles, threads, smem, st)
                : launch_axis_pass_spec<float, 3, false>(A, tiles, threads, smem, st);
  return pow2 ? launch_axis_pass_spec<float, 4, true>(A, tiles, threads, smem, st)
              : launch_axis_pass_spec<float, 4, false>(A, tiles, threads, smem, st);
}

pc_status launch_pass_vertex_f64(const PassArgs<double> &A, long long tiles, int threads, size_t smem,
                                 cudaStream_t st) {
  if (pass_family(A.kind) == 3) return launch_axis_pass_spec<double, 3, false>(A, tiles, threads, smem, st);
  return launch_axis_pass_spec<double, 4, false>(A, tiles, threads, smem, st);
}

pc_status prepare_pass_vertex(int lim) {
  PC_TRY((prepare_axis_pass_spec<float, 3, true>(lim)));
  PC_TRY((prepare_axis_pass_spec<float, 3, false>(lim)));
  PC_TRY((prepare_axis_pass_spec<float, 4, true>(lim)));
  PC_TRY((prepare_axis_pass_spec<float, 4, false>(lim)));
  PC_TRY((prepare_axis_pass_spec<double, 3, false>(lim)));
  return prepare_axis_pass_spec<double, 4, false>(lim);
}

}  // namespace pc
