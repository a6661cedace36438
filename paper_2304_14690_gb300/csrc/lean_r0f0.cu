// Lean FP32 transform passes of register class 0 and transform family 0 (see lean_pass.cuh),
// single and batched, in their own translation unit so the build stays parallel.
#include "lean_pass.cuh"

namespace pc {

pc_status launch_lean_r0f0(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                            unsigned grid, int threads, size_t smem, cudaStream_t st) {
  return lean::launch_kernel<0, 0>(A, dargs, ditems, grid, threads, smem, st);
}

pc_status prepare_lean_r0f0(int lim) {
  PC_CUDA_TRY(cudaFuncSetAttribute(lean::lean_kernel<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return PC_OK;
}

}  // namespace pc
