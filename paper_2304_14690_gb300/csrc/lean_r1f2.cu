// Lean FP32 transform passes of register class 1 and transform family 2 (see lean_pass.cuh),
// single and batched, in their own translation unit so the build stays parallel.
#include "lean_pass.cuh"

namespace pc {

pc_status launch_lean_r1f2(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                            unsigned grid, int threads, size_t smem, cudaStream_t st) {
  return lean::launch_kernel<1, 2>(A, dargs, ditems, grid, threads, smem, st);
}

pc_status prepare_lean_r1f2(int lim) {
  PC_CUDA_TRY(cudaFuncSetAttribute(lean::lean_kernel<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return PC_OK;
}

}  // namespace pc
