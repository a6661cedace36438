// Descriptors of one transform pass (see poisson.cu) shared with the batched executor.
#pragma once

#include <vector>

#include "fft.cuh"
#include "pc_internal.cuh"

namespace pc {

enum SrcMode { SRC_F32 = 0, SRC_F64 = 1, SRC_WORK = 2 };

constexpr int kMaxPassThreads = 512;   // CTA size limit of the transform passes
constexpr int kBatchPassEmax = 16;     // largest slots per thread of a batched pass kernel
constexpr int kBatchedThreads = 256;    // CTA size of the batched pass (4 resident per SM)
// DST_PAIR_*: the refinement iterate of the FP32 solves, kept as FP32 (hi, lo) pairs
// (double-float): SET stores the pass result, ADD adds it to the stored pair.
enum DstMode { DST_WORK = 0, DST_F64_SET = 1, DST_F64_ADD = 2, DST_PAIR_SET = 3, DST_PAIR_ADD = 4 };

template <typename Real>
struct PassArgs {
  using T = typename Cplx<Real>::T;
  int axis, kind, n, M, nst;
  StageInfo st[kMaxRadices];
  const T *tw;
  int dim;
  int shape[3];
  int stride;           // element stride along the axis
  int inner;            // column tiles: number of line positions f (= stride)
  int lines;            // row tiles: number of lines
  int L;                // lines per tile (power of two)
  int emax;             // slots per thread (power of two): selects the kernel instance
  int lbits;            // log2(L)
  int tpl_bits;         // log2(threads per line)
  int col;              // 1: column tile
  int tiles_per_outer;  // column tiles: ceil(inner / L)
  int do_fwd, do_div, do_inv;
  const Real *lam[3];
  int singular;
  int src_mode;
  const void *src;
  int dst_mode;
  void *dst;
  Real out_scale;       // normalisation of the inverse (2/n)
  double *f64;          // nullable (pair modes): also store the pair's value in FP64
  RefineGate gate;      // a refinement sweep's pass: nothing to do once the stopping rule ended it
  int chunk;            // single-problem launches: consecutive tiles per CTA (>= 1)
  int ntiles;           // tiles of the pass
  int lean;             // 0: general pass (axis_pass.cuh); else the lean kernel id (lean_pass.cuh)
};

// One pass of a solve: axis, phases, source and destination.
struct PassSpec {
  int axis;
  bool fwd, div, inv;
  int src_mode;
  const void *src;
  int dst_mode;
  void *dst;
  double *f64;          // nullable (pair modes): also store the result in FP64
  RefineGate gate;      // stopping-rule gate of PassArgs
  int chunk;            // tiles per CTA of a single-problem launch (0 or 1: one)
};

// The passes of one solve of plan p from src to dst, in launch order; f64 (nullable) goes to
// the final pass.
std::vector<PassSpec> solve_pass_specs(const Plan *p, bool fp32, int src_mode, const void *src,
                                       int dst_mode, void *dst, double *f64 = nullptr,
                                       RefineGate gate = RefineGate{nullptr, 0, 0.0f}, int chunk = 1);
// Fill the kernel arguments and launch shape of one pass (no launch). batch_threads > 0 sizes
// the tile to fill a CTA of that many threads (batched launches); 0 sizes it so that the
// problem alone fills the GPU.
template <typename Real>
pc_status build_pass(const Plan *p, const PassSpec &ps, PassArgs<Real> &A, long long &tiles, int &threads,
                     size_t &smem, int batch_threads);
// Single-problem FP32 pass of transform family 0 (real DFT), 1 (DCT-II/DST-II) or 2
// (DCT-IV/DST-IV), each compiled in its own translation unit (pass_f32_family*.cu), and the
// shared-memory attributes of their kernel instances. Families 3 and 4 (vertex grids) have
// their own unit.
pc_status launch_pass_f32_family0(const PassArgs<float> &A, long long tiles, int threads, size_t smem, cudaStream_t st);
pc_status launch_pass_f32_family1(const PassArgs<float> &A, long long tiles, int threads, size_t smem, cudaStream_t st);
pc_status launch_pass_f32_family2(const PassArgs<float> &A, long long tiles, int threads, size_t smem, cudaStream_t st);
pc_status prepare_pass_f32_family0(int lim);
pc_status prepare_pass_f32_family1(int lim);
pc_status prepare_pass_f32_family2(int lim);
// Passes along vertex-grid axes (families 3 and 4, pass_vertex.cu), FP32 and FP64.
pc_status launch_pass_vertex_f32(const PassArgs<float> &A, long long tiles, int threads, size_t smem, cudaStream_t st);
pc_status launch_pass_vertex_f64(const PassArgs<double> &A, long long tiles, int threads, size_t smem, cudaStream_t st);
pc_status prepare_pass_vertex(int lim);
// Batched FP32 pass over a work list of (args index, first tile, tiles) items of any family,
// length and dimension (one launch per pass for a whole batch, one CTA per item).
pc_status launch_batched_f32(const PassArgs<float> *dargs, const int4 *ditems, int nitems, int threads, size_t smem,
                             int emax, cudaStream_t st);
pc_status prepare_batched_f32(int lim);
// Lean FP32 passes (compile-time line length, lean_pass.cuh): one kernel per register class
// (r) and transform family (f) serves single-problem passes (dargs == ditems == nullptr, A the
// pass) and batched ones (one CTA per work item).
pc_status launch_lean_r0f0(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                            unsigned grid, int threads, size_t smem, cudaStream_t st);
pc_status prepare_lean_r0f0(int lim);
pc_status launch_lean_r0f1(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                            unsigned grid, int threads, size_t smem, cudaStream_t st);
pc_status prepare_lean_r0f1(int lim);
pc_status launch_lean_r0f2(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                            unsigned grid, int threads, size_t smem, cudaStream_t st);
pc_status prepare_lean_r0f2(int lim);
pc_status launch_lean_r1f0(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                            unsigned grid, int threads, size_t smem, cudaStream_t st);
pc_status prepare_lean_r1f0(int lim);
pc_status launch_lean_r1f1(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                            unsigned grid, int threads, size_t smem, cudaStream_t st);
pc_status prepare_lean_r1f1(int lim);
pc_status launch_lean_r1f2(const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                            unsigned grid, int threads, size_t smem, cudaStream_t st);
pc_status prepare_lean_r1f2(int lim);
// Launch of lean kernel id (PassArgs::lean: 1 + 3 * register class + family).
inline pc_status launch_lean(int id, const PassArgs<float> &A, const PassArgs<float> *dargs, const int4 *ditems,
                             unsigned grid, int threads, size_t smem, cudaStream_t st) {
  switch (id) {
    case 1: return launch_lean_r0f0(A, dargs, ditems, grid, threads, smem, st);
    case 2: return launch_lean_r0f1(A, dargs, ditems, grid, threads, smem, st);
    case 3: return launch_lean_r0f2(A, dargs, ditems, grid, threads, smem, st);
    case 4: return launch_lean_r1f0(A, dargs, ditems, grid, threads, smem, st);
    case 5: return launch_lean_r1f1(A, dargs, ditems, grid, threads, smem, st);
    default: return launch_lean_r1f2(A, dargs, ditems, grid, threads, smem, st);
  }
}
inline pc_status prepare_lean(int lim) {
  PC_TRY(prepare_lean_r0f0(lim));
  PC_TRY(prepare_lean_r0f1(lim));
  PC_TRY(prepare_lean_r0f2(lim));
  PC_TRY(prepare_lean_r1f0(lim));
  PC_TRY(prepare_lean_r1f1(lim));
  return prepare_lean_r1f2(lim);
}
// Transform family of a kind: 0 real DFT, 1 DCT-II/DST-II, 2 DCT-IV/DST-IV, 3 vertex DCT-I/DST-I,
// 4 vertex quarter-wave bases.
__host__ __device__ inline int pass_family(int kind) {
  if (kind == KIND_PP) return 0;
  if (kind == KIND_NN || kind == KIND_DD) return 1;
  if (kind == KIND_ND || kind == KIND_DN) return 2;
  return (kind == KIND_VNN || kind == KIND_VDD) ? 3 : 4;
}

}  // namespace pc
