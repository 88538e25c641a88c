// Launch functions of the line kernels (FC derivative, flux passes).  Each
// instantiation (dtype, FFT size n1, mode) is compiled in one of the
// fcs_lines_*.cu translation units so the build compiles them in parallel;
// fcs_api.cu only sees these declarations.
#pragma once

#include <cuda_runtime.h>

#include "fcs_device.cuh"

namespace fcs {

enum { MODE_RHS = 1, MODE_RK = 2, MODE_CHAIN = 4 };  // row-pass epilogue; MODE_CHAIN: chain-rule form

template <typename T>
struct StageArgs {
  int stage;
  T dt;
  const double* dt_dev;
  const T* e_n;
  T* acc;
  T* out;
};

// Shared-memory layout helpers of the line kernels (host and device agree).
// aux: per warp, the Stockham buffers (N1 = 0), nothing (32-lane FFT, odd N1)
// or four transpose tiles 8 x (B+1), B = 4 N1 (two-level FFT, even N1).
__host__ __device__ inline size_t aux_cx(int N1, int nfmax) {
  return N1 == 0 ? (size_t)2 * nfmax : (N1 % 2 ? 0 : (size_t)32 * (4 * N1 + 1));
}
__host__ __device__ inline size_t align16(size_t r) { return (r + 15) & ~size_t(15); }
constexpr int kRowsPerWarp = 2;  // rows a warp of the pass along q1 handles together
template <typename T>
__host__ __device__ inline size_t xpass_warp_bytes(int nmax, int nfmax, int N1) {
  return align16((size_t)kRowsPerWarp * 5 * nmax * sizeof(T)) + aux_cx(N1, nfmax) * 2 * sizeof(T);
}
template <typename T>
__host__ __device__ inline size_t deriv_warp_bytes(int nmax, int nfmax, int N1) {
  return align16((size_t)8 * nmax * sizeof(T)) + aux_cx(N1, nfmax) * 2 * sizeof(T);
}
template <typename T>
__host__ __device__ inline size_t cols_bytes(int n2max, int tw, int nfmax, int N1, int warps) {
  return align16((size_t)4 * n2max * (tw + 1) * sizeof(T)) + (size_t)warps * aux_cx(N1, nfmax) * 2 * sizeof(T);
}
template <typename T>
__host__ __device__ inline size_t ypass_bytes(int n2max, int tw, int nfmax, int N1, int warps) {
  return align16((size_t)5 * n2max * (tw + 1) * sizeof(T)) + (size_t)warps * aux_cx(N1, nfmax) * 2 * sizeof(T);
}
constexpr int kYWarps = 8;

// Blocks per SM the flux passes are compiled for (register budget 65536 /
// (threads x blocks)).  FP32 lines of n1 = 3, 5 take the paired-FP32 shuffle
// FFT (two line pairs per warp: twice the line registers of the pair path),
// so they get the budgets of the two-level FFT (even n1: 2 x 4 n1 values per
// lane); n1 = 3 rows take 96 registers; n1 = 7 and 9 (pair path) spill at
// lower budgets (ptxas).  Column passes of n1 <= 2 run 3 blocks of 8 warps
// (85 registers; 4 blocks spilled and measured 6 % slower on the Sod batch).
__host__ __device__ constexpr int ypass_min_blocks(size_t tsize, int N1) {
  return ((N1 >= 1 && N1 <= 2) || (N1 == 3 && tsize == 8)) ? 3 : 2;
}
__host__ __device__ constexpr int xpass_min_blocks(size_t tsize, int N1) {
  return (tsize == 4 && N1 == 3) ? 5 : 4;
}

struct LaunchCfg {
  unsigned grid;
  unsigned block;
  size_t smem;
  cudaStream_t stream;
};

// Set the dynamic shared-memory limit of the instantiations used by a context.
template <typename T, int N1>
cudaError_t prep_xpass(size_t smem);
template <typename T, int N1>
cudaError_t prep_ypass(size_t smem);
template <typename T, int N1>
cudaError_t prep_fc_deriv(size_t smem);
template <typename T, int N1>
cudaError_t prep_fc_cols(size_t smem);

template <typename T, int N1>
cudaError_t run_fc_deriv(const CtxDev& c, int dir, int order, const int4* pairs, int npairs, const T* in, T* out,
                         LaunchCfg g, const T* mu = nullptr);
template <typename T, int N1>
cudaError_t run_fc_cols(const CtxDev& c, int order, const int2* tiles, int ntiles, int nf, const T* in, T* out,
                        LaunchCfg g);
// The operator is the pass along q2 (writes R) followed by the pass along q1
// (completes L and takes the stage).
template <typename T, int MODE, int N1>
cudaError_t run_xpass(const CtxDev& c, int lbeg, int lcnt, const T* e, const T* mu, const T* R, T* G1, const T* G2,
                      StageArgs<T> st, LaunchCfg g);
template <typename T, int N1>
cudaError_t run_ypass(const CtxDev& c, const int2* tiles, int ntiles, const T* e, const T* mu, T* R, const T* G1,
                      T* G2, int chain, LaunchCfg g);

}  // namespace fcs
