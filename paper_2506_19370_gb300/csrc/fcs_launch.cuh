// Launch functions of the line kernels (FC derivative, flux passes).  Each
// instantiation (dtype, FFT size n1, mode) is compiled in one of the
// fcs_lines_*.cu translation units so the build compiles them in parallel;
// fcs_api.cu only sees these declarations.
#pragma once

#include <cuda_runtime.h>

#include "fcs_device.cuh"

namespace fcs {

enum { MODE_RHS = 1, MODE_RK = 2 };

template <typename T>
struct StageArgs {
  int stage;
  T dt;
  const double* dt_dev;
  const T* e_n;
  T* acc;
  T* out;
};

// Per-warp shared bytes of the line kernels: `lines` real lines of nmax values
// plus, when some plan uses it, the two complex buffers of the Stockham FFT.
template <typename T>
__host__ __device__ inline size_t warp_line_bytes(int lines, int nmax, int nfmax, int stockham) {
  size_t r = (size_t)lines * nmax * sizeof(T);
  r = (r + 15) & ~size_t(15);
  return r + (stockham ? (size_t)2 * nfmax * sizeof(Cx<T>) : 0);
}

// Shared bytes of the column pass: E and D tiles [4][n2max][tw+1], mu tile
// [n2max][tw+1], Stockham buffers of every warp.
template <typename T>
__host__ __device__ inline size_t ypass_bytes(int n2max, int tw, int nfmax, int stockham, int warps) {
  size_t r = (size_t)9 * n2max * (tw + 1) * sizeof(T);
  r = (r + 15) & ~size_t(15);
  return r + (stockham ? (size_t)warps * 2 * nfmax * sizeof(Cx<T>) : 0);
}
constexpr int kYWarps = 8;

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
cudaError_t run_fc_deriv(const CtxDev& c, int dir, int order, const int4* pairs, int npairs, const T* in, T* out,
                         LaunchCfg g);
template <typename T, int N1>
cudaError_t run_xpass(const CtxDev& c, const T* e, const T* mu, T* R, LaunchCfg g);
template <typename T, int MODE, int N1>
cudaError_t run_ypass(const CtxDev& c, const int2* tiles, int ntiles, const T* e, const T* mu, const T* R,
                      StageArgs<T> st, LaunchCfg g);

}  // namespace fcs
