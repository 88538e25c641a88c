// Definitions of the launch functions declared in fcs_launch.cuh, and the
// macro that instantiates them for one (dtype, n1) pair.
#pragma once

#include "fcs_line_kernels.cuh"
#include "fcs_launch.cuh"

namespace fcs {

template <typename T, int N1>
cudaError_t prep_xpass(size_t smem) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_xpass<T, MODE_RHS, N1>, a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xpass<T, MODE_RK, N1>, a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xpass<T, MODE_RHS | MODE_CHAIN, N1>, a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xpass<T, MODE_RK | MODE_CHAIN, N1>, a, (int)smem);
  return e;
}
template <typename T, int N1>
cudaError_t prep_ypass(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_ypass<T, 0, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_ypass<T, 1, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <typename T, int N1>
cudaError_t prep_fc_deriv(size_t smem) {
  return cudaFuncSetAttribute(k_fc_deriv<T, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int N1>
cudaError_t prep_fc_cols(size_t smem) {
  return cudaFuncSetAttribute(k_fc_cols<T, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <typename T, int N1>
cudaError_t run_fc_cols(const CtxDev& c, int order, const int2* tiles, int ntiles, int nf, const T* in, T* out,
                        LaunchCfg g) {
  k_fc_cols<T, N1><<<g.grid, g.block, g.smem, g.stream>>>(c, order, tiles, ntiles, nf, in, out);
  return cudaGetLastError();
}
template <typename T, int N1>
cudaError_t run_fc_deriv(const CtxDev& c, int dir, int order, const int4* pairs, int npairs, const T* in, T* out,
                         LaunchCfg g, const T* mu) {
  k_fc_deriv<T, N1><<<g.grid, g.block, g.smem, g.stream>>>(c, dir, order, pairs, npairs, in, out, mu);
  return cudaGetLastError();
}
template <typename T, int MODE, int N1>
cudaError_t run_xpass(const CtxDev& c, int lbeg, int lcnt, const T* e, const T* mu, const T* R, T* G1, const T* G2,
                      StageArgs<T> st, LaunchCfg g) {
  k_xpass<T, MODE, N1><<<g.grid, g.block, g.smem, g.stream>>>(c, lbeg, lcnt, e, mu, R, G1, G2, st);
  return cudaGetLastError();
}
template <typename T, int N1>
cudaError_t run_ypass(const CtxDev& c, const int2* tiles, int ntiles, const T* e, const T* mu, T* R, const T* G1,
                      T* G2, int chain, LaunchCfg g) {
  if (chain) k_ypass<T, 1, N1><<<g.grid, g.block, g.smem, g.stream>>>(c, tiles, ntiles, e, mu, R, G1, G2);
  else k_ypass<T, 0, N1><<<g.grid, g.block, g.smem, g.stream>>>(c, tiles, ntiles, e, mu, R, G1, G2);
  return cudaGetLastError();
}

}  // namespace fcs

#define FCS_INSTANTIATE_LINES(T, N1)                                                                          \
  template cudaError_t fcs::prep_xpass<T, N1>(size_t);                                                        \
  template cudaError_t fcs::prep_ypass<T, N1>(size_t);                                                        \
  template cudaError_t fcs::prep_fc_deriv<T, N1>(size_t);                                                     \
  template cudaError_t fcs::prep_fc_cols<T, N1>(size_t);                                                      \
  template cudaError_t fcs::run_fc_cols<T, N1>(const CtxDev&, int, const int2*, int, int, const T*, T*,        \
                                               LaunchCfg);                                                    \
  template cudaError_t fcs::run_fc_deriv<T, N1>(const CtxDev&, int, int, const int4*, int, const T*, T*,     \
                                                LaunchCfg, const T*);                                         \
  template cudaError_t fcs::run_ypass<T, N1>(const CtxDev&, const int2*, int, const T*, const T*, T*, const T*, \
                                             T*, int, LaunchCfg);                                             \
  template cudaError_t fcs::run_xpass<T, fcs::MODE_RHS, N1>(const CtxDev&, int, int, const T*, const T*,     \
                                                            const T*, T*, const T*, StageArgs<T>, LaunchCfg);  \
  template cudaError_t fcs::run_xpass<T, fcs::MODE_RK, N1>(const CtxDev&, int, int, const T*, const T*,      \
                                                           const T*, T*, const T*, StageArgs<T>, LaunchCfg);   \
  template cudaError_t fcs::run_xpass<T, fcs::MODE_RHS | fcs::MODE_CHAIN, N1>(                                \
      const CtxDev&, int, int, const T*, const T*, const T*, T*, const T*, StageArgs<T>, LaunchCfg);           \
  template cudaError_t fcs::run_xpass<T, fcs::MODE_RK | fcs::MODE_CHAIN, N1>(                                 \
      const CtxDev&, int, int, const T*, const T*, const T*, T*, const T*, StageArgs<T>, LaunchCfg);
