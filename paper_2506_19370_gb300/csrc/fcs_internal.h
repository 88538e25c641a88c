// Internal declarations shared by the host table builder (fcs_tables.cpp) and
// the CUDA translation unit (fcs_api.cu).
#pragma once

namespace fcs {

// Period P and highest mode K of the blend-to-zero fit for (d, C).
void fit_params(int d, int C, int* P, int* K);

// FP64 right-end continuation table A_R (C x d, row-major); 0 on success.
int build_table(int d, int C, double* A_R);

// e^{-2 pi i k / n}, k = 0..n-1, correctly rounded from double-double.
void twiddles(int n, double* re, double* im);

// v = hi + lo with hi = float(v), lo = float(v - hi).
void split_float(double v, float* hi, float* lo);

}  // namespace fcs
