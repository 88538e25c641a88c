// Internal declarations shared by the host parts (fcs_tables.cpp: FC-Gram
// tables, fcs_donors.cpp: donor search) and the CUDA translation unit
// (fcs_api.cu).
#pragma once

#include <vector>

#include "../../include/fcsdnn.h"

namespace fcs {

// Nodes per direction of the interpolation stencil of the fringe exchange.
constexpr int kStencil = 6;

struct FringeCopy {
  int dst_patch, dst_point, src_patch, src_point;  // points as j * n1 + i of their patch
};
struct FringeInterp {
  int dst_patch, dst_point, src_patch, src_point;  // src_point: first node of the stencil block
  double wi[kStencil], wj[kStencil];               // tensor Lagrange weights: node (a, b) has wi[a] * wj[b]
};

// 1 if (i, j) of patch q lies in an n_f-point fringe of an internal side.
bool is_receiver(const fcs_patch_desc& q, int n_f, int i, int j);

// Donor of every receiver (copies for coincident nodes, tensor Lagrange
// interpolation otherwise); -1 if some receiver has no donor.
int build_fringe(const fcs_patch_desc* pd, int npatch, int n_f, std::vector<FringeCopy>* copies,
                 std::vector<FringeInterp>* interp);

// Period P and highest mode K of the blend-to-zero fit for (d, C).
void fit_params(int d, int C, int* P, int* K);

// FP64 right-end continuation table A_R (C x d, row-major), and with A_R_lo
// the remainder of its double-double value; 0 on success.
int build_table(int d, int C, double* A_R, double* A_R_lo = nullptr);

// Gram basis of the d matching points (d x d, Q[m][k] = p_k(m), orthonormal
// columns of the Vandermonde matrix at m / (d - 1)) as double-double hi + lo.
void gram_basis_dd(int d, double* Qhi, double* Qlo);

// Row sums of A_R (C values: the continuation of a constant 1 from the right
// end), evaluated in double-double and rounded to FP64.
void row_sums(int d, int C, const double* ARhi, const double* ARlo, double* rs);

// Blend values of the Gram polynomials, T = A_R Q (C x d), evaluated in
// double-double and rounded to FP64.
void gram_blend(int d, int C, const double* ARhi, const double* ARlo, const double* Qhi, const double* Qlo,
                double* T);

// e^{-2 pi i k / n}, k = 0..n-1, correctly rounded from double-double.
void twiddles(int n, double* re, double* im);

// v = hi + lo with hi = float(v), lo = float(v - hi).
void split_float(double v, float* hi, float* lo);

}  // namespace fcs
