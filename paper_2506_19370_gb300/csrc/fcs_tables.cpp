// FC-Gram continuation tables and FFT twiddles, built on the host in
// double-double arithmetic (paper §2, FC-Gram; construction of Part I §I-2.2
// read as an oversampled, Tikhonov-regularised Fourier-extension fit).
//
// Problem solved (index units, matching points s = 0..d-1):
//   T(s) = a_0 + sum_{m=1..K} a_m cos(2 pi m s / P) + b_m sin(2 pi m s / P),
//   P = 2C + 4d - 1, K = floor((P - 9) / 3),
//   minimise  sum_{s in S_match} |T(s) - l_q(s)|^2 + sum_{s in S_zero} |T(s)|^2
//             + lam^2 |(a, b)|^2,       lam = 1e-14,
//   S_match = {i/20 : 0 <= i <= 20(d-1)},  S_zero = {d + C + i/20 : same i},
// for every Lagrange basis polynomial l_q of the d matching points; then
// A_R[c][q] = T_q(d + c), c = 0..C-1.  (The Gram polynomials of FC-Gram span
// the same space and the fit is linear in its targets, so the combined table
// is the same.)  The least-squares problem is solved by Householder QR with
// about 32 significant digits so that the FP64 table is exact to the last
// bits despite the exponential ill-conditioning of Fourier extension.
//
// Compiled with -ffp-contract=off: the error-free transformations below rely
// on every product and sum being rounded separately.
#include <cmath>
#include <cstdint>
#include <vector>

#include "fcs_internal.h"

namespace fcs {
namespace {

struct dd {
  double hi, lo;
};

inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  return {p, std::fma(a, b, -p)};
}
inline dd mk(double a) { return {a, 0.0}; }
inline dd add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
inline dd neg(dd a) { return {-a.hi, -a.lo}; }
inline dd sub(dd a, dd b) { return add(a, neg(b)); }
inline dd mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
inline dd mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}
inline dd div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = sub(a, mul_d(b, q1));
  double q2 = r.hi / b.hi;
  r = sub(r, mul_d(b, q2));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return add(q, mk(q3));
}
inline dd sqrt_dd(dd a) {
  if (a.hi <= 0.0) return mk(0.0);
  double x = std::sqrt(a.hi);
  dd xx = mk(x);
  // one Newton step doubles the number of correct digits
  dd r = sub(a, mul(xx, xx));
  return add(xx, mk(r.hi / (2.0 * x)));
}

// pi to double-double precision
const dd kPi = {3.141592653589793116e+00, 1.224646799147353207e-16};

// cos and sin of 2 pi k / M for integers k, M > 0: reduce to the nearest
// quarter turn with integer arithmetic, Taylor series on |x| <= pi/4.
void cos_sin_2pi(long long k, long long M, dd* c, dd* s) {
  k %= M;
  if (k < 0) k += M;
  long long q = (8 * k + M) / (2 * M);          // nearest quarter turn
  long long num = 4 * k - q * M;                 // x = (pi / (2M)) * num
  dd x = mul(kPi, div(mk((double)num), mk(2.0 * (double)M)));
  dd x2 = mul(x, x);
  dd sn = x, cs = mk(1.0), term_s = x, term_c = mk(1.0);
  for (int n = 1; n < 30; ++n) {
    term_s = div(mul(term_s, x2), mk(-(double)((2 * n) * (2 * n + 1))));
    term_c = div(mul(term_c, x2), mk(-(double)((2 * n - 1) * (2 * n))));
    sn = add(sn, term_s);
    cs = add(cs, term_c);
  }
  switch (((q % 4) + 4) % 4) {
    case 0: *c = cs; *s = sn; break;
    case 1: *c = neg(sn); *s = cs; break;
    case 2: *c = neg(cs); *s = neg(sn); break;
    default: *c = sn; *s = neg(cs); break;
  }
}

}  // namespace

void fit_params(int d, int C, int* P, int* K) {
  *P = 2 * C + 4 * d - 1;
  *K = (*P - 9) / 3;
}

int build_table(int d, int C, double* A_R, double* A_R_lo) {
  if (d < 2 || d > 12 || C < 2 || C > 64) return -1;
  int P, K;
  fit_params(d, C, &P, &K);
  const int nos = 20;
  const int nm = (d - 1) * nos + 1;  // samples per region
  const int ncol = 2 * K + 1;
  const int nrow = 2 * nm + ncol;
  std::vector<dd> A((size_t)nrow * ncol, mk(0.0)), B((size_t)nrow * d, mk(0.0));
  auto a = [&](int r, int c) -> dd& { return A[(size_t)r * ncol + c]; };
  auto b = [&](int r, int q) -> dd& { return B[(size_t)r * d + q]; };
  const long long M = (long long)nos * P;
  for (int r = 0; r < 2 * nm; ++r) {
    // sample s = off + i / nos with integer numerator t = nos * off + i
    long long i = r % nm;
    long long t = (r < nm) ? i : (long long)nos * (d + C) + i;
    a(r, 0) = mk(1.0);
    for (int m = 1; m <= K; ++m) {
      dd c, s;
      cos_sin_2pi((long long)m * t, M, &c, &s);
      a(r, 2 * m - 1) = c;
      a(r, 2 * m) = s;
    }
    if (r < nm) {
      dd sv = div(mk((double)i), mk((double)nos));
      for (int q = 0; q < d; ++q) {
        dd v = mk(1.0);
        for (int o = 0; o < d; ++o) {
          if (o == q) continue;
          v = mul(v, div(sub(sv, mk((double)o)), mk((double)(q - o))));
        }
        b(r, q) = v;
      }
    }
  }
  for (int c = 0; c < ncol; ++c) a(2 * nm + c, c) = mk(1e-14);

  // Householder QR: A = Q R, apply Q^T to B
  for (int k = 0; k < ncol; ++k) {
    dd nrm2 = mk(0.0);
    for (int r = k; r < nrow; ++r) nrm2 = add(nrm2, mul(a(r, k), a(r, k)));
    dd nrm = sqrt_dd(nrm2);
    if (nrm.hi == 0.0) continue;
    dd alpha = a(k, k).hi > 0 ? neg(nrm) : nrm;
    // v = x - alpha e_k, stored in column k below the diagonal
    a(k, k) = sub(a(k, k), alpha);
    dd vtv = mk(0.0);
    for (int r = k; r < nrow; ++r) vtv = add(vtv, mul(a(r, k), a(r, k)));
    dd beta = div(mk(2.0), vtv);
    for (int c = k + 1; c < ncol; ++c) {
      dd dot = mk(0.0);
      for (int r = k; r < nrow; ++r) dot = add(dot, mul(a(r, k), a(r, c)));
      dd f = mul(beta, dot);
      for (int r = k; r < nrow; ++r) a(r, c) = sub(a(r, c), mul(f, a(r, k)));
    }
    for (int q = 0; q < d; ++q) {
      dd dot = mk(0.0);
      for (int r = k; r < nrow; ++r) dot = add(dot, mul(a(r, k), b(r, q)));
      dd f = mul(beta, dot);
      for (int r = k; r < nrow; ++r) b(r, q) = sub(b(r, q), mul(f, a(r, k)));
    }
    // R(k,k) = alpha; the Householder vector is no longer needed
    a(k, k) = alpha;
  }
  // back substitution R x = (Q^T b)[0:ncol]
  std::vector<dd> X((size_t)ncol * d);
  for (int q = 0; q < d; ++q) {
    for (int k = ncol - 1; k >= 0; --k) {
      dd s = b(k, q);
      for (int c = k + 1; c < ncol; ++c) s = sub(s, mul(a(k, c), X[(size_t)c * d + q]));
      X[(size_t)k * d + q] = div(s, a(k, k));
    }
  }
  // evaluate at the gap points s = d + c
  for (int c = 0; c < C; ++c) {
    for (int q = 0; q < d; ++q) {
      dd v = X[q];
      for (int m = 1; m <= K; ++m) {
        dd cs, sn;
        cos_sin_2pi((long long)m * (d + c), P, &cs, &sn);
        v = add(v, add(mul(cs, X[(size_t)(2 * m - 1) * d + q]), mul(sn, X[(size_t)(2 * m) * d + q])));
      }
      A_R[c * d + q] = v.hi + v.lo;
      if (A_R_lo) A_R_lo[c * d + q] = v.lo - (A_R[c * d + q] - v.hi);
    }
  }
  return 0;
}

void gram_basis_dd(int d, double* Qhi, double* Qlo) {
  // Vandermonde matrix at s / (d - 1), s = 0..d-1, orthonormalised column by
  // column (modified Gram-Schmidt, twice for orthogonality to the last bits)
  std::vector<dd> Q((size_t)d * d);
  for (int i = 0; i < d; ++i) {
    const dd x = div(mk((double)i), mk((double)(d - 1)));
    dd v = mk(1.0);
    for (int j = 0; j < d; ++j) {
      Q[(size_t)i * d + j] = v;
      v = mul(v, x);
    }
  }
  for (int j = 0; j < d; ++j) {
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < j; ++k) {
        dd dot = mk(0.0);
        for (int i = 0; i < d; ++i) dot = add(dot, mul(Q[(size_t)i * d + k], Q[(size_t)i * d + j]));
        for (int i = 0; i < d; ++i) Q[(size_t)i * d + j] = sub(Q[(size_t)i * d + j], mul(dot, Q[(size_t)i * d + k]));
      }
    dd nrm2 = mk(0.0);
    for (int i = 0; i < d; ++i) nrm2 = add(nrm2, mul(Q[(size_t)i * d + j], Q[(size_t)i * d + j]));
    const dd nrm = sqrt_dd(nrm2);
    for (int i = 0; i < d; ++i) Q[(size_t)i * d + j] = div(Q[(size_t)i * d + j], nrm);
  }
  for (size_t k = 0; k < Q.size(); ++k) {
    Qhi[k] = Q[k].hi + Q[k].lo;
    Qlo[k] = Q[k].lo - (Qhi[k] - Q[k].hi);
  }
}

void row_sums(int d, int C, const double* ARhi, const double* ARlo, double* rs) {
  for (int c = 0; c < C; ++c) {
    dd v = mk(0.0);
    for (int m = 0; m < d; ++m) v = add(v, dd{ARhi[c * d + m], ARlo[c * d + m]});
    rs[c] = v.hi + v.lo;
  }
}

void gram_blend(int d, int C, const double* ARhi, const double* ARlo, const double* Qhi, const double* Qlo,
                double* T) {
  for (int c = 0; c < C; ++c)
    for (int k = 0; k < d; ++k) {
      dd v = mk(0.0);
      for (int m = 0; m < d; ++m)
        v = add(v, mul(dd{ARhi[c * d + m], ARlo[c * d + m]}, dd{Qhi[m * d + k], Qlo[m * d + k]}));
      T[c * d + k] = v.hi + v.lo;
    }
}

void twiddles(int n, double* re, double* im) {
  for (int k = 0; k < n; ++k) {
    dd c, s;
    cos_sin_2pi(-(long long)k, n, &c, &s);  // e^{-2 pi i k / n}
    re[k] = c.hi + c.lo;
    im[k] = s.hi + s.lo;
  }
}

void split_float(double v, float* hi, float* lo) {
  float h = (float)v;
  *hi = h;
  *lo = (float)(v - (double)h);
}

}  // namespace fcs
