// Donor search of the fringe exchange (paper §3.3, interpolation of I-3.4).
//
// Every point within n_f points of an internal side receives its values from
// another patch.  The donor is the lowest-numbered other patch that contains
// the point and either has a grid node there (copy) or whose 6 x 6 tensor
// Lagrange stencil around the point holds none of its own receivers (donors
// are never receivers; on an L-shaped donor every stencil node belongs to the
// patch).  The donor parameter of a point is the affine inverse
// on Cartesian patches and, on curvilinear ones, Newton's method on the
// tensor Lagrange interpolant of the donor's grid coordinates.  Host FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fcs_internal.h"

namespace fcs {
namespace {

constexpr int kS = kStencil;
constexpr double kCopyTol = 1e-9;    // index units: a node this close is copied
constexpr double kInsideTol = 1e-6;  // index units: slack of the inside test (curved maps)

struct PatchView {
  const fcs_patch_desc* d;
  double xmin, xmax, ymin, ymax;
  double X(int i, int j) const {
    return d->cartesian ? d->box[0] + (d->box[1] - d->box[0]) * i / (d->n1 - 1) : d->x[(size_t)j * d->n1 + i];
  }
  double Y(int i, int j) const {
    return d->cartesian ? d->box[2] + (d->box[3] - d->box[2]) * j / (d->n2 - 1) : d->y[(size_t)j * d->n1 + i];
  }
};

// Lagrange basis on the nodes 0..kS-1: values v[a] and derivatives dv[a] at t.
void basis(double t, double* v, double* dv) {
  for (int a = 0; a < kS; ++a) {
    double den = 1.0, num = 1.0, dsum = 0.0;
    for (int b = 0; b < kS; ++b) {
      if (b == a) continue;
      den *= (double)(a - b);
      num *= t - b;
    }
    // derivative of prod_{b != a} (t - b): sum over c of prod_{b != a, c}
    for (int c = 0; c < kS; ++c) {
      if (c == a) continue;
      double pr = 1.0;
      for (int b = 0; b < kS; ++b)
        if (b != a && b != c) pr *= t - b;
      dsum += pr;
    }
    v[a] = num / den;
    if (dv) dv[a] = dsum / den;
  }
}

int block_start(double f, int n) {
  const int s = (int)std::floor(f) - (kS / 2 - 1);
  return std::min(std::max(s, 0), n - kS);
}

bool lshaped(const fcs_patch_desc& q) { return q.lcut[0] > 0 && q.lcut[1] > 0; }

bool active(const fcs_patch_desc& q, int i, int j) { return !(lshaped(q) && i < q.lcut[0] && j < q.lcut[1]); }

// Donor block around (fi, fj): on an L-shaped patch a block reaching into the
// missing quadrant moves out of it along the direction needing the smaller
// shift (ties: along j).
void donor_block(const fcs_patch_desc& s, double fi, double fj, int* i0, int* j0) {
  *i0 = block_start(fi, s.n1);
  *j0 = block_start(fj, s.n2);
  if (lshaped(s) && *i0 < s.lcut[0] && *j0 < s.lcut[1]) {
    if (s.lcut[1] - *j0 <= s.lcut[0] - *i0) *j0 = s.lcut[1];
    else *i0 = s.lcut[0];
  }
}

// Fractional index (fi, fj) of (x, y) in patch P; false if not found.
bool locate(const PatchView& P, double x, double y, double* fi, double* fj) {
  const fcs_patch_desc& d = *P.d;
  if (d.cartesian) {
    *fi = (x - d.box[0]) * (d.n1 - 1) / (d.box[1] - d.box[0]);
    *fj = (y - d.box[2]) * (d.n2 - 1) / (d.box[3] - d.box[2]);
    return true;
  }
  // nearest node: coarse scan, then steepest descent over neighbours
  const int st = std::max(1, std::min(d.n1, d.n2) / 16);
  int bi = 0, bj = 0;
  double best = 1e300;
  for (int j = 0; j < d.n2; j += st)
    for (int i = 0; i < d.n1; i += st) {
      const double dx = P.X(i, j) - x, dy = P.Y(i, j) - y, r = dx * dx + dy * dy;
      if (r < best) { best = r; bi = i; bj = j; }
    }
  for (bool moved = true; moved;) {
    moved = false;
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int i = bi + di, j = bj + dj;
        if (i < 0 || j < 0 || i >= d.n1 || j >= d.n2) continue;
        const double dx = P.X(i, j) - x, dy = P.Y(i, j) - y, r = dx * dx + dy * dy;
        if (r < best) { best = r; bi = i; bj = j; moved = true; }
      }
  }
  double u = bi, w = bj;
  for (int it = 0; it < 40; ++it) {
    const int i0 = block_start(u, d.n1), j0 = block_start(w, d.n2);
    double vi[kS], dvi[kS], vj[kS], dvj[kS];
    basis(u - i0, vi, dvi);
    basis(w - j0, vj, dvj);
    double xm = 0, ym = 0, xu = 0, xw = 0, yu = 0, yw = 0;
    for (int b = 0; b < kS; ++b)
      for (int a = 0; a < kS; ++a) {
        const double px = P.X(i0 + a, j0 + b), py = P.Y(i0 + a, j0 + b);
        xm += vj[b] * vi[a] * px;
        ym += vj[b] * vi[a] * py;
        xu += vj[b] * dvi[a] * px;
        yu += vj[b] * dvi[a] * py;
        xw += dvj[b] * vi[a] * px;
        yw += dvj[b] * vi[a] * py;
      }
    const double det = xu * yw - xw * yu;
    if (det == 0.0 || !std::isfinite(det)) return false;
    const double rx = x - xm, ry = y - ym;
    const double du = (yw * rx - xw * ry) / det, dw = (-yu * rx + xu * ry) / det;
    u += du;
    w += dw;
    if (u < -2.0 || u > d.n1 + 1.0 || w < -2.0 || w > d.n2 + 1.0) return false;
    // converged to well below the interpolation accuracy (index units; a tighter
    // test can sit in the rounding noise of coordinates far from the origin)
    if (std::fabs(du) + std::fabs(dw) < 1e-10) {
      *fi = u;
      *fj = w;
      return true;
    }
  }
  return false;
}

}  // namespace

bool is_receiver(const fcs_patch_desc& q, int n_f, int i, int j) {
  if (!active(q, i, j)) return false;
  return (q.bc[0] == 0 && i < n_f) || (q.bc[1] == 0 && i >= q.n1 - n_f) || (q.bc[2] == 0 && j < n_f) ||
         (q.bc[3] == 0 && j >= q.n2 - n_f);
}

int build_fringe(const fcs_patch_desc* pd, int npatch, int n_f, std::vector<FringeCopy>* copies,
                 std::vector<FringeInterp>* interp) {
  std::vector<PatchView> V(npatch);
  for (int p = 0; p < npatch; ++p) {
    PatchView& v = V[p];
    v.d = &pd[p];
    v.xmin = v.ymin = 1e300;
    v.xmax = v.ymax = -1e300;
    for (int j = 0; j < pd[p].n2; ++j)
      for (int i = 0; i < pd[p].n1; ++i) {
        v.xmin = std::min(v.xmin, v.X(i, j));
        v.xmax = std::max(v.xmax, v.X(i, j));
        v.ymin = std::min(v.ymin, v.Y(i, j));
        v.ymax = std::max(v.ymax, v.Y(i, j));
      }
  }
  // bucket grid over the layout: each patch is listed in the buckets its
  // widened box touches (in patch order), so a receiver only tries the
  // patches of its bucket, lowest-numbered first
  double gx0 = 1e300, gx1 = -1e300, gy0 = 1e300, gy1 = -1e300, wsum = 0;
  std::vector<double> bx0(npatch), bx1(npatch), by0(npatch), by1(npatch);
  for (int p = 0; p < npatch; ++p) {
    const PatchView& D = V[p];
    // generous box: a curved side bulges past its nodes' extent
    const double mx = 0.05 * (D.xmax - D.xmin) + 1e-12, my = 0.05 * (D.ymax - D.ymin) + 1e-12;
    bx0[p] = D.xmin - mx;
    bx1[p] = D.xmax + mx;
    by0[p] = D.ymin - my;
    by1[p] = D.ymax + my;
    gx0 = std::min(gx0, bx0[p]);
    gx1 = std::max(gx1, bx1[p]);
    gy0 = std::min(gy0, by0[p]);
    gy1 = std::max(gy1, by1[p]);
    wsum += std::max(bx1[p] - bx0[p], by1[p] - by0[p]);
  }
  const double cell = std::max(wsum / npatch, 1e-12);
  const int nbx = std::max(1, std::min(4096, (int)std::ceil((gx1 - gx0) / cell)));
  const int nby = std::max(1, std::min(4096, (int)std::ceil((gy1 - gy0) / cell)));
  auto bxi = [&](double x) { return std::min(nbx - 1, std::max(0, (int)((x - gx0) / (gx1 - gx0 + 1e-300) * nbx))); };
  auto byi = [&](double y) { return std::min(nby - 1, std::max(0, (int)((y - gy0) / (gy1 - gy0 + 1e-300) * nby))); };
  std::vector<std::vector<int>> bucket((size_t)nbx * nby);
  for (int p = 0; p < npatch; ++p)
    for (int by = byi(by0[p]); by <= byi(by1[p]); ++by)
      for (int bx = bxi(bx0[p]); bx <= bxi(bx1[p]); ++bx) bucket[(size_t)by * nbx + bx].push_back(p);
  for (int p = 0; p < npatch; ++p) {
    const fcs_patch_desc& q = pd[p];
    for (int j = 0; j < q.n2; ++j)
      for (int i = 0; i < q.n1; ++i) {
        if (!is_receiver(q, n_f, i, j)) continue;   // (only points of the patch receive)
        const double x = V[p].X(i, j), y = V[p].Y(i, j);
        bool found = false;
        const std::vector<int>& cand = bucket[(size_t)byi(y) * nbx + bxi(x)];
        for (size_t ci = 0; ci < cand.size() && !found; ++ci) {
          const int r = cand[ci];
          if (r == p) continue;
          if (x < bx0[r] || x > bx1[r] || y < by0[r] || y > by1[r]) continue;
          double fi, fj;
          if (!locate(V[r], x, y, &fi, &fj)) continue;
          const fcs_patch_desc& s = pd[r];
          if (fi < -kInsideTol || fi > s.n1 - 1 + kInsideTol || fj < -kInsideTol || fj > s.n2 - 1 + kInsideTol)
            continue;
          if (lshaped(s) && fi < s.lcut[0] - kInsideTol && fj < s.lcut[1] - kInsideTol) continue;
          const long long ri = std::llround(fi), rj = std::llround(fj);
          if (std::fabs(fi - ri) <= kCopyTol && std::fabs(fj - rj) <= kCopyTol) {
            if (!active(s, (int)ri, (int)rj) || is_receiver(s, n_f, (int)ri, (int)rj)) continue;
            copies->push_back({p, j * q.n1 + i, r, (int)rj * s.n1 + (int)ri});
            found = true;
            break;
          }
          int i0, j0;
          donor_block(s, fi, fj, &i0, &j0);
          bool clean = true;
          for (int b = 0; b < kS && clean; ++b)
            for (int a = 0; a < kS && clean; ++a)
              clean = active(s, i0 + a, j0 + b) && !is_receiver(s, n_f, i0 + a, j0 + b);
          if (!clean) continue;
          FringeInterp e{};
          e.dst_patch = p;
          e.dst_point = j * q.n1 + i;
          e.src_patch = r;
          e.src_point = j0 * s.n1 + i0;
          basis(fi - i0, e.wi, nullptr);
          basis(fj - j0, e.wj, nullptr);
          interp->push_back(e);
          found = true;
        }
        if (!found) return -1;
      }
  }
  return 0;
}

}  // namespace fcs
