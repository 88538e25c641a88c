// Device code of the FC-SDNN stage library: line FFTs, FC derivatives, the
// Euler operator with the Runge-Kutta epilogue, exchange, reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fcs {

constexpr int kMaxStages = 12;
constexpr int kWarps = 4;             // warps per block of the line kernels
constexpr int kN1Classes = 10;        // FFT-size classes n1 = 0 (Stockham), 2..9 (register FFTs of n = 32 n1)
constexpr int kMaxLine = 512;         // most points per patch side

// ------------------------------------------------------------ descriptors
struct PatchDev {
  int n1, n2, cart, pad0;
  int bc[4];
  int plan[2];          // FFT plan of full lines along i (length n1) and along j (length n2)
  int m1, m2;           // L-shaped patch: points i < m1, j < m2 missing (0, 0: rectangle)
  int plan_s[2];        // L-shaped patch: plans of the short rows (n1 - m1) and columns (n2 - m2)
  int wx_off, wy_off;   // first x-window and first y-window of the patch (per instance)
  int wpl_x, wpl_y;     // windows per full x-line, per full y-line
  int wpl_xs, wpl_ys;   // windows per short x-line, short y-line (L-shaped patches)
  long long soff, qoff; // offsets in the state and scalar layouts (per instance)
  double hx, hy;        // derivative spacing along i and j (physical if Cartesian, parameter otherwise)
  double hmax;          // largest physical spacing (viscosity scale)
  double Lx, Ly;        // Cartesian box lengths (metrics x_q1, y_q2)
  // Lx, Ly, 1/(n1 - 1), 1/(n2 - 1), hmax in both types (pointwise kernels read
  // them per point: FP64 conversions run at 1/64 of the FP32 rate on this part)
  double cd[5];
  float cf[5];
  double inflowd[4];    // conserved inflow state of the patch's inflow sides
  float inflowf[4];
};

enum { PC_LX = 0, PC_LY = 1, PC_H1 = 2, PC_H2 = 3, PC_HMAX = 4 };
template <typename T>
__host__ __device__ __forceinline__ T pconst(const PatchDev& P, int k);
template <>
__host__ __device__ __forceinline__ double pconst<double>(const PatchDev& P, int k) { return P.cd[k]; }
template <>
__host__ __device__ __forceinline__ float pconst<float>(const PatchDev& P, int k) { return P.cf[k]; }

struct PlanDev {
  int N, C, n, nst;
  int radix[kMaxStages];
  int tw_off;           // offset of the n twiddles
  int tab_off;          // offset of the C x d continuation table (FP64, and its FP32 split)
  int n1reg;            // n = 32 * n1reg: register FFT (two-level for even n1reg); 0: Stockham FFT
  int tg_off;           // offset of the C x d Gram blend table (FP32)
  int rs_off;           // offset of the C values of the continuation of a constant 1 from the right end (FP32)
};

struct LineRef {
  int patch, line;
};

struct CtxDev {
  const PatchDev* patches;
  const PlanDev* plans;
  const double* tab64;
  const float* tabhi;
  const float* tablo;
  const double2* tw64;
  const float2* tw32;
  const double* flt64;    // per plan, n filter factors sigma(k) (same offsets as the twiddles)
  const float* flt32;
  const LineRef* lines0;  // rows (lines along i)
  const LineRef* lines1;  // columns (lines along j)
  const int4* windows;    // per window of one instance: patch, dir, line, start
  const double* metrics64;  // [5][scalar] x_q1, x_q2, y_q1, y_q2, J (instance 0 geometry)
  const float* metrics32;
  const unsigned char* fringe;  // 1 on receiver points (scalar layout, instance 0)
  int* status;
  int npatch, nlines0, nlines1, nwin;
  int instances, d;
  long long sstride, qstride;   // per-instance element counts of state and scalar layouts
  double gamma;
  float gm1f;             // gamma - 1 and the outlet pressure in FP32 (FP32 kernels read them per point)
  float p_outf;
  double inflow[4];
  double p_out;
  int ind_plan;                 // plan of the indicator (n = 16 + 26)
  int nmax;                     // longest line
  int nfmax;                    // longest FFT
  int stockham;                 // 1 if some plan needs the shared-memory FFT buffers
  int tw;                       // column-tile width of the pass along q2
  int n2max;                    // longest column (lines along q2)
  int gnmax[2][kN1Classes];     // per direction and FFT-size class: longest line
  int gnfmax[2][kN1Classes];    // ... and longest FFT (shared-memory layout of the line kernels)
  const float* gramQ;           // d x d Gram basis at the matching points (FP32)
  const float* gramT;           // Gram blend tables of all plans (FP32)
  const float* gramR;           // row sums of A_R of all plans (FP32): the continuation of a constant
  const double* gramQ64h;       // the Gram basis as double-double hi + lo
  const double* gramQ64l;
  const double* gramT64;        // Gram blend tables of all plans (FP64, same offsets as gramT)
  const int2* pblk;             // point blocks of 256 points: (patch, first point), one instance
  int npblk;
  const int4* nsw;              // no-slip wall points: (patch, point, inward stride in points, 0)
  int n_nsw;
  double nsw64[8];              // d weights of the derivative at node 0 on nodes 0..d-1
  float nsw32[8];
};

// Point handled by this thread in a pointwise kernel launched on
// (npblk, instances) blocks of 256 threads; 32-bit indexing within a patch.
// L-shaped patches: point membership, first index and plan of a line
// (dir 0: row `line`, dir 1: column `line`).  Rectangles have m1 = m2 = 0.
__host__ __device__ __forceinline__ bool pt_active(const PatchDev& P, int i, int j) {
  return !(i < P.m1 && j < P.m2);
}
__host__ __device__ __forceinline__ int line_start(const PatchDev& P, int dir, int line) {
  return dir == 0 ? (line < P.m2 ? P.m1 : 0) : (line < P.m1 ? P.m2 : 0);
}
__host__ __device__ __forceinline__ int line_plan(const PatchDev& P, int dir, int line) {
  return line_start(P, dir, line) ? P.plan_s[dir] : P.plan[dir];
}

struct PtIdx {
  int inst, patch, lq, i, j;
  bool ok;
};
__device__ __forceinline__ PtIdx pt_index(const CtxDev& c, const PatchDev** Pp) {
  const int2 pb = c.pblk[blockIdx.x];
  const PatchDev& P = c.patches[pb.x];
  *Pp = &P;
  PtIdx r;
  r.inst = blockIdx.y;
  r.patch = pb.x;
  r.lq = pb.y + (int)threadIdx.x;
  r.i = r.lq % P.n1;
  r.j = r.lq / P.n1;
  r.ok = r.lq < P.n1 * P.n2 && pt_active(P, r.i, r.j);
  return r;
}

template <typename T>
struct Cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename T>
__device__ __forceinline__ Cx<T> twid(const CtxDev& c, int idx);
template <>
__device__ __forceinline__ Cx<double> twid<double>(const CtxDev& c, int idx) {
  double2 v = __ldg(c.tw64 + idx);
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ Cx<float> twid<float>(const CtxDev& c, int idx) {
  float2 v = __ldg(c.tw32 + idx);
  return {v.x, v.y};
}

template <typename T>
__device__ __forceinline__ const T* metrics(const CtxDev& c);
template <>
__device__ __forceinline__ const double* metrics<double>(const CtxDev& c) { return c.metrics64; }
template <>
__device__ __forceinline__ const float* metrics<float>(const CtxDev& c) { return c.metrics32; }

// gamma - 1, inflow state k (k = 4: outlet pressure) in the kernel's type
template <typename T>
__device__ __forceinline__ T gm1_of(const CtxDev& c);
template <>
__device__ __forceinline__ double gm1_of<double>(const CtxDev& c) { return c.gamma - 1.0; }
template <>
__device__ __forceinline__ float gm1_of<float>(const CtxDev& c) { return c.gm1f; }
template <typename T>
__device__ __forceinline__ T p_out_of(const CtxDev& c);
template <>
__device__ __forceinline__ double p_out_of<double>(const CtxDev& c) { return c.p_out; }
template <>
__device__ __forceinline__ float p_out_of<float>(const CtxDev& c) { return c.p_outf; }
template <typename T>
__device__ __forceinline__ T inflow_of(const PatchDev& P, int k);
template <>
__device__ __forceinline__ double inflow_of<double>(const PatchDev& P, int k) { return P.inflowd[k]; }
template <>
__device__ __forceinline__ float inflow_of<float>(const PatchDev& P, int k) { return P.inflowf[k]; }

// ------------------------------------------------------------ FFT
// Small DFT of radix R in registers: v[q] <- sum_r v[r] W^{rq}, W = e^{-+2 pi i/R};
// the roots come from the length-n twiddle table (entry (rq mod R) n/R).
template <int R, typename T>
__device__ __forceinline__ void small_dft(Cx<T>* v, const CtxDev& c, int tw0, int n, bool inv) {
  if (R == 2) {
    Cx<T> a = v[0], b = v[1];
    v[0] = {a.x + b.x, a.y + b.y};
    v[1] = {a.x - b.x, a.y - b.y};
    return;
  }
  if (R == 4) {
    Cx<T> t0 = {v[0].x + v[2].x, v[0].y + v[2].y};
    Cx<T> t1 = {v[0].x - v[2].x, v[0].y - v[2].y};
    Cx<T> t2 = {v[1].x + v[3].x, v[1].y + v[3].y};
    Cx<T> t3 = {v[1].x - v[3].x, v[1].y - v[3].y};
    // -i t3 = (t3.y, -t3.x)
    Cx<T> mt3 = inv ? Cx<T>{-t3.y, t3.x} : Cx<T>{t3.y, -t3.x};
    v[0] = {t0.x + t2.x, t0.y + t2.y};
    v[2] = {t0.x - t2.x, t0.y - t2.y};
    v[1] = {t1.x + mt3.x, t1.y + mt3.y};
    v[3] = {t1.x - mt3.x, t1.y - mt3.y};
    return;
  }
  Cx<T> out[R];
  const int step = n / R;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    Cx<T> acc = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      Cx<T> w = twid<T>(c, tw0 + ((r * q) % R) * step);
      if (inv) w.y = -w.y;
      Cx<T> p = cmul(v[r], w);
      acc.x += p.x;
      acc.y += p.y;
    }
    out[q] = acc;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = out[q];
}

// One Stockham autosort stage of radix R: x -> y, Ns = product of earlier radices.
template <int R, typename T>
__device__ __forceinline__ void fft_stage(const Cx<T>* x, Cx<T>* y, const CtxDev& c, int tw0, int n, int Ns,
                                          bool inv, int lane) {
  const int nb = n / R;
  const int tstep = n / (Ns * R);
  for (int j = lane; j < nb; j += 32) {
    const int k = j % Ns;
    Cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      Cx<T> a = x[j + r * nb];
      if (r > 0 && k > 0) {
        Cx<T> w = twid<T>(c, tw0 + r * k * tstep);
        if (inv) w.y = -w.y;
        a = cmul(a, w);
      }
      v[r] = a;
    }
    small_dft<R, T>(v, c, tw0, n, inv);
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[base + r * Ns] = v[r];
  }
}

// Unnormalised FFT of length pl.n by one warp on shared buffers a, b; returns
// the buffer holding the result.
template <typename T>
__device__ Cx<T>* warp_fft(Cx<T>* a, Cx<T>* b, const CtxDev& c, const PlanDev& pl, bool inv, int lane) {
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 2: fft_stage<2, T>(a, b, c, pl.tw_off, pl.n, Ns, inv, lane); break;
      case 3: fft_stage<3, T>(a, b, c, pl.tw_off, pl.n, Ns, inv, lane); break;
      case 4: fft_stage<4, T>(a, b, c, pl.tw_off, pl.n, Ns, inv, lane); break;
      case 5: fft_stage<5, T>(a, b, c, pl.tw_off, pl.n, Ns, inv, lane); break;
      case 7: fft_stage<7, T>(a, b, c, pl.tw_off, pl.n, Ns, inv, lane); break;
      default: fft_stage<8, T>(a, b, c, pl.tw_off, pl.n, Ns, inv, lane); break;
    }
    __syncwarp();
    Cx<T>* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// ------------------------------------------------------------ FC continuation
// FP64 continuation in the Gram form of FC-Gram: the d end values of a line
// (v[m * sv], m = 0..d-1, matching point s = m) are projected on the Gram
// basis, a_k = sum_m Q[m][k] v_m, and the appended value at gap point q is
// sum_k T[q][k] a_k (right end) plus T[C-1-q][k] a_k of the reflected left
// end.  The projection cancels (the high-degree coefficients of smooth data
// are tiny differences of values of size |v|, and their blend values reach
// ~3e3), so it is a compensated dot product (Ogita-Rump-Oishi "Dot2":
// error-free products by fma, error-free sums) with the double-double basis
// Q = Qh + Ql; the blend sum T a is plain, since its large terms are small.
__device__ __forceinline__ double gram_coef64(const double* v, int sv, const double* Qh, const double* Ql, int d,
                                              int k) {
  double s = 0.0, e = 0.0;
  for (int m = 0; m < d; ++m) {
    const double x = v[m * sv];
    const double q = __ldg(Qh + m * d + k);
    const double p = __dmul_rn(q, x);
    const double pe = fma(q, x, -p);
    const double t = __dadd_rn(s, p);
    const double z = __dsub_rn(t, s);
    const double se = __dadd_rn(__dsub_rn(s, __dsub_rn(t, z)), __dsub_rn(p, z));
    s = t;
    e = __dadd_rn(e, __dadd_rn(pe, __dadd_rn(se, __dmul_rn(__ldg(Ql + m * d + k), x))));
  }
  return __dadd_rn(s, e);
}

// buf[0..N) holds two real lines as (re, im); append the C continuation
// values.  Every lane of the warp calls it: lanes k < d project, the others
// read the coefficients by shuffles.
__device__ __forceinline__ void continue_lines(Cx<double>* buf, const CtxDev& c, const PlanDev& pl, int d,
                                               int lane) {
  const double* Tg = c.gramT64 + pl.tg_off;
  const int N = pl.N, C = pl.C;
  double* f = reinterpret_cast<double*>(buf);   // line a at stride 2, line b at offset 1
  double aR = 0.0, aL = 0.0, bR = 0.0, bL = 0.0;
  if (lane < d) {
    aR = gram_coef64(f + 2 * (N - d), 2, c.gramQ64h, c.gramQ64l, d, lane);
    aL = gram_coef64(f + 2 * (d - 1), -2, c.gramQ64h, c.gramQ64l, d, lane);
    bR = gram_coef64(f + 2 * (N - d) + 1, 2, c.gramQ64h, c.gramQ64l, d, lane);
    bL = gram_coef64(f + 2 * (d - 1) + 1, -2, c.gramQ64h, c.gramQ64l, d, lane);
  }
  for (int q0 = 0; q0 < C; q0 += 32) {
    const int q = q0 + lane;
    const bool own = q < C;
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < d; ++k) {
      const double gaR = __shfl_sync(0xffffffffu, aR, k), gaL = __shfl_sync(0xffffffffu, aL, k);
      const double gbR = __shfl_sync(0xffffffffu, bR, k), gbL = __shfl_sync(0xffffffffu, bL, k);
      if (own) {
        const double tr = __ldg(Tg + q * d + k), tl = __ldg(Tg + (C - 1 - q) * d + k);
        sa = fma(tr, gaR, fma(tl, gaL, sa));
        sb = fma(tr, gbR, fma(tl, gbL, sb));
      }
    }
    if (own) buf[N + q] = {sa, sb};
  }
}

// FP32: compensated dot product (error-free product and sum, Ogita-Rump-Oishi
// "Dot2") with the FP64 table split into float hi + lo, so the continuation is
// accurate to about FP64 level although table entries reach ~1e3.
struct Dot2 {
  float s, e;
  __device__ __forceinline__ void add(float hi, float lo, float f) {
    const float p = __fmul_rn(hi, f);
    const float pe = fmaf(hi, f, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    e = __fadd_rn(e, __fadd_rn(pe, __fadd_rn(se, __fmul_rn(lo, f))));
  }
  __device__ __forceinline__ float get() const { return __fadd_rn(s, e); }
};

__device__ __forceinline__ void continue_lines(Cx<float>* buf, const CtxDev& c, const PlanDev& pl, int d,
                                               int lane) {
  const float* hi = c.tabhi + pl.tab_off;
  const float* lo = c.tablo + pl.tab_off;
  const int N = pl.N, C = pl.C;
  for (int q = lane; q < C; q += 32) {
    const int rr = q * d, rl = (C - 1 - q) * d;
    Dot2 a{0.f, 0.f}, b{0.f, 0.f};
    for (int m = 0; m < d; ++m) {
      const float hr = __ldg(hi + rr + m), lr = __ldg(lo + rr + m);
      const float hl = __ldg(hi + rl + m), ll = __ldg(lo + rl + m);
      const Cx<float> fr = buf[N - d + m], fl = buf[d - 1 - m];
      a.add(hr, lr, fr.x);
      b.add(hr, lr, fr.y);
      a.add(hl, ll, fl.x);
      b.add(hl, ll, fl.y);
    }
    buf[N + q] = {a.get(), b.get()};
  }
}

template <typename T>
struct Offset {
  // FP32 lines are shifted by the mean of their end values before the FFT of a
  // derivative (the FC derivative of a constant vanishes up to the fit
  // residual); FP64 lines, and filtered lines (the continuation of a constant
  // is not constant, so a filter does not commute with the shift), are
  // transformed as they are.
  static constexpr bool kShift = false;
};
template <>
struct Offset<float> {
  static constexpr bool kShift = true;
};

// Filter factor sigma(k) of the plan table at idx.
template <typename T>
__device__ __forceinline__ T flt_at(const CtxDev& c, int idx);
template <>
__device__ __forceinline__ double flt_at<double>(const CtxDev& c, int idx) { return __ldg(c.flt64 + idx); }
template <>
__device__ __forceinline__ float flt_at<float>(const CtxDev& c, int idx) { return __ldg(c.flt32 + idx); }

// FC derivative of two real lines packed in buf[0..N) (buf = a, scratch b):
// continuation, FFT, multiply by (i k)^order (order 0: by the filter factors
// sigma(k)), inverse FFT.  On return res[0..N) holds (d^order a, d^order b),
// already divided by n and scaled by (2 pi / (n h))^order; returns the result
// buffer.
template <typename T>
__device__ Cx<T>* fc_deriv_pair(Cx<T>* a, Cx<T>* b, const CtxDev& c, const PlanDev& pl, int d, T h, int order,
                                int lane) {
  const int N = pl.N, n = pl.n;
  T oa = T(0), ob = T(0);
  if (Offset<T>::kShift && order != 0) {
    const Cx<T> f0 = a[0], f1 = a[N - 1];
    oa = (f0.x + f1.x) * T(0.5);
    ob = (f0.y + f1.y) * T(0.5);
    __syncwarp();
    for (int t = lane; t < N; t += 32) a[t] = {a[t].x - oa, a[t].y - ob};
    __syncwarp();
  }
  continue_lines(a, c, pl, d, lane);
  __syncwarp();
  Cx<T>* r = warp_fft<T>(a, b, c, pl, false, lane);
  Cx<T>* s = (r == a) ? b : a;
  const T sc = T(6.283185307179586476925286766559) / (T(n) * h);
  const T inv_n = T(1) / T(n);
  for (int m = lane; m < n; m += 32) {
    const int km = (2 * m <= n) ? m : m - n;
    Cx<T> z = r[m];
    Cx<T> o;
    if (order == 1) {
      const T k = (2 * m == n) ? T(0) : T(km) * sc * inv_n;
      o = {-k * z.y, k * z.x};  // i k z
    } else if (order == 2) {
      const T k = T(km) * sc;
      const T f = -k * k * inv_n;
      o = {f * z.x, f * z.y};
    } else {
      const T f = flt_at<T>(c, pl.tw_off + m) * inv_n;
      o = {f * z.x, f * z.y};
    }
    r[m] = o;
  }
  __syncwarp();
  return warp_fft<T>(r, s, c, pl, true, lane);
}

// ------------------------------------------------------------ gas dynamics
template <typename T>
__device__ __forceinline__ T pressure(T rho, T mx, T my, T E, T gm1) {
  return gm1 * (E - T(0.5) * (mx * mx + my * my) / rho);
}

// Wall: remove the velocity component along the unit normal (nx, ny).
template <typename T>
__device__ __forceinline__ void wall_project(T* v, T nx, T ny) {
  const T nn = sqrt(nx * nx + ny * ny);
  nx /= nn;
  ny /= nn;
  const T mn = v[1] * nx + v[2] * ny;
  v[1] -= mn * nx;
  v[2] -= mn * ny;
}

// Apply the boundary conditions of the sides the point lies on, in the order
// left, right, bottom, top (paper §5 item 4: enforced at every stage), then
// for an L-shaped patch its inner wall edges i = m1 (j < m2) and j = m2
// (i < m1) and the corner node (m1, m2), a wall along the bisector of the
// two inward edge normals grad q1 / |grad q1| + grad q2 / |grad q2|.
// The work at a boundary point is out of line (called only there), so the
// inlined check keeps the update loops of the stage kernels short.
template <typename T>
__device__ __noinline__ void apply_bc_edge(const T* M, long long qs, T gm1, T pout, const PatchDev& P, int i, int j,
                                           long long q, T* v) {
  const bool on[4] = {i == 0 && j >= P.m2, i == P.n1 - 1, j == 0 && i >= P.m1, j == P.n2 - 1};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (!on[s]) continue;
    const int code = P.bc[s];
    if (code == 1) {  // wall
      if (P.cart) {
        v[s < 2 ? 1 : 2] = T(0);
      } else if (s < 2) {
        wall_project(v, M[3 * qs + q], -M[1 * qs + q]);
      } else {
        wall_project(v, -M[2 * qs + q], M[0 * qs + q]);
      }
    } else if (code == 2) {  // inflow
      v[0] = inflow_of<T>(P, 0);
      v[1] = inflow_of<T>(P, 1);
      v[2] = inflow_of<T>(P, 2);
      v[3] = inflow_of<T>(P, 3);
    } else if (code == 3) {  // outflow pressure
      v[3] = pout / gm1 + T(0.5) * (v[1] * v[1] + v[2] * v[2]) / v[0];
    } else if (code == 5) {  // no-slip wall: momentum (its temperature: k_noslip_temperature)
      v[1] = T(0);
      v[2] = T(0);
    }
  }
  if (P.m1 > 0) {
    if (i == P.m1 && j < P.m2) {
      if (P.cart) v[1] = T(0);
      else wall_project(v, M[3 * qs + q], -M[1 * qs + q]);
    } else if (j == P.m2 && i < P.m1) {
      if (P.cart) v[2] = T(0);
      else wall_project(v, -M[2 * qs + q], M[0 * qs + q]);
    } else if (i == P.m1 && j == P.m2) {
      T ax = T(1), ay = T(0), bx = T(0), by = T(1);
      if (!P.cart) {
        const T sg = M[4 * qs + q] < T(0) ? T(-1) : T(1);
        ax = sg * M[3 * qs + q];
        ay = -sg * M[1 * qs + q];
        bx = -sg * M[2 * qs + q];
        by = sg * M[0 * qs + q];
      }
      const T na = sqrt(ax * ax + ay * ay), nb = sqrt(bx * bx + by * by);
      wall_project(v, ax / na + bx / nb, ay / na + by / nb);
    }
  }
}
template <typename T>
__device__ __forceinline__ void apply_bc(const CtxDev& c, const PatchDev& P, int i, int j, long long q, T* v) {
  const bool edge = i == 0 || j == 0 || i == P.n1 - 1 || j == P.n2 - 1 ||
                    (P.m1 > 0 && ((i == P.m1 && j <= P.m2) || (j == P.m2 && i <= P.m1)));
  if (edge) apply_bc_edge<T>(metrics<T>(c), c.qstride, gm1_of<T>(c), p_out_of<T>(c), P, i, j, q, v);
}


// ------------------------------------------------------------ register FFT
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Everything one FC derivative of a line pair needs, by value (no pointer to
// the kernel's context, so nothing has to be spilled to local memory).
template <typename T>
struct LineOp {
  const Cx<T>* tw;      // the plan's n twiddles e^{-2 pi i k / n}
  const T* flt;         // the plan's n filter factors sigma(k)
  const double* t64;    // the plan's C x d table (FP64)
  const float* thi;     // FP32 split of the table (hi, lo)
  const float* tlo;
  const double* gQh;    // FP64 Gram basis (double-double) and the plan's FP64 Gram blend table
  const double* gQl;
  const double* gT64;
  const float* gQ32;    // FP32 Gram basis and the plan's FP32 Gram blend table
  const float* gT32;
  const float* gR32;    // the plan's continuation of a constant (row sums of A_R), FP32
  int N, C, n, d, n1reg;
  T h;                  // line spacing
};

template <typename T>
__device__ __forceinline__ LineOp<T> make_op(const CtxDev& c, const PlanDev& pl, T h);
template <>
__device__ __forceinline__ LineOp<double> make_op<double>(const CtxDev& c, const PlanDev& pl, double h) {
  return {reinterpret_cast<const Cx<double>*>(c.tw64 + pl.tw_off), c.flt64 + pl.tw_off, c.tab64 + pl.tab_off,
          c.tabhi + pl.tab_off, c.tablo + pl.tab_off, c.gramQ64h, c.gramQ64l, c.gramT64 + pl.tg_off,
          c.gramQ, c.gramT + pl.tg_off, c.gramR + pl.rs_off, pl.N, pl.C, pl.n, c.d, pl.n1reg, h};
}
template <>
__device__ __forceinline__ LineOp<float> make_op<float>(const CtxDev& c, const PlanDev& pl, float h) {
  return {reinterpret_cast<const Cx<float>*>(c.tw32 + pl.tw_off), c.flt32 + pl.tw_off, c.tab64 + pl.tab_off,
          c.tabhi + pl.tab_off, c.tablo + pl.tab_off, c.gramQ64h, c.gramQ64l, c.gramT64 + pl.tg_off,
          c.gramQ, c.gramT + pl.tg_off, c.gramR + pl.rs_off, pl.N, pl.C, pl.n, c.d, pl.n1reg, h};
}

template <typename T>
__device__ __forceinline__ Cx<T> ldtw(const Cx<T>* tw, int k) {
  return tw[k];
}

// Four-step FFT of length n = 32 * N1 held in registers: lane L holds
// x[L + 32 j1], j1 < N1.  Forward: length-N1 DFT per lane, twiddle
// w_n^{L k1}, 32-point DIF DFT across lanes by shuffles (lane L then holds
// X[k1 + N1 bitrev5(L)]).  Inverse: 32-point DIT DFT across lanes, conjugate
// twiddle, length-N1 DFT per lane, natural order again.  All roots come from
// the plan's length-n table: w_N1^m = tw[32 m], w_32^t = tw[N1 t].
template <typename T>
__device__ __forceinline__ Cx<T> shfl_xor_c(Cx<T> v, int m) {
  return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}

template <typename T, int N1>
__device__ __forceinline__ void lane_dft(Cx<T>* x, const Cx<T>* tw, bool inv) {
  Cx<T> W[N1];
#pragma unroll
  for (int m = 0; m < N1; ++m) {
    W[m] = ldtw(tw, 32 * m);
    if (inv) W[m].y = -W[m].y;
  }
  Cx<T> o[N1];
#pragma unroll
  for (int k = 0; k < N1; ++k) {
    Cx<T> acc = x[0];
#pragma unroll
    for (int j = 1; j < N1; ++j) {
      const Cx<T> p = cmul(x[j], W[(j * k) % N1]);
      acc.x += p.x;
      acc.y += p.y;
    }
    o[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < N1; ++k) x[k] = o[k];
}

// The radix-2 stages across lanes are written without a branch on the lane's
// half: forward (decimation in frequency) every lane forms w' (p + sg x) with
// sg = +1, w' = 1 in the lower half (x + p) and sg = -1, w' = w in the upper
// half ((p - x) w); inverse (decimation in time) every lane forms
// a + w'' b with (a, b, w'') = (x, p, w) below and (p, x, -w) above.
template <typename T, int N1>
__device__ __forceinline__ void reg_fft(Cx<T>* x, const Cx<T>* tw, bool inv, int lane) {
  if (!inv) {
    lane_dft<T, N1>(x, tw, false);
#pragma unroll
    for (int k = 1; k < N1; ++k) x[k] = cmul(x[k], ldtw(tw, lane * k));
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const bool hi = lane & s;
      const Cx<T> w0 = ldtw(tw, (lane & (s - 1)) * (16 / s) * N1);
      const Cx<T> w = hi ? w0 : Cx<T>{T(1), T(0)};
      const T sg = hi ? T(-1) : T(1);
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const Cx<T> p = shfl_xor_c(x[k], s);
        x[k] = cmul(Cx<T>{fma_t(sg, x[k].x, p.x), fma_t(sg, x[k].y, p.y)}, w);
      }
    }
  } else {
#pragma unroll
    for (int s = 1; s <= 16; s <<= 1) {
      const bool hi = lane & s;
      const Cx<T> w0 = ldtw(tw, (lane & (s - 1)) * (16 / s) * N1);
      const Cx<T> w = hi ? Cx<T>{-w0.x, w0.y} : Cx<T>{w0.x, -w0.y};   // -conj(w0) above, conj(w0) below
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const Cx<T> p = shfl_xor_c(x[k], s);
        const Cx<T> a = hi ? p : x[k], b = hi ? x[k] : p;
        x[k] = {fma_t(w.x, b.x, fma_t(-w.y, b.y, a.x)), fma_t(w.x, b.y, fma_t(w.y, b.x, a.y))};
      }
    }
#pragma unroll
    for (int k = 1; k < N1; ++k) {
      Cx<T> w = ldtw(tw, lane * k);
      w.y = -w.y;
      x[k] = cmul(x[k], w);
    }
    lane_dft<T, N1>(x, tw, true);
  }
}

__device__ __forceinline__ int bitrev5(int v) { return __brev(v) >> 27; }

// FC derivative of the lines a and b (b may be null) with the register FFT;
// results times `scale` go to oa[t*soa], ob[t*sob] for t < N.
template <typename T, int N1>
__device__ __forceinline__ void reg_deriv_pair(const T* a, int sa, const T* b, int sb, T* oa, int soa, T* ob, int sob,
                                               T scale, const LineOp<T>& op, int order, int lane) {
  const int N = op.N, n = 32 * N1;
  T offa = T(0), offb = T(0);
  if (Offset<T>::kShift && order != 0) {
    offa = (a[0] + a[(N - 1) * sa]) * T(0.5);
    if (b) offb = (b[0] + b[(N - 1) * sb]) * T(0.5);
  }
  Cx<T> x[N1];
  {
    // Gram form of the continuation: lanes k < d project the four line ends
    // on the Gram basis (FP64: compensated sums with the double-double basis;
    // FP32: plain sums of the shifted values, whose high-degree coefficients
    // are small for smooth data), every lane reads the coefficients of its
    // gap points by shuffles and sums the blend values T
    const int d = op.d;
    T aR = T(0), aL = T(0), bR = T(0), bL = T(0);
    if (lane < d) {
      if constexpr (sizeof(T) == 8) {
        aR = gram_coef64(a + (N - d) * sa, sa, op.gQh, op.gQl, d, lane);
        aL = gram_coef64(a + (d - 1) * sa, -sa, op.gQh, op.gQl, d, lane);
        if (b) {
          bR = gram_coef64(b + (N - d) * sb, sb, op.gQh, op.gQl, d, lane);
          bL = gram_coef64(b + (d - 1) * sb, -sb, op.gQh, op.gQl, d, lane);
        }
      } else {
        const float caR = a[(N - 1) * sa], caL = a[0];
        const float cbR = b ? b[(N - 1) * sb] : 0.f, cbL = b ? b[0] : 0.f;
        for (int m = 0; m < d; ++m) {
          const float q = __ldg(op.gQ32 + m * d + lane);
          aR = fmaf(q, a[(N - d + m) * sa] - caR, aR);
          aL = fmaf(q, a[(d - 1 - m) * sa] - caL, aL);
          if (b) {
            bR = fmaf(q, b[(N - d + m) * sb] - cbR, bR);
            bL = fmaf(q, b[(d - 1 - m) * sb] - cbL, bL);
          }
        }
      }
    }
    // FP32: the ends' values relative to the line offset, continued as constants
    T eaR = T(0), eaL = T(0), ebR = T(0), ebL = T(0);
    if constexpr (sizeof(T) == 4) {
      eaR = a[(N - 1) * sa] - offa;
      eaL = a[0] - offa;
      if (b) {
        ebR = b[(N - 1) * sb] - offb;
        ebL = b[0] - offb;
      }
    }
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int j = lane + 32 * j1;
      x[j1] = {T(0), T(0)};
      if (j < N) {
        x[j1].x = a[j * sa] - offa;
        x[j1].y = b ? b[j * sb] - offb : T(0);
      }
      if (32 * j1 + 31 >= N) {   // this register row holds gap points (uniform over the warp)
        const int q = j - N;
        T sa_ = T(0), sb_ = T(0);
        for (int k = 0; k < d; ++k) {
          const T gaR = __shfl_sync(0xffffffffu, aR, k), gaL = __shfl_sync(0xffffffffu, aL, k);
          const T gbR = __shfl_sync(0xffffffffu, bR, k), gbL = __shfl_sync(0xffffffffu, bL, k);
          if (q >= 0) {
            T tr, tl;
            if constexpr (sizeof(T) == 8) {
              tr = __ldg(op.gT64 + q * d + k);
              tl = __ldg(op.gT64 + (op.C - 1 - q) * d + k);
            } else {
              tr = __ldg(op.gT32 + q * d + k);
              tl = __ldg(op.gT32 + (op.C - 1 - q) * d + k);
            }
            sa_ = fma_t(tr, gaR, fma_t(tl, gaL, sa_));
            sb_ = fma_t(tr, gbR, fma_t(tl, gbL, sb_));
          }
        }
        if constexpr (sizeof(T) == 4) {
          if (q >= 0) {
            const float rr = __ldg(op.gR32 + q), rl = __ldg(op.gR32 + op.C - 1 - q);
            sa_ = fmaf(eaR, rr, fmaf(eaL, rl, sa_));
            sb_ = fmaf(ebR, rr, fmaf(ebL, rl, sb_));
          }
        }
        if (q >= 0) x[j1] = {sa_, b ? sb_ : T(0)};
      }
    }
  }
  reg_fft<T, N1>(x, op.tw, false, lane);
  const T sc = T(6.283185307179586476925286766559) / (T(n) * op.h);
  const T inv_n = scale / T(n);
  const int k2 = bitrev5(lane);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    const int k = k1 + N1 * k2;
    const int km = (2 * k <= n) ? k : k - n;
    const Cx<T> z = x[k1];
    if (order == 1) {
      const T kk = (2 * k == n) ? T(0) : T(km) * sc * inv_n;
      x[k1] = {-kk * z.y, kk * z.x};
    } else if (order == 2) {
      const T kk = T(km) * sc;
      const T f = -kk * kk * inv_n;
      x[k1] = {f * z.x, f * z.y};
    } else {
      const T f = __ldg(op.flt + k) * inv_n;
      x[k1] = {f * z.x, f * z.y};
    }
  }
  reg_fft<T, N1>(x, op.tw, true, lane);
#pragma unroll
  for (int j1 = 0; j1 < N1; ++j1) {
    const int j = lane + 32 * j1;
    if (j < N) {
      oa[j * soa] = x[j1].x;
      if (ob) ob[j * sob] = x[j1].y;
    }
  }
}

// ------------------------------------------------------------ paired FP32 FFT
// Two line pairs of one plan per warp (four real lines: the fields of one row
// or column), in the paired FP32 instructions of sm_100+ (add/mul/fma.f32x2:
// one instruction for both pairs).  C2 holds one complex value of each pair:
// re = (pair 0, pair 1), im likewise.  The 32-lane four-step FFT of
// reg_fft, with the radix-2 stages across lanes in the form
// out = partner's (w' x) + sg (w' x): every lane first multiplies its own
// value by w' (1 below, the stage twiddle above), so neither direction needs a
// select on the lane's half.
struct C2 {
  float2 re, im;
};
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
// a times the complex scalar w (the same for both pairs)
__device__ __forceinline__ C2 c2mul(C2 a, float wr, float wi) {
  return {__ffma2_rn(a.im, bc2(-wi), __fmul2_rn(a.re, bc2(wr))), __ffma2_rn(a.re, bc2(wi), __fmul2_rn(a.im, bc2(wr)))};
}
__device__ __forceinline__ C2 c2add(C2 a, C2 b) { return {__fadd2_rn(a.re, b.re), __fadd2_rn(a.im, b.im)}; }
__device__ __forceinline__ C2 shfl_xor_c2(C2 v, int m) {
  return {make_float2(__shfl_xor_sync(0xffffffffu, v.re.x, m), __shfl_xor_sync(0xffffffffu, v.re.y, m)),
          make_float2(__shfl_xor_sync(0xffffffffu, v.im.x, m), __shfl_xor_sync(0xffffffffu, v.im.y, m))};
}

template <int N1>
__device__ __forceinline__ void lane_dft2(C2* x, const Cx<float>* tw, bool inv) {
  Cx<float> W[N1];
#pragma unroll
  for (int m = 0; m < N1; ++m) {
    W[m] = ldtw(tw, 32 * m);
    if (inv) W[m].y = -W[m].y;
  }
  C2 o[N1];
#pragma unroll
  for (int k = 0; k < N1; ++k) {
    C2 acc = x[0];
#pragma unroll
    for (int j = 1; j < N1; ++j) acc = c2add(acc, c2mul(x[j], W[(j * k) % N1].x, W[(j * k) % N1].y));
    o[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < N1; ++k) x[k] = o[k];
}

template <int N1>
__device__ __forceinline__ void reg_fft2(C2* x, const Cx<float>* tw, bool inv, int lane) {
  if (!inv) {
    lane_dft2<N1>(x, tw, false);
#pragma unroll
    for (int k = 1; k < N1; ++k) {
      const Cx<float> w = ldtw(tw, lane * k);
      x[k] = c2mul(x[k], w.x, w.y);
    }
    // decimation in frequency: lower lane x + p, upper lane (p - x) w
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const bool hi = lane & s;
      const Cx<float> w0 = ldtw(tw, (lane & (s - 1)) * (16 / s) * N1);
      const float wr = hi ? w0.x : 1.f, wi = hi ? w0.y : 0.f;
      const float2 sg = bc2(hi ? -1.f : 1.f);
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const C2 p = shfl_xor_c2(x[k], s);
        x[k] = c2mul({__ffma2_rn(sg, x[k].re, p.re), __ffma2_rn(sg, x[k].im, p.im)}, wr, wi);
      }
    }
  } else {
    // decimation in time: lower lane x + conj(w0) p, upper lane p - conj(w0) x
#pragma unroll
    for (int s = 1; s <= 16; s <<= 1) {
      const bool hi = lane & s;
      const Cx<float> w0 = ldtw(tw, (lane & (s - 1)) * (16 / s) * N1);
      const float wr = hi ? w0.x : 1.f, wi = hi ? -w0.y : 0.f;
      const float2 sg = bc2(hi ? -1.f : 1.f);
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const C2 v = c2mul(x[k], wr, wi);
        const C2 p = shfl_xor_c2(v, s);
        x[k] = {__ffma2_rn(sg, v.re, p.re), __ffma2_rn(sg, v.im, p.im)};
      }
    }
#pragma unroll
    for (int k = 1; k < N1; ++k) {
      const Cx<float> w = ldtw(tw, lane * k);
      x[k] = c2mul(x[k], w.x, -w.y);
    }
    lane_dft2<N1>(x, tw, true);
  }
}

// FC derivative of the line pairs (a, b) and (c, e) of one plan (b, c, e may
// be null), the FP32 form of reg_deriv_pair for two pairs at once: the same
// continuation (Gram coefficients of the end values relative to each end's own
// value, blend table, continuation of the constant part), FFT, (i k)^order
// and inverse FFT; results times `scale` go to oa[t*soa] ... oe[t*soe].
template <int N1>
__device__ __forceinline__ void reg_deriv_quad(const float* a, int sa, const float* b, int sb, const float* c, int sc_,
                                               const float* e, int se, float* oa, int soa, float* ob, int sob,
                                               float* oc, int soc, float* oe, int soe, float scale,
                                               const LineOp<float>& op, int order, int lane) {
  const int N = op.N, n = 32 * N1, d = op.d;
  float off[4] = {0.f, 0.f, 0.f, 0.f};
  if (order != 0) {   // shift by the mean of the end values (Offset<float>)
    off[0] = (a[0] + a[(N - 1) * sa]) * 0.5f;
    if (b) off[1] = (b[0] + b[(N - 1) * sb]) * 0.5f;
    if (c) off[2] = (c[0] + c[(N - 1) * sc_]) * 0.5f;
    if (e) off[3] = (e[0] + e[(N - 1) * se]) * 0.5f;
  }
  const float* L[4] = {a, b, c, e};
  const int S[4] = {sa, sb, sc_, se};
  // lanes k < d: Gram coefficient k of every line at both ends, of the values
  // relative to that end's own value
  float gR[4] = {0.f, 0.f, 0.f, 0.f}, gL[4] = {0.f, 0.f, 0.f, 0.f};
  if (lane < d) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      if (!L[l]) continue;
      const float cR = L[l][(N - 1) * S[l]], cL = L[l][0];
      for (int m = 0; m < d; ++m) {
        const float q = __ldg(op.gQ32 + m * d + lane);
        gR[l] = fmaf(q, L[l][(N - d + m) * S[l]] - cR, gR[l]);
        gL[l] = fmaf(q, L[l][(d - 1 - m) * S[l]] - cL, gL[l]);
      }
    }
  }
  // the ends' values relative to the line offsets, continued as constants
  float eR[4] = {0.f, 0.f, 0.f, 0.f}, eL[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int l = 0; l < 4; ++l)
    if (L[l]) {
      eR[l] = L[l][(N - 1) * S[l]] - off[l];
      eL[l] = L[l][0] - off[l];
    }
  C2 x[N1];
#pragma unroll
  for (int j1 = 0; j1 < N1; ++j1) {
    const int j = lane + 32 * j1;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (j < N) {
#pragma unroll
      for (int l = 0; l < 4; ++l)
        if (L[l]) v[l] = L[l][j * S[l]] - off[l];
    }
    if (32 * j1 + 31 >= N) {   // this register row holds gap points (uniform over the warp)
      const int q = j - N;
      float2 sre = bc2(0.f), sim = bc2(0.f);   // (a, c) and (b, e) gap values
      for (int k = 0; k < d; ++k) {
        const float2 rRe = make_float2(__shfl_sync(0xffffffffu, gR[0], k), __shfl_sync(0xffffffffu, gR[2], k));
        const float2 rIm = make_float2(__shfl_sync(0xffffffffu, gR[1], k), __shfl_sync(0xffffffffu, gR[3], k));
        const float2 lRe = make_float2(__shfl_sync(0xffffffffu, gL[0], k), __shfl_sync(0xffffffffu, gL[2], k));
        const float2 lIm = make_float2(__shfl_sync(0xffffffffu, gL[1], k), __shfl_sync(0xffffffffu, gL[3], k));
        if (q >= 0) {
          const float2 tr = bc2(__ldg(op.gT32 + q * d + k)), tl = bc2(__ldg(op.gT32 + (op.C - 1 - q) * d + k));
          sre = __ffma2_rn(tr, rRe, __ffma2_rn(tl, lRe, sre));
          sim = __ffma2_rn(tr, rIm, __ffma2_rn(tl, lIm, sim));
        }
      }
      if (q >= 0) {
        const float2 rr = bc2(__ldg(op.gR32 + q)), rl = bc2(__ldg(op.gR32 + op.C - 1 - q));
        sre = __ffma2_rn(make_float2(eR[0], eR[2]), rr, __ffma2_rn(make_float2(eL[0], eL[2]), rl, sre));
        sim = __ffma2_rn(make_float2(eR[1], eR[3]), rr, __ffma2_rn(make_float2(eL[1], eL[3]), rl, sim));
        v[0] = sre.x;
        v[2] = c ? sre.y : 0.f;
        v[1] = b ? sim.x : 0.f;
        v[3] = e ? sim.y : 0.f;
      }
    }
    x[j1] = {make_float2(v[0], v[2]), make_float2(v[1], v[3])};
  }
  reg_fft2<N1>(x, op.tw, false, lane);
  const float sc = 6.283185307179586476925286766559f / (float(n) * op.h);
  const float inv_n = scale / float(n);
  const int k2 = bitrev5(lane);
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    const int k = k1 + N1 * k2;
    const int km = (2 * k <= n) ? k : k - n;
    const C2 z = x[k1];
    if (order == 1) {
      const float kk = (2 * k == n) ? 0.f : float(km) * sc * inv_n;
      x[k1] = {__fmul2_rn(bc2(-kk), z.im), __fmul2_rn(bc2(kk), z.re)};
    } else if (order == 2) {
      const float kk = float(km) * sc;
      const float f = -kk * kk * inv_n;
      x[k1] = {__fmul2_rn(bc2(f), z.re), __fmul2_rn(bc2(f), z.im)};
    } else {
      const float f = __ldg(op.flt + k) * inv_n;
      x[k1] = {__fmul2_rn(bc2(f), z.re), __fmul2_rn(bc2(f), z.im)};
    }
  }
  reg_fft2<N1>(x, op.tw, true, lane);
#pragma unroll
  for (int j1 = 0; j1 < N1; ++j1) {
    const int j = lane + 32 * j1;
    if (j < N) {
      oa[j * soa] = x[j1].re.x;
      if (ob) ob[j * sob] = x[j1].im.x;
      if (oc) oc[j * soc] = x[j1].re.y;
      if (oe) oe[j * soe] = x[j1].im.y;
    }
  }
}

// Shared-memory Stockham path for lengths that are not 32 * N1.
template <typename T>
__device__ void stk_deriv_pair(const T* a, int sa, const T* b, int sb, T* oa, int soa, T* ob, int sob, T scale,
                               const CtxDev& c, const PlanDev& pl, T h, int order, int lane, Cx<T>* buf0,
                               Cx<T>* buf1) {
  const int N = pl.N;
  for (int t = lane; t < N; t += 32) buf0[t] = {a[t * sa], b ? b[t * sb] : T(0)};
  __syncwarp();
  Cx<T>* r = fc_deriv_pair<T>(buf0, buf1, c, pl, c.d, h, order, lane);
  for (int t = lane; t < N; t += 32) {
    oa[t * soa] = r[t].x * scale;
    if (ob) ob[t * sob] = r[t].y * scale;
  }
  __syncwarp();
}

}  // namespace fcs

#include <type_traits>

#include "fcs_roots.cuh"

namespace fcs {

// ------------------------------------------------------------ small register DFTs
// In-place DFT of N complex values held in registers, N a product of small
// primes.  rdft_fwd leaves X[k] at register position p with k = rsigma(N, p)
// (Cooley-Tukey N = R M, R the smallest prime factor: R-point DFTs on the
// stride-M subsets, twiddles w_N^{jm kr}, M-point DFTs on the contiguous
// blocks).  rdft_inv applies the adjoint steps in reverse order, so
// rdft_inv(rdft_fwd(x)) = N x and it takes the permuted layout back to the
// natural one.  Roots come from the constant tables of fcs_roots.cuh (uniform
// compile-time indices: constant-bank operands).
__host__ __device__ constexpr int spf(int n) {
  for (int p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}
// Iterative (not recursive) so that it inlines and folds to a constant under
// unrolling: peel one smallest prime factor R of the size per level.
__host__ __device__ constexpr int rsigma(int N, int p) {
  int res = 0, mult = 1;
  while (spf(N) != N) {
    const int R = spf(N), M = N / R;
    res += mult * (p / M);
    p %= M;
    mult *= R;
    N = M;
  }
  return res + mult * p;
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1, so the
// permutation and root indices below are template constants (always folded).
template <int I, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < E) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, E>(f);
  }
}
template <int N, int P>
struct Sigma {
  static constexpr int value = rsigma(N, P);
};

template <typename T, int N>
__device__ __forceinline__ Cx<T> root(int m) {
  constexpr int off = kRootOff(N);
  static_assert(off >= 0, "no root table for this size");
  if constexpr (sizeof(T) == 8) {
    const double2 v = kRoots64[off + m % N];
    return {v.x, v.y};
  } else {
    const float2 v = kRoots32[off + m % N];
    return {v.x, v.y};
  }
}

template <typename T, int R, bool INV>
__device__ __forceinline__ void prime_dft(Cx<T>* v) {
  if constexpr (R == 2) {
    const Cx<T> a = v[0], b = v[1];
    v[0] = {a.x + b.x, a.y + b.y};
    v[1] = {a.x - b.x, a.y - b.y};
  } else if constexpr (R == 3) {
    const T s = T(0.86602540378443864676372317075294);
    const Cx<T> a = v[0], b = v[1], c = v[2];
    const Cx<T> t1 = {b.x + c.x, b.y + c.y};
    const Cx<T> t2 = {a.x - T(0.5) * t1.x, a.y - T(0.5) * t1.y};
    // -i s (b - c) for the forward transform, +i s (b - c) for the inverse
    Cx<T> r = {s * (b.y - c.y), -s * (b.x - c.x)};
    if (INV) r = {-r.x, -r.y};
    v[0] = {a.x + t1.x, a.y + t1.y};
    v[1] = {t2.x + r.x, t2.y + r.y};
    v[2] = {t2.x - r.x, t2.y - r.y};
  } else {
    Cx<T> o[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      Cx<T> acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        Cx<T> w = root<T, R>((r * q) % R);
        if (INV) w.y = -w.y;
        const Cx<T> p = cmul(v[r], w);
        acc.x += p.x;
        acc.y += p.y;
      }
      o[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = o[q];
  }
}

template <typename T, int N>
__device__ __forceinline__ void rdft_fwd(Cx<T>* x) {
  if constexpr (spf(N) == N) {
    prime_dft<T, N, false>(x);
  } else {
    constexpr int R = spf(N), M = N / R;
#pragma unroll
    for (int jm = 0; jm < M; ++jm) {
      Cx<T> v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = x[jm + M * r];
      prime_dft<T, R, false>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) x[jm + M * r] = v[r];
    }
#pragma unroll
    for (int jm = 1; jm < M; ++jm)
#pragma unroll
      for (int kr = 1; kr < R; ++kr) x[jm + M * kr] = cmul(x[jm + M * kr], root<T, N>(jm * kr));
#pragma unroll
    for (int kr = 0; kr < R; ++kr) rdft_fwd<T, M>(x + kr * M);
  }
}

template <typename T, int N>
__device__ __forceinline__ void rdft_inv(Cx<T>* x) {
  if constexpr (spf(N) == N) {
    prime_dft<T, N, true>(x);
  } else {
    constexpr int R = spf(N), M = N / R;
#pragma unroll
    for (int kr = 0; kr < R; ++kr) rdft_inv<T, M>(x + kr * M);
#pragma unroll
    for (int jm = 1; jm < M; ++jm)
#pragma unroll
      for (int kr = 1; kr < R; ++kr) {
        Cx<T> w = root<T, N>(jm * kr);
        w.y = -w.y;
        x[jm + M * kr] = cmul(x[jm + M * kr], w);
      }
#pragma unroll
    for (int jm = 0; jm < M; ++jm) {
      Cx<T> v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = x[jm + M * r];
      prime_dft<T, R, true>(v);
#pragma unroll
      for (int r = 0; r < R; ++r) x[jm + M * r] = v[r];
    }
  }
}

// ------------------------------------------------------------ two-level line FFT
// Line pair of FFT length n = 8 B handled by a group of 8 lanes (4 groups per
// warp).  z[j], j = b + B a (a < 8, b < B).  Lane t of the group:
//   forward: for its b in {t, t+8, ...}: 8-point DFT over a, twiddle
//   w_n^{b ka}, store Y[ka][b] to the group's shared tile (row pitch B+1);
//   after the warp barrier, the B-point DFT over b of row ka = t, so the lane
//   holds X[t + 8 k_b] with k_b = rsigma(B, p) at register p.
//   inverse: adjoint steps in reverse (B-point inverse DFT, conjugate twiddle,
//   transpose back, 8-point inverse DFTs), natural order again.
// FP32 continuation: Gram coefficients of the d end values (Q^T f), then the
// blend table T = A_R Q (no cancellation for smooth data, so plain FP32
// sums suffice); FP64: the same two steps, the projection compensated
// (gram_coef64).
template <typename T>
struct GramOp {
  const float* Q;     // d x d Gram basis (values at the d matching points), FP32
  const float* Tg;    // C x d blend values of the Gram polynomials, FP32
  const double* Qh;   // the basis as double-double (FP64 lines)
  const double* Ql;
  const double* Tg64; // C x d blend values, FP64
  const float* Rs;    // C values: continuation of a constant 1 from the right end (FP32)
};

template <typename T, int B>
__device__ __forceinline__ void tl_deriv_pair(const T* a, int sa, const T* b, int sb, T* oa, int soa, T* ob, int sob,
                                              T scale, const LineOp<T>& op, const GramOp<T>& gop, int order, int t,
                                              Cx<T>* tile, bool active) {
  constexpr int NB = B / 8;
  constexpr int MAXD = 5;  // degree bound of this path (contexts with d > 5 use the Stockham kernels)
  const int N = op.N, n = 8 * B, d = op.d;
  // ---- end values and continuation coefficients
  T offa = T(0), offb = T(0);
  if (active && Offset<T>::kShift && order != 0) {
    offa = (a[0] + a[(N - 1) * sa]) * T(0.5);
    if (b) offb = (b[0] + b[(N - 1) * sb]) * T(0.5);
  }
  // lane t (< d) of the group computes Gram coefficient k = t of both lines
  // and both ends (FP64: compensated sums with the double-double basis;
  // FP32: plain sums of the values relative to the end's own value, whose
  // differences are small for smooth data, the constant part entering
  // through the continuation of a constant, e* Rs); the group then shares
  // them by shuffles
  T gaR[MAXD], gaL[MAXD], gbR[MAXD], gbL[MAXD];
  {
    T cR = T(0), cL = T(0), dR = T(0), dL = T(0);
    if (active && t < d) {
      if constexpr (sizeof(T) == 4) {
        const float caR = a[(N - 1) * sa], caL = a[0];
        const float cbR = b ? b[(N - 1) * sb] : 0.f, cbL = b ? b[0] : 0.f;
        for (int m = 0; m < d; ++m) {
          const float q = __ldg(gop.Q + m * d + t);
          cR = fmaf(q, a[(N - d + m) * sa] - caR, cR);
          cL = fmaf(q, a[(d - 1 - m) * sa] - caL, cL);
          if (b) {
            dR = fmaf(q, b[(N - d + m) * sb] - cbR, dR);
            dL = fmaf(q, b[(d - 1 - m) * sb] - cbL, dL);
          }
        }
      } else {
        cR = gram_coef64(a + (N - d) * sa, sa, gop.Qh, gop.Ql, d, t);
        cL = gram_coef64(a + (d - 1) * sa, -sa, gop.Qh, gop.Ql, d, t);
        if (b) {
          dR = gram_coef64(b + (N - d) * sb, sb, gop.Qh, gop.Ql, d, t);
          dL = gram_coef64(b + (d - 1) * sb, -sb, gop.Qh, gop.Ql, d, t);
        }
      }
    }
    const int base = (threadIdx.x & 31) & ~7;  // first lane of the group
#pragma unroll
    for (int k = 0; k < MAXD; ++k) {
      gaR[k] = __shfl_sync(0xffffffffu, cR, base + k);
      gaL[k] = __shfl_sync(0xffffffffu, cL, base + k);
      gbR[k] = __shfl_sync(0xffffffffu, dR, base + k);
      gbL[k] = __shfl_sync(0xffffffffu, dL, base + k);
    }
  }
  auto input = [&](int j) -> Cx<T> {
    Cx<T> z = {T(0), T(0)};
    if (!active) return z;
    if (j < N) {
      z.x = a[j * sa] - offa;
      z.y = b ? b[j * sb] - offb : T(0);
    } else {
      const int q = j - N;
      T sa_ = T(0), sb_ = T(0);
#pragma unroll
      for (int k = 0; k < MAXD; ++k) {
        if (k >= d) continue;
        T tr, tl;
        if constexpr (sizeof(T) == 4) {
          tr = __ldg(gop.Tg + q * d + k);
          tl = __ldg(gop.Tg + (op.C - 1 - q) * d + k);
        } else {
          tr = __ldg(gop.Tg64 + q * d + k);
          tl = __ldg(gop.Tg64 + (op.C - 1 - q) * d + k);
        }
        sa_ = fma_t(tr, gaR[k], fma_t(tl, gaL[k], sa_));
        sb_ = fma_t(tr, gbR[k], fma_t(tl, gbL[k], sb_));
      }
      if constexpr (sizeof(T) == 4) {
        // the ends' values relative to the line offset, continued as constants
        const float rr = __ldg(gop.Rs + q), rl = __ldg(gop.Rs + op.C - 1 - q);
        sa_ = fmaf(a[(N - 1) * sa] - offa, rr, fmaf(a[0] - offa, rl, sa_));
        if (b) sb_ = fmaf(b[(N - 1) * sb] - offb, rr, fmaf(b[0] - offb, rl, sb_));
      }
      z = {sa_, b ? sb_ : T(0)};
    }
    return z;
  };
  // ---- stage 1: 8-point DFTs over a for each owned b (a rolled loop over
  // the columns keeps one copy of its body: the unrolled FFT is large and
  // instruction fetch stalls the warps)
  Cx<T> x[B];
#pragma unroll 1
  for (int i = 0; i < NB; ++i) {
    const int bb = t + 8 * i;
    Cx<T> v[8];
#pragma unroll
    for (int aa = 0; aa < 8; ++aa) v[aa] = input(bb + B * aa);
    rdft_fwd<T, 8>(v);
    static_for<0, 8>([&](auto P) {
      constexpr int p = decltype(P)::value;
      constexpr int ka = Sigma<8, p>::value;
      if constexpr (ka != 0) v[p] = cmul(v[p], ldtw(op.tw, bb * ka));
      tile[ka * (B + 1) + bb] = v[p];
    });
  }
  __syncwarp();
  // ---- stage 2: B-point DFT of row ka = t
#pragma unroll
  for (int bb = 0; bb < B; ++bb) x[bb] = tile[t * (B + 1) + bb];
  rdft_fwd<T, B>(x);
  // ---- (i k)^order
  const T sc = T(6.283185307179586476925286766559) / (T(n) * op.h);
  const T inv_n = scale / T(n);
  static_for<0, B>([&](auto P) {
    constexpr int p = decltype(P)::value;
    const int k = t + 8 * Sigma<B, p>::value;
    const int km = (2 * k <= n) ? k : k - n;
    const Cx<T> z = x[p];
    if (order == 1) {
      const T kk = (2 * k == n) ? T(0) : T(km) * sc * inv_n;
      x[p] = {-kk * z.y, kk * z.x};
    } else if (order == 2) {
      const T kk = T(km) * sc;
      const T f = -kk * kk * inv_n;
      x[p] = {f * z.x, f * z.y};
    } else {
      const T f = __ldg(op.flt + k) * inv_n;
      x[p] = {f * z.x, f * z.y};
    }
  });
  // ---- inverse: B-point inverse DFT, conjugate twiddle, transpose back
  rdft_inv<T, B>(x);
  __syncwarp();
#pragma unroll
  for (int bb = 0; bb < B; ++bb) {
    Cx<T> w = ldtw(op.tw, bb * t);
    w.y = -w.y;
    tile[t * (B + 1) + bb] = cmul(x[bb], w);
  }
  __syncwarp();
#pragma unroll 1
  for (int i = 0; i < NB; ++i) {
    const int bb = t + 8 * i;
    Cx<T> v[8];
    static_for<0, 8>([&](auto P) {
      constexpr int p = decltype(P)::value;
      v[p] = tile[Sigma<8, p>::value * (B + 1) + bb];
    });
    rdft_inv<T, 8>(v);
    if (active) {
#pragma unroll
      for (int aa = 0; aa < 8; ++aa) {
        const int j = bb + B * aa;
        if (j < N) {
          oa[j * soa] = v[aa].x;
          if (ob) ob[j * sob] = v[aa].y;
        }
      }
    }
  }
  __syncwarp();
}

// Jobs (line pairs) a warp runs at once: 4 on the two-level FFT (even N1),
// 1 on the 32-lane shuffle FFT (odd N1) and on the Stockham FFT (N1 = 0).
__host__ __device__ constexpr int jobs_per_round(int N1) { return (N1 > 0 && N1 % 2 == 0) ? 4 : 1; }

// FC derivative of a line pair by the FFT variant N1 selects.  Every lane of
// the warp calls it together; `active` is false for lanes whose group has no
// job this round.  tile: the group's transpose tile (two-level path);
// buf0/buf1: the warp's Stockham buffers (N1 = 0).
template <typename T, int N1>
__device__ __forceinline__ void line_deriv_pair(const T* a, int sa, const T* b, int sb, T* oa, int soa, T* ob, int sob,
                                                T scale, const CtxDev& c, const PlanDev& pl, T h, int order, int lane,
                                                Cx<T>* buf0, Cx<T>* buf1, Cx<T>* tile, bool active) {
  if constexpr (N1 == 0) {
    if (active) stk_deriv_pair<T>(a, sa, b, sb, oa, soa, ob, sob, scale, c, pl, h, order, lane, buf0, buf1);
  } else if constexpr (N1 % 2 == 1) {
    const LineOp<T> op = make_op<T>(c, pl, h);
    if (active) reg_deriv_pair<T, N1>(a, sa, b, sb, oa, soa, ob, sob, scale, op, order, lane);
  } else {
    const LineOp<T> op = make_op<T>(c, pl, h);
    const GramOp<T> gop{c.gramQ, c.gramT + pl.tg_off, c.gramQ64h, c.gramQ64l, c.gramT64 + pl.tg_off,
                        c.gramR + pl.rs_off};
    tl_deriv_pair<T, 4 * N1>(a, sa, b, sb, oa, soa, ob, sob, scale, op, gop, order, lane & 7, tile, active);
  }
}

// FP32 lines of the 32-lane shuffle FFT with n1 = 3, 5 go two pairs per warp
// in paired FP32 arithmetic (reg_deriv_quad): the pass kernels give it the
// four fields of one row or column, or four adjacent columns, which share a
// plan.  (n1 = 7, 9 would spill at 128 registers.)
template <typename T, int N1>
__host__ __device__ constexpr bool quad_path() {
  return sizeof(T) == 4 && (N1 == 3 || N1 == 5);
}
template <typename T, int N1>
__device__ __forceinline__ void line_deriv_quad(const T* a, int sa, const T* b, int sb, const T* c, int sc, const T* e,
                                                int se, T* oa, int soa, T* ob, int sob, T* oc, int soc, T* oe, int soe,
                                                T scale, const CtxDev& ctx, const PlanDev& pl, T h, int order, int lane,
                                                bool active) {
  if constexpr (quad_path<T, N1>()) {
    const LineOp<float> op = make_op<float>(ctx, pl, h);
    if (active) reg_deriv_quad<N1>(a, sa, b, sb, c, sc, e, se, oa, soa, ob, sob, oc, soc, oe, soe, scale, op, order, lane);
  }
}

}  // namespace fcs
