// Device code of the FC-SDNN stage library: line FFTs, FC derivatives, the
// Euler operator with the Runge-Kutta epilogue, exchange, reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fcs {

constexpr int kMaxStages = 12;
constexpr int kWarps = 4;             // warps per block of the line kernels

// ------------------------------------------------------------ descriptors
struct PatchDev {
  int n1, n2, cart, pad0;
  int bc[4];
  int plan[2];          // FFT plan of lines along i (length n1) and along j (length n2)
  int wx_off, wy_off;   // first x-window and first y-window of the patch (per instance)
  int wpl_x, wpl_y;     // windows per x-line, per y-line
  long long soff, qoff; // offsets in the state and scalar layouts (per instance)
  double hx, hy;        // derivative spacing along i and j (physical if Cartesian, parameter otherwise)
  double hmax;          // largest physical spacing (viscosity scale)
  double Lx, Ly;        // Cartesian box lengths (metrics x_q1, y_q2)
};

struct PlanDev {
  int N, C, n, nst;
  int radix[kMaxStages];
  int tw_off;           // offset of the n twiddles
  int tab_off;          // offset of the C x d continuation table
  int n1reg;            // n = 32 * n1reg: register four-step FFT; 0: shared-memory Stockham FFT
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
  double inflow[4];
  double p_out;
  int ind_plan;                 // plan of the indicator (n = 16 + 26)
  int nmax;                     // longest line
  int nfmax;                    // longest FFT
  int stockham;                 // 1 if some plan needs the shared-memory FFT buffers
  int tw;                       // column-tile width of the pass along q2
  int n2max;                    // longest column (lines along q2)
};

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
// buf[0..N) holds two real lines as (re, im); append the C continuation values
//   cont[c] = sum_m A_R[c][m] f[N-d+m] + sum_m A_R[C-1-c][m] f[d-1-m]
// (FC-Gram right blend-to-zero plus the reflected left blend).
__device__ __forceinline__ void continue_lines(Cx<double>* buf, const CtxDev& c, const PlanDev& pl, int d,
                                               int lane) {
  const double* tab = c.tab64 + pl.tab_off;
  const int N = pl.N, C = pl.C;
  for (int q = lane; q < C; q += 32) {
    const double* tr = tab + q * d;
    const double* tl = tab + (C - 1 - q) * d;
    double sa = 0.0, sb = 0.0;
    for (int m = 0; m < d; ++m) {
      const double ar = __ldg(tr + m), al = __ldg(tl + m);
      const Cx<double> fr = buf[N - d + m], fl = buf[d - 1 - m];
      sa = fma(ar, fr.x, sa);
      sb = fma(ar, fr.y, sb);
      sa = fma(al, fl.x, sa);
      sb = fma(al, fl.y, sb);
    }
    buf[N + q] = {sa, sb};
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
  // FP32 lines are shifted by the mean of their end values before the FFT
  // (the FC derivative of a constant vanishes up to the fit residual); FP64
  // lines are transformed as they are.
  static constexpr bool kShift = false;
};
template <>
struct Offset<float> {
  static constexpr bool kShift = true;
};

// FC derivative of two real lines packed in buf[0..N) (buf = a, scratch b):
// continuation, FFT, multiply by (i k)^order, inverse FFT.  On return res[0..N)
// holds (d^order a, d^order b) / n... already divided by n and scaled by
// (2 pi / (n h))^order; returns the result buffer.
template <typename T>
__device__ Cx<T>* fc_deriv_pair(Cx<T>* a, Cx<T>* b, const CtxDev& c, const PlanDev& pl, int d, T h, int order,
                                int lane) {
  const int N = pl.N, n = pl.n;
  if (Offset<T>::kShift) {
    const Cx<T> f0 = a[0], f1 = a[N - 1];
    const T oa = (f0.x + f1.x) * T(0.5), ob = (f0.y + f1.y) * T(0.5);
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
    } else {
      const T k = T(km) * sc;
      const T f = -k * k * inv_n;
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

// ------------------------------------------------------------ register FFT
// Everything one FC derivative of a line pair needs, by value (no pointer to
// the kernel's context, so nothing has to be spilled to local memory).
template <typename T>
struct LineOp {
  const Cx<T>* tw;      // the plan's n twiddles e^{-2 pi i k / n}
  const double* t64;    // the plan's C x d table (FP64)
  const float* thi;     // FP32 split of the table (hi, lo)
  const float* tlo;
  int N, C, n, d, n1reg;
  T h;                  // line spacing
};

template <typename T>
__device__ __forceinline__ LineOp<T> make_op(const CtxDev& c, const PlanDev& pl, T h);
template <>
__device__ __forceinline__ LineOp<double> make_op<double>(const CtxDev& c, const PlanDev& pl, double h) {
  return {reinterpret_cast<const Cx<double>*>(c.tw64 + pl.tw_off), c.tab64 + pl.tab_off, c.tabhi + pl.tab_off,
          c.tablo + pl.tab_off, pl.N, pl.C, pl.n, c.d, pl.n1reg, h};
}
template <>
__device__ __forceinline__ LineOp<float> make_op<float>(const CtxDev& c, const PlanDev& pl, float h) {
  return {reinterpret_cast<const Cx<float>*>(c.tw32 + pl.tw_off), c.tab64 + pl.tab_off, c.tabhi + pl.tab_off,
          c.tablo + pl.tab_off, pl.N, pl.C, pl.n, c.d, pl.n1reg, h};
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

template <typename T, int N1>
__device__ __forceinline__ void reg_fft(Cx<T>* x, const Cx<T>* tw, bool inv, int lane) {
  if (!inv) {
    lane_dft<T, N1>(x, tw, false);
#pragma unroll
    for (int k = 1; k < N1; ++k) x[k] = cmul(x[k], ldtw(tw, lane * k));
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const Cx<T> w = ldtw(tw, (lane & (s - 1)) * (16 / s) * N1);
      const bool hi = lane & s;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const Cx<T> p = shfl_xor_c(x[k], s);
        if (!hi) x[k] = {x[k].x + p.x, x[k].y + p.y};
        else x[k] = cmul(Cx<T>{p.x - x[k].x, p.y - x[k].y}, w);
      }
    }
  } else {
#pragma unroll
    for (int s = 1; s <= 16; s <<= 1) {
      Cx<T> w = ldtw(tw, (lane & (s - 1)) * (16 / s) * N1);
      w.y = -w.y;
      const bool hi = lane & s;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const Cx<T> p = shfl_xor_c(x[k], s);
        if (!hi) {
          const Cx<T> q = cmul(p, w);
          x[k] = {x[k].x + q.x, x[k].y + q.y};
        } else {
          const Cx<T> q = cmul(x[k], w);
          x[k] = {p.x - q.x, p.y - q.y};
        }
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

// Continuation value q (0 <= q < C) of the line a (stride sa) minus offset o:
// sum_m A_R[q][m] a[N-d+m] + A_R[C-1-q][m] a[d-1-m]
__device__ __forceinline__ double cont_value(const double* a, int sa, double o, const LineOp<double>& op, int q) {
  const double* tr = op.t64 + q * op.d;
  const double* tl = op.t64 + (op.C - 1 - q) * op.d;
  double s = 0.0;
  for (int m = 0; m < op.d; ++m) {
    s = fma(__ldg(tr + m), a[(op.N - op.d + m) * sa] - o, s);
    s = fma(__ldg(tl + m), a[(op.d - 1 - m) * sa] - o, s);
  }
  return s;
}
__device__ __forceinline__ float cont_value(const float* a, int sa, float o, const LineOp<float>& op, int q) {
  const int rr = q * op.d, rl = (op.C - 1 - q) * op.d;
  Dot2 acc{0.f, 0.f};
  for (int m = 0; m < op.d; ++m) {
    acc.add(__ldg(op.thi + rr + m), __ldg(op.tlo + rr + m), __fsub_rn(a[(op.N - op.d + m) * sa], o));
    acc.add(__ldg(op.thi + rl + m), __ldg(op.tlo + rl + m), __fsub_rn(a[(op.d - 1 - m) * sa], o));
  }
  return acc.get();
}

// FC derivative of the lines a and b (b may be null) with the register FFT;
// results times `scale` go to oa[t*soa], ob[t*sob] for t < N.
template <typename T, int N1>
__device__ __forceinline__ void reg_deriv_pair(const T* a, int sa, const T* b, int sb, T* oa, int soa, T* ob, int sob,
                                               T scale, const LineOp<T>& op, int order, int lane) {
  const int N = op.N, n = 32 * N1;
  T offa = T(0), offb = T(0);
  if (Offset<T>::kShift) {
    offa = (a[0] + a[(N - 1) * sa]) * T(0.5);
    if (b) offb = (b[0] + b[(N - 1) * sb]) * T(0.5);
  }
  Cx<T> x[N1];
#pragma unroll
  for (int j1 = 0; j1 < N1; ++j1) {
    const int j = lane + 32 * j1;
    if (j < N) {
      x[j1].x = a[j * sa] - offa;
      x[j1].y = b ? b[j * sb] - offb : T(0);
    } else {
      x[j1].x = cont_value(a, sa, offa, op, j - N);
      x[j1].y = b ? cont_value(b, sb, offb, op, j - N) : T(0);
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
    } else {
      const T kk = T(km) * sc;
      const T f = -kk * kk * inv_n;
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

// FC derivative of a line pair: register FFT of length 32 * N1, or (N1 = 0)
// the shared-memory Stockham FFT, which handles any 7-smooth length.
template <typename T, int N1>
__device__ __forceinline__ void line_deriv_pair(const T* a, int sa, const T* b, int sb, T* oa, int soa, T* ob, int sob,
                                                T scale, const CtxDev& c, const PlanDev& pl, T h, int order, int lane,
                                                Cx<T>* buf0, Cx<T>* buf1) {
  if constexpr (N1 == 0) {
    stk_deriv_pair<T>(a, sa, b, sb, oa, soa, ob, sob, scale, c, pl, h, order, lane, buf0, buf1);
  } else {
    const LineOp<T> op = make_op<T>(c, pl, h);
    reg_deriv_pair<T, N1>(a, sa, b, sb, oa, soa, ob, sob, scale, op, order, lane);
  }
}

}  // namespace fcs
