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
};

struct PlanDev {
  int N, C, n, nst;
  int radix[kMaxStages];
  int tw_off;           // offset of the n twiddles
  int tab_off;          // offset of the C x d continuation table
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

}  // namespace fcs
