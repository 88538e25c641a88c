// Line kernels of the FC-SDNN stage library: FC derivative of line pairs and
// the two flux passes of the Euler operator (with the Runge-Kutta epilogue).
// Included only by the fcs_lines_*.cu translation units.
#pragma once

#include "fcs_device.cuh"
#include "fcs_launch.cuh"

namespace fcs {

// ============================================================ FC derivative
// One warp per pair of lines of one patch (two real lines -> one complex FFT).
template <typename T, int N1>
__global__ void __launch_bounds__(kWarps * 32) k_fc_deriv(CtxDev c, int dir, int order, const int4* __restrict__ pairs,
                                                           int npairs, const T* __restrict__ in, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * warp_line_bytes<T>(2, c.nmax, c.nfmax, N1 == 0);
  T* A = reinterpret_cast<T*>(base);
  T* B = A + c.nmax;
  Cx<T>* b0 = reinterpret_cast<Cx<T>*>(base + (((size_t)2 * c.nmax * sizeof(T) + 15) & ~size_t(15)));
  Cx<T>* b1 = b0 + c.nfmax;
  const long long total = (long long)c.instances * npairs;
  for (long long w = (long long)blockIdx.x * kWarps + warp; w < total; w += (long long)gridDim.x * kWarps) {
    const int inst = (int)(w / npairs);
    const int4 pr = pairs[w % npairs];
    const PatchDev P = c.patches[pr.x];
    const PlanDev pl = c.plans[P.plan[dir]];
    const int N = pl.N;
    const long long stride = dir == 0 ? 1 : P.n1;
    const long long la = dir == 0 ? (long long)pr.y * P.n1 : pr.y;
    const long long lb = pr.z < 0 ? -1 : (dir == 0 ? (long long)pr.z * P.n1 : pr.z);
    const T* src = in + inst * c.qstride + P.qoff;
    T* dst = out + inst * c.qstride + P.qoff;
    for (int t = lane; t < N; t += 32) {
      A[t] = src[la + t * stride];
      B[t] = lb >= 0 ? src[lb + t * stride] : T(0);
    }
    __syncwarp();
    const T h = T(1) / T(N - 1);
    line_deriv_pair<T, N1>(A, 1, lb >= 0 ? B : nullptr, 1, dst + la, (int)stride, lb >= 0 ? dst + lb : nullptr, (int)stride,
                       T(1), c, pl, h, order, lane, b0, b1);
    __syncwarp();
  }
}

// ============================================================ Euler operator

// Apply the boundary conditions of the sides the point lies on, in the order
// left, right, bottom, top (paper §5 item 4: enforced at every stage).
template <typename T>
__device__ __forceinline__ void apply_bc(const CtxDev& c, const PatchDev& P, int i, int j, long long q, T* v) {
  const T gm1 = T(c.gamma - 1.0);
  const bool on[4] = {i == 0, i == P.n1 - 1, j == 0, j == P.n2 - 1};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (!on[s]) continue;
    const int code = P.bc[s];
    if (code == 1) {  // wall
      if (P.cart) {
        v[s < 2 ? 1 : 2] = T(0);
      } else {
        const T* M = metrics<T>(c);
        const long long qs = c.qstride;
        T nx, ny;
        if (s < 2) {
          nx = M[3 * qs + q];
          ny = -M[1 * qs + q];
        } else {
          nx = -M[2 * qs + q];
          ny = M[0 * qs + q];
        }
        const T nn = sqrt(nx * nx + ny * ny);
        nx /= nn;
        ny /= nn;
        const T mn = v[1] * nx + v[2] * ny;
        v[1] -= mn * nx;
        v[2] -= mn * ny;
      }
    } else if (code == 2) {  // inflow
      v[0] = T(c.inflow[0]);
      v[1] = T(c.inflow[1]);
      v[2] = T(c.inflow[2]);
      v[3] = T(c.inflow[3]);
    } else if (code == 3) {  // outflow pressure
      v[3] = T(c.p_out) / gm1 + T(0.5) * (v[1] * v[1] + v[2] * v[2]) / v[0];
    }
  }
}

// Flux of Eq. (1) along direction DIR at one point, transformed for the
// parameter direction: DIR 0: y_q2 f - x_q2 g, DIR 1: -y_q1 f + x_q1 g;
// Cartesian: f resp. g, minus mu times the derivative dv (viscous flux).
template <typename T, int DIR>
__device__ __forceinline__ void point_flux(const CtxDev& c, const PatchDev& P, long long q, const T* v, const T* dv,
                                           T mu, bool visc, T* F) {
  const T gm1 = T(c.gamma - 1.0);
  const T rho = v[0], mx = v[1], my = v[2], En = v[3];
  const T u = mx / rho, w = my / rho;
  const T p = pressure<T>(rho, mx, my, En, gm1);
  if (P.cart) {
    if (DIR == 0) {
      F[0] = mx; F[1] = mx * u + p; F[2] = my * u; F[3] = (En + p) * u;
    } else {
      F[0] = my; F[1] = mx * w; F[2] = my * w + p; F[3] = (En + p) * w;
    }
    if (visc) {
#pragma unroll
      for (int f = 0; f < 4; ++f) F[f] -= mu * dv[f];
    }
  } else {
    const T* Mt = metrics<T>(c);
    T ca, cb;
    if (DIR == 0) {
      ca = Mt[3 * c.qstride + q];
      cb = -Mt[1 * c.qstride + q];
    } else {
      ca = -Mt[2 * c.qstride + q];
      cb = Mt[0 * c.qstride + q];
    }
    const T f0 = mx, f1 = mx * u + p, f2 = my * u, f3 = (En + p) * u;
    const T g0 = my, g1 = mx * w, g2 = my * w + p, g3 = (En + p) * w;
    F[0] = ca * f0 + cb * g0;
    F[1] = ca * f1 + cb * g1;
    F[2] = ca * f2 + cb * g2;
    F[3] = ca * f3 + cb * g3;
  }
}

// Pass along q1 (rows): R = -d/dq1 F1, one warp per row (rows are contiguous).
template <typename T, int N1>
__global__ void __launch_bounds__(kWarps * 32) k_xpass(CtxDev c, const T* __restrict__ e, const T* __restrict__ mu,
                                                        T* __restrict__ R) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nmax = c.nmax;
  unsigned char* base = smem_raw + (size_t)warp * warp_line_bytes<T>(9, nmax, c.nfmax, N1 == 0);
  T* E = reinterpret_cast<T*>(base);
  T* W = E + 4 * nmax;
  T* M = W + 4 * nmax;
  Cx<T>* b0 = reinterpret_cast<Cx<T>*>(base + (((size_t)9 * nmax * sizeof(T) + 15) & ~size_t(15)));
  Cx<T>* b1 = b0 + c.nfmax;
  const long long total = (long long)c.instances * c.nlines0;
  for (long long w = (long long)blockIdx.x * kWarps + warp; w < total; w += (long long)gridDim.x * kWarps) {
    const int inst = (int)(w / c.nlines0);
    const LineRef lr = c.lines0[w % c.nlines0];
    const PatchDev P = c.patches[lr.patch];
    const PlanDev pl = c.plans[P.plan[0]];
    const int N = pl.N;
    const long long np = (long long)P.n1 * P.n2;
    const long long l0 = (long long)lr.line * P.n1;
    const T* es = e + inst * c.sstride + P.soff + l0;
    const T h = T(P.hx);
    const bool visc = (mu != nullptr) && P.cart;
    for (int t = lane; t < N; t += 32) {
#pragma unroll
      for (int f = 0; f < 4; ++f) E[f * nmax + t] = es[f * np + t];
      if (visc) M[t] = mu[inst * c.qstride + P.qoff + l0 + t];
    }
    __syncwarp();
    T* Rs = R + inst * c.sstride + P.soff + l0;
    // jobs 0,1: W = d e/dx (viscous part, field pairs); jobs 2,3: R = -d F/dx
    for (int job = visc ? 0 : 2; job < 4; ++job) {
      if (job == 2) {
        for (int t = lane; t < N; t += 32) {
          T v[4], dv[4], F[4];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            v[f] = E[f * nmax + t];
            dv[f] = visc ? W[f * nmax + t] : T(0);
          }
          point_flux<T, 0>(c, P, P.qoff + l0 + t, v, dv, visc ? M[t] : T(0), visc, F);
#pragma unroll
          for (int f = 0; f < 4; ++f) W[f * nmax + t] = F[f];
        }
        __syncwarp();
      }
      const int pr = job & 1;
      const T* src = job < 2 ? E : W;
      T* oa = job < 2 ? W + 2 * pr * nmax : Rs + 2 * pr * np;
      T* ob = job < 2 ? W + (2 * pr + 1) * nmax : Rs + (2 * pr + 1) * np;
      line_deriv_pair<T, N1>(src + 2 * pr * nmax, 1, src + (2 * pr + 1) * nmax, 1, oa, 1, ob, 1, job < 2 ? T(1) : T(-1), c,
                         pl, h, 1, lane, b0, b1);
      __syncwarp();
    }
  }
}

// Pass along q2 on a tile of tw adjacent columns of one patch (coalesced row
// segments staged in shared memory): L = (R - d/dq2 F2)/J, then either L
// (MODE_RHS) or the Runge-Kutta stage with boundary conditions (MODE_RK).
template <typename T, int MODE, int N1>
__global__ void __launch_bounds__(kYWarps * 32) k_ypass(CtxDev c, const int2* __restrict__ tiles, int ntiles,
                                                         const T* __restrict__ e, const T* __restrict__ mu,
                                                         const T* __restrict__ R, StageArgs<T> st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tw = c.tw, ld = c.tw + 1, n2m = c.n2max;
  T* E = reinterpret_cast<T*>(smem_raw);           // [4][n2m][ld]
  T* D = E + 4 * n2m * ld;                         // [4][n2m][ld]
  T* M = D + 4 * n2m * ld;                         // [n2m][ld]
  Cx<T>* b0 = reinterpret_cast<Cx<T>*>(smem_raw + (((size_t)9 * n2m * ld * sizeof(T) + 15) & ~size_t(15))) +
              (size_t)warp * 2 * c.nfmax;
  Cx<T>* b1 = b0 + c.nfmax;
  const T gm1 = T(c.gamma - 1.0);
  const long long total = (long long)c.instances * ntiles;
  for (long long wk = blockIdx.x; wk < total; wk += gridDim.x) {
    const int inst = (int)(wk / ntiles);
    const int2 tl = tiles[wk % ntiles];
    const PatchDev P = c.patches[tl.x];
    const PlanDev pl = c.plans[P.plan[1]];
    const int N = P.n2, c0 = tl.y;
    const int width = min(tw, P.n1 - c0);
    const long long np = (long long)P.n1 * P.n2;
    const long long sbase = inst * c.sstride + P.soff + c0;
    const long long qbase = P.qoff + c0;
    const bool visc = (mu != nullptr) && P.cart;
    for (int k = threadIdx.x; k < 4 * N * tw; k += blockDim.x) {
      const int cc = k % tw, j = (k / tw) % N, f = k / (tw * N);
      if (cc < width) E[(f * n2m + j) * ld + cc] = e[sbase + f * np + (long long)j * P.n1 + cc];
    }
    if (visc)
      for (int k = threadIdx.x; k < N * tw; k += blockDim.x) {
        const int cc = k % tw, j = k / tw;
        if (cc < width) M[j * ld + cc] = mu[inst * c.qstride + qbase + (long long)j * P.n1 + cc];
      }
    __syncthreads();
    const T h = T(P.hy);
    // phase 0 (viscous): D = d e/dy; phase 1: E = d F2/dq2 with F2 formed in D
    for (int phase = visc ? 0 : 1; phase < 2; ++phase) {
      if (phase == 1) {
        for (int k = threadIdx.x; k < N * tw; k += blockDim.x) {
          const int cc = k % tw, j = k / tw;
          if (cc >= width) continue;
          T v[4], dv[4], F[4];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            v[f] = E[(f * n2m + j) * ld + cc];
            dv[f] = visc ? D[(f * n2m + j) * ld + cc] : T(0);
          }
          point_flux<T, 1>(c, P, qbase + (long long)j * P.n1 + cc, v, dv, visc ? M[j * ld + cc] : T(0), visc, F);
#pragma unroll
          for (int f = 0; f < 4; ++f) D[(f * n2m + j) * ld + cc] = F[f];
        }
        __syncthreads();
      }
      const T* src = phase == 0 ? E : D;
      T* dst = phase == 0 ? D : E;
      for (int u = warp; u < 2 * width; u += kYWarps) {
        const int cc = u >> 1, pr = u & 1;
        line_deriv_pair<T, N1>(src + (2 * pr) * n2m * ld + cc, ld, src + (2 * pr + 1) * n2m * ld + cc, ld,
                           dst + (2 * pr) * n2m * ld + cc, ld, dst + (2 * pr + 1) * n2m * ld + cc, ld, T(1), c, pl, h,
                           1, lane, b0, b1);
      }
      __syncthreads();
    }
    const T dtv = st.dt_dev ? T(st.dt_dev[inst]) : st.dt;
    for (int k = threadIdx.x; k < N * tw; k += blockDim.x) {
      const int cc = k % tw, j = k / tw;
      if (cc >= width) continue;
      const long long off = sbase + (long long)j * P.n1 + cc;
      const long long q = qbase + (long long)j * P.n1 + cc;
      const T invJ = P.cart ? T(1) : T(1) / metrics<T>(c)[4 * c.qstride + q];
      T kv[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) kv[f] = (R[off + f * np] - E[(f * n2m + j) * ld + cc]) * invJ;
      if (MODE == MODE_RHS) {
#pragma unroll
        for (int f = 0; f < 4; ++f) st.out[off + f * np] = kv[f];
        continue;
      }
      T v[4];
      const int s = st.stage;
      if (s == 0) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const T en = st.e_n[off + f * np];
          st.acc[off + f * np] = en + (dtv / T(6)) * kv[f];
          v[f] = en + (dtv / T(2)) * kv[f];
        }
      } else if (s < 3) {
        const T a = s == 1 ? dtv / T(2) : dtv;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          st.acc[off + f * np] = st.acc[off + f * np] + (dtv / T(3)) * kv[f];
          v[f] = st.e_n[off + f * np] + a * kv[f];
        }
      } else {
#pragma unroll
        for (int f = 0; f < 4; ++f) v[f] = st.acc[off + f * np] + (dtv / T(6)) * kv[f];
      }
      apply_bc<T>(c, P, c0 + cc, j, q, v);
      const T pr_ = pressure<T>(v[0], v[1], v[2], v[3], gm1);
      int flag = 0;
      if (!(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]))) flag |= 1;
      else if (!(v[0] > T(0)) || !(pr_ > T(0))) flag |= 2;
      if (flag) atomicOr(c.status, flag);
#pragma unroll
      for (int f = 0; f < 4; ++f) st.out[off + f * np] = v[f];
    }
    __syncthreads();
  }
}

}  // namespace fcs
