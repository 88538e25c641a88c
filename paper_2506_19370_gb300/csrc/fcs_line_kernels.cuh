// Line kernels of the FC-SDNN stage library: FC derivative of line pairs and
// the two flux passes of the Euler operator (with the Runge-Kutta epilogue).
// Included only by the fcs_lines_*.cu translation units.
#pragma once

#include "fcs_device.cuh"
#include "fcs_launch.cuh"

namespace fcs {

// Asynchronous copy of one element global -> shared (cp.async): a thread
// issues all its staging copies before waiting once, so their latencies
// overlap without holding registers.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ============================================================ FC derivative
// FC derivative (with respect to the patch parameter, spacing 1/(n1 - 1) or
// 1/(n2 - 1) also on the short lines of an L-shaped patch) of a scalar field:
// each warp takes jobs_per_round(N1) line pairs at a time (two real lines ->
// one complex FFT).  A pair (patch, line a,
// line b, w) reads the scalar layout if w < 0, else field w of the state layout.
// mu (scalar layout, may be null): transform only the pairs with mu != 0
// somewhere on their lines (the viscous gradients, which only ever meet mu).
template <typename T, int N1>
__global__ void __launch_bounds__(kWarps * 32) k_fc_deriv(CtxDev c, int dir, int order, const int4* __restrict__ pairs,
                                                           int npairs, const T* __restrict__ in, T* __restrict__ out,
                                                           const T* __restrict__ mu) {
  constexpr int JPR = jobs_per_round(N1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nmax = c.gnmax[dir][N1], nfmax = c.gnfmax[dir][N1];
  unsigned char* base = smem_raw + (size_t)warp * deriv_warp_bytes<T>(nmax, nfmax, N1);
  T* L = reinterpret_cast<T*>(base);  // [JPR][2][nmax]
  Cx<T>* aux = reinterpret_cast<Cx<T>*>(base + align16((size_t)8 * nmax * sizeof(T)));
  const int g = JPR == 4 ? (lane >> 3) : 0;
  Cx<T>* tile = aux + (size_t)g * 8 * (4 * N1 + 1);
  const long long total = (long long)c.instances * npairs;
  const long long rounds = (total + JPR - 1) / JPR;
  for (long long r = (long long)blockIdx.x * kWarps + warp; r < rounds; r += (long long)gridDim.x * kWarps) {
    unsigned vis = 0xffffffffu;   // bit k: pair k of the round is transformed
    if (mu) {
      vis = 0u;
      for (int k = 0; k < JPR; ++k) {
        const long long w = r * JPR + k;
        if (w >= total) break;
        const int inst = (int)(w / npairs);
        const int4 pr = pairs[w % npairs];
        const PatchDev& P = c.patches[pr.x];
        const int N = c.plans[line_plan(P, dir, pr.y)].N;
        const long long stride = dir == 0 ? 1 : P.n1;
        const long long s0 = (long long)line_start(P, dir, pr.y) * stride;
        const long long la = (dir == 0 ? (long long)pr.y * P.n1 : pr.y) + s0;
        const long long lb = pr.z < 0 ? -1 : (dir == 0 ? (long long)pr.z * P.n1 : pr.z) + s0;
        const T* m = mu + inst * c.qstride + P.qoff;
        bool any = false;
        for (int t = lane; t < N; t += 32) any |= m[la + t * stride] != T(0) || (lb >= 0 && m[lb + t * stride] != T(0));
        if (__any_sync(0xffffffffu, any)) vis |= 1u << k;
      }
    }
    // stage the JPR line pairs of this round (asynchronous copies: all of a
    // lane's loads are in flight together)
    for (int k = 0; k < JPR; ++k) {
      const long long w = r * JPR + k;
      if (w >= total) break;
      if (!(vis >> k & 1u)) continue;
      const int inst = (int)(w / npairs);
      const int4 pr = pairs[w % npairs];
      const PatchDev& P = c.patches[pr.x];
      const int N = c.plans[line_plan(P, dir, pr.y)].N;
      const long long stride = dir == 0 ? 1 : P.n1;
      const long long s0 = (long long)line_start(P, dir, pr.y) * stride;   // both lines of a pair share it
      const long long la = (dir == 0 ? (long long)pr.y * P.n1 : pr.y) + s0;
      const long long lb = pr.z < 0 ? -1 : (dir == 0 ? (long long)pr.z * P.n1 : pr.z) + s0;
      const T* src = in + (pr.w < 0 ? inst * c.qstride + P.qoff
                                    : inst * c.sstride + P.soff + (long long)pr.w * P.n1 * P.n2);
      for (int t = lane; t < N; t += 32) {
        cp_async_elem(&L[(2 * k) * nmax + t], src + la + t * stride);
        if (lb >= 0) cp_async_elem(&L[(2 * k + 1) * nmax + t], src + lb + t * stride);
      }
    }
    cp_async_wait_all();
    __syncwarp();
    const long long w = r * JPR + g;
    const bool active = w < total && (vis >> g & 1u);
    const long long wc = w < total ? w : r * JPR;
    const int inst = (int)(wc / npairs);
    const int4 pr = pairs[wc % npairs];
    const PatchDev& P = c.patches[pr.x];
    const PlanDev& pl = c.plans[line_plan(P, dir, pr.y)];
    const long long stride = dir == 0 ? 1 : P.n1;
    const long long s0 = (long long)line_start(P, dir, pr.y) * stride;
    const long long la = (dir == 0 ? (long long)pr.y * P.n1 : pr.y) + s0;
    const long long lb = pr.z < 0 ? -1 : (dir == 0 ? (long long)pr.z * P.n1 : pr.z) + s0;
    T* dst = out + (pr.w < 0 ? inst * c.qstride + P.qoff
                             : inst * c.sstride + P.soff + (long long)pr.w * P.n1 * P.n2);
    const T hq = T(1) / T((dir == 0 ? P.n1 : P.n2) - 1);
    line_deriv_pair<T, N1>(L + (2 * g) * nmax, 1, lb >= 0 ? L + (2 * g + 1) * nmax : nullptr, 1, dst + la, (int)stride,
                           lb >= 0 ? dst + lb : nullptr, (int)stride, T(1), c, pl, hq, order, lane, aux, aux + nfmax,
                           tile, active);
    __syncwarp();
  }
}

// FC derivative along q2 (spacing 1/(n2 - 1)) on tiles of tw adjacent
// columns of one patch, the layout of the pass along q2: the tile's row
// segments are staged in shared memory with coalesced copies, transformed in
// place, and written back as row segments.  nf = 1: one scalar-layout field,
// adjacent columns share a transform; nf = 4: the four fields of the state
// layout, field pairs (0, 1) and (2, 3) of a column share one.  order as in
// k_fc_deriv (0: the filter factors).
template <typename T, int N1>
__global__ void __launch_bounds__(kYWarps * 32, ypass_min_blocks(sizeof(T), N1))
    k_fc_cols(CtxDev c, int order, const int2* __restrict__ tiles, int ntiles, int nf, const T* __restrict__ in,
              T* __restrict__ out) {
  constexpr int JPR = jobs_per_round(N1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tw = c.tw, ld = c.tw + 1, n2m = c.gnmax[1][N1], nfmax = c.gnfmax[1][N1];
  T* E = reinterpret_cast<T*>(smem_raw);   // [nf][n2m][ld], then the warps' FFT buffers
  Cx<T>* aux = reinterpret_cast<Cx<T>*>(smem_raw + align16((size_t)nf * n2m * ld * sizeof(T))) +
               (size_t)warp * aux_cx(N1, nfmax);
  const int g = JPR == 4 ? (lane >> 3) : 0;
  Cx<T>* tile = aux + (size_t)g * 8 * (4 * N1 + 1);
  const long long total = (long long)c.instances * ntiles;
  for (long long wk = blockIdx.x; wk < total; wk += gridDim.x) {
    const int inst = (int)(wk / ntiles);
    const int2 tl = tiles[wk % ntiles];
    const PatchDev P = c.patches[tl.x];
    const int c0 = tl.y;
    const int j0 = line_start(P, 1, c0), N = P.n2 - j0;
    const PlanDev pl = c.plans[line_plan(P, 1, c0)];
    const int width = min(tw, (c0 < P.m1 ? P.m1 : P.n1) - c0);
    const long long fs = nf == 1 ? 0 : (long long)P.n1 * P.n2;
    const long long base = (nf == 1 ? inst * c.qstride + P.qoff : inst * c.sstride + P.soff) +
                           (long long)j0 * P.n1 + c0;
    const int cnt = nf * N * width;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {   // columns fastest: coalesced row segments
      const int cc = k % width, r = k / width, j = r % N, f = r / N;
      cp_async_elem(&E[(f * n2m + j) * ld + cc], in + base + f * fs + (long long)j * P.n1 + cc);
    }
    cp_async_wait_all();
    __syncthreads();
    const int njobs = nf == 1 ? (width + 1) / 2 : 2 * width;
    const T h = T(1) / T(P.n2 - 1);
    if constexpr (quad_path<T, N1>()) {   // a warp per column (4 fields) or per 4 adjacent columns
      const int nq = nf == 1 ? (width + 3) / 4 : width;
#pragma unroll 1
      for (int u = warp; u < nq; u += kYWarps) {
        T* l[4];
#pragma unroll
        for (int f = 0; f < 4; ++f)
          l[f] = nf == 1 ? (4 * u + f < width ? E + 4 * u + f : nullptr) : E + f * n2m * ld + u;
        line_deriv_quad<T, N1>(l[0], ld, l[1], ld, l[2], ld, l[3], ld, l[0], ld, l[1], ld, l[2], ld, l[3], ld, T(1), c,
                               pl, h, order, lane, true);
      }
    } else
#pragma unroll 1
    for (int u0 = warp * JPR; u0 < njobs; u0 += kYWarps * JPR) {
      const int u = u0 + g;
      const bool active = u < njobs;
      T* sa;
      T* sb;
      if (nf == 1) {
        const int cc = active ? 2 * u : 0;
        sa = E + cc;
        sb = cc + 1 < width ? E + cc + 1 : nullptr;
      } else {
        const int cc = active ? (u >> 1) : 0, pr = u & 1;
        sa = E + (2 * pr) * n2m * ld + cc;
        sb = sa + n2m * ld;
      }
      // a pair's values are all read before any is written: in place
      line_deriv_pair<T, N1>(sa, ld, sb, ld, sa, ld, sb, ld, T(1), c, pl, h, order, lane, aux, aux + nfmax, tile,
                             active);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      const int cc = k % width, r = k / width, j = r % N, f = r / N;
      out[base + f * fs + (long long)j * P.n1 + cc] = E[(f * n2m + j) * ld + cc];
    }
    __syncthreads();
  }
}

// Flux of Eq. (1) along direction DIR at one point, transformed for the
// parameter direction: DIR 0: y_q2 f - x_q2 g, DIR 1: -y_q1 f + x_q1 g;
// Cartesian: f resp. g.  With viscosity the physical fluxes become f - mu e_x,
// g - mu e_y: dv is the derivative of e along this direction's parameter and
// dvo (curvilinear only) along the other one; e_x, e_y follow by the chain
// rule.  t is the point's index along its line segment of N points, code_lo
// the boundary code at the segment's start (a wall for the short lines of an
// L-shaped patch): the normal viscous flux is zero on wall, outflow and free
// sides (the diffusion term needs a condition on every variable there; this
// one is impermeable and adiabatic).
template <typename T, int DIR>
__device__ __forceinline__ void point_flux(const CtxDev& c, const PatchDev& P, long long q, const T* v, const T* dv,
                                           const T* dvo, T mu, bool visc, T* F, int t, int N, int code_lo) {
  // fields whose viscous flux this point keeps: none on the closed end points
  // (wall, outflow, free), momentum only on a no-slip wall
  int vmask = 15;
  if (visc) {
    const int code = t == 0 ? code_lo : (t == N - 1 ? P.bc[2 * DIR + 1] : 0);
    if (code == 1 || code == 3 || code == 4) visc = false;
    if (code == 5) vmask = 6;
  }
  const T gm1 = gm1_of<T>(c);
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
      for (int f = 0; f < 4; ++f)
        if (vmask >> f & 1) F[f] -= mu * dv[f];
    }
  } else {
    const T* Mt = metrics<T>(c);
    const long long qs = c.qstride;
    const T x_q1 = Mt[q], x_q2 = Mt[qs + q], y_q1 = Mt[2 * qs + q], y_q2 = Mt[3 * qs + q];
    const T ca = DIR == 0 ? y_q2 : -y_q1;
    const T cb = DIR == 0 ? -x_q2 : x_q1;
    const T f0 = mx, f1 = mx * u + p, f2 = my * u, f3 = (En + p) * u;
    const T g0 = my, g1 = mx * w, g2 = my * w + p, g3 = (En + p) * w;
    F[0] = ca * f0 + cb * g0;
    F[1] = ca * f1 + cb * g1;
    F[2] = ca * f2 + cb * g2;
    F[3] = ca * f3 + cb * g3;
    if (visc) {
      const T invJ = T(1) / Mt[4 * qs + q];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const T d1 = DIR == 0 ? dv[f] : dvo[f], d2 = DIR == 0 ? dvo[f] : dv[f];
        const T ex = (y_q2 * d1 - y_q1 * d2) * invJ, ey = (-x_q2 * d1 + x_q1 * d2) * invJ;
        if (vmask >> f & 1) F[f] -= mu * (ca * ex + cb * ey);
      }
    }
  }
}

// Chain-rule form of the operator (Algorithm 5): with w = (rho, m, n, theta),
// m = rho u, n = rho v, theta = p / rho, the flux divergence is
// f_x + g_y = A(w) w_x + B(w) w_y, A = df/dw, B = dg/dw.  The derivative of w
// along one parameter direction enters with the weight ca A + cb B (Cartesian
// rows: A, columns: B; curvilinear rows: y_q2 A - x_q2 B, columns:
// -y_q1 A + x_q1 B, the rest of the inverse Jacobian, 1/J, comes at the end).
// out_i = sum_k (ca A_ik + cb B_ik) dw_k at the state v (conserved).
template <typename T>
__device__ __forceinline__ void chain_contract(const T* v, const T* dw, T ca, T cb, T gm1, T gg, T* out) {
  const T rho = v[0], u = v[1] / rho, vv = v[2] / rho;
  const T th = pressure<T>(v[0], v[1], v[2], v[3], gm1) / rho;
  const T q2 = u * u + vv * vv, uv = u * vv;
  out[0] = ca * dw[1] + cb * dw[2];
  out[1] = ca * ((th - u * u) * dw[0] + T(2) * u * dw[1] + rho * dw[3]) + cb * (-uv * dw[0] + vv * dw[1] + u * dw[2]);
  out[2] = ca * (-uv * dw[0] + vv * dw[1] + u * dw[2]) + cb * ((th - vv * vv) * dw[0] + T(2) * vv * dw[2] + rho * dw[3]);
  out[3] = ca * (-u * q2 * dw[0] + (gg * th + T(0.5) * (T(3) * u * u + vv * vv)) * dw[1] + uv * dw[2] + gg * rho * u * dw[3]) +
           cb * (-vv * q2 * dw[0] + uv * dw[1] + (gg * th + T(0.5) * (u * u + T(3) * vv * vv)) * dw[2] +
                 gg * rho * vv * dw[3]);
}

// Pass along q2, the first of the operator: a tile of tw adjacent columns of
// one patch (coalesced row segments staged in shared memory; blocks of 8
// warps, ypass_min_blocks of them per SM) writes the partial operator
// R = -d/dq2 F2 that the pass along q1 completes.
// The tile stages 5 values per point (state, then flux in its place, and mu).
// Viscous columns (mu != 0 somewhere on them) first take e_q2 into G2 (phase
// 0), which the pass along q1 reads on curvilinear patches; curvilinear
// viscous columns also read e_q1 from G1 (the row transform of those patches
// before this pass).
// CH = 1: chain-rule form (inviscid): w is staged and differentiated in
// place, and R = -(ca A + cb B) w_q2.
template <typename T, int CH, int N1>
__global__ void __launch_bounds__(kYWarps * 32, ypass_min_blocks(sizeof(T), N1))
    k_ypass(CtxDev c, const int2* __restrict__ tiles, int ntiles, const T* __restrict__ e, const T* __restrict__ mu,
            T* __restrict__ R, const T* __restrict__ G1, T* __restrict__ G2) {
  constexpr int JPR = jobs_per_round(N1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tw = c.tw, ld = c.tw + 1, n2m = c.gnmax[1][N1], nfmax = c.gnfmax[1][N1];
  T* E = reinterpret_cast<T*>(smem_raw);           // [4][n2m][ld]: state, flux, d flux/dq2
  T* M = E + 4 * n2m * ld;                         // [n2m][ld]
  Cx<T>* aux = reinterpret_cast<Cx<T>*>(smem_raw + align16((size_t)5 * n2m * ld * sizeof(T))) +
               (size_t)warp * aux_cx(N1, nfmax);
  const int g = JPR == 4 ? (lane >> 3) : 0;
  Cx<T>* tile = aux + (size_t)g * 8 * (4 * N1 + 1);
  const T gm1 = gm1_of<T>(c);
  const long long total = (long long)c.instances * ntiles;
  for (long long wk = blockIdx.x; wk < total; wk += gridDim.x) {
    const int inst = (int)(wk / ntiles);
    const int2 tl = tiles[wk % ntiles];
    const PatchDev P = c.patches[tl.x];
    const int c0 = tl.y;
    // all columns of a tile share their segment (tiles never straddle i = m1)
    const int j0 = line_start(P, 1, c0), N = P.n2 - j0;
    const PlanDev pl = c.plans[line_plan(P, 1, c0)];
    const int code_lo = j0 ? 1 : P.bc[2];
    const int width = min(tw, (c0 < P.m1 ? P.m1 : P.n1) - c0);
    const long long np = (long long)P.n1 * P.n2;
    const long long sbase = inst * c.sstride + P.soff + (long long)j0 * P.n1 + c0;   // row j0 of the tile
    const long long qbase = P.qoff + (long long)j0 * P.n1 + c0;
    const bool visc = mu != nullptr;
    // each thread keeps one column cc of the tile and strides over rows
    const int cc = threadIdx.x % tw, jr = threadIdx.x / tw, js = blockDim.x / tw;
    const bool colok = cc < width && jr < js;
    __shared__ int colv[32];   // column has mu != 0 somewhere (tw <= 32)
    __shared__ int act[32];    // compacted list of such columns
    __shared__ int nact;
    if (threadIdx.x < 32) colv[threadIdx.x] = 0;
    __syncthreads();
    if (colok)
      for (int j = jr; j < N; j += js) {
#pragma unroll
        for (int f = 0; f < 4; ++f)
          cp_async_elem(&E[(f * n2m + j) * ld + cc], e + sbase + f * np + (long long)j * P.n1 + cc);
        if (visc) cp_async_elem(&M[j * ld + cc], mu + inst * c.qstride + qbase + (long long)j * P.n1 + cc);
      }
    cp_async_wait_all();
    if (colok) {   // the thread's own staged points
      bool any_mu = false;
      for (int j = jr; j < N; j += js) {
        if (CH) {
          const T* v = E + j * ld + cc;
          const int fs = n2m * ld;
          E[(3 * n2m + j) * ld + cc] = pressure<T>(v[0], v[fs], v[2 * fs], v[3 * fs], gm1) / v[0];
        }
        if (visc) any_mu |= M[j * ld + cc] != T(0);
      }
      if (any_mu) atomicOr(&colv[cc], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {   // warp 0 compacts the viscous columns
      const bool v = threadIdx.x < width && colv[threadIdx.x];
      const unsigned bal = __ballot_sync(0xffffffffu, v);
      if (v) act[__popc(bal & ((1u << threadIdx.x) - 1u))] = threadIdx.x;
      if (threadIdx.x == 0) nact = __popc(bal);
    }
    __syncthreads();
    const T h = T(P.hy);
    // phase 0 (viscous columns only): G2 = d e/dq2; phase 1: F2 formed in
    // place of the state, then -d F2/dq2 (chain-rule form: +d w/dq2) in place
    for (int phase = (visc && nact > 0) ? 0 : 1; phase < 2; ++phase) {
      if (phase == 1 && !CH) {
        for (int j = jr; colok && j < N; j += js) {
          T v[4], dv[4], dvo[4], F[4];
          const bool vc = visc && colv[cc];
          const bool curv = vc && !P.cart;
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            v[f] = E[(f * n2m + j) * ld + cc];
            dv[f] = vc ? G2[sbase + f * np + (long long)j * P.n1 + cc] : T(0);
            dvo[f] = curv ? G1[sbase + f * np + (long long)j * P.n1 + cc] : T(0);
          }
          point_flux<T, 1>(c, P, qbase + (long long)j * P.n1 + cc, v, dv, dvo, vc ? M[j * ld + cc] : T(0), vc, F, j, N,
                           code_lo);
#pragma unroll
          for (int f = 0; f < 4; ++f) E[(f * n2m + j) * ld + cc] = F[f];
        }
        __syncthreads();
      }
      // jobs (column, field pair): phase 0 over the viscous columns only (a
      // line pair's values are all read before any is written, so phase 1
      // differentiates in place)
      const int ncol = phase == 0 ? nact : width;
      if constexpr (quad_path<T, N1>()) {   // a warp per column: its four fields at once
#pragma unroll 1
        for (int u = warp; u < ncol; u += kYWarps) {
          const int cc = phase == 0 ? act[u] : u;
          T* src = E + cc;
          const long long fo = (long long)n2m * ld;
          // one call for both phases (one inlined copy of the transform)
          T* o = phase == 0 ? G2 + sbase + cc : src;
          const long long of = phase == 0 ? np : fo;
          const int so = phase == 0 ? P.n1 : ld;
          line_deriv_quad<T, N1>(src, ld, src + fo, ld, src + 2 * fo, ld, src + 3 * fo, ld, o, so, o + of, so,
                                 o + 2 * of, so, o + 3 * of, so, (phase == 0 || CH) ? T(1) : T(-1), c, pl, h, 1,
                                 lane, true);
        }
      } else
#pragma unroll 1
      for (int u0 = warp * JPR; u0 < 2 * ncol; u0 += kYWarps * JPR) {
        const int u = u0 + g;
        const bool active = u < 2 * ncol;
        const int cc = active ? (phase == 0 ? act[u >> 1] : (u >> 1)) : 0, pr = u & 1;
        T* src = E + (2 * pr) * n2m * ld + cc;
        T* oa = phase == 0 ? G2 + sbase + (2 * pr) * np + cc : src;
        const int so = phase == 0 ? P.n1 : ld;
        const long long fo = phase == 0 ? np : (long long)n2m * ld;
        line_deriv_pair<T, N1>(src, ld, src + n2m * ld, ld, oa, so, oa + fo, so, (phase == 0 || CH) ? T(1) : T(-1), c,
                               pl, h, 1, lane, aux, aux + nfmax, tile, active);
      }
      __syncthreads();
    }
    for (int j = jr; colok && j < N; j += js) {
      const long long off = sbase + (long long)j * P.n1 + cc;
      if (CH) {   // -(ca A + cb B) w_q2 at the stage's input state
        const long long q = qbase + (long long)j * P.n1 + cc;
        T v[4], dw[4], out[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          v[f] = e[off + f * np];
          dw[f] = E[(f * n2m + j) * ld + cc];
        }
        const T* Mt = metrics<T>(c);
        const T ca = P.cart ? T(0) : -Mt[2 * c.qstride + q];
        const T cb = P.cart ? T(1) : Mt[q];
        chain_contract<T>(v, dw, ca, cb, gm1, T(c.gamma) / gm1, out);
#pragma unroll
        for (int f = 0; f < 4; ++f) R[off + f * np] = -out[f];
      } else {
#pragma unroll
        for (int f = 0; f < 4; ++f) R[off + f * np] = E[(f * n2m + j) * ld + cc];
      }
    }
    __syncthreads();
  }
}

// Stage update of one point from its operator value kv = L(e_s): MODE_RHS
// stores kv; MODE_RK takes stage st.stage of the classical 4-stage
// Runge-Kutta scheme (acc collects e_n + dt/6 (k1 + 2 k2 + 2 k3) on the way,
// out = the next stage's input, or e_{n+1} after the fourth), then the
// boundary conditions and the state check (non-finite: status bit 1,
// density or pressure not positive: bit 2).  en, ac: the point's e_n (stages
// 0-2) and acc (stages 1-3), loaded by the caller; (i, j) is the point, q
// its scalar-layout offset, off its state-layout offset, np the field stride.
template <typename T, int MODE>
__device__ __forceinline__ void stage_point(const CtxDev& c, const PatchDev& P, const StageArgs<T>& st, T dtv,
                                            long long off, long long np, long long q, int i, int j, const T* kv,
                                            const T* en, const T* ac) {
  if ((MODE & 3) == MODE_RHS) {
#pragma unroll
    for (int f = 0; f < 4; ++f) st.out[off + f * np] = kv[f];
    return;
  }
  T v[4];
  const int s = st.stage;
  if (s == 0) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      st.acc[off + f * np] = en[f] + (dtv / T(6)) * kv[f];
      v[f] = en[f] + (dtv / T(2)) * kv[f];
    }
  } else if (s < 3) {
    const T a = s == 1 ? dtv / T(2) : dtv;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      st.acc[off + f * np] = ac[f] + (dtv / T(3)) * kv[f];
      v[f] = en[f] + a * kv[f];
    }
  } else {
#pragma unroll
    for (int f = 0; f < 4; ++f) v[f] = ac[f] + (dtv / T(6)) * kv[f];
  }
  apply_bc<T>(c, P, i, j, q, v);
  const T pr = pressure<T>(v[0], v[1], v[2], v[3], gm1_of<T>(c));
  int flag = 0;
  if (!(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]))) flag |= 1;
  else if (!(v[0] > T(0)) || !(pr > T(0))) flag |= 2;
  if (flag) atomicOr(c.status, flag);
#pragma unroll
  for (int f = 0; f < 4; ++f) st.out[off + f * np] = v[f];
}

// Pass along q1, the second of the operator (rows lbeg .. lbeg + lcnt - 1 of
// the row list, one FFT-size group), with the stage epilogue: a warp takes
// kRowsPerWarp rows, staged in shared memory (5 values per point, so four
// blocks of 4 warps fit an SM), forms d/dq1 F1 in place and completes
// L = (R - d/dq1 F1)/J with the partial operator R = -d/dq2 F2 of the pass
// along q2, then stores L (MODE_RHS) or takes the Runge-Kutta stage
// (MODE_RK): each warp updates its own rows with coalesced loads and stores.
// Jobs of a phase: (row, field pair); phase 0 (viscous rows of Cartesian
// patches) G1 = d e/dq1 in global memory (curvilinear patches have it from
// their row transform before the pass along q2); phase 1 the flux in place of
// the staged state, then its derivative in place.  Curvilinear viscous rows
// read e_q2 from G2 (the pass along q2).
// MODE_CHAIN (or-ed into MODE): chain-rule form (inviscid): w is staged and
// differentiated in place, and the epilogue forms (ca A + cb B) w_q1.
template <typename T, int MODE, int N1>
__global__ void __launch_bounds__(kWarps * 32, xpass_min_blocks(sizeof(T), N1))
    k_xpass(CtxDev c, int lbeg, int lcnt, const T* __restrict__ e, const T* __restrict__ mu, const T* __restrict__ R,
            T* __restrict__ G1, const T* __restrict__ G2, StageArgs<T> st) {
  constexpr bool CH = (MODE & MODE_CHAIN) != 0;
  constexpr int JPR = jobs_per_round(N1);
  constexpr int RW = kRowsPerWarp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nmax = c.gnmax[0][N1], nfmax = c.gnfmax[0][N1];
  unsigned char* base = smem_raw + (size_t)warp * xpass_warp_bytes<T>(nmax, nfmax, N1);
  T* E = reinterpret_cast<T*>(base);   // [RW][4][nmax]: state, then flux, then its derivative
  T* M = E + RW * 4 * nmax;            // [RW][nmax]
  Cx<T>* aux = reinterpret_cast<Cx<T>*>(base + align16((size_t)RW * 5 * nmax * sizeof(T)));
  const int g = JPR == 4 ? (lane >> 3) : 0;
  Cx<T>* tile = aux + (size_t)g * 8 * (4 * N1 + 1);
  const T gm1 = gm1_of<T>(c);
  // the epilogue's operands: R always; e_n in stages 0-2, acc in stages 1-3
  constexpr bool rk = (MODE & 3) == MODE_RK;
  const unsigned arrs = 1u | (rk && st.stage < 3 ? 2u : 0u) | (rk && st.stage > 0 ? 4u : 0u);
  const long long groups = ((long long)lcnt + RW - 1) / RW;   // row groups per instance
  const long long total = (long long)c.instances * groups;
  for (long long w = (long long)blockIdx.x * kWarps + warp; w < total; w += (long long)gridDim.x * kWarps) {
    const int inst = (int)(w / groups);
    const int l0 = lbeg + (int)(w % groups) * RW;
    int pid[RW], row[RW], nk[RW];
    bool has[RW], vrow[RW], cart[RW];
#pragma unroll
    for (int k = 0; k < RW; ++k) {
      has[k] = l0 + k < lbeg + lcnt;
      const LineRef lr = c.lines0[has[k] ? l0 + k : l0];
      pid[k] = lr.patch;
      row[k] = lr.line;
      const PatchDev& P = c.patches[lr.patch];
      cart[k] = P.cart;
      const long long np = (long long)P.n1 * P.n2;
      const int s0 = line_start(P, 0, lr.line), N = P.n1 - s0;
      const long long so = inst * c.sstride + P.soff + (long long)lr.line * P.n1 + s0;
      const T* es = e + so;
      const T* ms = mu ? mu + inst * c.qstride + P.qoff + (long long)lr.line * P.n1 + s0 : nullptr;
      nk[k] = has[k] ? N : 0;
      for (int t = lane; t < nk[k]; t += 32) {
#pragma unroll
        for (int f = 0; f < 4; ++f) cp_async_elem(&E[(k * 4 + f) * nmax + t], es + f * np + t);
        if (ms) cp_async_elem(&M[k * nmax + t], ms + t);
      }
      // start moving the row's segments of the epilogue's operands into L2
      // while the row is transformed (one prefetch per 128-byte line)
      const int nl = nk[k] ? (nk[k] * (int)sizeof(T) + 127) / 128 + 1 : 0;
      for (int u = lane; u < 12 * nl; u += 32) {
        const int a = u / (4 * nl), f = (u / nl) & 3, sg = u % nl;
        if (!(arrs >> a & 1)) continue;
        const T* b = a == 0 ? R : (a == 1 ? st.e_n : st.acc);
        const T* p = b + so + f * np + min(sg * (int)(128 / sizeof(T)), nk[k] - 1);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
      }
    }
    cp_async_wait_all();
#pragma unroll
    for (int k = 0; k < RW; ++k) {   // the lane's own staged points
      bool any_mu = false;
      for (int t = lane; t < nk[k]; t += 32) {
        if (CH) {
          const T* v = E + k * 4 * nmax + t;
          E[(k * 4 + 3) * nmax + t] = pressure<T>(v[0], v[nmax], v[2 * nmax], v[3 * nmax], gm1) / v[0];
        }
        if (mu) any_mu |= M[k * nmax + t] != T(0);
      }
      // the viscous flux of a row with mu == 0 everywhere vanishes: skip its
      // derivatives (localized viscosity)
      vrow[k] = __any_sync(0xffffffffu, any_mu);
    }
    __syncwarp();
    const bool p0 = (vrow[0] && cart[0]) || (vrow[1] && cart[1]);
    for (int phase = p0 ? 0 : 1; phase < 2; ++phase) {
      if (phase == 1 && !CH) {
#pragma unroll 1
        for (int k = 0; k < RW; ++k) {   // rolled (one copy of the flux); row data by selects
          if (!(k ? has[1] : has[0])) continue;
          const int rowk = k ? row[1] : row[0];
          const PatchDev& P = c.patches[k ? pid[1] : pid[0]];
          const bool visc = k ? vrow[1] : vrow[0];
          const bool curv = visc && !P.cart;
          const int a0 = line_start(P, 0, rowk), N = P.n1 - a0;
          const int code_lo = a0 ? 1 : P.bc[0];
          const long long q0 = P.qoff + (long long)rowk * P.n1 + a0;
          const long long np = (long long)P.n1 * P.n2;
          const long long s0 = inst * c.sstride + P.soff + (long long)rowk * P.n1 + a0;
          for (int t = lane; t < N; t += 32) {
            T v[4], dv[4], dvo[4], F[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              v[f] = E[(k * 4 + f) * nmax + t];
              dv[f] = visc ? G1[s0 + f * np + t] : T(0);
              dvo[f] = curv ? G2[s0 + f * np + t] : T(0);
            }
            point_flux<T, 0>(c, P, q0 + t, v, dv, dvo, visc ? M[k * nmax + t] : T(0), visc, F, t, N, code_lo);
#pragma unroll
            for (int f = 0; f < 4; ++f) E[(k * 4 + f) * nmax + t] = F[f];
          }
        }
        __syncwarp();
      }
      // jobs: (row k, field pair pr), 2 RW of them (row data chosen by
      // selects, not by indexing, so the small per-row arrays stay in registers)
      static_assert(RW == 2, "row selection below assumes two rows per warp");
      if constexpr (quad_path<T, N1>()) {   // a row's four fields at once
#pragma unroll 1
        for (int kk = 0; kk < RW; ++kk) {
          const int pidk = kk ? pid[1] : pid[0], rowk = kk ? row[1] : row[0];
          bool active = kk ? has[1] : has[0];
          if (phase == 0 && !(kk ? (vrow[1] && cart[1]) : (vrow[0] && cart[0]))) active = false;
          const PatchDev& P = c.patches[pidk];
          const PlanDev& pl = c.plans[line_plan(P, 0, rowk)];
          const long long np = (long long)P.n1 * P.n2;
          T* src = E + kk * 4 * nmax;
          // one call for both phases (one inlined copy of the transform)
          T* o = phase == 0 ? G1 + inst * c.sstride + P.soff + (long long)rowk * P.n1 + line_start(P, 0, rowk) : src;
          const long long of = phase == 0 ? np : (long long)nmax;
          line_deriv_quad<T, N1>(src, 1, src + nmax, 1, src + 2 * nmax, 1, src + 3 * nmax, 1, o, 1, o + of, 1,
                                 o + 2 * of, 1, o + 3 * of, 1, T(1), c, pl, T(P.hx), 1, lane, active);
        }
      } else
#pragma unroll 1
      for (int r0 = 0; r0 < 2 * RW; r0 += JPR) {
        const int job = r0 + g;
        const int k = job >> 1, pr = job & 1;
        const int kk = k == 1 ? 1 : 0;
        const int pidk = kk ? pid[1] : pid[0], rowk = kk ? row[1] : row[0];
        bool active = job < 2 * RW && (kk ? has[1] : has[0]);
        const PatchDev& P = c.patches[pidk];
        const PlanDev& pl = c.plans[line_plan(P, 0, rowk)];
        if (phase == 0 && !(kk ? (vrow[1] && cart[1]) : (vrow[0] && cart[0]))) active = false;
        const long long np = (long long)P.n1 * P.n2;
        T* src = E + (kk * 4 + 2 * pr) * nmax;
        const long long orow = inst * c.sstride + P.soff + (long long)rowk * P.n1 + line_start(P, 0, rowk) +
                               (2 * pr) * np;
        // phase 1 in place (a pair's values are all read before any is written)
        T* oa = phase == 0 ? G1 + orow : src;
        const long long ob_off = phase == 0 ? np : (long long)nmax;
        line_deriv_pair<T, N1>(src, 1, src + nmax, 1, oa, 1, oa + ob_off, 1, T(1), c, pl, T(P.hx), 1, lane, aux,
                               aux + nfmax, tile, active);
      }
      __syncwarp();
    }
    // epilogue: L = (R - d/dq1 F1)/J (chain-rule form: (R - (ca A + cb B) w_q1)/J),
    // U points of a lane at a time, whose global loads are all issued before
    // the first of them is used
    constexpr int U = 2;   // measured faster than 4 points per batch (registers)
    const T dtv = st.dt_dev ? T(st.dt_dev[inst]) : st.dt;
    const T* Mt = metrics<T>(c);
    const bool ld_en = rk && st.stage < 3, ld_ac = rk && st.stage > 0;
#pragma unroll 1
    for (int k = 0; k < RW; ++k) {   // rolled (one copy of the update); row data by selects
      if (!(k ? has[1] : has[0])) continue;
      const int rowk = k ? row[1] : row[0];
      const PatchDev& P = c.patches[k ? pid[1] : pid[0]];
      const int a0 = line_start(P, 0, rowk), N = P.n1 - a0;
      const long long np = (long long)P.n1 * P.n2;
      const long long s0 = inst * c.sstride + P.soff + (long long)rowk * P.n1 + a0;
      const long long q0 = P.qoff + (long long)rowk * P.n1 + a0;
      for (int t0 = lane; t0 < N; t0 += 32 * U) {
        T r[U][4], en[U][4], ac[U][4], ev[U][4], ij[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int t = t0 + 32 * u;
          const long long off = s0 + t;
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            r[u][f] = t < N ? R[off + f * np] : T(0);
            en[u][f] = ld_en && t < N ? st.e_n[off + f * np] : T(0);
            ac[u][f] = ld_ac && t < N ? st.acc[off + f * np] : T(0);
            ev[u][f] = CH && t < N ? e[off + f * np] : T(0);
          }
          ij[u] = P.cart || t >= N ? T(1) : T(1) / Mt[4 * c.qstride + q0 + t];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int t = t0 + 32 * u;
          if (t >= N) continue;
          const long long off = s0 + t, q = q0 + t;
          T kv[4];
          if (CH) {
            T dw[4], out[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) dw[f] = E[(k * 4 + f) * nmax + t];
            const T ca = P.cart ? T(1) : Mt[3 * c.qstride + q];
            const T cb = P.cart ? T(0) : -Mt[c.qstride + q];
            chain_contract<T>(ev[u], dw, ca, cb, gm1, T(c.gamma) / gm1, out);
#pragma unroll
            for (int f = 0; f < 4; ++f) kv[f] = (r[u][f] - out[f]) * ij[u];
          } else {
#pragma unroll
            for (int f = 0; f < 4; ++f) kv[f] = (r[u][f] - E[(k * 4 + f) * nmax + t]) * ij[u];
          }
          stage_point<T, MODE>(c, P, st, dtv, off, np, q, a0 + t, rowk, kv, en[u], ac[u]);
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace fcs
