// C ABI of the FC-SDNN stage library: context setup and the entry points
// declared in include/fcsdnn.h.  Device code lives in fcs_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/fcsdnn.h"
#include "fcs_internal.h"
#include "fcs_kernels.cuh"
#include "fcs_launch.cuh"

using namespace fcs;

namespace {

constexpr int kNParams = 1732;
constexpr int kIndC = 26;   // continuation length of the indicator (16 + 26 = 42 = 2 * 3 * 7)
constexpr int kIndD = 5;
constexpr double kCflMu = 0.2;  // viscous limit: 1/dt = 1/dt_a + mu (1/s1^2 + 1/s2^2) / 0.2

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct HostPlan {
  PlanDev dev;
  std::vector<double> tab;     // C x d, FP64
  std::vector<double> tab_lo;  // remainder of the double-double table
};

// A contiguous range of a work list (rows, line pairs, column tiles) whose
// lines share one compile-time FFT size n1 (0: Stockham); one launch each.
struct Group {
  int n1, begin, count;
};

}  // namespace

struct fcs_ctx {
  // side streams of the pass launches: the FFT-size classes of one pass are
  // independent, so the smaller ones run next to the largest (forked from and
  // joined back into the caller's stream by events; captured graphs get
  // parallel branches)
  static constexpr int kSide = 3;
  cudaStream_t side[kSide] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kSide] = {};
  fcs_options opt{};
  int d = 0, C = 0, npatch = 0;
  size_t tsize = 4;  // sizeof(T)
  std::vector<PatchDev> patches;
  std::vector<HostPlan> plans;
  std::map<int, int> plan_of_len;  // line length -> plan index
  std::vector<int64_t> state_off, scalar_off, window_off;
  size_t sstride = 0, qstride = 0, nwin = 0;
  int nlines0 = 0, nlines1 = 0, npairs0 = 0, npairs1 = 0, nent = 0, ntiles = 0;
  int nmax = 0, nfmax = 0, n2max = 0, stockham = 0, tw = 32;
  // per direction and FFT-size class n1: longest line and longest FFT (the
  // line kernels size their shared-memory buffers by these)
  int gnmax[2][kN1Classes] = {}, gnfmax[2][kN1Classes] = {};
  std::vector<int> kind_n1[2][2];  // [dir][kind][patch]: FFT size of the full (kind 0) and short
                                   // (kind 1, L-shaped patches) lines along q1 / q2; -1: none
  std::vector<int> n1_dir[2];    // distinct FFT sizes per direction
  std::vector<Group> g_rows, g_pairs[2], g_tiles, g_vpairs;
  std::vector<int> tw_options;  // column-tile widths that fit in shared memory (widest first)
  CtxDev dev{};
  std::vector<void*> allocs;
  // device arrays
  int4* pairs0 = nullptr;
  int4* pairs1 = nullptr;
  int4* vpairs = nullptr;  // row pairs x fields of curvilinear patches (viscous gradient e_q1)
  int4* fpairs[2] = {nullptr, nullptr};  // row / column pairs x 4 fields of every patch (filter)
  std::vector<Group> g_fpairs[2];
  double* smr64 = nullptr;  // filter factors of the initial smearing (order smear_p), twiddle offsets
  float* smr32 = nullptr;
  void* G1 = nullptr;      // e_q1, e_q2 of the lines with viscosity (state-sized)
  void* G2 = nullptr;
  int2* tiles = nullptr;
  int2* pblk = nullptr;  // point blocks of the pointwise kernels
  int4* nsw = nullptr;   // no-slip wall points (patch, point, inward stride)
  int4* btiles = nullptr;  // 32 x 32 output tiles of the viscosity blend (patch, i0, j0)
  int nbtiles = 0;
  int4* fringe_ent[2] = {nullptr, nullptr};   // copies, resolved for the state [0] and scalar [1] layouts
  int4* interp_ent[2] = {nullptr, nullptr};   // interpolations (src: first node of the donor block), likewise
  double* interp_w64 = nullptr;   // 12 weights per interpolation (the two factors of the tensor stencil)
  float* interp_w32 = nullptr;
  int ninterp = 0;
  double* wq = nullptr;
  int2* woff = nullptr;
  double* bump = nullptr;
  void* R = nullptr;     // x-pass partial operator (state-sized)
  void* S = nullptr;     // stage buffer
  void* A = nullptr;     // Runge-Kutta accumulator
  void* av0 = nullptr;   // viscosity scratch (scalar-sized)
  void* av1 = nullptr;
  void* mu = nullptr;    // viscosity of the step
  signed char* tau = nullptr;
  signed char* tau_w = nullptr;
  unsigned long long* dtbest = nullptr;
  double* dt_internal = nullptr;
  float* Wm = nullptr;   // FP32 master weights
  float* Am = nullptr;   // Adam moments
  float* Av = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* Wb = nullptr;
  float* bias = nullptr;
  double* W64 = nullptr;
  float* acts = nullptr;
  float* loss_s = nullptr;
  double* gpart = nullptr;  // per batch-chunk partial gradients
  int adam_t = 0;
  bool sums_ok = true;  // every patch has a quadrature (L-shaped: m2 + 1 >= 2 d)
  // graph of fcs_step
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  void* g_e = nullptr;
  double g_dt = 0.0;
  double* g_dtdev = nullptr;
  int g_av = -1;
  cudaStream_t g_stream = nullptr;
};

namespace {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return FCS_OK;
  std::fprintf(stderr, "fcsdnn: CUDA error %s\n", cudaGetErrorString(e));
  return FCS_ECUDA;
}

#define FCS_CUDA(x)                        \
  do {                                     \
    int _rc = cuda_err((x));               \
    if (_rc != FCS_OK) return _rc;         \
  } while (0)

template <typename P>
int dalloc(fcs_ctx* c, P** out, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return FCS_ENOMEM;
  }
  cudaMemset(p, 0, bytes);
  c->allocs.push_back(p);
  *out = static_cast<P*>(p);
  return FCS_OK;
}

template <typename P>
int upload(fcs_ctx* c, P** out, const void* src, size_t bytes) {
  int rc = dalloc(c, out, bytes);
  if (rc) return rc;
  if (bytes) FCS_CUDA(cudaMemcpy(*out, src, bytes, cudaMemcpyHostToDevice));
  return FCS_OK;
}

bool factor_radices(int n, std::vector<int>* rad) {
  rad->clear();
  int m = n;
  while (m % 8 == 0) { rad->push_back(8); m /= 8; }
  while (m % 4 == 0) { rad->push_back(4); m /= 4; }
  while (m % 2 == 0) { rad->push_back(2); m /= 2; }
  for (int p : {3, 5, 7})
    while (m % p == 0) { rad->push_back(p); m /= p; }
  return m == 1 && (int)rad->size() <= kMaxStages;
}

bool smooth7(int n) {
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Continuation length of a line of N points.  Policy 0: C.  Policy 1: the
// smallest C' >= max(C - 4, 20) with N + C' = 32 n1, 2 <= n1 <= 9 (register
// FFT), else the smallest C' in [C, C + 16] with N + C' 7-smooth (Stockham).
int choose_c(const fcs_options& o, int C, int N) {
  if (o.c_policy == 0) return C;
  for (int c = std::max(C - 4, 20); c <= 64; ++c) {
    const int n = N + c;
    if (n % 32 == 0 && n / 32 >= 2 && n / 32 <= 9) return c;
  }
  for (int c = C; c <= C + 16; ++c)
    if (smooth7(N + c)) return c;
  return C;
}

// Host FP64 FC quadrature weights of a line of N points (integral over
// [0, 1] of the FC expansion), folded onto the data points.
std::vector<double> quad_weights(int N, int C, int d, const std::vector<double>& AR) {
  const int n = N + C;
  const double h = 1.0 / (N - 1), beta = n * h, PI = 3.14159265358979323846;
  std::vector<std::complex<double>> I(n);
  for (int k = 0; k < n; ++k) {
    const int kk = (2 * k <= n) ? k : k - n;
    if (kk == 0) I[k] = 1.0;
    else {
      const double th = 2 * PI * kk / beta;
      I[k] = (std::exp(std::complex<double>(0, th)) - 1.0) / std::complex<double>(0, th);
    }
  }
  if (n % 2 == 0) I[n / 2] = 0.0;
  std::vector<double> w(n);
  for (int j = 0; j < n; ++j) {
    std::complex<double> s = 0;
    for (int k = 0; k < n; ++k) s += std::exp(std::complex<double>(0, -2 * PI * (double)((long long)j * k % n) / n)) * I[k];
    w[j] = s.real() / n;
  }
  std::vector<double> W(w.begin(), w.begin() + N);
  for (int c = 0; c < C; ++c)
    for (int m = 0; m < d; ++m) {
      W[N - d + m] += AR[c * d + m] * w[N + c];           // right blend acts on the last d values
      W[m] += AR[(C - 1 - c) * d + (d - 1 - m)] * w[N + c];  // reflected left blend on the first d
    }
  return W;
}

int get_plan(fcs_ctx* c, int N, int C, int d) {
  const int key = N * 4096 + C * 16 + d;
  auto it = c->plan_of_len.find(key);
  if (it != c->plan_of_len.end()) return it->second;
  HostPlan hp{};
  hp.dev.N = N;
  hp.dev.C = C;
  hp.dev.n = N + C;
  std::vector<int> rad;
  const int n = N + C;
  const bool stk = factor_radices(n, &rad);
  hp.dev.n1reg = (n % 32 == 0 && n / 32 >= 2 && n / 32 <= 9) ? n / 32 : 0;
  if (!stk) {
    if (hp.dev.n1reg == 0) return FCS_EUNSUPPORTED;
    rad.clear();
  }
  hp.dev.nst = (int)rad.size();
  for (int s = 0; s < hp.dev.nst; ++s) hp.dev.radix[s] = rad[s];
  hp.tab.resize((size_t)C * d);
  hp.tab_lo.resize((size_t)C * d);
  if (build_table(d, C, hp.tab.data(), hp.tab_lo.data()) != 0) return FCS_EINVAL;
  c->plans.push_back(hp);
  const int idx = (int)c->plans.size() - 1;
  c->plan_of_len[key] = idx;
  return idx;
}

template <typename T>
size_t xpass_smem(const fcs_ctx* c, int n1) {
  return kWarps * xpass_warp_bytes<T>(c->gnmax[0][n1], c->gnfmax[0][n1], n1);
}
template <typename T>
size_t deriv_smem(const fcs_ctx* c, int n1) {
  return kWarps * std::max(deriv_warp_bytes<T>(c->gnmax[0][n1], c->gnfmax[0][n1], n1),
                           deriv_warp_bytes<T>(c->gnmax[1][n1], c->gnfmax[1][n1], n1));
}
template <typename T>
size_t ypass_smem(const fcs_ctx* c, int tw, int n1) {
  return ypass_bytes<T>(c->gnmax[1][n1], tw, c->gnfmax[1][n1], n1, kYWarps);
}
template <typename T>
size_t cols_smem(const fcs_ctx* c, int tw, int n1, int nf) {
  return cols_bytes<T>(c->gnmax[1][n1], tw, c->gnfmax[1][n1], n1, kYWarps) -
         align16((size_t)4 * c->gnmax[1][n1] * (tw + 1) * sizeof(T)) +
         align16((size_t)nf * c->gnmax[1][n1] * (tw + 1) * sizeof(T));
}
constexpr size_t kSmemMax = 227 * 1024;   // dynamic shared memory a block may use

size_t blend_smem(int r, size_t tsize) {
  const size_t w = kBlendTile + 4 * r;
  return 2 * w * w * tsize;
}

int grid_for(long long work, int per_block) {
  long long g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

// dispatch on the compile-time FFT size of a direction
#define FCS_N1_SWITCH(n1, CALL)            \
  switch (n1) {                            \
    case 0: { constexpr int K = 0; CALL; } \
    case 2: { constexpr int K = 2; CALL; } \
    case 3: { constexpr int K = 3; CALL; } \
    case 4: { constexpr int K = 4; CALL; } \
    case 5: { constexpr int K = 5; CALL; } \
    case 6: { constexpr int K = 6; CALL; } \
    case 7: { constexpr int K = 7; CALL; } \
    case 8: { constexpr int K = 8; CALL; } \
    case 9: { constexpr int K = 9; CALL; } \
    default: return FCS_EINVAL;            \
  }

template <typename T>
int set_smem_attrs(const fcs_ctx* c) {
  FCS_CUDA(cudaFuncSetAttribute(k_av_blend<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)blend_smem(kBlendMaxR, sizeof(T))));
  for (int n1 : c->n1_dir[0]) {
    FCS_N1_SWITCH(n1, FCS_CUDA((prep_xpass<T, K>(xpass_smem<T>(c, n1)))); break)
  }
  for (int n1 : c->n1_dir[1]) {
    FCS_N1_SWITCH(n1, FCS_CUDA((prep_ypass<T, K>(ypass_smem<T>(c, c->tw, n1)))); break)
  }
  for (int dir = 0; dir < 2; ++dir)
    for (int n1 : c->n1_dir[dir]) {
      FCS_N1_SWITCH(n1, FCS_CUDA((prep_fc_deriv<T, K>(deriv_smem<T>(c, n1)))); break)
    }
  const int twmax = c->tw_options.empty() ? c->tw : c->tw_options[0];
  for (int n1 : c->n1_dir[1]) {
    FCS_N1_SWITCH(n1, FCS_CUDA((prep_fc_cols<T, K>(cols_smem<T>(c, twmax, n1, 4)))); break)
  }
  return FCS_OK;
}

// Launch order of the FFT-size groups of a pass (dir 0: rows, 1: column
// tiles): ascending by points, so the largest group comes last, on the
// caller's stream, and the others on the side streams.
std::vector<int> pass_order(const fcs_ctx* c, int dir) {
  const std::vector<Group>& g = dir == 0 ? c->g_rows : c->g_tiles;
  std::vector<std::pair<long long, int>> w;
  for (size_t k = 0; k < g.size(); ++k)
    w.push_back({(long long)g[k].count * (dir == 0 ? 1 : c->tw) * c->gnmax[dir][g[k].n1], (int)k});
  std::sort(w.begin(), w.end());
  std::vector<int> o;
  for (const auto& x : w) o.push_back(x.second);
  return o;
}
// Stream of the k-th of n launches of a pass: the last (largest) on s, the
// others round-robin on the side streams.
cudaStream_t side_of(const fcs_ctx* c, cudaStream_t s, int k, int n) {
  return k == n - 1 ? s : c->side[k % fcs_ctx::kSide];
}
// Make the side streams (the first min(nside, kSide)) wait for the work
// issued so far on s, and s for everything issued on them.
cudaError_t fork_side(fcs_ctx* c, cudaStream_t s, int nside) {
  if (nside <= 0) return cudaSuccess;
  cudaError_t e = cudaEventRecord(c->ev_fork, s);
  for (int k = 0; k < std::min(nside, fcs_ctx::kSide) && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(c->side[k], c->ev_fork, 0);
  return e;
}
cudaError_t join_side(fcs_ctx* c, cudaStream_t s, int nside) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < std::min(nside, fcs_ctx::kSide) && e == cudaSuccess; ++k) {
    e = cudaEventRecord(c->ev_join[k], c->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join[k], 0);
  }
  return e;
}

// FC derivative of a scalar field: one launch per FFT-size group of line pairs
// (rows or columns; the column-tile kernel leaves most of its warps idle on a
// single field, whose adjacent columns share one transform).
template <typename T>
int launch_deriv(fcs_ctx* c, const void* in, void* out, int dir, int order, cudaStream_t s) {
  const int4* pr = dir == 0 ? c->pairs0 : c->pairs1;
  for (const Group& gr : c->g_pairs[dir]) {
    const long long work = ((long long)c->dev.instances * gr.count + jobs_per_round(gr.n1) - 1) / jobs_per_round(gr.n1);
    const LaunchCfg g{(unsigned)grid_for(work, kWarps), kWarps * 32, deriv_smem<T>(c, gr.n1), s};
    FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_fc_deriv<T, K>(c->dev, dir, order, pr + gr.begin, gr.count,
                                                      static_cast<const T*>(in), static_cast<T*>(out), g))); break)
  }
  return FCS_OK;
}

// The operator (and stage): column-tile passes (partial operator R), then
// row passes (L, and the stage update), one launch per FFT-size group; every
// column pass precedes every row pass in the stream.
template <typename T>
int launch_flux(fcs_ctx* c, const void* e, const void* mu, int mode, StageArgs<T> st, cudaStream_t s) {
  if (mu && c->opt.op_form == 1) return FCS_EUNSUPPORTED;  // the chain-rule form is inviscid
  const T* ep = static_cast<const T*>(e);
  const T* mp = static_cast<const T*>(mu);
  T* R = static_cast<T*>(c->R);
  T* G1 = static_cast<T*>(c->G1);
  T* G2 = static_cast<T*>(c->G2);
  if (mu) {  // viscous fluxes of curvilinear patches need e_q1 before the column pass (rows with mu != 0)
    for (const Group& gr : c->g_vpairs) {
      const long long work =
          ((long long)c->dev.instances * gr.count + jobs_per_round(gr.n1) - 1) / jobs_per_round(gr.n1);
      const LaunchCfg g{(unsigned)grid_for(work, kWarps), kWarps * 32, deriv_smem<T>(c, gr.n1), s};
      FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_fc_deriv<T, K>(c->dev, 0, 1, c->vpairs + gr.begin, gr.count, ep, G1, g, mp)));
                    break)
    }
  }
  const bool ch = c->opt.op_form == 1;
  // columns (all classes), then rows (all classes): each pass forks its
  // smaller classes onto the side streams, launched first so their few long
  // blocks start next to the largest class, and joins them back
  const std::vector<int> ocol = pass_order(c, 1), orow = pass_order(c, 0);
  FCS_CUDA(fork_side(c, s, (int)ocol.size() - 1));
  for (size_t k = 0; k < ocol.size(); ++k) {
    const Group& gr = c->g_tiles[ocol[k]];
    const cudaStream_t sk = side_of(c, s, (int)k, (int)ocol.size());
    const long long w1 = (long long)c->opt.instances * gr.count;
    const LaunchCfg gy{(unsigned)grid_for(w1, 1), kYWarps * 32, ypass_smem<T>(c, c->tw, gr.n1), sk};
    FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_ypass<T, K>(c->dev, c->tiles + gr.begin, gr.count, ep, mp, R, G1, G2, ch, gy)));
                  break)
  }
  FCS_CUDA(join_side(c, s, (int)ocol.size() - 1));
  FCS_CUDA(fork_side(c, s, (int)orow.size() - 1));
  for (size_t k = 0; k < orow.size(); ++k) {
    const Group& gr = c->g_rows[orow[k]];
    const cudaStream_t sk = side_of(c, s, (int)k, (int)orow.size());
    const long long w0 = (long long)c->opt.instances * ((gr.count + kRowsPerWarp - 1) / kRowsPerWarp);
    const LaunchCfg gx{(unsigned)grid_for(w0, kWarps), kWarps * 32, xpass_smem<T>(c, gr.n1), sk};
    const int b = gr.begin, n = gr.count;
    if (mode == MODE_RHS && !ch) {
      FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_xpass<T, MODE_RHS, K>(c->dev, b, n, ep, mp, R, G1, G2, st, gx))); break)
    } else if (mode == MODE_RHS) {
      FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_xpass<T, MODE_RHS | MODE_CHAIN, K>(c->dev, b, n, ep, mp, R, G1, G2, st, gx)));
                    break)
    } else if (!ch) {
      FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_xpass<T, MODE_RK, K>(c->dev, b, n, ep, mp, R, G1, G2, st, gx))); break)
    } else {
      FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_xpass<T, MODE_RK | MODE_CHAIN, K>(c->dev, b, n, ep, mp, R, G1, G2, st, gx)));
                    break)
    }
  }
  FCS_CUDA(join_side(c, s, (int)orow.size() - 1));
  if (mode == MODE_RK && c->dev.n_nsw > 0) {  // no-slip walls: temperature after every point's stage
    k_noslip_temperature<T><<<dim3((c->dev.n_nsw + 127) / 128, c->opt.instances), 128, 0, s>>>(c->dev, st.out);
    FCS_CUDA(cudaGetLastError());
  }
  return FCS_OK;
}

// Lines of kind 0 (full) or 1 (short, L-shaped patches only) of patch P along
// direction dir: rows j (dir 0) or columns i (dir 1) in [*lo, *hi).
void kind_range(const PatchDev& P, int dir, int kind, int* lo, int* hi) {
  if (dir == 0) {
    *lo = kind ? 0 : P.m2;
    *hi = kind ? P.m2 : P.n2;
  } else {
    *lo = kind ? 0 : P.m1;
    *hi = kind ? P.m1 : P.n1;
  }
}

// Group a per-line work list by FFT size: gen(p, lo, hi, out) emits the items
// of lines [lo, hi) of patch p; lines of size n1[0] come first, then n1[1], ...
// (patch order kept inside a group).
template <typename Item, typename Gen>
void grouped(const fcs_ctx* c, int dir, std::vector<Item>* out, std::vector<Group>* groups, Gen gen) {
  out->clear();
  groups->clear();
  for (int n1 : c->n1_dir[dir]) {
    Group g{n1, (int)out->size(), 0};
    for (int p = 0; p < c->npatch; ++p)
      for (int kind = 0; kind < 2; ++kind)
        if (c->kind_n1[dir][kind][p] == n1) {
          int lo, hi;
          kind_range(c->patches[p], dir, kind, &lo, &hi);
          gen(p, lo, hi, out);
        }
    g.count = (int)out->size() - g.begin;
    if (g.count) groups->push_back(g);
  }
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

namespace {
// Fringe exchange: copies, then interpolations (donors are never receivers, so
// the two launches write and read disjoint points).  clamp floors the
// interpolated values at zero (viscosity).
int exchange_impl(fcs_ctx* c, void* field, int nfields, int clamp, cudaStream_t s) {
  const long long I = c->opt.instances;
  const bool f64 = c->opt.dtype == FCS_F64;
  if (c->nent) {
    const int g = grid_for(I * c->nent * nfields, 256);
    const int4* en = c->fringe_ent[nfields == 4 ? 0 : 1];
    if (f64) k_exchange<double><<<g, 256, 0, s>>>(c->dev, en, c->nent, static_cast<double*>(field), nfields);
    else k_exchange<float><<<g, 256, 0, s>>>(c->dev, en, c->nent, static_cast<float*>(field), nfields);
  }
  if (c->ninterp) {
    const int g = grid_for(I * c->ninterp, 32);   // 4 entries per warp, 8 warps per block
    if (f64)
      k_interp<double><<<g, 256, 0, s>>>(c->dev, c->interp_ent[nfields == 4 ? 0 : 1], c->interp_w64, c->ninterp,
                                         static_cast<double*>(field), nfields, clamp);
    else
      k_interp<float><<<g, 256, 0, s>>>(c->dev, c->interp_ent[nfields == 4 ? 0 : 1], c->interp_w32, c->ninterp,
                                        static_cast<float*>(field), nfields, clamp);
  }
  return cuda_err(cudaGetLastError());
}

template <typename T>
int av_impl(fcs_ctx* c, const void* e, const int8_t* tau, void* mu, cudaStream_t s) {
  const dim3 g(c->dev.npblk, c->opt.instances);
  const int r = c->opt.av_radius;
  T* a0 = static_cast<T*>(c->av0);
  T* a1 = static_cast<T*>(c->av1);
  T* m = static_cast<T*>(mu);
  k_av_prelim<T><<<g, 256, 0, s>>>(c->dev, static_cast<const T*>(e), reinterpret_cast<const signed char*>(tau),
                                   T(c->opt.c_mu), T(c->opt.gamma), T(c->opt.gamma - 1.0), a1);
  if (r <= kBlendMaxR) {
    const size_t smem = blend_smem(r, sizeof(T));
    k_av_blend<T><<<grid_for((long long)c->opt.instances * c->nbtiles, 1), 256, smem, s>>>(c->dev, c->btiles,
                                                                                          c->nbtiles, a1, m, c->bump, r);
  } else {  // wide blends: the separable kernels
    k_av_boxmax<T><<<g, 256, 0, s>>>(c->dev, a1, a0, r, 0);
    k_av_boxmax<T><<<g, 256, 0, s>>>(c->dev, a0, a1, r, 1);
    k_av_bump<T><<<g, 256, 0, s>>>(c->dev, a1, a0, c->bump, r, 0);
    k_av_bump<T><<<g, 256, 0, s>>>(c->dev, a0, m, c->bump, r, 1);
  }
  FCS_CUDA(cudaGetLastError());
  return exchange_impl(c, mu, 1, 1, s);
}
}  // namespace

namespace {
int train_forward_backward(fcs_ctx* c, const float* x, const int8_t* lab, int B, float* loss, cudaStream_t s) {
  k_train_sample<<<(B + 127) / 128, 128, 0, s>>>(x, reinterpret_cast<const signed char*>(lab), B, c->Wm, c->acts,
                                                 c->loss_s);
  const int nchunk = (B + kGradChunk - 1) / kGradChunk;
  k_train_grad<<<dim3((kNParams + 127) / 128, nchunk), 128, 0, s>>>(c->acts, B, c->gpart);
  k_train_grad_final<<<(kNParams + 127) / 128, 128, 0, s>>>(c->gpart, nchunk, c->grad);
  k_train_loss<<<1, 256, 0, s>>>(c->loss_s, B, loss);
  return cuda_err(cudaGetLastError());
}
}  // namespace

// Column tiles of the pass along q2 for tile width tw (one instance),
// grouped by FFT size.
int set_tiles(fcs_ctx* c, int tw) {
  std::vector<int2> tiles;
  grouped(c, 1, &tiles, &c->g_tiles, [&](int p, int lo, int hi, std::vector<int2>* o) {
    for (int c0 = lo; c0 < hi; c0 += tw) o->push_back(make_int2(p, c0));
  });
  int2* t = nullptr;
  int rc = upload(c, &t, tiles.data(), tiles.size() * sizeof(int2));
  if (rc) return rc;
  c->tiles = t;
  c->ntiles = (int)tiles.size();
  c->tw = tw;
  c->dev.tw = tw;
  return FCS_OK;
}

template <typename T>
int time_rhs(fcs_ctx* c, float* ms) {
  cudaEvent_t a, b;
  FCS_CUDA(cudaEventCreate(&a));
  FCS_CUDA(cudaEventCreate(&b));
  StageArgs<T> st{0, T(0), nullptr, nullptr, nullptr, static_cast<T*>(c->A)};
  int rc = FCS_OK;
  for (int k = 0; k < 2 && !rc; ++k) rc = launch_flux<T>(c, c->S, nullptr, MODE_RHS, st, 0);
  cudaEventRecord(a, 0);
  for (int k = 0; k < 5 && !rc; ++k) rc = launch_flux<T>(c, c->S, nullptr, MODE_RHS, st, 0);
  cudaEventRecord(b, 0);
  cudaEventSynchronize(b);
  cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

// Autotuner of the lines per CTA of the pass along q2: time L(e) on a
// uniform state for every column-tile width that fits, keep the fastest.
// Results do not depend on the width (each column is transformed by the same
// lanes and instructions), only the work partition does.
int autotune_tile_width(fcs_ctx* c, const fcs_patch_desc* pd) {
  // uniform valid state (rho = 1, u = v = 0, p = 1) in the stage buffer
  std::vector<double> one(c->sstride * c->opt.instances, 0.0);
  for (size_t k = 0; k < (size_t)c->opt.instances; ++k)
    for (int p = 0; p < c->npatch; ++p) {
      const size_t np = (size_t)pd[p].n1 * pd[p].n2, base = k * c->sstride + c->state_off[p];
      for (size_t q = 0; q < np; ++q) {
        one[base + q] = 1.0;
        one[base + 3 * np + q] = 1.0 / (c->opt.gamma - 1.0);
      }
    }
  if (c->tsize == 8) {
    FCS_CUDA(cudaMemcpy(c->S, one.data(), one.size() * 8, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> f(one.begin(), one.end());
    FCS_CUDA(cudaMemcpy(c->S, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
  }
  float best = 1e30f;
  int best_tw = c->tw;
  for (int tw : c->tw_options) {
    int rc = set_tiles(c, tw);
    if (rc) return rc;
    float ms = 0.f;
    rc = c->tsize == 8 ? time_rhs<double>(c, &ms) : time_rhs<float>(c, &ms);
    if (rc) return rc;
    if (ms < best) {
      best = ms;
      best_tw = tw;
    }
  }
  return set_tiles(c, best_tw);
}

// =====================================================================
extern "C" {

void fcs_default_options(fcs_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->gamma = 1.4;
  o->cfl = 0.5;
  o->n_f = 5;
  o->dtype = FCS_F32;
  o->instances = 1;
  o->inflow[0] = 1.0;
  o->inflow[1] = 1.0;
  o->inflow[2] = 0.0;
  o->inflow[3] = 3.0;
  o->p_out = 1.0;
  o->c_mu = 1.0;
  o->av_radius = 4;
  o->c_policy = 0;
  o->train_batch_max = 4096;
  o->autotune = 0;
  o->filter_alpha = 16.0 * std::log(10.0);
  o->filter_p = 18;
  o->filter_step = 0;
  o->smear_p = 1;
  o->op_form = 0;
}

const char* fcs_strerror(int code) {
  switch (code) {
    case FCS_OK: return "ok";
    case FCS_EINVAL: return "invalid argument";
    case FCS_EOVERLAP: return "fringe point without a donor outside the donor's own fringe";
    case FCS_EUNSUPPORTED: return "unsupported configuration";
    case FCS_ECUDA: return "CUDA runtime error";
    case FCS_ENOMEM: return "device allocation failed";
    case FCS_ENONFINITE: return "non-finite value in the state";
    case FCS_ENEGATIVE: return "non-positive density or pressure";
    case FCS_ESCRATCH: return "batch larger than the fixed scratch of the no-allocation entry point";
    default: return "unknown error";
  }
}

int fcs_build_table(int d, int C, double* A_R_host) {
  if (!A_R_host) return FCS_EINVAL;
  return build_table(d, C, A_R_host) == 0 ? FCS_OK : FCS_EINVAL;
}

int fcs_line_c(const fcs_ctx* ctx, int N) {
  if (!ctx) return FCS_EINVAL;
  return choose_c(ctx->opt, ctx->C, N);
}

void fc_destroy(fcs_ctx* c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  for (int k = 0; k < fcs_ctx::kSide; ++k) {
    if (c->side[k]) cudaStreamDestroy(c->side[k]);
    if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
}

int fc_setup(fcs_ctx** out, int d, int C, const fcs_patch_desc* pd, int npatch, const fcs_options* opt) {
  if (!out) return FCS_EINVAL;
  *out = nullptr;
  if (!pd || npatch <= 0 || d < 2 || d > 8 || C < 2 || C > 64) return FCS_EINVAL;
  fcs_options o;
  if (opt) o = *opt;
  else fcs_default_options(&o);
  if (o.instances < 1 || (o.dtype != FCS_F32 && o.dtype != FCS_F64) || o.n_f < 1 || o.gamma <= 1.0 ||
      o.av_radius < 0 || o.av_radius > 32 || o.train_batch_max < 1 || !(o.filter_alpha >= 0.0) || o.filter_p < 1 ||
      o.filter_p > 64 || o.smear_p < 1 || o.smear_p > 64 || o.op_form < 0 || o.op_form > 1)
    return FCS_EINVAL;
  for (int p = 0; p < npatch; ++p) {
    const fcs_patch_desc& q = pd[p];
    if (q.n1 < 16 || q.n2 < 16 || q.n1 > kMaxLine || q.n2 > kMaxLine) return FCS_EINVAL;
    for (int s = 0; s < 4; ++s)
      if (q.bc[s] < 0 || q.bc[s] > 5) return FCS_EINVAL;
    if (q.cartesian) {
      if (!(q.box[1] > q.box[0]) || !(q.box[3] > q.box[2])) return FCS_EINVAL;
    } else {
      if (!q.x || !q.y) return FCS_EINVAL;
    }
    if (2 * o.n_f >= q.n1 || 2 * o.n_f >= q.n2) return FCS_EINVAL;
    if (q.lcut[0] != 0 || q.lcut[1] != 0) {  // L-shaped: both cuts, segments of >= 16 points
      if (q.lcut[0] <= 0 || q.lcut[1] <= 0 || q.n1 - q.lcut[0] < 16 || q.n2 - q.lcut[1] < 16) return FCS_EINVAL;
    }
    // no-slip walls: rectangular patches, never on two adjacent sides (a wall
    // point's inward line must hold no other wall point)
    const bool ns[4] = {q.bc[0] == 5, q.bc[1] == 5, q.bc[2] == 5, q.bc[3] == 5};
    if ((ns[0] || ns[1] || ns[2] || ns[3]) && (q.lcut[0] != 0 || q.lcut[1] != 0)) return FCS_EUNSUPPORTED;
    if ((ns[0] || ns[1]) && (ns[2] || ns[3])) return FCS_EUNSUPPORTED;
  }
  fcs_ctx* c = new fcs_ctx();
  c->opt = o;
  c->d = d;
  c->C = C;
  c->npatch = npatch;
  c->tsize = o.dtype == FCS_F64 ? 8 : 4;
  auto fail = [&](int rc) {
    fc_destroy(c);
    return rc;
  };

  // ---- plans, layout, patch descriptors
  size_t soff = 0, qoff = 0, woff_ = 0;
  const size_t align = 64;
  std::vector<LineRef> l0, l1;
  std::vector<int4> p0, p1, wins;
  for (int p = 0; p < npatch; ++p) {
    const fcs_patch_desc& q = pd[p];
    PatchDev P{};
    P.n1 = q.n1;
    P.n2 = q.n2;
    P.cart = q.cartesian ? 1 : 0;
    for (int s = 0; s < 4; ++s) P.bc[s] = q.bc[s];
    const bool lshape = q.lcut[0] > 0 && q.lcut[1] > 0;
    P.m1 = lshape ? q.lcut[0] : 0;
    P.m2 = lshape ? q.lcut[1] : 0;
    for (int dir = 0; dir < 2; ++dir)
      for (int kind = 0; kind < 2; ++kind) {
        if (kind == 1 && !lshape) {
          c->kind_n1[dir][kind].push_back(-1);
          continue;
        }
        const int N = (dir == 0 ? q.n1 : q.n2) - (kind ? (dir == 0 ? P.m1 : P.m2) : 0);
        const int pi = get_plan(c, N, choose_c(o, C, N), d);
        if (pi < 0) return fail(pi);
        (kind ? P.plan_s : P.plan)[dir] = pi;
        c->nmax = std::max(c->nmax, N);
        c->nfmax = std::max(c->nfmax, c->plans[pi].dev.n);
        int r = c->plans[pi].dev.n1reg;
        if (r % 2 == 0 && d > 5) r = 0;  // the two-level register FFT handles d <= 5
        c->gnmax[dir][r] = std::max(c->gnmax[dir][r], N);
        c->gnfmax[dir][r] = std::max(c->gnfmax[dir][r], c->plans[pi].dev.n);
        c->kind_n1[dir][kind].push_back(r);
        if (std::find(c->n1_dir[dir].begin(), c->n1_dir[dir].end(), r) == c->n1_dir[dir].end())
          c->n1_dir[dir].push_back(r);
      }
    c->n2max = std::max(c->n2max, q.n2);
    P.soff = (long long)soff;
    P.qoff = (long long)qoff;
    c->state_off.push_back((int64_t)soff);
    c->scalar_off.push_back((int64_t)qoff);
    soff += ((size_t)4 * q.n1 * q.n2 + align - 1) / align * align;
    qoff += ((size_t)q.n1 * q.n2 + align - 1) / align * align;
    if (q.cartesian) {
      P.Lx = q.box[1] - q.box[0];
      P.Ly = q.box[3] - q.box[2];
      P.hx = P.Lx / (q.n1 - 1);
      P.hy = P.Ly / (q.n2 - 1);
      P.hmax = std::max(P.hx, P.hy);
    } else {
      P.hx = 1.0 / (q.n1 - 1);
      P.hy = 1.0 / (q.n2 - 1);
      double hm = 0;
      for (int j = 0; j < q.n2; ++j)
        for (int i = 0; i < q.n1; ++i) {
          const long long k = (long long)j * q.n1 + i;
          if (!pt_active(P, i, j)) continue;
          if (i + 1 < q.n1) hm = std::max(hm, std::hypot(q.x[k + 1] - q.x[k], q.y[k + 1] - q.y[k]));
          if (j + 1 < q.n2) hm = std::max(hm, std::hypot(q.x[k + q.n1] - q.x[k], q.y[k + q.n1] - q.y[k]));
        }
      P.hmax = hm;
    }
    // windows: x-lines (j outer) then y-lines (i outer)
    auto starts = [](int N) {
      std::vector<int> s;
      for (int a = 0; a + 16 <= N; a += 16) s.push_back(a);
      if (s.back() + 16 < N) s.push_back(N - 16);
      return s;
    };
    for (int k = 0; k < 4; ++k) {
      P.inflowd[k] = q.inflow ? q.inflow[k] : o.inflow[k];
      P.inflowf[k] = (float)P.inflowd[k];
    }
    P.cd[PC_LX] = P.Lx;
    P.cd[PC_LY] = P.Ly;
    P.cd[PC_H1] = 1.0 / (q.n1 - 1);
    P.cd[PC_H2] = 1.0 / (q.n2 - 1);
    P.cd[PC_HMAX] = P.hmax;
    for (int k = 0; k < 5; ++k) P.cf[k] = (float)P.cd[k];
    // windows tile each line segment (rows j < m2 and columns i < m1 of an
    // L-shaped patch are short); the list is x-lines (j outer), then y-lines
    const std::vector<int> sx = starts(q.n1), sy = starts(q.n2);
    const std::vector<int> sxs = lshape ? starts(q.n1 - P.m1) : std::vector<int>();
    const std::vector<int> sys = lshape ? starts(q.n2 - P.m2) : std::vector<int>();
    P.wpl_x = (int)sx.size();
    P.wpl_y = (int)sy.size();
    P.wpl_xs = (int)sxs.size();
    P.wpl_ys = (int)sys.size();
    P.wx_off = (int)woff_;
    c->window_off.push_back((int64_t)woff_);
    for (int j = 0; j < q.n2; ++j) {
      const int a = line_start(P, 0, j);
      for (int s : (a ? sxs : sx)) wins.push_back(make_int4(p, 0, j, a + s));
    }
    P.wy_off = (int)wins.size();
    for (int i = 0; i < q.n1; ++i) {
      const int a = line_start(P, 1, i);
      for (int s : (a ? sys : sy)) wins.push_back(make_int4(p, 1, i, a + s));
    }
    woff_ = wins.size();
    for (int i = 0; i < q.n1; ++i) l1.push_back({p, i});
    c->patches.push_back(P);
  }
  // rows and line pairs grouped by FFT size (one launch per group)
  for (int dir = 0; dir < 2; ++dir) std::sort(c->n1_dir[dir].begin(), c->n1_dir[dir].end());
  // the two lines of a pair always have the same segment
  grouped(c, 0, &l0, &c->g_rows, [&](int p, int lo, int hi, std::vector<LineRef>* o) {
    for (int j = lo; j < hi; ++j) o->push_back({p, j});
  });
  grouped(c, 0, &p0, &c->g_pairs[0], [&](int p, int lo, int hi, std::vector<int4>* o) {
    for (int j = lo; j < hi; j += 2) o->push_back(make_int4(p, j, j + 1 < hi ? j + 1 : -1, -1));
  });
  grouped(c, 1, &p1, &c->g_pairs[1], [&](int p, int lo, int hi, std::vector<int4>* o) {
    for (int i = lo; i < hi; i += 2) o->push_back(make_int4(p, i, i + 1 < hi ? i + 1 : -1, -1));
  });
  std::vector<int4> fp[2];  // state-layout line pairs of every patch, 4 fields (filter)
  for (int dir = 0; dir < 2; ++dir)
    grouped(c, dir, &fp[dir], &c->g_fpairs[dir], [&](int p, int lo, int hi, std::vector<int4>* o) {
      for (int f = 0; f < 4; ++f)
        for (int l = lo; l < hi; l += 2) o->push_back(make_int4(p, l, l + 1 < hi ? l + 1 : -1, f));
    });
  std::vector<int4> vp;  // state-layout row pairs of curvilinear patches, 4 fields
  grouped(c, 0, &vp, &c->g_vpairs, [&](int p, int lo, int hi, std::vector<int4>* o) {
    if (pd[p].cartesian) return;
    for (int f = 0; f < 4; ++f)
      for (int i = lo; i < hi; i += 2) o->push_back(make_int4(p, i, i + 1 < hi ? i + 1 : -1, f));
  });
  // indicator plan (degree 5, C = 26 on 16-point windows; direct DFT)
  const int ind = get_plan(c, 16, kIndC, kIndD);
  if (ind < 0) return fail(ind);
  // lines in the Stockham group need a radix factorisation of their length
  for (int dir = 0; dir < 2; ++dir)
    for (int p = 0; p < npatch; ++p)
      for (int kind = 0; kind < 2; ++kind)
        if (c->kind_n1[dir][kind][p] == 0) {
          c->stockham = 1;
          const PatchDev& P = c->patches[p];
          if (c->plans[(kind ? P.plan_s : P.plan)[dir]].dev.nst == 0) return fail(FCS_EUNSUPPORTED);
        }
  // row passes and line-pair derivatives of every class must fit a block's
  // shared memory (long Stockham lines in FP64 may not)
  for (int n1 : c->n1_dir[0])
    if ((c->tsize == 8 ? xpass_smem<double>(c, n1) : xpass_smem<float>(c, n1)) > kSmemMax)
      return fail(FCS_EUNSUPPORTED);
  for (int dir = 0; dir < 2; ++dir)
    for (int n1 : c->n1_dir[dir])
      if ((c->tsize == 8 ? deriv_smem<double>(c, n1) : deriv_smem<float>(c, n1)) > kSmemMax)
        return fail(FCS_EUNSUPPORTED);
  // column-tile width of the pass along q2: widest of 32, 16, 8, 4 that fits
  // the 227 KB of shared memory a block may use (FP64 tiles of long columns
  // need the narrow widths)
  {
    const size_t esz = c->tsize, lim = kSmemMax;
    int tw = 0;
    for (int t : {32, 16, 8, 4}) {
      size_t b = 0;
      for (int n1 : c->n1_dir[1])
        b = std::max(b, esz == 8 ? ypass_smem<double>(c, t, n1) : ypass_smem<float>(c, t, n1));
      if (b <= lim) {
        if (!tw) tw = t;
        c->tw_options.push_back(t);
      }
    }
    if (!tw) return fail(FCS_EUNSUPPORTED);
    c->tw = tw;
  }
  {
    const int rc0 = set_tiles(c, c->tw);
    if (rc0) return fail(rc0);
  }
  std::vector<int2> pblk;
  for (int p = 0; p < npatch; ++p)
    for (int s0 = 0; s0 < pd[p].n1 * pd[p].n2; s0 += 256) pblk.push_back(make_int2(p, s0));
  // no-slip wall points: (patch, point, stride towards the interior)
  std::vector<int4> nsw;
  for (int p = 0; p < npatch; ++p) {
    const int n1 = pd[p].n1, n2 = pd[p].n2;
    for (int sd = 0; sd < 4; ++sd) {
      if (pd[p].bc[sd] != 5) continue;
      const int cnt = sd < 2 ? n2 : n1;
      for (int k = 0; k < cnt; ++k) {
        const int i = sd == 0 ? 0 : (sd == 1 ? n1 - 1 : k), j = sd == 2 ? 0 : (sd == 3 ? n2 - 1 : k);
        const int stride = sd == 0 ? 1 : (sd == 1 ? -1 : (sd == 2 ? n1 : -n1));
        nsw.push_back(make_int4(p, j * n1 + i, stride, 0));
      }
    }
  }
  std::vector<int4> btiles;  // blend tiles holding at least one point of the patch
  for (int p = 0; p < npatch; ++p)
    for (int j0 = 0; j0 < pd[p].n2; j0 += kBlendTile)
      for (int i0 = 0; i0 < pd[p].n1; i0 += kBlendTile) {
        const PatchDev& P = c->patches[p];
        if (i0 + kBlendTile <= P.m1 && j0 + kBlendTile <= P.m2) continue;  // inside the missing quadrant
        btiles.push_back(make_int4(p, i0, j0, 0));
      }
  c->nbtiles = (int)btiles.size();
  c->sstride = soff;
  c->qstride = qoff;
  c->nwin = wins.size();
  c->nlines0 = (int)l0.size();
  c->nlines1 = (int)l1.size();
  c->npairs0 = (int)p0.size();
  c->npairs1 = (int)p1.size();

  // ---- fringe map (§3.3): receivers within n_f points of an internal side;
  // donors by fcs_donors.cpp (copies on coincident nodes, else interpolation)
  std::vector<unsigned char> fringe(qoff, 0);
  for (int p = 0; p < npatch; ++p)
    for (int j = 0; j < pd[p].n2; ++j)
      for (int i = 0; i < pd[p].n1; ++i)
        if (is_receiver(pd[p], o.n_f, i, j)) fringe[c->scalar_off[p] + (long long)j * pd[p].n1 + i] = 1;
  std::vector<FringeCopy> fcopy;
  std::vector<FringeInterp> finterp;
  if (build_fringe(pd, npatch, o.n_f, &fcopy, &finterp) != 0) return fail(FCS_EOVERLAP);
  // entries resolved for the state layout (fields 4) and the scalar layout:
  // offsets within one instance (32-bit), field strides, the donor's row pitch
  if (soff > (size_t)INT32_MAX) return fail(FCS_EUNSUPPORTED);
  std::vector<int4> ent[2], ient[2];
  std::vector<double> iw64;
  auto resolved = [&](int lay, int dp, int dpt, int sp, int spt) {
    const long long dnp = (long long)pd[dp].n1 * pd[dp].n2, snp = (long long)pd[sp].n1 * pd[sp].n2;
    const int64_t* off = lay == 0 ? c->state_off.data() : c->scalar_off.data();
    return make_int4((int)(off[dp] + dpt), (int)(off[sp] + spt), (int)((lay == 0 ? dnp : 0) | ((long long)pd[sp].n1 << 19)),
                     (int)(lay == 0 ? snp : 0));
  };
  for (int lay = 0; lay < 2; ++lay) {
    for (const FringeCopy& f : fcopy) ent[lay].push_back(resolved(lay, f.dst_patch, f.dst_point, f.src_patch, f.src_point));
    for (const FringeInterp& f : finterp)
      ient[lay].push_back(resolved(lay, f.dst_patch, f.dst_point, f.src_patch, f.src_point));
  }
  for (const FringeInterp& f : finterp) {
    iw64.insert(iw64.end(), f.wi, f.wi + kStencil);   // 12 weights per entry: along i, then along j
    iw64.insert(iw64.end(), f.wj, f.wj + kStencil);
  }
  std::vector<float> iw32(iw64.begin(), iw64.end());
  c->nent = (int)ent[0].size();
  c->ninterp = (int)ient[0].size();

  // ---- Gram basis on the d matching points (orthonormalised Vandermonde
  // matrix, double-double) and per plan the blend values of the Gram
  // polynomials T = A_R Q (double-double, rounded to FP64 and FP32): the
  // continuation in the Gram form projects the d end values on the basis and
  // sums T times the coefficients
  std::vector<double> Qhi((size_t)d * d), Qlo((size_t)d * d);
  gram_basis_dd(d, Qhi.data(), Qlo.data());
  std::vector<float> gramQ(Qhi.begin(), Qhi.end()), gramT;
  std::vector<double> gramT64;
  std::vector<float> gramR;
  // ---- device tables
  std::vector<double> tab64;
  std::vector<float> thi, tlo;
  std::vector<double2> tw64;
  std::vector<float2> tw32;
  std::vector<double> flt64, smr64;
  std::vector<float> flt32, smr32;
  std::vector<PlanDev> plans;
  for (HostPlan& hp : c->plans) {
    hp.dev.tg_off = (int)gramT.size();
    {
      std::vector<double> Tb((size_t)hp.dev.C * d);
      gram_blend(d, hp.dev.C, hp.tab.data(), hp.tab_lo.data(), Qhi.data(), Qlo.data(), Tb.data());
      for (double v : Tb) {
        gramT.push_back((float)v);
        gramT64.push_back(v);
      }
    }
    hp.dev.rs_off = (int)gramR.size();
    {
      std::vector<double> rs(hp.dev.C);
      row_sums(d, hp.dev.C, hp.tab.data(), hp.tab_lo.data(), rs.data());
      for (double v : rs) gramR.push_back((float)v);
    }
    hp.dev.tab_off = (int)tab64.size();
    for (double v : hp.tab) {
      float a, b;
      split_float(v, &a, &b);
      tab64.push_back(v);
      thi.push_back(a);
      tlo.push_back(b);
    }
    hp.dev.tw_off = (int)tw64.size();
    std::vector<double> re(hp.dev.n), im(hp.dev.n);
    twiddles(hp.dev.n, re.data(), im.data());
    for (int k = 0; k < hp.dev.n; ++k) {
      tw64.push_back(make_double2(re[k], im[k]));
      tw32.push_back(make_float2((float)re[k], (float)im[k]));
      // filter factor of mode number min(k, n - k) (same offsets as the twiddles)
      const double kk = std::min(k, hp.dev.n - k) / (0.5 * hp.dev.n);
      const double sg = std::exp(-o.filter_alpha * std::pow(kk, 2.0 * o.filter_p));
      flt64.push_back(sg);
      flt32.push_back((float)sg);
      const double si = std::exp(-o.filter_alpha * std::pow(kk, 2.0 * o.smear_p));  // smearing filter
      smr64.push_back(si);
      smr32.push_back((float)si);
    }
    plans.push_back(hp.dev);
  }
  // quadrature weights per patch: rectangles, the FC quadratures of a row
  // and a column (tensor product); L-shaped patches, per point weights of
  // the union of the upper rectangle (rows j >= m2) and the lower right one
  // (rows j <= m2, columns i >= m1), each the tensor product of the FC
  // quadratures of its own line segments (marked by woff.y = -1)
  std::vector<double> wq;
  std::vector<int2> wo;
  for (int p = 0; p < npatch; ++p) {
    const PatchDev& P = c->patches[p];
    int2 w2;
    if (P.m1 > 0) {
      const int n1 = P.n1, n2 = P.n2, m1 = P.m1, m2 = P.m2;
      if (m2 + 1 < 2 * d) {   // too short a segment below the cut for a quadrature
        c->sums_ok = false;
        wo.push_back(make_int2(0, 0));
        continue;
      }
      auto seg = [&](int N, double len) {
        const int Cq = choose_c(o, C, N);
        std::vector<double> A((size_t)Cq * d);
        build_table(d, Cq, A.data());
        std::vector<double> W = quad_weights(N, Cq, d, A);
        for (double& x : W) x *= len;
        return W;
      };
      const std::vector<double> Wxf = seg(n1, 1.0), Wxs = seg(n1 - m1, double(n1 - 1 - m1) / (n1 - 1));
      const std::vector<double> Wyh = seg(n2 - m2, double(n2 - 1 - m2) / (n2 - 1)), Wyl = seg(m2 + 1, double(m2) / (n2 - 1));
      std::vector<double> w((size_t)n1 * n2, 0.0);
      for (int j = m2; j < n2; ++j)
        for (int i = 0; i < n1; ++i) w[(size_t)j * n1 + i] += Wyh[j - m2] * Wxf[i];
      for (int j = 0; j <= m2; ++j)
        for (int i = m1; i < n1; ++i) w[(size_t)j * n1 + i] += Wyl[j] * Wxs[i - m1];
      w2 = make_int2((int)wq.size(), -1);
      wq.insert(wq.end(), w.begin(), w.end());
    } else {
      for (int dir = 0; dir < 2; ++dir) {
        const HostPlan& hp = c->plans[P.plan[dir]];
        std::vector<double> W = quad_weights(hp.dev.N, hp.dev.C, d, hp.tab);
        (dir == 0 ? w2.x : w2.y) = (int)wq.size();
        wq.insert(wq.end(), W.begin(), W.end());
      }
    }
    wo.push_back(w2);
  }
  std::vector<double> bump(2 * o.av_radius + 1);
  for (int k = -o.av_radius; k <= o.av_radius; ++k) {
    const double t = k / (o.av_radius + 1.0);
    bump[k + o.av_radius] = std::exp(1.0 - 1.0 / (1.0 - t * t));
  }

  int rc;
  CtxDev& D = c->dev;
  PatchDev* dpatch;
  PlanDev* dplan;
  double *dtab64, *dW64;
  float *dthi, *dtlo;
  double2* dtw64;
  float2* dtw32;
  double* dflt64;
  float* dflt32;
  LineRef *dl0, *dl1;
  int4* dwin;
  unsigned char* dfr;
  int* dstatus;
  float *dgq, *dgt;
  double *dgqh, *dgql, *dgt64;
  float* dgr;
  if ((rc = upload(c, &dgq, gramQ.data(), gramQ.size() * 4)) || (rc = upload(c, &dgt, gramT.data(), gramT.size() * 4)) ||
      (rc = upload(c, &dgqh, Qhi.data(), Qhi.size() * 8)) || (rc = upload(c, &dgql, Qlo.data(), Qlo.size() * 8)) ||
      (rc = upload(c, &dgt64, gramT64.data(), gramT64.size() * 8)) ||
      (rc = upload(c, &dgr, gramR.data(), gramR.size() * 4)))
    return fail(rc);
  if ((rc = upload(c, &dpatch, c->patches.data(), c->patches.size() * sizeof(PatchDev))) ||
      (rc = upload(c, &dplan, plans.data(), plans.size() * sizeof(PlanDev))) ||
      (rc = upload(c, &dtab64, tab64.data(), tab64.size() * 8)) ||
      (rc = upload(c, &dthi, thi.data(), thi.size() * 4)) || (rc = upload(c, &dtlo, tlo.data(), tlo.size() * 4)) ||
      (rc = upload(c, &dtw64, tw64.data(), tw64.size() * sizeof(double2))) ||
      (rc = upload(c, &dtw32, tw32.data(), tw32.size() * sizeof(float2))) ||
      (rc = upload(c, &dflt64, flt64.data(), flt64.size() * 8)) || (rc = upload(c, &dflt32, flt32.data(), flt32.size() * 4)) ||
      (rc = upload(c, &c->smr64, smr64.data(), smr64.size() * 8)) ||
      (rc = upload(c, &c->smr32, smr32.data(), smr32.size() * 4)) ||
      (rc = upload(c, &dl0, l0.data(), l0.size() * sizeof(LineRef))) ||
      (rc = upload(c, &dl1, l1.data(), l1.size() * sizeof(LineRef))) ||
      (rc = upload(c, &c->pairs0, p0.data(), p0.size() * sizeof(int4))) ||
      (rc = upload(c, &c->pairs1, p1.data(), p1.size() * sizeof(int4))) ||
      (rc = upload(c, &c->vpairs, vp.data(), vp.size() * sizeof(int4))) ||
      (rc = upload(c, &c->fpairs[0], fp[0].data(), fp[0].size() * sizeof(int4))) ||
      (rc = upload(c, &c->fpairs[1], fp[1].data(), fp[1].size() * sizeof(int4))) ||
      (rc = upload(c, &c->pblk, pblk.data(), pblk.size() * sizeof(int2))) ||
      (rc = upload(c, &c->nsw, nsw.data(), nsw.size() * sizeof(int4))) ||
      (rc = upload(c, &c->btiles, btiles.data(), btiles.size() * sizeof(int4))) ||
      (rc = upload(c, &dwin, wins.data(), wins.size() * sizeof(int4))) ||
      (rc = upload(c, &dfr, fringe.data(), fringe.size())) ||
      (rc = upload(c, &c->fringe_ent[0], ent[0].data(), ent[0].size() * sizeof(int4))) ||
      (rc = upload(c, &c->fringe_ent[1], ent[1].data(), ent[1].size() * sizeof(int4))) ||
      (rc = upload(c, &c->interp_ent[0], ient[0].data(), ient[0].size() * sizeof(int4))) ||
      (rc = upload(c, &c->interp_ent[1], ient[1].data(), ient[1].size() * sizeof(int4))) ||
      (rc = upload(c, &c->interp_w64, iw64.data(), iw64.size() * 8)) ||
      (rc = upload(c, &c->interp_w32, iw32.data(), iw32.size() * 4)) ||
      (rc = upload(c, &c->wq, wq.data(), wq.size() * 8)) || (rc = upload(c, &c->woff, wo.data(), wo.size() * sizeof(int2))) ||
      (rc = upload(c, &c->bump, bump.data(), bump.size() * 8)) || (rc = dalloc(c, &dstatus, 16)))
    return fail(rc);
  const size_t I = (size_t)o.instances, ts = c->tsize;
  double *m64;
  float* m32;
  if ((rc = dalloc(c, &c->R, I * c->sstride * ts)) || (rc = dalloc(c, &c->S, I * c->sstride * ts)) ||
      (rc = dalloc(c, &c->A, I * c->sstride * ts)) || (rc = dalloc(c, &c->av0, I * c->qstride * ts)) ||
      (rc = dalloc(c, &c->av1, I * c->qstride * ts)) || (rc = dalloc(c, &c->mu, I * c->qstride * ts)) ||
      (rc = dalloc(c, &c->tau, I * c->qstride)) || (rc = dalloc(c, &c->tau_w, I * c->nwin)) ||
      (rc = dalloc(c, &c->dtbest, I * 8)) || (rc = dalloc(c, &c->dt_internal, I * 8)) ||
      (rc = dalloc(c, &c->Wm, kNParams * 4)) || (rc = dalloc(c, &c->Am, kNParams * 4)) ||
      (rc = dalloc(c, &c->Av, kNParams * 4)) || (rc = dalloc(c, &c->grad, kNParams * 4)) ||
      (rc = dalloc(c, &c->Wb, 1664 * 2)) || (rc = dalloc(c, &c->bias, 68 * 4)) ||
      (rc = dalloc(c, &dW64, kNParams * 8)) || (rc = dalloc(c, &c->acts, (size_t)o.train_batch_max * kActs * 4)) ||
      (rc = dalloc(c, &c->loss_s, (size_t)o.train_batch_max * 4)) ||
      (rc = dalloc(c, &c->gpart, (size_t)((o.train_batch_max + kGradChunk - 1) / kGradChunk) * kNParams * 8)) || (rc = dalloc(c, &m64, 5 * c->qstride * 8)) ||
      (rc = dalloc(c, &m32, 5 * c->qstride * 4)))
    return fail(rc);
  // G1, G2: e_q1, e_q2 of the lines with viscosity (viscous fluxes of both passes)
  if ((rc = dalloc(c, &c->G1, I * c->sstride * ts)) || (rc = dalloc(c, &c->G2, I * c->sstride * ts)))
    return fail(rc);
  c->W64 = dW64;
  D.patches = dpatch;
  D.plans = dplan;
  D.tab64 = dtab64;
  D.tabhi = dthi;
  D.tablo = dtlo;
  D.tw64 = dtw64;
  D.tw32 = dtw32;
  D.flt64 = dflt64;
  D.flt32 = dflt32;
  D.lines0 = dl0;
  D.lines1 = dl1;
  D.windows = dwin;
  D.metrics64 = m64;
  D.metrics32 = m32;
  D.fringe = dfr;
  D.status = dstatus;
  D.npatch = npatch;
  D.nlines0 = c->nlines0;
  D.nlines1 = c->nlines1;
  D.nwin = (int)c->nwin;
  D.instances = o.instances;
  D.d = d;
  D.sstride = (long long)c->sstride;
  D.qstride = (long long)c->qstride;
  D.gamma = o.gamma;
  D.gm1f = (float)(o.gamma - 1.0);
  D.p_outf = (float)o.p_out;
  for (int k = 0; k < 4; ++k) D.inflow[k] = o.inflow[k];
  D.p_out = o.p_out;
  D.ind_plan = ind;
  D.nmax = c->nmax;
  D.nfmax = c->nfmax;
  for (int dir = 0; dir < 2; ++dir)
    for (int k = 0; k < kN1Classes; ++k) {
      D.gnmax[dir][k] = c->gnmax[dir][k];
      D.gnfmax[dir][k] = c->gnfmax[dir][k];
    }
  D.stockham = c->stockham;
  D.gramQ = dgq;
  D.gramT = dgt;
  D.gramQ64h = dgqh;
  D.gramQ64l = dgql;
  D.gramT64 = dgt64;
  D.gramR = dgr;
  D.pblk = c->pblk;
  D.npblk = (int)pblk.size();
  D.nsw = c->nsw;
  D.n_nsw = (int)nsw.size();
  // derivative at node 0 of the interpolant on nodes 0..d-1: for node m > 0
  // its basis polynomial has the root 0, so the derivative there is the rest
  // of the product at 0 over m; node 0 takes minus the sum of the others
  // (a constant has zero derivative)
  {
    double w0 = 0.0;
    for (int m = 1; m < d; ++m) {
      double pr = 1.0 / m;
      for (int r = 1; r < d; ++r)
        if (r != m) pr *= (double)(-r) / (double)(m - r);
      D.nsw64[m] = pr;
      D.nsw32[m] = (float)pr;
      w0 -= pr;
    }
    D.nsw64[0] = w0;
    D.nsw32[0] = (float)w0;
  }
  D.tw = c->tw;
  D.n2max = c->n2max;
  if ((rc = (o.dtype == FCS_F64 ? set_smem_attrs<double>(c) : set_smem_attrs<float>(c)))) return fail(rc);
  if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) return fail(FCS_ECUDA);
  for (int k = 0; k < fcs_ctx::kSide; ++k)
    if (cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(FCS_ECUDA);
  if (o.dtype != FCS_F64) {  // the metrics use FP64 derivatives
    for (int dir = 0; dir < 2; ++dir)
      for (int n1 : c->n1_dir[dir]) {
        FCS_N1_SWITCH(n1, if (prep_fc_deriv<double, K>(deriv_smem<double>(c, n1)) != cudaSuccess) return fail(FCS_ECUDA); break)
      }
  }

  // ---- metrics of curvilinear patches: FP64 FC derivatives of x and y
  bool curvi = false;
  for (int p = 0; p < npatch; ++p) curvi |= !pd[p].cartesian;
  if (curvi) {
    std::vector<double> X(c->qstride, 0.0), Y(c->qstride, 0.0);
    for (int p = 0; p < npatch; ++p) {
      const fcs_patch_desc& q = pd[p];
      for (int j = 0; j < q.n2; ++j)
        for (int i = 0; i < q.n1; ++i) {
          const long long k = (long long)j * q.n1 + i;
          double xv, yv;
          if (q.cartesian) {
            xv = q.box[0] + (q.box[1] - q.box[0]) * i / (q.n1 - 1);
            yv = q.box[2] + (q.box[3] - q.box[2]) * j / (q.n2 - 1);
          } else {
            xv = q.x[k];
            yv = q.y[k];
          }
          X[c->scalar_off[p] + k] = xv;
          Y[c->scalar_off[p] + k] = yv;
        }
    }
    double *dX, *dY;
    if ((rc = upload(c, &dX, X.data(), X.size() * 8)) || (rc = upload(c, &dY, Y.data(), Y.size() * 8))) return fail(rc);
    // run with one instance: the geometry is shared by all instances
    CtxDev saved = D;
    D.instances = 1;
    const size_t Q = c->qstride;
    if ((rc = launch_deriv<double>(c, dX, m64 + 0 * Q, 0, 1, 0)) || (rc = launch_deriv<double>(c, dX, m64 + 1 * Q, 1, 1, 0)) ||
        (rc = launch_deriv<double>(c, dY, m64 + 2 * Q, 0, 1, 0)) || (rc = launch_deriv<double>(c, dY, m64 + 3 * Q, 1, 1, 0)))
      return fail(rc);
    D = saved;
    std::vector<double> Mh(5 * Q);
    if (cudaMemcpy(Mh.data(), m64, 4 * Q * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return fail(FCS_ECUDA);
    for (size_t k = 0; k < Q; ++k) Mh[4 * Q + k] = Mh[k] * Mh[3 * Q + k] - Mh[Q + k] * Mh[2 * Q + k];
    std::vector<float> Mf(Mh.begin(), Mh.end());
    if (cudaMemcpy(m64, Mh.data(), 5 * Q * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m32, Mf.data(), 5 * Q * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(FCS_ECUDA);
  }
  if (o.autotune && c->tw_options.size() > 1) {
    if ((rc = autotune_tile_width(c, pd))) return fail(rc);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(FCS_ECUDA);
  *out = c;
  return FCS_OK;
}

int fcs_get_layout(const fcs_ctx* c, fcs_layout* o) {
  if (!c || !o) return FCS_EINVAL;
  o->instances = c->opt.instances;
  o->npatch = c->npatch;
  o->dtype = c->opt.dtype;
  o->d = c->d;
  o->state_elems = c->sstride;
  o->scalar_elems = c->qstride;
  o->windows = c->nwin;
  o->state_off = c->state_off.data();
  o->scalar_off = c->scalar_off.data();
  o->window_off = c->window_off.data();
  o->tile_width = c->tw;
  o->launches_stage = (int)(c->g_rows.size() + c->g_tiles.size()) + (c->dev.n_nsw > 0);
  o->launches_stage_visc = o->launches_stage + (int)c->g_vpairs.size();
  o->launches_exchange = (c->nent > 0) + (c->ninterp > 0);
  o->launches_av = 1 + (c->opt.av_radius <= kBlendMaxR ? 1 : 4) + o->launches_exchange;
  return FCS_OK;
}

int fc_derivative(fcs_ctx* c, const void* in, void* out, int dir, int order, void* stream) {
  if (!c || !in || !out || in == out || (dir != 0 && dir != 1) || (order != 1 && order != 2)) return FCS_EINVAL;
  if (c->opt.dtype == FCS_F64) return launch_deriv<double>(c, in, out, dir, order, as_stream(stream));
  return launch_deriv<float>(c, in, out, dir, order, as_stream(stream));
}

int euler_rhs(fcs_ctx* c, const void* e, const void* mu, void* rhs, void* stream) {
  if (!c || !e || !rhs || e == rhs) return FCS_EINVAL;
  if (c->opt.dtype == FCS_F64) {
    StageArgs<double> st{0, 0.0, nullptr, nullptr, nullptr, static_cast<double*>(rhs)};
    return launch_flux<double>(c, e, mu, MODE_RHS, st, as_stream(stream));
  }
  StageArgs<float> st{0, 0.f, nullptr, nullptr, nullptr, static_cast<float*>(rhs)};
  return launch_flux<float>(c, e, mu, MODE_RHS, st, as_stream(stream));
}

int rk_stage(fcs_ctx* c, int stage, double dt, const double* dt_dev, const void* e_n, const void* e_s, void* acc,
             void* out, const void* mu, void* stream) {
  if (!c || stage < 0 || stage > 3 || !e_n || !e_s || !acc || !out) return FCS_EINVAL;
  if (stage == 0 && e_s != e_n) return FCS_EINVAL;
  if (out == e_n && stage != 3) return FCS_EINVAL;
  if (out == acc) return FCS_EINVAL;
  if (c->opt.dtype == FCS_F64) {
    StageArgs<double> st{stage, dt, dt_dev, static_cast<const double*>(e_n), static_cast<double*>(acc),
                         static_cast<double*>(out)};
    return launch_flux<double>(c, e_s, mu, MODE_RK, st, as_stream(stream));
  }
  StageArgs<float> st{stage, (float)dt, dt_dev, static_cast<const float*>(e_n), static_cast<float*>(acc),
                      static_cast<float*>(out)};
  return launch_flux<float>(c, e_s, mu, MODE_RK, st, as_stream(stream));
}

int patch_exchange(fcs_ctx* c, void* field, int nfields, void* stream) {
  if (!c || !field || (nfields != 1 && nfields != 4)) return FCS_EINVAL;
  return exchange_impl(c, field, nfields, 0, as_stream(stream));
}

int fcs_time_step(fcs_ctx* c, const void* e, const void* mu, double* dt_dev, void* stream) {
  if (!c || !e || !dt_dev) return FCS_EINVAL;
  cudaStream_t s = as_stream(stream);
  const int I = c->opt.instances;
  k_dt_init<<<(I + 127) / 128, 128, 0, s>>>(c->dtbest, I);
  const dim3 g(c->dev.npblk, I);
  const double gam = c->opt.gamma;
  if (c->opt.dtype == FCS_F64)
    k_dt<double><<<g, 256, 0, s>>>(c->dev, static_cast<const double*>(e), static_cast<const double*>(mu), c->opt.cfl,
                                   kCflMu, gam, gam - 1.0, c->dtbest);
  else
    k_dt<float><<<g, 256, 0, s>>>(c->dev, static_cast<const float*>(e), static_cast<const float*>(mu),
                                  (float)c->opt.cfl, (float)kCflMu, (float)gam, (float)(gam - 1.0), c->dtbest);
  k_dt_final<<<(I + 127) / 128, 128, 0, s>>>(c->dtbest, dt_dev, I);
  return cuda_err(cudaGetLastError());
}

int fcs_conservation_sums(fcs_ctx* c, const void* e, double* sums, void* stream) {
  if (!c || !e || !sums) return FCS_EINVAL;
  if (!c->sums_ok) return FCS_EUNSUPPORTED;  // an L-shaped patch cut too close to its bottom side
  const int blocks = c->opt.instances * c->npatch;
  if (c->opt.dtype == FCS_F64)
    k_sums<double><<<blocks, 256, 0, as_stream(stream)>>>(c->dev, static_cast<const double*>(e), c->wq, c->woff, sums);
  else
    k_sums<float><<<blocks, 256, 0, as_stream(stream)>>>(c->dev, static_cast<const float*>(e), c->wq, c->woff, sums);
  return cuda_err(cudaGetLastError());
}

int sdnn_set_weights(fcs_ctx* c, const float* w, size_t n) {
  if (!c || !w || n != (size_t)kNParams) return FCS_EINVAL;
  std::vector<__nv_bfloat16> wb(1664);
  std::vector<float> bias(68);
  std::vector<double> w64(kNParams);
  for (int t = 0; t < kNParams; ++t) {
    w64[t] = w[t];
    if (t < 512) wb[t] = __float2bfloat16_rn(w[t]);
    else if (t < 544) bias[t - 512] = w[t];
    else if (t < 1568) wb[512 + t - 544] = __float2bfloat16_rn(w[t]);
    else if (t < 1600) bias[32 + t - 1568] = w[t];
    else if (t < 1728) wb[1536 + t - 1600] = __float2bfloat16_rn(w[t]);
    else bias[64 + t - 1728] = w[t];
  }
  FCS_CUDA(cudaMemcpy(c->Wm, w, kNParams * 4, cudaMemcpyHostToDevice));
  FCS_CUDA(cudaMemcpy(c->Wb, wb.data(), 1664 * 2, cudaMemcpyHostToDevice));
  FCS_CUDA(cudaMemcpy(c->bias, bias.data(), 68 * 4, cudaMemcpyHostToDevice));
  FCS_CUDA(cudaMemcpy(c->W64, w64.data(), kNParams * 8, cudaMemcpyHostToDevice));
  FCS_CUDA(cudaMemset(c->Am, 0, kNParams * 4));
  FCS_CUDA(cudaMemset(c->Av, 0, kNParams * 4));
  c->adam_t = 0;
  return FCS_OK;
}

int sdnn_get_weights(fcs_ctx* c, float* w, size_t n) {
  if (!c || !w || n != (size_t)kNParams) return FCS_EINVAL;
  FCS_CUDA(cudaDeviceSynchronize());
  FCS_CUDA(cudaMemcpy(w, c->Wm, kNParams * 4, cudaMemcpyDeviceToHost));
  return FCS_OK;
}

int sdnn_classify(fcs_ctx* c, const void* e, int8_t* tau, void* logits, void* stream) {
  if (!c || !e || !tau) return FCS_EINVAL;
  cudaStream_t s = as_stream(stream);
  const long long nw = (long long)c->opt.instances * c->nwin;
  const dim3 gp(c->dev.npblk, c->opt.instances);
  if (c->opt.dtype == FCS_F64) {
    k_av_speed<double><<<gp, 256, 0, s>>>(c->dev, static_cast<const double*>(e), static_cast<double*>(c->av0), 1, c->opt.gamma,
                                          c->opt.gamma - 1.0);
    k_mlp64<double><<<grid_for(nw, 128), 128, 0, s>>>(c->dev, static_cast<const double*>(c->av0), c->W64, c->tau_w,
                                                      static_cast<double*>(logits));
  } else {
    k_av_speed<float><<<gp, 256, 0, s>>>(c->dev, static_cast<const float*>(e), static_cast<float*>(c->av0), 1, (float)c->opt.gamma,
                                         (float)(c->opt.gamma - 1.0));
    const long long groups = (nw + 15) / 16;
    k_mlp_bf16<<<grid_for(groups, 4), 128, 0, s>>>(c->dev, static_cast<const float*>(c->av0), c->Wb, c->bias,
                                                    c->tau_w, static_cast<float*>(logits));
  }
  FCS_CUDA(cudaGetLastError());
  k_tau_gather<<<gp, 256, 0, s>>>(c->dev, c->tau_w, reinterpret_cast<signed char*>(tau));
  return cuda_err(cudaGetLastError());
}

int sdnn_windows(fcs_ctx* c, const void* e, float* x, int8_t* flat, void* stream) {
  if (!c || !e || !x) return FCS_EINVAL;
  cudaStream_t s = as_stream(stream);
  const long long nw = (long long)c->opt.instances * c->nwin;
  const dim3 gp(c->dev.npblk, c->opt.instances);
  signed char* fl = reinterpret_cast<signed char*>(flat);
  if (c->opt.dtype == FCS_F64) {
    k_av_speed<double><<<gp, 256, 0, s>>>(c->dev, static_cast<const double*>(e), static_cast<double*>(c->av0), 1, c->opt.gamma,
                                          c->opt.gamma - 1.0);
    k_windows<double><<<grid_for(nw, 128), 128, 0, s>>>(c->dev, static_cast<const double*>(c->av0), x, fl);
  } else {
    k_av_speed<float><<<gp, 256, 0, s>>>(c->dev, static_cast<const float*>(e), static_cast<float*>(c->av0), 1, (float)c->opt.gamma,
                                         (float)(c->opt.gamma - 1.0));
    k_windows<float><<<grid_for(nw, 128), 128, 0, s>>>(c->dev, static_cast<const float*>(c->av0), x, fl);
  }
  return cuda_err(cudaGetLastError());
}

int sdnn_indicator(fcs_ctx* c, const void* e, int8_t* tau, void* s_out, void* stream) {
  if (!c || !e || !tau) return FCS_EINVAL;
  cudaStream_t s = as_stream(stream);
  const long long nw = (long long)c->opt.instances * c->nwin;
  const dim3 gp(c->dev.npblk, c->opt.instances);
  if (c->opt.dtype == FCS_F64) {
    k_av_speed<double><<<gp, 256, 0, s>>>(c->dev, static_cast<const double*>(e), static_cast<double*>(c->av0), 1, c->opt.gamma,
                                          c->opt.gamma - 1.0);
    k_indicator<double><<<grid_for(nw, 128), 128, 0, s>>>(c->dev, static_cast<const double*>(c->av0), c->tau_w,
                                                          static_cast<double*>(s_out));
  } else {
    k_av_speed<float><<<gp, 256, 0, s>>>(c->dev, static_cast<const float*>(e), static_cast<float*>(c->av0), 1, (float)c->opt.gamma,
                                         (float)(c->opt.gamma - 1.0));
    k_indicator<float><<<grid_for(nw, 128), 128, 0, s>>>(c->dev, static_cast<const float*>(c->av0), c->tau_w,
                                                         static_cast<float*>(s_out));
  }
  FCS_CUDA(cudaGetLastError());
  k_tau_gather<<<gp, 256, 0, s>>>(c->dev, c->tau_w, reinterpret_cast<signed char*>(tau));
  return cuda_err(cudaGetLastError());
}


int av_assemble(fcs_ctx* c, const void* e, const int8_t* tau, void* mu, void* stream) {
  if (!c || !e || !tau || !mu) return FCS_EINVAL;
  if (c->opt.dtype == FCS_F64) return av_impl<double>(c, e, tau, mu, as_stream(stream));
  return av_impl<float>(c, e, tau, mu, as_stream(stream));
}


int sdnn_gradient(fcs_ctx* c, const float* x, const int8_t* lab, int B, float* loss, float* grad, void* stream) {
  if (!c || !x || !lab || !grad || B < 1 || B > c->opt.train_batch_max) return FCS_EINVAL;
  cudaStream_t s = as_stream(stream);
  int rc = train_forward_backward(c, x, lab, B, loss, s);
  if (rc) return rc;
  return cuda_err(cudaMemcpyAsync(grad, c->grad, kNParams * 4, cudaMemcpyDeviceToDevice, s));
}

// ---- no-allocation variant of the classifier gradient.  Its scratch (per
// sample activations and losses) is a file-scope device array; host code only
// ever passes the array's device address, looked up once per device.
constexpr size_t kNoAllocActs = (size_t)FCS_NOALLOC_BATCH_MAX * kActs;
constexpr size_t kNoAllocChunks = (FCS_NOALLOC_BATCH_MAX + kGradChunk - 1) / kGradChunk;
// activations, per-sample losses, then (8-byte aligned) the FP64 partial gradients
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocActs + FCS_NOALLOC_BATCH_MAX +
                                                          2 * kNoAllocChunks * kNParams];
namespace {
constexpr int kMaxDevices = 64;
float* g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;
}  // namespace

int sdnn_gradient_noalloc(const float* w, const float* x, const int8_t* lab, int B, float* loss, float* grad,
                          void* stream) {
  if (!w || !x || !lab || !grad || B < 1) return FCS_EINVAL;
  if (B > FCS_NOALLOC_BATCH_MAX) return FCS_ESCRATCH;
  int dev = -1;
  FCS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FCS_EUNSUPPORTED;
  float* acts;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      FCS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[dev] = static_cast<float*>(p);
    }
    acts = g_noalloc_addr[dev];
  }
  cudaStream_t s = as_stream(stream);
  k_train_sample<<<(B + 127) / 128, 128, 0, s>>>(x, reinterpret_cast<const signed char*>(lab), B, w, acts,
                                                 acts + kNoAllocActs);
  double* part = reinterpret_cast<double*>(acts + kNoAllocActs + FCS_NOALLOC_BATCH_MAX);
  const int nchunk = (B + kGradChunk - 1) / kGradChunk;
  k_train_grad<<<dim3((kNParams + 127) / 128, nchunk), 128, 0, s>>>(acts, B, part);
  k_train_grad_final<<<(kNParams + 127) / 128, 128, 0, s>>>(part, nchunk, grad);
  k_train_loss<<<1, 256, 0, s>>>(acts + kNoAllocActs, B, loss);
  return cuda_err(cudaGetLastError());
}

int sdnn_train_step(fcs_ctx* c, const float* x, const int8_t* lab, int B, float lr, float* loss, void* stream) {
  if (!c || !x || !lab || B < 1 || B > c->opt.train_batch_max) return FCS_EINVAL;
  cudaStream_t s = as_stream(stream);
  int rc = train_forward_backward(c, x, lab, B, loss, s);
  if (rc) return rc;
  c->adam_t += 1;
  const float b1c = 1.f - std::pow(0.9f, (float)c->adam_t), b2c = 1.f - std::pow(0.999f, (float)c->adam_t);
  k_adam<<<(kNParams + 127) / 128, 128, 0, s>>>(c->Wm, c->Am, c->Av, c->grad, lr, b1c, b2c, c->Wb, c->bias, c->W64);
  return cuda_err(cudaGetLastError());
}

}  // extern "C"

namespace {
// Spectral filter with the factor tables of dev (the step filter or the
// smearing filter), blended into the state by w when w is not null.
int filter_impl(fcs_ctx* c, void* e, const CtxDev& dev, const void* w, cudaStream_t s) {
  const dim3 g(dev.npblk, c->opt.instances);
  const bool f64 = c->opt.dtype == FCS_F64;
  const double gm1 = c->opt.gamma - 1.0;
  if (f64) k_filter_prep<double><<<g, 256, 0, s>>>(dev, static_cast<const double*>(e), static_cast<double*>(c->R), gm1);
  else k_filter_prep<float><<<g, 256, 0, s>>>(dev, static_cast<const float*>(e), static_cast<float*>(c->R), (float)gm1);
  FCS_CUDA(cudaGetLastError());
  // rows R -> S, columns S -> R (order 0 of the line transform: filter)
  for (int dir = 0; dir < 2; ++dir) {
    void* src = dir == 0 ? c->R : c->S;
    void* dst = dir == 0 ? c->S : c->R;
    if (dir == 1) {   // columns: tiles of adjacent columns, the four fields of the state layout
      for (const Group& gr : c->g_tiles) {
        const unsigned grid = (unsigned)grid_for((long long)dev.instances * gr.count, 1);
        if (f64) {
          const LaunchCfg lc{grid, kYWarps * 32, cols_smem<double>(c, c->tw, gr.n1, 4), s};
          FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_fc_cols<double, K>(dev, 0, c->tiles + gr.begin, gr.count, 4,
                                                                static_cast<const double*>(src),
                                                                static_cast<double*>(dst), lc))); break)
        } else {
          const LaunchCfg lc{grid, kYWarps * 32, cols_smem<float>(c, c->tw, gr.n1, 4), s};
          FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_fc_cols<float, K>(dev, 0, c->tiles + gr.begin, gr.count, 4,
                                                               static_cast<const float*>(src),
                                                               static_cast<float*>(dst), lc))); break)
        }
      }
      continue;
    }
    for (const Group& gr : c->g_fpairs[dir]) {
      const long long work = ((long long)dev.instances * gr.count + jobs_per_round(gr.n1) - 1) / jobs_per_round(gr.n1);
      if (f64) {
        const LaunchCfg lc{(unsigned)grid_for(work, kWarps), kWarps * 32, deriv_smem<double>(c, gr.n1), s};
        FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_fc_deriv<double, K>(dev, dir, 0, c->fpairs[dir] + gr.begin, gr.count,
                                                               static_cast<const double*>(src),
                                                               static_cast<double*>(dst), lc))); break)
      } else {
        const LaunchCfg lc{(unsigned)grid_for(work, kWarps), kWarps * 32, deriv_smem<float>(c, gr.n1), s};
        FCS_N1_SWITCH(gr.n1, FCS_CUDA((run_fc_deriv<float, K>(dev, dir, 0, c->fpairs[dir] + gr.begin, gr.count,
                                                              static_cast<const float*>(src),
                                                              static_cast<float*>(dst), lc))); break)
      }
    }
  }
  if (f64)
    k_filter_done<double><<<g, 256, 0, s>>>(dev, static_cast<const double*>(c->R), static_cast<double*>(e), gm1,
                                            static_cast<const double*>(w));
  else
    k_filter_done<float><<<g, 256, 0, s>>>(dev, static_cast<const float*>(c->R), static_cast<float*>(e), (float)gm1,
                                           static_cast<const float*>(w));
  FCS_CUDA(cudaGetLastError());
  if (dev.n_nsw > 0) {  // no-slip walls: temperature from the filtered interior
    const dim3 gw((dev.n_nsw + 127) / 128, c->opt.instances);
    if (f64) k_noslip_temperature<double><<<gw, 128, 0, s>>>(dev, static_cast<double*>(e));
    else k_noslip_temperature<float><<<gw, 128, 0, s>>>(dev, static_cast<float*>(e));
    FCS_CUDA(cudaGetLastError());
  }
  return exchange_impl(c, e, 4, 0, s);
}

// Box maximum then bump average of a scalar field (the viscosity blend):
// in -> out, tmp as work space (the separable kernels overwrite in).
template <typename T>
int blend_impl(fcs_ctx* c, T* in, T* tmp, T* out, cudaStream_t s) {
  const int r = c->opt.av_radius;
  if (r <= kBlendMaxR) {
    k_av_blend<T><<<grid_for((long long)c->opt.instances * c->nbtiles, 1), 256, blend_smem(r, sizeof(T)), s>>>(
        c->dev, c->btiles, c->nbtiles, in, out, c->bump, r);
  } else {
    const dim3 g(c->dev.npblk, c->opt.instances);
    k_av_boxmax<T><<<g, 256, 0, s>>>(c->dev, in, tmp, r, 0);
    k_av_boxmax<T><<<g, 256, 0, s>>>(c->dev, tmp, in, r, 1);
    k_av_bump<T><<<g, 256, 0, s>>>(c->dev, in, tmp, c->bump, r, 0);
    k_av_bump<T><<<g, 256, 0, s>>>(c->dev, tmp, out, c->bump, r, 1);
  }
  return cuda_err(cudaGetLastError());
}
}  // namespace

extern "C" {

int fcs_filter(fcs_ctx* c, void* e, void* stream) {
  if (!c || !e) return FCS_EINVAL;
  return filter_impl(c, e, c->dev, nullptr, as_stream(stream));
}

int fcs_smear_initial(fcs_ctx* c, void* e, const int8_t* tau, void* stream) {
  if (!c || !e || !tau) return FCS_EINVAL;
  cudaStream_t s = as_stream(stream);
  const dim3 g(c->dev.npblk, c->opt.instances);
  const signed char* t = reinterpret_cast<const signed char*>(tau);
  int rc;
  if (c->opt.dtype == FCS_F64) {
    double *w0 = static_cast<double*>(c->av1), *tmp = static_cast<double*>(c->av0), *w = static_cast<double*>(c->mu);
    k_smear_seed<double><<<g, 256, 0, s>>>(c->dev, t, w0);
    if ((rc = blend_impl<double>(c, w0, tmp, w, s))) return rc;
  } else {
    float *w0 = static_cast<float*>(c->av1), *tmp = static_cast<float*>(c->av0), *w = static_cast<float*>(c->mu);
    k_smear_seed<float><<<g, 256, 0, s>>>(c->dev, t, w0);
    if ((rc = blend_impl<float>(c, w0, tmp, w, s))) return rc;
  }
  CtxDev dev = c->dev;  // the same context with the smearing filter's factors
  dev.flt64 = c->smr64;
  dev.flt32 = c->smr32;
  return filter_impl(c, e, dev, c->mu, s);
}

int fcs_step(fcs_ctx* c, void* e, double dt, double* dt_dev, int use_av, void* stream) {
  if (!c || !e) return FCS_EINVAL;
  if (!(dt > 0.0) && !dt_dev) return FCS_EINVAL;
  int rc;
  const void* mu = nullptr;
  if (use_av) {
    if ((rc = sdnn_classify(c, e, reinterpret_cast<int8_t*>(c->tau), nullptr, stream))) return rc;
    if ((rc = av_assemble(c, e, reinterpret_cast<int8_t*>(c->tau), c->mu, stream))) return rc;
    mu = c->mu;
  }
  const double* dtd = nullptr;
  if (!(dt > 0.0)) {
    if ((rc = fcs_time_step(c, e, mu, dt_dev, stream))) return rc;
    dtd = dt_dev;
  }
  for (int s = 0; s < 4; ++s) {
    const void* es = s == 0 ? e : c->S;
    void* out = s == 3 ? e : c->S;
    if ((rc = rk_stage(c, s, dt, dtd, e, es, c->A, out, mu, stream))) return rc;
    if ((rc = patch_exchange(c, out, 4, stream))) return rc;
  }
  if (c->opt.filter_step) return fcs_filter(c, e, stream);
  return FCS_OK;
}

int fcs_step_graph(fcs_ctx* c, void* e, double dt, double* dt_dev, int use_av, void* stream) {
  if (!c || !e || !stream) return FCS_EINVAL;
  cudaStream_t s = as_stream(stream);
  if (!c->gexec || c->g_e != e || c->g_dt != dt || c->g_dtdev != dt_dev || c->g_av != use_av || c->g_stream != s) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    FCS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = fcs_step(c, e, dt, dt_dev, use_av, stream);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    FCS_CUDA(ce);
    c->graph = g;
    FCS_CUDA(cudaGraphInstantiate(&c->gexec, g, 0));
    c->g_e = e;
    c->g_dt = dt;
    c->g_dtdev = dt_dev;
    c->g_av = use_av;
    c->g_stream = s;
  }
  return cuda_err(cudaGraphLaunch(c->gexec, s));
}

int fcs_alu_probe(int dtype, int blocks, int iters, void* out, void* stream) {
  if (blocks < 1 || iters < 1 || !out || (dtype != FCS_F32 && dtype != FCS_F64)) return FCS_EINVAL;
  if (dtype == FCS_F64) k_fma_probe<double><<<blocks, 256, 0, as_stream(stream)>>>(iters, static_cast<double*>(out));
  else k_fma_probe<float><<<blocks, 256, 0, as_stream(stream)>>>(iters, static_cast<float*>(out));
  FCS_CUDA(cudaGetLastError());
  return FCS_OK;
}

int fcs_status(fcs_ctx* c, int* flags) {
  if (!c) return FCS_EINVAL;
  FCS_CUDA(cudaDeviceSynchronize());
  int f = 0;
  FCS_CUDA(cudaMemcpy(&f, c->dev.status, sizeof(int), cudaMemcpyDeviceToHost));
  FCS_CUDA(cudaMemset(c->dev.status, 0, sizeof(int)));
  if (flags) *flags = f;
  if (f & 1) return FCS_ENONFINITE;
  if (f & 2) return FCS_ENEGATIVE;
  return FCS_OK;
}

}  // extern "C"
