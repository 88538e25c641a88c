/*
 * fcsdnn.h - C ABI of the GB300 (sm_103a) FC-SDNN Runge-Kutta stage library.
 *
 * The library evaluates the data-parallel hot path of the multi-patch FC-SDNN
 * scheme for the 2D compressible Euler equations (Leibovici & Bruno,
 * arXiv 2506.19370): FC-Gram continuation and FFT-based spectral derivatives
 * on every grid line, the Euler operator, the shock-detecting classifier,
 * smooth localized artificial viscosity, Runge-Kutta stages with boundary
 * conditions, and the exchange of fringe values between overlapping patches.
 *
 * Conventions shared by every entry point
 *  - Return value: FCS_OK (0) or a negative fcs_err code.  Argument and
 *    descriptor errors are reported synchronously; faults detected on the
 *    device (non-finite values, negative density or pressure) are latched in
 *    a status word that fcs_status() reads.  No call traps on the device.
 *  - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA
 *    tensors) owned by the caller; *_host pointers are host memory.  The
 *    library never frees caller memory.  A context owns its own device
 *    tables and work buffers, allocated in fc_setup and freed by fc_destroy;
 *    no other call allocates.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every compute call is asynchronous on that stream except
 *    fc_setup, fcs_status, sdnn_set_weights and sdnn_get_weights, which
 *    synchronise.
 *  - Floating-point arrays use the context's dtype (FCS_F32 -> float,
 *    FCS_F64 -> double) unless the signature says otherwise.
 *  - State layout ("state"): [instance][patch][field][j][i], field = rho,
 *    rho u, rho v, E (Eq. 1); i runs along the first parameter q1 and is
 *    contiguous; j runs along q2.  Offsets come from fcs_get_layout.
 *    Scalar fields (viscosity mu, classifier tau) use [instance][patch][j][i].
 *  - Every context handles `instances` independent copies of one patch
 *    layout in the same call (batched ensemble).
 */
#ifndef FCSDNN_H
#define FCSDNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fcs_ctx fcs_ctx;

typedef enum {
  FCS_OK = 0,
  FCS_EINVAL = -1,        /* bad argument or descriptor */
  FCS_EOVERLAP = -2,      /* a fringe point has no donor that is not itself a receiver (§3.3) */
  FCS_EUNSUPPORTED = -3,  /* valid request outside what this build implements */
  FCS_ECUDA = -4,         /* a CUDA runtime call failed */
  FCS_ENOMEM = -5,        /* device allocation failed in fc_setup */
  FCS_ENONFINITE = -6,    /* (status word) NaN or Inf met in the state */
  FCS_ENEGATIVE = -7,     /* (status word) non-positive density or pressure */
  FCS_ESCRATCH = -8       /* request larger than the fixed scratch of sdnn_gradient_noalloc */
} fcs_err;

typedef enum { FCS_F32 = 0, FCS_F64 = 1 } fcs_dtype;

/* Boundary-condition code of one patch side (left i=0, right i=n1-1,
 * bottom j=0, top j=n2-1).  Paper: §3.3 (internal sides, n_f-point fringes)
 * and §5 item 4 (boundary conditions enforced at every Runge-Kutta stage). */
typedef enum {
  FCS_BC_INTERNAL = 0,  /* fringe of n_f points filled from donor patches */
  FCS_BC_WALL = 1,      /* slip/reflecting wall: normal momentum set to 0 */
  FCS_BC_INFLOW = 2,    /* all conserved variables set to options.inflow */
  FCS_BC_OUTFLOW = 3,   /* pressure set to options.p_out, E recomputed */
  FCS_BC_FREE = 4,      /* nothing imposed */
  FCS_BC_NOSLIP = 5     /* no-slip adiabatic wall (paper §2, §7): momentum set
                           to 0; the temperature theta = p/rho of the wall point
                           is the value for which the polynomial through theta at
                           the d points of its inward grid line has zero
                           derivative there, E = rho theta/(gamma-1).  The
                           viscous mass and energy fluxes through the side are
                           zero, the momentum flux (wall shear) is kept.  Only
                           on rectangular patches, and never on two adjacent
                           sides of one patch (FCS_EUNSUPPORTED) */
} fcs_bc;

/* One patch (paper §3.1-3.2: patches are images of Cartesian parameter
 * grids).  Cartesian patches give their box; curvilinear patches give host
 * FP64 coordinates x[j*n1+i], y[j*n1+i] (copied in fc_setup, not retained).
 * 16 <= n1, n2 <= 256.
 * lcut = {m1, m2}, both > 0, makes an L-shaped corner patch (type C1 of
 * §3.2, parameter space L): the points i < m1, j < m2 do not belong to it
 * (they keep whatever the caller stores there and are never written), and
 * its inner edges i = m1 (j < m2) and j = m2 (i < m1) are walls; the corner
 * node (m1, m2) is a wall along the bisector of the two edge normals.  Each
 * remaining line segment needs at least 16 points.  Coordinates of
 * curvilinear L patches are given on the whole n1 x n2 grid (the patch map
 * extends over the missing quadrant).  {0, 0}: rectangular patch. */
typedef struct {
  int n1, n2;
  int bc[4];
  int cartesian;     /* 1: use box, 0: use x, y */
  double box[4];     /* x0, x1, y0, y1 */
  const double* x;   /* host, n1*n2, cartesian == 0 only */
  const double* y;
  int lcut[2];       /* {m1, m2}: L-shaped corner patch; {0, 0}: rectangle */
  const double* inflow; /* host, 4 conserved values for this patch's inflow sides
                           (copied in fc_setup); NULL: options.inflow */
} fcs_patch_desc;

typedef struct {
  double gamma;      /* heat-capacity ratio (1.4 in every test of the paper, §2) */
  double cfl;        /* CFL number of the time step (0.5, §7) */
  int n_f;           /* fringe width (5, §3.3) */
  int dtype;         /* fcs_dtype of every state-sized array */
  int instances;     /* independent copies of the layout handled per call */
  double inflow[4];  /* conserved inflow state for FCS_BC_INFLOW */
  double p_out;      /* pressure for FCS_BC_OUTFLOW */
  double c_mu;       /* artificial-viscosity scale (1.0) */
  int av_radius;     /* blend radius of the viscosity, grid points (4) */
  int c_policy;      /* 0: use C as given; 1: per line length, smallest C' >= C
                        making N + C' a product of 2, 3, 5, 7 (at most C + 16) */
  int train_batch_max; /* largest batch sdnn_train_step accepts (4096) */
  int autotune;      /* 1: fc_setup times the column-tile widths (lines per CTA of the
                        pass along q2) that fit and keeps the fastest; 0: widest (0) */
  double filter_alpha; /* spectral filter sigma(k) = exp(-alpha (|k|/k_max)^(2p))
                          (§5 item 3; I-(32) read with alpha = 16 ln 10) */
  int filter_p;        /* filter order p (18) */
  int filter_step;     /* 1: fcs_step ends with fcs_filter, so every step after
                          the first starts from filtered data; 0: off (0) */
  int smear_p;         /* order of the stronger filter of fcs_smear_initial (1) */
  int op_form;         /* form of the operator L(e): 0 conservative contravariant
                          flux form (0, the default); 1 chain-rule form of
                          Algorithm 5: FC derivatives of rho, rho u, rho v and
                          theta = p / rho along q1 and q2, physical derivatives
                          through the inverse Jacobian of the patch map, flux
                          divergence by the product rule (f_x + g_y = A w_x +
                          B w_y, A = df/dw, B = dg/dw).  Form 1 is inviscid:
                          calls with a viscosity return FCS_EUNSUPPORTED */
} fcs_options;

/* Defaults listed in the comments above. */
void fcs_default_options(fcs_options* opt);

/* Build a context (paper Algorithm 2, initialization): FC-Gram continuation
 * tables for degree d (2 <= d <= 8) and C continuation points (2 <= C <= 64;
 * paper §2; construction is a
 * Tikhonov-regularised oversampled Fourier-extension fit of the Gram
 * polynomials, solved in double-double arithmetic; the Gram basis and the
 * blend values of the Gram polynomials in double-double too), FFT plans,
 * metrics of curvilinear patches, fringe/donor maps (§3.3: a host donor
 * search over all patches; a receiver on a donor node is copied, any other
 * receiver is interpolated with a 6 x 6 tensor Lagrange stencil in the
 * donor's index space, Cartesian, curvilinear and L-shaped donors alike),
 * window tables of the classifier, device work buffers.  Patches have 16 to
 * 512 points per side.  Uses the current CUDA device.  Errors: FCS_EINVAL
 * (sizes, codes), FCS_EOVERLAP (a receiver without a donor that is not a
 * receiver itself), FCS_EUNSUPPORTED (FFT length with a prime factor above
 * 7; a line class whose buffers exceed a block's shared memory, possible
 * for FP64 lines near 512 points; no-slip walls on an L-shaped patch or on
 * two adjacent sides; more than 2^31 - 1 state elements per instance),
 * FCS_ENOMEM, FCS_ECUDA.  *out is NULL on error. */
int fc_setup(fcs_ctx** out, int d, int C, const fcs_patch_desc* patches, int npatch,
             const fcs_options* opt);

void fc_destroy(fcs_ctx* ctx);

typedef struct {
  int instances, npatch, dtype, d;
  size_t state_elems;         /* elements of one instance's state */
  size_t scalar_elems;        /* elements of one instance's scalar field */
  size_t windows;             /* classifier windows of one instance */
  const int64_t* state_off;   /* per patch offset in the state layout (host, ctx-owned) */
  const int64_t* scalar_off;  /* per patch offset in the scalar layout */
  const int64_t* window_off;  /* per patch offset of its first window */
  int tile_width;             /* columns per CTA of the pass along q2 (autotuned or widest) */
  int launches_stage;         /* kernel launches of one rk_stage call without viscosity (one row
                                 pass and one column pass per FFT-size group, plus the no-slip
                                 wall temperature when the layout has FCS_BC_NOSLIP sides;
                                 euler_rhs launches that one fewer) */
  int launches_stage_visc;    /* the same with viscosity (adds the e_q1 pass of curvilinear patches) */
  int launches_exchange;      /* kernel launches of one patch_exchange call (copies, interpolations) */
  int launches_av;            /* kernel launches of one av_assemble call (exchange included) */
} fcs_layout;

int fcs_get_layout(const fcs_ctx* ctx, fcs_layout* out);

/* Host-only: FP64 FC-Gram right-end continuation table A_R (C x d, row-major,
 * acting on the last d values of a line); the left-end table is its
 * reflection A_L[c][m] = A_R[C-1-c][d-1-m].  Paper §2.  Needs no GPU. */
int fcs_build_table(int d, int C, double* A_R_host);

/* Host-only: continuation length C' used for lines of N points under the
 * context's policy. */
int fcs_line_c(const fcs_ctx* ctx, int N);

/* FC spectral derivative (paper §2 and Algorithm 5: continuation, FFT,
 * multiplication by (ik)^order, inverse FFT, restriction) of a scalar field
 * on every line of every patch of every instance, along parameter direction
 * dir (0: q1/i, 1: q2/j), with respect to the parameter q in [0, 1]
 * (spacing 1/(n-1)).  in_dev/out_dev: scalar layout, may not alias.
 * order: 1 or 2. */
int fc_derivative(fcs_ctx* ctx, const void* in_dev, void* out_dev, int dir, int order, void* stream);

/* Euler operator L(e) (Eq. 1-3; Algorithm 5 operator step) on every patch:
 * conservative contravariant form -(1/J)[d_q1(y_q2 f - x_q2 g) +
 * d_q2(-y_q1 f + x_q1 g)], on Cartesian patches -(df/dx + dg/dy).  mu_dev
 * (scalar layout) adds the artificial-viscosity flux -mu grad e; NULL = off;
 * Cartesian patches only.  rhs_dev: state layout.  Boundary conditions are not
 * applied (they act on the state, see rk_stage). */
int euler_rhs(fcs_ctx* ctx, const void* e_dev, const void* mu_dev, void* rhs_dev, void* stream);

/* One stage (0..3) of the classical four-stage Runge-Kutta scheme (paper §5
 * item 4, Algorithm 5 stage update), fused with L(e_s):
 *   s=0: acc = e_n + dt/6 k;  out = e_n + dt/2 k      (e_s must equal e_n)
 *   s=1: acc += dt/3 k;       out = e_n + dt/2 k
 *   s=2: acc += dt/3 k;       out = e_n + dt k
 *   s=3:                      out = acc + dt/6 k
 * with k = L(e_s), then boundary conditions on out (sides left, right,
 * bottom, top).  dt: per instance from dt_dev (device, `instances` doubles)
 * or, if dt_dev is NULL, the scalar dt.  out may alias e_s but not e_n or acc.
 * Fringe exchange is a separate call (patch_exchange). */
int rk_stage(fcs_ctx* ctx, int stage, double dt, const double* dt_dev, const void* e_n_dev,
             const void* e_s_dev, void* acc_dev, void* out_dev, const void* mu_dev, void* stream);

/* Copy donor values into every fringe point (paper §3.3, Algorithm 1
 * exchange after each stage).  nfields = 4: state layout; nfields = 1:
 * scalar layout (used for the viscosity). */
int patch_exchange(fcs_ctx* ctx, void* field_dev, int nfields, void* stream);

/* Per-instance time step (Algorithm 1, the step-size evaluation; formula of
 * Part I (31) read as the CFL condition): dt = min over points of
 * 1 / (1/dt_a + 1/dt_v), dt_a = cfl * min_k h_k / (|U_k| + c |grad q_k|),
 * dt_v = 0.2 / (mu (1/s_1^2 + 1/s_2^2)); U_k the contravariant velocity, h_k
 * the parameter spacing, s_k the physical spacing along q_k; mu_dev (scalar
 * layout) may be NULL (no viscous limit).  Writes dt_dev (instances doubles). */
int fcs_time_step(fcs_ctx* ctx, const void* e_dev, const void* mu_dev, double* dt_dev, void* stream);

/* Spectral filter of the state, in place (§5 item 3, Algorithm 4 for t > 0):
 * on every line segment, along q1 then along q2, the FC-continued values of
 * rho, rho u, rho v and the temperature theta = p / rho are Fourier
 * transformed, multiplied by sigma(k) = exp(-filter_alpha (|k| / (n/2))^(2
 * filter_p)) for the mode numbers |k| <= n/2 of the continued line of n
 * points, transformed back and restricted; E follows from the filtered
 * theta, then the boundary conditions and the fringe exchange are applied.
 * Uses the context's work buffers (not concurrently with other calls). */
int fcs_filter(fcs_ctx* ctx, void* e_dev, void* stream);

/* Localized smearing of discontinuous initial data, in place (§5 item 3,
 * Algorithm 4 at t = 0; reading of I-(33)): e' = (1 - w) e + w F(e), with F
 * the spectral filter of fcs_filter at order smear_p (Gaussian for 1) and w
 * the smooth window around the points whose tau_dev (int8, scalar layout, as
 * written by sdnn_classify or sdnn_indicator) is 1 (jump): 1 there, spread by
 * the box maximum and the bump average of the viscosity blend (av_radius);
 * then boundary conditions and the fringe exchange. */
int fcs_smear_initial(fcs_ctx* ctx, void* e_dev, const int8_t* tau_dev, void* stream);

/* Per instance and patch, FP64 sums of each conserved field with the FC
 * quadrature weights times |J| (§7 energy test: integrals over the domain):
 * sums_dev[(instance * npatch + patch) * 4 + field].  Rectangular patches:
 * tensor product of the FC quadratures along q1 and q2.  L-shaped patches:
 * the union of the upper rectangle (rows j >= m2) and the lower right one
 * (rows j <= m2, columns i >= m1), each the tensor product of the FC
 * quadratures of its line segments.  Also checks the state and latches
 * FCS_ENONFINITE / FCS_ENEGATIVE into the status word.  FCS_EUNSUPPORTED if
 * an L-shaped patch has m2 + 1 < 2 d (no quadrature below its cut). */
int fcs_conservation_sums(fcs_ctx* ctx, const void* e_dev, double* sums_dev, void* stream);

/* Classifier weights (the paper's ANN, §4/§5 item 2): FP32 master copy,
 * layout W1[32][16], b1[32], W2[32][32], b2[32], W3[4][32], b3[4]
 * (1732 floats).  Synchronous. */
int sdnn_set_weights(fcs_ctx* ctx, const float* w_host, size_t n);
int sdnn_get_weights(fcs_ctx* ctx, float* w_host, size_t n);

/* Shock-detecting classification (Algorithm 3, proxy and smoothness steps):
 * Mach-number proxy, 16-point windows along every line in both directions,
 * normalisation, MLP 16-32-32-4, tau = 1 + argmax, per point the minimum over
 * the windows that cover it.  tau_dev: int8 scalar layout.  logits_dev:
 * optional [instance][window][4] in the context dtype (NULL to skip).  F32
 * contexts run the MLP on BF16 tensor cores with FP32 accumulation; F64
 * contexts in FP64. */
int sdnn_classify(fcs_ctx* ctx, const void* e_dev, int8_t* tau_dev, void* logits_dev, void* stream);

/* The classifier's input windows (Algorithm 3: the Mach-number proxy on
 * 16-point windows along every line, as sdnn_classify cuts them), before the
 * per-window normalisation that sdnn_classify and sdnn_train_step apply:
 * x_dev [instance][window][16] float, in the window order of the layout
 * (per patch: rows j = 0.. n2-1, each row's windows by start 0, 16, ...,
 * the last right-aligned, then the columns i = 0 .. n1-1 likewise; segments
 * of L-shaped patches as in the classifier).  flat_dev (int8
 * [instance][window], optional): 1 where the window is flat (classified
 * smooth without inference).  Used to build training data from states the
 * solver's own FC steps produced.  Work buffers are the context's. */
int sdnn_windows(fcs_ctx* ctx, const void* e_dev, float* x_dev, int8_t* flat_dev, void* stream);

/* Coefficient-decay smoothness indicator (fallback and judge of the
 * classifier; not in the paper): per window the decay rate s of the FC
 * spectrum of the raw proxy window, tau_hat 1 (s < 2.7), 2 (s < 4.4) or 4;
 * per point the minimum over covering windows.  s_dev optional
 * [instance][window] in the context dtype (+Inf for flat windows). */
int sdnn_indicator(fcs_ctx* ctx, const void* e_dev, int8_t* tau_dev, void* s_dev, void* stream);

/* Artificial viscosity (Algorithm 3, MWSB and viscosity steps; §4):
 * S = max over 3x3 of |u| + c, mu0 = c_mu h_max S w(tau), w = (1, 1/2, 0, 0),
 * zero on fringes, box maximum and normalised C-infinity bump average of
 * radius av_radius, fringe values from donors.  mu_dev: scalar layout. */
int av_assemble(fcs_ctx* ctx, const void* e_dev, const int8_t* tau_dev, void* mu_dev, void* stream);

/* One training step of the classifier (softmax cross-entropy, Adam with
 * lr, betas 0.9/0.999, eps 1e-8) on `batch` raw windows x_dev (float,
 * batch x 16, normalised inside like sdnn_classify) with labels_dev (int8,
 * 1..4).  Forward uses BF16-rounded inputs and weights, FP32 arithmetic;
 * master weights FP32.  loss_dev: optional device float receiving the mean
 * loss before the update.  batch <= options.train_batch_max. */
int sdnn_train_step(fcs_ctx* ctx, const float* x_dev, const int8_t* labels_dev, int batch, float lr,
                    float* loss_dev, void* stream);

/* Raw gradient of the mean loss at the current weights (no update), float
 * grad_dev[1732]; for checking against the CPU oracle. */
int sdnn_gradient(fcs_ctx* ctx, const float* x_dev, const int8_t* labels_dev, int batch, float* loss_dev,
                  float* grad_dev, void* stream);

/* Classifier gradient without any device allocation (no counterpart in the
 * paper: it exists for callers that cannot call cudaMalloc, such as hosts
 * that hand the library only buffers they allocated themselves from their own
 * memory arenas, or code that must not trigger the allocator's implicit
 * synchronisation).  Same result as sdnn_gradient, but the weights come in
 * as an argument (w_dev: 1732 floats, layout of sdnn_set_weights) and no
 * context is needed.  The per-sample activations live in one file-scope
 * device array sized for FCS_NOALLOC_BATCH_MAX samples (about 2.9 MB), which
 * every GPU that loads the library keeps until the process exits.
 *  - batch > FCS_NOALLOC_BATCH_MAX returns FCS_ESCRATCH; nothing is launched.
 *  - The first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - All calls share the array: calls that may overlap on the GPU (other
 *    streams, other host threads) race; serialise them.  Every value the
 *    kernels read from it is written earlier in the same call.
 *  - loss_dev may be NULL; grad_dev receives 1732 floats. */
#define FCS_NOALLOC_BATCH_MAX 4096
int sdnn_gradient_noalloc(const float* w_dev, const float* x_dev, const int8_t* labels_dev, int batch,
                          float* loss_dev, float* grad_dev, void* stream);

/* One full time step (Algorithm 1 loop body): if use_av, classify and
 * assemble the viscosity; the time step (dt_dev receives it) unless dt > 0
 * is given; four stages, each followed by the exchange.  e_dev is updated in
 * place.  Work buffers are the context's. */
int fcs_step(fcs_ctx* ctx, void* e_dev, double dt, double* dt_dev, int use_av, void* stream);

/* The same step captured once into a CUDA graph on `stream` and replayed;
 * recaptured when e_dev, dt, dt_dev or use_av change. */
int fcs_step_graph(fcs_ctx* ctx, void* e_dev, double dt, double* dt_dev, int use_av, void* stream);

/* Synchronous: device status word (bit 0 non-finite, bit 1 non-positive
 * density/pressure), then cleared.  Returns FCS_OK or the first error. */
int fcs_status(fcs_ctx* ctx, int* flags);

const char* fcs_strerror(int code);

/* Measurement helper (the paper has no counterpart): launches `blocks`
 * blocks of 256 threads that each run iters x 32 independent fused
 * multiply-adds per thread in FP32 (dtype FCS_F32) or FP64 (FCS_F64), i.e.
 * blocks x 256 x iters x 64 flops, asynchronously on `stream`.  Timed with
 * events around it, it gives the peak arithmetic rate that the roofline
 * fractions of the FC derivative and stage kernels are quoted against.
 * out_dev: device buffer of at least `blocks` elements of that type (never
 * written for these inputs).  FCS_EINVAL on a bad argument. */
int fcs_alu_probe(int dtype, int blocks, int iters, void* out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FCSDNN_H */
