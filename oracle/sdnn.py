"""Shock-detecting network, smoothness indicator and artificial viscosity (oracle).

Test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module.

Follows Algorithm 3 and §5 item 2 (the formulas themselves are in Part I,
§I-5, which is not available; the readings below fill them in):
  * proxy: the Mach number Phi = |u| sqrt(rho / (gamma p)) (§5 item 2);
  * windows: every grid line is cut into 16-point windows starting at 0, 16,
    32, ...; if the line length is not a multiple of 16 the last window is
    right-aligned.  A window is normalised as (Phi - mean) / (max - min);
    a window with max - min <= 1e-4 max(1, max|Phi|) is flat (its Mach-number
    variation is far below any shock) and gets tau = 4 without inference;
  * smoothness classifier (the ANN of §4): dense 16 -> 32 (ReLU) -> 32 (ReLU)
    -> 4, tau = 1 + argmax (1 jump, 2 kink, 3 C1 with a jump in the second
    derivative, 4 smooth); a point takes the smallest tau of all windows, in
    both directions, that contain it;
  * training: softmax cross-entropy, Adam (lr 1e-3, betas 0.9 / 0.999,
    eps 1e-8);
  * MWSB (I-(37)): S = max over the 3 x 3 neighbourhood of |u| + c;
  * preliminary viscosity (I-(38)): c_mu h_max S w(tau), w = (1, 1/2, 0, 0),
    zero on the n_f-point fringe;
  * smooth blend (I-(42), I-(44)): box maximum of radius r followed by a
    normalised separable C-infinity bump average of radius r
    (b(t) = exp(1 - 1/(1 - t^2)), t = k/(r+1)); fringe values then come
    from donors like the solution does;
  * coefficient-decay indicator (not in the paper; the fallback and judge of
    the classifier): FC continuation of the raw window with C = 26 (n = 42),
    band amplitudes E_lo (modes 2..5) and E_hi (modes 11..20) of the
    spectrum, floored at 1e-6 of the largest mode, decay rate
    s = log(E_lo / E_hi) / log(15.5 / 3.5); tau_hat = 1 for s < 2.7, 2 for
    2.7 <= s < 4.4 and 4 otherwise.  The cut points were calibrated on the
    seeded labelled windows; on 16 points the estimate does not separate C1
    profiles (class 3) from smooth ones, and both carry no viscosity.
"""
import numpy as np

from . import euler, fcgram

WINDOW = 16
HIDDEN = 32
CLASSES = 4
LAYER_SHAPES = ((HIDDEN, WINDOW), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (CLASSES, HIDDEN), (CLASSES,))
N_PARAMS = sum(int(np.prod(s)) for s in LAYER_SHAPES)
FLAT_TOL = 1e-4
VISC_WEIGHT = (1.0, 0.5, 0.0, 0.0)
IND_C = 26
IND_D = 5
IND_CUTS = (2.7, 4.4)


# ---------------------------------------------------------------- proxy + windows
def proxy(e, gamma):
    """Phi = |u| sqrt(rho/(gamma p)) (§5 item 2, Algorithm 3)."""
    rho, mx, my, _ = e
    p = euler.pressure(e, gamma)
    return np.sqrt(mx * mx + my * my) / rho * np.sqrt(rho / (gamma * p))


def window_starts(N, W=WINDOW):
    if N < W:
        raise ValueError("line shorter than a window")
    starts = list(range(0, N - W + 1, W))
    if starts[-1] + W < N:
        starts.append(N - W)
    return starts


def line_span(n1, n2, lcut, dirn, line):
    """(first index, length) of a grid line (row j for dirn 0, column i for
    dirn 1) of a patch, L-shaped when lcut = (m1, m2) > 0."""
    m1, m2 = lcut
    if dirn == 0:
        return (m1, n1 - m1) if (m1 > 0 and m2 > 0 and line < m2) else (0, n1)
    return (m2, n2 - m2) if (m1 > 0 and m2 > 0 and line < m1) else (0, n2)


def patch_windows(phi, lcut=(0, 0)):
    """All windows of one patch: x-lines (j outer) then y-lines (i outer);
    on an L-shaped patch the windows tile each line's segment.

    Returns (win (nwin, 16), cover) where cover[w] = (direction, line, start).
    """
    n2, n1 = phi.shape
    wins, cover = [], []
    for j in range(n2):
        a, N = line_span(n1, n2, lcut, 0, j)
        for s in window_starts(N):
            wins.append(phi[j, a + s:a + s + WINDOW])
            cover.append((0, j, a + s))
    for i in range(n1):
        a, N = line_span(n1, n2, lcut, 1, i)
        for s in window_starts(N):
            wins.append(phi[a + s:a + s + WINDOW, i])
            cover.append((1, i, a + s))
    return np.array(wins), cover


def normalise(win):
    """(Phi - mean)/(max - min) per window; flat windows flagged (zeros)."""
    mn = win.min(axis=1, keepdims=True)
    mx = win.max(axis=1, keepdims=True)
    mean = win.mean(axis=1, keepdims=True)
    amax = np.abs(win).max(axis=1, keepdims=True)
    flat = (mx - mn) <= FLAT_TOL * np.maximum(1.0, amax)
    rng = np.where(flat, 1.0, mx - mn)
    return np.where(flat, 0.0, (win - mean) / rng), flat[:, 0]


# ---------------------------------------------------------------- MLP
def unpack(params):
    out, o = [], 0
    for s in LAYER_SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(params[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def init_params(seed=0):
    """He-uniform weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in LAYER_SHAPES:
        if len(s) == 2:
            lim = np.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32).copy()
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_forward(params, x, bf16=False):
    """Logits (B, 4) and the hidden activations; bf16=True rounds inputs, weights
    and hidden activations to bfloat16 as the tensor-core kernel does."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = r(x)
    z1 = x @ r(W1).T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = r(h1) @ r(W2).T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = r(h2) @ r(W3).T + b3
    return z3, (x, z1, h1, z2, h2)


def classify_windows(params, win, bf16=False):
    """tau per window (1..4) and logits (flat windows: tau 4, logits 0)."""
    xn, flat = normalise(win)
    z, _ = mlp_forward(params, xn, bf16)
    z = np.where(flat[:, None], 0.0, z)
    tau = np.where(flat, 4, 1 + np.argmax(z, axis=1))
    return tau.astype(np.int8), z, flat


def classify_patch(params, e, gamma, bf16=False, lcut=(0, 0)):
    """Point-wise tau of one patch (min over covering windows) and window logits."""
    phi = proxy(e, gamma)
    win, cover = patch_windows(phi, lcut)
    tw, z, flat = classify_windows(params, win, bf16)
    tau = np.full(phi.shape, 4, dtype=np.int8)
    for t, (dirn, line, s) in zip(tw, cover):
        if dirn == 0:
            seg = tau[line, s:s + WINDOW]
        else:
            seg = tau[s:s + WINDOW, line]
        np.minimum(seg, t, out=seg)
    return tau, z, flat


def loss_and_grad(params, x, labels, bf16_weights=False):
    """Mean softmax cross-entropy and its gradient w.r.t. the flat parameters.

    With bf16_weights the forward pass uses bfloat16-rounded inputs and
    weights (hidden activations stay in full precision), as the training
    kernel does; the gradient is with respect to the unrounded weights
    (straight-through).
    """
    W1, b1, W2, b2, W3, b3 = unpack(params)
    r = bf16_round if bf16_weights else (lambda a: np.asarray(a, dtype=np.float64))
    W1r, W2r, W3r = r(W1), r(W2), r(W3)
    x = r(x)
    B = x.shape[0]
    z1 = x @ W1r.T + b1
    h1 = np.maximum(z1, 0)
    z2 = h1 @ W2r.T + b2
    h2 = np.maximum(z2, 0)
    z3 = h2 @ W3r.T + b3
    zmax = z3.max(axis=1, keepdims=True)
    ez = np.exp(z3 - zmax)
    P = ez / ez.sum(axis=1, keepdims=True)
    y = np.zeros_like(P)
    y[np.arange(B), np.asarray(labels, dtype=np.int64) - 1] = 1.0
    loss = float(np.mean(-np.log(P[np.arange(B), np.asarray(labels, dtype=np.int64) - 1])))
    dz3 = (P - y) / B
    gW3 = dz3.T @ h2
    gb3 = dz3.sum(0)
    dh2 = dz3 @ W3r
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dh1 = dz2 @ W2r
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad


class Adam:
    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, params, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return params - self.lr * mh / (np.sqrt(vh) + self.eps)


# ---------------------------------------------------------------- indicator
def decay_indicator(win):
    """Coefficient-decay smoothness estimate per window: (tau_hat, s)."""
    win = np.asarray(win, dtype=np.float64)
    y = fcgram.continue_lines(win, IND_D, IND_C)
    n = y.shape[-1]
    A = np.abs(np.fft.fft(y, axis=-1))[:, 1:n // 2]        # modes 1..20
    peak = A.max(axis=1, keepdims=True)
    amax = np.abs(win).max(axis=1)
    flat = (win.max(axis=1) - win.min(axis=1)) <= FLAT_TOL * np.maximum(1.0, amax)
    a = np.maximum(A, 1e-6 * peak)
    e_lo = np.sqrt(np.mean(a[:, 1:5] ** 2, axis=1))        # modes 2..5
    e_hi = np.sqrt(np.mean(a[:, 10:20] ** 2, axis=1))      # modes 11..20
    s = np.log(np.where(flat, 1.0, e_lo) / np.where(flat, 1.0, e_hi)) / np.log(15.5 / 3.5)
    tau = np.where(s < IND_CUTS[0], 1, np.where(s < IND_CUTS[1], 2, 4))
    tau = np.where(flat, 4, tau).astype(np.int8)
    s = np.where(flat, np.inf, s)
    return tau, s


# ---------------------------------------------------------------- viscosity
def _active(shape, lcut):
    m = np.ones(shape, dtype=bool)
    if lcut[0] > 0 and lcut[1] > 0:
        m[:lcut[1], :lcut[0]] = False
    return m


def mwsb(e, gamma, lcut=(0, 0)):
    """Max wave speed bound: max of |u| + c over the 3x3 neighbourhood (points
    of the patch only)."""
    rho, mx, my, _ = e
    act = _active(rho.shape, lcut)
    safe = np.where(act, 1.0, 0.0)
    rho_s = np.where(act, rho, 1.0)
    p = euler.pressure(np.stack([rho_s, mx * safe, my * safe, np.where(act, e[3], 2.5)]), gamma)
    s = np.where(act, np.sqrt(mx * mx + my * my) / rho_s + np.sqrt(gamma * p / rho_s), -np.inf)
    n2, n1 = s.shape
    pad = np.full((n2 + 2, n1 + 2), -np.inf)
    pad[1:-1, 1:-1] = s
    out = np.max([pad[1 + dj:n2 + 1 + dj, 1 + di:n1 + 1 + di] for dj in (-1, 0, 1) for di in (-1, 0, 1)], axis=0)
    return np.where(act, out, 0.0)


def _box_max(a, r, lcut=(0, 0)):
    """Maximum over a (2r+1) x (2r+1) box, taken separably (along the rows,
    then along the columns), each line restricted to its segment in the patch."""
    n2, n1 = a.shape
    if not (lcut[0] > 0 and lcut[1] > 0):    # rectangle: whole lines, shifted maxima
        tmp = a.copy()
        for k in range(1, r + 1):
            tmp[:, :n1 - k] = np.maximum(tmp[:, :n1 - k], a[:, k:])
            tmp[:, k:] = np.maximum(tmp[:, k:], a[:, :n1 - k])
        out = tmp.copy()
        for k in range(1, r + 1):
            out[:n2 - k, :] = np.maximum(out[:n2 - k, :], tmp[k:, :])
            out[k:, :] = np.maximum(out[k:, :], tmp[:n2 - k, :])
        return out
    tmp = np.zeros_like(a)
    for j in range(n2):
        s0, N = line_span(n1, n2, lcut, 0, j)
        row = a[j, s0:s0 + N]
        tmp[j, s0:s0 + N] = [row[max(0, t - r):t + r + 1].max() for t in range(N)]
    out = np.zeros_like(a)
    for i in range(n1):
        s0, N = line_span(n1, n2, lcut, 1, i)
        col = tmp[s0:s0 + N, i]
        out[s0:s0 + N, i] = [col[max(0, t - r):t + r + 1].max() for t in range(N)]
    return out


def bump_weights(r):
    t = np.arange(-r, r + 1) / (r + 1.0)
    return np.exp(1.0 - 1.0 / (1.0 - t * t))


def _bump_avg_line(v, r):
    """Normalised bump average along the last axis (one segment per line)."""
    b = bump_weights(r)
    n = v.shape[-1]
    num = np.zeros(v.shape)
    den = np.zeros(n)
    for k in range(-r, r + 1):
        lo, hi = max(0, -k), min(n, n - k)
        num[..., lo:hi] += b[k + r] * v[..., lo + k:hi + k]
        den[lo:hi] += b[k + r]
    return num / den


def _bump_avg(a, r, axis, lcut=(0, 0)):
    """Bump average along rows (axis 1) or columns (axis 0), segment by segment."""
    n2, n1 = a.shape
    if not (lcut[0] > 0 and lcut[1] > 0):    # rectangle: all lines at once
        return np.moveaxis(_bump_avg_line(np.moveaxis(a, axis, -1), r), -1, axis)
    out = np.zeros_like(a)
    if axis == 1:
        for j in range(n2):
            s0, N = line_span(n1, n2, lcut, 0, j)
            out[j, s0:s0 + N] = _bump_avg_line(a[j, s0:s0 + N], r)
    else:
        for i in range(n1):
            s0, N = line_span(n1, n2, lcut, 1, i)
            out[s0:s0 + N, i] = _bump_avg_line(a[s0:s0 + N, i], r)
    return out


def h_max(geom):
    """Largest physical grid spacing of a patch: the box spacings, or the
    largest distance between neighbouring nodes of the patch (curvilinear)."""
    if geom.patch.cartesian:
        return max(geom.hx, geom.hy)
    X, Y = geom.patch.coords()
    act = geom.active
    d1 = np.hypot(np.diff(X, axis=1), np.diff(Y, axis=1))[act[:, 1:] & act[:, :-1]]
    d2 = np.hypot(np.diff(X, axis=0), np.diff(Y, axis=0))[act[1:, :] & act[:-1, :]]
    return float(max(d1.max(), d2.max()))


def av_patch(e, tau, geom, gamma, n_f, c_mu=1.0, radius=4):
    """Smooth viscosity of one patch before the fringe exchange."""
    lc = tuple(geom.patch.lcut) if geom.patch.is_l else (0, 0)
    S = mwsb(e, gamma, lc)
    w = np.asarray(VISC_WEIGHT)[np.asarray(tau, dtype=np.int64) - 1]
    mu0 = c_mu * h_max(geom) * S * w
    mu0[euler.receiver_mask(geom.patch, n_f)] = 0.0
    mu0[~geom.active] = 0.0
    m = _box_max(mu0, radius, lc)
    return _bump_avg(_bump_avg(m, radius, 1, lc), radius, 0, lc)


def av_assemble(solver, state, taus, c_mu=1.0, radius=4):
    """Viscosity on every patch, fringe values from donors (Algorithm 3 + blend)."""
    mus = [av_patch(e, t, g, solver.inst.gamma, solver.n_f, c_mu, radius)
           for e, t, g in zip(state, taus, solver.geoms)]
    return euler.exchange(mus, solver.fmap, clamp=True)


# ---------------------------------------------------------------- initial smearing
SMEAR_P = 1   # order of the stronger filter used at t = 0 (reading of "somewhat more strongly filtered":
              # exp(-alpha (k/k_max)^2) spreads a jump over ~7 points without overshoot; orders >= 2 ring)


def smear_weight(tau, lcut=(0, 0), radius=4):
    """Smooth window near discontinuities: 1 where a point's tau is 1 (jump),
    spread by the box maximum and the normalised bump average of the viscosity
    blend (values in [0, 1])."""
    w0 = (np.asarray(tau) == 1).astype(np.float64)
    w0[~_active(w0.shape, lcut)] = 0.0
    return _bump_avg(_bump_avg(_box_max(w0, radius, lcut), radius, 1, lcut), radius, 0, lcut)


def smear_initial(solver, state, taus, p=SMEAR_P, radius=4):
    """Localized smearing of discontinuous initial data (§5 item 3, Algorithm 4
    at t = 0; reading of I-(33)): e' = (1 - w) e + w F_p(e), F_p the spectral
    filter of order p, w the smooth window near the points classified as jumps;
    then boundary conditions and the fringe exchange."""
    out = []
    for e, t, g in zip(state, taus, solver.geoms):
        lc = tuple(g.patch.lcut) if g.patch.is_l else (0, 0)
        w = smear_weight(t, lc, radius)
        f = euler.filter_state(e, g, solver.inst.gamma, p=p)
        out.append(np.where(g.active, (1.0 - w) * e + w * f, e))
    for e, g in zip(out, solver.geoms):
        euler.apply_bc(e, g, solver.inst)
    return euler.exchange(out, solver.fmap)
