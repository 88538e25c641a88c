"""FC-Gram Fourier continuation and FC spectral derivatives (oracle, FP64).

Test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module.

What the paper fixes (§2, FC-Gram paragraph): a line carries N values F_j at
x_j = j h, h = 1/(N-1), on [0, 1]; FC-Gram of degree d uses the d values at
each end of the line to build a Fourier expansion that is periodic on an
interval [0, β] strictly containing [0, 1]; derivatives are taken from that
expansion (Algorithm 5, FC-based differentiation).  The construction of the
continuation itself is in Part I (§I-2.2), which is not available, so this
module follows this reading of the FC(Gram) method of Bruno and Lyon:

  * the continued line has n = N + C points with period β = n h: the N data
    values followed by C continuation values;
  * Gram basis: the polynomials of degree < d that are orthonormal on the d
    matching points s = 0, ..., d-1 (index units), from the QR factorisation of
    the Vandermonde matrix there;
  * blend-to-zero: for each Gram polynomial p_k, the trigonometric polynomial
    T_k(s) = a_0 + sum_{m=1..K} a_m cos(2 pi m s / P) + b_m sin(2 pi m s / P),
    P = 2C + 4d - 1, K = floor((P - 9) / 3), minimising
      sum over S_match |T_k - p_k|^2 + sum over S_zero |T_k|^2 + lam^2 |coef|^2
    where S_match samples [0, d-1] and S_zero samples [d+C, 2d+C-1] with 20
    points per unit (oversampling), lam = 1e-14.  The continuation values are
    T_k(d + c), c = 0..C-1.  Because the fit is linear in its targets, the
    right-end table is A_R = T Q^T, acting on the last d data values;
  * left end by reflection: A_L[c][m] = A_R[C-1-c][d-1-m], acting on the first
    d data values; the appended values are A_R f_right + A_L f_left.

The fit is solved at 40 significant digits (mpmath) so that the FP64 tables
are correct to the last bit despite the ill-conditioning of Fourier
extension.

Continuation in the Gram form of FC(Gram): the d end values are projected
on the Gram basis (coefficients a = Q^T f_end) and the appended values are
sum_k T_k a_k for the right end plus the same for the reflected left end.
The projection cancels: for smooth data the high-degree coefficients are
small differences of values of size |f|, while their blend values T_k reach
~3e3 for d = 5, so an FP64 projection would leave rounding of ~1e-12 |f| in
the continuation.  The oracle therefore evaluates the projection in extended
precision (numpy longdouble: 64-bit significand on x86, IEEE binary128 on
Arm) with the 40-digit basis Q held as a double-double pair, rounds the
coefficients to FP64 once, and sums T a in FP64 (the terms T_k a_k are small
where T_k is large, so that sum keeps ~1 ulp of |f|).

Derivative: FFT of the continued line, multiply mode k by
(i 2 pi k / beta)^order, inverse FFT, keep the first N values.  For even n the
Nyquist mode is zeroed for odd orders and kept, times -(pi n/beta)^2, for the
second derivative (reading of a point the paper leaves open).
"""
import functools
import os

import mpmath as mp
import numpy as np

OVERSAMPLE = 20
LAMBDA = "1e-14"
DIGITS = 40


def policy_c(N, C):
    """Continuation length of an N-point line under the FFT-length policy.

    A choice of this implementation, not of the paper: the smallest
    C' >= max(C - 4, 20), C' <= 64, with N + C' = 32 n1 and 2 <= n1 <= 9 (an
    FFT held in registers of one warp); failing that the smallest C' in
    [C, C + 16] with N + C' a product of 2, 3, 5 and 7; failing that C.
    """
    for c in range(max(C - 4, 20), 65):
        if (N + c) % 32 == 0 and 2 <= (N + c) // 32 <= 9:
            return c
    for c in range(C, C + 17):
        m = N + c
        for q in (2, 3, 5, 7):
            while m % q == 0:
                m //= q
        if m == 1:
            return c
    return C


def fit_params(d, C):
    """Period P (index units) and highest mode K of the blend-to-zero fit."""
    P = 2 * C + 4 * d - 1
    K = (P - 9) // 3
    return P, K


@functools.lru_cache(maxsize=None)
def gram_basis(d):
    """Gram basis on the d matching points (FC-Gram, §2): returns (Q, Rinv).

    Q (d x d, orthonormal columns) holds the values of the Gram polynomials at
    s = 0..d-1; p_k(s) = sum_j (s/(d-1))^j Rinv[j, k] evaluates them anywhere.
    """
    if d < 2:
        raise ValueError("FC-Gram needs d >= 2")
    with mp.workdps(DIGITS):
        V = mp.matrix(d, d)
        for i in range(d):
            for j in range(d):
                V[i, j] = (mp.mpf(i) / (d - 1)) ** j
        Q, R = mp.qr(V)
        Rinv = R ** -1
    return Q, Rinv


def _gram_poly(Rinv, d, k, s):
    return mp.fsum((s / (d - 1)) ** j * Rinv[j, k] for j in range(d))


@functools.lru_cache(maxsize=None)
def blend_fit(d, C):
    """Blend-to-zero fit of every Gram polynomial (FC-Gram, §2).

    Returns (T, resid): T[c, k] = T_k(d + c) as mpmath numbers (C x d) and the
    largest fit residual on the matching and zero regions (a float).
    """
    P, K = fit_params(d, C)
    with mp.workdps(DIGITS):
        Q, Rinv = gram_basis(d)
        lam = mp.mpf(LAMBDA)
        s_match = [mp.mpf(i) / OVERSAMPLE for i in range((d - 1) * OVERSAMPLE + 1)]
        s_zero = [mp.mpf(d + C) + mp.mpf(i) / OVERSAMPLE for i in range((d - 1) * OVERSAMPLE + 1)]
        pts = s_match + s_zero
        ncol = 2 * K + 1
        two_pi_over_P = 2 * mp.pi / P

        def basis_row(s):
            row = [mp.mpf(1)]
            for m in range(1, K + 1):
                w = two_pi_over_P * m * s
                row += [mp.cos(w), mp.sin(w)]
            return row

        A = mp.matrix(len(pts) + ncol, ncol)
        for r, s in enumerate(pts):
            for c, v in enumerate(basis_row(s)):
                A[r, c] = v
        for c in range(ncol):
            A[len(pts) + c, c] = lam
        gap_rows = [basis_row(mp.mpf(d + c)) for c in range(C)]
        T = mp.matrix(C, d)
        resid = 0.0
        for k in range(d):
            b = mp.matrix(len(pts) + ncol, 1)
            for r, s in enumerate(s_match):
                b[r] = _gram_poly(Rinv, d, k, s)
            coef, _ = mp.qr_solve(A, b)
            for r in range(len(pts)):
                fit = mp.fsum(A[r, c] * coef[c] for c in range(ncol))
                resid = max(resid, float(abs(fit - b[r])))
            for c in range(C):
                T[c, k] = mp.fsum(gap_rows[c][j] * coef[j] for j in range(ncol))
    return T, resid


_STORE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fcgram_tables.npz")


@functools.lru_cache(maxsize=None)
def _stored():
    return dict(np.load(_STORE)) if os.path.exists(_STORE) else {}


@functools.lru_cache(maxsize=None)
def continuation_tables(d, C, use_store=True):
    """FP64 continuation tables (A_R, A_L), each C x d (FC-Gram, §2).

    With use_store the tables written by oracle/make_tables.py (this very
    function, run once) are read instead of redoing the 40-digit fit.
    """
    key = f"d{d}_C{C}"
    if use_store and key in _stored():
        A_R = _stored()[key].copy()
    else:
        T, _ = blend_fit(d, C)
        Q, _ = gram_basis(d)
        with mp.workdps(DIGITS):
            AR = T * Q.T
        A_R = np.array([[float(AR[c, m]) for m in range(d)] for c in range(C)], dtype=np.float64)
    A_L = A_R[::-1, ::-1].copy()
    return A_R, A_L


@functools.lru_cache(maxsize=None)
def gram_tables(d, C, use_store=True):
    """Gram form of the continuation (FC-Gram, §2): (Q_hi, Q_lo, T).

    Q = Q_hi + Q_lo (d x d, double-double of the 40-digit Gram basis: column
    k holds p_k at the matching points s = 0..d-1); T (C x d, FP64): T[c, k]
    = blend-to-zero continuation of p_k at s = d + c.  A_R = T Q^T.
    """
    Q, _ = gram_basis(d)
    with mp.workdps(DIGITS):
        Qhi = np.array([[float(Q[i, k]) for k in range(d)] for i in range(d)], dtype=np.float64)
        Qlo = np.array([[float(Q[i, k] - mp.mpf(Qhi[i, k])) for k in range(d)] for i in range(d)],
                       dtype=np.float64)
    key = f"T_d{d}_C{C}"
    if use_store and key in _stored():
        T = _stored()[key].copy()
    else:
        Tm, _ = blend_fit(d, C)
        T = np.array([[float(Tm[c, k]) for k in range(d)] for c in range(C)], dtype=np.float64)
    return Qhi, Qlo, T


def gram_coefficients(f_end, d):
    """a = Q^T f_end over the last axis (d values at s = 0..d-1), evaluated
    in extended precision with the double-double basis, rounded to FP64."""
    Qhi, Qlo, _ = gram_tables(d, 2 * d)
    Qx = Qhi.astype(np.longdouble) + Qlo.astype(np.longdouble)
    return (np.asarray(f_end, dtype=np.longdouble) @ Qx).astype(np.float64)


def continue_lines(f, d, C):
    """Append the C FC-Gram continuation values to each line (last axis).

    Right end: the Gram coefficients of the last d values (s = m at point
    N-d+m) continued by T; left end by reflection: the first d values read
    backwards (s = m at point d-1-m), continued by T read backwards.
    """
    f = np.asarray(f, dtype=np.float64)
    _, _, T = gram_tables(d, C)
    a_right = gram_coefficients(f[..., -d:], d)
    a_left = gram_coefficients(f[..., d - 1::-1], d)
    ext = a_right @ T.T + a_left @ T[::-1].T
    return np.concatenate([f, ext], axis=-1)


def spectral_multiplier(n, h, order):
    """(i k)^order for the n-point period beta = n h, k = 2 pi j / beta."""
    j = np.fft.fftfreq(n, d=1.0 / n)
    k = 2.0 * np.pi * j / (n * h)
    mult = (1j * k) ** order
    if n % 2 == 0 and order % 2 == 1:
        mult[n // 2] = 0.0
    return mult


def fc_derivative(f, h, d, C, order=1, extended=False):
    """FC derivative of every line of f along the last axis (Algorithm 5).

    f: (..., N) samples at spacing h (parameter space); returns (..., N), or
    with extended=True the derivative of the continued line at all n = N + C
    points of its period (the first N are the derivative values).
    """
    f = np.asarray(f, dtype=np.float64)
    N = f.shape[-1]
    y = continue_lines(f, d, C)
    n = y.shape[-1]
    Y = np.fft.fft(y, axis=-1)
    dy = np.fft.ifft(Y * spectral_multiplier(n, h, order), axis=-1).real
    return dy if extended else dy[..., :N]


def fc_derivative_axis(f, h, d, C, axis, order=1):
    """FC derivative along an arbitrary axis."""
    g = np.moveaxis(np.asarray(f, dtype=np.float64), axis, -1)
    return np.moveaxis(fc_derivative(g, h, d, C, order), -1, axis)


# spectral filter (§5 item 3, Algorithm 4; reading of I-(32)):
# sigma(k) = exp(-alpha (|k| / k_max)^(2p)), k the mode number in
# (-n/2, n/2], k_max = n/2
FILTER_ALPHA = 16.0 * np.log(10.0)
FILTER_P = 18


def filter_factors(n, alpha=FILTER_ALPHA, p=FILTER_P):
    """sigma(k) for the n FFT modes in numpy order."""
    k = np.abs(np.fft.fftfreq(n, d=1.0 / n))
    return np.exp(-alpha * (k / (n / 2.0)) ** (2 * p))


def filter_periodic(y, alpha=FILTER_ALPHA, p=FILTER_P):
    """Filter of periodic lines y (..., n): Fourier coefficients times sigma."""
    y = np.asarray(y, dtype=np.float64)
    return np.real(np.fft.ifft(np.fft.fft(y, axis=-1) * filter_factors(y.shape[-1], alpha, p), axis=-1))


def fc_filter(f, d, C, alpha=FILTER_ALPHA, p=FILTER_P):
    """Spectral filter of every line of f along the last axis: continue, filter
    the periodic extension, restrict to the N data points."""
    f = np.asarray(f, dtype=np.float64)
    return filter_periodic(continue_lines(f, d, C), alpha, p)[..., :f.shape[-1]]


def naive_dft(y, sign=-1):
    """O(n^2) DFT, sum_j y_j exp(sign 2 pi i j k / n); pins the FFT use."""
    y = np.asarray(y)
    n = y.shape[-1]
    jk = np.outer(np.arange(n), np.arange(n))
    W = np.exp(sign * 2j * np.pi * jk / n)
    return y @ W


def spectral_integral_weights(n, h, N):
    """I_j = integral over [0, (N-1) h] of exp(2 pi i k_j x / beta), beta = n h.

    The Nyquist mode (even n) is the real cosine cos(pi x / h), whose integral
    over [0, (N-1) h] vanishes.
    """
    j = np.fft.fftfreq(n, d=1.0 / n)
    beta = n * h
    L = (N - 1) * h
    I = np.empty(n, dtype=np.complex128)
    for idx, jj in enumerate(j):
        if jj == 0:
            I[idx] = L
        else:
            w = 2j * np.pi * jj / beta
            I[idx] = (np.exp(w * L) - 1.0) / w
    if n % 2 == 0:
        I[n // 2] = 0.0
    return I


def fc_quadrature_weights(N, d, C):
    """Weights W (N,) with W.f = integral over [0, 1] of the FC expansion of f."""
    n = N + C
    h = 1.0 / (N - 1)
    I = spectral_integral_weights(n, h, N)
    # integral = (1/n) sum_k Y_k I_k,  Y_k = sum_j y_j e^{-2 pi i j k/n}
    jk = np.outer(np.arange(n), np.fft.fftfreq(n, d=1.0 / n))
    w = (np.exp(-2j * np.pi * jk / n) @ I).real / n
    A_R, A_L = continuation_tables(d, C)
    W = w[:N].copy()
    W[N - d:] += A_R.T @ w[N:]
    W[:d] += A_L.T @ w[N:]
    return W
