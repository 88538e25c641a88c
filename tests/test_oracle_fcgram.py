"""Pins of the oracle's FC-Gram continuation and FC derivative (paper §2)."""
import mpmath as mp
import numpy as np
import pytest

from oracle import fcgram


@pytest.mark.parametrize("d", [2, 5])
def test_gram_basis_orthonormal_and_consistent(d):
    Q, Rinv = fcgram.gram_basis(d)
    q = np.array(Q.tolist(), dtype=float)
    assert np.allclose(q.T @ q, np.eye(d), atol=1e-15)
    # the polynomial form reproduces the tabulated values at the matching points
    with mp.workdps(40):
        for k in range(d):
            for m in range(d):
                v = fcgram._gram_poly(Rinv, d, k, mp.mpf(m))
                assert abs(v - Q[m, k]) < mp.mpf("1e-35")
    # p_k has degree k: its k-th finite difference is nonzero, (k+1)-th vanishes
    with mp.workdps(40):
        for k in range(d):
            vals = [fcgram._gram_poly(Rinv, d, k, mp.mpf(s) / 3) for s in range(3 * d)]
            diffs = vals
            for _ in range(k):
                diffs = [b - a for a, b in zip(diffs, diffs[1:])]
            assert min(abs(float(x)) for x in diffs) > 1e-6
            diffs = [b - a for a, b in zip(diffs, diffs[1:])]
            assert max(abs(float(x)) for x in diffs) < 1e-25


@pytest.mark.parametrize("d,C", [(5, 25), (2, 25), (5, 26)])
def test_blend_fit_matches_and_vanishes(d, C):
    # the blend-to-zero reproduces each Gram polynomial on the matching region
    # and vanishes on the zero region to far below FP64 derivative accuracy
    _, resid = fcgram.blend_fit(d, C)
    assert resid < 2e-12


def test_fft_matches_naive_dft():
    rng = np.random.default_rng(0)
    f = np.sin(np.linspace(0, 2, 101)) + 0.1 * rng.standard_normal(101)
    y = fcgram.continue_lines(f, 5, 25)
    Y = np.fft.fft(y)
    assert np.abs(Y - fcgram.naive_dft(y)).max() < 1e-13 * np.abs(Y).max() * y.size


def _errors(fn, dfn, Ns, d, C, order=1):
    errs = []
    for N in Ns:
        x = np.linspace(0.0, 1.0, N)
        errs.append(np.abs(fcgram.fc_derivative(fn(x), 1.0 / (N - 1), d, C, order) - dfn(x)).max())
    return np.array(errs)


@pytest.mark.parametrize("fn,dfn", [
    (lambda x: np.sin(3 * x + 1), lambda x: 3 * np.cos(3 * x + 1)),
    (lambda x: np.exp(x) * np.cos(5 * x), lambda x: np.exp(x) * (np.cos(5 * x) - 5 * np.sin(5 * x))),
])
def test_first_derivative_converges_at_fc_gram_order(fn, dfn):
    # FC-Gram of degree d: observed order >= d - 1 (d = 5)
    Ns = [25, 50, 100, 200]
    e = _errors(fn, dfn, Ns, 5, 25)
    order = np.log2(e[:-1] / e[1:])
    assert e[-1] < 2e-6
    assert np.all(order > 3.5), order


def test_second_derivative_converges():
    fn = lambda x: np.sin(3 * x + 1)
    d2 = lambda x: -9 * np.sin(3 * x + 1)
    e = _errors(fn, d2, [50, 100, 200], 5, 25, order=2)
    assert np.all(np.log2(e[:-1] / e[1:]) > 2.5), e


def test_low_degree_polynomial_derivative():
    # polynomials of degree < d are continued smoothly: derivative close to exact
    N = 101
    x = np.linspace(0, 1, N)
    f = 1 + 2 * x - 3 * x ** 2 + 0.5 * x ** 3 - x ** 4
    df = 2 - 6 * x + 1.5 * x ** 2 - 4 * x ** 3
    err = np.abs(fcgram.fc_derivative(f, 1 / (N - 1), 5, 25) - df).max()
    assert err < 1e-7


@pytest.mark.parametrize("N", [101, 57])
def test_spectral_integral_identity(N):
    # integral over [0,1] of the derivative of the FC expansion = f(1) - f(0):
    # pins the wavenumber scaling (period beta = n h) and that the expansion
    # interpolates the data; exact up to rounding for odd N
    rng = np.random.default_rng(N)
    x = np.linspace(0, 1, N)
    f = np.sin(2.3 * x + rng.uniform()) + 0.3 * x ** 2
    h = 1 / (N - 1)
    y = fcgram.continue_lines(f, 5, 25)
    n = y.size
    Y = np.fft.fft(y)
    I = fcgram.spectral_integral_weights(n, h, N)
    integral = np.sum(Y * fcgram.spectral_multiplier(n, h, 1) * I).real / n
    assert abs(integral - (f[-1] - f[0])) < 1e-12


def test_quadrature_weights():
    N = 101
    W = fcgram.fc_quadrature_weights(N, 5, 25)
    assert abs(W.sum() - 1.0) < 1e-12
    x = np.linspace(0, 1, N)
    exact = (np.cos(1.0) - np.cos(4.0)) / 3.0
    assert abs(W @ np.sin(3 * x + 1) - exact) < 1e-9


def test_tables_reflection():
    A_R, A_L = fcgram.continuation_tables(5, 25)
    assert A_R.shape == (25, 5)
    assert np.array_equal(A_L, A_R[::-1, ::-1])
    # a constant line: the continuation is mirror-symmetric and the FC
    # derivative on the data points vanishes up to the fit residual
    c = fcgram.continue_lines(np.full(40, 3.0), 5, 25)
    assert np.abs(c[40:] - c[40:][::-1]).max() < 5e-12
    assert np.abs(fcgram.fc_derivative(np.full(40, 3.0), 1 / 39, 5, 25)).max() < 5e-9


def test_stored_tables_match_fresh_fits():
    # the stored tables (oracle/make_tables.py) are this module's own fits
    for C in (20, 25, 33):
        stored, _ = fcgram.continuation_tables(5, C)
        fresh, _ = fcgram.continuation_tables(5, C, use_store=False)
        assert np.array_equal(stored, fresh)
        assert np.array_equal(fcgram.gram_tables(5, C)[2], fcgram.gram_tables(5, C, use_store=False)[2])


@pytest.mark.parametrize("d,C", [(5, 25), (2, 25)])
def test_continuation_matches_exact_40_digit_evaluation(d, C):
    # FC-Gram (§2): the appended values are A_R f_right + A_L f_left with
    # A_R = T Q^T.  Evaluated exactly (40 digits, the fit's own T and Q) on
    # smooth lines, lines offset by a large constant and a rough line, the
    # oracle's continuation is correct to a few ulps of the line's values;
    # a plain FP64 sum with the combined table (entries ~2e3) is not
    T_mp, _ = fcgram.blend_fit(d, C)
    Q_mp, _ = fcgram.gram_basis(d)
    rng = np.random.default_rng(11)
    N = 64
    x = np.linspace(0, 1, N)
    lines = [np.sin(3 * x + 1), 116.0 + 0.01 * np.cos(2 * x), np.exp(x) * np.cos(5 * x),
             rng.standard_normal(N)]
    A_R, A_L = fcgram.continuation_tables(d, C)
    worst_plain = 0.0
    for f in lines:
        got = fcgram.continue_lines(f, d, C)[N:]
        with mp.workdps(40):
            AR = T_mp * Q_mp.T
            exact = [mp.fsum(AR[c, m] * mp.mpf(f[N - d + m]) + AR[C - 1 - c, m] * mp.mpf(f[d - 1 - m])
                             for m in range(d)) for c in range(C)]
        ex = np.array([float(v) for v in exact])
        scale = np.abs(f).max()
        assert np.abs(got - ex).max() <= 8 * 2.0 ** -53 * max(scale, np.abs(ex).max()), f[:3]
        plain = f[-d:] @ A_R.T + f[:d] @ A_L.T
        worst_plain = max(worst_plain, np.abs(plain - ex).max() / scale)
    if d == 5:
        assert worst_plain > 1e-15   # the cancellation the Gram form avoids is real


def test_filter_factors_on_single_modes():
    # sigma(k) = exp(-16 ln 10 (|k| / (n/2))^36) multiplies mode k and -k alike
    n = 64
    j = np.arange(n)
    for k0 in (0, 3, 16, 28, 31, 32):
        y = np.cos(2 * np.pi * k0 * j / n + (0.3 if k0 not in (0, 32) else 0.0))
        sig = np.exp(-16 * np.log(10) * (k0 / 32) ** 36)
        assert np.allclose(fcgram.filter_periodic(y), sig * y, atol=1e-14)
    assert fcgram.filter_factors(n)[32] < 1.01e-16          # Nyquist: exp(-alpha) = 1e-16
    assert abs(fcgram.filter_factors(n)[16] - 1.0) < 1e-9   # half the band is untouched


def test_fc_filter_keeps_smooth_data_and_damps_grid_noise():
    N = 101
    x = np.linspace(0.0, 1.0, N)
    f = np.exp(x) * np.sin(3 * x + 0.2)
    g = fcgram.fc_filter(f, 5, 25)
    assert np.abs(g - f).max() < 1e-9
    noise = 1e-2 * (-1.0) ** np.arange(N)
    r = fcgram.fc_filter(f + noise, 5, 25) - f
    assert np.abs(r[10:-10]).max() < 0.2 * np.abs(noise).max()
