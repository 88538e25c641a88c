"""Pins of the oracle's proxy, windows, classifier MLP, indicator and viscosity."""
import numpy as np
import pytest

from oracle import euler, sdnn
from paper_2506_19370_gb300 import inputs as I

G = 1.4


def test_proxy_is_mach_number():
    # (1.4, M, 0, 1) has sound speed 1, so Phi = M (§7 Mach-M flow)
    e = I.conserved(*I.mach_flow_state(3.0)).reshape(4, 1, 1) * np.ones((4, 3, 5))
    assert np.allclose(sdnn.proxy(e, G), 3.0, rtol=1e-14)


def test_window_cover():
    assert sdnn.window_starts(40) == [0, 16, 24]
    assert sdnn.window_starts(160) == list(range(0, 160, 16))
    assert sdnn.window_starts(101) == [0, 16, 32, 48, 64, 80, 85]
    phi = np.random.default_rng(0).standard_normal((40, 101))
    win, cover = sdnn.patch_windows(phi)
    assert win.shape == (40 * 7 + 101 * 3, 16)
    d, line, s = cover[40 * 7 + 5]
    assert d == 1 and np.array_equal(win[40 * 7 + 5], phi[s:s + 16, line])


def test_bf16_rounding_against_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).integers(-8, 8, 10000)
    x = np.concatenate([x, [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(sdnn.bf16_round(x), ref)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = sdnn.init_params(3) + 0.01 * rng.standard_normal(sdnn.N_PARAMS)
    x = rng.standard_normal((64, 16))
    y = rng.integers(1, 5, 64)
    _, g = sdnn.loss_and_grad(params, x, y)
    idx = rng.choice(sdnn.N_PARAMS, 60, replace=False)
    for k in idx:
        h = 1e-6
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        fd = (sdnn.loss_and_grad(pp, x, y)[0] - sdnn.loss_and_grad(pm, x, y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])) + 1e-9


def test_adam_first_step():
    opt = sdnn.Adam(5, lr=1e-3)
    g = np.array([0.5, -2.0, 1e-3, -1e-5, 3.0])
    p = opt.step(np.zeros(5), g)
    assert np.allclose(p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_training_learns_the_classes():
    x, y = I.classifier_windows(4096, seed=11)
    xn, _ = sdnn.normalise(x)
    params = sdnn.init_params(0)
    opt = sdnn.Adam(sdnn.N_PARAMS, lr=3e-3)
    l0, _ = sdnn.loss_and_grad(params, xn, y)
    for _ in range(300):
        _, g = sdnn.loss_and_grad(params, xn, y)
        params = opt.step(params, g)
    l1, _ = sdnn.loss_and_grad(params, xn, y)
    tau, _, _ = sdnn.classify_windows(params, x)
    assert l1 < 0.6 * l0 and np.mean(tau == y) > 0.6


def test_indicator_on_clean_profiles():
    x = np.arange(16.0)
    wins = np.array([np.where(x > 7.3, 1.0, 0.0),          # jump
                     np.abs(x - 7.3) / 4,                   # kink
                     np.sin(0.2 * x) + 0.1 * x,              # smooth
                     np.full(16, 2.0)])                      # flat
    tau, s = sdnn.decay_indicator(wins)
    assert list(tau) == [1, 2, 4, 4]
    assert s[0] < s[1] < s[2]


def test_viscosity_closed_forms():
    p = I.Patch(30, 20, (I.BC_WALL,) * 4, box=(0.0, 1.0, 0.0, 0.5))
    g = euler.PatchGeom(p, 5, 25)
    e = I.conserved(np.full((20, 30), 1.4), 2.0, 0.0, 1.0)
    # MWSB of a uniform state: |u| + c
    assert np.allclose(sdnn.mwsb(e, G), 3.0)
    # smooth everywhere -> no viscosity
    assert np.all(sdnn.av_patch(e, np.full((20, 30), 4), g, G, 5) == 0)
    # all "jump" -> uniform c_mu h_max S (bump average of a constant is that constant)
    mu = sdnn.av_patch(e, np.full((20, 30), 1), g, G, 5, c_mu=0.7)
    assert np.allclose(mu, 0.7 * (1.0 / 29) * 3.0, rtol=1e-14)
    # a single flagged point spreads to a smooth, local bump of radius 2r
    tau = np.full((20, 30), 4)
    tau[10, 15] = 1
    mu = sdnn.av_patch(e, tau, g, G, 5, radius=3)
    assert mu[10, 15] > 0 and mu[10, 22] == 0 and mu[10, 21] > 0 and mu[3, 15] == 0
    assert np.allclose(mu, mu[::-1, :][::-1, :])


def test_classify_patch_min_over_windows():
    params = sdnn.init_params(0)
    inst = I.sod_instance(npatch=1, n1=40, n2=20)
    e = inst.state[0].copy()
    e[1] = 0.3 * e[0] * np.sin(np.arange(40) / 5.0)[None, :]
    tau, z, flat = sdnn.classify_patch(params, e, G)
    win, cover = sdnn.patch_windows(sdnn.proxy(e, G))
    tw, _, _ = sdnn.classify_windows(params, win)
    for (dirn, line, s), t in zip(cover, tw):
        seg = tau[line, s:s + 16] if dirn == 0 else tau[s:s + 16, line]
        assert np.all(seg <= t)


def test_l_patch_windows_and_viscosity():
    from oracle import euler
    n1, n2, m1, m2 = 60, 52, 24, 20
    p = I.Patch(n1, n2, (I.BC_WALL,) * 4, box=(0.0, 1.18, 0.0, 1.02), lcut=(m1, m2))
    act = p.active()
    phi = np.random.default_rng(2).uniform(size=(n2, n1))
    win, cover = sdnn.patch_windows(phi, (m1, m2))
    hits = [np.zeros((n2, n1), int), np.zeros((n2, n1), int)]
    for dirn, line, s in cover:
        if dirn == 0:
            hits[0][line, s:s + 16] += 1
        else:
            hits[1][s:s + 16, line] += 1
    for h in hits:
        assert np.all(h[act] >= 1) and np.all(h[~act] == 0)   # windows tile the segments only
    # constant wave speed and tau = 1 everywhere: mu = c_mu h S on every point
    e = I.conserved(np.full((n2, n1), 1.4), 0.0, 0.0, 1.0)            # c = 1
    g = euler.PatchGeom(p, 5, 25)
    mu = sdnn.av_patch(e, np.ones((n2, n1), dtype=np.int8), g, G, 5, c_mu=0.7)
    assert np.allclose(mu[act], 0.7 * 0.02 * 1.0, rtol=1e-13) and np.all(mu[~act] == 0.0)


def test_initial_smearing_is_local_and_smooths_jumps():
    from oracle import euler
    inst = I.sod_instance()                         # sharp Sod jump at x = 0.5
    solver = euler.Solver(inst, c_policy=1)
    flat = [np.full((p.n2, p.n1), 4, dtype=np.int8) for p in inst.patches]
    same = sdnn.smear_initial(solver, [e.copy() for e in inst.state], flat)
    assert all(np.array_equal(a, b) for a, b in zip(same, inst.state))     # no jump flagged: unchanged
    taus = []
    for p in inst.patches:
        X, _ = p.coords()
        taus.append(np.where(np.abs(X - 0.5) < 0.004, 1, 4).astype(np.int8))
    w = sdnn.smear_weight(taus[3])
    assert w.min() >= 0.0 and w.max() <= 1.0 + 1e-15 and w.max() > 0.99
    out = sdnn.smear_initial(solver, [e.copy() for e in inst.state], taus)
    for a, b, p in zip(out, inst.state, inst.patches):
        X, _ = p.coords()
        far = np.abs(X - 0.5) > 0.05
        assert np.array_equal(a[:, far], b[:, far])                        # local
    jump = lambda st: max(float(np.abs(np.diff(e[0], axis=1)).max()) for e in st)
    assert jump(out) < 0.2 * jump(inst.state)                              # the jump is spread
    assert min(float(e[0].min()) for e in out) > 0.125 - 1e-3               # without overshoot
    assert max(float(e[0].max()) for e in out) < 1.0 + 1e-3
