"""Pins of the oracle's Euler operator, boundary conditions, RK4, exchange, Δt."""
import numpy as np
import pytest

from oracle import euler, fcgram
from paper_2506_19370_gb300 import inputs as I

G = 1.4


def test_fluxes_closed_form():
    # rho=2, u=3, v=-1, p=5  ->  E = 5/0.4 + 0.5*2*10 = 22.5  (Eq. 1-2)
    e = I.conserved(2.0, 3.0, -1.0, 5.0).reshape(4, 1, 1)
    assert np.isclose(e[3, 0, 0], 22.5)
    f, g = euler.fluxes(e, G)
    assert np.allclose(f[:, 0, 0], [6.0, 23.0, -6.0, 82.5])
    assert np.allclose(g[:, 0, 0], [-2.0, -6.0, 7.0, -27.5])
    assert np.isclose(euler.pressure(e, G)[0, 0], 5.0)


def test_free_stream_cartesian():
    p = I.Patch(40, 33, (I.BC_FREE,) * 4, box=(0.0, 2.0, -1.0, 0.5))
    g = euler.PatchGeom(p, 5, 25)
    e = I.conserved(np.full((33, 40), 1.4), 3.0, -1.0, 1.0)
    assert np.abs(euler.rhs(e, g, 5, 25, G)).max() < 1e-8


def test_free_stream_curvilinear():
    # the metrics come from the same FC derivative, and FC derivatives along q1
    # and q2 commute on the tensor grid, so uniform flow stays uniform
    p = I.annulus_patch()
    g = euler.PatchGeom(p, 5, 25)
    e = I.conserved(np.full((p.n2, p.n1), 1.4), 3.0, -1.0, 1.0)
    L = euler.rhs(e, g, 5, 25, G)
    assert np.abs(L).max() < 1e-6
    # a perturbed state is not preserved (the check above is not vacuous)
    X, Y = p.coords()
    e2 = I.conserved(1.4 + 0.1 * np.sin(3 * X), 3.0, -1.0, 1.0)
    assert np.abs(euler.rhs(e2, g, 5, 25, G)).max() > 1e-2


def test_curvilinear_matches_cartesian_on_affine_map():
    # an affine map given as coordinates reproduces the Cartesian operator
    box = (0.2, 1.3, -0.4, 0.6)
    pc = I.Patch(48, 40, (I.BC_FREE,) * 4, box=box)
    X, Y = pc.coords()
    pg = I.Patch(48, 40, (I.BC_FREE,) * 4, x=X, y=Y)
    rng = np.random.default_rng(3)
    e = I.random_state(pc, rng)
    a = euler.rhs(e, euler.PatchGeom(pc, 5, 25), 5, 25, G)
    b = euler.rhs(e, euler.PatchGeom(pg, 5, 25), 5, 25, G)
    assert np.abs(a - b).max() < 1e-6 * np.abs(a).max()


def test_curvilinear_viscous_matches_cartesian_on_affine_map():
    box = (0.2, 1.3, -0.4, 0.6)
    pc = I.Patch(48, 40, (I.BC_WALL, I.BC_FREE, I.BC_INTERNAL, I.BC_OUTFLOW), box=box)
    X, Y = pc.coords()
    pg = I.Patch(48, 40, pc.bc, x=X, y=Y)
    e = I.random_state(pc, np.random.default_rng(4))
    mu = 0.01 * (1.0 + np.sin(3 * X) * np.cos(2 * Y))
    a = euler.rhs(e, euler.PatchGeom(pc, 5, 25), 5, 25, G, mu)
    b = euler.rhs(e, euler.PatchGeom(pg, 5, 25), 5, 25, G, mu)
    assert np.abs(a - b).max() < 1e-6 * np.abs(a).max()


def test_curvilinear_viscous_term_is_div_mu_grad():
    # at rest (u = v = 0) the density equation reduces to d_t rho =
    # div(mu grad rho): on an annulus patch (rotating, stretching metrics)
    # the operator must converge to the analytic value
    def rho(x, y):
        return 1.0 + 0.2 * np.sin(2 * x + 0.5) * np.cos(3 * y)

    def lap_term(x, y):
        # mu = 1 + 0.5 x y; div(mu grad rho) = mu lap(rho) + grad(mu) . grad(rho)
        s, c = np.sin(2 * x + 0.5), np.cos(3 * y)
        rx, ry = 0.4 * np.cos(2 * x + 0.5) * c, -0.6 * s * np.sin(3 * y)
        lap = -0.2 * 13.0 * s * c
        return (1.0 + 0.5 * x * y) * lap + 0.5 * y * rx + 0.5 * x * ry

    errs = []
    for n in (48, 96):
        p = I.annulus_patch(n, n * 5 // 6, bc=(I.BC_INTERNAL,) * 4)
        X, Y = p.coords()
        e = I.conserved(rho(X, Y), 0.0, 0.0, 1.0)
        mu = 1.0 + 0.5 * X * Y
        L = euler.rhs(e, euler.PatchGeom(p, 5, 25), 5, 25, G, mu)
        ref = lap_term(X, Y)
        errs.append(np.abs(L[0] - ref).max() / np.abs(ref).max())
    assert errs[0] < 1e-3 and errs[1] < errs[0] / 6   # second derivatives: order d - 2 = 3


def test_vortex_is_steady_in_moving_frame():
    # the isentropic vortex solves Euler exactly with d_t e = -u0 d_x e; the
    # operator residual converges to zero under refinement (a sign or term
    # error in the fluxes leaves an O(1) residual)
    res = []
    for n in (101, 201):
        inst = I.vortex_instance(n)
        g = euler.PatchGeom(inst.patches[0], 5, 25)
        e = inst.state[0]
        L = euler.rhs(e, g, 5, 25, G)
        dedx = fcgram.fc_derivative_axis(e, g.hx, 5, 25, axis=2)
        res.append(np.abs(L + dedx).max() / np.abs(L).max())
    assert res[0] < 1e-7 and res[1] < res[0] / 20


def test_rk4_amplification_factor():
    # with L(e) = lam e the four stages give the degree-4 Taylor polynomial
    inst = I.Instance([I.Patch(20, 20, (I.BC_FREE,) * 4, box=(0, 1, 0, 1))],
                      [np.ones((4, 20, 20))])
    s = euler.Solver(inst)
    lam = -0.7
    s.rhs_all = lambda st, mu=None: [lam * e for e in st]
    dt = 0.3
    out = s.step([np.ones((4, 20, 20))], dt)
    z = lam * dt
    assert np.allclose(out[0], 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24, rtol=1e-15, atol=0)


def test_boundary_conditions():
    inst = I.vortex_instance(21)
    s = euler.Solver(inst)
    e = I.random_state(inst.patches[0], np.random.default_rng(1))
    euler.apply_bc(e, s.geoms[0], inst)
    assert np.allclose(e[:, :, 0], np.array(inst.inflow)[:, None])          # inflow left
    p_right = euler.pressure(e[:, :, -1], G)
    assert np.allclose(p_right[1:-1], inst.p_out)                           # outflow right
    assert np.all(e[2, 0, :] == 0) and np.all(e[2, -1, :] == 0)             # walls


def test_sod_fringe_map():
    inst = I.sod_instance()
    fmap = euler.fringe_map(inst.patches, 5)
    # two fringes of 5 columns per internal interface, 40 rows each
    assert len(fmap) == 7 * 2 * 5 * 40 and not fmap.interp   # coincident grids: copies only
    masks = [euler.receiver_mask(p, 5) for p in inst.patches]
    for p, j, i, q, jj, ii in fmap.copies:
        assert masks[p][j, i] and not masks[q][jj, ii]       # donors are never receivers
        Xp, Yp = inst.patches[p].coords()
        Xq, Yq = inst.patches[q].coords()
        assert abs(Xp[j, i] - Xq[jj, ii]) < 1e-12 and abs(Yp[j, i] - Yq[jj, ii]) < 1e-12


def test_split_patch_exchange_is_exact():
    # one patch split in two overlapping patches: after the exchange every
    # fringe value equals the single-patch value at the same point (bitwise)
    whole = I.Patch(60, 20, (I.BC_WALL,) * 4, box=(0.0, 59.0, 0.0, 19.0))
    a = I.Patch(35, 20, (I.BC_WALL, I.BC_INTERNAL, I.BC_WALL, I.BC_WALL), box=(0.0, 34.0, 0.0, 19.0))
    b = I.Patch(35, 20, (I.BC_INTERNAL, I.BC_WALL, I.BC_WALL, I.BC_WALL), box=(25.0, 59.0, 0.0, 19.0))
    ew = I.random_state(whole, np.random.default_rng(5))
    sa = ew[:, :, :35].copy()
    sb = ew[:, :, 25:].copy()
    sa[:, :, 30:] = -1.0
    sb[:, :, :5] = -1.0
    fmap = euler.fringe_map([a, b], 5)
    st = euler.exchange([sa, sb], fmap)
    assert np.array_equal(st[0], ew[:, :, :35]) and np.array_equal(st[1], ew[:, :, 25:])


def test_time_step_closed_form():
    p = I.Patch(11, 21, (I.BC_FREE,) * 4, box=(0.0, 1.0, 0.0, 0.5))
    inst = I.Instance([p], [I.conserved(np.full((21, 11), 1.4), 2.0, -0.5, 1.0)])
    s = euler.Solver(inst, cfl=0.5)
    c = 1.0
    expect = 0.5 * min(0.1 / (2.0 + c), 0.025 / (0.5 + c))
    assert abs(s.dt(inst.state) - expect) < 1e-15


def test_conservation_sums_constant_state():
    # FC quadrature of a constant field over a Cartesian patch = area * value
    p = I.Patch(41, 31, (I.BC_FREE,) * 4, box=(0.0, 2.0, 0.0, 0.5))
    inst = I.Instance([p], [I.conserved(np.full((31, 41), 1.0), 0.0, 0.0, 0.4)])
    s = euler.Solver(inst)
    sums = s.conservation_sums(inst.state)
    assert np.allclose(sums[0], [1.0, 0.0, 0.0, 1.0], rtol=1e-11, atol=1e-12)


def test_sod_mean_energy():
    # §7 energy test: with the Sod states the exact mean energy density is 1.375
    inst = I.sod_instance(npatch=1, n1=201, n2=21)
    s = euler.Solver(inst)
    sums = s.conservation_sums(inst.state)
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    assert abs(sums[0, 3] / 0.1 - g["sod_mean_energy"]["E_mean"]) < 2e-2


# ---------------------------------------------------------------- interpolation
def test_lagrange_weights_reproduce_degree_five():
    # the 6-node Lagrange basis reproduces every polynomial of degree <= 5 and
    # its derivative, and no polynomial of degree 6
    a = np.arange(euler.STENCIL, dtype=np.float64)
    for t in (0.0, 0.37, 2.5, 4.91):
        w, dw = euler.lagrange_weights(t), euler.lagrange_dweights(t)
        for k in range(6):
            assert abs(w @ a ** k - t ** k) < 1e-11 * max(1.0, t ** k)
            assert abs(dw @ a ** k - (k * t ** (k - 1) if k else 0.0)) < 1e-10 * max(1.0, t ** k)
    assert abs(euler.lagrange_weights(2.5) @ a ** 6 - 2.5 ** 6) > 1.0


def test_strip_interpolation_exact_for_tensor_quintics():
    patches = I.strip_layout((96, 128, 80))
    fm = euler.fringe_map(patches, 5)
    assert len(fm.copies) == 0 and len(fm.interp) == 2 * 2 * 5 * 40
    masks = [euler.receiver_mask(p, 5) for p in patches]
    for p, j, i, q, j0, i0, W in fm.interp:   # donors are never receivers
        assert masks[p][j, i] and not masks[q][j0:j0 + 6, i0:i0 + 6].any()
        assert abs(W.sum() - 1.0) < 1e-13

    def f(x, y):
        return (1.0 + 3 * x - 2 * x ** 3 + 5 * x ** 5) * (2.0 - 40 * y ** 2 + 9e4 * y ** 5)

    st, ex = [], []
    for pt in patches:
        X, Y = pt.coords()
        ex.append(f(X, Y))
        s = f(X, Y)
        s[euler.receiver_mask(pt, 5)] = -99.0
        st.append(s)
    euler.exchange(st, fm)
    for a, b in zip(st, ex):
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_annulus_donor_index_matches_polar_inverse():
    ring = I.annulus_ring()
    pt = ring[1]
    th0, th1 = 2 * np.pi / 3 - 0.45, 4 * np.pi / 3 + 0.45
    rng = np.random.default_rng(3)
    for _ in range(40):
        th, r = rng.uniform(th0, th1), rng.uniform(0.5, 1.0)
        fi, fj = euler.donor_index(pt, r * np.cos(th), r * np.sin(th))
        assert abs(fi - (th - th0) / (th1 - th0) * (pt.n1 - 1)) < 1e-6
        assert abs(fj - (r - 0.5) / 0.5 * (pt.n2 - 1)) < 1e-6


def test_annulus_interpolation_converges_at_sixth_order():
    def f(x, y):
        return np.sin(2 * x + 0.3) * np.cos(3 * y) + x * y

    errs = []
    for s in (1, 2, 4):
        ring = I.annulus_ring(sizes=((64 * s, 24 * s), (56 * s, 20 * s), (72 * s, 28 * s)))
        fm = euler.fringe_map(ring, 5)
        assert len(fm.interp) > 0
        st, ex = [], []
        for pt in ring:
            X, Y = pt.coords()
            ex.append(f(X, Y))
            v = f(X, Y)
            v[euler.receiver_mask(pt, 5)] = 0.0
            st.append(v)
        euler.exchange(st, fm)
        errs.append(max(np.max(np.abs(a - b)) for a, b in zip(st, ex)))
    assert errs[0] / errs[1] > 2 ** 5 and errs[1] / errs[2] > 2 ** 5


def test_interpolated_viscosity_stays_non_negative():
    patches = I.strip_layout((96, 128, 80))
    fm = euler.fringe_map(patches, 5)
    mu = []
    for pt in patches:
        X, _ = pt.coords()
        mu.append(np.where(np.abs(X - 0.372) < 0.003, 1.0, 0.0))   # a sharp bump in the overlap
    raw = euler.exchange([m.copy() for m in mu], fm)
    clamped = euler.exchange([m.copy() for m in mu], fm, clamp=True)
    assert min(r.min() for r in raw) < 0.0                         # Lagrange overshoot
    assert min(c.min() for c in clamped) == 0.0


# ---------------------------------------------------------------- L-shaped patches
def _l_patch(curvilinear=False, bc=(I.BC_WALL,) * 4):
    # 60 x 52 bounding grid, points i < 24, j < 20 missing (corner at the
    # node (24, 20)); as a box, or as the same grid rotated by 90 degrees
    n1, n2, m1, m2 = 60, 52, 24, 20
    if not curvilinear:
        return I.Patch(n1, n2, bc, box=(0.1, 1.3, -0.2, 0.82), lcut=(m1, m2), kind="C1")
    q1 = np.arange(n1) / (n1 - 1)
    q2 = np.arange(n2) / (n2 - 1)
    Q1, Q2 = np.meshgrid(q1, q2)
    return I.Patch(n1, n2, bc, x=0.9 - 1.02 * Q2, y=-0.3 + 1.2 * Q1, lcut=(m1, m2), kind="C1")


def test_l_patch_derivative_exact_on_low_degree_polynomials():
    for curv in (False, True):
        p = _l_patch(curv)
        g = euler.PatchGeom(p, 5, 25, 1)
        X, Y = p.coords()
        f = X ** 3 * Y ** 2 - 2 * X * Y ** 3 + 0.5
        act = p.active()
        if curv:   # d/dq of x(q), y(q) affine in q
            fx, fy = 3 * X ** 2 * Y ** 2 - 2 * Y ** 3, 2 * X ** 3 * Y - 6 * X * Y ** 2
            d1 = fx * g.x_q1 + fy * g.y_q1
            d2 = fx * g.x_q2 + fy * g.y_q2
            got1, got2 = g.D(f, 0, g.h1), g.D(f, 1, g.h2)
        else:
            d1 = 3 * X ** 2 * Y ** 2 - 2 * Y ** 3
            d2 = 2 * X ** 3 * Y - 6 * X * Y ** 2
            got1, got2 = g.D(f, 0, g.hx), g.D(f, 1, g.hy)
        for got, ref in ((got1, d1), (got2, d2)):
            assert np.abs(got - ref)[act].max() < 2e-8 * np.abs(ref[act]).max()
            assert np.all(got[~act] == 0.0)


def test_l_patch_full_lines_match_rectangle():
    # where both lines through a point are full, the L patch and its bounding
    # rectangle apply the same operators to the same data
    p = _l_patch()
    r = I.Patch(p.n1, p.n2, p.bc, box=p.box)
    e = I.random_state(r, np.random.default_rng(8))
    mu = 0.01 * (1 + np.cos(3 * r.coords()[0]))
    a = euler.rhs(e, euler.PatchGeom(p, 5, 25, 1), 5, 25, G, mu)
    b = euler.rhs(e, euler.PatchGeom(r, 5, 25, 1), 5, 25, G, mu)
    m1, m2 = p.lcut
    assert np.array_equal(a[:, m2 + 1:-1, m1 + 1:-1], b[:, m2 + 1:-1, m1 + 1:-1])
    assert not np.allclose(a[:, :m2, m1 + 1:-1], b[:, :m2, m1 + 1:-1])   # short columns differ
    assert np.all(a[:, :m2, :m1] == 0.0)


def test_l_patch_free_stream_preserved():
    for curv in (False, True):
        p = _l_patch(curv, bc=(I.BC_INTERNAL,) * 4)
        e = I.conserved(np.full((p.n2, p.n1), 1.3), 0.7, -0.4, 1.1)
        L = euler.rhs(e, euler.PatchGeom(p, 5, 25, 1), 5, 25, G)
        assert np.abs(L).max() < 1e-6          # fit residual of FC-Gram times 1/h, as on rectangles
        X, _ = p.coords()
        e2 = I.conserved(1.3 + 0.1 * np.sin(3 * X), 0.7, -0.4, 1.1)
        assert np.abs(euler.rhs(e2, euler.PatchGeom(p, 5, 25, 1), 5, 25, G)).max() > 1e-2


def test_l_patch_inner_walls():
    for curv in (False, True):
        p = _l_patch(curv)
        inst = I.Instance([p], [I.conserved(np.ones((p.n2, p.n1)), 0.5, 0.3, 1.0)])
        s = euler.Solver(inst, c_policy=1)
        e = inst.state[0].copy()
        euler.apply_bc(e, s.geoms[0], inst)
        m1, m2 = p.lcut
        g = s.geoms[0]
        # inner vertical edge i = m1 (j < m2): velocity along grad q1 removed
        v = e[1:3, :m2, m1] / e[0, :m2, m1]
        n = np.stack([g.y_q2[:m2, m1], -g.x_q2[:m2, m1]])
        assert np.abs((v * n).sum(0)).max() < 1e-12
        v = e[1:3, m2, :m1] / e[0, m2, :m1]
        n = np.stack([-g.y_q1[m2, :m1], g.x_q1[m2, :m1]])
        assert np.abs((v * n).sum(0)).max() < 1e-12
        # the corner node keeps only the velocity across the bisector of the
        # two inward normals: for this grid (normals along the axes) u' = -v'
        n1 = np.array([g.y_q2[m2, m1], -g.x_q2[m2, m1]])
        n2 = np.array([-g.y_q1[m2, m1], g.x_q1[m2, m1]])
        nb = n1 / np.linalg.norm(n1) + n2 / np.linalg.norm(n2)
        assert abs(e[1:3, m2, m1] @ nb) < 1e-12 * np.abs(e[1:3, m2, m1]).max()
        assert np.abs(e[1:3, m2, m1]).max() > 0.1                  # not a stagnation point


def test_filter_state_keeps_uniform_and_smooth_states():
    p = I.Patch(48, 40, (I.BC_WALL,) * 4, box=(0.0, 1.0, 0.0, 0.8))
    g = euler.PatchGeom(p, 5, 25, 1)
    e = I.conserved(np.full((40, 48), 1.3), 0.4, -0.2, 0.9)
    assert np.abs(euler.filter_state(e, g, G) - e).max() < 1e-8 * np.abs(e).max()   # FC-Gram fit residual
    s = I.random_state(p, np.random.default_rng(3))
    assert np.abs(euler.filter_state(s, g, G) - s).max() < 1e-8
    lp = _l_patch()
    gl = euler.PatchGeom(lp, 5, 25, 1)
    sl = I.random_state(lp, np.random.default_rng(4))
    fl = euler.filter_state(sl, gl, G)
    assert np.abs(fl - sl).max() < 1e-8


def test_neumann_weights_are_the_one_sided_difference_formulas():
    # textbook one-sided first-derivative formulas on 2..6 points (unit spacing)
    table = {2: [-1, 1], 3: [-3 / 2, 2, -1 / 2], 4: [-11 / 6, 3, -3 / 2, 1 / 3],
             5: [-25 / 12, 4, -3, 4 / 3, -1 / 4], 6: [-137 / 60, 5, -5, 10 / 3, -5 / 4, 1 / 5]}
    for d, w in table.items():
        assert np.allclose(euler.neumann_weights(d), w, rtol=0, atol=1e-13)


def _theta(e):
    return euler.pressure(e, G) / e[0]


def _with_theta(rho, mx, my, theta):
    return np.stack([rho, mx, my, rho * theta / (G - 1) + 0.5 * (mx * mx + my * my) / rho])


def test_noslip_adiabatic_wall_on_curvilinear_sector():
    # wall at r = r0 (side 2, q2 = 0): theta along each radial line is a
    # cubic in the index j with zero slope at the wall, so the wall value the
    # Neumann condition gives is its value a(i) there
    ring = I.annulus_ring(wall=I.BC_NOSLIP)
    p = ring[0]
    inst = I.Instance(ring, [np.zeros((4, q.n2, q.n1)) for q in ring])
    s = euler.Solver(inst, c_policy=1)
    rng = np.random.default_rng(3)
    j = np.arange(p.n2)[:, None].astype(float)
    a = 1.0 + 0.2 * rng.random(p.n1)
    theta = a + 0.01 * j ** 2 - 0.001 * j ** 3
    theta[0] += 0.3                                   # wall value to be replaced
    rho = 1.0 + 0.1 * rng.random((p.n2, p.n1))
    e = _with_theta(rho, 0.4 * rng.standard_normal((p.n2, p.n1)), 0.2 * rng.standard_normal((p.n2, p.n1)), theta)
    before = e.copy()
    euler.apply_bc(e, s.geoms[0], inst)
    assert np.all(e[1:3, 0, :] == 0.0)                                      # no slip
    assert np.abs(_theta(e[:, 0, :]) - a).max() < 1e-12                     # adiabatic
    assert np.allclose(e[3, 0, :], e[0, 0, :] * a / (G - 1), rtol=1e-13)
    assert np.array_equal(e[:, 1:, :], before[:, 1:, :])                    # interior untouched
    assert np.array_equal(e[0], before[0])                                  # density free


def test_noslip_adiabatic_walls_on_opposite_sides():
    # left and right no-slip, bottom/top slip: theta = 1 + c i^2 (N - i)^2 has
    # zero slope at both ends and degree 4 < d, so both wall values are 1
    n1, n2 = 30, 12
    p = I.Patch(n1, n2, (I.BC_NOSLIP, I.BC_NOSLIP, I.BC_WALL, I.BC_WALL), box=(0.0, 1.0, 0.0, 0.4))
    inst = I.Instance([p], [np.zeros((4, n2, n1))])
    s = euler.Solver(inst)
    i = np.arange(n1)[None, :].astype(float)
    theta = np.broadcast_to(1.0 + 1e-5 * i ** 2 * (n1 - 1 - i) ** 2, (n2, n1)).copy()
    theta[:, 0] = theta[:, -1] = 7.0
    e = _with_theta(np.full((n2, n1), 1.3), np.full((n2, n1), 0.5), np.full((n2, n1), -0.2), theta)
    euler.apply_bc(e, s.geoms[0], inst)
    for col in (0, -1):
        assert np.all(e[1:3, :, col] == 0.0)
        # (corner rows excluded: their inward points lie on the slip walls,
        # whose condition removed kinetic energy and so changed theta there)
        assert np.abs(_theta(e[:, 1:-1, col]) - 1.0).max() < 1e-12
    assert np.all(e[2, 0, 1:-1] == 0.0) and np.all(e[2, -1, 1:-1] == 0.0)   # slip walls
    assert np.allclose(e[1, 0, 1:-1], 0.5)


def test_noslip_viscous_flux_keeps_wall_shear():
    p = I.Patch(8, 8, (I.BC_INTERNAL, I.BC_FREE, I.BC_NOSLIP, I.BC_WALL), box=(0.0, 1.0, 0.0, 1.0))
    V1, V2 = np.ones((4, 8, 8)), np.ones((4, 8, 8))
    euler._zero_normal_viscous(V1, V2, p)
    assert np.all(V2[[0, 3], 0, :] == 0.0) and np.all(V2[[1, 2], 0, :] == 1.0)   # no-slip: mass, energy
    assert np.all(V2[:, -1, :] == 0.0) and np.all(V1[:, :, -1] == 0.0)            # slip wall, free side
    assert np.all(V1[:, :, 0] == 1.0)                                             # internal side


def test_noslip_layout_checks():
    bad = I.Patch(8, 8, (I.BC_NOSLIP, I.BC_FREE, I.BC_NOSLIP, I.BC_FREE), box=(0.0, 1.0, 0.0, 1.0))
    with pytest.raises(ValueError):
        euler.Solver(I.Instance([bad], [np.zeros((4, 8, 8))]))
    lp = _l_patch(False)
    lp.bc = (I.BC_NOSLIP,) + tuple(lp.bc[1:])
    with pytest.raises(ValueError):
        euler.check_noslip(lp)


def test_noslip_ring_steps_keep_the_wall_conditions():
    patches = I.annulus_ring(wall=I.BC_NOSLIP)
    state = []
    for p in patches:
        X, Y = p.coords()
        r = np.hypot(X, Y)
        f = 1.0 - np.exp(-((r - 0.5) / 0.15) ** 2)
        state.append(I.conserved(np.full(X.shape, 1.4), 0.8 * f * (-Y / r), 0.8 * f * (X / r), 1.0))
    inst = I.Instance(patches, state)
    s = euler.Solver(inst, c_policy=1)
    st = [e.copy() for e in state]
    mu = [np.full((p.n2, p.n1), 2e-4) for p in patches]
    for _ in range(3):
        st = s.step(st, 2e-4, mu)
    w = euler.neumann_weights(5)
    for e in st:
        inner = slice(s.n_f, e.shape[2] - s.n_f)           # wall points outside the angle fringes
        assert np.all(e[1:3, 0, inner] == 0.0)
        th = _theta(e[:, :5, inner])
        assert np.abs(w @ th).max() < 1e-12 * np.abs(th).max()
        assert np.all(np.isfinite(e))


def _conserved_of_w(w):
    rho, m, n, th = w
    return np.stack([rho, m, n, rho * th / (G - 1) + 0.5 * (m * m + n * n) / rho])


def test_flux_jacobians_match_finite_differences():
    rng = np.random.default_rng(5)
    w = np.stack([rng.uniform(0.5, 2, 50), rng.uniform(-2, 2, 50), rng.uniform(-2, 2, 50), rng.uniform(0.3, 3, 50)])
    A, B = euler.flux_jacobians(w, G)
    for k in range(4):
        dw = np.zeros_like(w)
        dw[k] = 1e-6 * np.maximum(np.abs(w[k]), 1.0)
        fp, gp = euler.fluxes(_conserved_of_w(w + dw), G)
        fm, gm = euler.fluxes(_conserved_of_w(w - dw), G)
        dfa = (fp - fm) / (2 * dw[k])
        dga = (gp - gm) / (2 * dw[k])
        scale = 1.0 + np.abs(dfa) + np.abs(dga)
        assert np.abs(A[:, k] - dfa).max() / scale.max() < 1e-7
        assert np.abs(B[:, k] - dga).max() / scale.max() < 1e-7


def _exact_divergence():
    """-(f_x + g_y) of a smooth analytic state, differentiated symbolically."""
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    rho = 1.2 + 0.2 * sympy.sin(2 * x + 1) * sympy.cos(y)
    u = 0.6 + 0.2 * sympy.cos(3 * x - y)
    v = -0.3 + 0.2 * sympy.sin(x + 2 * y)
    p = 1.0 + 0.3 * sympy.cos(x) * sympy.sin(2 * y + 0.5)
    E = p / (G - 1) + rho * (u * u + v * v) / 2
    f = [rho * u, rho * u * u + p, rho * u * v, (E + p) * u]
    g = [rho * v, rho * u * v, rho * v * v + p, (E + p) * v]
    L = [-(sympy.diff(f[i], x) + sympy.diff(g[i], y)) for i in range(4)]
    state = sympy.lambdify((x, y), [rho, rho * u, rho * v, E], "numpy")
    div = sympy.lambdify((x, y), L, "numpy")
    return state, div


def _chain_error(patch, state, div, cart=True):
    inst = I.Instance([patch], [np.zeros((4, patch.n2, patch.n1))])
    s = euler.Solver(inst, c_policy=1, chain=True)
    X, Y = patch.coords()
    e = np.array([np.broadcast_to(a, X.shape) for a in state(X, Y)], dtype=np.float64)
    L = s.rhs_all([e])[0]
    ex = np.array([np.broadcast_to(a, X.shape) for a in div(X, Y)])
    return np.abs(L - ex).max() / np.abs(ex).max()


def test_chain_form_converges_to_the_exact_divergence_cartesian():
    state, div = _exact_divergence()
    errs = [_chain_error(I.Patch(n, n, (I.BC_FREE,) * 4, box=(0.0, 1.0, 0.0, 1.0)), state, div) for n in (24, 48, 96)]
    assert errs[-1] < 1e-6
    assert errs[0] / errs[1] > 6 and errs[1] / errs[2] > 6      # at least third order


def test_chain_form_converges_to_the_exact_divergence_curvilinear():
    state, div = _exact_divergence()
    errs = [_chain_error(I.annulus_patch(n, n, bc=(I.BC_FREE,) * 4), state, div) for n in (24, 48, 96)]
    assert errs[-1] < 1e-5
    assert errs[0] / errs[1] > 6 and errs[1] / errs[2] > 6


def test_chain_form_is_inviscid_only():
    inst = I.vortex_instance(21)
    s = euler.Solver(inst, chain=True)
    with pytest.raises(ValueError):
        s.rhs_all(inst.state, [np.zeros((21, 21))])
