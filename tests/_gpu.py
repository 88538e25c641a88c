"""Shared helpers of the GPU parity tests (seeded inputs, context builders)."""
import math

import numpy as np

from paper_2506_19370_gb300 import inputs as I

F32, F64 = 0, 1
EPS = {F64: 2.0 ** -53, F32: 2.0 ** -24}

LAYOUTS = ("vortex", "sod", "annulus")


def layout(name):
    """(instance, C policy) of a parity layout."""
    if name == "vortex":
        return I.vortex_instance(101), 0
    if name == "sod":
        return I.sod_instance(smear=3.0), 1
    if name == "annulus":
        p = I.annulus_patch(48, 40)
        X, _ = p.coords()
        e = I.conserved(1.4 + 0.0 * X, 2.0, 0.5, 1.0)
        return I.Instance([p], [e], name="annulus"), 1
    if name == "split":
        # two overlapping Cartesian patches in y and two in x (4 patches, corners)
        pts = [I.Patch(40, 36, (I.BC_WALL, I.BC_INTERNAL, I.BC_WALL, I.BC_INTERNAL), box=(0, 39 / 60, 0, 35 / 60)),
               I.Patch(32, 36, (I.BC_INTERNAL, I.BC_WALL, I.BC_WALL, I.BC_INTERNAL), box=(29 / 60, 1, 0, 35 / 60)),
               I.Patch(40, 36, (I.BC_WALL, I.BC_INTERNAL, I.BC_INTERNAL, I.BC_WALL), box=(0, 39 / 60, 25 / 60, 1)),
               I.Patch(32, 36, (I.BC_INTERNAL, I.BC_WALL, I.BC_INTERNAL, I.BC_WALL), box=(29 / 60, 1, 25 / 60, 1))]
        rng = np.random.default_rng(7)
        return I.Instance(pts, [I.random_state(p, rng) for p in pts], name="split"), 1
    if name == "strip":
        # Sod on three patches of 96, 128 and 80 points along x: non-coincident
        # grids (interpolated fringes) and two FFT sizes along x
        return I.sod_instance(smear=3.0, patches=I.strip_layout((96, 128, 80))), 1
    if name == "ring":
        # annulus covered by three curvilinear sectors of different resolutions
        # (interpolated fringes between curvilinear grids, two FFT sizes)
        pts = I.annulus_ring(sizes=((64, 24), (100, 30), (72, 28)))
        rng = np.random.default_rng(9)
        st = []
        for p in pts:
            X, Y = p.coords()
            a, b = rng.uniform(1, 3, 2)
            st.append(I.conserved(1.4 * (1 + 0.05 * np.sin(a * X + b * Y)), 0.4 + 0.05 * np.cos(b * X), 0.2,
                                  1.0 + 0.05 * np.cos(a * Y)))
        return I.Instance(pts, st, name="ring"), 1
    if name == "ringns":
        # the ring with a no-slip adiabatic wall at r = 0.5 and a swirling
        # flow brought to rest smoothly at the wall
        pts = I.annulus_ring(sizes=((64, 24), (100, 30), (72, 28)), wall=I.BC_NOSLIP)
        st = []
        for p in pts:
            X, Y = p.coords()
            r = np.hypot(X, Y)
            f = 1.0 - np.exp(-((r - 0.5) / 0.15) ** 2)
            st.append(I.conserved(1.4 * (1 + 0.05 * np.sin(3 * X + Y)), 0.6 * f * (-Y / r) + 0.1 * f,
                                  0.6 * f * (X / r), 1.0 + 0.05 * np.cos(2 * Y)))
        return I.Instance(pts, st, name="ringns"), 1
    if name == "splitns":
        # the four-patch split layout with no-slip adiabatic walls on the left
        # and right outer sides (slip walls at the bottom and top)
        inst, pol = layout("split")
        for p in inst.patches:
            p.bc = tuple(I.BC_NOSLIP if (k < 2 and b == I.BC_WALL) else b for k, b in enumerate(p.bc))
        inst.name = "splitns"
        return inst, pol
    if name == "cylns":
        # the Mach-10 cylinder with the paper's no-slip adiabatic body wall
        return I.cylinder_instance(h=0.03, wall=I.BC_NOSLIP), 1
    if name in ("lbox", "lcurv"):
        # one L-shaped corner patch (60 x 52 grid, points i < 24, j < 20
        # missing), as a box or on a grid rotated by 90 degrees, walls around
        n1, n2, m1, m2 = 60, 52, 24, 20
        if name == "lbox":
            p = I.Patch(n1, n2, (I.BC_WALL,) * 4, box=(0.1, 1.3, -0.2, 0.82), lcut=(m1, m2), kind="C1")
        else:
            Q1, Q2 = np.meshgrid(np.arange(n1) / (n1 - 1), np.arange(n2) / (n2 - 1))
            p = I.Patch(n1, n2, (I.BC_WALL,) * 4, x=0.9 - 1.02 * Q2, y=-0.3 + 1.2 * Q1, lcut=(m1, m2), kind="C1")
        rng = np.random.default_rng(13)
        return I.Instance([p], [I.random_state(p, rng)], name=name), 1
    if name == "cylinder":
        # Mach-10 flow past a cylinder: annular sectors + Cartesian far field
        return I.cylinder_instance(h=0.03), 1
    if name == "ensemble":
        # three independent step flows of different resolutions and Mach
        # numbers in one layout (per-patch inflow states)
        return I.ffs_ensemble((0.006, 0.005, 0.0045), (2.0, 3.0, 4.0), length=1.4), 1
    if name == "ffs":
        # forward-facing step at Mach 3, 32 patches of uneven resolution with
        # a C1 (L-shaped) and a C2 corner patch (coarse version of the
        # 64-patch, ~1M-point layout)
        return I.ffs_instance(h0=0.005, length=1.4), 1
    raise KeyError(name)


def active_only(arrs, inst):
    """Zero the points outside L-shaped patches (never written by the library)."""
    out = []
    for a, p in zip(arrs, inst.patches):
        a = np.array(a, dtype=np.float64, copy=True)
        a[..., ~p.active()] = 0.0
        out.append(a)
    return out


def random_fields(inst, seed):
    rng = np.random.default_rng(seed)
    out = []
    for p in inst.patches:
        X, Y = p.coords()
        a, b, c = rng.uniform(1, 4, 3)
        out.append(np.sin(a * X + 0.3) * np.cos(b * Y - c) + 0.2 * X * Y + 1.5)
    return out


def random_states(inst, seed):
    rng = np.random.default_rng(seed)
    return [I.random_state(p, rng) for p in inst.patches]


def rel_err(a, b):
    a = np.concatenate([np.ravel(x) for x in a])
    b = np.concatenate([np.ravel(x) for x in b])
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def table_gain(d, C):
    """Largest row sum of |A_R| + |A_L|: amplification of rounding in the continuation."""
    from oracle import fcgram
    A_R, A_L = fcgram.continuation_tables(d, C)
    return float(np.max(np.abs(A_R).sum(1) + np.abs(A_L).sum(1)))


def deriv_bound(dtype, fmax, h, n, order, gain=None):
    """Rounding bound of one FC derivative of a line with values up to fmax.

    Both precisions continue in the Gram form (FP64: compensated projection
    on the Gram basis; FP32: Gram coefficients of the shifted line, or
    compensated sums with a split table), so the continuation adds a few
    roundings of the line's values (the ill-conditioned combined table, whose
    row sums `gain` reach ~7e3, never meets the data directly).  Rounding
    errors of the FFT pair add up like a random walk over its log2(n) stages
    (standard deviation ~ eps sqrt(log2 n + 4) fmax per mode); the derivative
    weights mode k by k^order, whose root mean square over the band is
    (pi/h)^order / sqrt(2 order + 1); the largest of all the points of a line
    set stays within 4 standard deviations.
    """
    return (4.0 * EPS[dtype] * math.sqrt(math.log2(n) + 4.0) * fmax * (math.pi / h) ** order
            / math.sqrt(2 * order + 1))
