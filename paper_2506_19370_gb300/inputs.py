"""Seeded synthetic inputs: patch layouts, initial data and classifier windows.

This module is the one piece shared by the CUDA path and the CPU oracle.  It
holds no step of the FC-SDNN method: it only lays out patches, samples initial
conditions and draws labelled training windows from seeded generators.

Workloads (shapes follow the paper's problems, §7):
  * ``vortex_instance``: one Cartesian patch on [0,1]^2 with an isentropic
    vortex advected by a uniform flow (single-patch accuracy case);
  * ``sod_instance``: the shock tube on [0,1] x [0,0.1] split into overlapping
    Cartesian patches, Sod data (§7 energy-conservation test uses the same
    states), reflecting walls;
  * ``mach_shock_state`` / ``mach_flow_state``: the Mach-M initial states of §7
    (Eq. for the Mach-M flow and the Mach-M shock);
  * ``classifier_windows``: labelled 16-point windows of seeded smooth, C1,
    kink and jump profiles for training the smoothness classifier.
"""
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

GAMMA = 1.4
SEED = 2506

# boundary-condition codes, one per patch side (left i=0, right i=n1-1,
# bottom j=0, top j=n2-1); they match the FCS_BC_* values of the C ABI
BC_INTERNAL = 0   # side lies inside the domain: values come from donors
BC_WALL = 1       # slip / reflecting wall: normal momentum set to zero
BC_INFLOW = 2     # Dirichlet: all four conserved variables prescribed
BC_OUTFLOW = 3    # pressure prescribed, energy recomputed
BC_FREE = 4       # nothing imposed (supersonic outflow)
BC_NOSLIP = 5     # no-slip adiabatic wall: momentum zero, zero normal temperature derivative


@dataclass
class Patch:
    """One patch with an n1 x n2 parameter grid (i along q1).

    Cartesian patches carry their box; curvilinear ones carry the physical
    coordinates x[j, i], y[j, i] of every grid point.  lcut = (m1, m2) > 0
    makes an L-shaped corner patch (type C1 of §3.2, parameter space L of
    the paper): the points with i < m1 and j < m2 are not part of the patch
    and the two inner edges (i = m1, j < m2 and j = m2, i < m1) are walls.
    """
    n1: int
    n2: int
    bc: Sequence[int]
    box: Optional[Sequence[float]] = None          # (x0, x1, y0, y1)
    x: Optional[np.ndarray] = None
    y: Optional[np.ndarray] = None
    lcut: Sequence[int] = (0, 0)
    kind: str = ""                                   # S, C1, C2 or I (label only)
    inflow: Optional[Sequence[float]] = None         # conserved inflow state of this patch (None: the instance's)

    @property
    def cartesian(self):
        return self.box is not None

    @property
    def is_l(self):
        return self.lcut[0] > 0 and self.lcut[1] > 0

    def active(self):
        """Mask of the grid points that belong to the patch."""
        m = np.ones((self.n2, self.n1), dtype=bool)
        if self.is_l:
            m[:self.lcut[1], :self.lcut[0]] = False
        return m

    def coords(self):
        if self.cartesian:
            x0, x1, y0, y1 = self.box
            xs = x0 + (x1 - x0) * np.arange(self.n1) / (self.n1 - 1)
            ys = y0 + (y1 - y0) * np.arange(self.n2) / (self.n2 - 1)
            return np.meshgrid(xs, ys)
        return self.x, self.y


@dataclass
class Instance:
    """One flow problem: patches, gas constant, boundary data, initial state."""
    patches: List[Patch]
    state: List[np.ndarray]                       # per patch (4, n2, n1), conserved
    gamma: float = GAMMA
    inflow: Sequence[float] = (1.0, 1.0, 0.0, 2.5)  # conserved inflow state
    p_out: float = 1.0
    name: str = ""
    meta: dict = field(default_factory=dict)


def conserved(rho, u, v, p, gamma=GAMMA):
    """(rho, rho u, rho v, E) from primitives, E = p/(gamma-1) + rho|u|^2/2 (Eq. 2)."""
    rho, u, v, p = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (rho, u, v, p)))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def vortex_primitives(x, y, t, eps=5.0, R=0.05, x0=0.5, y0=0.5, u0=1.0, v0=0.0, gamma=GAMMA):
    """Isentropic vortex of strength eps and radius R advected by (u0, v0).

    Standard form: with (xb, yb) = ((x - x0 - u0 t)/R, (y - y0 - v0 t)/R) and
    r2 = xb^2 + yb^2, du = -eps/(2 pi) e^{(1-r2)/2} yb, dv = eps/(2 pi)
    e^{(1-r2)/2} xb, T = 1 - (gamma-1) eps^2/(8 gamma pi^2) e^{1-r2},
    rho = T^{1/(gamma-1)}, p = rho^gamma (free stream rho = p = 1).
    """
    xb = (x - x0 - u0 * t) / R
    yb = (y - y0 - v0 * t) / R
    r2 = xb * xb + yb * yb
    g = np.exp(0.5 * (1.0 - r2))
    u = u0 - eps / (2 * np.pi) * g * yb
    v = v0 + eps / (2 * np.pi) * g * xb
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi ** 2) * g * g
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return rho, u, v, p


def vortex_instance(n=101, eps=5.0, R=0.05):
    """Single Cartesian patch [0,1]^2, n x n points, vortex at (0.5, 0.5)."""
    patch = Patch(n, n, (BC_INFLOW, BC_OUTFLOW, BC_WALL, BC_WALL), box=(0.0, 1.0, 0.0, 1.0))
    X, Y = patch.coords()
    e = conserved(*vortex_primitives(X, Y, 0.0, eps=eps, R=R))
    inflow = tuple(float(a) for a in conserved(1.0, 1.0, 0.0, 1.0))
    return Instance([patch], [e], inflow=inflow, p_out=1.0, name=f"vortex_{n}x{n}",
                    meta=dict(eps=eps, R=R))


def sod_layout(npatch=8, n1=160, n2=40, overlap=10, length=1.0, height=0.1):
    """Overlapping Cartesian patches along x covering [0,length] x [0,height].

    Neighbouring patches share `overlap` grid columns; the global x grid has
    npatch*n1 - (npatch-1)*overlap points.
    """
    nx = npatch * n1 - (npatch - 1) * overlap
    hx = length / (nx - 1)
    patches = []
    for p in range(npatch):
        i0 = p * (n1 - overlap)
        bc = [BC_INTERNAL, BC_INTERNAL, BC_WALL, BC_WALL]
        if p == 0:
            bc[0] = BC_WALL
        if p == npatch - 1:
            bc[1] = BC_WALL
        patches.append(Patch(n1, n2, tuple(bc), box=(i0 * hx, (i0 + n1 - 1) * hx, 0.0, height)))
    return patches


def strip_layout(n1s, n2=40, length=1.0, height=0.1, overlap=0.08):
    """Overlapping Cartesian patches along x with different point counts.

    Patch k spans [a_k, a_k + w] (equal widths w, consecutive patches overlap
    by `overlap`), with n1s[k] points along x: the grids do not coincide, so
    fringes are filled by interpolation.  Outer ends and y sides are walls.
    """
    P = len(n1s)
    w = (length + (P - 1) * overlap) / P
    patches = []
    for k, n1 in enumerate(n1s):
        a = k * (w - overlap)
        bc = [BC_INTERNAL, BC_INTERNAL, BC_WALL, BC_WALL]
        if k == 0:
            bc[0] = BC_WALL
        if k == P - 1:
            bc[1] = BC_WALL
        patches.append(Patch(n1, n2, tuple(bc), box=(a, min(a + w, length) if k == P - 1 else a + w, 0.0, height)))
    return patches


def sod_instance(npatch=8, n1=160, n2=40, overlap=10, x_jump=0.5, height=0.1, perturb=0.0, seed=SEED,
                 smear=0.0, patches=None):
    """Sod shock tube (rho,u,p) = (1,0,1) | (0.125,0,0.1), jump at x_jump.

    `perturb` adds a seeded relative perturbation to the density (used to make
    batched instances distinct).  `smear` > 0 replaces the jump by a tanh
    profile `smear` grid spacings wide (a stand-in for the paper's localized
    smearing of discontinuous initial data, Algorithm 4, which is not part of
    the stage).  `patches` replaces the default layout (any Cartesian
    patches covering [0,1] x [0,height]); the smearing width then uses the
    finest x spacing.
    """
    if patches is None:
        patches = sod_layout(npatch, n1, n2, overlap, 1.0, height)
        nx = npatch * n1 - (npatch - 1) * overlap
        hx = 1.0 / (nx - 1)
    else:
        hx = min((p.box[1] - p.box[0]) / (p.n1 - 1) for p in patches)
    rng = np.random.default_rng(seed)
    state = []
    for pt in patches:
        X, Y = pt.coords()
        if smear > 0:
            w = 0.5 * (1.0 + np.tanh((X - x_jump) / (smear * hx)))
            rho = 1.0 + (0.125 - 1.0) * w
            p = 1.0 + (0.1 - 1.0) * w
        else:
            left = X < x_jump
            rho = np.where(left, 1.0, 0.125)
            p = np.where(left, 1.0, 0.1)
        if perturb:
            rho = rho * (1.0 + perturb * rng.uniform(-1.0, 1.0))
        state.append(conserved(rho, 0.0 * X, 0.0 * X, p))
    return Instance(patches, state, inflow=(1.0, 0.0, 0.0, 2.5), p_out=0.1, name="sod",
                    meta=dict(x_jump=x_jump))


def annulus_patch(n1=48, n2=32, r0=0.5, r1=1.0, th0=0.3, th1=1.4, bc=(BC_FREE,) * 4):
    """Curvilinear polar patch: q1 -> angle in [th0, th1], q2 -> radius in [r0, r1]."""
    q1 = np.arange(n1) / (n1 - 1)
    q2 = np.arange(n2) / (n2 - 1)
    Q1, Q2 = np.meshgrid(q1, q2)
    th = th0 + (th1 - th0) * Q1
    r = r0 + (r1 - r0) * Q2
    return Patch(n1, n2, tuple(bc), x=r * np.cos(th), y=r * np.sin(th))


def annulus_ring(sizes=((64, 24), (56, 20), (72, 28)), r0=0.5, r1=1.0, overlap=0.9, rot=0.0, wall=BC_WALL):
    """Annulus r0 <= r <= r1 covered by overlapping curvilinear sectors.

    Sector k has sizes[k] = (n1, n2) points (angle, radius) and spans the
    angles [k 2pi/P - overlap/2, (k+1) 2pi/P + overlap/2] + rot; the sectors'
    grids differ, so their fringes are filled by interpolation.  Angle sides
    are internal, r = r0 a wall of kind `wall` (the cylinder), r = r1 free.
    """
    P = len(sizes)
    patches = []
    for k, (n1, n2) in enumerate(sizes):
        th0 = rot + k * 2 * np.pi / P - overlap / 2
        th1 = rot + (k + 1) * 2 * np.pi / P + overlap / 2
        patches.append(annulus_patch(n1, n2, r0, r1, th0, th1, bc=(BC_INTERNAL, BC_INTERNAL, wall, BC_FREE)))
    return patches


def ffs_start_factor(X, Y, ell=0.05):
    """Smooth factor 1 - exp(-(d/ell)^2), d the distance to the step's front
    face (x = 0.6, 0 <= y <= 0.2): the velocity of the initial state is
    multiplied by it, so the data satisfy the wall condition on the face."""
    dy = np.maximum(Y - 0.2, 0.0)
    d = np.hypot(X - 0.6, dy)
    return 1.0 - np.exp(-(d / ell) ** 2)


def ffs_instance(h0=0.002, length=3.0, seed=SEED, delta_pts=8, jitter=0.15, mach=3.0, start="smooth"):
    """Mach-`mach` flow over a forward-facing step (§7 problem shape).

    Channel [0, length] x [0, 1] with a step [0.6, length] x [0, 0.2].  The
    flow region is cut into cells at x = 0.2, 0.4, ... and y = 0.1, 0.2, 0.4,
    0.6, 0.8; every cell becomes a Cartesian patch extended by delta on its
    internal sides, with its own seeded spacing h0 (1 +- jitter), so that
    neighbouring grids do not coincide.  The three cells around the step's
    top corner (0.6, 0.2) (interior angle 270 degrees) form one L-shaped C1
    corner patch (§3.2), on a grid rotated by 90 degrees so that the missing
    quadrant of its parameter space maps onto the step; the cell at the
    step's foot (0.6, 0) is the C2 corner patch (interior angle 90 degrees).
    Left: inflow, right: free (supersonic outflow), walls elsewhere.  Initial
    state: the Mach flow (1.4, mach, 0, 1) of §7, its velocity brought to rest
    smoothly at the step's front face (start="smooth", ffs_start_factor; a
    stand-in for the localized smearing of initial data, Algorithm 4, which the
    stage does not contain) or uniform (start="uniform": an impulsive start
    whose wall jump the FC derivatives cannot represent).
    """
    rng = np.random.default_rng(seed)
    hmax = h0 * (1 + jitter)
    k = int(round(0.1 / h0))
    hs = 0.1 / k                              # C1 spacing: the corner lines are grid lines
    dn = int(np.ceil(delta_pts * hmax / hs))
    delta = dn * hs
    xb = list(np.round(np.arange(0.0, length + 1e-9, 0.2), 12))
    yb = [0.0, 0.1, 0.2, 0.4, 0.6, 0.8, 1.0]
    corner_cells = {(0.4, 0.2), (0.6, 0.2), (0.4, 0.1)}   # (x0, y0) of the cells inside the C1 patch
    patches = []
    for iy in range(len(yb) - 1):
        for ix in range(len(xb) - 1):
            x0, x1, y0, y1 = xb[ix], xb[ix + 1], yb[iy], yb[iy + 1]
            if x0 >= 0.6 - 1e-12 and y1 <= 0.2 + 1e-12:
                continue                                  # inside the step
            if (round(x0, 6), round(y0, 6)) in corner_cells:
                continue
            on_step_top = x0 >= 0.6 - 1e-12 and abs(y0 - 0.2) < 1e-12
            on_face = abs(x1 - 0.6) < 1e-12 and y1 <= 0.2 + 1e-12
            bc = [BC_INTERNAL] * 4
            if x0 == 0.0:
                bc[0] = BC_INFLOW
            if abs(x1 - length) < 1e-12:
                bc[1] = BC_FREE
            if on_face:
                bc[1] = BC_WALL
            if y0 == 0.0 or on_step_top:
                bc[2] = BC_WALL
            if abs(y1 - 1.0) < 1e-12:
                bc[3] = BC_WALL
            box = [x0 - delta * (bc[0] == BC_INTERNAL), x1 + delta * (bc[1] == BC_INTERNAL),
                   y0 - delta * (bc[2] == BC_INTERNAL), y1 + delta * (bc[3] == BC_INTERNAL)]
            h = h0 * (1 + jitter * rng.uniform(-1.0, 1.0))
            n1 = int(round((box[1] - box[0]) / h)) + 1
            n2 = int(round((box[3] - box[2]) / h)) + 1
            kind = "C2" if (on_face and y0 == 0.0) else ("S" if BC_WALL in bc or BC_INFLOW in bc or BC_FREE in bc else "I")
            patches.append(Patch(n1, n2, tuple(bc), box=tuple(box), kind=kind))
    # C1 corner patch: x = xr - hs j, y = yb0 + hs i on the bounding square,
    # points i < m1 (y < 0.2) with j < m2 (x > 0.6) missing
    xr, yb0 = 0.8 + delta, 0.1 - delta
    m1, m2 = k + dn, 2 * k + dn
    n1, n2 = 3 * k + 2 * dn + 1, 4 * k + 2 * dn + 1
    I_, J_ = np.meshgrid(np.arange(n1), np.arange(n2))
    c1 = Patch(n1, n2, (BC_INTERNAL,) * 4, x=xr - hs * J_, y=yb0 + hs * I_, lcut=(m1, m2), kind="C1")
    patches.insert(0, c1)
    state = []
    for p in patches:
        X, Y = p.coords()
        f = ffs_start_factor(X, Y) if start == "smooth" else 1.0
        state.append(conserved(np.full(X.shape, 1.4), mach * f, 0.0, 1.0))
    return Instance(patches, state, inflow=tuple(float(a) for a in conserved(1.4, mach, 0.0, 1.0)), p_out=1.0,
                    name="ffs", meta=dict(h0=h0, delta=delta, length=length))


def ffs_ensemble(h0s, machs, length=3.0, gap=1.0):
    """Independent step flows of different resolutions and Mach numbers in one
    layout: flow k is moved up by k (1 + gap) so no patch of one flow meets
    another flow, and its patches carry its own inflow state."""
    patches, state = [], []
    for k, (h0, M) in enumerate(zip(h0s, machs)):
        inst = ffs_instance(h0=h0, length=length, mach=M, seed=SEED + k)
        dy = k * (1.0 + gap)
        for p, e in zip(inst.patches, inst.state):
            if p.cartesian:
                q = Patch(p.n1, p.n2, p.bc, box=(p.box[0], p.box[1], p.box[2] + dy, p.box[3] + dy), lcut=p.lcut,
                          kind=p.kind, inflow=inst.inflow)
            else:
                q = Patch(p.n1, p.n2, p.bc, x=p.x, y=p.y + dy, lcut=p.lcut, kind=p.kind, inflow=inst.inflow)
            patches.append(q)
            state.append(e)
    return Instance(patches, state, inflow=tuple(float(a) for a in conserved(1.4, machs[0], 0.0, 1.0)), p_out=1.0,
                    name="ffs_ensemble", meta=dict(h0s=list(h0s), machs=list(machs)))


def cylinder_instance(h=0.01, R=0.5, r_out=None, box=(-3.0, 4.0, -3.0, 3.0), sectors=16, mach=10.0, delta_pts=8,
                      seed=SEED, ell=0.15, wall=BC_WALL):
    """Mach-`mach` flow past a circular cylinder of radius R at the origin.

    Body-fitted curvilinear annular sectors (angle along q1, radius along q2,
    wall at r = R) cover R <= r <= r_out and overlap by at least 24 points in
    angle; the rest of `box` is cut into Cartesian cells, 0.25 wide within
    [-1.5, 1.5]^2 and 0.5 wide outside.  Every cell is a patch with a seeded
    spacing h (1 +- 0.15), extended by delta on its internal sides; cells whose
    extended box comes closer than R + 0.1 to the centre are left out (the
    annulus covers them: by default r_out leaves room for such a cell and the
    annulus fringe).  Left: inflow, right: free (supersonic outflow),
    bottom/top: slip walls; the cylinder: a wall of kind `wall` (BC_WALL slip,
    BC_NOSLIP no-slip adiabatic as in §7).  Initial state: the Mach flow (1.4, mach, 0, 1) of §7
    with the velocity brought to rest smoothly at the cylinder wall (factor
    1 - exp(-((r - R)/ell)^2)).
    """
    rng = np.random.default_rng(seed)
    hmax = h * 1.15
    delta = delta_pts * hmax
    r_ex = R + 0.1
    if r_out is None:
        r_out = max(1.2, r_ex + 0.25 * np.sqrt(2.0) + 2 * delta + 12 * hmax)
    r_mid = 0.5 * (R + r_out)
    patches = []
    n2 = int(round((r_out - R) / h)) + 1
    overlap = max(0.35, 24 * hmax / R)
    for k in range(sectors):
        th0 = k * 2 * np.pi / sectors - overlap / 2
        th1 = (k + 1) * 2 * np.pi / sectors + overlap / 2
        hs = h * (1 + 0.15 * rng.uniform(-1.0, 1.0))
        n1 = int(round((th1 - th0) * r_mid / hs)) + 1
        p = annulus_patch(n1, n2, R, r_out, th0, th1, bc=(BC_INTERNAL, BC_INTERNAL, wall, BC_INTERNAL))
        p.kind = "S"
        patches.append(p)
    x0, x1, y0, y1 = box
    cells = []
    for cy0 in np.arange(y0, y1 - 1e-9, 0.5):
        for cx0 in np.arange(x0, x1 - 1e-9, 0.5):
            if -1.5 - 1e-9 <= cx0 < 1.5 - 1e-9 and -1.5 - 1e-9 <= cy0 < 1.5 - 1e-9:
                cells += [(cx0 + a, cx0 + a + 0.25, cy0 + b, cy0 + b + 0.25) for b in (0.0, 0.25) for a in (0.0, 0.25)]
            else:
                cells.append((cx0, cx0 + 0.5, cy0, cy0 + 0.5))
    for cx0, cx1, cy0, cy1 in cells:
        ex0, ex1, ey0, ey1 = cx0 - delta, cx1 + delta, cy0 - delta, cy1 + delta
        dx = 0.0 if ex0 <= 0.0 <= ex1 else min(abs(ex0), abs(ex1))
        dy = 0.0 if ey0 <= 0.0 <= ey1 else min(abs(ey0), abs(ey1))
        if np.hypot(dx, dy) < r_ex:
            continue
        bc = [BC_INTERNAL] * 4
        if abs(cx0 - x0) < 1e-9:
            bc[0] = BC_INFLOW
        if abs(cx1 - x1) < 1e-9:
            bc[1] = BC_FREE
        if abs(cy0 - y0) < 1e-9:
            bc[2] = BC_WALL
        if abs(cy1 - y1) < 1e-9:
            bc[3] = BC_WALL
        b = (cx0 - delta * (bc[0] == BC_INTERNAL), cx1 + delta * (bc[1] == BC_INTERNAL),
             cy0 - delta * (bc[2] == BC_INTERNAL), cy1 + delta * (bc[3] == BC_INTERNAL))
        hh = h * (1 + 0.15 * rng.uniform(-1.0, 1.0))
        patches.append(Patch(int(round((b[1] - b[0]) / hh)) + 1, int(round((b[3] - b[2]) / hh)) + 1, tuple(bc), box=b,
                             kind="I" if all(c == BC_INTERNAL for c in bc) else "S"))
    state = []
    for p in patches:
        X, Y = p.coords()
        f = 1.0 - np.exp(-((np.hypot(X, Y) - R) / ell) ** 2)
        state.append(conserved(np.full(X.shape, 1.4), mach * f, 0.0, 1.0))
    return Instance(patches, state, inflow=tuple(float(a) for a in conserved(1.4, mach, 0.0, 1.0)), p_out=1.0,
                    name="cylinder", meta=dict(h=h, R=R, r_out=r_out, mach=mach, wall=wall))


def mach_flow_state(M, gamma=GAMMA):
    """Uniform Mach-M flow (rho, u, v, p) = (1.4, M, 0, 1) of §7 (sound speed 1)."""
    return (1.4, float(M), 0.0, 1.0)


def mach_shock_state(M, gamma=GAMMA):
    """Post-shock state of a Mach-M shock into (1.4, 0, 0, 1), as printed in §7.

    rho = (gamma+1) M^2 / ((gamma-1) M^2 + 2), u = (zeta-1)/(gamma M), p = zeta,
    zeta = (2 gamma M^2 - gamma + 1)/(gamma + 1).
    """
    zeta = (2 * gamma * M * M - gamma + 1) / (gamma + 1)
    rho = (gamma + 1) * M * M / ((gamma - 1) * M * M + 2)
    return (rho, (zeta - 1) / (gamma * M), 0.0, zeta)


def random_state(patch, rng, amp=0.05):
    """Smooth seeded perturbation of a uniform state (for parity tests)."""
    X, Y = patch.coords()
    k = rng.uniform(1.0, 4.0, size=(4, 2))
    ph = rng.uniform(0, 2 * np.pi, size=4)
    base = (1.0, 0.3, -0.2, 1.0)
    prim = [base[c] * (1 + amp * np.sin(k[c, 0] * X + k[c, 1] * Y + ph[c])) if c in (0, 3)
            else base[c] + amp * np.sin(k[c, 0] * X + k[c, 1] * Y + ph[c]) for c in range(4)]
    return conserved(*prim)


# --------------------------------------------------------------------------
# classifier training windows
# --------------------------------------------------------------------------
WINDOW = 16
CLASS_JUMP, CLASS_KINK, CLASS_C1, CLASS_SMOOTH = 1, 2, 3, 4


def classifier_windows(count, seed=SEED, window=WINDOW):
    """Seeded labelled windows of raw profile samples (count, window), labels 1..4.

    Each window samples s(x) + A * feature(x - x0) on x = 0..window-1, with s a
    random smooth function (sine + linear + constant) and the feature a jump
    (label 1), a kink |x| (label 2), a one-sided square (x)_+^2 (label 3) or
    nothing (label 4), located at a random x0 inside the window.
    """
    rng = np.random.default_rng(seed)
    x = np.arange(window, dtype=np.float64)
    lab = rng.integers(1, 5, size=count)
    amp_s = rng.uniform(0.0, 1.0, size=(count, 1))
    om = rng.uniform(0.0, 0.35, size=(count, 1))
    ph = rng.uniform(0.0, 2 * np.pi, size=(count, 1))
    slope = rng.uniform(-0.2, 0.2, size=(count, 1))
    off = rng.uniform(-1.0, 1.0, size=(count, 1))
    A = rng.uniform(0.3, 2.0, size=(count, 1)) * rng.choice([-1.0, 1.0], size=(count, 1))
    x0 = rng.uniform(3.0, window - 4.0, size=(count, 1))
    s = amp_s * np.sin(om * x + ph) + slope * x + off
    t = x - x0
    feat = np.zeros((count, window))
    feat = np.where(lab[:, None] == CLASS_JUMP, (t >= 0).astype(np.float64), feat)
    feat = np.where(lab[:, None] == CLASS_KINK, np.abs(t) / window * 4.0, feat)
    feat = np.where(lab[:, None] == CLASS_C1, np.maximum(t, 0.0) ** 2 / window ** 2 * 8.0, feat)
    return s + A * feat, lab.astype(np.int8)


# --------------------------------------------------------------------------
# flow states with features at known places (training data of the classifier)
# --------------------------------------------------------------------------
FEATURE_L = 0.03   # localisation length of the kink and C1 features


def feature_profiles(batch, seed=SEED, n1=256, n2=16, per_row=8, gamma=GAMMA):
    """Seeded flow states on one Cartesian patch [0,1] x [0, (n2-1)/(n1-1)]
    (free sides) with features at known places, for `batch` instances.

    Every instance has a smooth background (density, velocity, pressure) and
    `per_row` features on the lines x = a_k + b y (k = 0..per_row-1, a_k near
    the centres of per_row equal bins of [0,1], |b| <= 1, so successive rows
    see a feature up to a grid spacing apart), each of a seeded class: 1 a
    jump, 2 a kink (slope jump), 3 a jump of the second derivative (C1), 4
    none.  With s = x - a_k - b y and t = s / L, a feature changes log(rho),
    log(p) and u by A * f: f = H(s) - 1/2 (jump), |t| exp(-t^2) (kink) and
    t_+^2 exp(-t^2) (C1), L = FEATURE_L, so the features are localised and the
    states stay positive.  Float32 arithmetic (the library's FP32 contexts
    read float states).

    Returns (patch, states, features): states a list of (4, n2, n1) conserved
    arrays, features a dict with 'cls' (batch, per_row) int8, 'a' (batch,
    per_row) and 'b' (batch,) float64.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / (n1 - 1)
    patch = Patch(n1, n2, (BC_FREE,) * 4, box=(0.0, 1.0, 0.0, (n2 - 1) * h))
    X, Y = (c.astype(np.float32)[None] for c in patch.coords())
    B, K = batch, per_row
    cls = rng.integers(1, 5, size=(B, K)).astype(np.int8)
    a = (np.arange(K) + 0.5) / K + rng.uniform(-0.15, 0.15, size=(B, K)) / K
    b = rng.uniform(-1.0, 1.0, size=B)
    om = rng.uniform(0.5, 2.0, size=(B, 4))
    ph = rng.uniform(0.0, 2 * np.pi, size=(B, 4))
    ky = rng.uniform(-2.0, 2.0, size=(B, 4))
    amp = rng.uniform(0.1, 0.5, size=(B, K, 3)) * rng.choice([-1.0, 1.0], size=(B, K, 3))
    f32 = np.float32

    def col(v):
        return np.asarray(v, dtype=f32)[:, None, None]

    def bg(c, scale):
        return f32(scale) * np.sin(f32(2 * np.pi) * col(om[:, c]) * X + col(ky[:, c]) * Y + col(ph[:, c]))

    lrho, u, lp = bg(0, 0.15), f32(0.8) + bg(1, 0.3), bg(2, 0.15)
    v = bg(3, 0.1)
    for k in range(K):
        t = (X - col(a[:, k]) - col(b) * Y) / f32(FEATURE_L)
        g = np.exp(-t * t)
        c = cls[:, k]
        f = (col(c == CLASS_JUMP) * ((t >= 0).astype(f32) - f32(0.5)) + col(c == CLASS_KINK) * np.abs(t) * g
             + col(c == CLASS_C1) * np.square(np.maximum(t, f32(0))) * g)
        lrho += col(amp[:, k, 0]) * f
        u += col(amp[:, k, 1]) * f
        lp += col(amp[:, k, 2]) * f
    rho, p = np.exp(lrho), np.exp(lp)
    E = p / f32(gamma - 1.0) + f32(0.5) * rho * (u * u + v * v)
    st = np.stack([rho, rho * u, rho * v, E], axis=1)
    return patch, list(st), {"cls": cls, "a": a, "b": b}
