"""Euler operator, boundary conditions, RK stages, patch exchange, Δt, sums (oracle).

Test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module.

Follows:
  * Eq. (1)-(3): 2D Euler equations in conservative form, e = (rho, rho u,
    rho v, E), E = p/(gamma-1) + rho |u|^2 / 2;
  * Algorithm 5 / §5 item 1: the operator in parameter space built from FC
    derivatives and the Jacobian of the inverse patch map.  Reading used here:
    conservative contravariant form
        L(e) = -(1/J) [ d/dq1 (y_q2 f - x_q2 g) + d/dq2 (-y_q1 f + x_q1 g) ],
    J = x_q1 y_q2 - x_q2 y_q1, with the metrics obtained by the same FC
    derivative of the grid coordinates; on Cartesian patches this is
    L(e) = -(df/dx + dg/dy) with FC derivatives at the physical spacings;
  * artificial viscosity term (reading; the paper's form is in Part I):
    d_t e + div f = div(mu grad e), folded into the fluxes as
    f - mu de/dx, g - mu de/dy (on curvilinear patches the physical gradient
    comes from the chain rule with the same metrics); the normal viscous flux
    is zero on wall, outflow and free sides (impermeable, adiabatic for the
    diffusion term: the parabolic term needs a condition on every variable);
  * §5 item 4 / Algorithm 1: explicit four-stage Runge-Kutta (classical RK4
    coefficients, reading of "SSPRK-4"), boundary conditions enforced after
    every stage, exchange of fringe values after every stage;
  * §3.3: n_f-point fringes of internal sides receive values from donor points
    of other patches that are not themselves receivers; coincident grids copy,
    other grids interpolate (tensor Lagrange, 6 x 6 donor nodes, reading of
    I-3.4), the donor parameter found by Newton's method on the donor map;
  * Δt (reading of I-(31)): min over points of 1 / (1/dt_a + 1/dt_v) with
        dt_a = CFL min_k h_k / (|U_k| + c |grad q_k|),
        dt_v = CFL_MU / (mu (1/s_1^2 + 1/s_2^2))   (only where mu > 0),
    U_k the contravariant velocity along parameter direction k, h_k the
    parameter spacing, s_k the physical spacing along q_k and CFL_MU = 0.2: the
    FC diffusion operator has eigenvalues down to about -9.5/s^2 per direction,
    and RK4 is stable on the negative real axis down to -2.78.
"""
import numpy as np

from paper_2506_19370_gb300 import inputs as I
from . import fcgram

RK4_A = (0.5, 0.5, 1.0)          # e_{s+1} = e_n + a_s dt k_s
RK4_B = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


def pressure(e, gamma):
    rho, mx, my, E = e
    return (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / rho)


def fluxes(e, gamma):
    """Physical fluxes f (x) and g (y) of Eq. (1)."""
    rho, mx, my, E = e
    u = mx / rho
    v = my / rho
    p = pressure(e, gamma)
    f = np.stack([mx, mx * u + p, my * u, (E + p) * u])
    g = np.stack([my, mx * v, my * v + p, (E + p) * v])
    return f, g


class PatchGeom:
    """Per-patch quantities the operator needs: spacings, metrics, line segments.

    Grid lines of an L-shaped patch (§3.2, parameter space L) are the
    segments of the rows and columns that lie in the patch: rows j < m2 and
    columns i < m1 are shorter; every segment is differentiated on its own,
    with its own continuation length.
    """

    def __init__(self, patch, d, C, c_policy=0):
        self.patch = patch
        self.d, self.C, self.c_policy = d, C, c_policy
        # continuation length per direction (full lines along q1 have n1 points)
        self.C1 = self.C_of(patch.n1)
        self.C2 = self.C_of(patch.n2)
        self.n1, self.n2 = patch.n1, patch.n2
        self.h1 = 1.0 / (patch.n1 - 1)
        self.h2 = 1.0 / (patch.n2 - 1)
        self.active = patch.active()
        if patch.cartesian:
            x0, x1, y0, y1 = patch.box
            self.hx = (x1 - x0) / (patch.n1 - 1)
            self.hy = (y1 - y0) / (patch.n2 - 1)
            self.x_q1 = np.full((self.n2, self.n1), x1 - x0)
            self.y_q2 = np.full((self.n2, self.n1), y1 - y0)
            self.x_q2 = np.zeros((self.n2, self.n1))
            self.y_q1 = np.zeros((self.n2, self.n1))
        else:
            X, Y = patch.coords()
            self.x_q1 = self.D(X, 0, self.h1)
            self.x_q2 = self.D(X, 1, self.h2)
            self.y_q1 = self.D(Y, 0, self.h1)
            self.y_q2 = self.D(Y, 1, self.h2)
            for m in (self.x_q1, self.x_q2, self.y_q1, self.y_q2):
                m[~self.active] = 1.0 if m is self.x_q1 or m is self.y_q2 else 0.0
        self.J = self.x_q1 * self.y_q2 - self.x_q2 * self.y_q1

    def C_of(self, N):
        return fcgram.policy_c(N, self.C) if self.c_policy else self.C

    def segments(self, dirn):
        """(index block, line length) of the line segments along q1 (dirn 0) or q2 (1)."""
        n1, n2 = self.patch.n1, self.patch.n2
        m1, m2 = self.patch.lcut if self.patch.is_l else (0, 0)
        if dirn == 0:
            out = [((slice(m2, n2), slice(0, n1)), n1)]
            if m2:
                out.append(((slice(0, m2), slice(m1, n1)), n1 - m1))
        else:
            out = [((slice(0, n2), slice(m1, n1)), n2)]
            if m1:
                out.append(((slice(m2, n2), slice(0, m1)), n2 - m2))
        return out

    def D(self, a, dirn, h, order=1):
        """FC derivative of a (..., n2, n1) along q1 (dirn 0) or q2 (dirn 1),
        segment by segment; zero outside the patch."""
        a = np.asarray(a, dtype=np.float64)
        out = np.zeros_like(a)
        axis = a.ndim - 1 if dirn == 0 else a.ndim - 2
        for blk, N in self.segments(dirn):
            idx = (Ellipsis,) + blk
            out[idx] = fcgram.fc_derivative_axis(a[idx], h, self.d, self.C_of(N), axis=axis, order=order)
        return out


def _zero_normal_viscous(V1, V2, patch):
    """Zero normal viscous flux on wall, outflow and free sides, and on the
    inner (wall) edges of an L-shaped patch.  On a no-slip adiabatic wall only
    the mass and energy fluxes vanish (impermeable, adiabatic); the momentum
    flux, the wall shear of the viscous layer, stays."""
    noflux = (I.BC_WALL, I.BC_OUTFLOW, I.BC_FREE)
    bc = patch.bc
    for side, V, idx in ((0, V1, (slice(None), 0)), (1, V1, (slice(None), -1)),
                         (2, V2, (0, slice(None))), (3, V2, (-1, slice(None)))):
        if bc[side] in noflux:
            V[(slice(None),) + idx] = 0.0
        elif bc[side] == I.BC_NOSLIP:
            V[(0,) + idx] = 0.0
            V[(3,) + idx] = 0.0
    if patch.is_l:
        m1, m2 = patch.lcut
        V1[:, :m2, m1] = 0.0
        V2[:, m2, :m1] = 0.0


def rhs(e, geom, d, C, gamma, mu=None):
    """L(e) on one patch (Algorithm 5, operator evaluation); e is (4, n2, n1).

    Points outside an L-shaped patch get zero.
    """
    e = np.asarray(e, dtype=np.float64)
    if geom.patch.is_l:
        # outside values never enter a line segment; keep them harmless
        e = np.where(geom.active, e, np.array([1.0, 0.0, 0.0, 2.5])[:, None, None])
    f, g = fluxes(e, gamma)
    if geom.patch.cartesian:
        if mu is not None:
            vf = mu * geom.D(e, 0, geom.hx)
            vg = mu * geom.D(e, 1, geom.hy)
            _zero_normal_viscous(vf, vg, geom.patch)
            f = f - vf
            g = g - vg
        L = -(geom.D(f, 0, geom.hx) + geom.D(g, 1, geom.hy))
        return np.where(geom.active, L, 0.0)
    F1 = geom.y_q2 * f - geom.x_q2 * g
    F2 = -geom.y_q1 * f + geom.x_q1 * g
    if mu is not None:
        # physical gradient by the chain rule, e_x = (y_q2 e_q1 - y_q1 e_q2)/J,
        # e_y = (-x_q2 e_q1 + x_q1 e_q2)/J; viscous fluxes mu e_x, mu e_y in
        # the same contravariant combination as f, g
        e1 = geom.D(e, 0, geom.h1)
        e2 = geom.D(e, 1, geom.h2)
        ex = (geom.y_q2 * e1 - geom.y_q1 * e2) / geom.J
        ey = (-geom.x_q2 * e1 + geom.x_q1 * e2) / geom.J
        V1 = mu * (geom.y_q2 * ex - geom.x_q2 * ey)
        V2 = mu * (-geom.y_q1 * ex + geom.x_q1 * ey)
        _zero_normal_viscous(V1, V2, geom.patch)
        F1 = F1 - V1
        F2 = F2 - V2
    div = geom.D(F1, 0, geom.h1) + geom.D(F2, 1, geom.h2)
    return np.where(geom.active, -div / geom.J, 0.0)


def chain_variables(e, gamma):
    """w = (rho, rho u, rho v, theta = p / rho): the variables the chain-rule
    form of the operator differentiates (Algorithm 5: density, momenta and
    temperature)."""
    e = np.asarray(e, dtype=np.float64)
    return np.stack([e[0], e[1], e[2], pressure(e, gamma) / e[0]])


def flux_jacobians(w, gamma):
    """A[i][k] = d f_i / d w_k and B[i][k] = d g_i / d w_k at w = (rho, m, n,
    theta), m = rho u, n = rho v, for f, g of Eq. (1) written in w:
    p = rho theta, E = rho theta / (gamma - 1) + (m^2 + n^2) / (2 rho)."""
    rho, m, n, th = w
    u, v = m / rho, n / rho
    q2 = u * u + v * v
    gg = gamma / (gamma - 1.0)
    z, one = np.zeros_like(rho), np.ones_like(rho)
    A = [[z, one, z, z],
         [th - u * u, 2.0 * u, z, rho],
         [-u * v, v, u, z],
         [-u * q2, gg * th + 0.5 * (3.0 * u * u + v * v), u * v, gg * rho * u]]
    B = [[z, z, one, z],
         [-u * v, v, u, z],
         [th - v * v, z, 2.0 * v, rho],
         [-v * q2, u * v, gg * th + 0.5 * (u * u + 3.0 * v * v), gg * rho * v]]
    return np.array(A), np.array(B)


def rhs_chain(e, geom, gamma):
    """L(e) on one patch in the chain-rule form of Algorithm 5 (inviscid):
    FC derivatives of w = (rho, rho u, rho v, theta) along q1 and q2, physical
    derivatives through the inverse Jacobian of the patch map, w_x = (y_q2
    w_q1 - y_q1 w_q2) / J, w_y = (-x_q2 w_q1 + x_q1 w_q2) / J, and the flux
    divergence by the product rule, f_x + g_y = A(w) w_x + B(w) w_y.
    Cartesian patches differentiate at the physical spacings directly."""
    e = np.asarray(e, dtype=np.float64)
    if geom.patch.is_l:
        e = np.where(geom.active, e, np.array([1.0, 0.0, 0.0, 2.5])[:, None, None])
    w = chain_variables(e, gamma)
    A, B = flux_jacobians(w, gamma)
    if geom.patch.cartesian:
        wx = geom.D(w, 0, geom.hx)
        wy = geom.D(w, 1, geom.hy)
    else:
        w1 = geom.D(w, 0, geom.h1)
        w2 = geom.D(w, 1, geom.h2)
        wx = (geom.y_q2 * w1 - geom.y_q1 * w2) / geom.J
        wy = (-geom.x_q2 * w1 + geom.x_q1 * w2) / geom.J
    L = -(np.einsum("ik...,k...->i...", A, wx) + np.einsum("ik...,k...->i...", B, wy))
    return np.where(geom.active, L, 0.0)


def filter_state(e, geom, gamma, alpha=fcgram.FILTER_ALPHA, p=fcgram.FILTER_P):
    """Spectral filter of one patch's state (§5 item 3, Algorithm 4, t > 0).

    Filters rho, rho u, rho v and the temperature theta = p / rho (the energy
    follows from theta: E = rho theta / (gamma - 1) + |rho u|^2 / (2 rho)),
    along q1 then q2, each line segment with its own continuation.  Points
    outside an L-shaped patch keep their values.
    """
    e = np.asarray(e, dtype=np.float64)
    act = geom.active
    safe = np.where(act, e, np.array([1.0, 0.0, 0.0, 2.5])[:, None, None])
    w = np.stack([safe[0], safe[1], safe[2], pressure(safe, gamma) / safe[0]])
    for dirn in (0, 1):
        out = w.copy()
        axis = 2 if dirn == 0 else 1
        for blk, N in geom.segments(dirn):
            idx = (Ellipsis,) + blk
            sub = np.moveaxis(w[idx], axis, -1)
            out[idx] = np.moveaxis(fcgram.fc_filter(sub, geom.d, geom.C_of(N), alpha, p), -1, axis)
        w = out
    rho, mx, my, th = w
    f = np.stack([rho, mx, my, rho * th / (gamma - 1.0) + 0.5 * (mx * mx + my * my) / rho])
    return np.where(act, f, e)


def _side_index(side, n1, n2):
    if side == 0:
        return (slice(None), slice(None), 0)
    if side == 1:
        return (slice(None), slice(None), n1 - 1)
    if side == 2:
        return (slice(None), 0, slice(None))
    return (slice(None), n2 - 1, slice(None))


def _sides(patch):
    """(side, code, index) of every boundary side in application order: left,
    right, bottom, top, then for an L-shaped patch its inner vertical edge
    (i = m1, j < m2; a q1 = const side like left), inner horizontal edge
    (j = m2, i < m1; like bottom), both walls, and the corner node (m1, m2)
    (side -1: wall along the bisector of the two edge normals).  Outer sides
    of an L-shaped patch hold only its points (left: j >= m2, bottom:
    i >= m1)."""
    n1, n2 = patch.n1, patch.n2
    out = []
    for side, code in enumerate(patch.bc):
        idx = _side_index(side, n1, n2)
        if patch.is_l and side == 0:
            idx = (slice(None), slice(patch.lcut[1], n2), 0)
        if patch.is_l and side == 2:
            idx = (slice(None), 0, slice(patch.lcut[0], n1))
        out.append((side, code, idx))
    if patch.is_l:
        m1, m2 = patch.lcut
        out.append((0, I.BC_WALL, (slice(None), slice(0, m2), m1)))
        out.append((2, I.BC_WALL, (slice(None), m2, slice(0, m1))))
        out.append((-1, I.BC_WALL, (slice(None), m2, m1)))
    return out


def neumann_weights(d):
    """Weights w_0..w_{d-1} of the derivative at node 0 of the polynomial that
    interpolates values on the nodes 0, 1, ..., d-1 (unit spacing):
    p'(0) = sum_k w_k f_k.  These are the derivatives at 0 of the Lagrange
    basis polynomials, written out as sums of products."""
    w = np.zeros(d)
    for k in range(d):
        tot = 0.0
        for j in range(d):
            if j == k:
                continue
            term = 1.0 / (k - j)
            for m in range(d):
                if m != k and m != j:
                    term *= (0.0 - m) / (k - m)
            tot += term
        w[k] = tot
    return w


def _inward(side, k, n1, n2):
    """Index (rows, columns) of the points k steps inside from a side."""
    if side == 0:
        return (slice(None), k)
    if side == 1:
        return (slice(None), n1 - 1 - k)
    if side == 2:
        return (k, slice(None))
    return (n2 - 1 - k, slice(None))


def check_noslip(patch):
    """No-slip sides are supported on rectangular patches whose adjacent sides
    are not no-slip (each wall point's inward line then holds no other wall's
    point)."""
    bc = patch.bc
    if I.BC_NOSLIP not in bc:
        return
    if patch.is_l:
        raise ValueError("no-slip sides on an L-shaped patch are not supported")
    for a, b in ((0, 2), (0, 3), (1, 2), (1, 3)):
        if bc[a] == I.BC_NOSLIP and bc[b] == I.BC_NOSLIP:
            raise ValueError("adjacent no-slip sides are not supported")


def apply_bc(e, geom, inst):
    """Boundary conditions of one patch, sides in the order left, right, bottom,
    top (then the inner wall edges of an L-shaped patch).

    Wall: normal momentum removed (Cartesian: the normal component is set to
    zero); inflow: the prescribed conserved state; outflow: energy recomputed
    for the prescribed pressure; no-slip adiabatic wall (§2, §7: zero velocity,
    zero normal derivative of the temperature, enforced through E): momentum
    set to zero, then, once every side's pointwise condition is in place, the
    temperature theta = p / rho of each wall point is the value for which the
    polynomial through theta at the d points of its inward grid line (the
    matching points of the FC-Gram continuation there) has zero derivative
    along that line, and E = rho theta / (gamma - 1).  Acts in place on e
    (4, n2, n1).
    """
    gamma = inst.gamma
    for side, code, idx in _sides(geom.patch):
        if side == -1:
            # corner node of an L-shaped patch: both edge normals, as unit
            # vectors along grad q1 and grad q2 (pointing into the flow), are
            # summed; the velocity component along that bisector is removed
            j, i = idx[1], idx[2]
            sg = np.sign(geom.J[j, i])
            n1 = sg * np.array([geom.y_q2[j, i], -geom.x_q2[j, i]])
            n2 = sg * np.array([-geom.y_q1[j, i], geom.x_q1[j, i]])
            nb = n1 / np.hypot(*n1) + n2 / np.hypot(*n2)
            nb = nb / np.hypot(*nb)
            mn = e[1, j, i] * nb[0] + e[2, j, i] * nb[1]
            e[1, j, i] -= mn * nb[0]
            e[2, j, i] -= mn * nb[1]
            continue
        if code == I.BC_WALL:
            if geom.patch.cartesian:
                comp = 1 if side < 2 else 2
                e[(comp,) + idx[1:]] = 0.0
            else:
                if side < 2:
                    nx, ny = geom.y_q2[idx[1:]], -geom.x_q2[idx[1:]]
                else:
                    nx, ny = -geom.y_q1[idx[1:]], geom.x_q1[idx[1:]]
                nn = np.sqrt(nx * nx + ny * ny)
                nx, ny = nx / nn, ny / nn
                mn = e[(1,) + idx[1:]] * nx + e[(2,) + idx[1:]] * ny
                e[(1,) + idx[1:]] -= mn * nx
                e[(2,) + idx[1:]] -= mn * ny
        elif code == I.BC_INFLOW:
            state = geom.patch.inflow if geom.patch.inflow is not None else inst.inflow
            for c in range(4):
                e[(c,) + idx[1:]] = state[c]
        elif code == I.BC_OUTFLOW:
            rho = e[(0,) + idx[1:]]
            mx = e[(1,) + idx[1:]]
            my = e[(2,) + idx[1:]]
            e[(3,) + idx[1:]] = inst.p_out / (gamma - 1.0) + 0.5 * (mx * mx + my * my) / rho
        elif code == I.BC_NOSLIP:
            e[(1,) + idx[1:]] = 0.0
            e[(2,) + idx[1:]] = 0.0
    if I.BC_NOSLIP in geom.patch.bc:
        check_noslip(geom.patch)
        w = neumann_weights(geom.d)
        n1, n2 = geom.patch.n1, geom.patch.n2
        for side, code in enumerate(geom.patch.bc):
            if code != I.BC_NOSLIP:
                continue
            acc = 0.0
            for k in range(1, geom.d):
                ik = _inward(side, k, n1, n2)
                acc = acc + w[k] * pressure(e[(slice(None),) + ik], gamma) / e[(0,) + ik]
            i0 = _inward(side, 0, n1, n2)
            theta0 = -acc / w[0]
            e[(3,) + i0] = e[(0,) + i0] * theta0 / (gamma - 1.0)
    return e


def receiver_mask(patch, n_f):
    """Points within n_f points of an internal side (the n_f-point fringe, §3.3)."""
    m = np.zeros((patch.n2, patch.n1), dtype=bool)
    b = patch.bc
    if b[0] == I.BC_INTERNAL:
        m[:, :n_f] = True
    if b[1] == I.BC_INTERNAL:
        m[:, patch.n1 - n_f:] = True
    if b[2] == I.BC_INTERNAL:
        m[:n_f, :] = True
    if b[3] == I.BC_INTERNAL:
        m[patch.n2 - n_f:, :] = True
    return m & patch.active()


# ---------------------------------------------------------------------------
# donors and interpolation (§3.3; reading of I-3.4: tensor-product Lagrange
# interpolation on a STENCIL x STENCIL block of donor grid points, in the
# donor's parameter (index) space)
# ---------------------------------------------------------------------------
STENCIL = 6
COPY_TOL = 1e-9     # a receiver this close (in index units) to a donor node copies it
INSIDE_TOL = 1e-6   # slack of the inside-the-donor test (index units): the interpolated
                    # map of a curved donor misses its true boundary by rounding-level amounts


def lagrange_weights(t, m=STENCIL):
    """Values at t of the m Lagrange basis polynomials on the nodes 0..m-1."""
    w = np.ones(m)
    for a in range(m):
        for b in range(m):
            if b != a:
                w[a] *= (t - b) / (a - b)
    return w


def lagrange_dweights(t, m=STENCIL):
    """Derivatives at t of the m Lagrange basis polynomials on 0..m-1: the
    product rule applied factor by factor to prod_{b != a} (t - b), divided by
    prod_{b != a} (a - b)."""
    dw = np.zeros(m)
    for a in range(m):
        val, der, den = 1.0, 0.0, 1.0
        for b in range(m):
            if b != a:
                der = der * (t - b) + val
                val *= t - b
                den *= a - b
        dw[a] = der / den
    return dw


def stencil_start(f, n, m=STENCIL):
    """First node of the m-point stencil around fractional index f (clamped to the line)."""
    return min(max(int(np.floor(f)) - (m // 2 - 1), 0), n - m)


def stencil_block(patch, fi, fj):
    """First node (i0, j0) of the donor block around fractional index (fi, fj).

    On an L-shaped patch a block that would reach into the missing quadrant
    is moved out of it along the direction needing the smaller shift (ties:
    along j), so that every node belongs to the patch.
    """
    i0, j0 = stencil_start(fi, patch.n1), stencil_start(fj, patch.n2)
    if patch.is_l:
        m1, m2 = patch.lcut
        if i0 < m1 and j0 < m2:
            if m2 - j0 <= m1 - i0:
                j0 = m2
            else:
                i0 = m1
    return i0, j0


_CELL_DIAG = {}   # id(patch) -> (patch, largest cell diagonal); the patch is kept so the id stays valid


def donor_index(patch, x, y, max_iter=40):
    """Fractional grid index (fi, fj) of the physical point (x, y) in `patch`.

    Cartesian patches invert their affine map.  Curvilinear patches invert the
    tensor Lagrange interpolant of their grid coordinates by Newton's method,
    starting from the nearest grid point; the stencil follows the iterate.
    Returns None when the iteration leaves the patch or does not converge.
    """
    if patch.cartesian:
        x0, x1, y0, y1 = patch.box
        return (x - x0) / ((x1 - x0) / (patch.n1 - 1)), (y - y0) / ((y1 - y0) / (patch.n2 - 1))
    X, Y = patch.coords()
    d2 = (X - x) ** 2 + (Y - y) ** 2
    k = int(np.argmin(d2))
    # a point of the patch lies within one cell diagonal of a node: farther
    # points are outside (this only saves the Newton iterations)
    key = id(patch)
    if key not in _CELL_DIAG:
        _CELL_DIAG[key] = (patch, float(np.sqrt(max(np.max(np.diff(X, axis=1) ** 2 + np.diff(Y, axis=1) ** 2),
                                                    np.max(np.diff(X, axis=0) ** 2 + np.diff(Y, axis=0) ** 2)) * 2)))
    if d2.flat[k] > (1.01 * _CELL_DIAG[key][1]) ** 2:
        return None
    fj, fi = float(k // patch.n1), float(k % patch.n1)
    for _ in range(max_iter):
        i0, j0 = stencil_start(fi, patch.n1), stencil_start(fj, patch.n2)
        wi, wj = lagrange_weights(fi - i0), lagrange_weights(fj - j0)
        di, dj = lagrange_dweights(fi - i0), lagrange_dweights(fj - j0)
        bx = X[j0:j0 + STENCIL, i0:i0 + STENCIL]
        by = Y[j0:j0 + STENCIL, i0:i0 + STENCIL]
        xm, ym = wj @ bx @ wi, wj @ by @ wi
        a11, a12 = wj @ bx @ di, dj @ bx @ wi
        a21, a22 = wj @ by @ di, dj @ by @ wi
        det = a11 * a22 - a12 * a21
        rx, ry = x - xm, y - ym
        di_ = (a22 * rx - a12 * ry) / det
        dj_ = (-a21 * rx + a11 * ry) / det
        fi += di_
        fj += dj_
        if not (-2.0 <= fi <= patch.n1 + 1.0 and -2.0 <= fj <= patch.n2 + 1.0):
            return None
        # converged well below the interpolation accuracy (index units; a tighter
        # test can sit in the rounding noise of coordinates far from the origin)
        if abs(di_) + abs(dj_) < 1e-10:
            return fi, fj
    return None


class FringeMap:
    """Donor data of every fringe point of one layout.

    copies: int array of rows (dst patch, j, i, src patch, j', i');
    interp: list of (dst patch, j, i, src patch, j0, i0, W) with W the
            STENCIL x STENCIL tensor Lagrange weights on the donor block
            starting at (j0, i0).
    """

    def __init__(self, copies, interp):
        self.copies = np.array(copies, dtype=np.int64).reshape(-1, 6)
        self.interp = interp

    def __len__(self):
        return len(self.copies) + len(self.interp)


def fringe_map(patches, n_f=5):
    """Donor of every fringe point (§3.3: donors are never receivers).

    For each receiver, the donor is the lowest-numbered other patch that
    contains the point and either has a grid node there (copy) or whose
    interpolation stencil holds no receiver of its own (interpolation).
    """
    masks = [receiver_mask(p, n_f) for p in patches]
    usable = [p.active() & ~m for p, m in zip(patches, masks)]   # possible donor nodes
    # bounding boxes, widened generously (a curved side bulges past its nodes):
    # only a shortcut, every patch that can contain a point passes it
    boxes = []
    for p in patches:
        X, Y = p.coords()
        wx, wy = X.max() - X.min(), Y.max() - Y.min()
        boxes.append((X.min() - 0.05 * wx - 1e-12, X.max() + 0.05 * wx + 1e-12,
                      Y.min() - 0.05 * wy - 1e-12, Y.max() + 0.05 * wy + 1e-12))
    copies, interp = [], []
    for p, pt in enumerate(patches):
        X, Y = pt.coords()
        for j, i in zip(*np.nonzero(masks[p])):
            x, y = X[j, i], Y[j, i]
            found = False
            for q, qt in enumerate(patches):
                if q == p:
                    continue
                bx = boxes[q]
                if not (bx[0] <= x <= bx[1] and bx[2] <= y <= bx[3]):
                    continue
                loc = donor_index(qt, x, y)
                if loc is None:
                    continue
                fi, fj = loc
                if not (-INSIDE_TOL <= fi <= qt.n1 - 1 + INSIDE_TOL and -INSIDE_TOL <= fj <= qt.n2 - 1 + INSIDE_TOL):
                    continue
                if qt.is_l and fi < qt.lcut[0] - INSIDE_TOL and fj < qt.lcut[1] - INSIDE_TOL:
                    continue                                   # in the missing quadrant
                ri, rj = int(round(fi)), int(round(fj))
                if abs(fi - ri) <= COPY_TOL and abs(fj - rj) <= COPY_TOL:
                    if not usable[q][rj, ri]:
                        continue
                    copies.append((p, j, i, q, rj, ri))
                    found = True
                    break
                i0, j0 = stencil_block(qt, fi, fj)
                if not usable[q][j0:j0 + STENCIL, i0:i0 + STENCIL].all():
                    continue
                W = np.outer(lagrange_weights(fj - j0), lagrange_weights(fi - i0))
                interp.append((p, j, i, q, j0, i0, W))
                found = True
                break
            if not found:
                raise ValueError(f"no donor for patch {p} point ({j},{i})")
    return FringeMap(copies, interp)


def exchange(state, fmap, clamp=False):
    """Donor values into every fringe point (all leading components).

    Copies first, then interpolations; donors are never receivers, so the
    order does not matter.  clamp=True floors interpolated values at zero
    (used for the viscosity, which must stay non-negative).
    """
    for p, j, i, q, jj, ii in fmap.copies:
        state[p][..., j, i] = state[q][..., jj, ii]
    for p, j, i, q, j0, i0, W in fmap.interp:
        blk = state[q][..., j0:j0 + STENCIL, i0:i0 + STENCIL]
        v = np.sum(blk * W, axis=(-2, -1))
        state[p][..., j, i] = np.maximum(v, 0.0) if clamp else v
    return state


CFL_MU = 0.2


def time_step(state, geoms, gamma, cfl, mu=None):
    """Δt = min over points of 1/(1/dt_a + 1/dt_v) (advective and viscous limits)."""
    best = np.inf
    for k, (e, g) in enumerate(zip(state, geoms)):
        rho, mx, my, E = e
        u, v = mx / rho, my / rho
        c = np.sqrt(gamma * pressure(e, gamma) / rho)
        # grad q1 = (y_q2, -x_q2)/J, grad q2 = (-y_q1, x_q1)/J
        U1 = (g.y_q2 * u - g.x_q2 * v) / g.J
        U2 = (-g.y_q1 * u + g.x_q1 * v) / g.J
        n1 = np.sqrt(g.y_q2 ** 2 + g.x_q2 ** 2) / np.abs(g.J)
        n2 = np.sqrt(g.y_q1 ** 2 + g.x_q1 ** 2) / np.abs(g.J)
        adv = cfl * np.minimum(g.h1 / (np.abs(U1) + c * n1), g.h2 / (np.abs(U2) + c * n2))
        if mu is not None:
            s1 = g.h1 * np.sqrt(g.x_q1 ** 2 + g.y_q1 ** 2)
            s2 = g.h2 * np.sqrt(g.x_q2 ** 2 + g.y_q2 ** 2)
            # 1/dt = 1/dt_a + mu (1/s1^2 + 1/s2^2) / CFL_MU
            adv = 1.0 / (1.0 / adv + mu[k] * (1.0 / (s1 * s1) + 1.0 / (s2 * s2)) / CFL_MU)
        best = min(best, float(np.min(adv[g.active])))
    return best


def max_wave_speed(state, gamma):
    return max(float(np.max(np.sqrt(e[1] ** 2 + e[2] ** 2) / e[0]
                            + np.sqrt(gamma * pressure(e, gamma) / e[0]))) for e in state)


class Solver:
    """Multi-patch FC-SDNN stepping on one instance (Algorithms 1 and 5)."""

    def __init__(self, inst, d=5, C=25, n_f=5, cfl=0.5, c_policy=0, chain=False):
        self.inst = inst
        self.d, self.C, self.n_f, self.cfl = d, C, n_f, cfl
        self.chain = chain      # operator in the chain-rule form (inviscid only)
        for p in inst.patches:
            check_noslip(p)
        self.geoms = [PatchGeom(p, d, C, c_policy) for p in inst.patches]
        self.fmap = fringe_map(inst.patches, n_f)

    def rhs_all(self, state, mu=None):
        if self.chain:
            if mu is not None:
                raise ValueError("the chain-rule operator form is inviscid")
            return [rhs_chain(e, g, self.inst.gamma) for e, g in zip(state, self.geoms)]
        return [rhs(e, g, self.d, self.C, self.inst.gamma, None if mu is None else mu[k])
                for k, (e, g) in enumerate(zip(state, self.geoms))]

    def stage(self, s, dt, e_n, e_s, acc, mu=None):
        """One RK4 stage: returns (e_out, acc); BCs then exchange on e_out."""
        k = self.rhs_all(e_s, mu)
        out, acc_new = [], []
        for p in range(len(e_n)):
            if s == 0:
                a = e_n[p] + (RK4_B[0] * dt) * k[p]
            elif s < 3:
                a = acc[p] + (RK4_B[s] * dt) * k[p]
            else:
                a = None
            o = e_n[p] + (RK4_A[s] * dt) * k[p] if s < 3 else acc[p] + (RK4_B[3] * dt) * k[p]
            apply_bc(o, self.geoms[p], self.inst)
            out.append(o)
            acc_new.append(a)
        exchange(out, self.fmap)
        return out, acc_new

    def filter(self, state):
        """Filter every patch, then boundary conditions and fringe exchange."""
        out = [filter_state(e, g, self.inst.gamma) for e, g in zip(state, self.geoms)]
        for e, g in zip(out, self.geoms):
            apply_bc(e, g, self.inst)
        return exchange(out, self.fmap)

    def step(self, state, dt, mu=None):
        e_n = [e.copy() for e in state]
        e_s, acc = e_n, None
        for s in range(4):
            e_s, acc = self.stage(s, dt, e_n, e_s, acc, mu)
        return e_s

    def dt(self, state, mu=None):
        return time_step(state, self.geoms, self.inst.gamma, self.cfl, mu)

    def quadrature_weights(self, g):
        """Per-point weights of the FC quadrature over the patch's parameter
        space (times |J|: the integral over the patch in physical space; §7
        energy test).  Rectangles: tensor product of the FC quadratures of
        the rows and the columns.  L-shaped parameter space (reading): the
        union of the upper rectangle, rows j >= m2 (full rows), and the lower
        right one, rows j <= m2 and columns i >= m1, which share the segment
        of row m2 to the right of i = m1; each is integrated by the tensor
        product of the FC quadratures of its own line segments (every
        integrand is smooth on each rectangle, while the row integral of the
        whole L has a kink at row m2)."""
        d = self.d
        n1, n2 = g.n1, g.n2

        def W(N, length):
            return fcgram.fc_quadrature_weights(N, d, g.C_of(N)) * length

        if not g.patch.is_l:
            w = np.outer(W(n2, 1.0), W(n1, 1.0))
        else:
            m1, m2 = g.patch.lcut
            w = np.zeros((n2, n1))
            w[m2:, :] += np.outer(W(n2 - m2, (n2 - 1 - m2) / (n2 - 1)), W(n1, 1.0))
            w[:m2 + 1, m1:] += np.outer(W(m2 + 1, m2 / (n2 - 1)), W(n1 - m1, (n1 - 1 - m1) / (n1 - 1)))
        return w * np.abs(g.J)

    def conservation_sums(self, state):
        """Per patch: FC quadrature of each conserved field times |J| (4 sums)."""
        out = []
        for e, g in zip(state, self.geoms):
            w = self.quadrature_weights(g)
            out.append(np.array([np.sum(w * e[c]) for c in range(4)]))
        return np.array(out)
