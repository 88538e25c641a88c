"""Closed-form solutions used to pin the oracle (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module.

  * exact Riemann solver for the 1D Euler equations (Godunov's method as in
    Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", Ch. 4:
    pressure function, Newton iteration for p*, sampling in x/t) - pins the
    shock-tube workload (§7 energy test uses the Sod states);
  * oblique-shock relation of §7 (wedge test): tan(theta) = 2 cot(beta)
    (M^2 sin^2 beta - 1) / (M^2 (gamma + cos 2 beta) + 2), solved for the
    weak-shock angle beta;
  * Rankine-Hugoniot jump of a normal shock (checks the Mach-M shock states).
"""
import numpy as np


def _f_side(p, rho, pk, gamma):
    """Toro's pressure function f_K and its derivative for one side."""
    c = np.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = np.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    r = p / pk
    f = 2.0 * c / (gamma - 1.0) * (r ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
    df = 1.0 / (rho * c) * r ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def riemann_star(left, right, gamma=1.4, tol=1e-15):
    """Star-region (p*, u*) for primitive states (rho, u, p) on each side."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(tol, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _f_side(p, rl, pl, gamma)
        fr, dfr = _f_side(p, rr, pr, gamma)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, tol)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_side(p, rl, pl, gamma)
    fr, _ = _f_side(p, rr, pr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def riemann_sample(left, right, xi, gamma=1.4):
    """Primitive (rho, u, p) of the exact solution at similarity variable x/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = riemann_star(left, right, gamma)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    out = np.zeros((3, xi.size))
    g = gamma
    cl = np.sqrt(g * pl / rl)
    cr = np.sqrt(g * pr / rr)
    for n, s in enumerate(xi):
        if s <= us:
            if ps > pl:                                   # left shock
                sl = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    out[:, n] = (rl, ul, pl)
                else:
                    r = rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)
                    out[:, n] = (r, us, ps)
            else:                                         # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - cl:
                    out[:, n] = (rl, ul, pl)
                elif s >= us - csl:
                    out[:, n] = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    fac = 2 / (g + 1) + (g - 1) / ((g + 1) * cl) * (ul - s)
                    out[:, n] = (rl * fac ** (2 / (g - 1)),
                                 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s),
                                 pl * fac ** (2 * g / (g - 1)))
        else:
            if ps > pr:                                   # right shock
                sr = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    out[:, n] = (rr, ur, pr)
                else:
                    r = rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)
                    out[:, n] = (r, us, ps)
            else:                                         # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + cr:
                    out[:, n] = (rr, ur, pr)
                elif s <= us + csr:
                    out[:, n] = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    fac = 2 / (g + 1) - (g - 1) / ((g + 1) * cr) * (ur - s)
                    out[:, n] = (rr * fac ** (2 / (g - 1)),
                                 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s),
                                 pr * fac ** (2 * g / (g - 1)))
    return out


def right_shock_speed(left, right, gamma=1.4):
    ps, _ = riemann_star(left, right, gamma)
    rr, ur, pr = right
    cr = np.sqrt(gamma * pr / rr)
    return ur + cr * np.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))


def oblique_shock_angle(M, theta, gamma=1.4):
    """Weak-shock angle beta (radians) for deflection theta (radians), §7 wedge."""
    def resid(beta):
        return (2.0 / np.tan(beta) * (M * M * np.sin(beta) ** 2 - 1.0)
                / (M * M * (gamma + np.cos(2 * beta)) + 2.0) - np.tan(theta))
    lo = np.arcsin(1.0 / M) + 1e-12
    # the weak root lies below the angle of maximum deflection
    grid = np.linspace(lo, np.pi / 2 - 1e-9, 20001)
    vals = np.array([resid(b) for b in grid])
    k = int(np.argmax(vals > 0))
    a, b = grid[k - 1], grid[k]
    for _ in range(200):
        m = 0.5 * (a + b)
        if resid(m) > 0:
            b = m
        else:
            a = m
    return 0.5 * (a + b)


def normal_shock_jump(rho1, u1, p1, speed, gamma=1.4):
    """State behind a normal shock moving at `speed` into (rho1, u1, p1) (R-H)."""
    c1 = np.sqrt(gamma * p1 / rho1)
    M = (speed - u1) / c1
    rho2 = rho1 * (gamma + 1) * M * M / ((gamma - 1) * M * M + 2)
    p2 = p1 * (2 * gamma * M * M - (gamma - 1)) / (gamma + 1)
    u2 = speed - (speed - u1) * rho1 / rho2
    return rho2, u2, p2
