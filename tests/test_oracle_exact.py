"""Pins of the closed-form helpers (exact Riemann solver, shock relations)."""
import json
import os

import numpy as np

from oracle import exact
from paper_2506_19370_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
SOD_L = (1.0, 0.0, 1.0)
SOD_R = (0.125, 0.0, 0.1)


def test_sod_star_state_textbook_values():
    # star state of the Sod problem as tabulated by Toro (Table 4.3, test 1)
    ps, us = exact.riemann_star(SOD_L, SOD_R)
    assert abs(ps - 0.30313) < 1e-5 and abs(us - 0.92745) < 1e-5
    out = exact.riemann_sample(SOD_L, SOD_R, [us - 1e-9, us + 1e-9])
    assert abs(out[0, 0] - 0.42632) < 1e-5 and abs(out[0, 1] - 0.26557) < 1e-5
    assert abs(exact.right_shock_speed(SOD_L, SOD_R) - 1.75216) < 1e-5


def test_riemann_shock_satisfies_rankine_hugoniot():
    S = exact.right_shock_speed(SOD_L, SOD_R)
    behind = exact.riemann_sample(SOD_L, SOD_R, [S - 1e-9])[:, 0]
    rh = exact.normal_shock_jump(*SOD_R, S)
    assert np.allclose(behind, rh, rtol=1e-10)


def test_riemann_rarefaction_is_isentropic():
    xi = np.linspace(-1.1, 0.0, 50)
    rho, u, p = exact.riemann_sample(SOD_L, SOD_R, xi)
    assert np.allclose(p / rho ** 1.4, 1.0, rtol=1e-12)


def test_oblique_shock_angles_printed_in_paper():
    # §7 wedge test, theoretical shock angles for a 40 degree wedge
    # (20 degree deflection): 34.6 (M = 3.5) and 25.8 (M = 10)
    g = GOLDEN["oblique_shock_angle_deg"]
    for M, th in zip(g["mach"], g["theory_deg"]):
        b = np.degrees(exact.oblique_shock_angle(M, np.radians(g["wedge_half_angle_deg"])))
        assert abs(b - th) < g["printed_precision_deg"]


def test_mach_shock_states():
    # §7: zeta(10) = 116.5 and u = 8.25 behind a Mach-10 shock into (1.4, 0, 1)
    g = GOLDEN["mach10_shock"]
    rho, u, v, p = I.mach_shock_state(g["mach"])
    assert abs(p - g["zeta"]) < 1e-12 and abs(u - g["u"]) < 1e-12
    # u and p agree with Rankine-Hugoniot for a shock of speed M c = 10; the
    # printed density formula is the density ratio (ambient 1.4 gives 8.0)
    r2, u2, p2 = exact.normal_shock_jump(1.4, 0.0, 1.0, 10.0)
    assert abs(u2 - u) < 1e-12 and abs(p2 - p) < 1e-12
    assert abs(r2 / 1.4 - rho) < 1e-12


def test_subpatch_point_counts():
    # §7 tables: every unknown count is a whole number of 101 x 101 subpatches
    g = GOLDEN["subpatch_points"]
    assert [n // 101 ** 2 for n in g["N"]] == g["subpatches"]
    assert all(n % 101 ** 2 == 0 for n in g["N"])
