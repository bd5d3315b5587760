"""The heated cavity of Sec. 4.3 on the GPU at the grids of Table 1, run to
steady state and compared with the paper's own results in Table 2: mean
Nusselt number on the hot wall, mean pressure p*_ave, and the maximum
horizontal (vertical) velocity along the vertical (horizontal) midplane
with its position.

eps = 0.6, ideal gas, Sutherland viscosity, Pr = 0.71, gamma = 1.4,
first-order extrapolation, FP32 deviation storage.  The relaxation time and
the bulk-to-shear viscosity ratio follow this library's stability rule for
the cavity (tau0 from the cold-wall margin, varsigma/nu = 4) rather than the
paper's tau0, which the paper does not print; Table 2 is then met to within
1% (Nu) and 0.5% (p*).  Steady state: the relative change of u and T over
1000 steps below 1e-5, the level FP32 storage resolves at small Ra (its
stochastic rounding keeps the change near 7e-6 at Ra = 1e3), and the
hot-wall Nusselt number changing by less than 1e-4 over 10,000 steps.  (The
cold wall's discrete flux differs from the hot wall's by 0.6-1.5%: the
one-sided wall gradient with a conductivity that varies by a factor of 2.6
across the cavity; the paper's Table 2 reports the hot wall.)"""
import json
import os

import numpy as np
import pytest

from paper_1809_08683_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_1809_08683_gb300 import lbm as m
    m.build()
    m.load()
    return m


def table2():
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_cavity.json")
    with open(path) as fh:
        t = json.load(fh)
    return {int(round(np.log10(r[0]))): dict(zip(t["columns"], r)) for r in t["rows"]}


def midplane(a, axis):
    """Values on the midplane x = L/2 (axis=1) or y = L/2 (axis=0) of a
    [ny][nx] field: the middle column (row), or the mean of the two middle
    ones for an even lattice."""
    n = a.shape[axis]
    take = (lambda i: a[:, i]) if axis == 1 else (lambda i: a[i, :])
    if n % 2:
        return take(n // 2), n // 2
    return 0.5 * (take(n // 2 - 1) + take(n // 2)), n / 2 - 0.5


def peak(v):
    """Maximum of a sampled profile and its position (in nodes), refined by
    the parabola through the largest sample and its two neighbours."""
    i = int(np.argmax(v))
    if 0 < i < len(v) - 1:
        a, b, c = v[i - 1], v[i], v[i + 1]
        den = a - 2 * b + c
        if den < 0:
            d = 0.5 * (a - c) / den
            return b - 0.25 * (a - c) * d, i + d
    return v[i], float(i)


@pytest.mark.parametrize("decade", [3, 4, 5])
def test_cavity_table2(lbm, decade):
    import torch
    ref = table2()[decade]
    cfg = W.cavity(N=int(ref["N"]), Ra=ref["Ra"], eps=0.6, precision=1)
    assert cfg["Ra"] == ref["Ra"]                      # the rule does not lower Ra at these grids
    stream = torch.cuda.Stream()
    lat = lbm.Lattice(cfg, stream=stream)
    batch = lbm.Batch([lat], graph_steps=1000)
    lat.diagnostics(snapshot=True)
    residual, drift, steps, nu_prev = 1.0, 1.0, 0, 0.0
    # steady: u and T settled, and the hot-wall Nusselt number no longer
    # moving (by less than 1e-4 relative over 10,000 steps)
    while (residual > 1e-5 or drift > 1e-4) and steps < 2_000_000:
        batch.step(1000)
        steps += 1000
        residual = lat.diagnostics(snapshot=True)["residual"]
        if steps % 10000 == 0:
            nu_now = lat.nusselt(W.WALL_W)
            drift = abs(nu_now / nu_prev - 1) if nu_prev else 1.0
            nu_prev = nu_now
    assert residual <= 1e-5 and drift <= 1e-4, (steps, residual, drift)
    nu = lat.nusselt(W.WALL_W)
    pstar = lat.diagnostics()["pstar"]
    assert abs(nu / ref["Nu_ave"] - 1) < 0.01, (nu, ref["Nu_ave"])
    assert abs(pstar / ref["p_ave_star"] - 1) < 0.005, (pstar, ref["p_ave_star"])

    # midplane velocity maxima, u* = u / U_ref with U_ref = sqrt(Ra) mu0 / (rho0 L)
    # and positions x* = x / L (Sec. 4.3)
    N, L = cfg["nx"], cfg["nx"] - 1
    uref = np.sqrt(ref["Ra"]) * lat.derived()["mu0"] / (cfg["rho0"] * L)
    m = lat.macros()
    ux_mid, _ = midplane(m["ux"], axis=1)       # along the vertical midplane, as a function of y
    uy_mid, _ = midplane(m["uy"], axis=0)       # along the horizontal midplane, as a function of x
    umax_x, y_at = peak(np.abs(ux_mid))
    umax_y, x_at = peak(np.abs(uy_mid))
    # 2%: the published methods of Table 2 themselves spread by 1.3% on
    # |u_x*|_max at Ra = 1e3 (0.1639 to 0.1660)
    assert abs(umax_x / uref / ref["ux_max"] - 1) < 0.02, (umax_x / uref, ref["ux_max"])
    assert abs(umax_y / uref / ref["uy_max"] - 1) < 0.02, (umax_y / uref, ref["uy_max"])
    assert abs(y_at / L - ref["y_max"]) < 1.5 / L, (y_at / L, ref["y_max"])
    assert abs(x_at / L - ref["x_max"]) < 1.5 / L, (x_at / L, ref["x_max"])
    print(f"Ra {ref['Ra']:g} N {ref['N']}: {steps} steps, Nu {nu:.5f} ({ref['Nu_ave']}), p* {pstar:.5f} "
          f"({ref['p_ave_star']}), cold wall {-lat.nusselt(W.WALL_E):.5f}, ux* {umax_x / uref:.4f} "
          f"({ref['ux_max']}) at y* {y_at / L:.4f} ({ref['y_max']}), uy* {umax_y / uref:.4f} ({ref['uy_max']}) "
          f"at x* {x_at / L:.4f} ({ref['x_max']})")
    batch.close()
