"""The heated cavity of Sec. 4.3 on the GPU at the grids of Table 1, run to
steady state and compared with the paper's own results in Table 2 (mean
Nusselt number on the hot wall and mean pressure p*_ave).

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
    print(f"Ra {ref['Ra']:g} N {ref['N']}: {steps} steps, Nu {nu:.5f} ({ref['Nu_ave']}), p* {pstar:.5f} "
          f"({ref['p_ave_star']}), cold wall {-lat.nusselt(W.WALL_E):.5f}")
    batch.close()
