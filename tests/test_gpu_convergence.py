"""Solves run to residual targets of 1e-8, through the serving loop: FP32 deviation storage until its stochastic-rounding noise
floor stops the residual from falling, then FP64 storage from the same state
(lbm_copy_state) down to the target.  The results are checked against the
same problem solved in FP64 alone and against Table 2 of the paper."""
import numpy as np
import pytest

from paper_1809_08683_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1809_08683_gb300 import lbm, serve
    lbm.build()
    lbm.load()
    return lbm, serve


def _solve(serve, cfg, tol, max_steps):
    req = serve.Request(rid=0, cfg=cfg, tol=tol, max_steps=max_steps)
    srv = serve.Server(max_slots=1, chunk=1000, graph_steps=100, keep_fields=True)
    srv.run([req], realtime=False)
    return req


@pytest.mark.parametrize("kind", ["cavity", "channel"])
def test_fp32_then_fp64_matches_fp64_alone(mods, kind):
    lbm, serve = mods
    if kind == "cavity":
        cfg = W.cavity(N=64, Ra=1e3, eps=0.5, precision=1)
    else:
        cfg = W.poiseuille(nx=8, ny=48, eos=(W.EOS_IDEAL, ()), gamma=1.4, precision=1)
    mixed = _solve(serve, cfg, 1e-8, 400_000)
    alone = _solve(serve, dict(cfg, precision=0), 1e-8, 400_000)
    assert mixed.status == alone.status == "converged"
    assert mixed.switched_at is not None and mixed.switched_at < mixed.steps
    assert mixed.result["residual"] < 1e-8
    a, b = mixed.result["fields"], alone.result["fields"]
    umax = np.hypot(b["ux"], b["uy"]).max()
    assert max(np.abs(a["ux"] - b["ux"]).max(), np.abs(a["uy"] - b["uy"]).max()) / umax < 1e-5
    assert np.abs(a["T"] - b["T"]).max() / max(np.abs(b["T"] - 1).max(), 1e-300) < 1e-4
    assert np.abs(a["rho"] - b["rho"]).max() / np.abs(b["rho"] - 1).max() < 1e-4
    if kind == "cavity":
        assert abs(mixed.result["nusselt"] / alone.result["nusselt"] - 1) < 1e-5


def test_cavity512_ra1e6_reaches_1e8_and_table2(mods):
    """The 512^2 cavity at Ra = 1e6, eps = 0.6 to r < 1e-8 (Table 2:
    Nu_ave 8.7406, p*_ave 0.91820; agreement within 0.5%)."""
    lbm, serve = mods
    cfg = W.cavity(N=512, Ra=1e6, eps=0.6, precision=1)
    req = _solve(serve, cfg, 1e-8, 2_000_000)
    assert req.status == "converged" and req.result["residual"] < 1e-8
    assert req.switched_at is not None
    assert abs(req.result["nusselt"] / 8.7406 - 1) < 5e-3
    assert abs(req.result["pstar"] / 0.91820 - 1) < 5e-3
