"""Rounding mode of FP32 storage, state copies across precisions, and the
bounded-wait timeout path, through the C ABI."""
import numpy as np
import pytest

from paper_1809_08683_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module")
def lbm():
    from paper_1809_08683_gb300 import lbm as m
    m.build()
    m.load()
    return m


def maxrel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_nearest_rounding_changes_bits_not_results(orc, lbm):
    cfg = W.cavity(N=64, Ra=1e3, eps=0.6, precision=1)
    o = orc.Oracle(cfg, threads=8)
    assert o.step(1500) == 0
    mo = o.macros()
    out = {}
    for mode in (lbm.ROUND_STOCHASTIC, lbm.ROUND_NEAREST):
        g = lbm.Lattice(cfg)
        g.set_rounding(mode)
        g.step(1500)
        out[mode] = g.get_state()
        mg = g.macros()
        umax = np.hypot(mo["ux"], mo["uy"]).max()
        assert np.abs(mg["ux"] - mo["ux"]).max() / umax < TOL32
        assert maxrel(mg["T"], mo["T"]) < TOL32
        g.close()
    assert not np.array_equal(out[0][0], out[1][0])


def test_nearest_rounding_is_reproducible_and_batched_equal(lbm):
    import torch
    stream = torch.cuda.Stream()
    cfgs = [W.cavity(N=70, Ra=2e3, eps=0.4, precision=1), W.poiseuille(nx=5, ny=40, precision=1)]
    a = [lbm.Lattice(c, stream=stream) for c in cfgs]
    b = [lbm.Lattice(c, stream=stream) for c in cfgs]
    for lat in a + b:
        lat.set_rounding(lbm.ROUND_NEAREST)
    for lat in a:
        lat.step(300)
    batch = lbm.Batch(b, graph_steps=10)
    batch.step(300)
    stream.synchronize()
    for x, y in zip(a, b):
        fx, gx = x.get_state()
        fy, gy = y.get_state()
        assert np.array_equal(fx, fy) and np.array_equal(gx, gy)
    batch.close()


def test_set_rounding_rejects_unknown_mode(lbm):
    g = lbm.Lattice(W.periodic_box(8, 8, precision=1))
    assert g.L.lbm_set_rounding(g.h, 7) == lbm.LBM_EINVAL
    g.close()


def test_copy_state_fp32_to_fp64_then_fp64_matches_oracle(orc, lbm):
    """A solve started in FP32 storage and continued in FP64 from the copied
    state follows the FP64 oracle started from that same state to 1e-10."""
    cfg32 = W.cavity(N=61, Ra=3e3, eps=0.6, precision=1)
    cfg32["walls"][1]["u"] = (0.01, 0.0)
    cfg64 = dict(cfg32, precision=0)
    a = lbm.Lattice(cfg32)
    a.step(777)
    a.diagnostics(snapshot=True)
    a.step(100)
    r32 = a.diagnostics()["residual"]
    b = lbm.Lattice(cfg64)
    b.copy_state_from(a)
    assert b.steps == a.steps == 877
    # the residual snapshot moves with the state
    assert abs(b.diagnostics()["residual"] / r32 - 1) < 1e-6
    f, g = a.get_state()
    fb, gb = b.get_state()
    assert np.array_equal(f, fb) and np.array_equal(g, gb)   # FP32 -> FP64 is exact
    o = orc.Oracle(cfg64, threads=8)
    o.set_state(f, g)
    assert o.step(500) == 0
    b.step(500)
    mo, mb = o.macros(), b.macros()
    umax = np.hypot(mo["ux"], mo["uy"]).max()
    assert np.abs(mb["ux"] - mo["ux"]).max() / umax < TOL64
    assert np.abs(mb["uy"] - mo["uy"]).max() / umax < TOL64
    assert maxrel(mb["T"], mo["T"]) < TOL64
    assert maxrel(mb["rho"], mo["rho"]) < TOL64
    a.close()
    b.close()


def test_copy_state_fp64_to_fp32_rounds_once(lbm):
    cfg = W.poiseuille(nx=6, ny=33, precision=0)
    a = lbm.Lattice(cfg)
    a.step(301)
    b = lbm.Lattice(dict(cfg, precision=1))
    b.copy_state_from(a)
    f, g = a.get_state()
    fb, gb = b.get_state()
    # deviations round once to FP32: the full values agree to FP32 rounding
    # of the deviation, far below the FP32 tolerance
    assert np.abs(fb - f).max() < 1e-6 and np.abs(gb - g).max() < 1e-6
    assert b.steps == 301
    b.step(10)          # steps on from an odd count (the other buffer)
    b.sync()
    a.close()
    b.close()


def test_copy_state_rejects_another_problem(lbm):
    a = lbm.Lattice(W.cavity(N=40, Ra=1e3, eps=0.5, precision=1))
    b = lbm.Lattice(W.cavity(N=40, Ra=1e3, eps=0.4, precision=0))
    assert a.L.lbm_copy_state(b.h, a.h) == lbm.LBM_EINVAL
    c = lbm.Lattice(W.cavity(N=40, Ra=1e3, eps=0.5, eos=(W.EOS_CUBIC, (0.05, 0.2)), precision=0))
    assert a.L.lbm_copy_state(c.h, a.h) == lbm.LBM_EINVAL
    for lat in (a, b, c):
        lat.close()


def test_bounded_wait_gives_up_and_reports_timeout(lbm):
    """The fused kernels' bounded mbarrier wait, run on a barrier that no
    copy completes with a limit of a few thousand cycles: it returns, the
    status word reports the timeout, the context turns sticky, and
    re-initialisation clears it."""
    cfg = W.periodic_box(16, 8, precision=1)
    g = lbm.Lattice(cfg)
    assert g.L.lbm_wait_selftest(g.h, 4000) == lbm.LBM_ETIMEOUT
    assert b"bounded wait" in g.L.lbm_last_error()
    assert g.L.lbm_step(g.h, 1) == lbm.LBM_ETIMEOUT        # sticky
    assert g.L.lbm_wait_selftest(g.h, -1) == lbm.LBM_EINVAL
    g.init_macros(*W.random_macros(16, 8, 3))                # re-initialisation clears it
    assert g.status_step(5) == lbm.LBM_OK
    g.close()


def test_peak_rates_are_positive(lbm):
    r = lbm.peak_rates()
    assert all(np.isfinite(v) and v > 1e9 for v in r.values()), r

