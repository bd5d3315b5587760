"""Batch-level entry points through the C ABI: diagnostics of every member
in one pass (the serving loop's residual check)."""
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


def _mix():
    return [W.cavity(N=40, Ra=1e3, eps=0.6, tau0=0.7),
            W.cavity(N=70, Ra=2e3, eps=0.3, eos=(W.EOS_CUBIC, (0.05, 0.2)), precision=1),
            W.poiseuille(nx=5, ny=33),
            W.couette(nx=130, ny=12, precision=1),
            W.cavity(N=200, Ra=1e4, eps=0.5, precision=1)]


def test_batch_diagnostics_equal_lone_diagnostics(lbm):
    import torch
    stream = torch.cuda.Stream()
    cfgs = _mix()
    a = [lbm.Lattice(c, stream=stream) for c in cfgs]
    b = [lbm.Lattice(c, stream=stream) for c in cfgs]
    ba = lbm.Batch(a, graph_steps=0)
    bb = lbm.Batch(b, graph_steps=0)
    for rnd in range(3):
        ba.step(150)
        bb.step(150)
        lone = [lat.diagnostics(snapshot=True) for lat in a]
        batched = bb.diagnostics(snapshot=True)
        for (d, st), e in zip(batched, lone):
            assert st == lbm.LBM_OK
            for k in e:
                if rnd == 0 and k == "residual":
                    continue          # no snapshot before the first call
                assert d[k] == e[k], (k, d[k], e[k])
    assert batched[0][0]["residual"] > 0
    ba.close()
    bb.close()


def test_batch_diagnostics_reports_an_unstable_member(lbm):
    import torch
    stream = torch.cuda.Stream()
    cfgs = _mix()[:3]
    lats = [lbm.Lattice(c, stream=stream) for c in cfgs]
    f, g = lats[1].get_state()
    f[3, 5, 7] = np.nan
    lats[1].set_state(f, g)
    batch = lbm.Batch(lats, graph_steps=0)
    batch.step(2)
    out = batch.diagnostics()
    assert [st for _, st in out] == [lbm.LBM_OK, lbm.LBM_EUNSTABLE, lbm.LBM_OK]
    assert out[1][0]["nonfinite"] > 0 and out[0][0]["nonfinite"] == 0
    # sticky: the batch refuses to step, a second pass reports it again
    assert batch.L.lbm_batch_step(batch.h, 2) == lbm.LBM_EUNSTABLE
    out = batch.diagnostics()
    assert out[1][1] == lbm.LBM_EUNSTABLE and np.isnan(out[1][0]["mass"])
    batch.close()
