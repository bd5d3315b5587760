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


def test_graph_batch_of_large_lattices_equals_alone(lbm):
    """Lattices large enough for the batch's shortened last runs and its
    cavity-model launch group, replayed from a graph: every member gets the
    bits it gets stepped alone, FP32 and FP64 members alike, from odd and
    even starting steps, and per-step launches after the graph continue
    from the same step counts."""
    import torch
    stream = torch.cuda.Stream()
    cfgs = [W.cavity(N=1024, Ra=1e6, eps=0.5, precision=1),
            W.cavity(N=1024, Ra=3e6, eps=0.3, eos=(W.EOS_CUBIC, (0.05, 0.2)), precision=1),
            W.cavity(N=768, Ra=1e5, eps=0.6, precision=1),
            W.cavity(N=300, Ra=1e4, eps=0.5),
            W.poiseuille(nx=200, ny=190, precision=1)]
    alone = [lbm.Lattice(c, stream=stream) for c in cfgs]
    mixed = [lbm.Lattice(c, stream=stream) for c in cfgs]
    for a, m in zip(alone[::2], mixed[::2]):
        a.step(3)
        m.step(3)
    batch = lbm.Batch(mixed, graph_steps=10)
    batch.step(30)
    for a in alone:
        a.step(30)
    stream.synchronize()
    for a, m in zip(alone, mixed):
        assert a.steps == m.steps
        fa, ga = a.get_state()
        fm, gm = m.get_state()
        assert np.array_equal(fa, fm) and np.array_equal(ga, gm)
    # per-step launches after the graph continue from the same step counts
    batch.step_profiled(4)
    for a in alone:
        a.step(4)
    stream.synchronize()
    for a, m in zip(alone, mixed):
        fa, _ = a.get_state()
        fm, _ = m.get_state()
        assert np.array_equal(fa, fm)
    batch.close()
    for lat in alone + mixed:
        lat.close()


def test_batch_add_remove_keep_bits(lbm):
    """Members joined with lbm_batch_add or left with lbm_batch_remove get
    the same bits as lattices stepped alone; the handle stays usable."""
    import torch
    stream = torch.cuda.Stream()
    cfgs = _mix()[:4]
    alone = [lbm.Lattice(c, stream=stream) for c in cfgs]
    mixed = [lbm.Lattice(c, stream=stream) for c in cfgs]
    batch = lbm.Batch(mixed[:2], graph_steps=10)
    batch.step(20)
    for a in alone[:2]:
        a.step(20)
    mixed[2].step(5)
    alone[2].step(5)
    batch.add(mixed[2])                      # joins at an odd step count
    batch.add(mixed[3])
    batch.step(30)
    for a in alone[:4]:
        a.step(30)
    batch.remove(mixed[0])
    assert batch.L.lbm_batch_remove(batch.h, mixed[0].h) == lbm.LBM_EINVAL     # not a member any more
    assert batch.L.lbm_batch_add(batch.h, mixed[1].h) == lbm.LBM_EINVAL        # already one
    batch.step(10)
    for a in alone[1:]:
        a.step(10)
    mixed[0].step(10)                         # the removed lattice steps on alone
    alone[0].step(10)
    out = batch.diagnostics()
    assert [st for _, st in out] == [lbm.LBM_OK] * 3
    stream.synchronize()
    for a, m in zip(alone, mixed):
        assert a.steps == m.steps
        fa, ga = a.get_state()
        fm, gm = m.get_state()
        assert np.array_equal(fa, fm) and np.array_equal(ga, gm)
    for lat in mixed[1:3]:
        batch.remove(lat)
    assert batch.L.lbm_batch_remove(batch.h, mixed[3].h) == lbm.LBM_EINVAL     # the last member stays
    batch.close()


def test_batch_host_transfers_equal_lone_calls(lbm):
    """lbm_batch_init_macros and lbm_batch_macros give every member the
    bits lbm_init_macros and lbm_macros give it alone, FP32 and FP64
    members alike, pinned and pageable host arrays, with fields skipped
    for all members (a NULL array) or for one member (a NULL entry)."""
    import torch
    stream = torch.cuda.Stream()
    cfgs = _mix()
    alone = [lbm.Lattice(c, stream=stream) for c in cfgs]
    mixed = [lbm.Lattice(c, stream=stream) for c in cfgs]
    batch = lbm.Batch(mixed, graph_steps=0)
    fields = []
    for k, c in enumerate(cfgs):
        f = W.random_macros(c["nx"], c["ny"], seed=100 + k, drho=0.01, du=0.01, dT=0.02)
        if k % 2:   # pinned copies for every other member
            f = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in f]
        fields.append([np.ascontiguousarray(a) for a in f])
    for lat, f in zip(alone, fields):
        lat.init_macros(*f)
    batch.init_macros(fields)
    for a, m in zip(alone, mixed):
        fa, ga = a.get_state()
        fm, gm = m.get_state()
        assert np.array_equal(fa, fm) and np.array_equal(ga, gm)
    batch.step(40)
    for a in alone:
        a.step(40)
    stream.synchronize()
    out = []
    for k, c in enumerate(cfgs):
        keys = ("rho", "ux", "uy", "T") if k == 2 else ("rho", "ux", "uy", "T", "p")
        out.append({q: np.full((c["ny"], c["nx"]), np.nan) for q in keys})
    assert batch.macros(out) == [lbm.LBM_OK] * len(cfgs)
    for k, (a, o) in enumerate(zip(alone, out)):
        ref = a.macros()
        for q, v in o.items():
            assert np.array_equal(v, ref[q]), (k, q)
    only_T = [{"T": np.empty((c["ny"], c["nx"]))} for c in cfgs]
    assert batch.macros(only_T) == [lbm.LBM_OK] * len(cfgs)
    for a, o in zip(alone, only_T):
        assert np.array_equal(o["T"], a.macros()["T"])
    # a NULL entry of the required init fields is refused before any work
    bad = [list(f) for f in fields]
    n = len(cfgs)
    cols = [(lbm.C.POINTER(lbm.C.c_double) * n)(*[lbm._ptr(bad[k][q]) for k in range(n)]) for q in range(4)]
    cols[1][3] = None
    assert batch.L.lbm_batch_init_macros(batch.h, *cols) == lbm.LBM_EINVAL
    batch.close()
