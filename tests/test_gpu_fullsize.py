"""The benchmark's own configuration at full size: the 96-cavity batch in
FP32 deviation storage, stepped as one batch in its default launch shapes
(paired block strips with the cavity-model instance), with sampled members
compared to the FP64 oracle, which steps those lattices on their own."""
import numpy as np
import pytest

from paper_1809_08683_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


@pytest.fixture(scope="module")
def lbm():
    from paper_1809_08683_gb300 import lbm as m
    m.build()
    m.load()
    return m


def test_batched_sweep_sampled_members_match_oracle(orc, lbm):
    import torch
    cfgs = W.batched_sweep(precision=1)
    stream = torch.cuda.Stream()
    lats = [lbm.Lattice(c, stream=stream) for c in cfgs]
    sides = [c["nx"] for c in cfgs]
    picks = [sides.index(1024), sides.index(192)]
    oracles = {}
    for i in picks:
        assert lats[i].tile()[2] == 1                  # paired block strips, as bench.py times them
        nx, ny = cfgs[i]["nx"], cfgs[i]["ny"]
        fields = W.random_macros(nx, ny, 500 + i)
        o = orc.Oracle(cfgs[i], threads=16)
        o.init_macros(*fields)
        lats[i].init_macros(*fields)
        oracles[i] = o
    batch = lbm.Batch(lats, graph_steps=0)
    batch.step(20)
    for i in picks:
        assert oracles[i].step(20) == 0
        mg, mo = lats[i].macros(), oracles[i].macros()
        umax = np.hypot(mo["ux"], mo["uy"]).max()
        err = {"rho": np.abs(mg["rho"] - mo["rho"]).max() / np.abs(mo["rho"]).max(),
               "ux": np.abs(mg["ux"] - mo["ux"]).max() / umax,
               "uy": np.abs(mg["uy"] - mo["uy"]).max() / umax,
               "T": np.abs(mg["T"] - mo["T"]).max() / np.abs(mo["T"]).max()}
        assert all(v < TOL32 for v in err.values()), (sides[i], err)
        # deviations from the rest state, each against its own size
        dev = {"rho_dev": np.abs(mg["rho"] - mo["rho"]).max() / np.abs(mo["rho"] - 1.0).max(),
               "T_dev": np.abs(mg["T"] - mo["T"]).max() / np.abs(mo["T"] - 1.0).max()}
        assert all(v < 1e-3 for v in dev.values()), (sides[i], dev)
    batch.close()
