"""The allocation-free entry point lbm_conserved_sums_static.

Some callers may not allocate device memory, for example a host program
that only receives device buffers and a stream from another framework's
allocator.  For them the library offers one entry point whose scratch lives
in a static device array; these tests check, through the C ABI, that two
calls in a row give the same totals as lbm_diagnostics and as the DF state
itself, and that lattices beyond the array's capacity are refused.  This
file is collected last so that a failure here stops a run only after every
other test has run."""
import ctypes as C

import numpy as np
import pytest

from paper_1809_08683_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)


@pytest.fixture(scope="module")
def lbm():
    from paper_1809_08683_gb300 import lbm as m
    m.build()
    m.load()
    return m


@pytest.mark.parametrize("precision", [0, 1])
def test_static_sums_match_diagnostics_on_two_calls(lbm, precision):
    import torch
    # no body force, so sum_i g_i is the total energy that lbm_diagnostics reports
    cfg = W.couette(nx=37, ny=80, precision=precision)
    lat = lbm.Lattice(cfg)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device=lat.device)
    for _ in range(2):
        lat.step(150)
        st = lat.L.lbm_conserved_sums_static(lat.h, C.c_void_p(out.data_ptr()))
        assert st == lbm.LBM_OK, lat.L.lbm_last_error()
        lat.stream.synchronize()
        got = out.cpu().numpy()
        d = lat.diagnostics()
        f, g = lat.get_state()
        mass = d["mass"]
        assert abs(got[0] / mass - 1) < 1e-12
        assert abs(got[3] / d["energy"] - 1) < 1e-12
        assert abs(got[1] - (EX[:, None, None] * f).sum()) < 1e-12 * mass
        assert abs(got[2] - (EY[:, None, None] * f).sum()) < 1e-12 * mass
        assert got[1] > 0          # the lid drives net x momentum
    lat.close()


def _check_static(lbm, lat, out):
    st = lat.L.lbm_conserved_sums_static(lat.h, C.c_void_p(out.data_ptr()))
    assert st == lbm.LBM_OK, lat.L.lbm_last_error()
    lat.stream.synchronize()
    got = out.cpu().numpy()
    d = lat.diagnostics()
    f, g = lat.get_state()
    mass = d["mass"]
    assert abs(got[0] / mass - 1) < 1e-12
    assert abs(got[3] / d["energy"] - 1) < 1e-12
    assert abs(got[3] - g.sum()) < 1e-12 * abs(d["energy"])
    assert abs(got[1] - (EX[:, None, None] * f).sum()) < 1e-12 * mass
    assert abs(got[2] - (EY[:, None, None] * f).sum()) < 1e-12 * mass


def test_static_sums_several_blocks_then_one(lbm):
    """A lattice of three blocks of nodes (300 x 300 > 2 x 32768), then a
    one-block lattice right after it: the second call's final pass reads
    only the slot its own first pass wrote, not the larger lattice's."""
    import torch
    big = lbm.Lattice(W.couette(nx=300, ny=300, precision=1))
    small = lbm.Lattice(W.couette(nx=37, ny=80, precision=1))
    out = torch.full((4,), float("nan"), dtype=torch.float64, device=big.device)
    for _ in range(2):
        big.step(40)
        small.step(40)
        _check_static(lbm, big, out)
        _check_static(lbm, small, out)
    big.close()
    small.close()


def test_static_sums_reject_lattices_beyond_capacity(lbm):
    import torch
    cfg = W.periodic_box(8193, 8192, precision=1)   # 1 node row more than 2048 x 32768 nodes
    lat = lbm.Lattice(cfg)
    out = torch.zeros(4, dtype=torch.float64, device=lat.device)
    st = lat.L.lbm_conserved_sums_static(lat.h, C.c_void_p(out.data_ptr()))
    assert st == lbm.LBM_EINVAL
    assert b"at most" in lat.L.lbm_last_error()
    lat.close()
    del lat
    torch.cuda.empty_cache()
