"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, exports every function include/lbm.h declares, and rejects bad
configurations during validation (which runs before any CUDA call)."""
import ctypes as C
import os
import re

import pytest

from paper_1809_08683_gb300 import lbm
from paper_1809_08683_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    lbm.build()
    return lbm.load()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:lbm_status|long|const char\*)\s+(lbm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n
    assert set(lbm.EXPORTS) <= names


def _status(L, cfg):
    n = C.c_size_t()
    return L.lbm_workspace_bytes(C.byref(lbm.make_config(cfg)), C.byref(n)), n.value


def test_validation_accepts_the_workloads(L):
    for cfg in (W.couette(), W.poiseuille(), W.cavity(), W.periodic_box(1, 1), W.cavity(N=4)):
        st, n = _status(L, cfg)
        assert st == lbm.LBM_OK and n > 0


@pytest.mark.parametrize("mutate", [
    lambda c: c.update(nx=0),
    lambda c: c.update(tau0=0.5),
    lambda c: c.update(gamma=1.0),
    lambda c: c.update(ny=3),                        # walled extent below 4
    lambda c: c["walls"][2].update(periodic=0),      # periodic W facing a periodic E
    lambda c: c["walls"][0].update(extrap_order=3),
    lambda c: c.update(precision=7),
    lambda c: c.update(varpi=0.4),
])
def test_validation_rejects_bad_configs(L, mutate):
    cfg = W.couette()
    cfg["walls"] = [dict(w) for w in cfg["walls"]]
    mutate(cfg)
    st, _ = _status(L, cfg)
    assert st == lbm.LBM_EINVAL
    assert L.lbm_last_error()


def test_workspace_grows_with_lattice_and_precision(L):
    _, a = _status(L, W.cavity(N=64, precision=0))
    _, b = _status(L, W.cavity(N=64, precision=1))
    _, c = _status(L, W.cavity(N=128, precision=0))
    assert b < a < c


def test_batch_calls_reject_a_null_batch(L):
    # the argument checks of the batch-level calls run before any CUDA call
    assert L.lbm_batch_init_macros(None, None, None, None, None) == lbm.LBM_EINVAL
    assert L.lbm_batch_macros(None, None, None, None, None, None, None) == lbm.LBM_EINVAL
    assert L.lbm_batch_diagnostics(None, 0, None, None) == lbm.LBM_EINVAL
    assert L.lbm_last_error()


def test_host_field_checks():
    # the batch transfer calls pass host arrays by pointer: only C-contiguous
    # float64 arrays of the lattice's shape are accepted
    import numpy as np
    import types
    lat = types.SimpleNamespace(nx=5, ny=3)
    a = np.zeros((3, 5))
    assert lbm._host_field(a, lat) is a
    for bad in (np.zeros((3, 5), dtype=np.float32), np.zeros((5, 3)), np.zeros((3, 10))[:, ::2], [[0.0] * 5] * 3):
        with pytest.raises(ValueError):
            lbm._host_field(bad, lat)
    ro = np.zeros((3, 5))
    ro.flags.writeable = False
    lbm._host_field(ro, lat)
    with pytest.raises(ValueError):
        lbm._host_field(ro, lat, writable=True)
