"""Thin ctypes binding of the C ABI in include/lbm.h.

Argument marshalling only: every step of the lattice update runs in the CUDA
library (``csrc/lbm_gb300.cu``).  PyTorch supplies device memory (one
workspace tensor per lattice) and the CUDA stream.  There is no CPU fallback:
if the compiled library is missing or no GPU is visible, construction fails.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "lbm_gb300.cu")
_DEPS = [_SRC, os.path.join(_HERE, "csrc", "lbm_node.cuh"), os.path.join(_HERE, "csrc", "lbm_f2.cuh"),
         os.path.join(_HERE, "csrc", "lbm_ff.cuh"), os.path.join(os.path.dirname(_HERE), "include", "lbm.h")]
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "liblbm_gb300.so")
NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-shared"]

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT = 0, -1, -2, -3, -4, -5
FP64, FP32_DEV = 0, 1
ROUND_STOCHASTIC, ROUND_NEAREST = 0, 1

_lock = threading.Lock()
_lib = None


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (in-tree, git-ignored)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _DEPS)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([_nvcc(), *NVCC_FLAGS, "-o", tmp, _SRC])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lbm status {status}: {msg}")
        self.status = status


class WallBC(C.Structure):
    _fields_ = [("periodic", C.c_int32), ("thermal", C.c_int32), ("extrap_order", C.c_int32),
                ("reserved", C.c_int32), ("u", C.c_double * 2), ("T", C.c_double)]


class Config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("precision", C.c_int32),
                ("visc_law", C.c_int32), ("rho0", C.c_double), ("T0", C.c_double),
                ("Pr", C.c_double), ("gamma", C.c_double), ("tau0", C.c_double),
                ("visc_p", C.c_double * 2), ("bulk_ratio", C.c_double), ("varpi", C.c_double),
                ("gamma1", C.c_double), ("gamma2", C.c_double), ("force_mode", C.c_int32),
                ("corrections", C.c_int32), ("force", C.c_double * 2), ("wall", WallBC * 4)]


EXPORTS = ("lbm_workspace_bytes", "lbm_create", "lbm_set_eos", "lbm_step", "lbm_sync", "lbm_macros",
           "lbm_macros_device", "lbm_nusselt", "lbm_diagnostics", "lbm_get_state", "lbm_set_state",
           "lbm_init_macros", "lbm_derived", "lbm_set_tile", "lbm_get_tile", "lbm_step_count", "lbm_destroy",
           "lbm_last_error", "lbm_batch_create", "lbm_batch_step", "lbm_batch_step_profiled",
           "lbm_batch_destroy", "lbm_conserved_sums_static", "lbm_set_rounding", "lbm_copy_state",
           "lbm_wait_selftest", "lbm_batch_diagnostics", "lbm_batch_add", "lbm_batch_remove",
           "lbm_peak_rates", "lbm_batch_init_macros", "lbm_batch_macros")


def load(path: str | None = None):
    """Load the compiled library (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is None:
            path = os.environ.get("LBM_LIBRARY") or (LIB_PATH if os.path.exists(LIB_PATH) else build())
        L = C.CDLL(path)
        P = C.POINTER
        vp, dp, i, cfgp = C.c_void_p, P(C.c_double), C.c_int, P(Config)
        L.lbm_workspace_bytes.argtypes = [cfgp, P(C.c_size_t)]
        L.lbm_create.argtypes = [cfgp, vp, C.c_size_t, vp, P(vp)]
        L.lbm_set_eos.argtypes = [vp, i, dp, i]
        L.lbm_step.argtypes = [vp, C.c_long]
        L.lbm_sync.argtypes = [vp]
        L.lbm_macros.argtypes = [vp, dp, dp, dp, dp, dp]
        L.lbm_macros_device.argtypes = [vp, vp, vp, vp, vp, vp]
        L.lbm_nusselt.argtypes = [vp, i, dp]
        L.lbm_diagnostics.argtypes = [vp, i, dp]
        L.lbm_get_state.argtypes = [vp, dp, dp]
        L.lbm_set_state.argtypes = [vp, dp, dp]
        L.lbm_init_macros.argtypes = [vp, dp, dp, dp, dp]
        L.lbm_derived.argtypes = [vp, dp]
        L.lbm_set_tile.argtypes = [vp, i, i, i]
        L.lbm_get_tile.argtypes = [vp, P(i), P(i), P(i)]
        L.lbm_step_count.argtypes = [vp]
        L.lbm_step_count.restype = C.c_long
        L.lbm_destroy.argtypes = [vp]
        L.lbm_last_error.argtypes = []
        L.lbm_last_error.restype = C.c_char_p
        L.lbm_batch_create.argtypes = [P(vp), i, i, P(vp)]
        L.lbm_batch_step.argtypes = [vp, C.c_long]
        L.lbm_batch_step_profiled.argtypes = [vp, C.c_long, dp, dp]
        L.lbm_batch_destroy.argtypes = [vp]
        L.lbm_conserved_sums_static.argtypes = [vp, vp]
        L.lbm_set_rounding.argtypes = [vp, i]
        L.lbm_copy_state.argtypes = [vp, vp]
        L.lbm_wait_selftest.argtypes = [vp, C.c_longlong]
        L.lbm_batch_diagnostics.argtypes = [vp, i, dp, P(C.c_int)]
        L.lbm_batch_add.argtypes = [vp, vp]
        L.lbm_peak_rates.argtypes = [vp, dp]
        L.lbm_batch_remove.argtypes = [vp, vp]
        L.lbm_batch_init_macros.argtypes = [vp, P(dp), P(dp), P(dp), P(dp)]
        L.lbm_batch_macros.argtypes = [vp, P(dp), P(dp), P(dp), P(dp), P(dp), P(C.c_int)]
        _lib = L
        return L


def _check(L, st):
    if st != LBM_OK:
        raise LbmError(st, L.lbm_last_error().decode(errors="replace"))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _host_field(a, lat, writable=False):
    """Check that a is an FP64 C-contiguous host array of the lattice's
    shape (it is passed to the library by pointer, not copied)."""
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous \
            or a.shape != (lat.ny, lat.nx) or (writable and not a.flags.writeable):
        raise ValueError(f"expected a C-contiguous float64 array of shape {(lat.ny, lat.nx)}")
    return a


def make_config(cfg: dict) -> Config:
    k = Config()
    k.nx, k.ny = int(cfg["nx"]), int(cfg["ny"])
    k.precision = int(cfg.get("precision", FP64))
    k.visc_law = int(cfg.get("visc_law", 0))
    k.rho0, k.T0, k.Pr = cfg["rho0"], cfg["T0"], cfg["Pr"]
    k.gamma, k.tau0 = cfg["gamma"], cfg["tau0"]
    vp = cfg.get("visc_p", (0.0, 0.0))
    k.visc_p[0], k.visc_p[1] = vp[0], vp[1]
    k.bulk_ratio = cfg.get("bulk_ratio", 1.0)
    k.varpi = cfg.get("varpi", 1.0 / 6.0)
    k.gamma1 = cfg.get("gamma1", -2.0)
    k.gamma2 = cfg.get("gamma2", 2.0)
    k.force_mode = int(cfg.get("force_mode", 0))
    k.corrections = int(cfg.get("corrections", 1))
    fo = cfg.get("force", (0.0, 0.0))
    k.force[0], k.force[1] = fo[0], fo[1]
    for s, w in enumerate(cfg["walls"]):
        k.wall[s].periodic = int(w.get("periodic", 0))
        k.wall[s].thermal = int(w.get("thermal", 0))
        k.wall[s].extrap_order = int(w.get("extrap_order", 2))
        u = w.get("u", (0.0, 0.0))
        k.wall[s].u[0], k.wall[s].u[1] = u[0], u[1]
        k.wall[s].T = w.get("T", cfg["T0"])
    return k


def peak_rates(stream=None) -> dict:
    """FP64 FMA, FP32 FMA and double-float multiply-add rates per second of
    the current device (lbm_peak_rates)."""
    L = load()
    a = np.empty(3)
    _check(L, L.lbm_peak_rates(C.c_void_p(stream.cuda_stream if stream is not None else 0), _ptr(a)))
    return {"fp64_fma_per_s": float(a[0]), "fp32_fma_per_s": float(a[1]), "ff64_madd_per_s": float(a[2])}


def workspace_bytes(cfg: dict) -> int:
    L = load()
    n = C.c_size_t()
    _check(L, L.lbm_workspace_bytes(C.byref(make_config(cfg)), C.byref(n)))
    return int(n.value)


class Lattice:
    """One D2Q9 lattice (f and g) resident in HBM, advanced by the CUDA kernels."""

    def __init__(self, cfg: dict, stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the lattice-Boltzmann kernels need a CUDA GPU; none is visible")
        self.L = load()
        self.cfg = cfg
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self.device = torch.device(device or "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._k = make_config(cfg)
        nbytes = workspace_bytes(cfg)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        _check(self.L, self.L.lbm_create(C.byref(self._k), C.c_void_p(self.workspace.data_ptr()),
                                         C.c_size_t(nbytes), C.c_void_p(self.stream.cuda_stream),
                                         C.byref(h)))
        self.h = h
        eos = cfg.get("eos", {"kind": 1, "params": []})
        pr = np.ascontiguousarray(np.asarray(eos.get("params", []), dtype=np.float64))
        _check(self.L, self.L.lbm_set_eos(self.h, int(eos["kind"]), _ptr(pr) if pr.size else None,
                                          int(pr.size)))

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        _check(self.L, st)

    def step(self, n: int):
        _check(self.L, self.L.lbm_step(self.h, int(n)))

    def sync(self):
        _check(self.L, self.L.lbm_sync(self.h))

    def status_step(self, n: int) -> int:
        """Step and synchronise, returning the raw status instead of raising."""
        st = self.L.lbm_step(self.h, int(n))
        if st != LBM_OK:
            return st
        return self.L.lbm_sync(self.h)

    @property
    def steps(self) -> int:
        return int(self.L.lbm_step_count(self.h))

    def macros(self) -> dict:
        out = {k: np.empty((self.ny, self.nx)) for k in ("rho", "ux", "uy", "T", "p")}
        _check(self.L, self.L.lbm_macros(self.h, *(_ptr(out[k]) for k in ("rho", "ux", "uy", "T", "p"))))
        return out

    def macros_device(self, out=None):
        import torch
        if out is None:
            out = {k: torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
                   for k in ("rho", "ux", "uy", "T", "p")}
        ptrs = [C.c_void_p(out[k].data_ptr()) if k in out else None for k in ("rho", "ux", "uy", "T", "p")]
        _check(self.L, self.L.lbm_macros_device(self.h, *ptrs))
        return out

    def nusselt(self, wall: int) -> float:
        v = C.c_double()
        _check(self.L, self.L.lbm_nusselt(self.h, int(wall), C.byref(v)))
        return float(v.value)

    def diagnostics(self, snapshot: bool = False) -> dict:
        a = np.empty(8)
        _check(self.L, self.L.lbm_diagnostics(self.h, int(bool(snapshot)), _ptr(a)))
        return dict(zip(("mass", "energy", "pstar", "residual", "nonfinite", "umax", "Tmean", "steps"),
                        a.tolist()))

    def get_state(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        _check(self.L, self.L.lbm_get_state(self.h, _ptr(f), _ptr(g)))
        return f, g

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx) and g.shape == f.shape
        _check(self.L, self.L.lbm_set_state(self.h, _ptr(f), _ptr(g)))

    def init_macros(self, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.ny, self.nx) for a in (rho, ux, uy, T)]
        _check(self.L, self.L.lbm_init_macros(self.h, *(_ptr(a) for a in arrs)))

    def derived(self) -> dict:
        a = np.empty(8)
        _check(self.L, self.L.lbm_derived(self.h, _ptr(a)))
        return dict(zip(("R", "Cv", "Cp", "mu0", "p0", "eta0", "lambda0", "cs2"), a.tolist()))

    def set_tile(self, bx: int, by: int, pair: int = 0):
        _check(self.L, self.L.lbm_set_tile(self.h, int(bx), int(by), int(pair)))

    def tile(self) -> tuple:
        """(bx, by, pair) of the launch shape in use."""
        bx, by, pr = C.c_int(), C.c_int(), C.c_int()
        _check(self.L, self.L.lbm_get_tile(self.h, C.byref(bx), C.byref(by), C.byref(pr)))
        return bx.value, by.value, pr.value

    def set_rounding(self, mode: int):
        """ROUND_STOCHASTIC (default) or ROUND_NEAREST for FP32 stores."""
        _check(self.L, self.L.lbm_set_rounding(self.h, int(mode)))

    def copy_state_from(self, other: "Lattice"):
        """Take the state, step count and residual snapshot of another lattice
        of the same problem, converting the storage precision."""
        _check(self.L, self.L.lbm_copy_state(self.h, other.h))

    def conserved_sums_static(self, out):
        """Total mass, x and y momentum and sum of g into the device tensor
        ``out`` (4 doubles) without any allocation; asynchronous."""
        _check(self.L, self.L.lbm_conserved_sums_static(self.h, C.c_void_p(out.data_ptr())))


class Batch:
    """Several lattices on one stream advanced together: one fused launch per
    (precision, strip width) and one wall-pass launch per precision each step,
    optionally captured as a CUDA graph of ``graph_steps`` steps."""

    def __init__(self, lattices, graph_steps: int = 0):
        self.L = load()
        self.lattices = list(lattices)
        arr = (C.c_void_p * len(self.lattices))(*[lat.h.value for lat in self.lattices])
        h = C.c_void_p()
        _check(self.L, self.L.lbm_batch_create(arr, len(self.lattices), int(graph_steps), C.byref(h)))
        self.h = h
        self.graph_steps = int(graph_steps)

    def step(self, n: int):
        _check(self.L, self.L.lbm_batch_step(self.h, int(n)))

    def step_profiled(self, n: int):
        """Step n times with per-step CUDA events; returns (ms in the fused
        kernels, ms in the wall pass), summed over the n steps."""
        a, b = C.c_double(), C.c_double()
        _check(self.L, self.L.lbm_batch_step_profiled(self.h, int(n), C.byref(a), C.byref(b)))
        return a.value, b.value

    def add(self, lattice):
        """Append a member (launch tables and graph rebuilt)."""
        _check(self.L, self.L.lbm_batch_add(self.h, lattice.h))
        self.lattices.append(lattice)

    def remove(self, lattice):
        """Drop a member; the others keep their order."""
        _check(self.L, self.L.lbm_batch_remove(self.h, lattice.h))
        self.lattices.remove(lattice)

    def diagnostics(self, snapshot: bool = False):
        """lbm_diagnostics of every member in one pass: a list of (dict,
        status) in member order; status is LBM_OK or the member's sticky
        error."""
        n = len(self.lattices)
        a = np.empty(n * 8)
        st = (C.c_int * n)()
        _check(self.L, self.L.lbm_batch_diagnostics(self.h, int(bool(snapshot)), _ptr(a), st))
        keys = ("mass", "energy", "pstar", "residual", "nonfinite", "umax", "Tmean", "steps")
        return [(dict(zip(keys, a[8 * k:8 * k + 8].tolist())), int(st[k])) for k in range(n)]

    def init_macros(self, fields):
        """lbm_init_macros of every member with one synchronisation:
        ``fields[k]`` is (rho, ux, uy, T) of member k, FP64 C-contiguous
        host arrays [ny][nx] (pinned memory copies fastest)."""
        n = len(self.lattices)
        arrs = [[_host_field(a, lat) for a in f] for f, lat in zip(fields, self.lattices)]
        if len(arrs) != n or any(len(f) != 4 for f in arrs):
            raise ValueError("one (rho, ux, uy, T) per member")
        cols = [(C.POINTER(C.c_double) * n)(*[_ptr(arrs[k][q]) for k in range(n)]) for q in range(4)]
        _check(self.L, self.L.lbm_batch_init_macros(self.h, *cols))

    def macros(self, out):
        """lbm_macros of every member with one synchronisation: ``out[k]``
        maps 'rho', 'ux', 'uy', 'T', 'p' (any subset) of member k to FP64
        C-contiguous host arrays [ny][nx] that receive the fields.  Returns
        each member's status (LBM_OK or its sticky error)."""
        n = len(self.lattices)
        if len(out) != n:
            raise ValueError("one output dict per member")
        keys = ("rho", "ux", "uy", "T", "p")
        for o, lat in zip(out, self.lattices):
            for k, a in o.items():
                if k not in keys:
                    raise ValueError(f"unknown field {k}")
                _host_field(a, lat, writable=True)
        cols = []
        for k in keys:
            if any(k in o for o in out):
                cols.append((C.POINTER(C.c_double) * n)(*[_ptr(o.get(k)) for o in out]))
            else:
                cols.append(None)
        st = (C.c_int * n)()
        _check(self.L, self.L.lbm_batch_macros(self.h, *cols, st))
        return [int(v) for v in st]

    def close(self):
        if getattr(self, "h", None):
            self.L.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
