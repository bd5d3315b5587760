"""ctypes binding of the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` import this module.  It imports nothing
from the CUDA package: configurations arrive as plain dictionaries (see
``paper_1809_08683_gb300.workloads`` for the layout) and are marshalled into
this module's own ctypes image of ``orc_config``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OrcWall(C.Structure):
    _fields_ = [("periodic", C.c_int32), ("thermal", C.c_int32), ("extrap_order", C.c_int32),
                ("reserved", C.c_int32), ("u", C.c_double * 2), ("T", C.c_double)]


class OrcConfig(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("precision", C.c_int32),
                ("visc_law", C.c_int32), ("rho0", C.c_double), ("T0", C.c_double),
                ("Pr", C.c_double), ("gamma", C.c_double), ("tau0", C.c_double),
                ("visc_p", C.c_double * 2), ("bulk_ratio", C.c_double), ("varpi", C.c_double),
                ("gamma1", C.c_double), ("gamma2", C.c_double), ("force_mode", C.c_int32),
                ("corrections", C.c_int32), ("force", C.c_double * 2), ("wall", OrcWall * 4)]


class OrcNodeInfo(C.Structure):
    _fields_ = ([(n, C.c_double) for n in
                 ("rho", "ux", "uy", "Fx", "Fy", "qe", "E", "T", "p", "eta", "H")]
                + [("s", C.c_double * 9), ("sig", C.c_double * 9)]
                + [(n, C.c_double * 9) for n in ("m", "meq", "Fm", "mbar", "n", "neq", "Qm", "nbar")]
                + [(n, C.c_double * 81) for n in ("S", "R", "L", "Y")]
                + [("Tm", C.c_double * 18), ("Xm", C.c_double * 18)]
                + [("IS2inv", C.c_double * 81), ("IL2inv", C.c_double * 81)]
                + [("fbar", C.c_double * 9), ("gbar", C.c_double * 9)])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            dp = P(C.c_double)
            L.orc_create.argtypes = [P(OrcConfig), P(C.c_void_p)]
            L.orc_set_eos.argtypes = [C.c_void_p, C.c_int, dp, C.c_int]
            L.orc_step.argtypes = [C.c_void_p, C.c_long]
            L.orc_macros.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
            L.orc_nusselt.argtypes = [C.c_void_p, C.c_int, dp]
            L.orc_get_state.argtypes = [C.c_void_p, dp, dp]
            L.orc_set_state.argtypes = [C.c_void_p, dp, dp]
            L.orc_init_macros.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_step_count.argtypes = [C.c_void_p]
            L.orc_step_count.restype = C.c_long
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_derived.argtypes = [C.c_void_p, dp]
            L.orc_boundary_pass.argtypes = [C.c_void_p]
            L.orc_grad_field.argtypes = [C.c_void_p, dp, dp, dp]
            L.orc_eq_moments.argtypes = [C.c_void_p] + [C.c_double] * 6 + [dp] * 4
            L.orc_matrix_M.argtypes = [dp]
            L.orc_matrix_Minv.argtypes = [dp]
            L.orc_node.argtypes = [C.c_void_p, dp, dp, dp, dp, P(OrcNodeInfo)]
            _lib = L
        return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_config(cfg: dict) -> OrcConfig:
    k = OrcConfig()
    k.nx, k.ny = int(cfg["nx"]), int(cfg["ny"])
    k.precision = 0
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


class Oracle:
    """One lattice advanced by the plain CPU oracle."""

    def __init__(self, cfg: dict, threads: int | None = None):
        self.L = lib()
        if threads is not None:
            self.L.orc_set_threads(int(threads))
        self.cfg = cfg
        self.nx, self.ny = int(cfg["nx"]), int(cfg["ny"])
        self._k = make_config(cfg)
        h = C.c_void_p()
        st = self.L.orc_create(C.byref(self._k), C.byref(h))
        if st != 0:
            raise ValueError(f"orc_create failed ({st})")
        self.h = h
        eos = cfg.get("eos", {"kind": 1, "params": []})
        pr = np.ascontiguousarray(np.asarray(eos.get("params", []), dtype=np.float64))
        st = self.L.orc_set_eos(self.h, int(eos["kind"]), _ptr(pr) if pr.size else None, int(pr.size))
        if st != 0:
            raise ValueError(f"orc_set_eos failed ({st})")

    def close(self):
        if getattr(self, "h", None):
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int) -> int:
        return int(self.L.orc_step(self.h, int(n)))

    @property
    def steps(self) -> int:
        return int(self.L.orc_step_count(self.h))

    def macros(self) -> dict:
        sh = (self.ny, self.nx)
        out = {k: np.empty(sh) for k in ("rho", "ux", "uy", "T", "p")}
        st = self.L.orc_macros(self.h, *(_ptr(out[k]) for k in ("rho", "ux", "uy", "T", "p")))
        if st != 0:
            raise RuntimeError(f"orc_macros failed ({st})")
        return out

    def get_state(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        self.L.orc_get_state(self.h, _ptr(f), _ptr(g))
        return f, g

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx) and g.shape == f.shape
        st = self.L.orc_set_state(self.h, _ptr(f), _ptr(g))
        if st != 0:
            raise RuntimeError("orc_set_state failed")

    def init_macros(self, rho, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.ny, self.nx)
                for a in (rho, ux, uy, T)]
        st = self.L.orc_init_macros(self.h, *(_ptr(a) for a in arrs))
        if st != 0:
            raise RuntimeError("orc_init_macros failed")

    def nusselt(self, wall: int) -> float:
        v = C.c_double()
        st = self.L.orc_nusselt(self.h, int(wall), C.byref(v))
        if st != 0:
            raise RuntimeError(f"orc_nusselt failed ({st})")
        return float(v.value)

    def derived(self) -> dict:
        a = np.empty(8)
        self.L.orc_derived(self.h, _ptr(a))
        return dict(zip(("R", "Cv", "Cp", "mu0", "p0", "eta0", "lambda0", "cs2"), a.tolist()))

    def boundary_pass(self):
        self.L.orc_boundary_pass(self.h)

    def grad_field(self, phi):
        """(d phi/dx, d phi/dy) at every node with the oracle's gradient
        stencil; phi is [ny][nx]."""
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        gx, gy = np.empty_like(phi), np.empty_like(phi)
        if self.L.orc_grad_field(self.h, _ptr(phi), _ptr(gx), _ptr(gy)) != 0:
            raise RuntimeError("orc_grad_field failed")
        return gx, gy

    def eq_moments(self, rho, ux, uy, T, Fx=0.0, Fy=0.0) -> dict:
        out = {k: np.empty(9) for k in ("meq", "Fm", "neq", "Qm")}
        st = self.L.orc_eq_moments(self.h, rho, ux, uy, T, Fx, Fy,
                                   *(_ptr(out[k]) for k in ("meq", "Fm", "neq", "Qm")))
        if st != 0:
            raise RuntimeError("orc_eq_moments failed")
        return out

    def node(self, f9, g9, grad_rho=(0.0, 0.0), grad_p=(0.0, 0.0)) -> dict:
        info = OrcNodeInfo()
        f9 = np.ascontiguousarray(f9, dtype=np.float64)
        g9 = np.ascontiguousarray(g9, dtype=np.float64)
        gr = np.ascontiguousarray(grad_rho, dtype=np.float64)
        gp = np.ascontiguousarray(grad_p, dtype=np.float64)
        st = self.L.orc_node(self.h, _ptr(f9), _ptr(g9), _ptr(gr), _ptr(gp), C.byref(info))
        if st != 0:
            raise RuntimeError("orc_node failed")
        out = {}
        for name, typ in OrcNodeInfo._fields_:
            v = getattr(info, name)
            if isinstance(v, float):
                out[name] = v
            else:
                a = np.array(v[:], dtype=np.float64)
                if a.size == 81:
                    a = a.reshape(9, 9)
                elif a.size == 18:
                    a = a.reshape(9, 2)
                out[name] = a
        return out


def matrix_M() -> np.ndarray:
    a = np.empty(81)
    lib().orc_matrix_M(_ptr(a))
    return a.reshape(9, 9)


def matrix_Minv() -> np.ndarray:
    a = np.empty(81)
    lib().orc_matrix_Minv(_ptr(a))
    return a.reshape(9, 9)
