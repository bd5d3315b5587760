"""Continuous-batching serving loop for lattice solves.

Requests (a cavity or channel configuration, a residual target and a step
cap) arrive over time.  The server keeps every admitted lattice resident in
HBM and advances all resident lattices together: one batched fused launch
per launch group and one batched wall-pass launch per time step, replayed
from a CUDA graph in chunks of ``chunk`` steps.  After each chunk one
batched diagnostics pass (one synchronisation) gives the FP64 residual of
every resident lattice (relative change of u and T over the chunk); the
server retires converged, capped or unstable solves and admits arrived
requests while slots and device memory allow, first fit in arrival order,
so a small request is not held back behind a large one that does not fit
yet.  The batch is rebuilt only when the resident set changes.

Precision: a request whose configuration asks for FP32 deviation storage is
stepped in FP32 while FP32 makes progress; stochastic rounding leaves FP32
residuals on a noise floor (about 1e-6 for heated cavities, 1e-5 for
channels, whose temperature variation is small).  If the target lies below
what FP32 reaches (the residual stops falling below ``fp32_stall``), the
solve is finished in FP64 from the FP32 state (lbm_copy_state), so that
every result meets its stated target.  A
request's result is bitwise the same alone and in any mix: per-node
arithmetic does not depend on the batch, residual checks fall on the same
step counts, and stochastic rounding draws from (node, absolute step) only.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

from . import lbm


@dataclass
class Request:
    rid: int
    cfg: dict
    arrival: float = 0.0      # seconds after the start of the run
    tol: float = 1e-7         # residual target
    max_steps: int = 2_000_000
    min_steps: int = 0
    # filled by the server
    admitted: float | None = None
    finished: float | None = None
    steps: int = 0
    converged: bool = False
    status: str = "pending"
    switched_at: int | None = None   # step count at which an FP32 solve moved to FP64
    result: dict = field(default_factory=dict)
    history: list = field(default_factory=list)   # residual after each chunk

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival

    @property
    def nodes(self):
        return int(self.cfg["nx"]) * int(self.cfg["ny"])


def summarise(lat, req, d=None):
    """Result of a finished solve: its last residual, the FP64 diagnostics
    (taken now unless `d`, the last diagnostics of the current state, is
    given) and the hot-wall Nusselt number when two Dirichlet walls differ."""
    out = {"residual": req.result.get("residual")}
    if d is None:
        d = lat.diagnostics()
    out.update({"mass": d["mass"], "pstar": d["pstar"], "umax": d["umax"], "Tmean": d["Tmean"]})
    walls = req.cfg["walls"]
    dirichlet = [s for s in range(4) if not walls[s]["periodic"] and walls[s]["thermal"] == 0]
    Ts = {walls[s]["T"] for s in dirichlet}
    if len(dirichlet) >= 2 and len(Ts) >= 2:
        out["nusselt"] = lat.nusselt(max(dirichlet, key=lambda s: walls[s]["T"]))
    return out


def fp32_stalled(history, ceiling=1e-4, window=20, gain=0.8):
    """Whether an FP32 solve has reached what FP32 storage can resolve: its
    residual is below `ceiling` and the best residual of the last `window`
    checks is no better than `gain` times the best of the `window` before.
    Stochastic rounding puts the FP32 noise floor near 1e-6 for heated
    cavities and 1e-5 for channels; above `ceiling` a slow or oscillating
    start-up transient is not taken for that floor.  None: never."""
    if ceiling is None or len(history) < 2 * window or history[-1] >= ceiling:
        return False
    return min(history[-window:]) > gain * min(history[-2 * window:-window])


def stall_window(cfg, base=20, ref_nodes=512 * 512):
    """Residual checks that fp32_stalled compares for this lattice: `base`
    up to 512^2 nodes, in proportion to the node count above.  The slowest
    modes of a heated cavity relax on a diffusive time that grows with its
    area: the 512^2 cavity at Ra = 1e6 loses a decade of residual in about
    70,000 FP32 steps, and if that time scales with the area a 1024^2 one
    loses it in about 280,000, a fall of less than 20% per 20 checks that a
    fixed window of 20 would take for the noise floor."""
    nodes = int(cfg["nx"]) * int(cfg["ny"])
    return max(base, int(round(base * nodes / ref_nodes)))


def _fp64(cfg):
    c = dict(cfg)
    c["precision"] = lbm.FP64
    return c



class _Timer:
    """Device time between start() and stop() on the serving stream (CUDA
    events); wall-clock time when the stream is not a CUDA stream."""

    def __init__(self, stream):
        import torch
        self.cuda = isinstance(stream, torch.cuda.Stream)
        self.stream = stream
        if self.cuda:
            self.e0 = torch.cuda.Event(enable_timing=True)
            self.e1 = torch.cuda.Event(enable_timing=True)

    def start(self):
        if self.cuda:
            self.e0.record(self.stream)
        else:
            self.t0 = time.perf_counter()

    def stop(self):
        if self.cuda:
            self.e1.record(self.stream)
        else:
            self.t1 = time.perf_counter()

    def ms(self):
        if self.cuda:
            self.e1.synchronize()
            return self.e0.elapsed_time(self.e1)
        return (self.t1 - self.t0) * 1e3


class _Slot:
    __slots__ = ("req", "lat", "bytes")

    def __init__(self, req, lat, nbytes):
        self.req, self.lat, self.bytes = req, lat, nbytes


class Server:
    """max_slots: resident lattices at most.  mem_fraction: share of the
    device memory free at construction that resident lattices may take; the
    memory free at each admission (minus the rest of the device as
    headroom) is checked as well, so memory that other work takes or frees
    later is seen.  fp32_stall: the residual below which an FP32 solve that
    stops improving moves to FP64 (fp32_stalled); None keeps FP32 to the
    end.  starvation_s: a request that has waited this long stops later
    arrivals from overtaking it (None: never).  finish_tile_fn: launch shape
    of the FP64 lattice an FP32 solve finishes in (None: the FP64
    default)."""

    def __init__(self, max_slots: int = 64, mem_fraction: float = 0.85, chunk: int = 1000,
                 graph_steps: int = 10, stream=None, tile_fn=None, keep_fields: bool = False,
                 fp32_stall: float | None = 1e-4, starvation_s: float | None = None,
                 finish_tile_fn=None):
        import torch
        self.torch = torch
        self.max_slots = max_slots
        self.mem_fraction = mem_fraction
        self.chunk = chunk
        self.graph_steps = graph_steps if graph_steps and chunk % graph_steps == 0 else 0
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.tile_fn = tile_fn
        self.keep_fields = keep_fields
        self.fp32_stall = fp32_stall
        self.finish_tile_fn = finish_tile_fn
        self.starvation_s = starvation_s
        free, total = torch.cuda.mem_get_info()
        self.total = total
        self.budget = int(free * mem_fraction)
        self.headroom = int(total * (1.0 - mem_fraction))
        self.in_use = 0
        self.node_steps = 0
        self.gpu_ms = 0.0          # device time of the stepping, summed over chunks
        self.chunks = 0
        self.rebuilds = 0
        # host seconds between one chunk's diagnostics and the next chunk's
        # launch (the device idles), and where they went
        self.host_s = {"between_chunks": 0.0, "admit": 0.0, "retire": 0.0, "rebuild": 0.0}
        self.log = []

    # -- device memory ----------------------------------------------------
    def _live_free(self):
        """Device memory free now, counting what the caching allocator holds
        unused as free."""
        free, _ = self.torch.cuda.mem_get_info()
        try:
            cached = self.torch.cuda.memory_reserved() - self.torch.cuda.memory_allocated()
        except Exception:
            cached = 0
        return free + max(0, cached)

    def _fits(self, nbytes):
        return (self.in_use + nbytes <= self.budget) and (nbytes <= self._live_free() - self.headroom)

    def _new_lattice(self, cfg):
        if isinstance(self.stream, self.torch.cuda.Stream):
            # the workspace belongs to the serving stream, so the caching
            # allocator reuses it only in that stream's order
            with self.torch.cuda.stream(self.stream):
                lat = lbm.Lattice(cfg, stream=self.stream)
        else:
            lat = lbm.Lattice(cfg, stream=self.stream)
        if self.tile_fn is not None:
            lat.set_tile(*self.tile_fn(cfg))
        return lat

    # -- the loop ----------------------------------------------------------
    def run(self, requests, realtime: bool = True, deadline_s: float | None = None):
        """Serve the requests; arrival times are honoured against the wall
        clock when realtime is True, otherwise every request is available at
        once.  deadline_s: after this many seconds of wall time the run
        stops between chunks; resident solves are closed with status
        "stopped" and requests not yet admitted stay "pending".  Returns the
        list of requests with their results filled."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        resident: list[_Slot] = []
        batch = None
        dirty = True
        timer = _Timer(self.stream)
        t0 = time.perf_counter()
        t_diag = None           # when the last chunk's diagnostics returned
        while pending or resident:
            now = time.perf_counter() - t0
            if deadline_s is not None and now > deadline_s:
                if batch is not None:
                    batch.close()
                    batch = None
                for slot in resident:
                    slot.req.status = "stopped"
                    self.in_use -= slot.bytes
                    slot.lat.close()
                resident = []
                break
            ta = time.perf_counter()
            # admission: first fit in arrival order
            i = 0
            while i < len(pending) and len(resident) < self.max_slots:
                r = pending[i]
                if realtime and r.arrival > now:
                    break
                nbytes = lbm.workspace_bytes(r.cfg)
                if not self._fits(nbytes):
                    if self.starvation_s is not None and now - r.arrival > self.starvation_s:
                        break
                    i += 1
                    continue
                pending.pop(i)
                lat = self._new_lattice(r.cfg)
                self.in_use += nbytes
                r.admitted = time.perf_counter() - t0
                r.status = "running"
                resident.append(_Slot(r, lat, nbytes))
                dirty = True
            self.host_s["admit"] += time.perf_counter() - ta
            if not resident:
                future = [r for r in pending if realtime and r.arrival > now]
                if not future:
                    # everything has arrived, nothing is resident, nothing fits
                    raise RuntimeError(f"request {pending[0].rid} does not fit the device budget")
                t_diag = None   # waiting for arrivals is not host overhead
                time.sleep(max(0.0, min(0.01, future[0].arrival - now)))
                continue
            if dirty:
                tb = time.perf_counter()
                if batch is not None:
                    batch.close()
                batch = lbm.Batch([s.lat for s in resident], graph_steps=self.graph_steps)
                self.rebuilds += 1
                dirty = False
                self.host_s["rebuild"] += time.perf_counter() - tb
            if t_diag is not None:
                self.host_s["between_chunks"] += time.perf_counter() - t_diag
            timer.start()
            batch.step(self.chunk)
            timer.stop()
            diags = batch.diagnostics(snapshot=True)
            t_diag = time.perf_counter()
            self.gpu_ms += timer.ms()
            self.chunks += 1
            self.node_steps += self.chunk * sum(s.req.nodes for s in resident)
            keep = []
            for slot, (d, st) in zip(resident, diags):
                r = slot.req
                r.steps += self.chunk
                if st != lbm.LBM_OK:
                    r.status = "unstable"
                    r.result["error"] = f"lbm status {st}"
                else:
                    # the first check of a solve has no snapshot to compare with
                    res = d["residual"] if r.steps > self.chunk else float("inf")
                    r.result["residual"] = res
                    r.history.append(res)
                    fp32 = int(slot.lat.cfg.get("precision", 0)) == lbm.FP32_DEV
                    if r.steps >= r.min_steps and res < r.tol:
                        r.converged = True
                        r.status = "converged"
                    elif (fp32 and fp32_stalled(r.history, self.fp32_stall, stall_window(r.cfg))
                          and self._switch_to_fp64(slot)):
                        r.switched_at = r.steps
                        dirty = True
                    if r.status == "running" and r.steps >= r.max_steps:
                        r.status = "capped"
                if r.status == "running":
                    keep.append(slot)
                    continue
                r.finished = time.perf_counter() - t0
                tr = time.perf_counter()
                if r.status != "unstable":
                    r.result.update(summarise(slot.lat, r, d))
                    if self.keep_fields:
                        r.result["fields"] = slot.lat.macros()
                self.in_use -= slot.bytes
                slot.lat.close()
                dirty = True
                self.host_s["retire"] += time.perf_counter() - tr
            if dirty and batch is not None:
                batch.close()
                batch = None
            resident = keep
            self.log.append((time.perf_counter() - t0, len(resident), len(pending)))
        if batch is not None:
            batch.close()
        self.wall = time.perf_counter() - t0
        return requests

    def _switch_to_fp64(self, slot):
        """Move a stalled FP32 solve to FP64 storage (state, step count and
        residual snapshot copied); False when the FP64 lattice does not fit
        now (the solve then stays in FP32 and retries after the next chunk)."""
        cfg = _fp64(slot.lat.cfg)
        nbytes = lbm.workspace_bytes(cfg)
        if not self._fits(nbytes):
            return False
        lat = self._new_lattice(cfg)
        if self.finish_tile_fn is not None:
            lat.set_tile(*self.finish_tile_fn(cfg))
        lat.copy_state_from(slot.lat)
        slot.lat.close()
        self.in_use += nbytes - slot.bytes
        slot.lat, slot.bytes = lat, nbytes
        return True

    @property
    def host_overhead(self):
        """Share of the wall time the device waited for the host between two
        chunks: the results loop, retirements, admissions and the batch
        rebuild.  (Time with nothing resident, waiting for arrivals, is not
        counted; device_busy includes it.)"""
        return self.host_s["between_chunks"] / self.wall if getattr(self, "wall", 0) else None

    @property
    def device_busy(self):
        """Share of the wall time the device spent stepping lattices."""
        return self.gpu_ms * 1e-3 / self.wall if getattr(self, "wall", 0) else None


def solve_sequential(req: Request, chunk: int = 1000, keep_fields: bool = False, fp32_stall: float | None = 1e-4,
                     finish_tile_fn=None):
    """Plain per-request solve: the lattice alone, per-step launches, the
    same residual schedule (and the same move from FP32 to FP64 once FP32
    stalls).  The baseline the batched server is compared to."""
    t0 = time.perf_counter()
    lat = lbm.Lattice(req.cfg)
    while True:
        lat.step(chunk)
        req.steps += chunk
        d = lat.diagnostics(snapshot=True)
        # the first check of a solve has no snapshot to compare with
        res = d["residual"] if req.steps > chunk else float("inf")
        req.result["residual"] = res
        req.history.append(res)
        if req.steps >= req.min_steps and res < req.tol:
            req.converged = True
            req.status = "converged"
            break
        if req.steps >= req.max_steps:
            req.status = "capped"
            break
        if (int(lat.cfg.get("precision", 0)) == lbm.FP32_DEV
                and fp32_stalled(req.history, fp32_stall, stall_window(req.cfg))):
            lat64 = lbm.Lattice(_fp64(lat.cfg))
            if finish_tile_fn is not None:
                lat64.set_tile(*finish_tile_fn(lat64.cfg))
            lat64.copy_state_from(lat)
            lat.close()
            lat = lat64
            req.switched_at = req.steps
    req.result.update(summarise(lat, req, d))
    if keep_fields:
        req.result["fields"] = lat.macros()
    req.result["solve_s"] = time.perf_counter() - t0
    lat.close()
    return req


def percentiles(values, ps=(50, 99)):
    import numpy as np
    v = np.asarray([x for x in values if x is not None], dtype=float)
    if v.size == 0:
        return {f"p{p}": None for p in ps}
    return {f"p{p}": float(np.percentile(v, p)) for p in ps}
