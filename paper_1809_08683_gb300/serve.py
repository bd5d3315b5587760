"""Continuous-batching serving loop for lattice solves.

Requests (a cavity or channel configuration, a residual target and a step
cap) arrive over time.  The server keeps every admitted lattice resident in
HBM and advances all resident lattices together: one batched fused launch
and one batched wall-pass launch per time step, replayed from a CUDA graph in
chunks of ``chunk`` steps.  After each chunk it evaluates the FP64 residual of
every resident lattice (relative change of u and T over the chunk), retires
converged or capped solves, and admits newly arrived requests while slots and
device memory allow.  A request that arrives while others run joins at the
next chunk boundary.  Per-node arithmetic does not depend on the batch, so a
request's result is bitwise the same alone and in any mix.
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
    result: dict = field(default_factory=dict)

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival

    @property
    def nodes(self):
        return int(self.cfg["nx"]) * int(self.cfg["ny"])


def summarise(lat, req):
    out = {"residual": req.result.get("residual")}
    d = lat.diagnostics()
    out.update({"mass": d["mass"], "pstar": d["pstar"], "umax": d["umax"], "Tmean": d["Tmean"]})
    walls = req.cfg["walls"]
    dirichlet = [s for s in range(4) if not walls[s]["periodic"] and walls[s]["thermal"] == 0]
    Ts = {walls[s]["T"] for s in dirichlet}
    if len(dirichlet) >= 2 and len(Ts) >= 2:
        out["nusselt"] = lat.nusselt(max(dirichlet, key=lambda s: walls[s]["T"]))
    return out


class Server:
    def __init__(self, max_slots: int = 64, mem_fraction: float = 0.85, chunk: int = 1000,
                 graph_steps: int = 100, stream=None, tile_fn=None, keep_fields: bool = False):
        import torch
        self.torch = torch
        self.max_slots = max_slots
        self.mem_fraction = mem_fraction
        self.chunk = chunk
        self.graph_steps = graph_steps if graph_steps and chunk % graph_steps == 0 else 0
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.tile_fn = tile_fn
        self.keep_fields = keep_fields
        free, total = torch.cuda.mem_get_info()
        self.budget = int(free * mem_fraction)
        self.in_use = 0
        self.node_steps = 0
        self.log = []

    def _fits(self, req):
        return self.in_use + lbm.workspace_bytes(req.cfg) <= self.budget

    def run(self, requests, realtime: bool = True):
        """Serve the requests; arrival times are honoured against the wall
        clock when realtime is True, otherwise every request is available at
        once.  Returns the list of requests with their results filled."""
        pending = sorted(requests, key=lambda r: r.arrival)
        resident = []          # (request, lattice)
        batch = None
        dirty = True
        t0 = time.perf_counter()
        while pending or resident:
            now = time.perf_counter() - t0
            while (pending and (not realtime or pending[0].arrival <= now)
                   and len(resident) < self.max_slots and self._fits(pending[0])):
                r = pending.pop(0)
                lat = lbm.Lattice(r.cfg, stream=self.stream)
                if self.tile_fn is not None:
                    lat.set_tile(*self.tile_fn(r.cfg))
                lat.diagnostics(snapshot=True)
                self.in_use += lbm.workspace_bytes(r.cfg)
                r.admitted = time.perf_counter() - t0
                r.status = "running"
                resident.append((r, lat))
                dirty = True
            if not resident:
                if pending:
                    if realtime:
                        time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                    else:
                        raise RuntimeError(f"request {pending[0].rid} does not fit the device budget")
                continue
            if dirty:
                if batch is not None:
                    batch.close()
                batch = lbm.Batch([lat for _, lat in resident], graph_steps=self.graph_steps)
                dirty = False
            batch.step(self.chunk)
            self.node_steps += self.chunk * sum(r.nodes for r, _ in resident)
            keep = []
            for r, lat in resident:
                r.steps += self.chunk
                try:
                    d = lat.diagnostics(snapshot=True)
                    r.result["residual"] = d["residual"]
                    done = (r.steps >= r.min_steps and d["residual"] < r.tol)
                    r.converged = done
                    if done or r.steps >= r.max_steps:
                        r.status = "converged" if done else "capped"
                except lbm.LbmError as e:
                    r.status = "unstable"
                    r.result["error"] = str(e)
                if r.status == "running":
                    keep.append((r, lat))
                    continue
                r.finished = time.perf_counter() - t0
                if r.status != "unstable":
                    r.result.update(summarise(lat, r))
                    if self.keep_fields:
                        r.result["fields"] = lat.macros()
                self.in_use -= lbm.workspace_bytes(r.cfg)
                lat.close()
                dirty = True
            if dirty and batch is not None:
                batch.close()
                batch = None
            resident = keep
            self.log.append((time.perf_counter() - t0, len(resident), len(pending)))
        if batch is not None:
            batch.close()
        self.wall = time.perf_counter() - t0
        return requests


def solve_sequential(req: Request, chunk: int = 1000, keep_fields: bool = False):
    """Plain per-request solve: FP64 lattice alone, per-step launches, the
    same residual schedule.  The baseline the batched server is compared to."""
    lat = lbm.Lattice(req.cfg)
    lat.diagnostics(snapshot=True)
    t0 = time.perf_counter()
    while True:
        lat.step(chunk)
        req.steps += chunk
        d = lat.diagnostics(snapshot=True)
        req.result["residual"] = d["residual"]
        if req.steps >= req.min_steps and d["residual"] < req.tol:
            req.converged = True
            req.status = "converged"
            break
        if req.steps >= req.max_steps:
            req.status = "capped"
            break
    req.result.update(summarise(lat, req))
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
