"""Host scheduling of the continuous-batching server (serve.Server.run) on the
CPU: the library is replaced by a scripted fake (lattices whose residual
falls at a set rate, or that turn unstable), so admission by free slots and
device memory, arrival order, retirement on convergence, on the step cap and
on instability, and the memory ledger are checked without a GPU."""
import time
import types

import pytest

from paper_1809_08683_gb300 import serve
from paper_1809_08683_gb300 import workloads as W


class FakeError(RuntimeError):
    pass


def fake_library(trace):
    """A stand-in for the lbm module: each config carries its script under
    cfg["fake"] = {"bytes": workspace bytes, "decay": residual factor per
    1000 steps, "unstable_at": step count at which diagnostics fail,
    "floor": residual below which FP32 storage does not get}.  A FP64
    configuration takes twice the bytes of its FP32 one."""

    class Lattice:
        def __init__(self, cfg, stream=None):
            self.cfg, self.steps, self.closed = cfg, 0, False
            trace["created"].append((cfg["rid"], int(cfg.get("precision", 0))))

        def set_tile(self, *a):
            pass

        def copy_state_from(self, other):
            self.steps = other.steps
            trace["copied"].append(self.cfg["rid"])

        def residual(self):
            s = self.cfg["fake"]
            r = 1.0 * s["decay"] ** (self.steps / 1000.0) if self.steps else 1.0
            if int(self.cfg.get("precision", 0)) == 1:
                r = max(r, s.get("floor", 0.0))
            return r

        def unstable(self):
            s = self.cfg["fake"]
            return s.get("unstable_at") is not None and self.steps >= s["unstable_at"]

        def diagnostics(self, snapshot=False):
            if self.unstable():
                raise FakeError("non-finite state")
            return {"residual": self.residual(), "mass": 1.0, "pstar": 1.0, "umax": 0.0, "Tmean": 1.0}

        def nusselt(self, wall):
            return 1.0

        def macros(self):
            return {}

        def close(self):
            self.closed = True

    class Batch:
        def __init__(self, lattices, graph_steps=0):
            self.lattices = list(lattices)
            trace["batches"].append(sorted(l.cfg["rid"] for l in self.lattices))

        def step(self, n):
            time.sleep(trace.get("step_sleep", 0.0))
            for l in self.lattices:
                assert not l.closed
                l.steps += n

        def diagnostics(self, snapshot=False):
            trace["diag_calls"] += 1
            return [({}, -4) if l.unstable() else
                    ({"residual": l.residual(), "mass": 1.0, "pstar": 1.0, "umax": 0.0, "Tmean": 1.0}, 0)
                    for l in self.lattices]

        def close(self):
            pass

    def workspace_bytes(cfg):
        # a request made in FP32 storage takes twice its bytes once in FP64
        b = cfg["fake"]["bytes"]
        return 2 * b if (cfg["fake"]["fp32"] and int(cfg.get("precision", 0)) == 0) else b

    return types.SimpleNamespace(Lattice=Lattice, Batch=Batch, LbmError=FakeError, LBM_OK=0, FP64=0, FP32_DEV=1,
                                 workspace_bytes=workspace_bytes)


def make_requests(specs, precision=0, tol=1.5e-3, floor=0.0):
    reqs = []
    for rid, (arrival, bytes_, decay, unstable_at, max_steps) in enumerate(specs):
        cfg = W.couette(nx=4, ny=8, precision=precision)
        cfg["rid"] = rid
        cfg["fake"] = {"bytes": bytes_, "decay": decay, "unstable_at": unstable_at, "floor": floor,
                       "fp32": precision == 1}
        reqs.append(serve.Request(rid=rid, cfg=cfg, arrival=arrival, tol=tol, max_steps=max_steps))
    return reqs


@pytest.fixture
def server_factory(monkeypatch):
    import torch
    trace = {"created": [], "batches": [], "copied": [], "diag_calls": 0}
    monkeypatch.setattr(serve, "lbm", fake_library(trace))
    monkeypatch.setattr(torch.cuda, "memory_reserved", lambda *a: 0)
    monkeypatch.setattr(torch.cuda, "memory_allocated", lambda *a: 0)

    def make(free_bytes, free_fn=None, **kw):
        monkeypatch.setattr(torch.cuda, "mem_get_info",
                            free_fn or (lambda *a: (free_bytes, free_bytes)))
        return serve.Server(stream=object(), **kw)

    return make, trace


def test_outcomes_slots_and_ledger(server_factory):
    make, trace = server_factory
    # residual 0.1 per 1000 steps meets the 1.5e-3 target after 3000 steps
    # (checked at chunk boundaries of 1000); 0.9 per 1000 steps is capped at
    # 5000; the third turns non-finite at 2000
    reqs = make_requests([(0.0, 100, 0.1, None, 10000), (0.0, 100, 0.9, None, 5000),
                          (0.0, 100, 0.1, 2000, 10000), (0.0, 100, 0.1, None, 10000),
                          (0.0, 100, 0.1, None, 10000)])
    srv = make(10_000, max_slots=2, mem_fraction=1.0, chunk=1000, graph_steps=0)
    srv.run(reqs, realtime=False)
    status = [r.status for r in reqs]
    assert status == ["converged", "capped", "unstable", "converged", "converged"]
    assert [r.steps for r in reqs] == [3000, 5000, 2000, 3000, 3000]
    assert all(r.finished is not None and r.admitted is not None for r in reqs)
    assert max(n for _, n, _ in srv.log) <= 2               # never more than max_slots resident
    assert [rid for rid, _ in trace["created"]] == [0, 1, 2, 3, 4]   # admitted in arrival order
    assert srv.in_use == 0                                    # every admission released
    assert "error" in reqs[2].result and "mass" in reqs[0].result
    # one batched diagnostics pass per chunk, whatever the number resident
    assert trace["diag_calls"] == len(srv.log)


def test_memory_budget_limits_admission(server_factory):
    make, trace = server_factory
    # three requests of 400 bytes against a budget of 1000: two at a time
    reqs = make_requests([(0.0, 400, 0.1, None, 10000)] * 3)
    srv = make(1000, max_slots=8, mem_fraction=1.0, chunk=1000, graph_steps=0)
    srv.run(reqs, realtime=False)
    assert all(r.status == "converged" for r in reqs)
    assert max(len(b) for b in trace["batches"]) == 2
    # the batch is rebuilt only when the resident set changes
    assert len(trace["batches"]) == 2
    assert reqs[2].admitted >= reqs[0].finished              # the third waited for room


def test_request_that_never_fits_is_reported(server_factory):
    make, _ = server_factory
    reqs = make_requests([(0.0, 5000, 0.1, None, 10000)])
    srv = make(1000, max_slots=8, mem_fraction=1.0, chunk=1000, graph_steps=0)
    with pytest.raises(RuntimeError, match="does not fit"):
        srv.run(reqs, realtime=False)


def test_late_arrival_joins_at_a_chunk_boundary(server_factory):
    make, trace = server_factory
    # the second request arrives after the first is already running (each
    # chunk takes 10 ms; the first needs 10 chunks)
    trace["step_sleep"] = 0.01
    reqs = make_requests([(0.0, 100, 0.5, None, 40000), (0.05, 100, 0.1, None, 10000)])
    srv = make(10_000, max_slots=4, mem_fraction=1.0, chunk=1000, graph_steps=0)
    srv.run(reqs, realtime=True)
    assert reqs[1].admitted >= 0.05 and reqs[1].admitted > reqs[0].admitted
    assert [0] in trace["batches"] and [0, 1] in trace["batches"]   # rebuilt when it joined
    assert all(r.status == "converged" for r in reqs)


def test_percentiles_skip_missing_values():
    p = serve.percentiles([1.0, None, 3.0, 2.0])
    assert p["p50"] == 2.0 and abs(p["p99"] - 2.98) < 1e-12
    assert serve.percentiles([None]) == {"p50": None, "p99": None}


def test_small_request_overtakes_one_that_does_not_fit(server_factory):
    make, trace = server_factory
    # a running request of 600 bytes leaves 400 of 1000; the next arrival
    # (500 bytes) does not fit, the one after it (300 bytes) does and is
    # admitted at once instead of waiting behind it
    reqs = make_requests([(0.0, 600, 0.5, None, 20000), (0.0, 500, 0.1, None, 10000),
                          (0.0, 300, 0.1, None, 10000)])
    srv = make(1000, max_slots=8, mem_fraction=1.0, chunk=1000, graph_steps=0)
    srv.run(reqs, realtime=False)
    assert all(r.status == "converged" for r in reqs)
    assert reqs[2].admitted < reqs[0].finished                # overtook request 1
    assert reqs[1].admitted >= reqs[0].finished               # which waited for room
    assert [rid for rid, _ in trace["created"]] == [0, 2, 1]


def test_starvation_limit_stops_overtaking(server_factory):
    make, trace = server_factory
    reqs = make_requests([(0.0, 600, 0.5, None, 20000), (0.0, 500, 0.1, None, 10000),
                          (0.0, 300, 0.1, None, 10000)])
    srv = make(1000, max_slots=8, mem_fraction=1.0, chunk=1000, graph_steps=0, starvation_s=0.0)
    srv.run(reqs, realtime=False)
    assert [rid for rid, _ in trace["created"]] == [0, 1, 2]


def test_admission_sees_memory_taken_by_others(server_factory):
    make, trace = server_factory
    # the ledger alone would admit both requests at once; another user of
    # the device takes 800 of the 1000 free bytes right after the first
    # admission and gives them back when the first request retires, so the
    # second request waits for the live free memory, not for the ledger
    state = {"free": 1000}
    reqs = make_requests([(0.0, 300, 0.1, None, 10000), (0.0, 300, 0.1, None, 10000)])
    srv = make(1000, free_fn=lambda *a: (state["free"], 1000), max_slots=8, mem_fraction=1.0, chunk=1000,
               graph_steps=0)
    orig_new, orig_close = serve.Server._new_lattice, serve.lbm.Lattice.close

    def take_memory(self, cfg):
        lat = orig_new(self, cfg)
        if cfg["rid"] == 0:
            state["free"] = 200
        return lat

    def give_back(lat):
        orig_close(lat)
        if lat.cfg["rid"] == 0:
            state["free"] = 1000

    serve.Server._new_lattice = take_memory
    serve.lbm.Lattice.close = give_back
    try:
        srv.run(reqs, realtime=False)
    finally:
        serve.Server._new_lattice = orig_new
        serve.lbm.Lattice.close = orig_close
    assert all(r.status == "converged" for r in reqs)
    assert trace["batches"][0] == [0]
    assert reqs[1].admitted >= reqs[0].finished


def test_fp32_solve_below_its_floor_finishes_in_fp64(server_factory):
    make, trace = server_factory
    # FP32 stalls at a residual of 1e-6 (reached after 6000 steps); the
    # target is 1e-8: once 20 checks bring no gain over the 20 before, the
    # solve moves to FP64 storage and finishes there
    reqs = make_requests([(0.0, 100, 0.1, None, 80000), (0.0, 100, 0.1, None, 80000)],
                         precision=1, tol=1e-8, floor=1e-6)
    reqs[1].tol = 2e-5                       # above the floor: stays FP32
    srv = make(10_000, max_slots=8, mem_fraction=1.0, chunk=1000, graph_steps=0, fp32_stall=1e-4)
    srv.run(reqs, realtime=False)
    assert [r.status for r in reqs] == ["converged", "converged"]
    assert reqs[0].switched_at == 40000 and reqs[0].steps == 41000
    assert reqs[1].switched_at is None and reqs[1].steps == 5000
    assert (0, 0) in trace["created"] and (1, 0) not in trace["created"]
    assert trace["copied"] == [0]
    assert srv.in_use == 0


def test_fp32_without_a_floor_caps(server_factory):
    make, _ = server_factory
    reqs = make_requests([(0.0, 100, 0.1, None, 60000)], precision=1, tol=1e-8, floor=1e-6)
    srv = make(10_000, max_slots=8, mem_fraction=1.0, chunk=1000, graph_steps=0, fp32_stall=None)
    srv.run(reqs, realtime=False)
    assert reqs[0].status == "capped" and reqs[0].switched_at is None


def test_fp32_plateau_above_the_floor_also_finishes_in_fp64(server_factory):
    make, trace = server_factory
    # a channel-like FP32 solve whose noise floor lies at 2e-5: the residual
    # stops falling and the solve moves to FP64
    reqs = make_requests([(0.0, 100, 0.5, None, 200000)], precision=1, tol=1e-7, floor=2e-5)
    srv = make(10_000, max_slots=8, mem_fraction=1.0, chunk=1000, graph_steps=0, fp32_stall=1e-4)
    srv.run(reqs, realtime=False)
    r = reqs[0]
    assert r.status == "converged" and r.switched_at is not None
    # 0.5 per 1000 steps reaches the 2e-5 floor after 16 chunks; the stall is
    # seen 40 checks in at the earliest
    assert 40000 <= r.switched_at <= 60000
    assert r.steps < r.switched_at + 30000


def test_stall_rule():
    assert not serve.fp32_stalled([1e-5] * 39)                 # too short to tell
    assert serve.fp32_stalled([1e-5] * 40)                     # flat below the ceiling
    assert not serve.fp32_stalled([3e-4] * 40)                 # flat above it: a start-up transient
    decaying = [10 ** (-3 - k / 20) for k in range(40)]        # a decade per 20 checks
    assert not serve.fp32_stalled(decaying)
    slow = [10 ** (-3 - k / 100) for k in range(40)]           # a decade per 100 checks: 0.63 per 20
    assert not serve.fp32_stalled(slow)
    assert not serve.fp32_stalled([1e-5] * 40, None)


def test_stall_window_grows_with_the_lattice():
    assert serve.stall_window(W.cavity(N=128)) == 20
    assert serve.stall_window(W.cavity(N=512)) == 20
    assert serve.stall_window(W.cavity(N=1024)) == 80
    # a decade per 280 checks, the 512^2 rate of a decade per 70 checks
    # scaled by the area of a 1024^2 lattice: below the ceiling the fixed
    # window took it for the floor, the scaled one does not
    slow = [10 ** (-4.2 - k / 280) for k in range(200)]
    assert serve.fp32_stalled(slow, window=20)
    assert not serve.fp32_stalled(slow, window=serve.stall_window(W.cavity(N=1024)))
    # a flat floor is still seen, after twice the longer window
    assert not serve.fp32_stalled([1e-6] * 159, window=80)
    assert serve.fp32_stalled([1e-6] * 160, window=80)


def test_deadline_stops_resident_solves(server_factory):
    make, trace = server_factory
    # two solves that never reach the target and a third that waits for a slot
    reqs = make_requests([(0.0, 100, 0.999, None, 10**9), (0.0, 100, 0.999, None, 10**9),
                          (0.0, 100, 0.1, None, 10**9)])
    trace["step_sleep"] = 0.01
    srv = make(10_000, max_slots=2, mem_fraction=1.0, chunk=1000, graph_steps=0)
    t0 = time.perf_counter()
    srv.run(reqs, realtime=False, deadline_s=0.2)
    assert time.perf_counter() - t0 < 5.0
    assert [r.status for r in reqs] == ["stopped", "stopped", "pending"]
    assert reqs[0].steps > 0 and reqs[2].steps == 0
    assert srv.in_use == 0
