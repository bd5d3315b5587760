"""Benchmark of the thermal MRT lattice-Boltzmann hot path (arXiv:1809.08683)
on GB300.

Default workload: the batched sweep of 96 heated cavities (sides 192..1024
from Ra log-uniform in [1e3, 1e8], eps in [0.1, 0.6], ideal or cubic EOS,
FP32 deviation storage; 39.2M nodes, 11 GB of DFs), advanced together.  One
bench step = `--chunk` time steps of every cavity.  Metric: MLUPS, one
lattice-node update of both f and g per node per time step.

Fields of the JSON line (rank 0):
  value     device-timed MLUPS over the timed region: the batch replayed
            from a CUDA graph of `chunk` time steps (one fused launch per
            launch group and one wall-pass launch per time step), in the
            launch shape the batch autotuner picked; CUDA events, inputs
            resident in HBM, state 11 GB >> 129 MB L2 (no flush needed)
  autotune  the batch's launch shape: default, pick, ms per step of each
  ungraphed the same batch stepped with per-step launches and per-step
            CUDA events, which also give the fused/wall-pass split
  e2e       same metric through the public API with host buffers: per bench
            step, equilibrium initialisation of every cavity from pinned host
            fields (H2D, lbm_batch_init_macros), the chunk of time steps, and
            the macroscopic fields back (D2H, lbm_batch_macros); with the rate
            of a plain pinned copy of the same bytes each way on this machine
  roofline  the fused kernel's algorithmic bytes (18 DF reads + 18 DF writes
            per node) over its CUDA-event duration, against the measured HBM
            copy bandwidth
  time_to_steady  the 512^2 Ra = 1e6 cavity run to residual 1e-8 (FP32, then
            FP64 once FP32 stalls), and the sweep's members of side <= 256 as
            one batch to residual 1e-5: p50/p99 seconds per solve
  serving   a Poisson stream of cavity and channel solves to residual 1e-7
            through the continuous-batching server; a subset solved four
            ways (batched or one at a time, FP32 then FP64 or FP64 only)
  fp64_path the FP64-storage kernel on a 2048^2 cavity against the probed
            FP64 FMA rate
  cpu_baseline  the FP64 CPU oracle on a bounded sample (rank 0, N = 1)
`--impl reference` times that oracle alone (the reference arm).
Multi-GPU: instances are independent, so each rank advances its own copy of
the batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import hashlib
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1809_08683_gb300 import workloads as W  # noqa: E402

BYTES_PER_NODE = {0: 288, 1: 144}   # 18 DF reads + 18 DF writes, FP64 / FP32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_sweep",
                    choices=["batched_sweep", "cavity512", "cavity4096", "poiseuille"])
    ap.add_argument("--precision", type=int, default=None, help="0 FP64, 1 FP32-deviation")
    ap.add_argument("--chunk", type=int, default=None, help="time steps per bench step")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tile", default=None, help="bx,by[,pair] for every lattice (default: batch autotuner)")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--serving", type=int, default=200,
                    help="requests in the served Poisson stream (0 to skip)")
    ap.add_argument("--serving-sides", default="64,128", help="smallest,largest side of the served stream")
    ap.add_argument("--serving-compare", type=int, default=6,
                    help="requests of the stream also solved batched/one at a time x FP32/FP64")
    ap.add_argument("--no-steady", action="store_true", help="skip the time-to-steady runs")
    ap.add_argument("--table2", type=float, default=None,
                    help="instead of the benchmark: run the Table 2 cavity at this Ra (1e3..1e8) on its Table 1 "
                         "grid and print time-averaged Nu and p* (--table2-steps, averaged over the last half)")
    ap.add_argument("--table2-steps", type=int, default=2_000_000)
    ap.add_argument("--sweep-steady", type=int, default=None, metavar="SIDE",
                    help="instead of the benchmark: serve the 96-cavity sweep's members of side <= SIDE as one "
                         "batch from rest to residual --sweep-steady-tol and print p50/p99 time to steady")
    ap.add_argument("--sweep-steady-tol", type=float, default=1e-5)
    ap.add_argument("--sweep-steady-deadline", type=float, default=None, help="seconds after which it stops")
    return ap.parse_args()


def workload(name, precision):
    if name == "batched_sweep":
        p = 1 if precision is None else precision
        cfgs = W.batched_sweep(precision=p)
        desc = {"workload": "batched_sweep_96_cavities", "instances": len(cfgs), "seed": 1809,
                "sides": "192..1024 from Ra in [1e3,1e8]", "eos": "ideal|cubic(a=0.05,b=0.2)",
                "precision": "fp32_dev" if p else "fp64"}
        return cfgs, desc, 100
    if name == "cavity512":
        p = 1 if precision is None else precision
        cfgs = [W.cavity(N=512, Ra=1e6, eps=0.6, precision=p)]
        return cfgs, {"workload": "cavity_512x512_Ra1e6_eps0.6", "precision": "fp32_dev" if p else "fp64"}, 1000
    if name == "cavity4096":
        p = 1 if precision is None else precision
        cfgs = [W.cavity(N=4096, Ra=1e8, eps=0.6, precision=p)]
        return cfgs, {"workload": "cavity_4096x4096_Ra1e8_eps0.6", "precision": "fp32_dev" if p else "fp64"}, 20
    p = 0 if precision is None else precision
    cfgs = [W.poiseuille(nx=4, ny=128, precision=p)]
    return cfgs, {"workload": "poiseuille_4x128_cubic", "precision": "fp32_dev" if p else "fp64"}, 1000


KERNEL_OF_PAIR = {0: "k_collide_stream", 1: "k_collide_pair", 2: "k_collide_pair", 3: "k_collide_stream",
                  4: "k_collide_warp", 5: "k_collide_warp2"}
KERNEL_SOURCES = ("lbm_gb300.cu", "lbm_node.cuh", "lbm_f2.cuh")


def kernel_source_hash():
    """SHA-256 over the kernel sources with comments and blank space
    removed, to tell whether a stored ncu figure still describes the
    kernels being run (a comment edit does not change the code)."""
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1809_08683_gb300", "csrc", name), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def read_traffic(workload, kernel):
    """DRAM bytes per fused launch from the committed ncu summary of this
    workload, or None when there is none or the kernels changed since."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    try:
        kv = {}
        with open(path) as fh:
            for line in fh:
                if "=" in line and not line.lstrip().startswith("#"):
                    k, v = line.split("=", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel") != kernel or kv.get("source_sha256") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lbm_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 7 and parts[0].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][1]), "reasons": reasons,
                "samples": len(rows)}


def _oracle_rate(cfg, threads, budget_s):
    import oracle
    o = oracle.Oracle(cfg, threads=threads)
    nodes = cfg["nx"] * cfg["ny"]
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > budget_s or steps >= 100000:
            break
    o.close()
    return nodes * steps / el / 1e6, steps, el


def cpu_baseline(cfgs, budget_s=12.0, single_s=4.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample: the first
    lattice of the workload, stepped until about budget_s seconds pass on
    every host core, and for about single_s seconds on one."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.build()
    cfg = dict(cfgs[0])
    v, steps, el = _oracle_rate(cfg, cores, budget_s)
    v1, steps1, el1 = _oracle_rate(cfg, 1, single_s)
    return {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{cfg['nx']}x{cfg['ny']} lattice (first of the workload), {steps} steps, FP64, "
                      f"{el:.1f} s",
            "single_core": {"value": v1, "steps": steps1, "s": el1}}


def _requests(mix, precision):
    from paper_1809_08683_gb300 import serve
    out = []
    for m in mix:
        c = dict(m["cfg"])
        c["precision"] = precision
        out.append(serve.Request(rid=m["rid"], cfg=c, arrival=m["arrival"], tol=m["tol"], max_steps=m["max_steps"]))
    return out


def _field_errors(a, b):
    """Errors of fields a against reference fields b: velocity relative to
    the largest speed, rho - 1 and T - 1 each relative to their own size."""
    umax = max(np.hypot(b["ux"], b["uy"]).max(), 1e-300)
    return {"u": float(max(np.abs(a["ux"] - b["ux"]).max(), np.abs(a["uy"] - b["uy"]).max()) / umax),
            "rho_dev": float(np.abs(a["rho"] - b["rho"]).max() / max(np.abs(b["rho"] - 1.0).max(), 1e-300)),
            "T_dev": float(np.abs(a["T"] - b["T"]).max() / max(np.abs(b["T"] - 1.0).max(), 1e-300))}


def serving_run(n, n_compare, sides=(24, 96)):
    """Continuous batching of a seeded Poisson stream of n cavity and channel
    solves (mean inter-arrival 50 ms, sides log-uniform in `sides` (24..96 by
    default), FP32 deviation storage
    finished in FP64 where FP32 stalls, residual target 1e-7, cap 600,000
    steps), honouring arrival times.  The first n_compare requests are also
    solved three more ways for the attribution of the speed-up: batched in
    FP64 only, and one at a time with per-step launches, FP32-then-FP64 and
    FP64 only (all with every request available at once); each FP32 result
    is compared with its own FP64 solve."""
    from paper_1809_08683_gb300 import serve
    mix = W.serving_mix(n=n, seed=1810, min_side=sides[0], max_side=sides[1],
                        mean_interarrival=0.05, tol=1e-7, max_steps=600_000, precision=1)
    reqs = _requests(mix, 1)
    srv = serve.Server(max_slots=64, chunk=1000, graph_steps=10)
    srv.run(reqs, realtime=True)
    lat = [r.latency for r in reqs]
    node_steps = sum(r.steps * r.nodes for r in reqs)
    out = {"requests": n, "tol": 1e-7, "wall_s": srv.wall, "mlups": node_steps / srv.wall / 1e6,
           **{k + "_latency_s": v for k, v in serve.percentiles(lat).items()},
           "converged": sum(r.status == "converged" for r in reqs),
           "capped": sum(r.status == "capped" for r in reqs),
           "unstable": sum(r.status == "unstable" for r in reqs),
           "finished_in_fp64": sum(r.switched_at is not None for r in reqs),
           "host_overhead": srv.host_overhead, "device_busy": srv.device_busy, "host_s": srv.host_s,
           "chunks": srv.chunks,
           "batch_rebuilds": srv.rebuilds,
           "mix": f"Poisson stream (mean 50 ms), cavities and channels, sides {sides[0]}..{sides[1]}, "
                  f"seed 1810, FP32 then FP64 where FP32 stalls"}
    if n_compare <= 0:
        return out
    sub = mix[:n_compare]
    cells = {}
    # batched, FP32 then FP64 (the same requests as above, all at once)
    b32 = _requests(sub, 1)
    s32 = serve.Server(max_slots=64, chunk=1000, graph_steps=10, keep_fields=True)
    s32.run(b32, realtime=False)
    cells["batched_fp32_then_fp64"] = s32.wall
    b64 = _requests(sub, 0)
    s64 = serve.Server(max_slots=64, chunk=1000, graph_steps=10, keep_fields=True)
    s64.run(b64, realtime=False)
    cells["batched_fp64"] = s64.wall
    for prec, name in ((1, "sequential_fp32_then_fp64"), (0, "sequential_fp64")):
        t0 = time.perf_counter()
        for r in _requests(sub, prec):
            serve.solve_sequential(r)
        cells[name] = time.perf_counter() - t0
    errs = []
    for a, b in zip(b32, b64):
        if a.status == "converged" and b.status == "converged":
            e = _field_errors(a.result["fields"], b.result["fields"])
            if "nusselt" in b.result:
                e["nu"] = abs(a.result["nusselt"] / b.result["nusselt"] - 1.0)
            errs.append(e)
    worst = {k: max((e[k] for e in errs if k in e), default=None) for k in ("u", "rho_dev", "T_dev", "nu")}
    out["compare"] = {
        "requests": n_compare, "wall_s": cells,
        "speedup_vs_sequential_fp64": cells["sequential_fp64"] / cells["batched_fp32_then_fp64"],
        "from_batching_fp32": cells["sequential_fp32_then_fp64"] / cells["batched_fp32_then_fp64"],
        "from_fp32_batched": cells["batched_fp64"] / cells["batched_fp32_then_fp64"],
        "converged": {"fp32_then_fp64": sum(r.status == "converged" for r in b32),
                      "fp64": sum(r.status == "converged" for r in b64)},
        "max_error_vs_own_fp64_solve": worst, "compared": len(errs),
        "within_tolerance": all((e["u"] <= 1e-4 and e["rho_dev"] <= 1e-3 and e["T_dev"] <= 1e-3
                                 and e.get("nu", 0.0) <= 5e-3) for e in errs)}
    return out


def steady_cavity512(tol=1e-8):
    """The 512^2 heated cavity at Ra = 1e6, eps = 0.6, ideal gas,
    Sutherland viscosity, run from rest to residual `tol` in FP32 deviation
    storage, finished in FP64 once FP32 stalls; its lone launch shape from
    the autotuner.  Nu_ave and p*_ave against Table 2."""
    from paper_1809_08683_gb300 import autotune, serve
    cfg = W.cavity(N=512, Ra=1e6, eps=0.6, precision=1)
    req = serve.Request(rid=0, cfg=cfg, tol=tol, max_steps=3_000_000)
    srv = serve.Server(max_slots=1, chunk=1000, graph_steps=1000, tile_fn=lambda c: autotune.tune(c, steps=10))
    for prec in (1, 0):                 # tune outside the timed solve
        autotune.tune(dict(cfg, precision=prec), steps=10)
    srv.run([req], realtime=False)
    nu, ps = req.result.get("nusselt"), req.result.get("pstar")
    return {"workload": "cavity_512x512_Ra1e6_eps0.6", "tol": tol, "status": req.status, "s": req.latency,
            "steps": req.steps, "fp64_from_step": req.switched_at, "nu": nu, "pstar": ps,
            "table2": {"nu": 8.7406, "pstar": 0.91820},
            "nu_vs_table2": None if nu is None else nu / 8.7406 - 1.0,
            "pstar_vs_table2": None if ps is None else ps / 0.91820 - 1.0}


TABLE2 = {1e3: (128, 1.1063, 0.93443), 1e4: (192, 2.2123, 0.91144), 1e5: (256, 4.4836, 0.91719),
          1e6: (512, 8.7406, 0.91820), 1e7: (1024, 16.4373, 0.91425), 1e8: (4096, 29.9435, 0.91609)}


def table2_run(Ra, steps, every=20_000):
    """The heated cavity of Sec. 4.3 at Ra on its Table 1 grid (eps = 0.6,
    ideal gas, Sutherland viscosity, varsigma/nu of Table 1 from the
    stability rule), FP32 deviation storage, from rest: hot- and cold-wall
    Nu and p* every `every` steps, averaged over the second half of the
    run (at Ra = 1e8 the flow is unsteady), against Table 2."""
    import torch
    from paper_1809_08683_gb300 import lbm
    N, nu_ref, p_ref = TABLE2[Ra]
    tau0, ra_run = W.tau_for(N, Ra, 0.6)
    # the exact Ra with the stability rule's tau0 where its velocity bound
    # would lower Ra (Ra = 1e7: tau0 = 0.744, varsigma/nu of Table 1)
    cfg = W.cavity(N=N, Ra=Ra, eps=0.6, precision=1, tau0=None if ra_run >= Ra else tau0)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        lat = lbm.Lattice(cfg, stream=st)
    batch = lbm.Batch([lat], graph_steps=1000)
    rec = []
    t0 = time.perf_counter()
    for n in range(every, steps + 1, every):
        batch.step(every)
        d = lat.diagnostics()
        rec.append((n, lat.nusselt(W.WALL_W), lat.nusselt(W.WALL_E), d["pstar"]))
    wall = time.perf_counter() - t0
    batch.close()
    lat.close()
    second = [r for r in rec if r[0] > steps // 2]
    nu = float(np.mean([r[1] for r in second]))
    ps = float(np.mean([r[3] for r in second]))
    return {"Ra": Ra, "grid": N, "tau0": cfg["tau0"], "bulk_ratio": cfg["bulk_ratio"], "steps": steps,
            "average_over_steps": [second[0][0], second[-1][0]], "nu_hot": nu,
            "nu_hot_std": float(np.std([r[1] for r in second])),
            "nu_cold": float(np.mean([r[2] for r in second])), "pstar": ps,
            "table2": {"nu": nu_ref, "pstar": p_ref}, "nu_vs_table2": nu / nu_ref - 1.0,
            "pstar_vs_table2": ps / p_ref - 1.0, "wall_s": wall,
            "series": [[r[0], round(r[1], 5), round(r[2], 5), round(r[3], 6)] for r in rec[::5]]}


# FP64 operations per node update of the heated-cavity model, counted by
# instantiating the node templates with an operation-counting number type:
# 308 additions, 289 multiplications, 10 divisions, 1 square root, and
# about 36 for the gradient stencil.
FP64_OPS_PER_NODE = 644


def fp64_path(n_side=2048, steps=10):
    """The FP64-storage fused kernel on an n_side^2 heated cavity (Ra =
    1e8, eps = 0.6, block strips): per-step time and counted FP64 operation
    rate against the device's probed FP64 FMA rate, which bounds it."""
    import torch
    from paper_1809_08683_gb300 import lbm
    st = torch.cuda.Stream()
    rates = lbm.peak_rates(st)
    cfg = W.cavity(N=n_side, Ra=1e8, eps=0.6, precision=0)
    out = {"workload": f"cavity_{n_side}x{n_side}_Ra1e8_eps0.6_fp64", "rates": rates,
           "ops_per_node": FP64_OPS_PER_NODE}
    with torch.cuda.stream(st):
        lat = lbm.Lattice(cfg, stream=st)
    for name, tile in (("native_fp64", (128, 8, 0)),):
        lat.set_tile(*tile)
        b = lbm.Batch([lat], graph_steps=0)
        b.step_profiled(3)
        ms, _ = b.step_profiled(steps)
        b.close()
        mlups = n_side * n_side * steps / (ms * 1e-3) / 1e6
        out[name] = {"tile": list(tile), "fused_ms_per_step": ms / steps, "mlups": mlups,
                     "counted_gflops": mlups * FP64_OPS_PER_NODE / 1e3}
    lat.close()
    # FP64 FMA counts two operations
    out["native_fp64"]["frac_of_fp64_peak"] = out["native_fp64"]["counted_gflops"] * 1e9 / (2 * rates["fp64_fma_per_s"])
    return out


def steady_sweep_subset(tol=1e-5, max_side=256, deadline_s=None):
    """The 96-cavity sweep's members of side <= max_side served as one batch from rest
    to residual `tol` (FP32, FP64 finish where FP32 stalls): p50/p99 of the
    per-member time to steady.  deadline_s stops the run after that many
    seconds; percentiles then cover the members that finished."""
    from paper_1809_08683_gb300 import serve
    cfgs = [c for c in W.batched_sweep(precision=1) if c["nx"] <= max_side]
    reqs = [serve.Request(rid=i, cfg=c, tol=tol, max_steps=1_000_000) for i, c in enumerate(cfgs)]
    srv = serve.Server(max_slots=len(reqs), chunk=1000, graph_steps=1000)
    srv.run(reqs, realtime=False, deadline_s=deadline_s)
    out = {"workload": f"batched_sweep_96_cavities members of side <= {max_side}", "members": len(reqs),
           "tol": tol, **{k + "_s": v for k, v in serve.percentiles([r.latency for r in reqs]).items()},
           "wall_s": srv.wall, "converged": sum(r.status == "converged" for r in reqs),
           "capped": sum(r.status == "capped" for r in reqs),
           "unstable": sum(r.status == "unstable" for r in reqs),
           "finished_in_fp64": sum(r.switched_at is not None for r in reqs),
           "mlups": sum(r.steps * r.nodes for r in reqs) / srv.wall / 1e6}
    if deadline_s is not None:
        out["deadline_s"] = deadline_s
        out["stopped"] = sum(r.status == "stopped" for r in reqs)
        out["stopped_sides"] = sorted({r.cfg["nx"] for r in reqs if r.status == "stopped"})
        out["stopped_in_fp64"] = sum(r.status == "stopped" and r.switched_at is not None for r in reqs)
    return out


def host_link(h2d_bytes, d2h_bytes, dev, stream):
    """Rate of one plain pinned-host copy of the end-to-end step's byte
    counts in each direction (GB/s, best of 3): the copy floor that the
    end-to-end figure carries on this machine."""
    import torch
    hi = torch.empty(h2d_bytes // 8, dtype=torch.float64).pin_memory()
    ho = torch.empty(d2h_bytes // 8, dtype=torch.float64).pin_memory()
    d = torch.empty(max(hi.numel(), ho.numel()), dtype=torch.float64, device=dev)
    out = {}
    with torch.cuda.stream(stream):
        for name, fn, nbytes in (("h2d", lambda: d[:hi.numel()].copy_(hi, non_blocking=True), h2d_bytes),
                                 ("d2h", lambda: ho.copy_(d[:ho.numel()], non_blocking=True), d2h_bytes)):
            best = None
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            out[name] = nbytes / (best * 1e-3) / 1e9
    del hi, ho, d
    return out


def max_over_ranks(value, world, dist=None, device=None):
    """The largest of a per-rank float over all ranks (all_reduce MAX), the
    bench's rule for timed regions; `value` itself when world == 1."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, time_steps, world, ms):
    """Whole-job lattice updates per second (millions): every rank advances
    its own replica of the workload, over the slowest rank's time."""
    return nodes_per_rank * time_steps * world / (ms * 1e-3) / 1e6


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfgs, desc, _ = workload(args.workload, args.precision)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    cfg = dict(cfgs[0])
    o = oracle.Oracle(cfg, threads=cores)
    nodes = cfg["nx"] * cfg["ny"]
    per_step = max(1, int(2e6 // nodes))   # about 1-2 s of oracle work per bench step
    for _ in range(args.warmup):
        o.step(per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per_step)
    el = time.perf_counter() - t0
    v = nodes * per_step * args.steps / el / 1e6
    sample = f"{cfg['nx']}x{cfg['ny']} lattice (first of the workload), {per_step} time steps per bench step, FP64"
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": desc,
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_1809_08683_gb300 import autotune, lbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    lbm.build()
    lbm.load()
    if args.table2 is not None:
        if rank == 0:
            print(json.dumps(table2_run(args.table2, args.table2_steps)))
        return 0
    if args.sweep_steady is not None:
        if rank == 0:
            print(json.dumps(steady_sweep_subset(tol=args.sweep_steady_tol, max_side=args.sweep_steady,
                                                 deadline_s=args.sweep_steady_deadline)))
        return 0

    cfgs, desc, chunk = workload(args.workload, args.precision)
    chunk = args.chunk or chunk
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        lats = [lbm.Lattice(c, stream=stream, device=dev) for c in cfgs]
    tuned = None
    if args.tile:
        t = [int(v) for v in args.tile.split(",")]
        for lat in lats:
            lat.set_tile(t[0], t[1], t[2] if len(t) > 2 else 0)
    elif not args.no_tune:
        best, res = autotune.tune_batch(lats)
        tuned = {"pick": None if best is None else list(best), "ms_per_step": {
            ("default" if k is None else ",".join(map(str, k))): v for k, v in res.items()},
            "default_ms": res[None], "pick_ms": res[best]}
    nodes = sum(c["nx"] * c["ny"] for c in cfgs)
    prec = int(cfgs[0].get("precision", 0))
    graph_steps = chunk if chunk % 2 == 0 else 0
    batch = lbm.Batch(lats, graph_steps=graph_steps)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        batch.step(chunk)
    barrier()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            batch.step(chunk)
        ev1.record(stream)
        ev1.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    for lat in lats:        # a run that produced NaN/Inf is not a measurement
        lat.sync()
    ms = max_over_ranks(ms, world, dist, dev)
    steps_total = args.steps * chunk
    value = whole_job_mlups(nodes, steps_total, world, ms)
    clocks = clk.summary()

    # the same batch with per-step launches and events: fused / wall-pass split
    pbatch = lbm.Batch(lats, graph_steps=0)
    psteps = min(steps_total, 5 * chunk)
    pbatch.step_profiled(chunk)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t_collide, t_wall = pbatch.step_profiled(psteps)
    e1.record(stream)
    e1.synchronize()
    pbatch.close()
    ungraphed = {"value": nodes * psteps / (e0.elapsed_time(e1) * 1e-3) / 1e6, "steps": psteps,
                 "fused_ms_per_step": t_collide / psteps, "wall_pass_ms_per_step": t_wall / psteps}

    # fused kernel against the HBM roofline
    peak, peak_kind = read_peaks()
    avg_collide_ms = t_collide / psteps
    alg_bytes = nodes * BYTES_PER_NODE[prec]
    achieved = alg_bytes / (avg_collide_ms * 1e-3) / 1e9
    kernels = sorted({KERNEL_OF_PAIR[lat.tile()[2]] for lat in lats})
    kernel = "+".join(kernels)
    n_collide_launches = len({(lat.tile()[0], lat.tile()[2], lat.cfg.get("precision", 0)) for lat in lats})
    gpu_launches = steps_total * (n_collide_launches + 1)
    traffic = read_traffic(desc["workload"], kernel)

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        host_in = []
        for c in cfgs:
            shp = (c["ny"], c["nx"])
            fields = []
            for v in (1.0, 0.0, 0.0, 1.0):
                t = torch.full(shp, v, dtype=torch.float64).pin_memory()
                fields.append(t.numpy())
            host_in.append(fields)
        host_out = [{k: torch.empty((c["ny"], c["nx"]), dtype=torch.float64).pin_memory().numpy()
                     for k in ("rho", "ux", "uy", "T", "p")} for c in cfgs]

        def e2e_step():
            # every member's fields up and results down, one round trip each way
            batch.init_macros(host_in)
            batch.step(chunk)
            st = batch.macros(host_out)
            if any(v != lbm.LBM_OK for v in st):
                raise lbm.LbmError(max(st, key=abs), "a member failed during the end-to-end run")

        e2e_step()  # untimed warm-up: the first host round trip of a process runs slow
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        barrier()
        el = time.perf_counter() - t0
        el = max_over_ranks(el, world, dist, dev)
        e2e = {"value": whole_job_mlups(nodes, chunk * args.e2e_steps, world, el * 1e3), "unit": "MLUPS",
               "h2d_bytes_per_step": nodes * 4 * 8, "d2h_bytes_per_step": nodes * 5 * 8,
               "host_link_gbps": host_link(nodes * 4 * 8, nodes * 5 * 8, dev, stream)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(cfgs)

    batch.close()
    for lat in lats:
        lat.close()
    lats, batch = [], None
    torch.cuda.empty_cache()

    fp64 = None
    if rank == 0 and not args.no_steady and args.workload == "batched_sweep":
        fp64 = fp64_path()
    steady = None
    if rank == 0 and not args.no_steady and args.workload == "batched_sweep":
        steady = {"cavity512": steady_cavity512(), "sweep_subset": steady_sweep_subset()}
    serving = None
    if rank == 0 and args.serving > 0:
        serving = serving_run(args.serving, args.serving_compare,
                              tuple(int(v) for v in args.serving_sides.split(",")))

    if rank == 0:
        desc = dict(desc)
        desc.update({"nodes": nodes, "time_steps_per_bench_step": chunk, "graph_steps": graph_steps,
                     "l2": "state larger than L2 (no flush)" if alg_bytes > 2 * 129e6 else "state may be L2-resident"})
        out = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec else "f64",
            "data": "synthetic", "config": desc,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                         "kernel": kernel, "alg_bytes_per_launch": alg_bytes,
                         "avg_launch_ms": avg_collide_ms, "wall_pass_ms_per_step": t_wall / psteps},
            "autotune": tuned, "ungraphed": ungraphed,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches, "clocks": clocks,
            "time_to_steady": steady, "fp64_path": fp64, "serving": serving,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
