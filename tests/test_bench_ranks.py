"""Host-side rules of bench.py, without a GPU: on two CPU ranks (gloo) the
timed region's duration is the slowest rank's and the whole-job rate counts
every rank's replica of the workload; the reference arm runs on rank 0 only;
the clock record reports the median SM clock and the throttle reasons seen."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, dist, "cpu")
        rate = bench.whole_job_mlups(1000, 100, world, ms)
        with open(os.path.join(outdir, f"r{rank}"), "w") as fh:
            fh.write(f"{ms!r} {rate!r}")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for rank in range(world):
        ms, rate = (float(v) for v in (tmp_path / f"r{rank}").read_text().split())
        assert ms == 15.0                                   # the slower rank's time
        assert rate == pytest.approx(1000 * 100 * 2 / 15e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_mlups(10, 20, 1, 2.0) == pytest.approx(10 * 20 / 2e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import sys
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(bench.parse()) == 0        # no oracle work, no line
    assert capsys.readouterr().out == ""


def test_clock_summary_reads_samples_and_reasons(tmp_path):
    # nvidia-smi --format=csv,noheader,nounits lines: sm, max sm, power,
    # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    c.proc = object()                                   # as if the sampler ran
    (tmp_path / "clocks.csv").write_text(
        "2070, 2070, 950.1, Not Active, Not Active, Not Active, Not Active\n"
        "1980, 2070, 1399.8, Not Active, Not Active, Not Active, Active\n"
        "[N/A], 2070, 0.0, Not Active, Not Active, Not Active, Not Active\n"
        "2055, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active\n")
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]             # kept and noted, not a rejection reason


def test_clock_summary_without_a_sampler():
    with bench.Clocks(0) as c:                          # no nvidia-smi here, or no GPU behind it
        pass
    s = c.summary()
    assert s["sm_mhz"] is None and s["reasons"]


def test_traffic_figure_follows_the_kernel_code_not_its_comments(tmp_path, monkeypatch):
    import shutil
    src = tmp_path / "paper_1809_08683_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_1809_08683_gb300", "csrc", name), src / name)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic_demo.txt").write_text(
        f"# a summary\nkernel = k_demo\nworkload = demo\nsource_sha256 = {h}\ndram_bytes_per_launch = 12345\n")
    assert bench.read_traffic("demo", "k_demo") == 12345.0
    assert bench.read_traffic("demo", "k_other") is None and bench.read_traffic("other", "k_demo") is None
    first = src / bench.KERNEL_SOURCES[0]
    text = first.read_text()
    first.write_text("// a new comment line\n" + text.replace("\n", "\n  ", 3) + "\n/* block */\n")
    assert bench.kernel_source_hash() == h                # comments and blank space do not count
    assert bench.read_traffic("demo", "k_demo") == 12345.0
    first.write_text(text + "\nstatic int changed_code = 1;\n")
    assert bench.kernel_source_hash() != h
    assert bench.read_traffic("demo", "k_demo") is None    # the stored figure no longer applies
