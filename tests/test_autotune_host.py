"""Host logic of the launch-shape autotuner on the CPU: candidate shapes,
size classes, choice of the fastest measured shape, and the per-class cache
(timing itself is replaced by a scripted function)."""
import json

import pytest

from paper_1809_08683_gb300 import autotune
from paper_1809_08683_gb300 import workloads as W


def test_size_class_and_key():
    assert [autotune.size_class(n) for n in (1, 16, 17, 100, 128, 129)] == [16, 16, 32, 128, 128, 256]
    assert autotune.key_for(W.cavity(N=100, precision=1)) == "p1_x128_y128"
    assert autotune.key_for(W.couette(nx=4, ny=64)) == "p0_x16_y64"


def test_candidates_follow_precision_and_size():
    c64 = autotune.candidates(W.cavity(N=300))                 # FP64
    assert {p for _, _, p in c64} == {0, 4}                     # no packed-FP32 shapes
    c32 = autotune.candidates(W.cavity(N=300, precision=1))
    assert {p for _, _, p in c32} == {0, 1, 2, 3, 4, 5}
    assert set(c64) < set(c32)
    # narrow lattice: strips more than twice as wide as the lattice are skipped
    narrow = autotune.candidates(W.couette(nx=40, ny=12, precision=1))
    assert all(bx <= 32 or 40 > bx // 2 for bx, _, _ in narrow)
    assert (128, 4, 0) not in narrow and (32, 4, 0) in narrow
    # runs longer than the lattice is tall are skipped, except the shortest
    assert all(by <= 12 or by == autotune.BY_CANDIDATES[0] for _, by, _ in narrow)


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_CACHE_PATH", str(tmp_path / "tiles.json"))
    calls = []

    def fake_measure(cfg, bx, by, pair=0, steps=20, stream=None):
        calls.append((bx, by, pair))
        # one shape is 50 MLUPS faster than the rest; longer runs a little slower
        return 1000.0 + (50.0 if (bx, by, pair) == (64, 8, 0) else 0.0) - by * 0.1

    monkeypatch.setattr(autotune, "measure", fake_measure)
    cfg = W.cavity(N=300, precision=1)
    best = autotune.tune(cfg, steps=2)
    assert best == (64, 8, 0)
    assert len(calls) == len(autotune.candidates(cfg))         # every candidate timed once
    n = len(calls)
    assert autotune.tune(cfg) == best and len(calls) == n      # served from the cache
    with open(tmp_path / "tiles.json") as fh:
        entry = json.load(fh)[autotune.key_for(cfg)]
    assert entry["tile"] == [64, 8, 0] and entry["mlups"] == pytest.approx(1049.2)
    # another lattice of the same size class shares the entry
    assert autotune.tune(W.cavity(N=290, precision=1)) == best and len(calls) == n
    # force re-measures
    autotune.tune(cfg, force=True)
    assert len(calls) == 2 * n


def test_apply_sets_every_lattice(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "_CACHE_PATH", str(tmp_path / "tiles.json"))
    monkeypatch.setattr(autotune, "measure", lambda cfg, bx, by, pair=0, steps=20, stream=None: float(bx + by))

    class FakeLattice:
        def __init__(self, cfg):
            self.cfg, self.stream, self.tile = cfg, None, None

        def set_tile(self, bx, by, pair):
            self.tile = (bx, by, pair)

    lats = [FakeLattice(W.cavity(N=300)), FakeLattice(W.couette(nx=40, ny=12))]
    autotune.apply(lats, steps=2)
    for lat in lats:
        assert lat.tile == max(autotune.candidates(lat.cfg), key=lambda t: t[0] + t[1])


def test_tune_batch_picks_fastest_shape_and_applies_it(monkeypatch):
    timings = {None: 1.30, (128, 16, 1): 1.31, (128, 24, 1): 1.28, (128, 32, 1): 1.25, (128, 48, 1): 1.27,
               (256, 32, 1): 1.40, (128, 24, 0): 1.39}
    seen = []

    def fake_measure(lattices, shape, steps=10, warmup=3):
        seen.append(shape)
        return timings[shape]

    class FakeLattice:
        def __init__(self, precision):
            self.cfg, self.tiles = {"precision": precision}, []

        def set_tile(self, *t):
            self.tiles.append(t)

    monkeypatch.setattr(autotune, "measure_batch", fake_measure)
    lats = [FakeLattice(1), FakeLattice(1)]
    best, res = autotune.tune_batch(lats)
    assert best == (128, 32, 1) and res[best] == 1.25
    assert seen == list(autotune.BATCH_SHAPES)
    assert all(l.tiles[-1] == (128, 32, 1) for l in lats)
    # an FP64 member rules out the packed-FP32 shapes; the default can win
    seen.clear()
    lats = [FakeLattice(1), FakeLattice(0)]
    best, res = autotune.tune_batch(lats)
    assert set(res) == {None, (128, 24, 0)} and best is None
    assert all(l.tiles[-1] == (0, 0, 0) for l in lats)
