"""The seeded synthetic inputs (the input recipe): determinism, the sizes the
benchmark quotes, and the parameter rules that derive gravity, tau0 and the
grid from Ra."""
import math

import numpy as np

from paper_1809_08683_gb300 import workloads as W


def test_batched_sweep_is_deterministic_and_sized_as_quoted():
    a, b = W.batched_sweep(), W.batched_sweep()
    assert len(a) == 96 and a == b
    assert sum(c["nx"] * c["ny"] for c in a) == 39_165_952
    assert {c["nx"] for c in a} <= set(W.SIZES)
    assert all(c["nx"] == c["ny"] and c["precision"] == 1 for c in a)
    kinds = {c["eos"]["kind"] for c in a}
    assert kinds == {W.EOS_IDEAL, W.EOS_CUBIC}
    assert all(1e3 <= c["Ra_requested"] <= 1e8 and 0.1 <= c["eps"] <= 0.6 for c in a)
    assert W.batched_sweep(seed=7) != a


def test_cavity_gravity_reproduces_ra():
    # Ra = Pr g rho0^2 (T_h - T_c) L^3 / (T0 mu0^2), rho0 = T0 = 1, T_h - T_c = 2 eps
    for N, Ra, eps, tau0 in ((33, 1e3, 0.6, 0.8), (257, 1e6, 0.3, 0.62)):
        g = W.cavity_gravity(N, Ra, eps, Pr=0.71, tau0=tau0)
        mu0 = (tau0 - 0.5) / 3.0
        assert abs(0.71 * g * 2 * eps * (N - 1) ** 3 / mu0 ** 2 / Ra - 1) < 1e-12
    cfg = W.cavity(N=65, Ra=1e4, eps=0.5, tau0=0.7)
    assert cfg["force"][0] == 0.0 and cfg["force"][1] < 0 and cfg["force_mode"] == 1


def test_tau_rule_keeps_the_cold_wall_margin_and_lowers_ra_only_when_needed():
    for N, Ra, eps, eos in ((512, 1e6, 0.6, W.EOS_IDEAL), (64, 1e8, 0.6, W.EOS_CUBIC), (1024, 1e3, 0.1, W.EOS_IDEAL)):
        tau0, Ra_run = W.tau_for(N, Ra, eps, eos=eos)
        Tc = 1.0 - eps
        margin = W.COLD_MARGIN[eos]
        assert tau0 >= 0.65 - 1e-12
        assert tau0 >= 0.5 + margin / (W.sutherland_ratio(Tc) * Tc) - 1e-12
        assert Ra_run <= Ra * (1 + 1e-12)
    # a lattice far too coarse for the requested Ra gets a lower one
    _, Ra_run = W.tau_for(64, 1e8, 0.6)
    assert Ra_run < 1e8
    assert abs(W.sutherland_ratio(1.0) - 1.0) < 1e-15


def test_grid_rule_is_monotone_and_capped():
    sides = [W.grid_for_Ra(10 ** e) for e in np.linspace(3, 8, 41)]
    assert all(s in W.SIZES for s in sides)
    assert sides == sorted(sides) and max(sides) <= 1024
    assert W.grid_for_Ra(1e8, cap=512) == 512


def test_serving_mix_is_a_seeded_poisson_stream():
    a = W.serving_mix(n=200, seed=3, min_side=48, max_side=160)
    assert a == W.serving_mix(n=200, seed=3, min_side=48, max_side=160)
    t = [r["arrival"] for r in a]
    assert all(x < y for x, y in zip(t, t[1:]))
    assert {r["kind"] for r in a} == {"cavity", "channel"}
    assert all(48 <= r["cfg"]["ny"] <= 160 for r in a)
    assert abs(np.mean(np.diff([0.0] + t)) / 0.05 - 1) < 0.25   # mean inter-arrival 50 ms


def test_poiseuille_force_gives_the_centreline_velocity():
    # U0 = F_x W^2 / (8 mu), mu = rho0 (tau0 - 1/2) / 3
    F = W.poiseuille_force(128, 0.05, 0.8)
    assert abs(F * 127 ** 2 / (8 * 0.1) - 0.05) < 1e-15
    cfg = W.poiseuille(nx=4, ny=128, Th=1.01)
    assert cfg["walls"][0]["T"] == 1.0 and cfg["walls"][1]["T"] == 1.01


def test_couette_variable_mu_lid_speed():
    c = W.couette_variable_mu(Ma_e=0.1)
    assert abs(c["walls"][1]["u"][0] - 0.1 * math.sqrt(1.4 / 0.4 / 3.0)) < 1e-15
    assert c["walls"][0]["thermal"] == 1 and c["walls"][1]["thermal"] == 0 and c["visc_law"] == W.VISC_LINEAR
    c = W.couette_variable_mu(Ma_e=0.1, cp=3.5 / 3.0)
    assert abs(c["walls"][1]["u"][0] - 0.1 * math.sqrt(3.5 / 3.0)) < 1e-15
