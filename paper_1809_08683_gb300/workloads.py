"""Seeded synthetic workloads: the lattice problems of Sec. 4 of
arXiv:1809.08683 (thermal Couette, thermal Poiseuille, heated cavity) and the
batched / serving mixes built from them.

This module is shared by the tests, the oracle driver and bench.py.  It holds
problem set-up only (sizes, wall data, body forces, random draws) and none of
the lattice-Boltzmann arithmetic.  A configuration is a plain dict with the
fields of ``lbm_config`` (include/lbm.h) plus ``eos = {"kind", "params"}``.

Lattice units: dx = dt = 1, rho0 = T0 = 1.  Walls are wet nodes, so a walled
extent of n nodes has physical width n - 1.
"""
from __future__ import annotations

import math

import numpy as np

EOS_DECOUPLING, EOS_IDEAL, EOS_CS, EOS_CUBIC = 0, 1, 2, 3
WALL_S, WALL_N, WALL_W, WALL_E = 0, 1, 2, 3
VISC_CONST, VISC_LINEAR, VISC_SUTHERLAND = 0, 1, 2
SUTHERLAND_S_OVER_T0 = 110.5 / 600.0   # Sutherland constant over T0 = 600 K (Sec. 4.3)


def periodic():
    return {"periodic": 1, "thermal": 1, "extrap_order": 2, "u": (0.0, 0.0), "T": 1.0}


def wall(u=(0.0, 0.0), T=1.0, thermal=0, order=2):
    return {"periodic": 0, "thermal": int(thermal), "extrap_order": int(order),
            "u": (float(u[0]), float(u[1])), "T": float(T)}


def base(nx, ny, **kw):
    cfg = {
        "nx": int(nx), "ny": int(ny), "precision": 0, "visc_law": VISC_CONST,
        "rho0": 1.0, "T0": 1.0, "Pr": 0.71, "gamma": 1.4, "tau0": 0.8,
        "visc_p": (0.0, 0.0), "bulk_ratio": 1.0, "varpi": 1.0 / 6.0,
        "gamma1": -2.0, "gamma2": 2.0, "force_mode": 0, "corrections": 1,
        "force": (0.0, 0.0),
        "walls": [periodic(), periodic(), periodic(), periodic()],
        "eos": {"kind": EOS_IDEAL, "params": []},
    }
    cfg.update(kw)
    return cfg


def couette(nx=4, ny=64, U=0.05, T=1.0, tau0=0.8, Pr=0.71, gamma=1.4, precision=0):
    """Thermal Couette flow, both walls isothermal at T, lid at u = (U, 0)
    (north), periodic in x, second-order extrapolation, ideal gas."""
    return base(nx, ny, tau0=tau0, Pr=Pr, gamma=gamma, precision=precision,
                walls=[wall((0, 0), T, 0, 2), wall((U, 0), T, 0, 2), periodic(), periodic()],
                eos={"kind": EOS_IDEAL, "params": []})


def couette_variable_mu(nx=1, ny=32, Ma_e=0.1, tau0=0.8, Pr=0.71, gamma=1.4, eos=(EOS_IDEAL, ()), precision=0,
                        cp=None):
    """Thermal Couette flow with mu / mu0 = T / T0 (Sec. 4.2): adiabatic lower
    wall at rest (south, Neumann), upper wall moving at u = (U0, 0) and held
    at T0 = 1 (north, Dirichlet), periodic in x, second-order extrapolation,
    tau0 = 0.8 for mu0.  U0 = Ma_e sqrt(Cp T0).  cp is the heat capacity the
    configuration produces; the default, gamma / (gamma - 1) c_s^2 / T0, is
    that of the ideal and decoupling EOS at rho0 = T0 = 1.  For another EOS
    pass it (the paper's Eq. Cp gives 3.5 c_s^2 / T0 = 7/6 with the gamma
    it quotes for each EOS)."""
    if cp is None:
        cp = gamma / (gamma - 1.0) / 3.0
    U0 = Ma_e * math.sqrt(cp)
    return base(nx, ny, tau0=tau0, Pr=Pr, gamma=gamma, precision=precision, visc_law=VISC_LINEAR,
                walls=[wall((0, 0), 1.0, 1, 2), wall((U0, 0), 1.0, 0, 2), periodic(), periodic()],
                eos={"kind": int(eos[0]), "params": list(eos[1])})


def poiseuille_force(ny, U0, tau0, rho0=1.0):
    """Body force F_x giving centreline velocity U0 in a channel of width
    W = ny - 1 for dynamic viscosity mu = rho0 (tau0 - 1/2) / 3:
    U0 = F_x W^2 / (8 mu)."""
    W = ny - 1
    mu = rho0 * (tau0 - 0.5) / 3.0
    return 8.0 * mu * U0 / (W * W)


def poiseuille(nx=4, ny=128, U0=0.05, T=1.0, tau0=0.8, Pr=0.7, gamma=1.3,
               eos=(EOS_CUBIC, (0.05, 0.2)), precision=0, Th=None):
    """Thermal Poiseuille flow, walls at rest, lower wall at T (= T_c) and
    upper wall at Th (default T), constant body force, periodic in x,
    second-order extrapolation; default EOS is the cubic
    rho R T/(1 - b rho) - a rho^2 with a = 0.05, b = 0.2."""
    Fx = poiseuille_force(ny, U0, tau0)
    return base(nx, ny, tau0=tau0, Pr=Pr, gamma=gamma, precision=precision,
                force=(Fx, 0.0), force_mode=0,
                walls=[wall((0, 0), T, 0, 2), wall((0, 0), T if Th is None else Th, 0, 2), periodic(), periodic()],
                eos={"kind": int(eos[0]), "params": list(eos[1])})


def bulk_ratio_for(Ra, stable=True):
    """varsigma/nu per Table 1, extended to any Ra by decade.  With stable=True
    it is raised to 4 for every cavity: Sec. 4.3 raises varsigma/nu to enhance
    stability, and at eps up to 0.6 on lattices coarser than Table 1 the extra
    bulk damping of the impulsive start is what keeps the scheme stable."""
    if Ra <= 1e6 * (1 + 1e-9):
        r = 1.0
    elif Ra <= 1e7 * (1 + 1e-9):
        r = 2.0
    else:
        r = 4.0
    return max(r, 4.0) if stable else r


def cavity_gravity(N, Ra, eps, Pr=0.71, tau0=0.6):
    """Lattice gravity for Ra = Pr g rho0^2 (T_h - T_c) L^3 / (T0 mu0^2)
    with rho0 = T0 = 1, T_h - T_c = 2 eps, L = N - 1, mu0 = (tau0 - 1/2)/3."""
    L = N - 1
    mu0 = (tau0 - 0.5) / 3.0
    return Ra * mu0 * mu0 / (Pr * 2.0 * eps * L ** 3)


def sutherland_ratio(theta, S=SUTHERLAND_S_OVER_T0):
    """mu / mu0 at T / T0 = theta (Sec. 4.3, ratio form)."""
    return theta * math.sqrt(theta) * (1.0 + S) / (theta + S)


COLD_MARGIN = {EOS_IDEAL: 0.05, EOS_CUBIC: 0.068}


def tau_for(N, Ra, eps, tau_min=0.65, dtau_cold=None, u_peak=0.065, u_peak_over_uref=0.32,
            strat=0.15, Pr=0.71, eos=EOS_IDEAL):
    """Relaxation time at (rho0, T0) for a heated cavity of side N, and the
    Rayleigh number actually run.

    Lower bound: tau0 >= tau_min, and at the cold wall (T = 1 - eps,
    rho ~ 1/T, Sutherland mu) the local 1/s_p - 1/2 stays >= dtau_cold.
    Upper bound: the peak velocity, about 0.32 U_ref with
    U_ref = sqrt(Ra) nu0 / L (Table 2), stays below u_peak and the hydrostatic
    stratification 3 g L = 3 U_ref^2 / (Pr 2 eps) below strat.  tau0 is the
    lower bound; when it exceeds the upper bound (Ra too high for the
    lattice), Ra is lowered to the largest value that meets it.  The bounds
    come from GPU stability scans of eps up to 0.6 with varsigma/nu = 4 over
    6e4 steps, with about 10% headroom: the cold-wall margin is 0.05 for the
    ideal gas and 0.068 for the cubic EOS, whose cold, dense fluid has a
    much smaller p / rho."""
    if dtau_cold is None:
        dtau_cold = COLD_MARGIN.get(eos, 0.068)
    L = N - 1
    Tc = 1.0 - eps
    lo = max(tau_min, 0.5 + dtau_cold / (sutherland_ratio(Tc) * Tc))
    uref_max = min(u_peak / u_peak_over_uref, math.sqrt(strat * Pr * 2.0 * eps / 3.0))
    hi = 0.5 + 3.0 * L * uref_max / math.sqrt(Ra)
    if lo <= hi:
        return lo, Ra
    return lo, (3.0 * L * uref_max / (lo - 0.5)) ** 2


def cavity(N=512, Ra=1e6, eps=0.6, Pr=0.71, gamma=1.4, tau0=None,
           eos=(EOS_IDEAL, ()), precision=0, order=1):
    """Heated square cavity (Sec. 4.3): west wall hot T0(1+eps), east wall
    cold T0(1-eps), adiabatic south/north walls, all at rest; F = rho g with
    g = (0, -g); Sutherland viscosity; first-order extrapolation.  tau0=None
    picks tau0 (and, if the lattice is too coarse, a lower Ra) by tau_for."""
    Ra_req = Ra
    if tau0 is None:
        tau0, Ra = tau_for(N, Ra, eps, Pr=Pr, eos=int(eos[0]))
        bulk = bulk_ratio_for(Ra, stable=True)
    else:
        bulk = bulk_ratio_for(Ra, stable=False)
    g = cavity_gravity(N, Ra, eps, Pr, tau0)
    return base(N, N, tau0=tau0, Pr=Pr, gamma=gamma, precision=precision,
                visc_law=VISC_SUTHERLAND, visc_p=(SUTHERLAND_S_OVER_T0, 0.0),
                bulk_ratio=bulk, force_mode=1, force=(0.0, -g),
                walls=[wall((0, 0), 1.0, 1, order), wall((0, 0), 1.0, 1, order),
                       wall((0, 0), 1.0 + eps, 0, order), wall((0, 0), 1.0 - eps, 0, order)],
                eos={"kind": int(eos[0]), "params": list(eos[1])}, Ra=float(Ra), Ra_requested=float(Ra_req),
                eps=float(eps))


def periodic_box(nx, ny, tau0=0.8, Pr=0.71, gamma=1.4, eos=(EOS_IDEAL, ()), precision=0,
                 visc_law=VISC_CONST, force=(0.0, 0.0), force_mode=0, corrections=1):
    return base(nx, ny, tau0=tau0, Pr=Pr, gamma=gamma, precision=precision, visc_law=visc_law,
                visc_p=(SUTHERLAND_S_OVER_T0, 0.0), force=force, force_mode=force_mode,
                corrections=corrections, eos={"kind": int(eos[0]), "params": list(eos[1])})


def random_macros(nx, ny, seed, drho=0.02, du=0.03, dT=0.05, smooth=True):
    """Seeded random macroscopic fields (rho, ux, uy, T) around (1, 0, 0, 1):
    a few random Fourier modes (smooth) plus optional white noise."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx]
    out = []
    for amp, base_v in ((drho, 1.0), (du, 0.0), (du, 0.0), (dT, 1.0)):
        field = np.zeros((ny, nx))
        for _ in range(4):
            kx = rng.integers(0, 3) * 2 * math.pi / nx
            ky = rng.integers(0, 3) * 2 * math.pi / ny
            ph = rng.uniform(0, 2 * math.pi)
            field += rng.uniform(-1, 1) * np.cos(kx * x + ky * y + ph)
        field *= amp / 4.0
        if not smooth:
            field += 0.25 * amp * rng.uniform(-1, 1, size=(ny, nx))
        out.append(base_v + field)
    return tuple(out)


def df_noise(nx, ny, seed, amp=1e-4):
    """Seeded white noise for the 9 f and 9 g populations, [q][y][x]."""
    rng = np.random.default_rng(seed)
    return (amp * rng.standard_normal((9, ny, nx)), amp * rng.standard_normal((9, ny, nx)))


# --- batched sweep and serving mix --------------------------------------

SIZES = (128, 192, 256, 384, 512, 768, 1024)
TABLE1 = ((1e3, 128), (1e4, 192), (1e5, 256), (1e6, 512), (1e7, 1024), (1e8, 4096))


def grid_for_Ra(Ra, cap=1024):
    """Smallest lattice side in SIZES not below the Table-1 grid for Ra,
    log-interpolated between decades, capped at `cap`."""
    lr = math.log10(Ra)
    pts = [(math.log10(r), math.log2(n)) for r, n in TABLE1]
    if lr <= pts[0][0]:
        need = 2 ** pts[0][1]
    elif lr >= pts[-1][0]:
        need = 2 ** pts[-1][1]
    else:
        for (a, na), (b, nb) in zip(pts, pts[1:]):
            if a <= lr <= b:
                need = 2 ** (na + (nb - na) * (lr - a) / (b - a))
                break
    for s in SIZES:
        if s >= need - 1e-9 and s <= cap:
            return s
    return cap


def batched_sweep(n=96, seed=1809, precision=1, cap=1024):
    """96 heated cavities: Ra log-uniform in [1e3, 1e8], side from Ra,
    eps uniform in [0.1, 0.6], EOS ideal or cubic(0.05, 0.2) with p = 1/2."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        Ra = 10 ** rng.uniform(3, 8)
        eps = rng.uniform(0.1, 0.6)
        cubic = rng.uniform() < 0.5
        N = grid_for_Ra(Ra, cap)
        eos = (EOS_CUBIC, (0.05, 0.2)) if cubic else (EOS_IDEAL, ())
        out.append(cavity(N=N, Ra=Ra, eps=eps, eos=eos, precision=precision))
    return out


def serving_mix(n=2000, seed=1810, min_side=64, max_side=2048, mean_interarrival=0.05,
                tol=1e-7, max_steps=2_000_000, precision=1):
    """Poisson stream of cavity and channel solves: sides log-uniform in
    [min_side, max_side], Ra log-linear in the side from 1e3 (64) to 1e8
    (2048) for cavities, eps and EOS as in the batched sweep, channels of
    4..64 periodic columns (Poiseuille with the same EOS mix).  Returns a list
    of dicts {rid, cfg, arrival, tol, max_steps, kind}."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(mean_interarrival)
        side = int(round(math.exp(rng.uniform(math.log(min_side), math.log(max_side)))))
        side = max(8, side)
        eps = rng.uniform(0.1, 0.6)
        cubic = rng.uniform() < 0.5
        eos = (EOS_CUBIC, (0.05, 0.2)) if cubic else (EOS_IDEAL, ())
        if rng.uniform() < 0.5:
            Ra = 10 ** (3 + 5 * math.log(side / 64.0) / math.log(2048 / 64.0))
            Ra = max(Ra, 1e3)
            cfg = cavity(N=side, Ra=Ra, eps=eps, eos=eos, precision=precision)
            kind = "cavity"
        else:
            nx = int(rng.integers(4, 65))
            cfg = poiseuille(nx=nx, ny=side, eos=eos, gamma=1.3 if cubic else 1.4, precision=precision)
            kind = "channel"
        out.append({"rid": rid, "cfg": cfg, "arrival": t, "tol": tol, "max_steps": max_steps, "kind": kind})
    return out
