"""Closed-form solutions of the paper's validation flows, shared by the
oracle pins and the GPU tests (test infrastructure, not the method)."""
import numpy as np


def couette_mu_profile(xi, Ma_e, Pr):
    """Closed form of Sec. 4.2's thermal Couette flow with mu / mu0 = T / T0,
    Pr and Cp constant, lower wall adiabatic and at rest, lid at U0 and T0
    (Eq. Couette.u.T): s = u_x / U0 solves
    s + (Pr Ma_e^2 / 2)(s - s^3 / 3) = (1 + Pr Ma_e^2 / 3) xi,  xi = y / W,
    and T / T0 = 1 + (Pr Ma_e^2 / 2)(1 - s^2).  The left side increases with
    s on [0, 1], so Newton's method from s = xi converges."""
    a = 0.5 * Pr * Ma_e * Ma_e
    rhs = (1.0 + Pr * Ma_e * Ma_e / 3.0) * np.asarray(xi, dtype=np.float64)
    s = rhs.copy()
    for _ in range(50):
        s = s - (s + a * (s - s ** 3 / 3.0) - rhs) / (1.0 + a * (1.0 - s * s))
    return s, 1.0 + a * (1.0 - s * s)


def cs_pressure(rho, T, R, b):
    """Carnahan-Starling EOS p = Z rho R T, Z = (1 + e + e^2 - e^3) / (1 - e)^3,
    e = b rho / 4 (Eq. EOSs.3)."""
    e = b * rho / 4.0
    return (1.0 + e + e * e - e ** 3) / (1.0 - e) ** 3 * rho * R * T


def uniform_pressure_density(T, mean_rho, pressure, rho_max=None):
    """Density profile of a channel at rest in x with uniform pressure and a
    given mean density (Eq. rho.analytical.3): for a trial pressure p each
    node's rho solves pressure(rho, T) = p by bisection on [0, rho_max]
    (default 4 mean_rho; the pressure must increase with rho there), and p is
    found by bisection so that the mean of rho matches."""
    T = np.asarray(T, dtype=np.float64)
    rho_max = 4.0 * mean_rho if rho_max is None else rho_max

    def rho_of(p):
        lo, hi = np.zeros_like(T), np.full_like(T, rho_max)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            below = pressure(mid, T) < p
            lo, hi = np.where(below, mid, lo), np.where(below, hi, mid)
        return 0.5 * (lo + hi)

    p_lo, p_hi = 0.0, float(pressure(rho_max, T.min()))
    for _ in range(200):
        p = 0.5 * (p_lo + p_hi)
        if rho_of(p).mean() < mean_rho:
            p_lo = p
        else:
            p_hi = p
    return rho_of(0.5 * (p_lo + p_hi))
