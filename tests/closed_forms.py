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
