"""Algebraic pins of the FP64 oracle: each check compares the oracle with a
fact the paper or the mathematics fixes independently of the oracle's own
formulas (orthogonality of M, moments of the equilibria, the product rule
behind F_m, the closed-form inverses of App. B, the step sequence of App. C,
the collision invariants)."""
import numpy as np
import pytest

from paper_1809_08683_gb300 import workloads as W

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)


def _oracle(orc, **kw):
    return orc.Oracle(W.periodic_box(4, 4, **kw))


def test_M_orthogonal_rows(orc):
    # Eq. (M): rows are mutually orthogonal with norms 9, 36, 36, 6, 12, 6, 12, 4, 4
    M = orc.matrix_M()
    G = M @ M.T
    assert np.array_equal(G, np.diag([9.0, 36, 36, 6, 12, 6, 12, 4, 4]))
    # rows 3 and 5 are the momentum moments e_x, e_y (Eq. 1)
    assert np.array_equal(M[3], EX) and np.array_equal(M[5], EY)
    Minv = orc.matrix_Minv()
    assert np.abs(Minv @ M - np.eye(9)).max() < 1e-15


@pytest.mark.parametrize("eos", [(W.EOS_IDEAL, ()), (W.EOS_CUBIC, (0.05, 0.2)),
                                 (W.EOS_CS, ()), (W.EOS_DECOUPLING, ())])
def test_density_equilibrium_moments(orc, eos):
    # Sec. 2.1: the equilibrium must carry rho, rho u and the momentum flux
    # p_EOS I + rho u u (the self-tuning EOS, p_LBE = p_EOS), and the D2Q9
    # third moments rho u_b / 3 + rho u_a^2 u_b.
    o = _oracle(orc, eos=eos)
    Minv = orc.matrix_Minv()
    rng = np.random.default_rng(5)
    for _ in range(20):
        rho = rng.uniform(0.6, 1.4)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        T = rng.uniform(0.5, 1.5)
        q = o.eq_moments(rho, ux, uy, T)
        feq = Minv @ q["meq"]
        # p from an independent evaluation of the same EOS through the node hook
        node = o.node(feq, Minv @ q["neq"])
        p = node["p"]
        assert abs(feq.sum() - rho) < 1e-14
        assert abs((EX * feq).sum() - rho * ux) < 1e-14
        assert abs((EY * feq).sum() - rho * uy) < 1e-14
        assert abs((EX * EX * feq).sum() - (p + rho * ux * ux)) < 1e-13
        assert abs((EY * EY * feq).sum() - (p + rho * uy * uy)) < 1e-13
        assert abs((EX * EY * feq).sum() - rho * ux * uy) < 1e-14
        assert abs((EX * EX * EY * feq).sum() - (rho * uy / 3 + rho * ux * ux * uy)) < 1e-14
        assert abs((EX * EY * EY * feq).sum() - (rho * ux / 3 + rho * ux * uy * uy)) < 1e-14


def _eos_value(kind, params, rho, T, R, T0=1.0):
    if kind == W.EOS_DECOUPLING:
        return rho * R * T0
    if kind == W.EOS_IDEAL:
        return rho * R * T
    if kind == W.EOS_CS:
        b = params[0] if params else np.sqrt(2) * np.pi / 3
        e = b * rho / 4
        return (1 + e + e * e - e ** 3) / (1 - e) ** 3 * rho * R * T
    a, b = params
    return rho * R * T / (1 - b * rho) - a * rho * rho


@pytest.mark.parametrize("eos", [(W.EOS_IDEAL, ()), (W.EOS_CUBIC, (0.05, 0.2)),
                                 (W.EOS_CS, ()), (W.EOS_DECOUPLING, ())])
def test_eos_sound_speed_and_heat_capacities(orc, eos):
    # Eq. (cs): d p_EOS / d rho at (rho0, T0) equals c_s^2 = 1/3 (checked by a
    # central finite difference of the EOS evaluated through the node hook);
    # Cp - Cv = p0 / (rho0 T0) and Cp / Cv = gamma.
    o = _oracle(orc, eos=eos, gamma=1.3)
    d = o.derived()
    Minv = orc.matrix_Minv()

    def p_of(rho, T):
        q = o.eq_moments(rho, 0.0, 0.0, T)
        return o.node(Minv @ q["meq"], Minv @ q["neq"])["p"]

    h = 1e-5
    dp = (p_of(1 + h, 1.0) - p_of(1 - h, 1.0)) / (2 * h)
    assert abs(dp - 1.0 / 3.0) < 1e-8
    assert abs(p_of(1.0, 1.0) - d["p0"]) < 1e-14
    # the EOS itself, retyped from Eqs. (EOSs.1-3) and the cubic form
    for rho, T in ((0.8, 1.2), (1.1, 0.7)):
        assert abs(p_of(rho, T) - _eos_value(eos[0], eos[1], rho, T, d["R"])) < 1e-13
    assert abs(d["Cp"] - d["Cv"] - d["p0"]) < 1e-14
    assert abs(d["Cp"] / d["Cv"] - 1.3) < 1e-14


def test_energy_equilibrium_moments(orc):
    # Sec. 2.2: sum g^eq = rho E, sum e g^eq = rho H u, and with gamma1 = -2
    # the second moment is isotropic rho0 Cp0 T / 3.
    o = _oracle(orc, eos=(W.EOS_CUBIC, (0.05, 0.2)), gamma=1.3)
    d = o.derived()
    Minv = orc.matrix_Minv()
    rng = np.random.default_rng(7)
    for _ in range(20):
        rho = rng.uniform(0.7, 1.3)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        T = rng.uniform(0.6, 1.4)
        q = o.eq_moments(rho, ux, uy, T)
        geq = Minv @ q["neq"]
        E = d["Cv"] * T + 0.5 * (ux * ux + uy * uy)
        p = _eos_value(W.EOS_CUBIC, (0.05, 0.2), rho, T, d["R"])
        H = E + p / rho
        assert abs(geq.sum() - rho * E) < 1e-14
        assert abs((EX * geq).sum() - rho * H * ux) < 1e-14
        assert abs((EY * geq).sum() - rho * H * uy) < 1e-14
        assert abs((EX * EX * geq).sum() - d["Cp"] * T / 3) < 1e-14
        assert abs((EY * EY * geq).sum() - d["Cp"] * T / 3) < 1e-14
        assert abs((EX * EY * geq).sum()) < 1e-14


def test_force_moments_product_rule(orc):
    # F_m of Sec. 2.1 with the bracket read by the product rule (the printed
    # example of [F u u u]_xxyy): each velocity-dependent entry of m^eq is
    # rho phi_k(u) and F_m,k = sum_a F_a d phi_k / d u_a.  Checked against a
    # central finite difference of m^eq in u, for arbitrary force directions.
    o = _oracle(orc)
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(10):
        rho = rng.uniform(0.7, 1.3)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        T = rng.uniform(0.8, 1.2)
        Fx, Fy = rng.uniform(-1, 1, 2)
        Fm = o.eq_moments(rho, ux, uy, T, Fx, Fy)["Fm"]
        # eta (from p) depends on T only, not on u: finite difference in u at fixed rho, T
        def meq(a, b):
            return o.eq_moments(rho, a, b, T)["meq"] / rho
        dphi_dx = (meq(ux + h, uy) - meq(ux - h, uy)) / (2 * h)
        dphi_dy = (meq(ux, uy + h) - meq(ux, uy - h)) / (2 * h)
        fd = Fx * dphi_dx + Fy * dphi_dy
        fd[0] = 0.0
        # the internal energy is held fixed, so m^eq_1,2 change only through rho|u|^2 terms
        assert np.abs(Fm - fd).max() < 1e-8, (Fm, fd)
        # discrete force: zero mass source, momentum source F
        Minv = orc.matrix_Minv()
        fF = Minv @ Fm
        assert abs(fF.sum()) < 1e-15
        assert abs((EX * fF).sum() - Fx) < 1e-14 and abs((EY * fF).sum() - Fy) < 1e-14


def test_source_moments(orc):
    # Q_m of Sec. 2.2: its zeroth moment is q_e and its first moment q_e u
    o = _oracle(orc)
    Minv = orc.matrix_Minv()
    q = o.eq_moments(1.1, 0.05, -0.03, 1.0, 0.2, -0.1)
    qe = 0.05 * 0.2 + (-0.03) * (-0.1)
    gQ = Minv @ q["Qm"]
    assert abs(gQ.sum() - qe) < 1e-16
    assert abs((EX * gQ).sum() - qe * 0.05) < 1e-16
    assert abs((EY * gQ).sum() - qe * (-0.03)) < 1e-16


def _random_node(orc, o, seed):
    rng = np.random.default_rng(seed)
    Minv = orc.matrix_Minv()
    q = o.eq_moments(rng.uniform(0.8, 1.2), *rng.uniform(-0.1, 0.1, 2), rng.uniform(0.8, 1.2))
    f = Minv @ q["meq"] + 1e-2 * rng.standard_normal(9)
    g = Minv @ q["neq"] + 1e-2 * rng.standard_normal(9)
    return f, g, rng.uniform(-0.05, 0.05, 2), rng.uniform(-0.05, 0.05, 2)


@pytest.mark.parametrize("visc_law", [0, 1, 2])
def test_appendix_B_inverses(orc, visc_law):
    # App. B gives (I - S/2)^-1 and (I - L/2)^-1 in closed form; the oracle
    # inverts the dense matrices of Sec. 2.1/2.2 numerically.
    o = orc.Oracle(W.periodic_box(4, 4, visc_law=visc_law, force=(1e-3, -2e-3)))
    c = o.cfg
    k = 1 - c["varpi"]
    h = 6 * c["varpi"] * (1 - c["varpi"]) / (1 - 3 * c["varpi"])
    b = (1 - c["varpi"]) / (1 - 3 * c["varpi"])
    for seed in range(6):
        f, g, gr, gp = _random_node(orc, o, seed)
        nd = o.node(f, g, gr, gp)
        s, sig, ux, uy = nd["s"], nd["sig"], nd["ux"], nd["uy"]
        P = np.eye(9)
        P[1, 2] = -k * s[2] / 2
        P[1, 4] = -h * ux * s[4] / 2
        P[1, 6] = -h * uy * s[4] / 2
        P[7, 4] = -b * ux * s[4]
        P[7, 6] = b * uy * s[4]
        P[8, 4] = -b * uy * s[4] / 2
        P[8, 6] = -b * ux * s[4] / 2
        closed = P @ np.diag(1.0 / (1.0 - s / 2))
        assert np.abs(closed - nd["IS2inv"]).max() < 1e-14
        Q = np.eye(9)
        Q[3, 4] = -sig[4] / 2
        Q[5, 6] = -sig[6] / 2
        closedL = Q @ np.diag(1.0 / (1.0 - sig / 2))
        assert np.abs(closedL - nd["IL2inv"]).max() < 1e-14


@pytest.mark.parametrize("visc_law", [0, 2])
def test_appendix_C_sequence(orc, visc_law):
    # App. C: the four assignment steps reproduce the dense collision of
    # Eq. (LBE.T.c) computed by the oracle.
    o = orc.Oracle(W.periodic_box(4, 4, visc_law=visc_law, force=(1e-3, 5e-4)))
    for seed in range(8):
        f, g, gr, gp = _random_node(orc, o, 100 + seed)
        nd = o.node(f, g, gr, gp)
        sig, ux, uy = nd["sig"], nd["ux"], nd["uy"]
        n = nd["n"].copy()
        nb = n.copy()
        n = n - nd["neq"]
        nb = nb - 2 * n
        n = n + nd["Qm"] / 2
        n[3] += sig[4] * n[4] / 2
        n[5] += sig[6] * n[6] / 2
        n = (1 - sig / 2) * n
        nb = nb + 2 * n
        G = (nd["m"] + nd["mbar"]) / 2 - nd["meq"]
        Y3 = ux / 3 * G[1] + ux * G[7] + 2 * uy * G[8]
        Y5 = uy / 3 * G[1] - uy * G[7] + 2 * ux * G[8]
        nb[3] += Y3
        nb[4] -= Y3
        nb[5] += Y5
        nb[6] -= Y5
        assert np.abs(nb - nd["nbar"]).max() < 1e-14


def test_collision_invariants(orc):
    # Eq. (LBE.u.c) keeps mass and adds the force impulse to momentum;
    # Eq. (LBE.T.c) adds the source q_e to the total energy.
    o = orc.Oracle(W.periodic_box(4, 4, force=(2e-3, -1e-3), visc_law=2))
    for seed in range(10):
        f, g, gr, gp = _random_node(orc, o, 200 + seed)
        nd = o.node(f, g, gr, gp)
        assert abs(nd["mbar"][0] - nd["m"][0]) < 1e-15
        assert abs(nd["mbar"][3] - (nd["m"][3] + nd["Fx"])) < 1e-15
        assert abs(nd["mbar"][5] - (nd["m"][5] + nd["Fy"])) < 1e-15
        assert abs(nd["nbar"][0] - (nd["n"][0] + nd["qe"])) < 1e-15


def test_relaxation_rate_rules(orc):
    # Sec. 4 parameter rules: s0 = sj = 1, (1/sp - 1/2)(1/sq - 1/2) = 1/12,
    # s_eps = s_e with varsigma = varpi c_s^2 (1/s_e - 1/2) = (varsigma/nu) nu,
    # sigma_0 = 1, (1/sj - 1/2)(1/se - 1/2) = 1/4, sigma_eps = sigma_p = sigma_e,
    # sigma_q = sigma_j, lambda = Cp mu / Pr = rho0 Cp0 c_s^2 (1/sigma_j - 1/2).
    cfg = W.periodic_box(4, 4, tau0=0.7, Pr=0.9, visc_law=2)
    cfg["bulk_ratio"] = 2.0
    o = orc.Oracle(cfg)
    d = o.derived()
    f, g, gr, gp = _random_node(orc, o, 300)
    nd = o.node(f, g, gr, gp)
    s, sig = nd["s"], nd["sig"]
    T = nd["T"]
    S_ = 110.5 / 600
    mu = d["mu0"] * T ** 1.5 * (1 + S_) / (T + S_)
    nu = mu / nd["rho"]
    assert abs((1 / s[7] - 0.5) / 3 - nu) < 1e-15
    assert s[0] == 1 and s[3] == 1 and s[5] == 1 and s[1] == s[2] and s[4] == s[6] and s[7] == s[8]
    assert abs((1 / s[7] - 0.5) * (1 / s[4] - 0.5) - 1 / 12) < 1e-15
    assert abs(cfg["varpi"] / 3 * (1 / s[1] - 0.5) - 2.0 * nu) < 1e-15
    lam = d["Cp"] * mu / 0.9
    assert abs(d["Cp"] / 3 * (1 / sig[3] - 0.5) - lam) < 1e-15
    assert abs((1 / sig[3] - 0.5) * (1 / sig[1] - 0.5) - 0.25) < 1e-14
    assert sig[0] == 1 and sig[1] == sig[2] == sig[7] == sig[8] and sig[3] == sig[4] == sig[5] == sig[6]


def _quadratic(nx, ny, c):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    a, b, cy, d, e, f = c
    phi = a + b * x + cy * y + d * x * x + e * x * y + f * y * y
    return phi, b + 2 * d * x + e * y, cy + e * x + 2 * f * y


@pytest.mark.parametrize("nx,ny", [(9, 7), (5, 5), (13, 4)])
def test_gradient_stencil_exact_on_quadratics(orc, nx, ny):
    # Step 2 of the oracle (the stencil the paper leaves to cited work,
    # reading R3): the isotropic interior stencil 3 sum_i w_i e_i phi(x + e_i),
    # the one-sided second-order difference along a wall normal and the
    # central one along the wall are all exact for a quadratic field, at
    # interior nodes, on every wall and in the corners.  The x and y
    # coefficients differ, so a swapped axis, a wrong sign of the inward
    # normal, a dropped diagonal weight or a first-order wall formula fails.
    o = orc.Oracle(W.cavity(N=8, Ra=1e3, eps=0.5) | {"nx": nx, "ny": ny})
    rng = np.random.default_rng(nx * 31 + ny)
    for _ in range(3):
        c = rng.uniform(-1, 1, 6)
        phi, gx_ref, gy_ref = _quadratic(nx, ny, c)
        gx, gy = o.grad_field(phi)
        assert np.abs(gx - gx_ref).max() < 1e-12
        assert np.abs(gy - gy_ref).max() < 1e-12
    # a cubic term along x is not differentiated exactly by a second-order
    # formula: the check above is not vacuous
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    gx, _ = o.grad_field(x ** 3)
    assert np.abs(gx - 3 * x ** 2).max() > 0.5
    o.close()


def test_gradient_stencil_periodic_fourier_mode(orc):
    # On a periodic lattice the stencil applied to sin(k x) (or sin(k y))
    # gives exactly sin(k) cos(k x): the weights 1/9 (axis) and 1/36
    # (diagonal) sum to 1/6 per side, 3 * 2 * (1/6) = 1, times the central
    # difference (phi(x+1) - phi(x-1)) / 2 = sin(k) cos(k x).  The wrap
    # across the periodic edge takes part at both ends.
    nx, ny = 12, 10
    o = orc.Oracle(W.periodic_box(nx, ny))
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    kx, ky = 2 * np.pi * 2 / nx, 2 * np.pi / ny
    gx, gy = o.grad_field(np.sin(kx * x) + 0.5 * np.sin(ky * y))
    assert np.abs(gx - np.sin(kx) * np.cos(kx * x)).max() < 1e-13
    assert np.abs(gy - 0.5 * np.sin(ky) * np.cos(ky * y)).max() < 1e-13
    o.close()
