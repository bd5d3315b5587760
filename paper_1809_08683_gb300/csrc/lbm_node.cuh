// Per-node arithmetic of the thermal MRT lattice-Boltzmann model of
// arXiv:1809.08683, written in deviation form for the GPU kernels.
//
// Storage convention: a node holds f'_i = f_i - f^r_i and g'_i = g_i - g^r_i,
// where f^r = M^-1 m^eq(rho0, u = 0, T0) and g^r = M^-1 n^eq(rho0 E0, u = 0, T0)
// are the rest equilibria.  M f^r has only rows 0, 1, 2 nonzero, so
// m' = M f' equals m - m^r and every cancellation-prone difference
// (rho - rho0, T - T0, p - p0, eta - eta0, rho E - rho0 E0) is formed from
// small quantities.  The same code serves FP64 and FP32 storage.
//
// The collision uses the sparse forms of the modified matrices:
//  (I - S/2) d  from the block structure of S (Sec. 2.1; App. B),
//  S d = 2 (d - (I - S/2) d),
//  ((m + m_bar)/2 - m^eq)_a = G_a - C_a / 2 for a = 1, 7, 8, where
//  G = (I - S/2) d and C = R G + T grad(rho) + X grad(p),
//  L applied as diag(L) plus the two sigma_q omega_j couplings (Sec. 2.2),
//  M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define LBM_HD __host__ __device__ __forceinline__
#else
#define LBM_HD inline
#endif

namespace lbm {

// Division in the per-node arithmetic.  FP32: the fast hardware division
// (a few ulp), which the FP32 path's 1e-4 tolerance absorbs.  FP64 on the
// device: a * (1/b), with 1/b from the hardware's approximate FP64
// reciprocal (PTX rcp.approx.ftz.f64, about 20 correct bits) refined by two
// Newton-Raphson steps y <- y + y (1 - b y), each of which doubles the
// correct bits (20 -> 40 -> beyond 53): within 2 ulp of the quotient.  The
// divisors are O(1) lattice quantities (densities, temperatures, 1 + eta/rho
// terms), never subnormal.
LBM_HD double fdiv(double a, double b) {
#if defined(__CUDA_ARCH__)
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(b));
    double e = fma(-b, y, 1.0);
    y = fma(y, e, y);
    e = fma(-b, y, 1.0);
    y = fma(y, e, y);
    return a * y;
#else
    return a / b;
#endif
}
LBM_HD float fdiv(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

// Constants of one lattice, in the arithmetic type R.
template <typename R>
struct Params {
    R rho0, T0, E0, Cv, inv_Cv, Rg, eos_a, eos_b, p0, rho0E0_p0, rho0Cp0;
    R mu0, inv_T0, visc_S, lam_fac, tj_fac, e_fac;
    R alpha1, beta1, alpha2, beta2, kk, hh, bb, gamma1, gamma2;
    R cR11, cR17, cR18, cR71, cR77, cR81, cR88;
    R Fx, Fy;
    R cs_b0;  // 1 - b rho0 (cubic EOS)
    R dither; // FP32 storage: 1 rounds the stored deviations stochastically, 0 to nearest
    int eos, visc, force_mode, corrections;
};

enum { EOS_DECOUPLING = 0, EOS_IDEAL = 1, EOS_CS = 2, EOS_CUBIC = 3 };

// Model classes.  MODEL_ANY reads the EOS, the viscosity law, the force
// mode and the corrections flag from the parameters at run time.
// MODEL_CAVITY fixes the heated-cavity model at compile time (Sutherland
// viscosity, F = rho g with vertical g, corrections on) and keeps only the
// ideal-gas and cubic EOS, chosen at run time.  The arithmetic is the same;
// a fixed model drops the branches and the code of the others, and the
// terms of F_x = 0.
enum { MODEL_ANY = 0, MODEL_CAVITY = 1 };
template <int MC, typename R>
LBM_HD int visc_law(const Params<R>& P) { return MC != MODEL_ANY ? 2 : P.visc; }
template <int MC, typename R>
LBM_HD bool force_is_rho_g(const Params<R>& P) { return MC != MODEL_ANY || P.force_mode != 0; }
template <int MC, typename R>
LBM_HD bool corrections_on(const Params<R>& P) { return MC != MODEL_ANY || P.corrections != 0; }

// Macroscopic state of one node in deviation form.
template <typename R>
struct Mac {
    R rho_d, rho, ir, ux, uy, Fx, Fy, qe, rhoE_d, T_d, T, p_d, eta_d, rhoH;
};

// The part of Mac that the fused kernels keep in registers from a row's
// macro pass to its collision; expand() rebuilds the rest with the same
// operations as macros(), so an expanded state equals the original bit
// for bit.
template <typename R>
struct MacC {
    R rho_d, ir, ux, uy, rhoE_d, T_d, p_d;
};

// Carnahan-Starling deviation p - p0 with p = Z(e) rho R T, e = b rho / 4
// (Eq. EOSs.3).  The density part is differenced in FP64 to avoid
// cancellation when the arithmetic type is FP32.
LBM_HD double cs_dev1(double b, double rho0, double Rg, double rho_d, double T, double T_d) {
    double r = rho0 + rho_d;
    double e = b * r / 4.0, e0 = b * rho0 / 4.0;
    double z = (1.0 + e + e * e - e * e * e) / ((1.0 - e) * (1.0 - e) * (1.0 - e));
    double z0 = (1.0 + e0 + e0 * e0 - e0 * e0 * e0) / ((1.0 - e0) * (1.0 - e0) * (1.0 - e0));
    return Rg * ((z * r - z0 * rho0) * T + z0 * rho0 * T_d);
}
LBM_HD double cs_dev(double b, double rho0, double Rg, double rho_d, double T, double T_d) {
    return cs_dev1(b, rho0, Rg, rho_d, T, T_d);
}
LBM_HD float cs_dev(float b, float rho0, float Rg, float rho_d, float T, float T_d) {
    return (float)cs_dev1(b, rho0, Rg, rho_d, T, T_d);
}

// p_EOS(rho, T) - p0.
template <int MC = MODEL_ANY, typename R>
LBM_HD R eos_dev(const Params<R>& P, R rho_d, R rho, R T_d, R T) {
    const int kind = MC == MODEL_CAVITY ? (P.eos == EOS_CUBIC ? EOS_CUBIC : EOS_IDEAL) : P.eos;
    if (MC == MODEL_CAVITY && kind == EOS_IDEAL) return P.Rg * (rho_d * T + P.rho0 * T_d);
    switch (kind) {
    case EOS_DECOUPLING:
        return P.Rg * P.T0 * rho_d;
    case EOS_IDEAL:
        return P.Rg * (rho_d * T + P.rho0 * T_d);
    case EOS_CS:
        return cs_dev(P.eos_b, P.rho0, P.Rg, rho_d, T, T_d);
    default: {
        // rho R T / (1 - b rho) - a rho^2, differenced exactly:
        // [rho T (1 - b rho0) - rho0 T0 (1 - b rho)] = rho_d T + rho0 T_d - b rho rho0 T_d
        R om = R(1) - P.eos_b * rho;
        R num = rho_d * T + P.rho0 * T_d - P.eos_b * rho * P.rho0 * T_d;
        return fdiv(P.Rg * num, om * P.cs_b0) - P.eos_a * rho_d * (rho + P.rho0);
    }
    }
}

// Body force F = rho g (force_mode 1) or F = g, and q = u . F.
template <int MC = MODEL_ANY, typename R>
LBM_HD void mac_force(const Params<R>& P, Mac<R>& m) {
    if (MC == MODEL_CAVITY) { m.Fx = R(0); m.Fy = m.rho * P.Fy; }
    else if (force_is_rho_g<MC>(P)) { m.Fx = m.rho * P.Fx; m.Fy = m.rho * P.Fy; }
    else { m.Fx = P.Fx; m.Fy = P.Fy; }
}
template <int MC = MODEL_ANY, typename R>
LBM_HD void mac_qe(Mac<R>& m) {
    if (MC == MODEL_CAVITY) m.qe = m.uy * m.Fy;
    else m.qe = m.ux * m.Fx + m.uy * m.Fy;
}

// eta' = (3 p' - (2 + alpha1) rho') / beta1 and rho H - rho0 H0 + p0.
template <typename R>
LBM_HD void mac_tail(const Params<R>& P, Mac<R>& m) {
    m.eta_d = fdiv(R(3) * m.p_d - (R(2) + P.alpha1) * m.rho_d, P.beta1);
    m.rhoH = P.rho0E0_p0 + m.rhoE_d + m.p_d;
}

// Eq. (rho.u), Eq. (E), T = eps / Cv, p_EOS, eta = (p / c_s^2 - (2 + alpha1) rho) / beta1.
template <int MC = MODEL_ANY, typename R>
LBM_HD void macros(const Params<R>& P, R rho_d, R jx, R jy, R sg, Mac<R>& m) {
    m.rho_d = rho_d;
    m.rho = P.rho0 + rho_d;
    m.ir = fdiv(R(1), m.rho);
    mac_force<MC>(P, m);
    m.ux = MC == MODEL_CAVITY ? jx * m.ir : (jx + R(0.5) * m.Fx) * m.ir;
    m.uy = (jy + R(0.5) * m.Fy) * m.ir;
    mac_qe<MC>(m);
    m.rhoE_d = sg + R(0.5) * m.qe;
    R E_d = (m.rhoE_d - rho_d * P.E0) * m.ir;
    m.T_d = (E_d - R(0.5) * (m.ux * m.ux + m.uy * m.uy)) * P.inv_Cv;
    m.T = P.T0 + m.T_d;
    m.p_d = eos_dev<MC>(P, rho_d, m.rho, m.T_d, m.T);
    mac_tail(P, m);
}

template <typename R>
LBM_HD void compress(const Mac<R>& m, MacC<R>& c) {
    c.rho_d = m.rho_d; c.ir = m.ir; c.ux = m.ux; c.uy = m.uy;
    c.rhoE_d = m.rhoE_d; c.T_d = m.T_d; c.p_d = m.p_d;
}

template <int MC = MODEL_ANY, typename R>
LBM_HD void expand(const Params<R>& P, const MacC<R>& c, Mac<R>& m) {
    m.rho_d = c.rho_d;
    m.rho = P.rho0 + c.rho_d;
    m.ir = c.ir;
    mac_force<MC>(P, m);
    m.ux = c.ux;
    m.uy = c.uy;
    mac_qe<MC>(m);
    m.rhoE_d = c.rhoE_d;
    m.T_d = c.T_d;
    m.T = P.T0 + c.T_d;
    m.p_d = c.p_d;
    mac_tail(P, m);
}

// Macros of a wall node whose density, velocity and total energy are fixed
// by the wall data (Sec. 3.1).
template <typename R>
LBM_HD void wall_macros(const Params<R>& P, R rho_d, R ux, R uy, R rhoE_d, Mac<R>& m) {
    m.rho_d = rho_d;
    m.rho = P.rho0 + rho_d;
    m.ir = fdiv(R(1), m.rho);
    if (P.force_mode) { m.Fx = m.rho * P.Fx; m.Fy = m.rho * P.Fy; }
    else { m.Fx = P.Fx; m.Fy = P.Fy; }
    m.ux = ux;
    m.uy = uy;
    m.qe = ux * m.Fx + uy * m.Fy;
    m.rhoE_d = rhoE_d;
    R E_d = (rhoE_d - rho_d * P.E0) * m.ir;
    m.T_d = (E_d - R(0.5) * (ux * ux + uy * uy)) * P.inv_Cv;
    m.T = P.T0 + m.T_d;
    m.p_d = eos_dev(P, rho_d, m.rho, m.T_d, m.T);
    m.eta_d = fdiv(R(3) * m.p_d - (R(2) + P.alpha1) * rho_d, P.beta1);
    m.rhoH = P.rho0E0_p0 + m.rhoE_d + m.p_d;
}

// Relaxation rates of Sec. 4: s_p = 1/tau, (1/s_p - 1/2)(1/s_q - 1/2) = 1/12,
// s_eps = s_e from varsigma = varpi c_s^2 (1/s_e - 1/2) = (varsigma/nu) nu,
// lambda = Cp mu / Pr = coef rho0 Cp0 (1/sigma_j - 1/2), sigma_q = sigma_j,
// (1/sigma_j - 1/2)(1/sigma_e - 1/2) = 1/4, sigma_eps = sigma_p = sigma_e.
template <typename R>
struct Rates {
    R se, sq, sp, sj, sE;
};

template <int MC = MODEL_ANY, typename R>
LBM_HD R viscosity(const Params<R>& P, R T) {
    const int law = visc_law<MC>(P);
    if (law == 1) return P.mu0 * T * P.inv_T0;
    if (law == 2) {
        R th = T * P.inv_T0;
        return fdiv(P.mu0 * th * sqrt(th) * (R(1) + P.visc_S), th + P.visc_S);
    }
    return P.mu0;
}

template <int MC = MODEL_ANY, typename R>
LBM_HD void rates(const Params<R>& P, R rho_ir, R T, Rates<R>& r) {
    R mu = viscosity<MC>(P, T);
    R nu = mu * rho_ir;
    r.sp = fdiv(R(1), R(0.5) + R(3) * nu);
    r.sq = fdiv(R(36) * nu, R(18) * nu + R(1));
    r.se = fdiv(R(1), R(0.5) + P.e_fac * nu);
    R a = P.lam_fac * mu * P.tj_fac;  // 1/sigma_j - 1/2
    r.sj = fdiv(R(1), R(0.5) + a);
    r.sE = fdiv(R(4) * a, R(2) * a + R(1));
}

// Rows 1, 2, 4, 6, 7, 8 of m - m^eq + F_m/2 (rows 0, 3, 5 vanish identically
// by the definitions of rho and u) and the force moments used by the caller.
template <typename R>
struct Dev {
    R d1, d2, d4, d6, d7, d8;
    R me1, me2, me4, me6, me7, me8;  // deviation equilibrium rows
    R F1, F2, F4, F6, F7, F8;        // F_m rows (F_m3 = Fx, F_m5 = Fy)
};

template <int MC = MODEL_ANY, typename R>
LBM_HD void neq_density(const Params<R>& P, const Mac<R>& m, R m1, R m2, R m4, R m6, R m7, R m8,
                        Dev<R>& d) {
    R ux = m.ux, uy = m.uy, rho = m.rho;
    R ux2 = ux * ux, uy2 = uy * uy, u2 = ux2 + uy2;
    // m^eq - m^r, Sec. 2.1
    d.me1 = R(2) * P.alpha1 * m.rho_d + R(2) * P.beta1 * m.eta_d + R(3) * rho * u2;
    d.me2 = P.alpha2 * m.rho_d + P.beta2 * m.eta_d - R(3) * rho * u2 + R(9) * rho * ux2 * uy2;
    d.me4 = -rho * ux + R(3) * rho * ux * uy2;
    d.me6 = -rho * uy + R(3) * rho * uy * ux2;
    d.me7 = rho * (ux2 - uy2);
    d.me8 = rho * ux * uy;
    // F_m, Sec. 2.1, bracket by the product rule
    R Fx = m.Fx, Fy = m.Fy;
    if (MC == MODEL_CAVITY) {
        // the same terms with F_x = 0
        R Fu = Fy * uy;
        d.F1 = R(6) * Fu;
        d.F2 = -R(6) * Fu + R(18) * (Fy * uy * ux2);
        d.F4 = R(3) * (R(2) * Fy * ux * uy);
        d.F6 = -Fy + R(3) * (Fy * ux2);
        d.F7 = R(2) * (-Fy * uy);
        d.F8 = Fy * ux;
    } else {
        R Fu = Fx * ux + Fy * uy;
        d.F1 = R(6) * Fu;
        d.F2 = -R(6) * Fu + R(18) * (Fx * ux * uy2 + Fy * uy * ux2);
        d.F4 = -Fx + R(3) * (Fx * uy2 + R(2) * Fy * ux * uy);
        d.F6 = -Fy + R(3) * (Fy * ux2 + R(2) * Fx * ux * uy);
        d.F7 = R(2) * (Fx * ux - Fy * uy);
        d.F8 = Fx * uy + Fy * ux;
    }
    d.d1 = m1 - d.me1 + R(0.5) * d.F1;
    d.d2 = m2 - d.me2 + R(0.5) * d.F2;
    d.d4 = m4 - d.me4 + R(0.5) * d.F4;
    d.d6 = m6 - d.me6 + R(0.5) * d.F6;
    d.d7 = m7 - d.me7 + R(0.5) * d.F7;
    d.d8 = m8 - d.me8 + R(0.5) * d.F8;
}

// G = (I - S/2) d on rows 1, 2, 4, 6, 7, 8 (Sec. 2.1 S; App. B block structure).
template <typename R>
struct Gv {
    R G1, G2, G4, G6, G7, G8;
};

template <typename R>
LBM_HD void apply_IS2(const Params<R>& P, const Rates<R>& r, R ux, R uy, const Dev<R>& d, Gv<R>& G) {
    R he = R(1) - R(0.5) * r.se, hq = R(1) - R(0.5) * r.sq, hp = R(1) - R(0.5) * r.sp;
    G.G1 = he * (d.d1 + R(0.5) * (P.kk * r.se * d.d2 + P.hh * r.sq * (ux * d.d4 + uy * d.d6)));
    G.G2 = he * d.d2;
    G.G4 = hq * d.d4;
    G.G6 = hq * d.d6;
    G.G7 = hp * (d.d7 + P.bb * r.sq * (ux * d.d4 - uy * d.d6));
    G.G8 = hp * (d.d8 + R(0.5) * P.bb * r.sq * (uy * d.d4 + ux * d.d6));
}

// Moments m' = M f' (Eq. M).
template <typename R>
LBM_HD void moments(const R* f, R* m) {
    R a = f[1] + f[2] + f[3] + f[4];
    R b = f[5] + f[6] + f[7] + f[8];
    m[0] = f[0] + a + b;
    m[1] = -R(4) * f[0] - a + R(2) * b;
    m[2] = R(4) * f[0] - R(2) * a + b;
    R dx = f[5] - f[6] - f[7] + f[8];
    R dy = f[5] + f[6] - f[7] - f[8];
    m[3] = f[1] - f[3] + dx;
    m[4] = R(-2) * (f[1] - f[3]) + dx;
    m[5] = f[2] - f[4] + dy;
    m[6] = R(-2) * (f[2] - f[4]) + dy;
    m[7] = f[1] - f[2] + f[3] - f[4];
    m[8] = f[5] - f[6] + f[7] - f[8];
}

// f = M^-1 m with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
template <typename R>
LBM_HD void inverse_moments(const R* m, R* f) {
    R a0 = m[0] * R(1.0 / 9.0), a1 = m[1] * R(1.0 / 36.0), a2 = m[2] * R(1.0 / 36.0);
    R a3 = m[3] * R(1.0 / 6.0), a4 = m[4] * R(1.0 / 12.0), a5 = m[5] * R(1.0 / 6.0);
    R a6 = m[6] * R(1.0 / 12.0), a7 = m[7] * R(0.25), a8 = m[8] * R(0.25);
    R A = a0 - a1 - R(2) * a2;
    R B = a0 + R(2) * a1 + a2;
    R X = a3 - R(2) * a4, Y = a5 - R(2) * a6;
    R Pp = a3 + a4, Q = a5 + a6;
    f[0] = a0 - R(4) * a1 + R(4) * a2;
    f[1] = A + X + a7;
    f[3] = A - X + a7;
    f[2] = A + Y - a7;
    f[4] = A - Y - a7;
    f[5] = B + Pp + Q + a8;
    f[6] = B - Pp + Q - a8;
    f[7] = B - Pp - Q + a8;
    f[8] = B + Pp - Q - a8;
}

// Sec. 2.2: n^eq - n^r and Q_m for a node.
template <typename R>
struct EDev {
    R ne1, ne2, ne3, ne5;  // ne4 = -ne3, ne6 = -ne5, ne7 = ne8 = 0
    R Q0, Q1, Q2, Q3, Q5;  // Q4 = -Q3, Q6 = -Q5
};

template <typename R>
LBM_HD void energy_eq(const Params<R>& P, const Mac<R>& m, EDev<R>& e) {
    R ref_d = P.rho0Cp0 * m.T_d;
    e.ne1 = -R(4) * (m.rhoE_d - ref_d) + P.gamma1 * ref_d;
    e.ne2 = R(4) * (m.rhoE_d - ref_d) + P.gamma2 * ref_d;
    e.ne3 = m.rhoH * m.ux;
    e.ne5 = m.rhoH * m.uy;
    e.Q0 = m.qe;
    e.Q1 = P.gamma1 * m.qe;
    e.Q2 = P.gamma2 * m.qe;
    e.Q3 = m.qe * m.ux;
    e.Q5 = m.qe * m.uy;
}

// Plain update: new = old + delta, rounded to nearest, for the pair
// (f_i, g_i) of one link.
struct AddNearest {
    template <typename R>
    LBM_HD void operator()(R& f, R df, R& g, R dg) const {
        f = f + df;
        g = g + dg;
    }
};

// Leaves f and g as they are between the moments and the final update.
struct KeepDFs {
    template <typename R>
    LBM_HD void operator()(R*, R*) const {}
};

// Full collision of one node (Eqs. LBE.u.c, LBE.T.c) in increment form: the
// moment changes m_bar - m and n_bar - n are formed from small quantities
// only (force and source moments, non-equilibrium parts, corrections), then
// mapped back with M^-1 and added to the stored deviations through `add`,
// which may round stochastically.  f, g hold deviations on entry and the
// post-collision deviations on exit.  f and g are read twice: for the
// moments, and for the final update after `reload(f, g)`; a caller that can
// fetch them again (from shared memory) passes a reload that does so, and
// the values need not stay in registers through the collision.
template <int MC = MODEL_ANY, typename R, typename Add, typename Reload = KeepDFs>
LBM_HD void collide(const Params<R>& P, const Mac<R>& mc, R* f, R* g, R grx, R gry, R gpx, R gpy,
                    const Add& add, const Reload& reload = Reload()) {
    Rates<R> r;
    rates<MC>(P, mc.ir, mc.T, r);
    R m[9], n[9];
    moments(f, m);
    moments(g, n);
    Dev<R> d;
    neq_density<MC>(P, mc, m[1], m[2], m[4], m[6], m[7], m[8], d);
    Gv<R> G;
    const R ux = mc.ux, uy = mc.uy;
    apply_IS2(P, r, ux, uy, d, G);

    // corrections C = R G + T grad(rho) + X grad(p) on rows 1, 7, 8 (Sec. 2.1)
    R C1 = R(0), C7 = R(0), C8 = R(0);
    if (corrections_on<MC>(P)) {
        R ux2 = ux * ux, uy2 = uy * uy, sum2 = ux2 + uy2, dif2 = ux2 - uy2, xy = ux * uy;
        R tse = R(2) - r.se, tsp = R(2) - r.sp;
        R q1 = fdiv(r.sp * tse, tsp), q7 = fdiv(r.se * tsp, tse);
        R R11 = P.cR11 * r.se * sum2;
        R R17 = P.cR17 * q1 * dif2;
        R R18 = P.cR18 * q1 * xy;
        R R71 = P.cR71 * q7 * dif2;
        R R77 = P.cR77 * r.sp * sum2;
        R R81 = P.cR81 * q7 * xy;
        R R88 = P.cR88 * r.sp * sum2;
        R t1 = R(1.5) * tse, k2h = R(2) * P.kk + P.hh, omk = R(1) - P.kk;
        R T1x = t1 * (omk * ux2 * ux - k2h * ux * uy2);
        R T1y = t1 * (omk * uy2 * uy - k2h * ux2 * uy);
        R t7 = R(0.5) * tsp;
        R T7x = t7 * (ux2 * ux + R(2) * P.bb * ux * uy2);
        R T7y = -t7 * (uy2 * uy + R(2) * P.bb * ux2 * uy);
        R v8x = uy2 * uy + R(2) * ux2 * uy, v8y = ux2 * ux + R(2) * ux * uy2;
        R x1 = R(4.5) * k2h * tse;
        R x7 = -R(3) * P.bb * tsp;
        // T8 = -(b (2 - s_p)/2) v8 and X8 = (3 b (2 - s_p)/2) v8
        R b8 = R(0.5) * P.bb * tsp;
        C1 = R11 * G.G1 + R17 * G.G7 + R18 * G.G8 + T1x * grx + T1y * gry
           + x1 * (ux * uy2 * gpx + ux2 * uy * gpy);
        C7 = R71 * G.G1 + R77 * G.G7 + T7x * grx + T7y * gry + x7 * (ux * uy2 * gpx - ux2 * uy * gpy);
        C8 = R81 * G.G1 + R88 * G.G8 + b8 * (v8x * (R(3) * gpx - grx) + v8y * (R(3) * gpy - gry));
    }

    // m_bar - m = F_m - S d - C with S d = 2 (d - G); rows 0, 3, 5: 0, Fx, Fy
    R dm[9];
    dm[0] = R(0);
    dm[3] = mc.Fx;
    dm[5] = mc.Fy;
    dm[1] = d.F1 - R(2) * d.d1 + R(2) * G.G1 - C1;
    dm[2] = d.F2 - R(2) * d.d2 + R(2) * G.G2;
    dm[4] = d.F4 - R(2) * d.d4 + R(2) * G.G4;
    dm[6] = d.F6 - R(2) * d.d6 + R(2) * G.G6;
    dm[7] = d.F7 - R(2) * d.d7 + R(2) * G.G7 - C7;
    dm[8] = d.F8 - R(2) * d.d8 + R(2) * G.G8 - C8;

    // (m + m_bar)/2 - m^eq on rows 1, 7, 8
    R Gt1 = G.G1 - R(0.5) * C1, Gt7 = G.G7 - R(0.5) * C7, Gt8 = G.G8 - R(0.5) * C8;

    // total-energy DF: n_bar - n = Q - L (n - n^eq + Q/2) + Y ((m + m_bar)/2 - m^eq)
    EDev<R> e;
    energy_eq(P, mc, e);
    R dn1 = n[1] - e.ne1 + R(0.5) * e.Q1;
    R dn2 = n[2] - e.ne2 + R(0.5) * e.Q2;
    R dn3 = n[3] - e.ne3 + R(0.5) * e.Q3;
    R dn4 = n[4] + e.ne3 - R(0.5) * e.Q3;
    R dn5 = n[5] - e.ne5 + R(0.5) * e.Q5;
    R dn6 = n[6] + e.ne5 - R(0.5) * e.Q5;
    R wj = R(0.5) * r.sj - R(1);
    R Y3 = ux * (Gt1 * R(1.0 / 3.0) + Gt7) + R(2) * uy * Gt8;
    R Y5 = uy * (Gt1 * R(1.0 / 3.0) - Gt7) + R(2) * ux * Gt8;
    R nb[9];
    nb[0] = e.Q0;
    nb[1] = e.Q1 - r.sE * dn1;
    nb[2] = e.Q2 - r.sE * dn2;
    nb[3] = e.Q3 - (r.sj * dn3 + r.sj * wj * dn4) + Y3;
    nb[4] = -e.Q3 - r.sj * dn4 - Y3;
    nb[5] = e.Q5 - (r.sj * dn5 + r.sj * wj * dn6) + Y5;
    nb[6] = -e.Q5 - r.sj * dn6 - Y5;
    nb[7] = -r.sE * n[7];
    nb[8] = -r.sE * n[8];

    R df[9], dg[9];
    inverse_moments(dm, df);
    inverse_moments(nb, dg);
    reload(f, g);
#pragma unroll
    for (int i = 0; i < 9; ++i) add(f[i], df[i], g[i], dg[i]);
}

template <typename R>
LBM_HD void collide(const Params<R>& P, const Mac<R>& mc, R* f, R* g, R grx, R gry, R gpx, R gpy) {
    collide(P, mc, f, g, grx, gry, gpx, gpy, AddNearest());
}

// Redefined non-equilibrium moments of Eq. (neq.redefinition) at a fluid
// node: mt = (I - S/2) m^neq, nt = (I - L/2) n^neq + (Y/2) mt, with
// m^neq = m - m^eq + F_m/2 and n^neq = n - n^eq + Q_m/2 (Eq. decompose).
// Rows 0, 3, 5 of mt and row 0 of nt vanish identically.
template <typename R>
LBM_HD void tilde_neq(const Params<R>& P, const Mac<R>& mc, const R* f, const R* g, R* mt, R* nt) {
    Rates<R> r;
    rates(P, mc.ir, mc.T, r);
    R m[9];
    moments(f, m);
    Dev<R> d;
    neq_density(P, mc, m[1], m[2], m[4], m[6], m[7], m[8], d);
    Gv<R> G;
    apply_IS2(P, r, mc.ux, mc.uy, d, G);
    mt[0] = R(0); mt[3] = R(0); mt[5] = R(0);
    mt[1] = G.G1; mt[2] = G.G2; mt[4] = G.G4; mt[6] = G.G6; mt[7] = G.G7; mt[8] = G.G8;
    R n[9];
    moments(g, n);
    EDev<R> e;
    energy_eq(P, mc, e);
    R dn1 = n[1] - e.ne1 + R(0.5) * e.Q1;
    R dn2 = n[2] - e.ne2 + R(0.5) * e.Q2;
    R dn3 = n[3] - e.ne3 + R(0.5) * e.Q3;
    R dn4 = n[4] + e.ne3 - R(0.5) * e.Q3;
    R dn5 = n[5] - e.ne5 + R(0.5) * e.Q5;
    R dn6 = n[6] + e.ne5 - R(0.5) * e.Q5;
    R hE = R(1) - R(0.5) * r.sE, hj = R(1) - R(0.5) * r.sj;
    R wj = R(0.5) * r.sj - R(1);
    R ux = mc.ux, uy = mc.uy;
    R Y3 = ux * (mt[1] * R(1.0 / 3.0) + mt[7]) + R(2) * uy * mt[8];
    R Y5 = uy * (mt[1] * R(1.0 / 3.0) - mt[7]) + R(2) * ux * mt[8];
    nt[0] = R(0);
    nt[1] = hE * dn1;
    nt[2] = hE * dn2;
    nt[3] = hj * dn3 - R(0.5) * r.sj * wj * dn4 + R(0.5) * Y3;
    nt[4] = hj * dn4 - R(0.5) * Y3;
    nt[5] = hj * dn5 - R(0.5) * r.sj * wj * dn6 + R(0.5) * Y5;
    nt[6] = hj * dn6 - R(0.5) * Y5;
    nt[7] = hE * n[7];
    nt[8] = hE * n[8];
}

// Rebuild all 18 DFs of a wall node from its macroscopic state mb and the
// extrapolated redefined non-equilibrium moments mt, nt (Sec. 3.2):
// m^neq = (I - S/2)^-1 mt, n^neq = (I - L/2)^-1 (nt - (Y/2) mt) with the
// closed forms of App. B, then m = m^eq - F_m/2 + m^neq, n = n^eq - Q_m/2 + n^neq.
template <typename R>
LBM_HD void rebuild(const Params<R>& P, const Mac<R>& mb, const R* mt, const R* nt, R* f, R* g) {
    Rates<R> r;
    rates(P, mb.ir, mb.T, r);
    const R ux = mb.ux, uy = mb.uy;
    R he = R(1) - R(0.5) * r.se, hq = R(1) - R(0.5) * r.sq, hp = R(1) - R(0.5) * r.sp;
    const R ihe = fdiv(R(1), he), ihq = fdiv(R(1), hq), ihp = fdiv(R(1), hp);
    R v1 = mt[1] * ihe, v2 = mt[2] * ihe, v4 = mt[4] * ihq, v6 = mt[6] * ihq;
    R v7 = mt[7] * ihp, v8 = mt[8] * ihp;
    R mn1 = v1 - R(0.5) * P.kk * r.se * v2 - R(0.5) * P.hh * r.sq * (ux * v4 + uy * v6);
    R mn7 = v7 - P.bb * r.sq * (ux * v4 - uy * v6);
    R mn8 = v8 - R(0.5) * P.bb * r.sq * (uy * v4 + ux * v6);

    Dev<R> d;
    neq_density(P, mb, R(0), R(0), R(0), R(0), R(0), R(0), d);
    R m[9];
    m[0] = mb.rho_d;
    m[1] = d.me1 - R(0.5) * d.F1 + mn1;
    m[2] = d.me2 - R(0.5) * d.F2 + v2;
    m[3] = mb.rho * ux - R(0.5) * mb.Fx;
    m[4] = d.me4 - R(0.5) * d.F4 + v4;
    m[5] = mb.rho * uy - R(0.5) * mb.Fy;
    m[6] = d.me6 - R(0.5) * d.F6 + v6;
    m[7] = d.me7 - R(0.5) * d.F7 + mn7;
    m[8] = d.me8 - R(0.5) * d.F8 + mn8;

    R Y3 = ux * (mt[1] * R(1.0 / 3.0) + mt[7]) + R(2) * uy * mt[8];
    R Y5 = uy * (mt[1] * R(1.0 / 3.0) - mt[7]) + R(2) * ux * mt[8];
    R hE = R(1) - R(0.5) * r.sE, hj = R(1) - R(0.5) * r.sj;
    const R ihE = fdiv(R(1), hE), ihj = fdiv(R(1), hj);
    R w1 = nt[1] * ihE, w2 = nt[2] * ihE, w7 = nt[7] * ihE, w8 = nt[8] * ihE;
    R w3 = (nt[3] - R(0.5) * Y3) * ihj, w4 = (nt[4] + R(0.5) * Y3) * ihj;
    R w5 = (nt[5] - R(0.5) * Y5) * ihj, w6 = (nt[6] + R(0.5) * Y5) * ihj;
    R nn3 = w3 - R(0.5) * r.sj * w4;
    R nn5 = w5 - R(0.5) * r.sj * w6;
    EDev<R> e;
    energy_eq(P, mb, e);
    R n[9];
    n[0] = mb.rhoE_d - R(0.5) * e.Q0;
    n[1] = e.ne1 - R(0.5) * e.Q1 + w1;
    n[2] = e.ne2 - R(0.5) * e.Q2 + w2;
    n[3] = e.ne3 - R(0.5) * e.Q3 + nn3;
    n[4] = -e.ne3 + R(0.5) * e.Q3 + w4;
    n[5] = e.ne5 - R(0.5) * e.Q5 + nn5;
    n[6] = -e.ne5 + R(0.5) * e.Q5 + w6;
    n[7] = w7;
    n[8] = w8;
    inverse_moments(m, f);
    inverse_moments(n, g);
}

// Equilibrium deviations with zero non-equilibrium part (Eq. decompose):
// f' = M^-1 (m^eq - m^r - F_m/2), g' = M^-1 (n^eq - n^r - Q_m/2).
template <typename R>
LBM_HD void equilibrium(const Params<R>& P, const Mac<R>& mb, R* f, R* g) {
    Dev<R> d;
    neq_density(P, mb, R(0), R(0), R(0), R(0), R(0), R(0), d);
    R m[9];
    m[0] = mb.rho_d;
    m[1] = d.me1 - R(0.5) * d.F1;
    m[2] = d.me2 - R(0.5) * d.F2;
    m[3] = mb.rho * mb.ux - R(0.5) * mb.Fx;
    m[4] = d.me4 - R(0.5) * d.F4;
    m[5] = mb.rho * mb.uy - R(0.5) * mb.Fy;
    m[6] = d.me6 - R(0.5) * d.F6;
    m[7] = d.me7 - R(0.5) * d.F7;
    m[8] = d.me8 - R(0.5) * d.F8;
    EDev<R> e;
    energy_eq(P, mb, e);
    R n[9];
    n[0] = mb.rhoE_d - R(0.5) * e.Q0;
    n[1] = e.ne1 - R(0.5) * e.Q1;
    n[2] = e.ne2 - R(0.5) * e.Q2;
    n[3] = e.ne3 - R(0.5) * e.Q3;
    n[4] = -e.ne3 + R(0.5) * e.Q3;
    n[5] = e.ne5 - R(0.5) * e.Q5;
    n[6] = -e.ne5 + R(0.5) * e.Q5;
    n[7] = R(0);
    n[8] = R(0);
    inverse_moments(m, f);
    inverse_moments(n, g);
}

// Sums over the 9 populations of a node: rho', j, sum g'.
template <typename R>
LBM_HD void node_sums(const R* f, const R* g, R& rd, R& jx, R& jy, R& sg) {
    rd = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    sg = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
}

}  // namespace lbm
