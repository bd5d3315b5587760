/*
 * Plain FP64 CPU oracle of arXiv:1809.08683 (thermal MRT LB, D2Q9, f + g).
 *
 * TEST INFRASTRUCTURE ONLY: see lbm_oracle.h.  Built with -ffp-contract=off.
 *
 * Per time step (phase order: collide all nodes -> stream -> wall pass):
 *   1. macros of every node from its post-boundary DFs (Eqs. rho.u, E);
 *   2. grad(rho) and grad(p) of every node (9-point isotropic stencil in the
 *      interior, one-sided second order along a wall normal);
 *   3. dense MRT collision of f (Eq. LBE.u.c) and g (Eq. LBE.T.c), with the
 *      9x9 matrices S, R, L, Y and the 9x2 matrices T, X written out from
 *      Sec. 2.1/2.2 entry by entry;  f_bar = M^-1 m_bar with M^-1 from a
 *      numeric inversion of M (Eq. M);
 *   4. push streaming into a second lattice (Eqs. LBE.u.s, LBE.T.s); a
 *      population whose target lies outside the domain is bounced back
 *      into the node's own opposite slot (Eqs. BB.f, BB.g);
 *   5. wall pass at every wall node (Sec. 3): density from the bounced
 *      sums, u and (Dirichlet) T from the wall data or (Neumann) total
 *      energy from the bounced g sums, non-equilibrium parts redefined by
 *      Eq. (neq.redefinition) at x_f (and x_ff), extrapolated by
 *      Eq. (neq.extrapolation), converted back with numerically inverted
 *      (I-S/2) and (I-L/2), recombined by Eq. (decompose).
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 velocities, Eq. (1): rest, 4 axis links, 4 diagonals (counter-clockwise). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* Transformation matrix of Eq. (M), row by row as printed. */
static const double MROWS[81] = {
     1,  1,  1,  1,  1,  1,  1,  1,  1,
    -4, -1, -1, -1, -1,  2,  2,  2,  2,
     4, -2, -2, -2, -2,  1,  1,  1,  1,
     0,  1,  0, -1,  0,  1, -1, -1,  1,
     0, -2,  0,  2,  0,  1, -1, -1,  1,
     0,  0,  1,  0, -1,  1,  1, -1, -1,
     0,  0, -2,  0,  2,  1,  1, -1, -1,
     0,  1, -1,  1, -1,  0,  0,  0,  0,
     0,  0,  0,  0,  0,  1, -1,  1, -1,
};

static const double CS2 = 1.0 / 3.0;

/* index of the link with e_j = -e_i */
static int opposite(int i) {
    for (int j = 0; j < 9; ++j)
        if (EX[j] == -EX[i] && EY[j] == -EY[i]) return j;
    return -1;
}

struct orc_ctx {
    orc_config cfg;
    int px, py;
    int eos_kind, eos_set;
    double eos_a, eos_b;
    double R, Cv, Cp, Cp0, mu0, p0, eta0, lambda0;
    double alpha1, beta1, alpha2, beta2, kk, hh, bb;
    double Minv[81];
    double *f, *g, *f2, *g2;   /* [y][x][9] */
    double *rho_f, *p_f;       /* per-node macro scratch for the gradients */
    long step;
    int unstable;
};

/* ------------------------------------------------------------------ */
/* small dense linear algebra                                         */
/* ------------------------------------------------------------------ */

static void matvec9(const double* A, const double* x, double* y) {
    for (int r = 0; r < 9; ++r) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += A[r * 9 + k] * x[k];
        y[r] = s;
    }
}

/* Gauss-Jordan inversion with partial pivoting; returns 0 on success. */
static int invert9(const double* A, double* Ainv) {
    double a[9][18];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 18; ++c)
            a[r][c] = c < 9 ? A[r * 9 + c] : (c - 9 == r ? 1.0 : 0.0);
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 18; ++c) {
                double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t;
            }
        double d = a[col][col];
        for (int c = 0; c < 18; ++c) a[col][c] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == col) continue;
            double fct = a[r][col];
            if (fct == 0.0) continue;
            for (int c = 0; c < 18; ++c) a[r][c] -= fct * a[col][c];
        }
    }
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) Ainv[r * 9 + c] = a[r][c + 9];
    return 0;
}

void orc_matrix_M(double* out81) { memcpy(out81, MROWS, sizeof(MROWS)); }

void orc_matrix_Minv(double* out81) { invert9(MROWS, out81); }

/* ------------------------------------------------------------------ */
/* thermodynamic closures (Sec. 2.2, Eqs. EOSs, cs, Cp; Sutherland)    */
/* ------------------------------------------------------------------ */

/* p_EOS(rho, T).  kind: 0 decoupling (EOSs.1), 1 ideal gas (EOSs.2),
 * 2 Carnahan-Starling (EOSs.3), 3 cubic rho R T/(1 - b rho) - a rho^2. */
static double eos_p(const orc_ctx* c, double rho, double T) {
    switch (c->eos_kind) {
    case 0: return rho * c->R * c->cfg.T0;
    case 1: return rho * c->R * T;
    case 2: {
        double e = c->eos_b * rho / 4.0;
        double om = 1.0 - e;
        double Z = (1.0 + e + e * e - e * e * e) / (om * om * om);
        return Z * rho * c->R * T;
    }
    default:
        return rho * c->R * T / (1.0 - c->eos_b * rho) - c->eos_a * rho * rho;
    }
}

/* d p_EOS / d rho at fixed T, per unit R for the R-proportional part.
 * Returns A, B with dp/drho = R * A + B. */
static void eos_dpdrho_parts(const orc_ctx* c, double rho, double T, double* A, double* B) {
    switch (c->eos_kind) {
    case 0: *A = c->cfg.T0; *B = 0.0; break;
    case 1: *A = T; *B = 0.0; break;
    case 2: {
        /* d(rho Z)/d rho with e = b rho / 4:  Z + e dZ/de */
        double e = c->eos_b * rho / 4.0;
        double om = 1.0 - e;
        double N = 1.0 + e + e * e - e * e * e;
        double Z = N / (om * om * om);
        double dZ = (1.0 + 2.0 * e - 3.0 * e * e) / (om * om * om) + 3.0 * N / (om * om * om * om);
        *A = (Z + e * dZ) * T;
        *B = 0.0;
        break;
    }
    default: {
        double om = 1.0 - c->eos_b * rho;
        *A = T / (om * om);
        *B = -2.0 * c->eos_a * rho;
        break;
    }
    }
}

static double viscosity(const orc_ctx* c, double T) {
    double th = T / c->cfg.T0;
    switch (c->cfg.visc_law) {
    case 1: return c->mu0 * th;
    case 2: {
        double S = c->cfg.visc_p[0];
        return c->mu0 * th * sqrt(th) * (1.0 + S) / (th + S);
    }
    default: return c->mu0;
    }
}

/* ------------------------------------------------------------------ */
/* per-node quantities                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    double rho, ux, uy, Fx, Fy, qe, E, T, p, eta, H;
} macro_t;

static void force_at(const orc_ctx* c, double rho, double* Fx, double* Fy) {
    if (c->cfg.force_mode == 1) { *Fx = rho * c->cfg.force[0]; *Fy = rho * c->cfg.force[1]; }
    else { *Fx = c->cfg.force[0]; *Fy = c->cfg.force[1]; }
}

/* Eq. (rho.u), Eq. (E), T = eps / Cv, H = E + p / rho, eta from Sec. 2.2 end. */
static void node_macros(const orc_ctx* c, const double* f, const double* g, macro_t* o) {
    double rho = 0, jx = 0, jy = 0, sg = 0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += EX[i] * f[i];
        jy += EY[i] * f[i];
        sg += g[i];
    }
    double Fx, Fy;
    force_at(c, rho, &Fx, &Fy);
    o->rho = rho;
    o->Fx = Fx; o->Fy = Fy;
    o->ux = (jx + 0.5 * Fx) / rho;
    o->uy = (jy + 0.5 * Fy) / rho;
    o->qe = o->ux * Fx + o->uy * Fy;
    o->E = (sg + 0.5 * o->qe) / rho;
    o->T = (o->E - 0.5 * (o->ux * o->ux + o->uy * o->uy)) / c->Cv;
    o->p = eos_p(c, rho, o->T);
    o->eta = (o->p / CS2 - (2.0 + c->alpha1) * rho) / c->beta1;
    o->H = o->E + o->p / rho;
}

/* Macros of a wall node given its density, velocity and total energy. */
static void wall_macros(const orc_ctx* c, double rho, double ux, double uy, double E, macro_t* o) {
    double Fx, Fy;
    force_at(c, rho, &Fx, &Fy);
    o->rho = rho; o->ux = ux; o->uy = uy; o->Fx = Fx; o->Fy = Fy;
    o->qe = ux * Fx + uy * Fy;
    o->E = E;
    o->T = (E - 0.5 * (ux * ux + uy * uy)) / c->Cv;
    o->p = eos_p(c, rho, o->T);
    o->eta = (o->p / CS2 - (2.0 + c->alpha1) * rho) / c->beta1;
    o->H = E + o->p / rho;
}

/* Relaxation rates (Sec. 4 parameter rules; nu = c_s^2 (1/s_p - 1/2),
 * varsigma = varpi c_s^2 (1/s_e - 1/2), lambda = (2/3 + g1/2 + g2/3) rho0 Cp0 (1/sigma_j - 1/2)). */
static void node_rates(const orc_ctx* c, const macro_t* m, double* s, double* sig) {
    double mu = viscosity(c, m->T);
    double nu = mu / m->rho;
    double tau_p = 0.5 + nu / CS2;                     /* 1/s_p */
    double tau_q = 0.5 + 1.0 / (12.0 * (tau_p - 0.5)); /* (1/s_p-1/2)(1/s_q-1/2) = 1/12 */
    double varsig = c->cfg.bulk_ratio * nu;
    double tau_e = 0.5 + varsig / (c->cfg.varpi * CS2);
    double sp = 1.0 / tau_p, sq = 1.0 / tau_q, se = 1.0 / tau_e;
    s[0] = 1.0; s[1] = se; s[2] = se; s[3] = 1.0; s[4] = sq; s[5] = 1.0; s[6] = sq; s[7] = sp; s[8] = sp;

    double lam = c->Cp * mu / c->cfg.Pr;
    double coef = 2.0 / 3.0 + c->cfg.gamma1 / 2.0 + c->cfg.gamma2 / 3.0;
    double tj = 0.5 + lam / (coef * c->cfg.rho0 * c->Cp0);  /* 1/sigma_j */
    double te = 0.5 + 1.0 / (4.0 * (tj - 0.5));             /* (1/sj-1/2)(1/se-1/2) = 1/4 */
    double sj = 1.0 / tj, sgE = 1.0 / te;
    sig[0] = 1.0; sig[1] = sgE; sig[2] = sgE; sig[3] = sj; sig[4] = sj; sig[5] = sj; sig[6] = sj;
    sig[7] = sgE; sig[8] = sgE;
}

/* m^eq of Sec. 2.1. */
static void build_meq(const orc_ctx* c, const macro_t* m, double* meq) {
    double r = m->rho, ux = m->ux, uy = m->uy, u2 = ux * ux + uy * uy;
    meq[0] = r;
    meq[1] = 2.0 * c->alpha1 * r + 2.0 * c->beta1 * m->eta + 3.0 * r * u2;
    meq[2] = c->alpha2 * r + c->beta2 * m->eta - 3.0 * r * u2 + 9.0 * r * ux * ux * uy * uy;
    meq[3] = r * ux;
    meq[4] = -r * ux + 3.0 * r * ux * uy * uy;
    meq[5] = r * uy;
    meq[6] = -r * uy + 3.0 * r * uy * ux * ux;
    meq[7] = r * (ux * ux - uy * uy);
    meq[8] = r * ux * uy;
}

/* F_m of Sec. 2.1 with the bracket read by the product rule of m^eq. */
static void build_Fm(const macro_t* m, double* Fm) {
    double Fx = m->Fx, Fy = m->Fy, ux = m->ux, uy = m->uy;
    double Fu = Fx * ux + Fy * uy;
    double b_xxyy = 2.0 * Fx * ux * uy * uy + 2.0 * Fy * uy * ux * ux;
    double b_xyy = Fx * uy * uy + 2.0 * Fy * ux * uy;
    double b_xxy = Fy * ux * ux + 2.0 * Fx * ux * uy;
    Fm[0] = 0.0;
    Fm[1] = 6.0 * Fu;
    Fm[2] = -6.0 * Fu + 9.0 * b_xxyy;
    Fm[3] = Fx;
    Fm[4] = -Fx + 3.0 * b_xyy;
    Fm[5] = Fy;
    Fm[6] = -Fy + 3.0 * b_xxy;
    Fm[7] = 2.0 * (Fx * ux - Fy * uy);
    Fm[8] = Fx * uy + Fy * ux;
}

/* Modified collision matrix S of Sec. 2.1. */
static void build_S(const orc_ctx* c, const macro_t* m, const double* s, double* S) {
    memset(S, 0, 81 * sizeof(double));
    double se = s[1], seps = s[2], sq = s[4], sp = s[7];
    double we = se / 2.0 - 1.0, wp = sp / 2.0 - 1.0;
    for (int k = 0; k < 9; ++k) S[k * 9 + k] = s[k];
    S[1 * 9 + 2] = c->kk * seps * we;
    S[1 * 9 + 4] = c->hh * m->ux * sq * we;
    S[1 * 9 + 6] = c->hh * m->uy * sq * we;
    S[7 * 9 + 4] = 2.0 * c->bb * m->ux * sq * wp;
    S[7 * 9 + 6] = -2.0 * c->bb * m->uy * sq * wp;
    S[8 * 9 + 4] = c->bb * m->uy * sq * wp;
    S[8 * 9 + 6] = c->bb * m->ux * sq * wp;
}

/* Correction matrix R of Sec. 2.1 (nonzero rows/cols 1, 7, 8). */
static void build_R(const orc_ctx* c, const macro_t* m, const double* s, double* R) {
    memset(R, 0, 81 * sizeof(double));
    double k = c->kk, h = c->hh, b = c->bb, w = c->cfg.varpi;
    double se = s[1], sp = s[7];
    double ux = m->ux, uy = m->uy;
    double sum2 = ux * ux + uy * uy, dif2 = ux * ux - uy * uy, xy = ux * uy;
    R[1 * 9 + 1] = -((9.0 - 15.0 * k - 2.0 * h) * se / (4.0 * w)) * sum2;
    R[1 * 9 + 7] = -(3.0 * (9.0 - 3.0 * k + 2.0 * h) * sp * (2.0 - se) / (4.0 * (2.0 - sp))) * dif2;
    R[1 * 9 + 8] = (12.0 * (3.0 * k + h) * sp * (2.0 - se) / (2.0 - sp)) * xy;
    R[7 * 9 + 1] = -((3.0 - 4.0 * b) * se * (2.0 - sp) / (4.0 * w * (2.0 - se))) * dif2;
    R[7 * 9 + 7] = -(3.0 * (3.0 + 4.0 * b) * sp / 4.0) * sum2;
    R[7 * 9 + 8] = 0.0;
    R[8 * 9 + 1] = (b * se * (2.0 - sp) / (w * (2.0 - se))) * xy;
    R[8 * 9 + 7] = 0.0;
    R[8 * 9 + 8] = 6.0 * b * sp * sum2;
}

/* Correction matrices T and X (9 x 2) of Sec. 2.1; rows 1, 7, 8 nonzero. */
static void build_TX(const orc_ctx* c, const macro_t* m, const double* s, double* Tm, double* Xm) {
    memset(Tm, 0, 18 * sizeof(double));
    memset(Xm, 0, 18 * sizeof(double));
    double k = c->kk, h = c->hh, b = c->bb;
    double se = s[1], sp = s[7];
    double ux = m->ux, uy = m->uy;
    double ux2 = ux * ux, uy2 = uy * uy;
    double t1 = 3.0 * (2.0 - se) / 2.0;
    Tm[1 * 2 + 0] = t1 * ((1.0 - k) * ux2 * ux - (2.0 * k + h) * ux * uy2);
    Tm[1 * 2 + 1] = t1 * ((1.0 - k) * uy2 * uy - (2.0 * k + h) * ux2 * uy);
    double t7 = (2.0 - sp) / 2.0;
    Tm[7 * 2 + 0] = t7 * (ux2 * ux + 2.0 * b * ux * uy2);
    Tm[7 * 2 + 1] = t7 * (-uy2 * uy - 2.0 * b * ux2 * uy);
    double t8 = -b * (2.0 - sp) / 2.0;
    Tm[8 * 2 + 0] = t8 * (uy2 * uy + 2.0 * ux2 * uy);
    Tm[8 * 2 + 1] = t8 * (ux2 * ux + 2.0 * ux * uy2);

    double x1 = 9.0 * (2.0 * k + h) * (2.0 - se) / 2.0;
    Xm[1 * 2 + 0] = x1 * (ux * uy2);
    Xm[1 * 2 + 1] = x1 * (ux2 * uy);
    double x7 = -3.0 * b * (2.0 - sp);
    Xm[7 * 2 + 0] = x7 * (ux * uy2);
    Xm[7 * 2 + 1] = x7 * (-ux2 * uy);
    double x8 = 3.0 * b * (2.0 - sp) / 2.0;
    Xm[8 * 2 + 0] = x8 * (uy2 * uy + 2.0 * ux2 * uy);
    Xm[8 * 2 + 1] = x8 * (ux2 * ux + 2.0 * ux * uy2);
}

/* n^eq and Q_m of Sec. 2.2. */
static void build_neq(const orc_ctx* c, const macro_t* m, double* neq) {
    double rE = m->rho * m->E;
    double ref = c->cfg.rho0 * c->Cp0 * m->T;
    double rH = m->rho * m->H;
    neq[0] = rE;
    neq[1] = -4.0 * (rE - ref) + c->cfg.gamma1 * ref;
    neq[2] = 4.0 * (rE - ref) + c->cfg.gamma2 * ref;
    neq[3] = rH * m->ux;
    neq[4] = -rH * m->ux;
    neq[5] = rH * m->uy;
    neq[6] = -rH * m->uy;
    neq[7] = 0.0;
    neq[8] = 0.0;
}

static void build_Qm(const orc_ctx* c, const macro_t* m, double* Qm) {
    double q = m->qe;
    Qm[0] = q;
    Qm[1] = c->cfg.gamma1 * q;
    Qm[2] = c->cfg.gamma2 * q;
    Qm[3] = q * m->ux;
    Qm[4] = -q * m->ux;
    Qm[5] = q * m->uy;
    Qm[6] = -q * m->uy;
    Qm[7] = 0.0;
    Qm[8] = 0.0;
}

/* Modified collision matrix L of Sec. 2.2. */
static void build_L(const double* sig, double* L) {
    memset(L, 0, 81 * sizeof(double));
    for (int k = 0; k < 9; ++k) L[k * 9 + k] = sig[k];
    double wj = sig[3] / 2.0 - 1.0;
    L[3 * 9 + 4] = sig[4] * wj;
    L[5 * 9 + 6] = sig[6] * wj;
}

/* Viscous-dissipation matrix Y, Eq. (Y.nonzero), with Y_4a = -Y_3a, Y_6a = -Y_5a. */
static void build_Y(const macro_t* m, double* Y) {
    memset(Y, 0, 81 * sizeof(double));
    double ux = m->ux, uy = m->uy;
    Y[3 * 9 + 1] = ux / 3.0;
    Y[3 * 9 + 7] = ux;
    Y[3 * 9 + 8] = 2.0 * uy;
    Y[5 * 9 + 1] = uy / 3.0;
    Y[5 * 9 + 7] = -uy;
    Y[5 * 9 + 8] = 2.0 * ux;
    for (int a = 0; a < 9; ++a) {
        Y[4 * 9 + a] = -Y[3 * 9 + a];
        Y[6 * 9 + a] = -Y[5 * 9 + a];
    }
}

static void I_minus_half(const double* A, double* out) {
    for (int r = 0; r < 9; ++r)
        for (int k = 0; k < 9; ++k) out[r * 9 + k] = (r == k ? 1.0 : 0.0) - 0.5 * A[r * 9 + k];
}

/* Dense collision of one node, Eqs. (LBE.u.c) and (LBE.T.c). */
static void collide_node(const orc_ctx* c, const double* f, const double* g,
                         const double* grho, const double* gp, orc_node_info* o) {
    macro_t mc;
    node_macros(c, f, g, &mc);
    o->rho = mc.rho; o->ux = mc.ux; o->uy = mc.uy; o->Fx = mc.Fx; o->Fy = mc.Fy;
    o->qe = mc.qe; o->E = mc.E; o->T = mc.T; o->p = mc.p; o->eta = mc.eta; o->H = mc.H;
    node_rates(c, &mc, o->s, o->sig);

    matvec9(MROWS, f, o->m);
    matvec9(MROWS, g, o->n);
    build_meq(c, &mc, o->meq);
    build_Fm(&mc, o->Fm);
    build_S(c, &mc, o->s, o->S);
    build_R(c, &mc, o->s, o->R);
    build_TX(c, &mc, o->s, o->Tm, o->Xm);
    build_neq(c, &mc, o->neq);
    build_Qm(c, &mc, o->Qm);
    build_L(o->sig, o->L);
    build_Y(&mc, o->Y);

    double d[9], Sd[9], IS2[81], IS2d[9], RIS2d[9];
    for (int k = 0; k < 9; ++k) d[k] = o->m[k] - o->meq[k] + 0.5 * o->Fm[k];
    matvec9(o->S, d, Sd);
    I_minus_half(o->S, IS2);
    matvec9(IS2, d, IS2d);
    matvec9(o->R, IS2d, RIS2d);
    int corr = c->cfg.corrections;
    for (int k = 0; k < 9; ++k) {
        double v = o->m[k] + o->Fm[k] - Sd[k];
        if (corr) {
            v -= RIS2d[k];
            v -= o->Tm[k * 2 + 0] * grho[0] + o->Tm[k * 2 + 1] * grho[1];
            v -= o->Xm[k * 2 + 0] * gp[0] + o->Xm[k * 2 + 1] * gp[1];
        }
        o->mbar[k] = v;
    }

    double dn[9], Ldn[9], Gt[9], YG[9];
    for (int k = 0; k < 9; ++k) dn[k] = o->n[k] - o->neq[k] + 0.5 * o->Qm[k];
    matvec9(o->L, dn, Ldn);
    for (int k = 0; k < 9; ++k) Gt[k] = 0.5 * (o->m[k] + o->mbar[k]) - o->meq[k];
    matvec9(o->Y, Gt, YG);
    for (int k = 0; k < 9; ++k) o->nbar[k] = o->n[k] + o->Qm[k] - Ldn[k] + YG[k];

    matvec9(c->Minv, o->mbar, o->fbar);
    matvec9(c->Minv, o->nbar, o->gbar);

    double IL2[81];
    I_minus_half(o->L, IL2);
    invert9(IS2, o->IS2inv);
    invert9(IL2, o->IL2inv);
}

int orc_node(const orc_ctx* c, const double* f9, const double* g9,
             const double* grad_rho, const double* grad_p, orc_node_info* out) {
    if (!c || !c->eos_set) return -1;
    double z[2] = {0.0, 0.0};
    collide_node(c, f9, g9, grad_rho ? grad_rho : z, grad_p ? grad_p : z, out);
    return 0;
}

int orc_eq_moments(const orc_ctx* c, double rho, double ux, double uy, double T,
                   double Fx, double Fy, double* meq, double* Fm, double* neq, double* Qm) {
    if (!c || !c->eos_set) return -1;
    macro_t mc;
    double E = c->Cv * T + 0.5 * (ux * ux + uy * uy);
    wall_macros(c, rho, ux, uy, E, &mc);
    mc.Fx = Fx;
    mc.Fy = Fy;
    mc.qe = ux * Fx + uy * Fy;
    if (meq) build_meq(c, &mc, meq);
    if (Fm) build_Fm(&mc, Fm);
    if (neq) build_neq(c, &mc, neq);
    if (Qm) build_Qm(c, &mc, Qm);
    return 0;
}

/* ------------------------------------------------------------------ */
/* lattice geometry                                                   */
/* ------------------------------------------------------------------ */

static inline long nidx(const orc_ctx* c, int x, int y) { return ((long)y * c->cfg.nx + x) * 9; }

typedef struct {
    int is_wall, corner;
    int dx, dy;            /* inward normal */
    double ux, uy;         /* wall velocity */
    int thermal;           /* 0 Dirichlet, 1 Neumann */
    double T;
    int order;
} wall_info;

/* Wall data of node (x, y): straight walls use their side's data; corners
 * take velocity 0, the x-side's extrapolation order, and a Dirichlet
 * temperature from whichever adjacent side is Dirichlet (x-side first). */
static void node_wall(const orc_ctx* c, int x, int y, wall_info* w) {
    const orc_config* k = &c->cfg;
    int onS = !c->py && y == 0, onN = !c->py && y == k->ny - 1;
    int onW = !c->px && x == 0, onE = !c->px && x == k->nx - 1;
    memset(w, 0, sizeof(*w));
    if (!(onS || onN || onW || onE)) return;
    w->is_wall = 1;
    w->dx = onW ? 1 : (onE ? -1 : 0);
    w->dy = onS ? 1 : (onN ? -1 : 0);
    const orc_wall* ws = onS ? &k->wall[0] : (onN ? &k->wall[1] : NULL);
    const orc_wall* wx = onW ? &k->wall[2] : (onE ? &k->wall[3] : NULL);
    if (ws && wx) {
        w->corner = 1;
        w->ux = 0.0; w->uy = 0.0;
        w->order = wx->extrap_order;
        if (wx->thermal == 0) { w->thermal = 0; w->T = wx->T; }
        else if (ws->thermal == 0) { w->thermal = 0; w->T = ws->T; }
        else { w->thermal = 1; w->T = 0.0; }
    } else {
        const orc_wall* ww = ws ? ws : wx;
        w->ux = ww->u[0]; w->uy = ww->u[1];
        w->thermal = ww->thermal; w->T = ww->T;
        w->order = ww->extrap_order;
    }
}

static inline int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* Gradient of a node field phi at (x, y): 9-point isotropic stencil
 * grad = 3 sum_i w_i e_i phi(x + e_i) in the interior (periodic wrap);
 * along a wall normal one-sided second order, tangentially central. */
static void node_grad(const orc_ctx* c, const double* phi, int x, int y, double* gr) {
    static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    int nx = c->cfg.nx, ny = c->cfg.ny;
    wall_info w;
    node_wall(c, x, y, &w);
    if (!w.is_wall) {
        double gx = 0, gy = 0;
        for (int i = 1; i < 9; ++i) {
            int xn = c->px ? wrap(x + EX[i], nx) : x + EX[i];
            int yn = c->py ? wrap(y + EY[i], ny) : y + EY[i];
            double v = phi[(long)yn * nx + xn];
            gx += W[i] * EX[i] * v;
            gy += W[i] * EY[i] * v;
        }
        gr[0] = 3.0 * gx;
        gr[1] = 3.0 * gy;
        return;
    }
#define PHI(xx, yy) phi[(long)(yy) * nx + (xx)]
    if (w.dx != 0) {
        double p0 = PHI(x, y), p1 = PHI(x + w.dx, y), p2 = PHI(x + 2 * w.dx, y);
        gr[0] = w.dx * (-3.0 * p0 + 4.0 * p1 - p2) / 2.0;
    } else {
        int xa = c->px ? wrap(x + 1, nx) : x + 1;
        int xb = c->px ? wrap(x - 1, nx) : x - 1;
        gr[0] = (PHI(xa, y) - PHI(xb, y)) / 2.0;
    }
    if (w.dy != 0) {
        double p0 = PHI(x, y), p1 = PHI(x, y + w.dy), p2 = PHI(x, y + 2 * w.dy);
        gr[1] = w.dy * (-3.0 * p0 + 4.0 * p1 - p2) / 2.0;
    } else {
        int ya = c->py ? wrap(y + 1, ny) : y + 1;
        int yb = c->py ? wrap(y - 1, ny) : y - 1;
        gr[1] = (PHI(x, ya) - PHI(x, yb)) / 2.0;
    }
#undef PHI
}

/* The gradient of one field [ny][nx] at every node by node_grad, for the
 * tests that pin the stencil on fields whose gradient is known exactly. */
int orc_grad_field(const orc_ctx* c, const double* phi, double* gx, double* gy) {
    if (!c || !phi || !gx || !gy) return -1;
    for (int y = 0; y < c->cfg.ny; ++y)
        for (int x = 0; x < c->cfg.nx; ++x) {
            double gr[2];
            node_grad(c, phi, x, y, gr);
            gx[(long)y * c->cfg.nx + x] = gr[0];
            gy[(long)y * c->cfg.nx + x] = gr[1];
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* wall pass (Sec. 3)                                                 */
/* ------------------------------------------------------------------ */

/* Redefined non-equilibrium moments of Eq. (neq.redefinition) at a node
 * whose post-streaming DFs are f, g. */
static void node_tilde_neq(const orc_ctx* c, const double* f, const double* g,
                           double* mt, double* nt) {
    macro_t mc;
    node_macros(c, f, g, &mc);
    double s[9], sig[9], m[9], n[9], meq[9], Fm[9], neq[9], Qm[9];
    double S[81], L[81], Y[81], IS2[81], IL2[81];
    node_rates(c, &mc, s, sig);
    matvec9(MROWS, f, m);
    matvec9(MROWS, g, n);
    build_meq(c, &mc, meq);
    build_Fm(&mc, Fm);
    build_neq(c, &mc, neq);
    build_Qm(c, &mc, Qm);
    build_S(c, &mc, s, S);
    build_L(sig, L);
    build_Y(&mc, Y);
    I_minus_half(S, IS2);
    I_minus_half(L, IL2);
    double mneq[9], nneq[9], a[9], bvec[9];
    for (int k = 0; k < 9; ++k) {
        mneq[k] = m[k] - meq[k] + 0.5 * Fm[k];
        nneq[k] = n[k] - neq[k] + 0.5 * Qm[k];
    }
    matvec9(IS2, mneq, mt);
    matvec9(IL2, nneq, a);
    matvec9(Y, mt, bvec);
    for (int k = 0; k < 9; ++k) nt[k] = a[k] + 0.5 * bvec[k];
}

static void wall_node_rebuild(const orc_ctx* c, double* F, double* G, int x, int y, const wall_info* w) {
    double* fb = F + nidx(c, x, y);
    double* gb = G + nidx(c, x, y);
    /* density and (Neumann) total energy from the bounced-back populations */
    double rho = 0.0, sg = 0.0;
    for (int i = 0; i < 9; ++i) { rho += fb[i]; sg += gb[i]; }
    double ux = w->ux, uy = w->uy, E;
    if (w->thermal == 0) {
        E = c->Cv * w->T + 0.5 * (ux * ux + uy * uy);
    } else {
        double Fx, Fy;
        force_at(c, rho, &Fx, &Fy);
        double qe = ux * Fx + uy * Fy;
        E = (sg + 0.5 * qe) / rho;
    }
    macro_t mb;
    wall_macros(c, rho, ux, uy, E, &mb);

    /* extrapolated redefined non-equilibrium parts */
    double mt_f[9], nt_f[9], mt[9], nt[9];
    int xf = x + w->dx, yf = y + w->dy;
    node_tilde_neq(c, F + nidx(c, xf, yf), G + nidx(c, xf, yf), mt_f, nt_f);
    if (w->order == 2) {
        double mt_ff[9], nt_ff[9];
        int xff = x + 2 * w->dx, yff = y + 2 * w->dy;
        node_tilde_neq(c, F + nidx(c, xff, yff), G + nidx(c, xff, yff), mt_ff, nt_ff);
        for (int k = 0; k < 9; ++k) {
            mt[k] = 2.0 * mt_f[k] - mt_ff[k];
            nt[k] = 2.0 * nt_f[k] - nt_ff[k];
        }
    } else {
        memcpy(mt, mt_f, sizeof(mt));
        memcpy(nt, nt_f, sizeof(nt));
    }

    /* back to m^neq, n^neq with the wall node's own S, L, Y */
    double s[9], sig[9], S[81], L[81], Y[81], IS2[81], IL2[81], IS2i[81], IL2i[81];
    node_rates(c, &mb, s, sig);
    build_S(c, &mb, s, S);
    build_L(sig, L);
    build_Y(&mb, Y);
    I_minus_half(S, IS2);
    I_minus_half(L, IL2);
    invert9(IS2, IS2i);
    invert9(IL2, IL2i);
    double mneq[9], Ymt[9], rhs[9], nneq[9];
    matvec9(IS2i, mt, mneq);
    matvec9(Y, mt, Ymt);
    for (int k = 0; k < 9; ++k) rhs[k] = nt[k] - 0.5 * Ymt[k];
    matvec9(IL2i, rhs, nneq);

    double meq[9], Fm[9], neq[9], Qm[9], m[9], n[9];
    build_meq(c, &mb, meq);
    build_Fm(&mb, Fm);
    build_neq(c, &mb, neq);
    build_Qm(c, &mb, Qm);
    for (int k = 0; k < 9; ++k) {
        m[k] = meq[k] - 0.5 * Fm[k] + mneq[k];
        n[k] = neq[k] - 0.5 * Qm[k] + nneq[k];
    }
    matvec9(c->Minv, m, fb);
    matvec9(c->Minv, n, gb);
}

static void boundary_pass(orc_ctx* c, double* F, double* G) {
    int nx = c->cfg.nx, ny = c->cfg.ny;
    if (c->px && c->py) return;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            wall_info w;
            node_wall(c, x, y, &w);
            if (w.is_wall) wall_node_rebuild(c, F, G, x, y, &w);
        }
}

int orc_boundary_pass(orc_ctx* c) {
    if (!c || !c->eos_set) return -1;
    boundary_pass(c, c->f, c->g);
    return 0;
}

/* ------------------------------------------------------------------ */
/* API                                                                */
/* ------------------------------------------------------------------ */

int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_create(const orc_config* cfg, orc_ctx** out) {
    if (!cfg || !out) return -1;
    *out = NULL;
    int px = cfg->wall[2].periodic != 0, pxe = cfg->wall[3].periodic != 0;
    int py = cfg->wall[0].periodic != 0, pyn = cfg->wall[1].periodic != 0;
    if (px != pxe || py != pyn) return -1;
    if (cfg->nx < 1 || cfg->ny < 1) return -1;
    for (int s = 0; s < 4; ++s) {
        if (cfg->wall[s].periodic) continue;
        if (cfg->wall[s].extrap_order != 1 && cfg->wall[s].extrap_order != 2) return -1;
    }
    if (!px && cfg->nx < 4) return -1;
    if (!py && cfg->ny < 4) return -1;
    if (!(cfg->tau0 > 0.5) || !(cfg->rho0 > 0) || !(cfg->T0 > 0) || !(cfg->gamma > 1.0)) return -1;
    orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    if (!c) return -2;
    c->cfg = *cfg;
    c->px = px; c->py = py;
    long nn = (long)cfg->nx * cfg->ny;
    c->f = (double*)calloc((size_t)nn * 9, sizeof(double));
    c->g = (double*)calloc((size_t)nn * 9, sizeof(double));
    c->f2 = (double*)calloc((size_t)nn * 9, sizeof(double));
    c->g2 = (double*)calloc((size_t)nn * 9, sizeof(double));
    c->rho_f = (double*)calloc((size_t)nn, sizeof(double));
    c->p_f = (double*)calloc((size_t)nn, sizeof(double));
    if (!c->f || !c->g || !c->f2 || !c->g2 || !c->rho_f || !c->p_f) { orc_destroy(c); return -2; }
    if (invert9(MROWS, c->Minv) != 0) { orc_destroy(c); return -1; }
    /* Eq. (LBE.u.coefficients) with alpha1 = -1, beta1 = 1 */
    double w = cfg->varpi;
    c->alpha1 = -1.0;
    c->beta1 = 1.0;
    c->alpha2 = -(2.0 * c->alpha1 + w + 1.0) / (1.0 - w);
    c->beta2 = -2.0 * c->beta1 / (1.0 - w);
    c->kk = 1.0 - w;
    c->hh = 6.0 * w * (1.0 - w) / (1.0 - 3.0 * w);
    c->bb = (1.0 - w) / (1.0 - 3.0 * w);
    *out = c;
    return 0;
}

int orc_destroy(orc_ctx* c) {
    if (!c) return 0;
    free(c->f); free(c->g); free(c->f2); free(c->g2); free(c->rho_f); free(c->p_f);
    free(c);
    return 0;
}

/* Rest-state initialisation (zero non-equilibrium part, Eq. decompose):
 * f = M^-1 (m^eq - F_m/2), g = M^-1 (n^eq - Q_m/2) at (rho0, u = 0, T0). */
static void init_rest(orc_ctx* c) {
    macro_t mc;
    double E0 = c->Cv * c->cfg.T0;
    wall_macros(c, c->cfg.rho0, 0.0, 0.0, E0, &mc);
    double meq[9], Fm[9], neq[9], Qm[9], m[9], n[9], f[9], g[9];
    build_meq(c, &mc, meq);
    build_Fm(&mc, Fm);
    build_neq(c, &mc, neq);
    build_Qm(c, &mc, Qm);
    for (int k = 0; k < 9; ++k) { m[k] = meq[k] - 0.5 * Fm[k]; n[k] = neq[k] - 0.5 * Qm[k]; }
    matvec9(c->Minv, m, f);
    matvec9(c->Minv, n, g);
    long nn = (long)c->cfg.nx * c->cfg.ny;
    for (long j = 0; j < nn; ++j)
        for (int i = 0; i < 9; ++i) { c->f[j * 9 + i] = f[i]; c->g[j * 9 + i] = g[i]; }
    c->step = 0;
    c->unstable = 0;
}

/* EOS selection and the derived thermodynamic constants (Eqs. cs, Cp):
 * R such that d p_EOS / d rho = c_s^2 = 1/3 at (rho0, T0);
 * Cp - Cv = p0 / (rho0 T0) with Cp / Cv = gamma. */
int orc_set_eos(orc_ctx* c, int kind, const double* params, int np) {
    if (!c || kind < 0 || kind > 3) return -1;
    c->eos_kind = kind;
    c->eos_a = 0.0;
    c->eos_b = 0.0;
    if (kind == 2) {
        c->eos_b = (np >= 1 && params) ? params[0] : sqrt(2.0) * M_PI / (3.0 * c->cfg.rho0);
    } else if (kind == 3) {
        if (np < 2 || !params) return -1;
        c->eos_a = params[0];
        c->eos_b = params[1];
        if (!(c->eos_b * c->cfg.rho0 < 1.0)) return -1;
    }
    double A, B;
    c->R = 1.0;
    eos_dpdrho_parts(c, c->cfg.rho0, c->cfg.T0, &A, &B);
    if (!(A > 0)) return -1;
    c->R = (CS2 - B) / A;
    if (!(c->R > 0)) return -1;
    c->p0 = eos_p(c, c->cfg.rho0, c->cfg.T0);
    c->Cv = (c->p0 / (c->cfg.rho0 * c->cfg.T0)) / (c->cfg.gamma - 1.0);
    c->Cp = c->cfg.gamma * c->Cv;
    c->Cp0 = c->Cp;
    c->mu0 = c->cfg.rho0 * (c->cfg.tau0 - 0.5) * CS2;
    c->eta0 = (c->p0 / CS2 - (2.0 + c->alpha1) * c->cfg.rho0) / c->beta1;
    c->lambda0 = c->Cp * c->mu0 / c->cfg.Pr;
    c->eos_set = 1;
    init_rest(c);
    return 0;
}

int orc_derived(const orc_ctx* c, double* out8) {
    if (!c || !c->eos_set) return -1;
    out8[0] = c->R; out8[1] = c->Cv; out8[2] = c->Cp; out8[3] = c->mu0;
    out8[4] = c->p0; out8[5] = c->eta0; out8[6] = c->lambda0; out8[7] = CS2;
    return 0;
}

long orc_step_count(const orc_ctx* c) { return c ? c->step : -1; }

static int one_step(orc_ctx* c) {
    int nx = c->cfg.nx, ny = c->cfg.ny;
    long nn = (long)nx * ny;
    int bad = 0;

    /* 1-2: macros and gradients at time t */
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long j = 0; j < nn; ++j) {
        macro_t mc;
        node_macros(c, c->f + j * 9, c->g + j * 9, &mc);
        c->rho_f[j] = mc.rho;
        c->p_f[j] = mc.p;
        if (!isfinite(mc.rho) || !isfinite(mc.T) || !isfinite(mc.ux) || !isfinite(mc.uy)) bad |= 1;
    }
    if (bad) return -4;

    /* 3-4: collide every node and push into the second lattice */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        orc_node_info o;
        for (int x = 0; x < nx; ++x) {
            double gr[2], gp[2];
            node_grad(c, c->rho_f, x, y, gr);
            node_grad(c, c->p_f, x, y, gp);
            collide_node(c, c->f + nidx(c, x, y), c->g + nidx(c, x, y), gr, gp, &o);
            for (int i = 0; i < 9; ++i) {
                int xd = x + EX[i], yd = y + EY[i];
                int out = 0;
                if (c->px) xd = wrap(xd, nx); else if (xd < 0 || xd >= nx) out = 1;
                if (c->py) yd = wrap(yd, ny); else if (yd < 0 || yd >= ny) out = 1;
                if (out) {
                    /* Eqs. (BB.f), (BB.g): reverse into the own opposite slot */
                    int ib = opposite(i);
                    c->f2[nidx(c, x, y) + ib] = o.fbar[i];
                    c->g2[nidx(c, x, y) + ib] = o.gbar[i];
                } else {
                    c->f2[nidx(c, xd, yd) + i] = o.fbar[i];
                    c->g2[nidx(c, xd, yd) + i] = o.gbar[i];
                }
            }
        }
    }

    /* 5: wall pass on the streamed lattice */
    boundary_pass(c, c->f2, c->g2);

    double* t;
    t = c->f; c->f = c->f2; c->f2 = t;
    t = c->g; c->g = c->g2; c->g2 = t;
    c->step += 1;
    return 0;
}

int orc_step(orc_ctx* c, long nsteps) {
    if (!c || !c->eos_set) return -1;
    if (c->unstable) return -4;
    for (long s = 0; s < nsteps; ++s) {
        int st = one_step(c);
        if (st != 0) { c->unstable = 1; return st; }
    }
    return 0;
}

int orc_macros(orc_ctx* c, double* rho, double* ux, double* uy, double* T, double* p) {
    if (!c || !c->eos_set) return -1;
    long nn = (long)c->cfg.nx * c->cfg.ny;
    for (long j = 0; j < nn; ++j) {
        macro_t mc;
        node_macros(c, c->f + j * 9, c->g + j * 9, &mc);
        if (rho) rho[j] = mc.rho;
        if (ux) ux[j] = mc.ux;
        if (uy) uy[j] = mc.uy;
        if (T) T[j] = mc.T;
        if (p) p[j] = mc.p;
    }
    return 0;
}

/* Equilibrium initialisation from macroscopic fields (Eq. decompose with a
 * zero non-equilibrium part): f = M^-1 (m^eq - F_m/2), g = M^-1 (n^eq - Q_m/2). */
int orc_init_macros(orc_ctx* c, const double* rho, const double* ux, const double* uy, const double* T) {
    if (!c || !c->eos_set || !rho || !ux || !uy || !T) return -1;
    long nn = (long)c->cfg.nx * c->cfg.ny;
    for (long j = 0; j < nn; ++j) {
        macro_t mc;
        double E = c->Cv * T[j] + 0.5 * (ux[j] * ux[j] + uy[j] * uy[j]);
        wall_macros(c, rho[j], ux[j], uy[j], E, &mc);
        double meq[9], Fm[9], neq[9], Qm[9], m[9], n[9];
        build_meq(c, &mc, meq);
        build_Fm(&mc, Fm);
        build_neq(c, &mc, neq);
        build_Qm(c, &mc, Qm);
        for (int k = 0; k < 9; ++k) { m[k] = meq[k] - 0.5 * Fm[k]; n[k] = neq[k] - 0.5 * Qm[k]; }
        matvec9(c->Minv, m, c->f + j * 9);
        matvec9(c->Minv, n, c->g + j * 9);
    }
    c->unstable = 0;
    return 0;
}

int orc_get_state(orc_ctx* c, double* f, double* g) {
    if (!c) return -1;
    long nn = (long)c->cfg.nx * c->cfg.ny;
    for (long j = 0; j < nn; ++j)
        for (int i = 0; i < 9; ++i) {
            if (f) f[(long)i * nn + j] = c->f[j * 9 + i];
            if (g) g[(long)i * nn + j] = c->g[j * 9 + i];
        }
    return 0;
}

int orc_set_state(orc_ctx* c, const double* f, const double* g) {
    if (!c || !f || !g) return -1;
    long nn = (long)c->cfg.nx * c->cfg.ny;
    for (long j = 0; j < nn; ++j)
        for (int i = 0; i < 9; ++i) {
            c->f[j * 9 + i] = f[(long)i * nn + j];
            c->g[j * 9 + i] = g[(long)i * nn + j];
        }
    c->unstable = 0;
    return 0;
}

/* Mean Nusselt number through a Dirichlet wall (Sec. 4.3): the inward heat
 * flux -lambda(T_wall) dT/dn with a one-sided second-order difference along
 * the inward normal, integrated along the wall by the trapezoid rule over
 * L = N - 1 and divided by lambda(T0) (T_hot - T_cold). */
int orc_nusselt(orc_ctx* c, int wall, double* nu) {
    if (!c || !c->eos_set || !nu || wall < 0 || wall > 3) return -1;
    const orc_config* k = &c->cfg;
    if (k->wall[wall].periodic) return -1;
    double tmax = -1e300, tmin = 1e300;
    int nd = 0;
    for (int s = 0; s < 4; ++s)
        if (!k->wall[s].periodic && k->wall[s].thermal == 0) {
            nd++;
            if (k->wall[s].T > tmax) tmax = k->wall[s].T;
            if (k->wall[s].T < tmin) tmin = k->wall[s].T;
        }
    if (nd < 2 || !(tmax > tmin)) return -1;
    int nx = k->nx, ny = k->ny;
    long nn = (long)nx * ny;
    double* T = (double*)malloc((size_t)nn * sizeof(double));
    if (!T) return -2;
    orc_macros(c, NULL, NULL, NULL, T, NULL);
    int along_y = (wall == 2 || wall == 3);
    int len = along_y ? ny : nx;
    double sum = 0.0;
    for (int t = 0; t < len; ++t) {
        int x0, y0, dx, dy;
        if (wall == 0) { x0 = t; y0 = 0; dx = 0; dy = 1; }
        else if (wall == 1) { x0 = t; y0 = ny - 1; dx = 0; dy = -1; }
        else if (wall == 2) { x0 = 0; y0 = t; dx = 1; dy = 0; }
        else { x0 = nx - 1; y0 = t; dx = -1; dy = 0; }
        double T0v = T[(long)y0 * nx + x0];
        double T1v = T[(long)(y0 + dy) * nx + (x0 + dx)];
        double T2v = T[(long)(y0 + 2 * dy) * nx + (x0 + 2 * dx)];
        double dTdn = (-3.0 * T0v + 4.0 * T1v - T2v) / 2.0;
        double lam = c->Cp * viscosity(c, T0v) / k->Pr;
        double q = -lam * dTdn;
        double wgt = (t == 0 || t == len - 1) ? 0.5 : 1.0;
        sum += wgt * q;
    }
    free(T);
    *nu = sum / (c->lambda0 * (tmax - tmin));
    return 0;
}
