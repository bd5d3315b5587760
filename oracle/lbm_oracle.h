/*
 * Plain FP64 CPU oracle of the thermal MRT lattice-Boltzmann model of
 * Huang, Wu & Adams (arXiv:1809.08683): D2Q9 density DF f_i (Sec. 2.1),
 * total-energy DF g_i (Sec. 2.2) and the wall treatment of Sec. 3.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this library; only the tests, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py do.  It shares no code, header or constant
 * table with the CUDA library: every matrix is built densely from the
 * paper's printed entries and M^-1, (I-S/2)^-1, (I-L/2)^-1 are obtained by
 * numeric Gauss-Jordan inversion, never from the closed forms of App. B.
 *
 * Lattice units throughout: c = dx = dt = 1, c_s^2 = 1/3.
 * DF arrays exchanged through this API are [q][ny][nx] (x fastest), FP64.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t periodic;     /* 1: this side is periodic (its opposite must be too) */
    int32_t thermal;      /* 0 Dirichlet (T given), 1 Neumann (adiabatic) */
    int32_t extrap_order; /* 1 or 2, Eq. (neq.extrapolation) */
    int32_t reserved;
    double u[2];          /* wall velocity */
    double T;             /* Dirichlet temperature */
} orc_wall;

typedef struct {
    int32_t nx, ny;
    int32_t precision;    /* ignored: the oracle always computes in FP64 */
    int32_t visc_law;     /* 0 constant mu, 1 mu ~ T, 2 Sutherland ratio form */
    double rho0, T0, Pr, gamma, tau0;
    double visc_p[2];     /* Sutherland: visc_p[0] = S / T0 */
    double bulk_ratio;    /* varsigma / nu */
    double varpi, gamma1, gamma2;
    int32_t force_mode;   /* 0: F = force, 1: F = rho * force (gravity) */
    int32_t corrections;  /* 1: keep R, T, X terms of Eq. (LBE.u.c) */
    double force[2];
    orc_wall wall[4];     /* S, N, W, E */
} orc_config;

/* Per-node intermediate quantities, for the algebraic pins. */
typedef struct {
    double rho, ux, uy, Fx, Fy, qe, E, T, p, eta, H;
    double s[9];          /* diag of S: s0 se seps sj sq sj sq sp sp */
    double sig[9];        /* diag of L */
    double m[9], meq[9], Fm[9], mbar[9];
    double n[9], neq[9], Qm[9], nbar[9];
    double S[81], R[81], L[81], Y[81];
    double Tm[18], Xm[18];          /* rows k: (k,x),(k,y) */
    double IS2inv[81], IL2inv[81];  /* numeric inverses of I-S/2, I-L/2 */
    double fbar[9], gbar[9];
} orc_node_info;

typedef struct orc_ctx orc_ctx;

int  orc_create(const orc_config* cfg, orc_ctx** out);
int  orc_set_eos(orc_ctx* c, int kind, const double* params, int np);
int  orc_step(orc_ctx* c, long nsteps);
int  orc_macros(orc_ctx* c, double* rho, double* ux, double* uy, double* T, double* p);
int  orc_nusselt(orc_ctx* c, int wall, double* nu);
int  orc_get_state(orc_ctx* c, double* f, double* g);
int  orc_set_state(orc_ctx* c, const double* f, const double* g);
int  orc_init_macros(orc_ctx* c, const double* rho, const double* ux, const double* uy, const double* T);
int  orc_destroy(orc_ctx* c);
long orc_step_count(const orc_ctx* c);
int  orc_set_threads(int n);
int  orc_derived(const orc_ctx* c, double* out8); /* R, Cv, Cp, mu0, p0, eta0, lambda0, cs2 */

/* Boundary-pass-only hook: apply Sec. 3 at every wall node of the current state. */
int  orc_boundary_pass(orc_ctx* c);
/* grad(phi) of a field [ny][nx] at every node with the stencil of step 2
 * (interior, walls, corners, periodic wraps), for the stencil's pins. */
int  orc_grad_field(const orc_ctx* c, const double* phi, double* gx, double* gy);

/* Node-level hooks for the algebraic pins. */
/* m^eq, F_m, n^eq, Q_m at given (rho, u, T) and force (Fx, Fy). */
int  orc_eq_moments(const orc_ctx* c, double rho, double ux, double uy, double T,
                    double Fx, double Fy, double* meq, double* Fm, double* neq, double* Qm);
void orc_matrix_M(double* out81);
void orc_matrix_Minv(double* out81);
int  orc_node(const orc_ctx* c, const double* f9, const double* g9,
              const double* grad_rho, const double* grad_p, orc_node_info* out);

#ifdef __cplusplus
}
#endif
#endif
