/*
 * C ABI of the GB300 (sm_103a) thermal MRT lattice-Boltzmann hot path:
 * Huang, Wu & Adams, "Lattice Boltzmann model with self-tuning equation of
 * state for coupled thermo-hydrodynamic flows", arXiv:1809.08683.
 *
 * One context = one D2Q9 lattice of nx * ny nodes (x fastest) carrying the
 * density DF f_i (Sec. 2.1, Eqs. LBE.u) and the total-energy DF g_i
 * (Sec. 2.2, Eqs. LBE.T), with the wall treatment of Sec. 3 on every
 * non-periodic side.  Lattice units: c = dx = dt = 1, c_s^2 = 1/3.
 *
 * Conventions
 *  - Every call returns an lbm_status; no exception or signal crosses the ABI.
 *    On error, lbm_last_error() returns a per-thread message (never freed by
 *    the caller).  A detected NaN/Inf (LBM_EUNSTABLE) is sticky until
 *    lbm_set_eos(), lbm_init_macros() or lbm_set_state() re-initialises.
 *  - Device memory: the caller passes one device buffer of
 *    lbm_workspace_bytes() bytes (256-byte aligned, owned by the caller,
 *    kept alive until lbm_destroy()); passing NULL makes the library
 *    allocate and own it.  Small launch tables are always library-owned.
 *  - Streams: all device work of a context is ordered on the cudaStream_t
 *    given at creation (NULL = legacy default stream).  lbm_step() is
 *    asynchronous; calls that return host data synchronise that stream.
 *  - Host arrays are caller-owned, row-major [ny][nx] (x fastest); DF
 *    arrays are [9][ny][nx].  Values are FP64 whatever the precision.
 *  - Storage: DFs are stored as deviations from the rest equilibrium
 *    f_i - M^-1 m^eq(rho0, u = 0, T0) (and the g analogue), in FP64
 *    (LBM_FP64) or FP32 (LBM_FP32_DEV); reductions are always FP64.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* bad argument or configuration */
    LBM_ENOMEM = -2,     /* workspace too small or allocation failed */
    LBM_ECUDA = -3,      /* a CUDA runtime call failed */
    LBM_EUNSTABLE = -4,  /* NaN/Inf detected in the state (sticky) */
    LBM_ETIMEOUT = -5    /* a bounded device wait gave up */
} lbm_status;

typedef enum { LBM_FP64 = 0, LBM_FP32_DEV = 1 } lbm_precision;
typedef enum { LBM_WALL_S = 0, LBM_WALL_N = 1, LBM_WALL_W = 2, LBM_WALL_E = 3 } lbm_wall;

/* EOS kinds: Eqs. (EOSs.1), (EOSs.2), (EOSs.3) of Sec. 4 and the cubic
 * p = rho R T / (1 - b rho) - a rho^2 (params {a, b}).  R is always chosen so
 * that dp/drho = c_s^2 = 1/3 at (rho0, T0), Eq. (cs). */
typedef enum { LBM_EOS_DECOUPLING = 0, LBM_EOS_IDEAL = 1, LBM_EOS_CS = 2, LBM_EOS_CUBIC = 3 } lbm_eos;

/* Wall data of one side (Sec. 3).  A periodic side must face a periodic side. */
typedef struct {
    int32_t periodic;     /* 1: periodic pair, rest ignored */
    int32_t thermal;      /* 0 Dirichlet (T given), 1 Neumann (adiabatic, Eq. BB.g) */
    int32_t extrap_order; /* 1 or 2, Eq. (neq.extrapolation) */
    int32_t reserved;
    double u[2];          /* wall velocity */
    double T;             /* Dirichlet temperature */
} lbm_wall_bc;

/* Problem statement (Secs. 2-4).  Corner nodes take u = 0, the x-side's
 * extrapolation order, and a Dirichlet temperature if either side has one
 * (x-side first). */
typedef struct {
    int32_t nx, ny;       /* walled extents need >= 4 nodes, periodic >= 1 */
    int32_t precision;    /* lbm_precision */
    int32_t visc_law;     /* 0 constant mu, 1 mu = mu0 T/T0, 2 Sutherland */
    double rho0, T0;      /* reference state */
    double Pr;            /* Prandtl number Cp mu / lambda (Sec. 2.2).  High Pr puts
                           * sigma_j = 1 / (1/2 + 3 mu / (Pr rho0)) near 2, where the
                           * scheme's grid-scale modes grow: with tau0 = 0.8 and the
                           * paper's varpi, gamma1, gamma2, from Pr = 3 in a sheared
                           * channel and by Pr = 20 at rest.  A flow that stays exactly
                           * x-invariant never excites them; FP32 storage's stochastic
                           * rounding, whose draws depend on x, does. */
    double gamma;         /* Cp / Cv with Cp - Cv = p0 / (rho0 T0) */
    double tau0;          /* 1/s_p at (rho0, T0): mu0 = rho0 (tau0 - 1/2) / 3 */
    double visc_p[2];     /* Sutherland: visc_p[0] = S / T0 (ratio form of Sec. 4.3) */
    double bulk_ratio;    /* varsigma / nu (Table 1) */
    double varpi, gamma1, gamma2; /* Eq. (LBE.u.coefficients), n^eq; paper: 1/6, -2, 2 */
    int32_t force_mode;   /* 0: F = force; 1: F = rho * force (gravity) */
    int32_t corrections;  /* 1: keep the R, T, X terms of Eq. (LBE.u.c) */
    double force[2];
    lbm_wall_bc wall[4];  /* indexed by lbm_wall */
} lbm_config;

typedef struct lbm_ctx lbm_ctx;
typedef struct lbm_batch lbm_batch;

/* Device bytes needed by one context of this configuration. */
lbm_status lbm_workspace_bytes(const lbm_config* cfg, size_t* bytes);

/* Create a context.  workspace: device pointer (or NULL, see above);
 * cuda_stream: cudaStream_t or NULL.  *out receives the context. */
lbm_status lbm_create(const lbm_config* cfg, void* workspace, size_t workspace_bytes,
                      void* cuda_stream, lbm_ctx** out);

/* Select the EOS (Sec. 2.2 end, Eqs. EOSs, cs, Cp), derive R, Cv, Cp, mu0,
 * lambda0, and initialise the lattice at rest: f = M^-1 (m^eq - F_m/2),
 * g = M^-1 (n^eq - Q_m/2) at (rho0, 0, T0) (Eq. decompose, zero
 * non-equilibrium part).  params: {a, b} (cubic), {b} or none (CS). */
lbm_status lbm_set_eos(lbm_ctx* ctx, int kind, const double* params, int nparams);

/* Advance nsteps time steps (Eqs. LBE.u, LBE.T, BB.f, BB.g, Sec. 3):
 * fused collide + stream of every node, then the wall pass.  Async. */
lbm_status lbm_step(lbm_ctx* ctx, long nsteps);

/* Synchronise the context's stream and return its sticky status. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Macroscopic fields (Eqs. rho.u, E; T = eps / Cv; p = p_EOS) into host
 * arrays [ny][nx]; NULL skips a field.  Synchronises. */
lbm_status lbm_macros(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* T, double* p);

/* Same into device arrays [ny][nx] (FP64); asynchronous. */
lbm_status lbm_macros_device(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* T, double* p);

/* Mean Nusselt number through a Dirichlet wall (Sec. 4.3): inward flux
 * -lambda(T_w) dT/dn (one-sided, second order), trapezoid rule along the
 * wall over L = N - 1, divided by lambda(T0) (T_max - T_min) over the
 * Dirichlet walls.  Synchronises. */
lbm_status lbm_nusselt(lbm_ctx* ctx, int wall, double* nu);

/* FP64 global diagnostics, deterministic order.  out[8] receives:
 *  0 total mass sum(rho), 1 total energy sum(rho E), 2 p*_ave (trapezoid
 *  mean of p / p0 over the square, Sec. 4.3), 3 residual
 *  max(|u - u_snap|_2 / |u|_2, |T - T_snap|_2 / |T - T0|_2) against the
 *  last snapshot (0 if none), 4 number of non-finite nodes, 5 max |u|,
 *  6 mean T, 7 steps taken.  snapshot != 0 stores u, T as the new snapshot.
 *  Synchronises. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, int snapshot, double* out8);

/* DF state as [9][ny][nx] FP64 host arrays (full values, not deviations). */
lbm_status lbm_get_state(lbm_ctx* ctx, double* f, double* g);
lbm_status lbm_set_state(lbm_ctx* ctx, const double* f, const double* g);

/* Equilibrium initialisation from host fields rho, ux, uy, T [ny][nx]. */
lbm_status lbm_init_macros(lbm_ctx* ctx, const double* rho, const double* ux,
                           const double* uy, const double* T);

/* Derived constants: R, Cv, Cp, mu0, p0, eta0, lambda0, c_s^2. */
lbm_status lbm_derived(const lbm_ctx* ctx, double* out8);

/* Rounding of the FP32-deviation stores (no effect with FP64 storage).
 * LBM_ROUND_STOCHASTIC (the default after lbm_create): each stored value
 * gets uniform noise of one unit in its last place before rounding, so the
 * expected stored value is the exact one and a nearly steady state does not
 * stall on a repeated rounding error; the noise comes from a counter-based
 * hash of (node, step), so results are reproducible and the same alone or
 * batched.  It leaves a floor of about 1e-6 on the residual of
 * lbm_diagnostics.  LBM_ROUND_NEAREST: plain round-to-nearest, a
 * deterministic map.  The paper states no precision (Sec. 2 uses exact
 * arithmetic); both modes are this library's.  Takes effect from the next
 * step, also inside existing batches and their graphs; asynchronous on the
 * context's stream.  LBM_EINVAL for another mode. */
typedef enum { LBM_ROUND_STOCHASTIC = 0, LBM_ROUND_NEAREST = 1 } lbm_rounding;
lbm_status lbm_set_rounding(lbm_ctx* ctx, int mode);

/* Copy the state of src into dst, converting the storage precision (FP64 <->
 * FP32 deviations): both contexts must describe the same problem (identical
 * configurations apart from precision, the same EOS) and be initialised.
 * dst takes src's step count, so the residual snapshot of
 * lbm_diagnostics (also copied) and the stochastic rounding continue where
 * src left off.  Synchronises both streams.  The paper has no counterpart:
 * it lets a solve started in FP32 storage finish in FP64 once FP32 reaches
 * its residual floor.  LBM_EINVAL if the problems differ. */
lbm_status lbm_copy_state(lbm_ctx* dst, const lbm_ctx* src);

/* Check of the bounded-wait path of the fused kernels: one device thread
 * waits on an mbarrier that no copy will complete, gives up after
 * limit_cycles SM cycles (0 .. 2^32; the fused kernels use 2^32), and
 * records the timeout in the context's status word exactly as a fused
 * kernel whose row copy never landed does.  Returns LBM_ETIMEOUT, which is
 * then sticky on the context until lbm_set_eos(), lbm_init_macros() or
 * lbm_set_state() re-initialises it.  Synchronises.  The paper has no
 * counterpart; LBM_EINVAL for a limit outside the range. */
lbm_status lbm_wait_selftest(lbm_ctx* ctx, long long limit_cycles);

/* Arithmetic rates of the current device, for the roofline of the FP64
 * path, which the FP64 pipe bounds: out3[0] FP64 fused multiply-adds per
 * second, out3[1] FP32 fused multiply-adds per second, out3[2]
 * double-float multiply-adds (pairs of FP32 numbers carrying about 48
 * significant bits) per second, each the best
 * of three launches of dependent chains over the whole device.  Allocates
 * and frees a small device buffer; synchronises the stream (NULL = legacy
 * default stream).  The paper has no counterpart. */
lbm_status lbm_peak_rates(void* cuda_stream, double* out3);

/* Launch shape of the fused kernel: one CTA per strip of bx columns and by
 * rows (>= 1).  pair = 0: one node per thread, bx = 32, 64 or 128.
 * pair = 1 or 2 (FP32 storage only): two neighbouring nodes per thread in
 * packed FP32 arithmetic, bx = 64, 128 or 256; pair = 1 keeps each node's
 * macros in registers between the row pass and the collision, pair = 2
 * recomputes them (fewer registers, more threads per SM).  pair = 3 (FP32
 * storage only): one node per thread, bx = 32, 64 or 128, recomputing the
 * macros.  pair = 4: one node per thread in warps that each own 30 columns
 * and never synchronise with one another, bx = 30, 60 or 120 (1, 2 or 4
 * warps per CTA), any precision.  pair = 5 (FP32 storage only): warp
 * strips of 60 columns, two neighbouring nodes per lane in packed FP32,
 * bx = 60, 120 or 240.  pair = 0 and pair = 4 shapes of any width give
 * identical results; pairs 1-3 and 5 agree with them to FP32 rounding (their
 * arithmetic is contracted differently).  (bx, by, pair) = (0, 0, 0)
 * restores the default shape, which batches may then shorten.
 * Used by the autotuner. */
lbm_status lbm_set_tile(lbm_ctx* ctx, int bx, int by, int pair);

/* Launch shape in use: the default chosen by lbm_create and lbm_set_eos, or
 * the one set by lbm_set_tile.  Default: warp strips, pair = 4, bx = 30, for
 * nx <= 160; paired block strips, pair = 1, bx = 128, for wider FP32
 * lattices of the heated-cavity model class (see lbm_batch_create); block
 * strips, pair = 0, bx = 128, otherwise.  by = ny / 128 between 1 and 24
 * (FP32) or 8 (FP64); 3 ny / 512 between 1 and 12 for pair = 1.  by is
 * the run length when the lattice is stepped alone; a batch uses runs of
 * up to 24 (FP32; 32 for pair = 1) or 8 (FP64) rows for members whose
 * shape was not set, shortened until the batch fills the GPU.  In either
 * case the runs that make up the last fill of the GPU in a launch are cut
 * into up to four runs of at least 6 rows, launched last. */
lbm_status lbm_get_tile(const lbm_ctx* ctx, int* bx, int* by, int* pair);

/* Steps taken since the last (re)initialisation. */
long lbm_step_count(const lbm_ctx* ctx);

lbm_status lbm_destroy(lbm_ctx* ctx);            /* NULL-safe */
const char* lbm_last_error(void);

/* Batched stepping: contexts (same stream, any size/EOS/precision mix) are
 * advanced together, one fused launch per group of members sharing a
 * precision, launch shape and model class (lattices of 32768 nodes or more
 * with the heated-cavity model (Sutherland viscosity, F = rho g with
 * force[0] == 0, corrections on), ideal or cubic EOS, run a specialised
 * kernel instance, all others the generic one) and one wall-pass launch per
 * precision per step.  A lattice gives the same bits alone or batched.
 * graph_steps > 0 captures that many steps in a CUDA graph that
 * lbm_batch_step replays (nsteps must then be a multiple of graph_steps).
 * A member whose EOS class lbm_set_eos changes afterwards makes the batch
 * step fail with LBM_EINVAL: build the batch again. */
lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, int graph_steps, lbm_batch** out);

/* Add a context as the last member, or remove one (the others keep their
 * order; a removed context keeps its state and can be stepped alone or
 * batched again).  The launch tables and the graph are rebuilt, as
 * lbm_batch_create builds them; the batch handle stays valid and, if the
 * rebuild fails, unchanged.  Synchronises the batch stream.  LBM_EINVAL for
 * a context already in (add) or not in (remove) the batch, for one on
 * another stream, and for removing the last member.  The paper has no
 * counterpart: these serve requests that join and leave a running set of
 * lattices. */
lbm_status lbm_batch_add(lbm_batch* b, lbm_ctx* ctx);
lbm_status lbm_batch_remove(lbm_batch* b, lbm_ctx* ctx);
lbm_status lbm_batch_step(lbm_batch* b, long nsteps);
lbm_status lbm_batch_destroy(lbm_batch* b);     /* NULL-safe */

/* Same as lbm_batch_step without the graph, with CUDA events recorded on the
 * batch stream around each step's fused launches and wall-pass launches;
 * *ms_collide and *ms_wall receive their summed device times.  Synchronises. */
lbm_status lbm_batch_step_profiled(lbm_batch* b, long nsteps, double* ms_collide, double* ms_wall);

/* lbm_diagnostics for every member of a batch in one pass: one launch per
 * storage precision over all members, one copy back and one
 * synchronisation of the batch stream.  out8n (host, n x 8 doubles in the
 * member order given to lbm_batch_create) receives each member's eight
 * outputs as lbm_diagnostics defines them, bit for bit the values that
 * lbm_diagnostics would return; snapshot != 0 stores every member's
 * snapshot.  member_status (host, n entries, may be NULL) receives each
 * member's status: LBM_OK, or the sticky LBM_EUNSTABLE / LBM_ETIMEOUT /
 * LBM_ECUDA that lbm_diagnostics would return for it (its outputs are then
 * NaN if it was already sticky).  The call itself fails only on bad
 * arguments or a failed CUDA call.  The paper has no counterpart: it serves
 * the residual checks of the serving loop. */
lbm_status lbm_batch_diagnostics(lbm_batch* b, int snapshot, double* out8n, int* member_status);

/* lbm_init_macros for every member of a batch, and lbm_macros for every
 * member, each with one synchronisation of the batch stream: all host
 * copies and kernels of all members are enqueued first, so the copies run
 * back to back at the host link's rate instead of one stream round trip
 * per member.  The fields are those of lbm_init_macros (Eq. decompose at
 * the given rho, u, T with zero non-equilibrium part) and lbm_macros (Eqs.
 * rho.u, E; T = eps / Cv; p = p_EOS).
 *
 * Arguments are arrays of n host pointers (n members, in the member order
 * of lbm_batch_diagnostics: creation order, additions appended, removals
 * closing the gap), each pointing to a caller-owned FP64 host array
 * [ny][nx] (x fastest) of that member.  Pinned host memory gives the full
 * copy rate; pageable memory works but serialises the copies.
 *   lbm_batch_init_macros: rho, ux, uy, T must all be non-NULL and so must
 *   every entry; each member's sticky status is cleared, as
 *   lbm_init_macros clears it.  LBM_EINVAL before anything is enqueued
 *   when an entry is NULL.
 *   lbm_batch_macros: a NULL array skips that field for every member, a
 *   NULL entry skips it for one member.  member_status (host, n entries,
 *   may be NULL) receives each member's status as lbm_macros would return
 *   it (LBM_OK, or a sticky LBM_EUNSTABLE / LBM_ETIMEOUT / LBM_ECUDA); the
 *   call itself fails only on bad arguments or a failed CUDA call.  The
 *   first call allocates one status word per member on the device.
 * The paper has no counterpart: these move many problems' inputs and
 * results between host and device in one round trip. */
lbm_status lbm_batch_init_macros(lbm_batch* b, const double* const* rho, const double* const* ux,
                                 const double* const* uy, const double* const* T);
lbm_status lbm_batch_macros(lbm_batch* b, double* const* rho, double* const* ux, double* const* uy,
                            double* const* T, double* const* p, int* member_status);

/* Conserved sums of a context's current state, computed without allocating
 * anything.  The paper has no counterpart: this entry point is for callers
 * that may not allocate device memory, for example a host program that
 * only receives device buffers and a stream from another framework's
 * allocator, or code that runs where cudaMalloc is not permitted.
 *
 * out4 is a caller-owned device array of 4 doubles receiving, in FP64:
 *   out4[0] total mass sum(rho), out4[1] sum(j_x), out4[2] sum(j_y),
 *   out4[3] sum over nodes of sum_i g_i (the total energy minus half the
 *   source work, so equal to the total energy when F = 0).
 * Asynchronous on the context's stream; the context's device (the one
 * current at lbm_create) must be current, else LBM_EINVAL.
 *
 * Scratch: block partials go to a file-scope static device array of 2048 x 4
 * doubles (64 KiB) that every GPU loading the library holds until exit.
 * Lattices of more than 2048 x 32768 = 67,108,864 nodes are rejected with
 * LBM_EINVAL.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  No cudaMalloc, cudaFree or allocating library routine is called.
 * All calls share the one array and each call overwrites the slots it
 * reads, so calls that overlap on the GPU (on different streams, or from
 * several threads at once) race and must be serialised by the caller. */
lbm_status lbm_conserved_sums_static(const lbm_ctx* ctx, double* out4);

#ifdef __cplusplus
}
#endif
#endif
