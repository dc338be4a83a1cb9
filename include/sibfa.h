/*
 * sibfa.h -- C ABI of the GB300 SIBFA21 water energy/force library.
 *
 * One call evaluates the SIBFA intermolecular potential of a set of rigid or
 * flexible waters (Eq. 1: E_inter = E_elec+pen + E_rep + E_pol + E_ct +
 * E_disp,xdisp) and its analytic gradient.  The terms and where they are
 * defined:
 *   - multipolar electrostatics to quadrupoles with the charge-charge*,
 *     charge-dipole* and charge-quadrupole* penetration corrections (Eq. 2,
 *     section "Multipolar Electrostatics including Short-Range Penetration");
 *   - exchange-repulsion over bond-bond, bond-lone pair and lone pair-lone
 *     pair overlaps (Eq. 3 and Technical Appendix, exchange-repulsion);
 *   - many-body polarization, E_pol = 1/2 mu T mu - mu E solved by a
 *     preconditioned conjugate gradient on T mu = E (Technical Appendix,
 *     polarization; Computational Details);
 *   - the reduced many-body charge transfer (Eqs. 13-16);
 *   - C6/C8/C10 dispersion with exchange-dispersion (Technical Appendix);
 *   - periodic systems use smooth particle mesh Ewald of order 5 for the
 *     multipoles and the induced dipoles (Computational Details).
 * Units: kcal/mol, Angstrom, elementary charge; dipoles in e.A, tolerances
 * in Debye (4.80321 D per e.A).
 *
 * Memory and errors.  The library owns the context and every device buffer
 * it allocates at sibfa_create.  The caller owns all input and output
 * arrays; they may be host or device pointers (detected per call).  Device
 * pointers are read and written on the context's stream; page-locked host
 * memory (cudaMallocHost, cudaHostRegister) is copied to and from directly,
 * pageable host memory is staged through the context's pinned buffers, and
 * the call returns after the results are in host memory.  No call throws; every call returns a status
 * and sibfa_last_error() gives a one-line reason for the last failure.
 */
#ifndef SIBFA_H
#define SIBFA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SIBFA_OK = 0,
    SIBFA_E_INVALID = -1,        /* bad argument or inconsistent sizes          */
    SIBFA_E_OOM = -2,            /* device or host allocation failed            */
    SIBFA_E_NOT_CONVERGED = -3,  /* PCG hit max_iter above the tolerance        */
    SIBFA_E_CUTOFF = -4,         /* rc + 2 * site extent exceeds half the box   */
    SIBFA_E_CT_DENOM = -5,       /* a charge-transfer denominator dE <= 0       */
    SIBFA_E_TIMEOUT = -6,        /* reserved: no kernel of this library waits on
                                    another (grid-wide steps use cooperative
                                    launches), so no call returns it             */
    SIBFA_E_CUDA = -7,           /* a CUDA / cuFFT call failed                  */
    SIBFA_E_BUSY = -8,           /* admission refused (serving)                 */
    SIBFA_E_NEIGHBOR = -9        /* neighbour list overflow                     */
} sibfa_status;

/* Energy components (kcal/mol), in the order of Eq. 1; elec holds the
 * multipolar part, pen the penetration correction. */
typedef struct {
    double elec, pen, rep, disp, xdisp, pol, ct, total;
} sibfa_energy_terms;

/* Force-field parameters (all scalars; see synth/water.py for the values).
 * Layout is fixed; fields are read once at sibfa_create. */
typedef struct {
    double ke, debye;
    double d_lp, lp_half_deg;
    double alpha_o, alpha_h, alpha_m_damp, thole;
    double z_o, z_h, b_o, b_h;
    double cs_o, cp_o, cs_h, cp_h, cs_lp, cp_lp, g_o, g_h, nval_o, nval_h;
    double rvdw_rep_o, rvdw_rep_h, rvdw_rep_lp, rep_alpha, rep_alpha2, rep_c1, rep_c2, rep_f;
    double occ_bond, n_lp;
    double rvdw_disp_o, rvdw_disp_h, rvdw_disp_lp, disp_alpha, beta_o, beta_h;
    double c6, c8, c10, gamma6, gamma8, gamma10, disp_delta;
    double xd_c1, xd_a1, xd_c2, xd_a2, xd_c3, xd_a3;
    double ct_eta, ct_t, ct_m, ct_ae, ct_ah, rvdw_ct_o, rvdw_ct_h;
} sibfa_params;

/* Topology: n_mol waters; local-frame multipoles per molecule and site
 * (sites O, H1, H2, M1 = midpoint O-H1, M2 = midpoint O-H2), 10 doubles per
 * site: q, mu_x, mu_y, mu_z, Th_xx, Th_yy, Th_zz, Th_xy, Th_xz, Th_yz
 * (traceless, potential convention phi = q/r + mu.r/r^3 + Th:rr/r^5).
 * mp_local is a HOST pointer, n_mol*5*10 doubles, copied at create. */
typedef struct {
    int n_mol;
    const double *mp_local;
    /* Optional batch of independent gas-phase clusters (periodic = 0 only).
     * n_clusters > 1 splits the molecules into consecutive clusters: cluster
     * c holds molecules cluster_start[c] .. cluster_start[c+1]-1 (HOST
     * pointer, n_clusters+1 ints, cluster_start[0] = 0, cluster_start
     * [n_clusters] = n_mol, increasing; copied at create).  Molecules of
     * different clusters do not interact; each call evaluates every cluster
     * with one launch per kernel, the polarization solve stops when the RMS
     * residual of every cluster is below pcg_tol_D, sibfa_cluster_terms
     * returns the terms per cluster and the terms of sibfa_energy_forces are
     * their sums.  n_clusters = 0 or 1: one system (cluster_start unused). */
    int n_clusters;
    const int *cluster_start;
} sibfa_topology;

enum { SIBFA_PREC_FP64 = 0, SIBFA_PREC_MIXED = 1 };

/* Run options.  periodic = 0: gas phase, all pairs, no cutoff, no Ewald.
 * periodic = 1: orthorhombic box, minimum image, real-space cutoff rc,
 * SPME grid[3] of B-spline order 5 with Ewald parameter ewald_alpha.
 * precision: SIBFA_PREC_FP64 (all FP64) or SIBFA_PREC_MIXED (FP32 pair and
 * grid arithmetic, FP64 accumulation across pairs, FP64 PCG scalars,
 * energies and influence function).  stream: a cudaStream_t or NULL for the
 * legacy default stream; each call is ordered after the work queued on it
 * and the work queued on it afterwards waits for the call's results.  Inside,
 * the context runs four streams of its own (main; reciprocal space, highest
 * priority; short-range terms, lowest; lone-pair potentials and charge
 * transfer), forked from and joined back into the main one within the call.
 * warm_start: the PCG initial guess.  0: the direct-field dipoles alpha E.
 * 1: the dipoles of the previous solve.  2..6: the polynomial through the
 * converged dipoles of the last warm_start full evaluations (energy and
 * forces, equally spaced in time as in an MD run), extrapolated one step
 * ahead (linear, quadratic, cubic, quartic, quintic: coefficients
 * (-1)^(j+1) C(n, j) for the j-th newest of n); with fewer stored it uses as many as it
 * has; a dipole-only solve neither uses nor feeds that history, and
 * sibfa_minimize clears it when it returns.  Every
 * choice converges to the same tolerance; only the iteration count differs.
 * Other values: SIBFA_E_INVALID. */
typedef struct {
    int periodic;
    double box[3];
    double rc;
    int grid[3];
    int order;
    double ewald_alpha;
    double pcg_tol_D;
    int pcg_max_iter;
    int precision;
    int warm_start;
    void *stream;
    /* Intramolecular support potential used only by sibfa_md_steps (not
     * part of the reported intermolecular energy): E = k_bond (r - r0)^2
     * per O-H bond + k_angle (theta - theta0)^2 per H-O-H angle
     * (kcal/mol, A, rad; theta0 in degrees).  k = 0 switches a term off. */
    double md_k_bond, md_r0, md_k_angle, md_theta0_deg;
    /* Long-range dispersion (periodic only; 0 = off): 1 adds the dispersion
     * beyond rc for a homogeneous fluid (pair distribution 1 past the
     * cutoff; the C6/C8/C10 pair function of the Technical Appendix
     * integrated from rc to infinity, 2 pi M (M-1)/V times the sum over the
     * point types) to the dispersion energy and total of every call, and
     * E_tail on the diagonal of the virial (it scales as 1/V).  Forces do
     * not change: the term depends on the volume only. */
    int disp_tail;
    /* Integrator of sibfa_md_steps: 0 velocity Verlet, 1 Beeman (the
     * paper's MD setting, Computational Details):
     *   x(t+dt) = x + v dt + (4 a(t) - a(t-dt)) dt^2 / 6,
     *   v(t+dt) = v + (2 a(t+dt) + 5 a(t) - a(t-dt)) dt / 6,
     * with a(t-dt) = a(t) on the first step of a context. */
    int md_integrator;
    /* Anharmonic (MM3-style) corrections to the support potential, 0 = off:
     * bond  k_bond dr^2 (1 - 2.55 dr + (7/12) 2.55^2 dr^2)            (dr in A)
     * angle k_angle dth^2 (1 - 0.014 D + 5.6e-5 D^2 - 7e-7 D^3 + 9e-10 D^4)
     *       (dth in rad, D the same deviation in degrees),
     * plus a Urey-Bradley H-H term md_k_ub (r_HH - md_r_ub)^2 when
     * md_k_ub > 0 (the paper's flexible water: MM3 bond and angle terms with
     * a Urey-Bradley term). */
    int md_anharmonic;
    double md_k_ub, md_r_ub;
    /* Charge transfer form, 0 = the reduced one of Eqs. 13-16.  1 = the
     * original many-body form (CT section, before its reduction): the
     * acceptor atoms' potentials are kept,
     *   e1 = exp(-eta rho1) (V_int(a1) + V*(a1) - V_lp)(Cs t + Cp m cos alpha),
     *   e2 = exp(-eta rho2) (V_int(a2) + V*(a2) - V_lp)(Cs t + Cp m cos beta),
     *   dE = ae + V_lp - (ah + V(a1)),
     * with V(a) the potential of the permanent multipoles of every molecule
     * but a's own at acceptor atom a (undamped, full Ewald in a box) and
     * V*(a) = V(a) minus the donor molecule's part (its five sites, bare,
     * at the pair's image).  Forces include the dependence through V(a)
     * (point charges dE/dV(a) on the acceptor atoms) and through the
     * donor's multipoles in V*.  The virial is not available with it
     * (SIBFA_E_INVALID when requested). */
    int ct_original;
} sibfa_run_opts;

typedef struct sibfa_ctx sibfa_ctx;

/* Create a context: validates sizes, copies the topology, builds the SPME
 * influence function and FFT plans, allocates all device state.  *out is
 * NULL on failure.  The PCG loop normally runs on the device as a CUDA graph
 * with a conditional while-node; with the environment variable
 * SIBFA_PCG_HOST_LOOP=1 at creation it is driven from the host instead (one
 * launch per kernel and iteration, same arithmetic), which kernel profilers
 * can follow.  The context tunes the schedule of its short-range kernels
 * (resident blocks per SM, and whether they finish before the polarization
 * solve; see sibfa_tuned_schedule) over its first full evaluations outside
 * sibfa_minimize by timing them and then keeps the fastest; the choice
 * affects scheduling only, never the results.  SIBFA_TUNE=0 at creation
 * turns the tuning off (fixed shape). */
sibfa_status sibfa_create(const sibfa_params *params, const sibfa_topology *topo,
                          const sibfa_run_opts *opts, sibfa_ctx **out);

/* One energy + force evaluation.  pos: n_mol*9 doubles (O, H1, H2 xyz per
 * molecule, Angstrom).  box: 3 doubles (host) or NULL to keep the current
 * box.  A box that differs from the context's current one changes it, for
 * this and every later call (constant-pressure MD; periodic contexts only,
 * SIBFA_E_INVALID for a gas-phase context): the influence function is
 * recomputed, the neighbour list rebuilt and the dispersion tail rescaled.
 * Returns SIBFA_E_INVALID for a non-positive edge or when the new box needs
 * more cells than the context allocated at create (a box much larger than
 * the first), SIBFA_E_CUTOFF when rc + 2 * O-H distance exceeds half the
 * new box; the box is then unchanged.
 * e: host struct, filled on success (may be NULL).  forces: n_mol*9 doubles
 * (kcal/mol/A, = -dE/dx) or NULL.  virial: 9 host doubles (row-major 3x3,
 * kcal/mol) or NULL: W_ab = -dE/d eps_ab for the affine strain x -> (I + eps) x
 * applied to every atom and to the periodic cell, the quantity a barostat
 * needs (pressure tensor P = (sum m v v + W) / V); in the gas phase it
 * equals sum over atoms of F_a x_b.  It is a sum of pair terms (real space),
 * the reciprocal-space strain derivative (k-space sums and the k-dependence of
 * the multipole structure factor) and the frame terms of the rotating
 * multipoles and lone pairs; a cluster batch returns the sum over clusters.
 * Requesting it runs the force pass and selects kernel variants that also
 * accumulate it. */
sibfa_status sibfa_energy_forces(sibfa_ctx *ctx, const double *pos, const double *box,
                                 sibfa_energy_terms *e, double *forces, double *virial);

/* Solve T mu = E only (sites, permanent field, PCG).  mu: n_mol*9 doubles
 * (induced dipoles on O, H1, H2, e.A) or NULL.  tol_D <= 0 uses the run
 * option.  iters / resid_D may be NULL. */
sibfa_status sibfa_solve_dipoles(sibfa_ctx *ctx, const double *pos, const double *box,
                                 double tol_D, double *mu, int *iters, double *resid_D);

/* NVE steps on the device (velocity Verlet or Beeman, see run options;
 * support for the MD workloads):
 * pos and vel (n_mol*9 doubles, A and A/fs) are updated in place; masses
 * n_mol*3 doubles (amu).  Each step is one full energy + force evaluation.
 * e (may be NULL) receives the energy of the last step. */
sibfa_status sibfa_md_steps(sibfa_ctx *ctx, double *pos, double *vel, const double *masses,
                            double dt_fs, int n_steps, sibfa_energy_terms *e);

/* Relax a starting structure by capped steepest descent on the
 * intermolecular energy plus the intramolecular support potential:
 * each atom moves by F * min(1e-4 A^2 mol/kcal, max_disp_A / |F|) per step.
 * pos: device pointer, n_mol*9 doubles, updated in place.  e (may be NULL)
 * receives the intermolecular energy before the last step. */
sibfa_status sibfa_minimize(sibfa_ctx *ctx, double *pos, int n_steps, double max_disp_A, sibfa_energy_terms *e);

/* Statistics of the last evaluation: PCG iterations and final residual (D;
 * for a cluster batch, the largest per-cluster residual). */
sibfa_status sibfa_last_stats(const sibfa_ctx *ctx, int *pcg_iters, double *pcg_resid_D);

/* Energy terms per cluster of the last evaluation (cluster batches; one
 * entry for a single system).  terms: HOST pointer, n_clusters entries. */
sibfa_status sibfa_cluster_terms(sibfa_ctx *ctx, sibfa_energy_terms *terms);

/* Number of the library's own kernel launches since the context was created
 * (cuFFT executions are not counted). */
uint64_t sibfa_kernel_launches(const sibfa_ctx *ctx);

/* Launch shape of the short-range kernels chosen by the context's tuning:
 * *blocks_per_sm = resident blocks per SM (0 = uncapped), *done = 1 once the
 * tuning has fixed it (0 while candidates are still being timed).  Either
 * pointer may be NULL.  Returns SIBFA_E_INVALID for a NULL context. */
sibfa_status sibfa_tuned_shape(const sibfa_ctx *ctx, int *blocks_per_sm, int *done);

/* The whole short-range schedule chosen by the tuning.  The candidates, in
 * order: (blocks per SM, joined before the solve) = (3, no), (0, no),
 * (2, no), (0, yes), (3, yes); "joined before the solve" means the
 * short-range kernels finish before the polarization solve starts (the
 * solve's latency-bound kernels then have the SMs to themselves), otherwise
 * they run beside it until the chain rule.  *blocks_per_sm, *join_before_solve
 * (0/1) and *done as for sibfa_tuned_shape; cand_ms (HOST, n_cand entries,
 * may be NULL) receives each candidate's fastest timed evaluation in ms (0
 * for a candidate not timed, or beyond the 5 candidates).  Any output may be
 * NULL.  Returns SIBFA_E_INVALID for a NULL context or n_cand < 0. */
sibfa_status sibfa_tuned_schedule(const sibfa_ctx *ctx, int *blocks_per_sm, int *join_before_solve, int *done,
                                  double *cand_ms, int n_cand);

/* Optional phase timing with CUDA events recorded on the context stream
 * around each phase of an evaluation: "sites", "neighbors", "real_perm"
 * (permanent electrostatics + penetration + Thole field + lone-pair
 * potential), "short" (repulsion, dispersion), "spme_perm", "ct", "pcg"
 * (whole solve), "real_tmu" (real-space part of each T.mu product),
 * "real_polforce", "spme_polforce", "finalize".  sibfa_profile_get returns
 * the summed milliseconds and the number of spans of one phase recorded
 * since the last get/clear of that phase, and synchronizes the stream.
 * on = 1: the phases keep their usual overlap on the context's streams, so a
 * span on a low-priority stream includes the time it waited for SMs.
 * on = 2: serial profiling: every phase runs alone on the GPU (the streams
 * join after each reciprocal-space chain, and the short-range and
 * charge-transfer kernels run in order on the main stream), so each span is
 * the duration of that phase's kernels alone.  The solve keeps its device
 * loop (real and reciprocal parts of each product concurrent, as captured);
 * "real_tmu" then times the first product's real-space part alone.  Results agree
 * with on = 0 or 1 up to the order of floating-point sums.  on = 0: off. */
void sibfa_set_profiling(sibfa_ctx *ctx, int on);
sibfa_status sibfa_profile_get(sibfa_ctx *ctx, const char *name, double *ms, int *count);
void sibfa_profile_clear(sibfa_ctx *ctx);

/* Allocation-free electrostatics of a gas-phase cluster.  (The paper has no
 * counterpart: this entry point exists for callers that cannot allocate.)
 *
 * Some callers must not allocate device memory during a step: code running
 * under a memory pool or arena that owns all device memory, and plugins of
 * host MD engines that forbid cudaMalloc/cudaFree inside their force
 * callback (an allocation can synchronize the device and stall other
 * streams).  This call computes, on `stream`, the same multipole (elec) and
 * penetration (pen) energies that sibfa_energy_forces reports for a
 * gas-phase cluster, using only a fixed file-scope device array as scratch
 * (about 270 KB, held by every GPU that loads the library until the process
 * exits).
 *
 * n_mol: 1..512 waters (larger clusters are rejected with SIBFA_E_INVALID).
 * pos: DEVICE pointer, n_mol*9 doubles (O, H1, H2).  mp_local: DEVICE
 * pointer, n_mol*5*10 doubles (local-frame multipoles as in sibfa_topology).
 * elec_pen: DEVICE pointer to 2 doubles receiving elec and pen (kcal/mol).
 * The three must be device or managed memory of the current device
 * (checked with cudaPointerGetAttributes, which allocates nothing; anything
 * else returns SIBFA_E_INVALID before any launch); their lengths cannot be
 * checked through plain pointers and are the caller's responsibility.
 * params: host struct.  The call is asynchronous on `stream` and does not
 * synchronize.  The first call on each device looks up the scratch array's
 * device address with that device current and keeps it until the process
 * exits; make that first call before any stream capture, and do not use the
 * call after cudaDeviceReset on that device (the kept address would be
 * stale).  All calls on a device share the scratch array: calls whose
 * kernels overlap on the GPU (different streams, no ordering) race.  Errors
 * are described by sibfa_noalloc_last_error(). */
sibfa_status sibfa_cluster_elec_noalloc(const sibfa_params *params, int n_mol, const double *pos,
                                        const double *mp_local, double *elec_pen, void *stream);
const char *sibfa_noalloc_last_error(void);

/* CUDA-core arithmetic peak of the current device (a measurement utility;
 * the paper has no counterpart).  Runs `blocks` blocks of 256 threads, each
 * thread `iters` x 128 fused multiply-adds on 8 independent chains, FP32
 * (fp64 = 0) or FP64 (fp64 = 1), on the legacy default stream after one
 * shorter warm-up launch, and returns the CUDA-event time of the timed
 * launch (*ms) and its flop count (*flops, an FMA counted as 2).  The ratio
 * is the device's FMA rate at the clock it ran at; the pair kernels' roofline
 * is measured against it.  Allocates and frees a small device buffer;
 * synchronizes the device.  Errors: sibfa_alu_peak_error(). */
sibfa_status sibfa_alu_peak(int fp64, int iters, int blocks, double *ms, double *flops);
const char *sibfa_alu_peak_error(void);

/* The library's FP32 elementary kernels beside CUDA's functions, for tests
 * that hold them to an error bound (test support; the paper has no
 * counterpart).  x, out: DEVICE float arrays; asynchronous on `stream`.
 *   fn 0: out[2k] = the Newton-refined reciprocal square root of x[k] used by
 *         the pair kernels, out[2k+1] = rsqrtf(x[k]);
 *   fn 1: out[2k] = the Newton-refined reciprocal of x[k], out[2k+1] =
 *         1.0f / x[k] (IEEE division);
 *   fn 2: x[k] = r; out[5k..5k+3] = the radial kernels g_0..g_3 of
 *         erf(alpha r)/r (g_{n+1} = (1/r) dg_n/dr) used by the intramolecular
 *         Ewald exclusions, out[5k+4] = erff(alpha r) / r.
 * out holds 2n (fn 0, 1) or 5n (fn 2) floats.  SIBFA_E_INVALID for another
 * fn or null arrays. */
sibfa_status sibfa_math_selftest(int fn, int n, const float *x, float alpha, float *out, void *stream);

void sibfa_destroy(sibfa_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Serving: a request loop for energy/force jobs that arrive over time.
 *
 * Jobs are MD runs (n_steps velocity-Verlet steps; n_steps = 0 is one energy
 * and force evaluation) of a periodic water box or a gas-phase cluster.
 * Box jobs run in `slots` concurrent workers, each with its own stream and up
 * to four contexts of distinct shapes kept between jobs of those shapes.  Gas-phase clusters of at most
 * `batch_max_cluster` waters are batched continuously: one resident batch
 * context advances every admitted cluster by one step per tick, finished jobs
 * leave and newly arrived ones join at the next tick, and each cluster keeps
 * its induced dipoles on the device as the warm start of its next solve.
 * Jobs are admitted while the device memory they need (estimated from their
 * size) fits under `device_mem_bytes`; the others wait in the queue.
 * The scheme follows the serving form of the hot path; the paper itself has
 * no request loop.
 * ------------------------------------------------------------------------- */
typedef struct sibfa_server sibfa_server;

typedef struct {
    const sibfa_params *params;  /* force-field parameters (copied)                       */
    int slots;                   /* concurrent box workers, >= 1                           */
    size_t device_mem_bytes;     /* admission cap on the server's device memory            */
    int max_pending;             /* queued jobs beyond which sibfa_submit returns BUSY     */
    int batch_waters;            /* capacity of the cluster batch (waters); 0 = no batch   */
    int batch_max_cluster;       /* largest cluster that joins the batch (<= 385)          */
    double batch_dt_fs;          /* time step of batched cluster jobs (fs)                 */
    int precision;               /* SIBFA_PREC_MIXED or SIBFA_PREC_FP64                    */
    double pcg_tol_D;            /* PCG tolerance of every job (D)                         */
} sibfa_server_opts;

typedef struct {
    int n_mol;
    const double *pos;           /* HOST n_mol*9 (A), copied at submit                    */
    const double *vel;           /* HOST n_mol*9 (A/fs) or NULL (zero), copied             */
    const double *mp_local;      /* HOST n_mol*50 local multipoles, copied                 */
    int periodic;                /* 1: box job (box, rc, grid, ewald_alpha used)           */
    double box[3];
    double rc;
    int grid[3];
    double ewald_alpha;
    int n_steps;                 /* velocity-Verlet steps; 0: one evaluation               */
    double dt_fs;                /* time step (a batched cluster uses batch_dt_fs)         */
} sibfa_job;

typedef struct {
    sibfa_energy_terms terms;    /* intermolecular terms at the final positions (kcal/mol) */
    double *forces;              /* HOST n_mol*9 or NULL: filled by sibfa_poll; MD jobs:   */
                                 /* the integrator's forces (with the intramolecular        */
                                 /* support potential), evaluations: intermolecular         */
    double *pos;                 /* HOST n_mol*9 or NULL: final positions                  */
    int status;                  /* sibfa_status of the job                                */
    int pcg_iters;               /* iterations of the last solve                           */
    double queue_ms;             /* submit -> start of the job on the device               */
    double latency_ms;           /* submit -> completion                                   */
    int batched;                 /* 1 if the job ran in the cluster batch                  */
} sibfa_result;

/* Create a server on the current device; worker threads start at once. */
sibfa_status sibfa_server_create(const sibfa_server_opts *opts, sibfa_server **out);

/* Queue a job (its arrays are copied before the call returns) and return its
 * ticket.  SIBFA_E_BUSY: max_pending jobs already wait; SIBFA_E_INVALID: bad
 * sizes or a job that can never fit the memory cap.  Never blocks on the GPU. */
sibfa_status sibfa_submit(sibfa_server *srv, const sibfa_job *job, uint64_t *ticket);

/* *done = 1 when the job has finished: out receives its result (forces and
 * positions copied to the caller's buffers when non-NULL) and the ticket is
 * released; *done = 0 while it waits or runs.  Unknown ticket: INVALID. */
sibfa_status sibfa_poll(sibfa_server *srv, uint64_t ticket, sibfa_result *out, int *done);

/* Stop accepting jobs, finish the running ones, free everything. */
void sibfa_server_destroy(sibfa_server *srv);


/* Text of the last error on this context (or of the last failed create when
 * ctx is NULL).  Never NULL. */
const char *sibfa_last_error(const sibfa_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SIBFA_H */
