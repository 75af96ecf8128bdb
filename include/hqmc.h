/*
 * hqmc.h - C ABI of the GB300 hybrid quantum Monte Carlo hot path.
 *
 * The library applies the fermion matrix of a compact (or non-compact) U(1)
 * gauge field theta on the spatial bonds of an L x L x Ntau lattice coupled to
 * fermions, solves (M^dagger M) X = phi by conjugate gradients, computes the
 * pseudofermion force and runs leapfrog / Metropolis HMC trajectories, all in
 * CUDA kernels for sm_103a (arXiv 2508.16298, Methods and Supplement SI).
 *
 * Layouts (all arrays contiguous, caller-owned DEVICE memory unless stated):
 *   theta, p, F : double[Ntau][L][L][2]; index [tau][y][x][c], c = 0 the bond
 *                 (x,y)->(x+1,y), c = 1 the bond (x,y)->(x,y+1); periodic in x, y.
 *   vectors     : complex[Ntau][L][L], interleaved (re, im); complex double
 *                 (16 B) for HQMC_FP64, complex float (8 B) for HQMC_FP32.
 *   0-based slices: slice tau carries the paper's B_{tau+1}.
 * Every pointer must be 16-byte aligned.  Arrays must not overlap unless a
 * function says otherwise.  Scalars returned through *_info structs are host
 * memory owned by the caller.
 *
 * Stream semantics: every call is ordered on `stream` (a cudaStream_t passed
 * as void*; NULL is the legacy default stream).  Functions that return
 * host-side results (solve and trajectory info) synchronise that stream
 * before returning; the others only enqueue work.
 *
 * Errors: every function returns an hqmc_status.  No C++ exception crosses
 * the ABI.  After HQMC_ECUDA the CUDA error text is in hqmc_last_error(cfg).
 * The config is single-threaded: calls on one config must not run
 * concurrently from several host threads.
 */
#ifndef HQMC_H
#define HQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HQMC_API __attribute__((visibility("default")))
#else
#define HQMC_API
#endif

typedef enum {
    HQMC_OK = 0,
    HQMC_EINVAL = 1,       /* bad parameter: odd or too large L, Ntau < 2, NULL or misaligned pointer */
    HQMC_ENOTCONV = 2,     /* CG used up maxit; x holds the last iterate, info the true residual */
    HQMC_EBREAKDOWN = 3,   /* CG met <d, O d> <= 0 */
    HQMC_ENONFINITE = 4,   /* a NaN or Inf reached a CG reduction or the Hamiltonian */
    HQMC_ETIMEOUT = 5,     /* a bounded device-side wait (about 1 s) gave up: the kernel wrote NaN
                              into its outputs and set the config's error word; the next solve
                              (hqmc_cg_solve, hqmc_leapfrog, hqmc_trajectory, hqmc_estimate)
                              returns this code and clears the word */
    HQMC_ECUDA = 6,        /* a CUDA runtime call failed (text in hqmc_last_error) */
    HQMC_ENOMEM = 7,       /* workspace allocation failed (hqmc_make_config, hqmc_make_batch,
                              hqmc_net_create, hqmc_set_preconditioner) */
    HQMC_EUNSUPPORTED = 8, /* option not available for these sizes or this device */
    HQMC_EIO = 9           /* checkpoint file missing, unwritable, truncated or corrupted */
} hqmc_status;

enum { HQMC_FP64 = 0, HQMC_FP32 = 1 };
enum { HQMC_ACTION_COMPACT = 0, HQMC_ACTION_NONCOMPACT = 1 };

/* Solver selection for hqmc_cg_solve / hqmc_leapfrog / hqmc_trajectory. */
enum {
    HQMC_SOLVER_CG64 = 0,    /* plain CG, every vector and reduction in FP64 */
    HQMC_SOLVER_MIXED = 1,   /* CG with M^dagger M in FP32 (complex float) and FP64 reliable
                                residual updates every params.reliable_interval iterations */
    HQMC_SOLVER_LEARNED = 2, /* the attached net (hqmc_set_preconditioner) corrects the initial
                                guess, x <- x + z with z = K(theta) r0, r0 = phi - O x, kept only if
                                ||r0 - O z|| < ||r0|| (both from the FP32 apply: they only decide);
                                then the mixed solver, whose FP64 true residual judges convergence.
                                Inside hqmc_leapfrog / hqmc_trajectory with the chronological guess
                                (hqmc_set_guess_history), the net is not tried again in that
                                integration after two consecutive tries that did not cut the
                                residual norm at least in half (kept or not) */
    /* The same three with the tau-line preconditioner Otilde^{-1} of hqmc_apply_precond in the
     * preconditioned CG of Methods Eq. (pCG): directions from z = Otilde^{-1} r, step lengths
     * from <r, z>; convergence is still judged on ||r|| and the FP64 true residual. */
    HQMC_SOLVER_PCG64 = 3,
    HQMC_SOLVER_PMIXED = 4,
    HQMC_SOLVER_PLEARNED = 5,
    /* Flexible CG (Notay 2000) with one kept direction, i.e. the Polak-Ribiere
     * beta_k = Re<z_k, r_k - r_{k-1}> / Re<z_{k-1}, r_{k-1}>, which stays valid
     * when the preconditioner changes from one iteration to the next: z = K(theta) r
     * from the attached net on iterations c with c % net_interval == 0 of every
     * reliable_interval-long segment (hqmc_set_net_interval; default 1, every
     * iteration) and z = Otilde^{-1} r (tau-line) on the others.  FP32 recurrence
     * with FP64 reliable updates, after the learned initial guess of
     * HQMC_SOLVER_LEARNED.  If the net makes Re<r, z> or <p, O p> non-positive or
     * stalls the recurrence, the solve continues as HQMC_SOLVER_PMIXED from the
     * current x (info.fcg_fallback = 1).  The FP64 true residual judges
     * convergence.  Not a method of the paper (spec extension). */
    HQMC_SOLVER_FLEARNED = 6
};

/* Model and lattice (Results "Model"; Methods "Model and partition function"). */
typedef struct hqmc_params {
    int L;                 /* spatial extent: even, 4 <= L <= 68 (FP64 path limit) */
    int Ntau;              /* number of imaginary-time slices, >= 2 */
    double dtau;           /* Trotter step Delta tau (> 0); the paper uses 0.1 */
    double t;              /* hopping amplitude (the paper's energy unit, 1) */
    double J;              /* gauge coupling (> 0) */
    double K;              /* plaquette coupling (0 in the compact runs here) */
    int action;            /* HQMC_ACTION_COMPACT or HQMC_ACTION_NONCOMPACT */
    int reliable_interval; /* mixed solver: FP64 residual update period; <= 0 means 50 */
    int autotune;          /* 1: time every admissible launch shape of the fused M^dagger M in
                              hqmc_make_config and keep the fastest; 0: built-in choice */
    int variant;           /* fused M^dagger M kernel: 0 any, 1 generic only, 2 register-blocked
                              only (HQMC_EUNSUPPORTED if no strip shape fits L), 3 FP32 on the
                              persistent tau-walking kernel (HQMC_EUNSUPPORTED if it does not fit
                              L; FP64 as for 0) */
} hqmc_params;

/* Opaque configuration: geometry, launch shapes and the device workspace
 * (CG vectors, link tables, reduction partials).  It is bound to the device
 * that was current in hqmc_make_config; use it only with that device current. */
typedef struct hqmc_config hqmc_config;

typedef struct hqmc_solve_info {
    int status;                /* hqmc_status of the solve */
    int iterations;            /* applications of M^dagger M to a search direction */
    int restarts;              /* mixed solver: restarts after an FP32 breakdown or stall */
    int reliable_updates;      /* mixed solver: FP64 residual recomputations */
    double true_residual;      /* ||phi - (M^dagger M) x|| / ||phi||, computed in FP64 */
    double recursive_residual; /* the recurrence's estimate at exit */
    int fp64_fallback;         /* mixed solver: 1 if FP32 breakdowns, or a true residual cut
                                  by less than 2x over eight reliable updates, handed the
                                  rest of the solve to the FP64 recurrence */
    int net_guess_used;        /* learned solver: 1 if the net's correction of the initial
                                  guess lowered the residual and was kept */
    int fcg_fallback;          /* flexible CG: 1 if it handed the solve to HQMC_SOLVER_PMIXED */
} hqmc_solve_info;

typedef struct hqmc_traj_info {
    int status;            /* worst hqmc_status of the solves in the trajectory */
    int accepted;          /* 1 if the Metropolis test accepted the end point */
    int cg_solves;         /* number of CG solves (nsteps + 1) */
    int cg_iterations;     /* total CG iterations */
    double H0, H1, dH;     /* Hamiltonian at start and end, dH = H1 - H0 */
    double u;              /* the uniform number used by the Metropolis test */
    double max_true_residual;
    int net_guesses_tried; /* learned solvers: solves that applied the net to their initial residual */
    int net_guesses_used;  /* ... and kept its correction */
} hqmc_traj_info;

/* ---- configuration ----------------------------------------------------- */

/* Validates *p, chooses launch shapes for the current device and allocates
 * the workspace.  On a config, device memory is allocated only here and, for
 * the learned net's activation fields, in hqmc_set_preconditioner and, for the
 * chronological guess, in hqmc_set_guess_history; no apply, solve, force,
 * leapfrog, trajectory or net call allocates.
 * *out receives the config; free it with hqmc_free_config.
 * Errors: HQMC_EINVAL (parameters), HQMC_EUNSUPPORTED (device is not
 * compute capability 10.x, the sm_103a build's family), HQMC_ENOMEM, HQMC_ECUDA. */
HQMC_API int hqmc_make_config(const hqmc_params* p, hqmc_config** out);

/* Releases the workspace.  NULL is accepted.  Waits for the device. */
HQMC_API int hqmc_free_config(hqmc_config* cfg);

/* Static description of a status code. */
HQMC_API const char* hqmc_strerror(int status);

/* Detail text of the last error on this config ("" if none). */
HQMC_API const char* hqmc_last_error(const hqmc_config* cfg);

/* Number of lattice sites Ntau*L*L of the config (host query, no device work). */
HQMC_API long long hqmc_num_sites(const hqmc_config* cfg);

/* Number of CUDA kernels this config has enqueued since it was made (host
 * counter; no device work).  Differences around a region count its launches. */
HQMC_API long long hqmc_launch_count(const hqmc_config* cfg);

/* Launch shape of the fused M^dagger M for one precision (host query):
 * *variant >= 100: persistent tau-walking kernel (FP32) with strips of
 * *variant - 100 2x2 blocks, one contiguous range of slices per CTA;
 * 0 < *variant < 100: register-blocked kernel with strips of *variant 2x2 blocks;
 * *variant <= 0: generic kernel holding -*variant bonds per family in registers
 * (0: links re-read from memory).  *cluster: CTAs (slices) per cluster;
 * *threads: block size; *tuned_us: autotuner's time of one apply (0 if not
 * tuned).  Any output may be NULL. */
HQMC_API int hqmc_get_launch_shape(const hqmc_config* cfg, int precision, int* variant, int* cluster,
                                   int* threads, float* tuned_us);

/* ---- operators (Methods, Eq. (M_alpha) and the checkerboard Eq. (eq24)) -- */

/* y = M x (dagger = 0) or y = M^dagger x (dagger = 1), where
 * (M x)_tau = x_tau - B_{tau-1} x_{tau-1} for tau >= 1 and
 * (M x)_0 = x_0 + B_{Ntau-1} x_{Ntau-1}, and B_tau is the symmetric checkerboard
 * product e^{V4/2} e^{V3/2} e^{V2/2} e^{V1} e^{V2/2} e^{V3/2} e^{V4/2} of 2x2 bond
 * exponentials [[cosh a, e^{i theta} sinh a], [e^{-i theta} sinh a, cosh a]] with
 * a = dtau*t (halved for families 2-4).  precision: HQMC_FP64 (x, y complex
 * double) or HQMC_FP32 (complex float).  theta is always double.  x and y
 * must not overlap. */
HQMC_API int hqmc_apply_M(hqmc_config* cfg, const double* theta, const void* x, void* y,
                 int dagger, int precision, void* stream);

/* y = (M^dagger M) x in one fused kernel (Methods, "Matrix-free representation
 * of M^dagger M v"):  y_tau = x_tau + B_tau^2 x_tau - s_tau B_{tau-1} x_{tau-1}
 * - s'_tau B_tau x_{tau+1} with s_0 = -1, s'_{Ntau-1} = -1, else +1. */
HQMC_API int hqmc_apply_MdagM(hqmc_config* cfg, const double* theta, const void* x, void* y,
                     int precision, void* stream);

/* Tau-line preconditioner (Methods, "CG method and preconditioner").  It is built
 * once per config from O = M^dagger M at the pi-flux field (theta_y(x,y) = pi (x mod 2),
 * theta_x = 0), where every site is equivalent.  The same-site part of O there is the
 * tau-line matrix T = a - b (S + S^dagger), with a = 1 + sum_j |B_js|^2, b = B_ss and
 * S the antiperiodic tau shift.  Its bulk Cholesky factor is
 * L = sqrt(b/rho)(1 - rho S) with rho + 1/rho = a/b.  The Neumann series of L^{-1}
 * keeps the entries sqrt(rho/b) rho^m >= 1e-3 (m <= W), so on every site's tau line
 *     z = Otilde^{-1} r = (rho/b) F_W^dagger F_W r,   F_W = sum_{m=0}^{W} rho^m S^m,
 * which is Hermitian positive definite.
 *   r, z: device vectors (complex double for HQMC_FP64, complex float for HQMC_FP32),
 *   16-byte aligned, not overlapping.  The call uses config workspace (the FP64 or
 *   FP32 CG direction buffer) and is stream-ordered like every other call. */
HQMC_API int hqmc_apply_precond(hqmc_config* cfg, const void* r, void* z, int precision, void* stream);

/* The preconditioner's coefficients (host query): a, b, rho and W as above.  Any
 * output may be NULL. */
HQMC_API int hqmc_get_precond(const hqmc_config* cfg, double* a, double* b, double* rho, int* W);

/* Launch shape of the tau-line preconditioner (Methods, "CG method and
 * preconditioner") for one precision, a host query with no device work: slices
 * per tile of the separate kernel (*tile_slices; chosen per config, for FP32
 * timed by the autotuner when it runs) and whether preconditioned CG fuses the
 * vector update with the preconditioner (*fused, 0 or 1; the autotuner's
 * choice, 0 under variant 1).  Any output may be NULL.  Returns HQMC_EINVAL for
 * a NULL cfg or a precision other than HQMC_FP64 / HQMC_FP32. */
HQMC_API int hqmc_get_precond_shape(const hqmc_config* cfg, int precision, int* tile_slices, int* fused);

/* Overrides the autotuner's choice between the fused and the separate vector
 * update of preconditioned CG for one precision (fused: 1 or 0), e.g. to check
 * both forms on one lattice.  Host-only; takes effect at the next solve.
 * Returns HQMC_EINVAL for a NULL cfg, a bad precision or fused not 0/1, and
 * HQMC_EUNSUPPORTED for fused = 1 on a variant-1 config (generic kernels only). */
HQMC_API int hqmc_set_precond_fused(hqmc_config* cfg, int precision, int fused);

/* y = (M^dagger M) x in FP64 without a config and without allocating device
 * memory (HQMC_EUNSUPPORTED on a device that is not compute capability 10.x;
 * HQMC_EINVAL for a non-finite or non-positive dtau * t).  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate, such as code running while another component owns the
 * device allocator (a memory pool that must not be bypassed, or a budget that is
 * already handed out), plug-ins that are only given device pointers, or code
 * that must not let cudaMalloc/cudaFree synchronise the device.  The fused
 * apply's only scratch, the gauge field's FP64 link table, lives in a
 * fixed-size device array that every device loading the library holds until
 * the process exits.
 *   p: model and lattice (autotune, variant and reliable_interval are ignored);
 *   theta (double), x, y (complex double): caller device memory as for
 *   hqmc_apply_MdagM; x and y must not overlap.
 * Limit: Ntau * L * L <= 262144 sites (8 MiB of scratch); larger lattices
 * return HQMC_EUNSUPPORTED without touching the device.  Every call fully
 * rewrites the scratch before reading it, but all calls on a device share it:
 * calls whose executions overlap on the GPU (different streams with no
 * ordering) race and give wrong results, so order them on one stream.  The
 * first call on each device looks up the scratch address (cudaGetSymbolAddress,
 * once per device); make that first call before any stream capture.  The call
 * only enqueues work on `stream`. */
HQMC_API int hqmc_apply_MdagM_static(const hqmc_params* p, const double* theta, const void* x, void* y,
                                     void* stream);

/* ---- solver (Methods, "CG method and preconditioner", Eq. (pCG)) ------- */

/* Solves (M^dagger M) x = phi.  phi and x are complex double.  x holds the
 * initial guess on entry (zeros for the paper's X_0 = 0) and the solution on
 * exit.  Stops when ||r|| <= tol ||phi|| for the FP64 true residual
 * r = phi - (M^dagger M) x; HQMC_SOLVER_CG64 restarts from the true residual if
 * the recursive one has drifted.  maxit bounds the iterations.  *info (host,
 * may be NULL) is filled.  Synchronises the stream.  Returns HQMC_ENOTCONV,
 * HQMC_EBREAKDOWN or HQMC_ENONFINITE on failure with x holding the last iterate. */
HQMC_API int hqmc_cg_solve(hqmc_config* cfg, const double* theta, const void* phi, void* x,
                  double tol, int maxit, int solver, hqmc_solve_info* info, void* stream);

/* Stochastic estimation of fermionic observables (Methods, "Stochastic estimation
 * of fermionic observables").  For k = 0..nrv-1 a random vector xi_k ~ CN(0, 1) is
 * drawn per site from Philox4x32-10 (key = seed, counter = (site, 3, counter + k)),
 * R_k = M^dagger xi_k is formed, and X_k = (M^dagger M)^{-1} R_k = M^{-1} xi_k is
 * solved with `solver` to `tol` (each solve starting from the previous X).
 * (M^{-1} xi)_i conj(xi_j) is an unbiased estimate of (M^{-1})_ij.
 * Outputs (each nullable):
 *   Gxi:    device, nrv x N complex double, the X_k;
 *   xi:     device, nrv x N complex double, the draws;
 *   g_host: host double[2], the estimate of the mean diagonal of M^{-1},
 *           (1 / (nrv N)) sum_k <xi_k, X_k> (re, im); its real part has expectation
 *           exactly 1/2 at half filling on this bipartite lattice;
 *   infos:  host, nrv solve infos.
 * Returns HQMC_ENOTCONV if any solve missed tol.  Synchronises the stream. */
HQMC_API int hqmc_estimate(hqmc_config* cfg, const double* theta, uint64_t seed, uint64_t counter, int nrv,
                           double tol, int maxit, int solver, void* Gxi, void* xi, double* g_host,
                           hqmc_solve_info* infos, void* stream);

/* The same estimate with the right-hand sides solved as a set on one field:
 * every solve after the first starts from the Galerkin projection of its solution
 * onto the earlier ones, x0 = sum_{i<k} c_i X_i with G c = (<X_i, R_k>)_i and
 * G_ij = <X_i, (M^dagger M) X_j> = <X_i, R_j> (known from the earlier solves, no
 * extra operator application).  The solutions share the lowest modes of
 * M^dagger M, which dominate them and set the iteration count, so x0 already
 * carries most of them (not a method of the paper: its Methods solve the
 * N_rv = 40 systems independently).  Gxi is required (the earlier solutions are
 * the projection basis).  If the small Hermitian system is numerically singular
 * (pivot below 1e-12), or 2 nrv (blocks + 1) doubles exceed the config's scratch
 * vector (not at the paper's sizes), a solve starts from the previous solution as
 * in hqmc_estimate.  Outputs, errors and synchronisation as hqmc_estimate. */
HQMC_API int hqmc_estimate_projected(hqmc_config* cfg, const double* theta, uint64_t seed, uint64_t counter,
                                     int nrv, double tol, int maxit, int solver, void* Gxi, void* xi,
                                     double* g_host, hqmc_solve_info* infos, void* stream);

/* ---- systems solved together on one field ------------------------------
 * Methods, "Stochastic estimation of fermionic observables": the N_rv systems
 * (M^dagger M) X_k = R_k of an estimate share theta.  Solved together, one
 * CG iteration of all of them is one tau-walking M^dagger M launch (CTA b walks
 * slice range b / nrhs of system b % nrhs, so the CTAs resident together read
 * the same theta slices, and each walks a longer range than a one-system launch
 * could give it), one update launch and (PMIXED) one preconditioner launch; each
 * loop body ends with one FP64 reliable-update launch for all systems.  Every
 * system keeps its own scalars, CG state and convergence test on its own FP64
 * true residual. */

/* Allocates the workspace of up to nmax systems on this config (about 96 bytes
 * per site and system: six FP32 and three FP64 vectors) and their descriptor
 * tables; nmax = 0 frees it, a smaller nmax keeps the larger workspace.  The only
 * call of this group that allocates.  Needs the tau-walking FP32 kernel (every
 * even L that fits one slice per CTA; not with params.variant 1 or 2).
 * Synchronises the device.  Errors: HQMC_EINVAL (nmax outside [0, 1024]),
 * HQMC_EUNSUPPORTED (no tau-walking shape), HQMC_ENOMEM. */
HQMC_API int hqmc_set_multi_rhs(hqmc_config* cfg, int nmax);

/* Solves (M^dagger M) x_k = phi_k for k < nrhs on one theta.  phi and x are
 * device arrays of nrhs complex double vectors back to back (nrhs x Ntau x L x L);
 * x holds the guesses on entry and the solutions on exit.  solver is
 * HQMC_SOLVER_MIXED or HQMC_SOLVER_PMIXED (otherwise HQMC_EUNSUPPORTED).  A system
 * stops when its FP64 true residual ||phi_k - O x_k|| <= tol ||phi_k||; a system
 * whose FP32 recurrence breaks down or stalls is finished alone by the solver of
 * hqmc_cg_solve from its current iterate.  infos (host, nullable) receives nrhs
 * solve infos.  Needs hqmc_set_multi_rhs(cfg, >= nrhs) (HQMC_EINVAL otherwise).
 * Returns the first failure of hqmc_cg_solve's kinds over the systems;
 * synchronises the stream. */
HQMC_API int hqmc_cg_solve_multi(hqmc_config* cfg, const double* theta, int nrhs, const void* phi, void* x,
                                 double tol, int maxit, int solver, hqmc_solve_info* infos, void* stream);

/* hqmc_estimate with its systems solved together in groups of up to the
 * workspace's nmax (hqmc_set_multi_rhs), each from X = 0: the same draws xi_k,
 * R_k = M^dagger xi_k and estimate; outputs, errors and synchronisation as
 * hqmc_estimate; solver as hqmc_cg_solve_multi. */
HQMC_API int hqmc_estimate_multi(hqmc_config* cfg, const double* theta, uint64_t seed, uint64_t counter, int nrv,
                                 double tol, int maxit, int solver, void* Gxi, void* xi, double* g_host,
                                 hqmc_solve_info* infos, void* stream);

/* Fixes the slice ranges per system of the multi-system walk launch (each
 * system's Ntau slices split into `ranges` contiguous ranges, one CTA each);
 * 0 restores the default, the ranges with the fewest rounds of sweeps the device
 * needs: about ceil(nrhs ranges / resident CTAs) x (2 ceil(Ntau / ranges) + 1).
 * Results do not depend on it beyond FP32 rounding of the partial sums.
 * HQMC_EINVAL outside [0, Ntau].  Host only. */
HQMC_API int hqmc_set_multi_ranges(hqmc_config* cfg, int ranges);

/* Launch shape of a multi-system solve of nrhs systems: slice ranges per system
 * (*ranges), block size and strip height of the tau-walking kernel.
 * HQMC_EUNSUPPORTED without a tau-walking shape.  Host only. */
HQMC_API int hqmc_multi_launch_shape(const hqmc_config* cfg, int nrhs, int* ranges, int* threads, int* nby);

/* ---- force (Supplement SI, Eqs. (force&CG) and (fermion_force)) -------- */

/* Given X = (M^dagger M)^{-1} phi (complex double), writes the total force
 * F = -dS_B/dtheta - dS_f/dtheta with S_f = phi^dagger (M^dagger M)^{-1} phi and
 * S_B the bosonic action (compact: (1/(J dtau)) sum[1 - cos(theta_{tau+1} -
 * theta_tau)], non-compact: (1/(J dtau)) sum (theta_{tau+1} - theta_tau)^2, plus
 * K dtau sum_plaquettes cos(curl theta)).  dSf (nullable) receives dS_f/dtheta
 * alone.  F and dSf are double[Ntau][L][L][2] and may not alias theta. */
HQMC_API int hqmc_force(hqmc_config* cfg, const double* theta, const void* X, double* F,
               double* dSf, void* stream);

/* Hamiltonian terms of Eq. (H_hmc) at (theta, p) with fermion part phi^dagger X:
 * out_host[0] = S_B(theta), out_host[1] = sum p^2, out_host[2] = Re phi^dagger X.
 * p, phi or X may be NULL (the term is then 0).  Synchronises the stream. */
HQMC_API int hqmc_action_terms(hqmc_config* cfg, const double* theta, const double* p,
                      const void* phi, const void* X, double* out_host, void* stream);

/* ---- HMC (Methods, "HQMC algorithm": steps (i)-(iv), Eq. (leapfrog)) ---- */

/* Gaussian draws of step (i) from the counter-based Philox4x32-10 generator
 * (key = seed, counter = (element, stream, traj_counter)): p ~ N(0, 1/2) per
 * bond and R ~ CN(0, 1) per site (complex double).  Either output may be NULL.
 * *u_host (nullable) receives the Metropolis uniform of that trajectory. */
HQMC_API int hqmc_draw(hqmc_config* cfg, uint64_t seed, uint64_t traj_counter, double* p, void* R,
              double* u_host, void* stream);

/* nsteps leapfrog steps of size dt on (theta, p) in place:
 * p += F dt/2; theta += 2 p dt; solve; p += F dt/2, with F the total force.
 * X (complex double, in/out) is the CG initial guess on entry and
 * (M^dagger M)^{-1} phi at the final theta on exit.  Every solve uses tol,
 * maxit and solver as in hqmc_cg_solve.  *info (nullable): cg_solves,
 * cg_iterations, status, max_true_residual.  Synchronises the stream. */
HQMC_API int hqmc_leapfrog(hqmc_config* cfg, double* theta, double* p, const void* phi, void* X,
                  int nsteps, double dt, double tol, int maxit, int solver,
                  hqmc_traj_info* info, void* stream);

/* One HQMC update from theta (in/out).  Draws p and R with hqmc_draw(seed,
 * traj_counter) unless p_in (double, device) / R_in (complex double, device) /
 * u_in (host) are given; phi = M^dagger R; H0 = S_B + sum p^2 + R^dagger R;
 * nsteps leapfrog steps; H1 = S_B + sum p^2 + phi^dagger X; accepts iff
 * u < exp(H0 - H1), else restores theta.  Synchronises the stream. */
HQMC_API int hqmc_trajectory(hqmc_config* cfg, double* theta, uint64_t seed, uint64_t traj_counter,
                    const double* p_in, const void* R_in, const double* u_in, int nsteps,
                    double dt, double tol, int maxit, int solver, hqmc_traj_info* info,
                    void* stream);

/* ---- batches of independent chains (many lattices, one launch per CG step) */

/* A batch of nchains independent chains, chain c described by params[c] (L and
 * Ntau may differ; the batched kernels are the generic fused ones and every
 * chain gets the same cluster size, by default the smallest the chains admit).
 * If any params[c].autotune is set, hqmc_make_batch times the batched fused
 * launch at every cluster size 1, 2, 4, 8 the device co-schedules and every
 * tile order (hqmc_batch_launch_shape) and keeps the fastest; results do not
 * depend on that choice.  Each chain owns a config's workspace.  Inside a CG solve every iteration is ONE
 * launch of the fused M^dagger M over a tile table covering every chain's
 * slices plus ONE launch of the vector update over every chain's blocks, under
 * a device-side WHILE loop that runs while any chain is unconverged.  Every
 * chain's arithmetic and reduction order equal those of its own single-chain
 * config, so a batch reproduces independent runs bit for bit. */
typedef struct hqmc_batch hqmc_batch;

HQMC_API int hqmc_make_batch(const hqmc_params* params, int nchains, hqmc_batch** out);
HQMC_API int hqmc_free_batch(hqmc_batch* b);
HQMC_API const char* hqmc_batch_last_error(const hqmc_batch* b);

/* Solver of the batch's CG loop: HQMC_SOLVER_CG64 (default) or HQMC_SOLVER_PCG64, the
 * FP64 CG preconditioned with each chain's tau-line preconditioner (hqmc_apply_precond),
 * applied to all chains in one launch per iteration.  A chain's results are those of
 * its own config made with variant 1 and the same solver. */
HQMC_API int hqmc_batch_set_solver(hqmc_batch* b, int solver);
/* Kernels the batch has enqueued (including its chains' configs). */
HQMC_API long long hqmc_batch_launch_count(const hqmc_batch* b);
/* Tile shape of the batch's fused M^dagger M launch: cluster size along tau
 * (slices per tile), tile order (0 chain by chain, 1 chains with the most sites
 * per slice first, 2 round robin over the chains), block size, and the
 * autotuner's time of one launch in microseconds (0 without autotune).  Any
 * output pointer may be NULL.  HQMC_EINVAL for a NULL batch. */
HQMC_API int hqmc_batch_launch_shape(const hqmc_batch* b, int* cluster, int* order, int* threads, float* tuned_us);

/* CG on every chain: theta[c], phi[c], x[c] are HOST arrays of device
 * pointers with chain c's layouts (as in hqmc_cg_solve); infos (host, nchains
 * entries, nullable).  Returns the worst chain status.  Synchronises. */
HQMC_API int hqmc_batch_cg_solve(hqmc_batch* b, const double* const* theta, const void* const* phi, void* const* x,
                                 double tol, int maxit, hqmc_solve_info* infos, void* stream);

/* One HQMC update of every chain (as hqmc_trajectory with device draws:
 * seeds[c], the shared traj_counter, nsteps steps of dt[c]); theta[c] in/out;
 * infos (host, nchains entries, nullable).  The whole trajectory of all chains is
 * ONE CUDA graph launch (Methods, "CUDA Graph acceleration"): batched draws, link
 * tables, phi = M^dagger R, Hamiltonian terms, forces and kicks over a table of
 * every chain's blocks or slices, the N_lf + 1 batched solves as conditional WHILE
 * nodes, and the Metropolis test and restore on the device.  The graph is captured
 * on first use for (nsteps, tol, maxit, solver) and replayed; per-chain field
 * pointers, seeds, dt and the counter are uploaded before each launch.  A chain
 * whose solve fails is rejected (its status in infos[c]).  Returns the worst chain
 * status.  Synchronises once. */
HQMC_API int hqmc_batch_trajectory(hqmc_batch* b, double* const* theta, const uint64_t* seeds, uint64_t traj_counter,
                                   int nsteps, const double* dt, double tol, int maxit, hqmc_traj_info* infos,
                                   void* stream);

/* ---- learned preconditioner (spec extension; not in the paper) ----- */

/* A 3D periodic convolution network on the space-time lattice: 4 layers with
 * 1 -> 16 -> 16 -> 16 -> 1 complex channels; each layer is a 7-point stencil
 * (centre, +-x, +-y, +-tau) whose neighbour values are parallel-transported by
 * e^{i theta} (antiperiodic sign across tau = 0) and mixed by real 16x16
 * matrices.  It is gauge covariant and linear in its input, K(theta) r.
 * Weights are BF16 (FP32 master copy for training); arithmetic is FP32.
 * Weight layout per layer: [7][c_out][c_in], layers in order, 3808 floats. */
typedef struct hqmc_net hqmc_net;

/* Net on the current device, initialised near the identity map (seeded). */
HQMC_API int hqmc_net_create(uint64_t seed, hqmc_net** out);
HQMC_API int hqmc_net_free(hqmc_net* net);
HQMC_API int hqmc_net_num_weights(const hqmc_net* net);
/* FP32 master weights to / from host memory (n == hqmc_net_num_weights). */
HQMC_API int hqmc_net_get_weights(const hqmc_net* net, float* host, int n);
HQMC_API int hqmc_net_set_weights(hqmc_net* net, const float* host, int n);
/* z = K(theta) r (complex double in and out; computed in FP32).  Needs the net
 * workspace of the config: attach a net with hqmc_set_preconditioner first
 * (HQMC_EINVAL otherwise).  Allocates nothing. */
HQMC_API int hqmc_net_apply(hqmc_config* cfg, hqmc_net* net, const double* theta, const void* r, void* z,
                            void* stream);
/* One Adam step (lr; betas 0.9, 0.999) on loss = ||K(theta) phi - x||^2 / ||x||^2
 * for one (theta, phi, x) triple with x = (M^dagger M)^{-1} phi; *loss_host
 * (nullable) receives the loss before the step (then the call synchronises).
 * Like hqmc_net_apply it needs the config's net workspace and allocates nothing. */
HQMC_API int hqmc_net_train_step(hqmc_config* cfg, hqmc_net* net, const double* theta, const void* phi,
                                 const void* x, double lr, double* loss_host, void* stream);
/* Flexible CG (HQMC_SOLVER_FLEARNED): the net preconditions iterations c with
 * c % k == 0 of each reliable-update segment, the tau-line preconditioner the
 * others (k >= 1; 1 = every iteration).  Host-only; HQMC_EINVAL for k < 1. */
HQMC_API int hqmc_set_net_interval(hqmc_config* cfg, int k);
/* Arithmetic of the net's inference layers (hqmc_net_apply, the learned guess and
 * flexible CG): on = 1 (default) stores the 16-channel activations in BF16 and
 * runs the layers that read them (16 -> 16 and 16 -> 1) on tensor cores: BF16
 * activations times BF16 weights with FP32 accumulation (warp-level mma, 16
 * output channels x 8 sites per product), the transport phases applied to the
 * FP32 products.  on = 0 keeps every layer and activation in FP32 on CUDA cores.
 * Training stays in FP32.  Host-only; HQMC_EINVAL unless on is 0 or 1. */
HQMC_API int hqmc_set_net_tensor_cores(hqmc_config* cfg, int on);

/* Chronological initial guess of the solves inside hqmc_leapfrog and
 * hqmc_trajectory (Brower, Ivanenko, Levi and Orginos, "Chronological inversion
 * method for the Dirac matrix in hybrid Monte Carlo", Nucl. Phys. B 484 (1997);
 * not a method of the paper, which starts every pCG from X_0 = 0).  With k >= 2
 * the last k solutions of the current integration are kept; every solve after
 * the first starts from the Galerkin solution in their span with the current
 * operator: Q an orthonormal basis of them, G = Q^dagger (M^dagger M) Q (O applied
 * in FP32, k applies), x0 = Q G^{-1} Q^dagger phi.  k = 0 (the default) keeps the
 * previous solution as the guess; k = 1 is the same.  The first call with a
 * given k allocates 2 k vectors (complex double) on the config, kept until
 * hqmc_free_config; make it before any stream capture.  The solves' own
 * tolerance and FP64 true residual are unchanged, so only the iteration counts
 * change.  0 <= k <= 8.  Errors: HQMC_EINVAL, HQMC_ENOMEM, HQMC_EUNSUPPORTED
 * (a lattice whose scratch vector cannot hold the k-vector dot partials). */
HQMC_API int hqmc_set_guess_history(hqmc_config* cfg, int k);

/* Attaches (or with NULL detaches) the net used by HQMC_SOLVER_LEARNED.  The
 * first attach on a config allocates the net workspace (activation and gradient
 * fields, 5 + 32 complex-float channels per site, about 300 B per site), which the
 * config keeps until hqmc_free_config; make this call before any stream capture.
 * The net must belong to the config's device.  Errors: HQMC_EINVAL, HQMC_ENOMEM. */
HQMC_API int hqmc_set_preconditioner(hqmc_config* cfg, hqmc_net* net);

/* ---- checkpoint / resume (not in the paper; its production runs imply it) -- */

/* Everything that fixes a chain's future besides theta: the model, the Philox
 * key and the counter of the next trajectory (every random number of trajectory
 * k is a function of (seed, k), so a resumed chain continues bit for bit), the
 * leapfrog parameters and the acceptance statistics. */
typedef struct hqmc_checkpoint {
    int L, Ntau;
    double dtau, t, J, K;
    int action;
    int n_weights;            /* learned net's FP32 master weights stored after theta (0: none) */
    uint64_t seed;            /* Philox key of the chain */
    uint64_t traj_counter;    /* counter of the next trajectory */
    double dt;                /* leapfrog step */
    int nsteps;               /* leapfrog steps per trajectory */
    int solver;               /* HQMC_SOLVER_* of the chain */
    long long trajectories;   /* trajectories run so far */
    long long accepted;       /* of which accepted */
    int version;              /* file format version (1) */
    int reserved;
} hqmc_checkpoint;

/* Writes the checkpoint: magic, *c, theta (HOST, double[Ntau][L][L][2]), the
 * weights (HOST, c->n_weights floats, nullable when 0) and a 64-bit FNV-1a hash
 * of the rest.  Host-only; HQMC_EINVAL for a bad header, HQMC_EIO on a file
 * error. */
HQMC_API int hqmc_checkpoint_write(const char* path, const hqmc_checkpoint* c, const double* theta_host,
                                   const float* weights_host);

/* Reads a checkpoint into *c.  With theta_host NULL only the header is read (to
 * size the buffers); otherwise theta (HOST, 2 Ntau L L doubles) and, if
 * weights_host is given, the weights are read and the hash is checked.
 * HQMC_EIO for a missing, truncated or corrupted file (nothing written to *c). */
HQMC_API int hqmc_checkpoint_read(const char* path, hqmc_checkpoint* c, double* theta_host, float* weights_host);

/* ---- instrumentation ---------------------------------------------------- */

/* Timed kernel classes: the fused M^dagger M in FP64 (applies, CG directions,
 * residuals), the fused M^dagger M in FP32, the CG vector update, the force,
 * and the two passes of the tau-line preconditioner inside CG iterations. */
enum { HQMC_TIMER_MDAGM = 0, HQMC_TIMER_CG_UPDATE = 1, HQMC_TIMER_FORCE = 2, HQMC_TIMER_MDAGM32 = 3,
       HQMC_TIMER_PRECOND = 4, HQMC_TIMER_COUNT = 5 };

/* Enables (1) or disables (0) CUDA-event timing of kernel launches and resets
 * the counters.  Events are recorded on the launching stream around every
 * launch of the timed kernel classes. */
HQMC_API int hqmc_set_timing(hqmc_config* cfg, int enable);

/* Synchronises the device and returns, for one kernel class, the number of
 * timed launches and their summed duration in milliseconds. */
HQMC_API int hqmc_get_timing(hqmc_config* cfg, int timer, long long* launches, double* total_ms);

/* Synchronises the device and writes the durations (microseconds) of the first
 * min(max_n, launches) timed launches of one kernel class, in launch order, to
 * us (host); *n_out (nullable) receives the number of timed launches.  Launches
 * that found their solve finished (the rest of a loop body after convergence)
 * are among them: a median over the samples is the time of a launch that works. */
HQMC_API int hqmc_get_timing_samples(hqmc_config* cfg, int timer, float* us, int max_n, int* n_out);

/* Measures the device's FP64 fused-multiply-add throughput (TFLOP/s, 2 flops
 * per FMA) with a short kernel of independent FMA chains on the default
 * stream; used as the roofline denominator of the FP64 (ALU-bound) kernels.
 * Synchronises the device. */
HQMC_API int hqmc_probe_fp64_rate(hqmc_config* cfg, double* tflops_out);

#ifdef __cplusplus
}
#endif

#endif /* HQMC_H */
