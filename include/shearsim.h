/*
 * shearsim.h — C ABI of the GB300 (sm_103a) coupled velocity solve of
 * Korolkovas, "Giant fluctuations in sheared viscoelastic fluids emerging in
 * a mesoscale simulation" (arXiv 1808.06381).
 *
 * One particle per polymer chain (§Method).  Every time step:
 *   1. finds all pairs closer than the truncation radius r_c under sheared
 *      (Lees-Edwards) periodic images (§Method: weights truncated below 5 %,
 *      "standard Lees-Edwards boundary conditions");
 *   2. evaluates the forces of Eq. F (noise, excluded volume Eq. exvol, shear
 *      body force) and assembles Eq. vc as the sparse symmetric positive-
 *      definite system of Eq. algebra, A v = b, with
 *        A_ii = 1 + alpha sum_j w_ij,  A_ij = -alpha w_ij,
 *        b_i  = F_i / zeta + alpha sum_j V_ij w_ij,
 *        w_ij = exp(-R_ij^2 / 2 lambda^2),  V_ij = kappa L_y round(y_ij / L_y) x;
 *   3. solves it for all velocities with Jacobi-preconditioned conjugate
 *      gradients on the GPU;
 *   4. advances R += v dt (first order in time) with the Lees-Edwards wrap.
 *
 * Units: lengths in r_c; lambda^2 = r_c^2 / (2 ln 20) follows from the 5 %
 * truncation; the excluded-volume parameter v/lambda^3 is 0.1 (§Method) times
 * eps; the thermal noise is sqrt(2 zeta kT / dt) N(0,1) per Cartesian
 * component (the discrete form of sqrt(6 zeta kT) W_c(t) with <W.W> = delta).
 *
 * Conventions for every call:
 *   - returns SP_OK (0) or a negative sp_status; nothing is thrown across the ABI;
 *   - sp_last_error() gives a one-line description of the last failure;
 *   - arrays called *_host are caller-owned host memory (pinned or pageable),
 *     copied before the call returns; arrays called *_dev are caller-owned
 *     device memory on the simulation's device, read or written on the
 *     simulation's stream;
 *   - per-particle host arrays are indexed by particle id (the row order of
 *     the positions given to sp_sim_create) and laid out [n][3] row-major;
 *   - the library owns every device buffer of a simulation and frees them in
 *     sp_sim_destroy;
 *   - calls on one simulation must not run concurrently from several threads.
 */
#ifndef SHEARSIM_H
#define SHEARSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sp_status {
    SP_OK = 0,
    SP_ERR_INVALID_ARG = -1,    /* a null pointer, n <= 0, a non-positive box edge, ... */
    SP_ERR_CUDA = -2,           /* a CUDA runtime call failed (sp_last_error has the text) */
    SP_ERR_NOT_CONVERGED = -3,  /* CG hit cg_max_iter before ||b - Av|| <= cg_tol ||b|| */
    SP_ERR_NONFINITE = -4,      /* a NaN or infinity appeared in the solve */
    SP_ERR_OOM = -5,            /* device allocation failed */
    SP_ERR_BOX_TOO_SMALL = -6,  /* some box edge is below 2 r_c: the minimum image is ambiguous */
    SP_ERR_NO_DEVICE = -7,      /* no CUDA device, or the requested ordinal does not exist */
    SP_ERR_TIMEOUT = -8         /* a device-side wait of the persistent solver ran past its limit
                                   (sp_set_wait_limit) */
} sp_status;

enum sp_precision {
    SP_PREC_FP64 = 0,   /* matrix, vectors and dots in FP64 */
    SP_PREC_MIXED = 1   /* FP32 SpMV, axpy and Jacobi; double-float (FP32 pipes) assembly, normals, dots,
                           x and residual replacement; FP64 positions */
};

enum sp_warm_start {
    SP_WARM_NONE = 0,   /* CG starts from v = 0 */
    SP_WARM_PREV = 1    /* CG starts from the previous step's velocities */
};

/* Model and solver parameters (§Method).  kappa is the shear rate in units of
 * kT / (zeta r_c^2); sp_kappa_from_kappa_tau converts the paper's kappa*tau. */
typedef struct sp_params {
    int64_t n;            /* particles (chains), >= 2 */
    double L[3];          /* box edges L_x, L_y, L_z; each >= 2 r_c */
    double rc;            /* truncation radius (w = 5 % there) */
    double alpha;         /* entanglement strength (4 in the paper's shear runs), >= 0 */
    double eps;           /* multiplies the paper's v/lambda^3 = 0.1 */
    double zeta;          /* friction coefficient, > 0 */
    double kT;            /* temperature, >= 0 */
    double kappa;         /* shear rate in the xy plane (x flow, y gradient) */
    double dt;            /* time step, > 0 */
    uint64_t seed;        /* key of the counter-based noise generator */
    int32_t precision;    /* enum sp_precision */
    int32_t warm_start;   /* enum sp_warm_start */
    double cg_tol;        /* stop at ||b - A v||_2 <= cg_tol ||b||_2 over all 3n entries */
    int32_t cg_max_iter;  /* iteration cap per solve (e.g. 1000) */
    int32_t device;       /* CUDA device ordinal */
    void* stream;         /* cudaStream_t to run on; NULL: the library creates its own */
} sp_params;

typedef struct sp_solve_info {
    int32_t status;       /* sp_status of the solve */
    int32_t iterations;   /* CG iterations of this solve */
    double residual;      /* final true relative residual ||b - A v|| / ||b|| (FP64) */
    double bnorm;         /* ||b||_2 */
    int32_t offchip_blocks; /* on-chip solver configuration: blocks some of whose entries (the
                               chunks that found no room) or all of them did not fit on their SM
                               and were gathered from global memory (0 otherwise) */
    int32_t host_driven;    /* 1: the solve's CG loop was driven from the host (graph capture
                               unavailable, or SHEARSIM_HOST_LOOP=1); 0: it ran as one CUDA graph */
} sp_solve_info;

typedef struct sp_step_info {
    int32_t status;          /* first non-OK status of the steps, else SP_OK */
    int32_t max_iterations;  /* largest CG iteration count of the steps */
    int64_t steps_done;      /* steps completed by this call */
    int64_t cg_iterations;   /* CG iterations summed over the steps */
    double last_residual;    /* true relative residual of the last solve */
    double stress_xy;        /* shear stress of the last step (pair virial, see sp_stress_xy) */
    int64_t kernel_launches; /* kernels this call ran on the GPU */
    double delta;            /* Lees-Edwards offset after the steps (as sp_get_state) */
    int64_t step;            /* step counter after the steps (as sp_get_state) */
    int32_t host_driven;     /* 1: the steps' kernels were launched from a host loop (graph capture
                                unavailable, or SHEARSIM_HOST_LOOP=1); 0: each step ran as one CUDA
                                graph with the CG loop inside it */
} sp_step_info;

typedef struct sp_sim sp_sim;

/* kappa = kappa_tau / tau with tau = lambda^2 zeta / kT, lambda^2 = rc^2 / (2 ln 20)
 * (§Method: tau is the Rouse time).  Returns NaN if kT <= 0. */
double sp_kappa_from_kappa_tau(double kappa_tau, double rc, double zeta, double kT);

/* Create a simulation on p->device.  pos_host: [n][3] initial positions in
 * [0, L) (copied), or NULL for positions uniform in the box drawn from the
 * counter-based generator keyed by p->seed.  The Lees-Edwards offset starts at
 * 0 and the step counter at 0.  On success *out owns all device memory. */
int sp_sim_create(const sp_params* p, const double* pos_host, sp_sim** out);

/* Free everything; NULL is allowed. */
int sp_sim_destroy(sp_sim* sim);

/* One line describing the last failure on this simulation ("" if none);
 * valid until the next call on it.  sim may be NULL (creation errors). */
const char* sp_last_error(const sp_sim* sim);

/* Step 1 for the current positions: cell list with sheared periodic images,
 * then all pairs with |R_ij|^2 < r_c^2 (§Method, 5 % truncation). */
int sp_build_neighbors(sp_sim* sim);

/* Step 2 for the current pairs: forces of Eq. F with the noise of the current
 * step counter, and Eq. algebra (A, b, Jacobi diagonal).  Requires
 * sp_build_neighbors since the last position change. */
int sp_assemble(sp_sim* sim);

/* Step 3: solve Eq. algebra by Jacobi-PCG (FP64 or mixed, per p->precision).
 * v0_dev: optional start vector, device [3][n] planes in the library's
 * current particle order (see sp_get_order), or NULL for the configured warm
 * start.  info may be NULL.  Returns SP_ERR_NOT_CONVERGED if the iteration
 * cap is hit; the velocities are kept either way. */
int sp_solve_velocities(sp_sim* sim, const double* v0_dev, sp_solve_info* info);

/* Step 3 by flexible conjugate gradients (FCG(1), Notay 2000) in FP64 with a
 * preconditioner that may change between iterations: the learned network
 * (sp_mpnn_enable) applied to the current residual at iterations k with
 * net_every > 0 and k % net_every == 0 (the network maps a right-hand side to
 * an approximation of A^-1 of it; its previous-velocity feature is 0 here),
 * Jacobi D^-1 otherwise; net_every = 0 is Jacobi throughout (PCG in exact
 * arithmetic).  Each new direction is A-orthogonalised against the previous
 * one.  Not in the paper (its solver is unnamed); an alternative to the
 * warm start for the learned part.  Starts from the configured warm start,
 * stops at ||r|| <= cg_tol ||b|| on the recurrence residual, and reports the
 * true residual b - A x (SP_ERR_NOT_CONVERGED if it is above cg_tol or
 * cg_max_iter is reached).  The iteration is driven from the host (state
 * polled every 8 iterations).  Requires an SP_PREC_FP64 simulation and
 * sp_assemble; info->host_driven is 1.  Errors: SP_ERR_INVALID_ARG (mixed
 * precision, no assembled system, net_every > 0 without a network),
 * SP_ERR_NOT_CONVERGED, SP_ERR_NONFINITE, SP_ERR_OOM, SP_ERR_CUDA. */
int sp_solve_flexible(sp_sim* sim, int32_t net_every, sp_solve_info* info);

/* nsteps full time steps (steps 1-4), each run as one CUDA graph launch with
 * the CG loop inside the graph.  The noise of step k is keyed by the step
 * counter, which advances by one per step.  info may be NULL.  Stops early on
 * the first failing step (info->steps_done tells how many finished). */
int sp_step(sp_sim* sim, int32_t nsteps, sp_step_info* info);
/* The same steps from and to host memory in one call: pos_in [n][3] by
 * particle id (each in [0, L)) and the Lees-Edwards offset delta in [0, L_x)
 * replace the state, nsteps steps run, and the positions after them are
 * written to pos_out [n][3] by particle id (may alias pos_in).  One
 * synchronisation in the common case (the host arrays are read and written
 * before the call returns).  The positions are checked on the device as in
 * sp_set_positions, inside the same synchronisation: invalid ones return
 * SP_ERR_INVALID_ARG with no step taken.  Errors: those of sp_set_positions
 * and sp_step. */
int sp_step_host(sp_sim* sim, const double* pos_in, double delta, int32_t nsteps, double* pos_out,
                 sp_step_info* info);
/* Bytes of the state record (step statistics, CG scalars, flags) that
 * sp_step and sp_step_host copy to the host once per call. */
int64_t sp_state_record_bytes(void);

/* Eq. Sfactor at q_z = 0 on the sheared reciprocal lattice of the current
 * positions: q_x = 2 pi kx / L_x, q_y = 2 pi ky / L_y - (delta / L_y) q_x for
 * kx in [-nkx, nkx], ky in [-nky, nky].  Outputs (host, (2nkx+1)(2nky+1)
 * entries, kx slowest): S_host = |sum_c exp(-i q . R_c)|^2 / n, qx_host, qy_host
 * (either q array may be NULL).
 * grid > 0: the density is spread on a grid x grid mesh of the sheared frame
 * x' = x - (delta/L_y) y by cloud-in-cell (z summed), transformed, and the CIC
 * window divided out; |kx|, |ky| must stay below grid / 4 (aliasing grows
 * towards the mesh's Nyquist limit).  grid = 0: exact direct sum over the
 * particles for every mode (cost n x modes). */
int sp_structure_factor(sp_sim* sim, int32_t nkx, int32_t nky, int32_t grid, double* S_host,
                        double* qx_host, double* qy_host);

/* Shear stress sigma_xy of the current state: -(1/V) sum_{i<j} y_ij f_ij,x with
 * f_ij = eps 0.1 kT/lambda^2 R_ij w_ij + zeta alpha w_ij (v_j - v_i + V_ij), the
 * pair forces of Eq. F and Eq. vc, using the velocities of the last solve.
 * The paper defines no stress; this is the pair virial of its pair forces. */
int sp_stress_xy(sp_sim* sim, double* sigma_xy);

/* FDT-consistent thermal noise (not in the paper, which draws the noise of
 * Eq. F independently per particle): xi = p(A) g ~ A^(1/2) g for the current
 * assembled matrix A of Eq. algebra, p the degree-`degree` Chebyshev
 * interpolant of sqrt on [1, lambda_max] (Chebyshev points of the first kind;
 * lambda_max = max_i (A_ii + alpha sum_j w_ij), Gershgorin's bound; the
 * spectrum starts at 1 because A = I + alpha L_w with L_w positive
 * semidefinite).  If g has covariance I, xi has covariance p(A)^2 ~ A; passing
 * xi to sp_set_noise and assembling again gives a step whose noise is
 * correlated like the friction.  g_host, xi_host: [n][3] in particle order
 * (host).  lambda_max (may be NULL) receives the interval's upper end; when it
 * is 1 (no coupling) xi = g.  One sliced-layout SpMV per degree (FP64 for the
 * FP64 path, double-float on the FP32 pipes for the mixed path); steps_ms (may be NULL)
 * receives their time (CUDA events on the simulation's stream).  Errors:
 * SP_ERR_INVALID_ARG (NULL pointer, degree outside [1, 4096], no assembled
 * system), SP_ERR_OOM, SP_ERR_CUDA. */
int sp_sqrt_apply(sp_sim* sim, int32_t degree, const double* g_host, double* xi_host, double* lambda_max,
                  double* steps_ms);

/* Steps with A^(1/2)-correlated noise: with degree > 0 every step of sp_step /
 * sp_step_host replaces the independent normals g in its right-hand side by
 * xi = p(A) g as sp_sqrt_apply forms it (on the device, inside the step's
 * graph): b += (noise amplitude / zeta) (xi - g) after the assembly.  degree =
 * 0 restores the paper's independent noise (the default).  Costs one SpMV
 * per degree per step.  Batched steps (sp_batch_step) keep the independent
 * noise.  Errors: SP_ERR_INVALID_ARG (degree outside [0, 4096]),
 * SP_ERR_OOM. */
int sp_set_fdt_noise(sp_sim* sim, int32_t degree);

/* Velocity cross-correlation versus distance (§Results, Fig. vv): the average
 * inter-chain velocity product <v_c . v_c'> / <v_c^2> against |R_cc'|.
 * u_c = v_c - kappa (y_c - L_y/2) x is the velocity relative to the imposed
 * flow (the lab velocity at kappa = 0; a Lees-Edwards image carries the same
 * u).  Every pair c < c' whose minimum-image distance r is below rmax adds
 * u_c . u_c' to bin k = floor(r nbins / rmax) (nbins - 1 where that rounds up
 * to nbins) and counts there; the correlation of bin k is
 * sum_host[k] / (count_host[k] vsq_host) with vsq_host = <|u|^2> over all
 * particles.  All n^2 / 2 pairs are visited.  The counts are exact (a pair
 * whose FP32 distance lies near a bin edge, the cut-off or an image boundary
 * is decided with the FP64 operations of the definition); each product enters
 * its sum rounded to a fixed point of 2^-20 of the largest |u|^2 (absolute
 * error per pair below 2^-19 max |u|^2, independent of the order of the sums).
 * Uses the simulation's current positions and the velocities of its last
 * solve.  Outputs (host): sum_host[nbins], count_host[nbins], vsq_host; info
 * may be NULL.  Errors: SP_ERR_INVALID_ARG (NULL pointer, nbins outside
 * [1, 1024], rmax <= 0), SP_ERR_OOM, SP_ERR_CUDA. */
typedef struct sp_vcorr_info {
    double pairs_ms;          /* the all-pairs kernel, CUDA events on the simulation's stream */
    int64_t boundary_pairs;   /* pairs decided in FP64 */
    int64_t pairs;            /* pairs visited, n (n - 1) / 2 */
} sp_vcorr_info;
int sp_velocity_correlation(sp_sim* sim, int32_t nbins, double rmax, double* sum_host, int64_t* count_host,
                            double* vsq_host, sp_vcorr_info* info);

/* The same for given positions and velocities (host arrays pos_host[n][3] with
 * every coordinate in [0, L_a), v_host[n][3]) in the box L3[3] with shift delta
 * (0 <= delta < L_x) and shear rate kappa, on device `device`.  Allocates and
 * frees its own device memory.  Errors as above, SP_ERR_INVALID_ARG also for a
 * position outside the box, SP_ERR_NO_DEVICE. */
int sp_velocity_correlation_host(int32_t device, int64_t n, const double* L3, double delta, double kappa,
                                 const double* pos_host, const double* v_host, int32_t nbins, double rmax,
                                 double* sum_host, int64_t* count_host, double* vsq_host, sp_vcorr_info* info);

/* Per-kernel timing of one time step (a diagnostic for roofline reports).
 * Runs one full step (it advances the simulation exactly like sp_step(sim, 1))
 * with the CG loop driven from the host and a CUDA event pair on the
 * simulation's stream around every kernel launch; times are sums in ms. */
typedef struct sp_kernel_profile {
    int32_t spmv_launches;           /* q = A p (the solver's SpMV) */
    int32_t update_launches;         /* x, r update with the r.r, r.z partial sums */
    int32_t direction_launches;      /* p = z + beta p */
    int32_t true_residual_launches;  /* r = b - A x checks */
    double spmv_ms, update_ms, direction_ms, true_residual_ms;
    double build_ms;                 /* cell list, pair search and assembly */
    double other_ms;                 /* solver set-up, stress, position update */
    int64_t n;                       /* rows */
    int64_t nnz;                     /* off-diagonal entries (2 x pairs) */
    int32_t cg_iterations;
    int32_t precision;               /* enum sp_precision of the solver */
    double sort_ms;                  /* part of build_ms: binning and the counting sort into cell order */
    double count_ms;                 /* part of build_ms: the pair search (counts and partners) and the slice plan */
    double fill_ms;                  /* part of build_ms: a separate pair fill (0: the assembly places the pairs) */
    int64_t nnz_slots;               /* stored entries including the sliced layout's padding */
    int32_t probe_reps;              /* back-to-back launches timed for the two fields below */
    double spmv_probe_ms;            /* average SpMV kernel time, launched back to back */
    double update_probe_ms;          /* average update kernel time, launched back to back */
    double persistent_ms;            /* the persistent mixed solver kernel (0 when not used) */
    int32_t true_checks;             /* FP64 true-residual computations of the solve */
    int32_t persistent_blocks;       /* its grid (cooperative launch), 0 when not used */
    double init_ms;                  /* part of other_ms: solver set-up (r = b - A x0, or the split of x0) */
    double stress_ms;                /* part of other_ms: the stress kernel */
    double integrate_ms;             /* part of other_ms: the position update */
    double mpnn_ms;                  /* the learned warm start's inference (0 when not used) */
    double assemble_ms;              /* part of build_ms: FP64 assembly of the matrix and right-hand side */
    int32_t persistent_init;         /* 1: the persistent (on-chip) solve formed r = b - A x0 itself, as in
                                        sp_step; init_ms then holds only the split of x0 */
} sp_kernel_profile;
int sp_profile_step(sp_sim* sim, sp_kernel_profile* out);

/* ---- autotuning of the persistent solver's tiles ----
 *
 * Not in the paper (an implementation parameter).  The mixed-precision
 * solve runs as one cooperative persistent kernel compiled in several tile
 * configurations: gathers in flight per thread against resident blocks per
 * SM, with or without requesting the next batch of matrix columns while the
 * current gathers are in flight, and blocks of 256 or 1024 threads (one or
 * four windows of rows at a time; fewer, larger blocks make the grid-wide
 * reductions cheaper).  All of them run the same iteration with the same
 * per-row arithmetic; the grid-wide dot products are summed per block, so a
 * configuration with another block count rounds them differently (results
 * agree to about 1e-13 relative), and each configuration is deterministic.
 * One configuration (resident = 1) keeps each block's rows on its SM for the
 * whole solve: their solver vectors in registers, their z = D^-1 r and the
 * matrix entries between two of them in shared memory, so that only entries
 * to other blocks' rows are gathered from global memory; it serves systems of
 * at most 2048 rows per SM and is not timed (ms 0) for larger ones.
 * Two configurations (matrix_free = 1) stream only the columns in the
 * iteration and recompute each pair weight w_ij = exp(-|R_ij|^2 / 2 lambda^2)
 * (arXiv 1808.06381, §Method) in FP32 from the positions in 32-bit fixed
 * point (~3e-7 of the assembled weight); their residual replacements use the
 * assembled weights, so they meet the same tolerance on the same system.
 * sp_autotune builds the pair list
 * and the system for the current positions, times `trials` solves from a
 * zero start with every configuration on the simulation's stream, keeps the
 * fastest for this simulation, and leaves positions, step counter and the
 * previous velocities (the warm start) unchanged.  With the environment
 * variable SHEARSIM_TUNE_CACHE naming a file, choices are looked up there
 * first, keyed by device name, SM count, n and the mean row length, and new
 * choices are appended (one line per key).  For SP_PREC_FP64, or with
 * trials < 1, nothing is timed and configuration 0 is kept.  Errors:
 * SP_ERR_INVALID_ARG (NULL sim), SP_ERR_CUDA, and those of the solve. */
#define SP_TUNE_MAX_CONFIGS 12
typedef struct sp_tune_info {
    int32_t config;              /* chosen configuration (index) */
    int32_t gathers_in_flight;   /* its gathers in flight per thread */
    int32_t blocks_per_sm;       /* its resident blocks per SM */
    int32_t from_cache;          /* 1: taken from the tuning cache, nothing timed */
    int32_t num_configs;         /* configurations available */
    double ms[SP_TUNE_MAX_CONFIGS]; /* best time of one solve per configuration (0: not timed) */
    int32_t pipelined;           /* 1: the next batch of columns is requested during the current gathers */
    int32_t block_threads;       /* threads per block (256 per window processed at once) */
    int32_t resident;            /* 1: rows, their vectors and the entries between them kept on chip */
    int32_t matrix_free;         /* 1: streaming solve whose SpMV recomputes the pair weights w_ij from
                                    the positions every iteration (reads only the columns) */
} sp_tune_info;
int sp_autotune(sp_sim* sim, int32_t trials, sp_tune_info* info);
/* Select tile configuration `config` (0 .. num_configs - 1) of the persistent
 * solver for this simulation without timing, e.g. one an earlier sp_autotune
 * chose for the same system.  info (may be NULL) receives its description
 * (ms all 0).  A configuration that cannot serve the system (the on-chip one
 * beyond 2048 rows per SM) falls back to configuration 0 at each solve.
 * Errors: SP_ERR_INVALID_ARG (NULL sim, config out of range). */
int sp_set_solver_config(sp_sim* sim, int32_t config, sp_tune_info* info);

/* ---- state access (test hooks and checkpointing) ---- */

/* Positions [n][3] by particle id. */
int sp_get_positions(sp_sim* sim, double* pos_host);
/* Replace positions ([n][3] by particle id, each in [0, L)) and the
 * Lees-Edwards offset delta in [0, L_x).  Every coordinate is checked on the
 * device as it is gathered: a NaN, an infinity or a value outside [0, L_a)
 * returns SP_ERR_INVALID_ARG, after which the simulation's positions are
 * undefined until valid ones are set (the simulation itself stays usable). */
int sp_set_positions(sp_sim* sim, const double* pos_host, double delta);
/* Velocities of the last solve [n][3] by particle id. */
int sp_get_velocities(sp_sim* sim, double* v_host);
/* Lees-Edwards offset and step counter (the noise key). */
int sp_get_state(sp_sim* sim, double* delta, int64_t* step);
/* Architecture of the device code that `device` runs for this library
 * (cudaFuncGetAttributes of one of its kernels): *binary_version = 10 x major +
 * minor of the machine code (103 for a build for sm_103a on a GB300),
 * *ptx_version likewise for the virtual architecture it was compiled from.
 * Not in the paper (a build check).  Errors: SP_ERR_INVALID_ARG (NULL
 * output), SP_ERR_NO_DEVICE, SP_ERR_CUDA (no code for this device). */
int sp_device_code_version(int32_t device, int32_t* binary_version, int32_t* ptx_version);

/* Set the step counter, e.g. to resume a checkpoint (positions via sp_set_positions). */
int sp_set_step(sp_sim* sim, int64_t step);
/* Limit of one device-side wait of the persistent solvers (a block waiting at
 * a grid barrier for the other blocks), in seconds, (0, 60]; 2 s by default.
 * A wait that runs past it makes the solve return SP_ERR_TIMEOUT instead of
 * waiting on; the simulation stays usable.  Not in the paper (a safety bound
 * of the implementation).  Errors: SP_ERR_INVALID_ARG. */
int sp_set_wait_limit(sp_sim* sim, double seconds);
/* Particle id of each internal row, [n] (rows are kept in cell order). */
int sp_get_order(sp_sim* sim, int64_t* ids_host);
/* Number of pairs i < j found by the last sp_build_neighbors / sp_step. */
int sp_get_num_pairs(sp_sim* sim, int64_t* npairs);
/* The pairs (by particle id, i < j, unsorted) [npairs][2]; cap = capacity in pairs. */
int sp_get_neighbors(sp_sim* sim, int64_t cap, int64_t* pairs_host, int64_t* npairs);
/* The assembled system by particle id: diag_host [n] (A_ii), b_host [n][3],
 * w_host [npairs] weight of each pair in the order of sp_get_neighbors
 * (any output may be NULL). */
int sp_get_system(sp_sim* sim, double* diag_host, double* b_host, double* w_host);
/* Noise override: xi_host [n][3] standard normals by particle id used by
 * every following assembly instead of the generator; NULL returns to the
 * generator. */
int sp_set_noise(sp_sim* sim, const double* xi_host);
/* Raw counter-based generator (Philox4x64-10, Salmon et al. SC'11), for
 * checking: out_host[4 * k ...] = Philox(ctr = (ids[k], step, 0, 0), key = (seed, 0)). */
int sp_philox_blocks(int32_t device, uint64_t seed, uint64_t step, int64_t count,
                     const int64_t* ids_host, uint64_t* out_host);
/* The thermal normals of Eq. F (Box-Muller on the Philox block above: two
 * 53-bit uniforms per pair) for particle ids at `step`, as a simulation of
 * the given precision draws them: SP_PREC_FP64 in FP64, SP_PREC_MIXED in
 * double-float arithmetic on the FP32 pipes (within ~1e-13 of the FP64
 * ones).  out_host[3 * k + c], for checking.  Errors: SP_ERR_INVALID_ARG,
 * SP_ERR_NO_DEVICE, SP_ERR_OOM, SP_ERR_CUDA. */
int sp_normals(int32_t device, uint64_t seed, uint64_t step, int64_t count, const int64_t* ids_host,
               int32_t precision, double* out_host);

/* ---- learned warm start ----
 *
 * The paper solves Eq. algebra with no learned part; this optional network
 * guesses the velocities before CG, which then runs from the guess to the
 * same tolerance (CG alone decides convergence).  For node i and Cartesian
 * component c, with shared weights: s = RMS of b; x0 = (b/A_ii, vprev, b)/s;
 * a0 = M x0 with (M u)_i = sum_j alpha w_ij / A_ii u_j; y = tanh(tanh([x0,a0] W1)
 * W2) W3 (6 -> 64 -> 64 -> 4, BF16 tensor cores, FP32 accumulation); a1 = M y;
 * guess = s [y, a1, x0] . o.  Flat FP32 weights: W1 [6][64], W2 [64][64],
 * W3 [64][4], o [11], row-major in that order (sp_mpnn_num_params() floats).
 * Training minimises the mean square of (guess - v*)/s over the rows, v* the
 * converged velocities, with Adam on FP32 master weights. */
int sp_mpnn_num_params(void);
/* Attach the network (weights_host: sp_mpnn_num_params() floats, or NULL for
 * a seeded start whose readout returns the previous velocities); from then on
 * every step runs it before the solve and CG starts from its guess. */
int sp_mpnn_enable(sp_sim* sim, uint64_t seed, const float* weights_host);
int sp_mpnn_disable(sp_sim* sim);
/* use_vprev = 0: the network's previous-velocity feature is 0 in every
 * inference and training step from now on (a network trained that way maps a
 * right-hand side alone to its solution, as the preconditioner of
 * sp_solve_flexible applies it); 1 (the default after sp_mpnn_enable): the
 * feature is the previous velocities.  Errors: SP_ERR_INVALID_ARG. */
int sp_mpnn_set_prior(sp_sim* sim, int32_t use_vprev);
int sp_mpnn_get_weights(sp_sim* sim, float* weights_host);
int sp_mpnn_set_weights(sp_sim* sim, const float* weights_host);
/* Run the network on the assembled system (after sp_assemble); its guess
 * becomes the start vector of the next sp_solve_velocities.  guess_host:
 * [n][3] by particle id, or NULL. */
int sp_mpnn_forward(sp_sim* sim, double* guess_host);
/* One training step on the last solve (call after sp_step(sim, 1), or after
 * sp_mpnn_forward then sp_solve_velocities): loss of the guess against the
 * converged velocities, gradient (grad_host may be NULL), Adam with learning
 * rate lr (lr = 0 computes the gradient only). */
int sp_mpnn_train_step(sp_sim* sim, float lr, double* loss, float* grad_host);

/* ---- batches of independent replicas ----
 *
 * Ensembles of simulations with their own box, particle count, shear rate
 * and seed, advanced together: one time step of the whole batch is one CUDA
 * graph whose pair searches and assemblies run as parallel branches and
 * whose velocity solves of all replicas are one cooperative persistent launch
 * (blocks shared out in proportion to each replica's rows; every replica
 * keeps its own CG scalars and convergence).  Every replica must use
 * SP_PREC_MIXED on the same device; params[k].stream is ignored (the batch
 * owns its stream). */
typedef struct sp_batch sp_batch;

/* R replicas (1 <= R <= 4096); pos_host: NULL, or R pointers to [n_k][3]
 * initial positions (entries may be NULL for positions drawn from the seed). */
int sp_batch_create(int32_t R, const sp_params* params, const double* const* pos_host, sp_batch** out);
int sp_batch_destroy(sp_batch* b);
/* nsteps steps of every replica; info: NULL or [R] step infos.  A replica whose
 * pair storage overflows is regrown and catches up on its own. */
int sp_batch_step(sp_batch* b, int32_t nsteps, sp_step_info* info);
/* Replica k as a simulation handle for state access (owned by the batch;
 * never pass it to sp_sim_destroy). */
int sp_batch_get_sim(sp_batch* b, int32_t k, sp_sim** sim);
/* Blocks of the cooperative launch given to each replica, [R]. */
int sp_batch_blocks(sp_batch* b, int32_t* blocks);
/* Tile configuration of the batched solver, chosen by timing (not in the
 * paper; an implementation parameter): the batched solve runs in several
 * compiled configurations (gathers in flight per thread, resident blocks per
 * SM, threads per block: 256, 512 or 1024; fewer, larger blocks give each
 * replica fewer blocks to synchronise), and the blocks of the cooperative
 * launch are shared out in proportion to the replicas' rows within that
 * configuration's co-resident capacity.  sp_batch_autotune builds every
 * replica's pair list and system for its current positions, times `trials`
 * batched solves from a zero start per configuration (CUDA events on the
 * batch's stream), keeps the fastest and re-shares the blocks; positions,
 * offsets, step counters and the previous velocities are unchanged.
 * info (may be NULL): chosen config, its gathers_in_flight, blocks_per_sm and
 * block_threads, num_configs, and ms[k] the best solve time of configuration
 * k (0: not timed, e.g. fewer resident blocks than replicas).  trials < 1
 * keeps the current configuration.  The configurations round the dot
 * products differently (results agree to ~1e-13 relative); each is
 * deterministic.  sp_batch_set_config selects configuration `config` without
 * timing.  Errors: SP_ERR_INVALID_ARG, SP_ERR_CUDA, and those of a build. */
int sp_batch_autotune(sp_batch* b, int32_t trials, sp_tune_info* info);
int sp_batch_set_config(sp_batch* b, int32_t config);
const char* sp_batch_last_error(const sp_batch* b);

/* ---- allocation-free solve ----
 *
 * No counterpart in the paper: an entry point for callers that cannot
 * allocate device memory (a host framework that owns every device allocation
 * through its own pool, a real-time loop that forbids allocation after
 * start-up, or an embedding that must not touch the caller's allocator).
 *
 * Solves (A (x) I_3) x = b by Jacobi-preconditioned CG in FP64 from x = 0,
 * stopping at ||b - A x||_2 <= tol ||b||_2 (checked on the exactly recomputed
 * residual), for A = diag - alpha W with W given in CSR (off-diagonal weights
 * only; A_ij = -alpha w_ij; A must be symmetric positive definite):
 *   row_ptr_dev [n+1], col_dev [nnz] (int32), w_dev [nnz], diag_dev [n] (A_ii),
 *   b_dev [3][n] and x_dev [3][n] (x, y, z planes) — all caller-owned device
 *   memory on `device`; x_dev is overwritten.  stream: a cudaStream_t or NULL.
 *   row_ptr must start at 0 and never decrease, and every col entry must lie
 *   in [0, n); a call that breaks either returns SP_ERR_INVALID_ARG before
 *   any gather through the CSR (row_ptr[n] itself is the caller's to bound by
 *   the real length of col_dev and w_dev).
 *
 * It allocates nothing: its working vectors live in one fixed device array
 * (about 3.2 MB) that every device context loading this library holds until
 * the process exits.  Hence:
 *   - n must be <= 32768, else SP_ERR_INVALID_ARG (sp_last_error(NULL) says why);
 *   - every call on a device shares that array, so calls that may overlap on
 *     the GPU (several streams or host threads) race; serialise them;
 *   - the first call on a device looks up the array's address with that device
 *     current (the caller's current device is restored);
 *   - every call reads the solver state back and synchronises `stream`, so it
 *     can never be made while that stream is being captured into a CUDA graph
 *     (such a call returns SP_ERR_INVALID_ARG and leaves the capture intact);
 *   - device must be in [0, 63].
 * Returns SP_OK; SP_ERR_INVALID_ARG (n, a pointer, tol, max_iter, alpha or
 * device out of range, a malformed CSR, a capturing stream); SP_ERR_NOT_CONVERGED
 * when max_iter iterations are reached, or when the exactly recomputed residual
 * is still above tol after the restart limit (info->iterations is then below
 * max_iter); SP_ERR_NONFINITE; SP_ERR_NO_DEVICE; SP_ERR_CUDA.  info (may be
 * NULL) receives iterations and the true residual. */
int sp_solve_csr_noalloc(int32_t device, void* stream, int64_t n, const int32_t* row_ptr_dev,
                         const int32_t* col_dev, const double* w_dev, const double* diag_dev, double alpha,
                         const double* b_dev, double* x_dev, double tol, int32_t max_iter,
                         sp_solve_info* info);

#ifdef __cplusplus
}
#endif

#endif /* SHEARSIM_H */
