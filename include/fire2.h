/*
 * fire2.h -- C ABI of the GB300 FIRE 2.0 relaxation library.
 *
 * The library relaxes one atomistic configuration to a local energy minimum
 * with FIRE 2.0 (Guenole et al., Algorithm 2), integrated with the
 * semi-implicit Euler scheme of Algorithm 4 and the parameters of Table 1.
 * Every iteration of the relaxation -- neighbour-list maintenance, the force
 * evaluation F = -grad E (Sec. 2.1), the reductions of P = F.v, |F|^2, |v|^2
 * and the stopping norms (Sec. 3.4), the dt / alpha control, the half step
 * back on P <= 0, and the mixing + integration -- runs on the GPU; the host
 * launches one CUDA graph per call and reads the result once at the end.
 *
 * Conventions for every entry point:
 *   - Every function returns a fire_status and never throws or aborts across
 *     the ABI.  On failure, fire_last_error(h) returns a message that stays
 *     valid until the next call on the same handle.
 *   - Host buffers are owned by the caller; the library copies in and out
 *     and keeps no caller pointer after returning.  Device buffers passed to
 *     the *_dev variants are owned by the caller and must stay valid until
 *     the call returns (the call synchronises its stream before returning).
 *   - The handle owns all device memory it allocates (fire_init) and frees
 *     it in fire_destroy.  A handle must not be used by two threads at once.
 *   - Positions are N x 3 row-major doubles (x0 y0 z0 x1 y1 z1 ...).  Boxes
 *     are orthorhombic with lengths box[3]; a periodic axis must be at least
 *     twice the interaction cut-off long (minimum-image convention).  On an
 *     open axis the length only sets the extent of the cell grid of the
 *     neighbour search: atoms may lie outside [0, L) there (they share the
 *     edge cells, which costs time, not correctness).
 *   - Units are the caller's.  `mass` is expressed so that the acceleration
 *     is F / mass (for metal units with masses in amu divide the mass by
 *     9648.533212 to get eV ps^2 / A^2).
 */
#ifndef FIRE2_GB300_H
#define FIRE2_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FIRE2_ABI_VERSION 9

typedef enum {
    FIRE_OK = 0,
    FIRE_ERR_ARG = 1,           /* invalid argument (NULL, size, box, parameter) */
    FIRE_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    FIRE_ERR_NOMEM = 3,         /* device or host allocation failed */
    FIRE_ERR_NONFINITE = 4,     /* a force, energy or position became NaN/Inf */
    FIRE_ERR_NBR_OVERFLOW = 5,  /* a neighbour list or cell exceeded its capacity */
    FIRE_ERR_TIMEOUT = 6,       /* the device loop exceeded its wall-clock budget */
    FIRE_ERR_STATE = 7,         /* call not valid for this handle (e.g. wrong size) */
    FIRE_ERR_NOT_CONVERGED = 8  /* an inner iterative solve stopped before its tolerance */
} fire_status;

/* Stop reasons (Algorithm 2 and Sec. 3.4). */
typedef enum {
    FIRE_STOP_FTOL = 0,         /* force norm fell below ftol ("converged") */
    FIRE_STOP_MAXITER = 1,      /* maxiter iterations done */
    FIRE_STOP_MAXVDOTF = 2      /* more than vdfmax consecutive passes with P <= 0 */
} fire_stop;

/* Force norm used by the convergence test (Sec. 3.4). */
typedef enum {
    FIRE_NORM_MAX_ATOM = 0,     /* max_i |F_i| (Euclidean per atom) */
    FIRE_NORM_TWO = 1,          /* f2norm: Euclidean norm of the 3N force vector */
    FIRE_NORM_INF = 2           /* largest Cartesian force component */
} fire_norm;

typedef enum {
    FIRE_POT_LJ = 0,            /* 12-6 Lennard-Jones, energy shifted to 0 at rc */
    FIRE_POT_RGL = 1,           /* second-moment (RGL) EAM, quintic taper on [rs, rc) */
    FIRE_POT_SW = 2             /* Stillinger-Weber three-body (Sec. 4 case 5 family), FP64 */
} fire_pot_kind;

/* How the RGL pair functions phi(r), g(r) and their derivatives are
 * evaluated.  FIRE_PAIR_TABLE: piecewise quintic Hermite polynomials in
 * u = r^2 - r0^2 (knots every ~0.04 A^2, on rs and rc, matching value, first
 * and second derivative at every knot; interpolation error ~1e-13 relative
 * for values, ~1e-11 for derivatives), no square root or exponential per
 * pair; pairs closer than r0/2 use the analytic functions.  In the FP64
 * precision the table terms are computed from exact fixed-point separations
 * (2^-44 A) in double-float arithmetic (float pairs, ~2^-44 relative), with
 * FP64 sums, reductions and integration.
 * FIRE_PAIR_ANALYTIC: the exponentials and the taper per pair, IEEE FP64 in
 * the FP64 precision. */
typedef enum {
    FIRE_PAIR_TABLE = 0,
    FIRE_PAIR_ANALYTIC = 1
} fire_pair_eval;

/* Neighbour lists of the FP64 tabulated form (other forms ignore it).
 * FIRE_NEWTON_ON: each pair once (half list), its terms added to both atoms
 * by FP64 atomics.  FIRE_NEWTON_OFF: full list, every pair from both ends,
 * no atomics (results reproducible bit for bit).  FIRE_NEWTON_AUTO: the
 * library's default for this part (FIRE_NEWTON_ON). */
typedef enum {
    FIRE_NEWTON_AUTO = 0,
    FIRE_NEWTON_ON = 1,
    FIRE_NEWTON_OFF = 2
} fire_newton;

typedef enum {
    FIRE_PREC_FP64 = 0,         /* FP64 results: positions, densities, forces, energies,
                                   reductions, control and integration in FP64.  The
                                   pair terms follow pot.pair_eval: with the default
                                   FIRE_PAIR_TABLE they are double-float (float pairs,
                                   ~2^-44 relative) from table interpolation on exact
                                   fixed-point separations; FIRE_PAIR_ANALYTIC computes
                                   them with IEEE-FP64 exponentials */
    FIRE_PREC_FP32_PAIR = 1     /* pair/embedding math in FP32; positions, sums, control FP64 */
} fire_precision;

/* Integrators of the appendix (Algorithms 3-6); Sec. 3.1 compares them. */
typedef enum {
    FIRE_INT_EULER_IMPLICIT = 0, /* Algorithm 4, semi-implicit (symplectic) Euler (default) */
    FIRE_INT_EULER_EXPLICIT = 1, /* Algorithm 3, explicit Euler: mix v(t), x += dt v(t),
                                    v += dt F(x(t)) / m */
    FIRE_INT_VERLET = 2,         /* Algorithm 6, velocity Verlet */
    FIRE_INT_LEAPFROG = 3        /* Algorithm 5, Leapfrog: as Algorithm 4 with the initial
                                    v(-dt/2) = -dt/2 F / m in place of v = 0 */
} fire_integrator;

/* How an FP32-pair relaxation reaches an FP64-checked ftol
 * (fire_params_t.confirm64; the paper's stopping test at tight ftol is what
 * FP32 pair terms cannot settle alone: their force error, ~5e-7 eV/A at
 * relaxed Cu structures, is comparable to ftol = 1e-6).
 * FIRE_FP64_CHECK_OFF: stop on the FP32-pair forces.
 * FIRE_FP64_CHECK_CONFIRM: when the FP32-pair forces meet ftol, the same
 *   configuration is evaluated once more in FP64 (double-float table terms,
 *   full list) and the relaxation stops only if those forces meet ftol too;
 *   otherwise it tightens its FP32 threshold by the FP32-FP64 difference seen
 *   there and goes on.  Each confirmation is one force evaluation that is not
 *   an iteration.  The batched form confirms per system.
 * FIRE_FP64_CHECK_FINISH: FP32-pair forces while the force norm is at least
 *   3 ftol, FP64 forces (double-float table terms, full list) from the first
 *   evaluation below it to the end; a precision schedule (per system in the
 *   batched form).  The default: below 3 ftol the FP32-pair force error
 *   starts to steer FIRE, and with CONFIRM the number of iterations in that
 *   tail depends on the trajectory's rounding (1M-atom Cu box to 1e-6 eV/A:
 *   435 or 664 iterations after a change in the last bit of the update
 *   arithmetic) where FINISH takes 353 both times, against 349 in FP64. */
typedef enum {
    FIRE_FP64_CHECK_OFF = 0,
    FIRE_FP64_CHECK_CONFIRM = 1,
    FIRE_FP64_CHECK_FINISH = 2
} fire_fp64_check;

/* Minimizer variant. */
typedef enum {
    FIRE_VARIANT_FIRE2 = 0,      /* FIRE 2.0, Algorithm 2 (default) */
    FIRE_VARIANT_FIRE1 = 1       /* the original FIRE, Algorithm 1: mixing of v(t) at the
                                    start of a P > 0 step, dt *= f_dec, alpha reset and
                                    v = 0 on P <= 0; no N_P<=0 cap, no initial delay, no
                                    dt_min, no half step back */
} fire_variant;

typedef struct {
    int64_t n_atoms;            /* N >= 1 */
    double mass;                /* uniform mass (Sec. 2.1), > 0 */
    int32_t periodic[3];        /* 1 = periodic axis, 0 = open */
    int32_t reserved;
} fire_system_t;

typedef struct {
    int32_t kind;               /* fire_pot_kind */
    int32_t precision;          /* fire_precision */
    /* LJ: phi(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - phi(rc_lj), r < rc_lj */
    double eps, sigma, rc_lj;
    /* RGL: E_i = sum_j A e^{-p(r/r0-1)} S(r) - sqrt(sum_j xi^2 e^{-2q(r/r0-1)} S(r)),
     * S = 1 - 10t^3 + 15t^4 - 6t^5, t = (r - rs)/(rc - rs) on [rs, rc) */
    double A, xi, p, q, r0, rs, rc;
    double skin;                /* neighbour-list skin (>= 0); lists rebuilt after
                                   any atom moved more than skin/2 */
    int32_t pair_eval;          /* fire_pair_eval (RGL): FIRE_PAIR_TABLE (default) or
                                   FIRE_PAIR_ANALYTIC */
    int32_t newton;             /* fire_newton (FP64 tabulated RGL only) */
    /* SW (with eps, sigma above): E = sum_{i<j} phi2(r_ij) + sum_i sum_{j<k} phi3,
     * phi2 = sw_A eps [sw_B (sigma/r)^sw_p - (sigma/r)^sw_q] exp(sigma / (r - sw_a sigma)),
     * phi3 = sw_lambda eps (cos theta_jik + 1/3)^2 exp(sw_gamma sigma / (r_ij - sw_a sigma))
     *        exp(sw_gamma sigma / (r_ik - sw_a sigma)); cut-off sw_a sigma.  FP64 only. */
    double sw_A, sw_B, sw_p, sw_q, sw_a, sw_lambda, sw_gamma;
} fire_potential_t;

/* FIRE 2.0 parameters: Table 1 names; dt_start is the MD timestep. */
typedef struct {
    double dt_start;            /* initial timestep, > 0 */
    double tmax;                /* dt_max = tmax * dt_start          (default 10) */
    double tmin;                /* dt_min = tmin * dt_start          (default 0.02) */
    double dtgrow;              /* f_inc                             (default 1.1) */
    double dtshrink;            /* f_dec                             (default 0.5) */
    double alpha0;              /* alpha_start                       (default 0.25) */
    double alphashrink;         /* f_alpha                           (default 0.99) */
    int32_t delaystep;          /* N_delay                           (default 20) */
    int32_t vdfmax;             /* N_P<=0,max                        (default 2000) */
    int32_t halfstepback;       /* 1 = correct uphill motion         (default 1) */
    int32_t initialdelay;       /* 1 = no dt/alpha change while i < N_delay (default 1) */
    int32_t integrator;         /* fire_integrator                   (default 0) */
    int32_t norm;               /* fire_norm for the ftol test       (default 0) */
    int32_t variant;            /* fire_variant                      (default 0) */
    int32_t confirm64;          /* fire_fp64_check, FP32-pair form only (default
                                   FIRE_FP64_CHECK_FINISH) */
    double dmax;                /* maximum displacement of any atom per step (the
                                   paper's dmax, Sec. 4 cases 1 and 7), 0 = no cap
                                   (default 0): the drift x += dt v uses
                                   min(dt, dmax / max_i |v_i|); the FIRE dt is
                                   not changed by the cap */
} fire_params_t;

/* Result of a relaxation.  Energy and norms are those of the last force
 * evaluation, which for an FP32-pair relaxation stopped on ftol with an FP64
 * check (confirm64) is the FP64 one. */
typedef struct {
    double energy;              /* E at the returned positions */
    int64_t iterations;         /* completed FIRE iterations (= force evaluations - 1,
                                   less the FP64 confirmations of FP32-pair stops) */
    int64_t force_evals;        /* force evaluations including the initial one */
    int64_t nbr_builds;         /* neighbour-list builds during the call */
    int32_t stop;               /* fire_stop */
    int32_t reserved;
    double fmax_atom;           /* max_i |F_i| at the returned positions */
    double f2norm;              /* |F| of the 3N vector */
    double finf;                /* max |F_i,d| */
    double dt_final, alpha_final;
} fire_result_t;

typedef struct fire_handle fire_handle_t;

/* Fills *out with the Table 1 defaults and the given dt_start.
 * Returns FIRE_ERR_ARG if out is NULL or dt_start <= 0. */
fire_status fire_default_params(fire_params_t* out, double dt_start);

/* Creates a handle for systems of sys->n_atoms atoms with the given potential
 * and FIRE parameters; allocates all device buffers on the current device.
 * Errors: FIRE_ERR_ARG (bad field), FIRE_ERR_NOMEM, FIRE_ERR_CUDA. */
fire_status fire_init(fire_handle_t** h, const fire_system_t* sys,
                      const fire_potential_t* pot, const fire_params_t* params);

/* Relaxes pos (host, N x 3, in/out) in box[3] until the chosen force norm is
 * below ftol, maxiter iterations are done, or MAXVDOTF triggers (Alg. 2).
 * pos is overwritten only when FIRE_OK is returned; a MAXITER or MAXVDOTF stop
 * is FIRE_OK with out->stop set.  out may not be NULL.  pos in page-locked
 * host memory (cudaMallocHost, cudaHostRegister) is copied to and from the
 * device directly; other host memory takes a staging copy on the way back.
 * Errors: FIRE_ERR_ARG (ftol < 0, maxiter < 0, box), FIRE_ERR_NONFINITE,
 * FIRE_ERR_NBR_OVERFLOW, FIRE_ERR_TIMEOUT, FIRE_ERR_CUDA. */
fire_status fire_minimize(fire_handle_t* h, double* pos, const double box[3], double ftol,
                          int64_t maxiter, fire_result_t* out);

/* Same as fire_minimize with pos on the device (N x 3 doubles, in/out),
 * running on `stream` (a cudaStream_t, NULL = legacy default stream).  The
 * call returns after the stream has finished the relaxation. */
fire_status fire_minimize_dev(fire_handle_t* h, double* d_pos, const double box[3], double ftol,
                              int64_t maxiter, fire_result_t* out, void* stream);

/* One force evaluation F = -grad E (Sec. 2.1) at pos (host, N x 3).
 * forces (host, N x 3) may be NULL; energy may be NULL.
 * Errors: FIRE_ERR_ARG, FIRE_ERR_NONFINITE, FIRE_ERR_NBR_OVERFLOW, FIRE_ERR_CUDA. */
fire_status fire_energy_forces(fire_handle_t* h, const double* pos, const double box[3],
                               double* forces, double* energy);

/* Device-pointer variant: d_pos, d_forces (N x 3 doubles) and d_energy (one
 * double) are device buffers; d_forces / d_energy may be NULL. */
fire_status fire_energy_forces_dev(fire_handle_t* h, const double* d_pos, const double box[3],
                                   double* d_forces, double* d_energy, void* stream);

/* How fire_minimize drives the iterations on the device. */
typedef enum {
    FIRE_EXEC_GRAPH_WHILE = 0,  /* one CUDA graph with a conditional WHILE node (default):
                                   no host synchronisation until the relaxation ends */
    FIRE_EXEC_CHUNKED = 1       /* plain CUDA graphs of `chunk` iterations; the host reads
                                   the stop flag once per chunk (for profilers, which
                                   cannot look inside conditional graphs) */
} fire_exec_mode;

/* Selects the execution mode of later fire_minimize* calls on h.  chunk is,
 * in FIRE_EXEC_CHUNKED, the number of iterations per graph launch (1..4096);
 * in FIRE_EXEC_GRAPH_WHILE, the number of iterations per launch of the WHILE
 * node's body (0..64), each with its cell-list build and the FP64 confirming
 * passes of FP32-pair handles under conditional IF nodes (an all-pairs list
 * build, used for boxes under three cells per axis, is launched in every
 * iteration and returns at once unless due; iterations past the stop return
 * at once too); 0 (the default) takes 8.  Results do not depend on the mode.
 * The paper has no counterpart (it describes the loop of Algorithm 2, not how
 * it is driven).  Errors: FIRE_ERR_ARG. */
fire_status fire_set_exec_mode(fire_handle_t* h, int32_t mode, int32_t chunk);

/* Threads per atom in the RGL pair passes of the FP64 table form and of the
 * FP32-pair form with exponentials, and in the LJ force pass: tpa = 1, 2, 4,
 * 8, 16 or 32, or 0 for the
 * automatic choice, which handles start with (the fewest that give a pass at
 * least 1024 threads per SM in the FP64 form, 512 in the FP32-pair form, at
 * most 8 for RGL and 32 for LJ: on a 152-SM device one thread per atom from
 * about 155,000 and 78,000 atoms, 8 below about 39,000 and 19,000, and for
 * LJ 32 below about 4,900 atoms).  The threads of an atom
 * take every tpa-th entry of its neighbour list and their partial sums are
 * added in FP64, so results change only in the rounding of the per-atom sums
 * (far below the FP64 form's 1e-10 relative force error).  Other forms run
 * one thread per atom and report 1.  *chosen (may be NULL) receives the value
 * in effect.  Applies to later calls on h; the paper has no counterpart (it
 * does not say how force evaluation is parallelised).
 * Errors: FIRE_ERR_ARG (another tpa; batched handles, which take their launch
 * shape from fire_batch_set_tuning). */
fire_status fire_set_threads_per_atom(fire_handle_t* h, int32_t tpa, int32_t* chosen);

/* Shared-memory tiles of the FP64 form's half-list passes (pot.precision =
 * FIRE_PREC_FP64, pair_eval = FIRE_PAIR_TABLE, newton on; other forms ignore
 * the setting).  F = -grad E (Sec. 2.1) on a half list owes each pair's term
 * to both atoms.  With tiles the atoms are taken brick of cells by brick of
 * cells (4 x 4 x 2 list cells): a brick's atoms and every neighbour their
 * lists name are staged in shared memory, the neighbours' terms are summed
 * there exactly (two 32-bit fixed-point words per component, 2^-40 units),
 * and each staged atom's sum goes to global memory with one FP64 atomic per
 * component, in place of one per pair.  Neighbours beyond stage_cap distinct
 * atoms per brick, and terms of 15 or more (eV/A) per component, take the
 * per-pair FP64 atomics.  Forces and densities agree with the untiled
 * passes to the rounding of their sums (well inside the 1e-10 relative
 * force bar).  mode: FIRE_TILES_ON (whenever the list is in cell mode and
 * the handle holds one system), FIRE_TILES_OFF, or FIRE_TILES_AUTO (the
 * default: the library's choice, which is the untiled passes -- on GB300
 * both passes are bound by the issue of their double-float arithmetic, and
 * the tiles' staging and fixed-point splits cost more issue than the FP64
 * additions and atomics they remove: 0.60 against 0.51 ms for the force
 * pass of the 1M-atom box).  stage_cap: 0 for the largest
 * stage (1920 atoms), else 64..1920 (smaller stages send more pairs down
 * the per-pair path; a testing aid).  Applies to later calls on h; the
 * paper has no counterpart.  Errors: FIRE_ERR_ARG (mode, stage_cap, batched
 * handle). */
typedef enum {
    FIRE_TILES_AUTO = 0,
    FIRE_TILES_ON = 1,
    FIRE_TILES_OFF = 2
} fire_tiles;
fire_status fire_set_pair_tiles(fire_handle_t* h, int32_t mode, int32_t stage_cap);

/* Wall-clock budget of one device relaxation loop (default 3600 s, 0 = none).
 * When exceeded, the loop stops at the next iteration boundary and the call
 * returns FIRE_ERR_TIMEOUT.  Errors: FIRE_ERR_ARG (h NULL or seconds < 0). */
fire_status fire_set_time_budget(fire_handle_t* h, double seconds);

/* Frozen degrees of freedom for later fire_minimize* calls on h (Sec. 4,
 * cases 1 and 7: border atoms frozen in x and y).  mask: host, one byte per
 * atom, bit d (0 = x, 1 = y, 2 = z) set = that component is frozen; the
 * library copies it.  Frozen force components are set to zero after every
 * force evaluation of a relaxation, so they enter neither P, the force norms
 * (ftol test, result norms) nor the motion.  fire_energy_forces* still
 * return the full forces.  mask = NULL frees every component again.
 * Errors: FIRE_ERR_ARG (h NULL, a batched handle, a byte above 7),
 * FIRE_ERR_NOMEM / FIRE_ERR_CUDA. */
fire_status fire_set_dof_mask(fire_handle_t* h, const uint8_t* mask);

/* Stages timed by fire_profile_stages. */
typedef enum {
    FIRE_STAGE_BUILD = 0,       /* cell binning + neighbour-list build */
    FIRE_STAGE_DENSITY = 1,     /* RGL density pass (0 for LJ) */
    FIRE_STAGE_EMBED = 2,       /* RGL embedding derivative (0 for LJ) */
    FIRE_STAGE_FORCE = 3,       /* force pass (RGL pass 2, or LJ) */
    FIRE_STAGE_REDUCE = 4,      /* FP64 reductions of P, |F|^2, |v|^2, max|F_i|, with the
                                   scalar FIRE control (Algorithm 2) in the same launch */
    FIRE_STAGE_CONTROL = 5,     /* ~0: the control runs in the last block of the reduction
                                   launch (for NEB handles, of the projection launch), whose
                                   time FIRE_STAGE_REDUCE holds */
    FIRE_STAGE_UPDATE = 6,      /* element-wise half step back / kick / mix / drift */
    FIRE_NSTAGES = 7
} fire_stage;

/* Diagnostic: runs the kernels of one relaxation iteration `reps` times at
 * pos (host, N x 3) on the handle's stream, each kernel bracketed by CUDA
 * events, and writes the mean device time of each stage in milliseconds to
 * stage_ms[FIRE_NSTAGES].  The neighbour list is rebuilt in every repetition
 * (so FIRE_STAGE_BUILD is the cost of one rebuild); the update runs with
 * dt = 0 so the positions stay fixed.  The paper has no counterpart (its cost
 * metric is the number of force evaluations, Sec. 5.3).
 * Errors: as fire_energy_forces; FIRE_ERR_ARG if reps < 1 or stage_ms NULL. */
fire_status fire_profile_stages(fire_handle_t* h, const double* pos, const double box[3],
                                int32_t reps, double* stage_ms);

/* Diagnostic: measured issue rate of dependent-free fused multiply-adds on
 * the current device, in floating-point operations per second (2 per FMA):
 * which = 0 for FP64, 1 for FP32.  Used as the ALU roofline denominator of
 * the force kernels.  The paper has no counterpart.
 * Errors: FIRE_ERR_ARG (which, out), FIRE_ERR_CUDA. */
fire_status fire_diag_fma_peak(int32_t which, double* flops_per_s);

/* Energy and forces of one configuration without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc when they need forces -- plug-ins whose host
 * program's memory pool owns all device memory and forbids stray
 * allocations, and latency-critical loops where an allocation could
 * synchronise the device or fail under memory pressure.
 * It needs no handle: the caller passes the potential, the periodic flags,
 * device buffers d_pos (n_atoms x 3 doubles, row-major, read) and d_forces
 * (n_atoms x 3, written; may be NULL) and d_energy (one double, written; may
 * be NULL), and the stream to run on (a cudaStream_t, NULL = legacy default).
 * The call only enqueues kernels; the results are ready when the stream is.
 * Forces come from an all-pairs (minimum-image) sum, FP64 only.
 * Scratch: a static device array inside the library sized for at most 32768
 * atoms (~0.5 MiB, held by every GPU that loads the library until the
 * process exits).  It is shared by all calls and keeps the last call's
 * contents; every value a call reads is written earlier in the same call, so
 * nothing needs clearing between calls, but calls that overlap on the GPU
 * race on it and must be serialised by the caller.  The first call on each
 * device, and the first after a device reset (a new context), looks up the
 * array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture on that device.  A CUDA error left pending by
 * the caller's earlier work is neither reported as this call's nor cleared.
 * Errors (message in fire_last_error(NULL)): FIRE_ERR_ARG for NULL
 * arguments, n_atoms outside [1, 32768], precision other than FP64, bad
 * potential parameters or a periodic box shorter than twice the cut-off;
 * FIRE_ERR_CUDA if a CUDA call or a kernel launch fails. */
fire_status fire_energy_forces_noalloc(const fire_potential_t* pot, int64_t n_atoms,
                                       const int32_t periodic[3], const double* d_pos,
                                       const double box[3], double* d_forces, double* d_energy,
                                       void* stream);

/* Diagnostic: evaluates the library's FP64 exponential (the table-driven
 * method of P. T. P. Tang, ACM TOMS 15(2), 1989, used by the RGL pair terms)
 * at n points: d_x and d_out are device arrays of n doubles; valid for
 * |x| < 700.  Synchronises `stream` before returning.  The paper has no
 * counterpart.  Errors: FIRE_ERR_ARG, FIRE_ERR_NOMEM, FIRE_ERR_CUDA. */
fire_status fire_diag_exp(int64_t n, const double* d_x, double* d_out, void* stream);

/* ---- Batched form ----------------------------------------------------------
 * Hundreds of independent relaxations (Algorithm 2 + Algorithm 4 each, with
 * its own dt, alpha, counters, neighbour list and stop reason) of uneven atom
 * counts in one persistent kernel launch: each CTA takes the next system from
 * a device queue (largest first) and relaxes it to its own stop.  RGL
 * potential only; FP64 or FP32-pair precision as in fire_potential_t, and in
 * FP64 the pair evaluation of pot->pair_eval (FIRE_PAIR_TABLE: double-float
 * table terms on exact fixed-point separations, as in the single-system
 * FP64 form; FIRE_PAIR_ANALYTIC: IEEE-FP64 exponentials).  The
 * paper relaxes one configuration per run; the batch is this library's
 * throughput form (e.g. for ensembles of defect configurations). */

/* Launch shape of the batched kernel. */
typedef struct {
    int32_t threads_per_block;  /* multiple of 32 in [32, 1024] (default 256);
                                   above 512 only without clusters and with
                                   threads_per_block x ctas_per_sm <= 1024.
                                   The kernel exists in three register budgets:
                                   128 registers per thread (up to 512 threads
                                   per SM), 80 (768) and 64 (1024); a tuning
                                   without clusters runs the smallest budget
                                   that holds threads_per_block x ctas_per_sm
                                   threads, or the 128-register one when that
                                   product exceeds 1024 (fewer CTAs are then
                                   resident); clusters always run the
                                   128-register one */
    int32_t ctas_per_sm;        /* resident CTAs per SM, 1..32 (default 2) */
    int32_t cluster_size;       /* CTAs per thread-block cluster sharing each system:
                                   1 (or 0): one CTA per system; 2, 4 or 8: the
                                   cluster splits every system's atoms and combines
                                   its reductions through distributed shared memory */
    int32_t reserved;
} fire_batch_tuning_t;

/* Creates a batched handle for n_sys systems; system s owns atoms
 * atom_offsets[s] .. atom_offsets[s+1]-1 of the packed position arrays
 * (atom_offsets has n_sys + 1 entries, atom_offsets[0] = 0, every system
 * >= 1 atom).  sys->mass and sys->periodic apply to every system
 * (sys->n_atoms is ignored).  Only fire_minimize_batch*, fire_batch_* and
 * fire_destroy / fire_last_error / fire_set_time_budget accept the handle.
 * Errors: FIRE_ERR_ARG, FIRE_ERR_NOMEM, FIRE_ERR_CUDA. */
fire_status fire_batch_init(fire_handle_t** h, int32_t n_sys, const int64_t* atom_offsets,
                            const fire_system_t* sys, const fire_potential_t* pot,
                            const fire_params_t* params);

/* Relaxes every system of the batch: pos (host, packed N_total x 3, in/out),
 * boxes (host, n_sys x 3 orthorhombic lengths), the shared ftol / maxiter,
 * out[n_sys] per-system results (out[s].reserved holds the system's device
 * status, 0 = ok), forces (host, packed N_total x 3, optional: forces at the
 * returned positions).  pos is written only on FIRE_OK; the call fails with
 * the first system's error code if any system failed.
 * Errors: FIRE_ERR_STATE (not a batched handle), FIRE_ERR_ARG, FIRE_ERR_NONFINITE,
 * FIRE_ERR_NBR_OVERFLOW, FIRE_ERR_TIMEOUT, FIRE_ERR_CUDA. */
fire_status fire_minimize_batch(fire_handle_t* h, double* pos, const double* boxes, double ftol,
                                int64_t maxiter, fire_result_t* out, double* forces);

/* Device-pointer variant: d_pos and d_forces (optional) are device buffers of
 * N_total x 3 doubles, boxes and out stay on the host; runs on `stream` and
 * synchronises it before returning. */
fire_status fire_minimize_batch_dev(fire_handle_t* h, double* d_pos, const double* boxes,
                                    double ftol, int64_t maxiter, fire_result_t* out,
                                    double* d_forces, void* stream);

/* Sets the launch shape of later batched calls.  Errors: FIRE_ERR_STATE, FIRE_ERR_ARG. */
fire_status fire_batch_set_tuning(fire_handle_t* h, const fire_batch_tuning_t* tuning);

/* Autotuner: times every candidate launch shape (threads per CTA 64..512,
 * CTAs per SM 1..8, at most 2048 threads per SM, clusters of 1, 2 or 4 CTAs
 * where the device can co-schedule them; 768 threads per SM as 768 x 1,
 * 384 x 2, 256 x 3, 192 x 4 or 128 x 6; and 1024 x 1) on this batch
 * -- positions
 * pos and boxes as for fire_minimize_batch, `iters` FIRE iterations of every
 * system from the same start -- keeps the fastest for later calls and
 * returns it in *chosen (may be NULL).  pos is not modified.
 * Errors: FIRE_ERR_STATE, FIRE_ERR_ARG, FIRE_ERR_CUDA. */
fire_status fire_batch_autotune(fire_handle_t* h, const double* pos, const double* boxes,
                                int32_t iters, fire_batch_tuning_t* chosen);

/* ---- Differentiable form (RGL, FP64) ------------------------------------------
 * theta = (A, xi, p, q) are the RGL parameters of fire_potential_t.  The
 * paper treats the force field as fixed; these entry points add gradients
 * with respect to it: dE/dtheta (the hand-written backward of E(x, theta)),
 * the Hessian-vector product H u = (d^2 E / dx^2) u, and the implicit
 * gradient of a loss L(x*) of the relaxed configuration x*(theta): at a
 * minimum the forces vanish, so dL/dtheta = lambda . dF/dtheta with
 * H lambda = dL/dx, solved by conjugate gradients in FP64 with the three
 * translation modes projected out (H is singular along them).  All take
 * device arrays of N x 3 doubles (row-major) and run on `stream` (a
 * cudaStream_t), synchronising it before returning; they use a full
 * neighbour list built at d_pos on each call.  Handle: a single-system RGL
 * handle (either precision; the derivatives are always FP64). */

/* Replaces the RGL parameters A, xi, p, q of h (later relaxations and
 * evaluations use them).  Errors: FIRE_ERR_ARG (not RGL, xi <= 0, A < 0,
 * exponents out of range). */
fire_status fire_set_rgl_params(fire_handle_t* h, const double theta[4]);

/* E(x, theta) (*energy, host, may be NULL), dE/dtheta (host, 4 doubles, may
 * be NULL) and F = -dE/dx (d_forces, device, may be NULL) at d_pos.
 * Errors: FIRE_ERR_ARG, FIRE_ERR_NONFINITE, FIRE_ERR_NBR_OVERFLOW, FIRE_ERR_CUDA. */
fire_status fire_rgl_energy_grad_dev(fire_handle_t* h, const double* d_pos, const double box[3],
                                     const double theta[4], double* d_forces, double* energy,
                                     double dE_dtheta[4], void* stream);

/* d_hu = H(d_pos, theta) d_u (device arrays, N x 3).  Errors: as above. */
fire_status fire_rgl_hvp_dev(fire_handle_t* h, const double* d_pos, const double box[3],
                             const double theta[4], const double* d_u, double* d_hu,
                             void* stream);

/* Implicit gradient at a relaxed d_pos: d_g = dL/dx (device, N x 3),
 * CG until |r| <= tol |g| or maxit iterations; dL_dtheta (host, 4) receives
 * lambda . dF/dtheta, d_lambda (device, N x 3, may be NULL) the solution,
 * *cg_iters (may be NULL) the iteration count.  Returns FIRE_OK only when
 * the residual met tol.  FIRE_ERR_NOT_CONVERGED when CG stopped first:
 * either maxit iterations left |r| > tol |g|, or CG broke down (p.Hp <= 0
 * or not finite along a search direction, i.e. d_pos is not at a minimum).
 * In both cases the outputs hold the last iterate, and fire_last_error(h)
 * names the cause and the final relative residual.
 * Errors: FIRE_ERR_ARG (tol <= 0, maxit < 1, NULL), FIRE_ERR_NONFINITE (d_g),
 * FIRE_ERR_NOT_CONVERGED, FIRE_ERR_NBR_OVERFLOW, FIRE_ERR_CUDA. */
fire_status fire_rgl_implicit_grad_dev(fire_handle_t* h, const double* d_pos, const double box[3],
                                       const double theta[4], const double* d_g, double tol,
                                       int64_t maxit, double dL_dtheta[4], double* d_lambda,
                                       int64_t* cg_iters, void* stream);

/* Diagnostic, host only (no GPU needed): evaluates the FP64 pair-function
 * table the library builds for pot at n distances r (host arrays) into
 * out[4 n] = (phi, g, dphi/dr, dg/dr) per distance, zero at r >= rc.  The
 * paper has no counterpart.  Errors: FIRE_ERR_ARG. */
fire_status fire_diag_rgl_table(const fire_potential_t* pot, int64_t n, const double* r,
                                double* out);

/* ---- Nudged elastic band (Sec. 4, cases 7 and 8) ------------------------
 * FIRE 2.0 relaxation of an ensemble of n_img movable images of one system
 * between two fixed end states "with modified forces".  The paper cites
 * Sheppard et al. (2008) and states no formulas; the library uses that
 * reference's standard forces: the improved tangent of Henkelman and Jonsson
 * (2000) from the neighbouring images and energies, F - (F.t) t plus the
 * spring force k (|R_{i+1} - R_i| - |R_i - R_{i-1}|) t, and optionally a
 * climbing image (the movable image of highest energy: F - 2 (F.t) t).  All
 * movable images form one system for FIRE (one dt, alpha and P), and the
 * stopping norm is taken over every image. */

/* Creates a NEB handle for n_img >= 1 movable images of sys->n_atoms atoms
 * each (n_img x n_atoms <= 2^25 - 1); k_spring >= 0 (energy / length^2);
 * climb != 0 enables the climbing image.  fire_set_dof_mask takes one
 * image's mask (n_atoms bytes) and applies it to every image;
 * fire_set_time_budget and fire_set_exec_mode apply as for single systems.
 * Errors: FIRE_ERR_ARG, FIRE_ERR_NOMEM, FIRE_ERR_CUDA. */
fire_status fire_neb_init(fire_handle_t** h, int32_t n_img, const fire_system_t* sys,
                          const fire_potential_t* pot, const fire_params_t* params,
                          double k_spring, int32_t climb);

/* Relaxes the band.  path: host, (n_img + 2) x n_atoms x 3 row-major, image 0
 * and image n_img + 1 are the fixed end states (read only), images 1..n_img
 * are relaxed in place (updated only on FIRE_OK).  energies: host, n_img + 2
 * values out (may be NULL); climber: out, the index 1..n_img of the climbing
 * image at the last evaluation, 0 without climbing (may be NULL).
 * out->energy is the sum of the movable images' energies, the norms are
 * those of the NEB forces.  Errors: as fire_minimize, FIRE_ERR_STATE for a
 * handle not made by fire_neb_init. */
fire_status fire_neb_minimize(fire_handle_t* h, double* path, const double box[3], double ftol,
                              int64_t maxiter, fire_result_t* out, double* energies,
                              int32_t* climber);

/* As fire_neb_minimize with path on the device (same layout), ordered on
 * `stream` (cudaStream_t); energies and climber are host pointers. */
fire_status fire_neb_minimize_dev(fire_handle_t* h, double* d_path, const double box[3],
                                  double ftol, int64_t maxiter, fire_result_t* out,
                                  double* energies, int32_t* climber, void* stream);

/* Message of the last failed call on h (or of the last failed fire_init when
 * h is NULL).  Never NULL. */
const char* fire_last_error(const fire_handle_t* h);

/* Frees the handle and its device memory.  NULL is accepted. */
void fire_destroy(fire_handle_t* h);

/* FIRE2_ABI_VERSION of the loaded library. */
int32_t fire_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FIRE2_GB300_H */
