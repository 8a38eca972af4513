/*
 * FIRE 2.0 reference oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised FP64 CPU implementation of what the
 * GPU library computes.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA path.
 *
 * What it follows (Guenole et al., "Assessment and optimization of the fast
 * inertial relaxation engine (FIRE) for energy minimization in atomistic
 * simulations and its implementation in LAMMPS"):
 *   - Sec. 2.1, Eq. 1:   F = -grad E; the power P = F . v decides uphill motion.
 *   - Algorithm 2:       FIRE 2.0 control loop (counters N_P>0 / N_P<=0, dt and
 *                        alpha adaptation, N_P<=0 cap, initial delay, dt_min
 *                        guard, half step back on P <= 0).
 *   - Algorithm 4:       semi-implicit (symplectic) Euler with the mixing
 *                        placed just before the position update (Sec. 3.3);
 *                        Algorithms 3, 5, 6: explicit Euler, Leapfrog and
 *                        velocity Verlet; Algorithm 1: the original FIRE.
 *   - Table 1:           parameter names and defaults.
 *   - Sec. 3.4:          f2norm and per-atom maximum force stopping norms.
 *   - Sec. 5.2:          EAM = pair term + embedding functional of the local
 *                        density; here in the second-moment (RGL) form.
 *
 * Readings where the paper is silent or garbled (all shared with the GPU path,
 * listed again in the design notes):
 *   - Algorithm 4 writes the mixing line with v(t); it is applied to the kicked
 *     velocity, with the norm of the kicked velocity (as Algorithms 5 and 6 do).
 *   - Mixing only when P > 0 (after P <= 0, v is zeroed, so the kicked v is
 *     parallel to F and the mixing would be a no-op).
 *   - The half step back uses the dt after the shrink (literal order of Alg. 2).
 *   - The force is not re-evaluated after the half step back.
 *   - dt is left unchanged (not clamped) when dt*f_dec < dt_min; alpha is
 *     still reset.
 *   - Convergence is tested once before the first iteration and after each
 *     force evaluation.
 *   - Algorithm 3's velocity update is written with F(x(t+dt)) before that
 *     force is computed; it uses the force at x(t) (forward Euler, the
 *     non-symplectic scheme the paper advises against).
 *   - The Leapfrog initialisation v(-dt/2) = -dt/2 F/m of Algorithm 5 is
 *     applied once, in place of v = 0 at the start of the run.
 *   - Algorithm 1 (original FIRE) has no N_P<=0 counter, initial delay,
 *     dt_min guard or half step back, and mixes v(t) at the start of the
 *     step (before the integration) when P > 0.
 *
 * Force routines are O(N^2) all-pairs with the minimum-image convention
 * (FORCE_BRUTE).  A cell-grid variant (FORCE_CELLS) visits the same candidate
 * pairs in the same ascending-j order, so its results are bit-identical to
 * the all-pairs routine; tests check that on boxes where both run.
 *
 * Parity status per function:
 *   ora_energy_forces   pinned (finite differences, sum F = 0, zero force on
 *                       perfect lattices, closed-form cohesive energies).
 *   ora_fire2           pinned (hand-traced iterations of Alg. 2 + Alg. 4 on
 *                       quadratic wells, MAXVDOTF and dt_min traces, LJ dimer
 *                       bond length).
 *   ora_rgl_param_derivs  pinned (central differences of E and F in theta).
 *   ora_rgl_hvp         pinned (central differences of F along u, symmetry
 *                       u.Hv = v.Hu, zero translation mode).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { POT_LJ = 0, POT_RGL = 1, POT_QUAD = 2, POT_DWELL = 3, POT_SW = 4 };
enum { FORCE_BRUTE = 0, FORCE_CELLS = 1 };
enum { STOP_FTOL = 0, STOP_MAXITER = 1, STOP_MAXVDOTF = 2 };
enum { NORM_MAX_ATOM = 0, NORM_TWO = 1, NORM_INF = 2 };
enum { INT_EULER_IMPLICIT = 0, INT_EULER_EXPLICIT = 1, INT_VERLET = 2, INT_LEAPFROG = 3 };
enum { VAR_FIRE2 = 0, VAR_FIRE1 = 1 };

typedef struct {
    int64_t n;          /* number of atoms */
    double box[3];      /* orthorhombic box lengths */
    int32_t periodic[3];
    double mass;        /* uniform mass, in units where a = F / mass */
} ora_sys;

typedef struct {
    int32_t kind;
    /* Lennard-Jones 12-6, energy shifted to zero at rc */
    double eps, sigma, rc_lj;
    /* second-moment (RGL) EAM with a quintic taper on [rs, rc) */
    double A, xi, p, q, r0, rs, rc;
    /* quadratic test well E = 1/2 sum_d k_d (x_d - x0_d)^2 (control-flow tests) */
    const double *quad_k, *quad_x0;
    /* double-well test surface per atom (NEB tests), dwell = {h, a, c, ky, kz}:
     * E = h ((x/a)^2 - 1)^2 + ky (y - c x^2)^2 + kz z^2; minima (+-a, c a^2, 0)
     * with E = 0, first-order saddle (0, 0, 0) with E = h. */
    const double *dwell;
    /* Stillinger-Weber (the paper's three-body family, Sec. 4 case 5), with
     * eps and sigma above: E = sum_{i<j} phi2(r_ij) + sum_i sum_{j<k} phi3,
     * phi2 = A eps [B (sigma/r)^p - (sigma/r)^q] exp(sigma / (r - a sigma)),
     * phi3 = lambda eps (cos theta_jik + 1/3)^2
     *        exp(gamma sigma / (r_ij - a sigma)) exp(gamma sigma / (r_ik - a sigma)),
     * every term zero beyond r = a sigma. */
    double sw_A, sw_B, sw_p, sw_q, sw_a, sw_lambda, sw_gamma;
} ora_pot;

typedef struct {
    double dt_start, tmax, tmin, dtgrow, dtshrink, alpha0, alphashrink;
    int32_t delaystep, vdfmax, halfstepback, initialdelay, integrator, norm;
    int32_t variant, pad;   /* VAR_FIRE2 (Algorithm 2) or VAR_FIRE1 (Algorithm 1) */
    /* Maximum displacement of any atom per step (the paper's dmax, Sec. 4
     * cases 1 and 7); 0 = no cap.  The drift x += dt v of the step then uses
     * dt_eff = min(dt, dmax / max_i |v_i|); the FIRE dt is unchanged. */
    double dmax;
    /* Frozen degrees of freedom (Sec. 4 cases 1 and 7: borders frozen in x
     * and y): NULL, or one byte per atom with bit d set = component d
     * frozen.  Frozen force components are set to zero after every force
     * evaluation, so they enter neither P, the norms nor the motion. */
    const uint8_t *frozen;
} ora_params;

typedef struct {
    double energy;
    int64_t iterations, force_evals;
    int32_t stop, pad;
    double fmax_atom, f2norm, finf, dt_final, alpha_final;
} ora_result;

typedef struct {
    int64_t i, npos, nneg;
    double P, dt, alpha, energy, fnorm;
} ora_trace;

static double dot3n(const double *a, const double *b, int64_t n3);

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */

static double min_image(double d, double L, int periodic) {
    if (periodic) d -= L * nearbyint(d / L);
    return d;
}

static double pot_cutoff(const ora_pot *pot) {
    if (pot->kind == POT_SW) return pot->sw_a * pot->sigma;
    return pot->kind == POT_LJ ? pot->rc_lj : pot->rc;
}

/* Quintic taper S(r) = 1 - 10 t^3 + 15 t^4 - 6 t^5, t = (r - rs)/(rc - rs):
 * 1 below rs, 0 at and above rc, C2-continuous at both ends. */
static void taper(const ora_pot *pot, double r, double *S, double *dS) {
    if (r <= pot->rs) { *S = 1.0; *dS = 0.0; return; }
    if (r >= pot->rc) { *S = 0.0; *dS = 0.0; return; }
    double w = pot->rc - pot->rs;
    double t = (r - pot->rs) / w;
    *S = 1.0 - 10.0 * t * t * t + 15.0 * t * t * t * t - 6.0 * t * t * t * t * t;
    *dS = (-30.0 * t * t + 60.0 * t * t * t - 30.0 * t * t * t * t) / w;
}

/* RGL pair functions of Sec. 5.2's EAM family in second-moment form:
 *   phi(r) = A exp(-p (r/r0 - 1)) S(r)         (repulsive pair term)
 *   g(r)   = xi^2 exp(-2q (r/r0 - 1)) S(r)     (density contribution)   */
static void rgl_pair(const ora_pot *pot, double r, double *phi, double *dphi,
                     double *g, double *dg) {
    double S, dS;
    taper(pot, r, &S, &dS);
    double s = r / pot->r0 - 1.0;
    double ep = pot->A * exp(-pot->p * s);
    double eq = pot->xi * pot->xi * exp(-2.0 * pot->q * s);
    *phi = ep * S;
    *dphi = ep * (-pot->p / pot->r0 * S + dS);
    *g = eq * S;
    *dg = eq * (-2.0 * pot->q / pot->r0 * S + dS);
}

/* phi, g, phi', g' at n distances (out[4 i + 0..3]); zero at r >= rc. */
int ora_rgl_pair_terms(const ora_pot *pot, int64_t n, const double *r, double *out) {
    if (pot->kind != POT_RGL) return -1;
    for (int64_t i = 0; i < n; ++i) {
        double phi = 0.0, dphi = 0.0, g = 0.0, dg = 0.0;
        if (r[i] < pot->rc) rgl_pair(pot, r[i], &phi, &dphi, &g, &dg);
        out[4 * i] = phi;
        out[4 * i + 1] = g;
        out[4 * i + 2] = dphi;
        out[4 * i + 3] = dg;
    }
    return 0;
}

/* LJ: phi(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - phi(rc) for r < rc. */
static double lj_phi(const ora_pot *pot, double r) {
    double sr6 = pow(pot->sigma / r, 6.0);
    return 4.0 * pot->eps * (sr6 * sr6 - sr6);
}

/* ------------------------------------------------------------------------ */
/* Candidate-neighbour enumeration.  Both modes yield, for atom i, every j != i
 * in ascending order; the caller applies the cutoff test itself.             */

typedef struct {
    int mode;
    int64_t n;
    int nc[3];
    int64_t *cell_start; /* ncell + 1 */
    int64_t *cell_atoms; /* n, ascending within each cell */
} ora_grid;

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int64_t cell_coord(double x, double L, int nc) {
    double u = x / L;
    u -= floor(u);
    int64_t c = (int64_t)(u * nc);
    if (c >= nc) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

static void grid_build(ora_grid *g, const ora_sys *sys, const double *x, double rc, int mode) {
    memset(g, 0, sizeof(*g));
    g->n = sys->n;
    g->mode = FORCE_BRUTE;
    if (mode != FORCE_CELLS) return;
    for (int d = 0; d < 3; ++d) {
        if (!sys->periodic[d]) return;
        g->nc[d] = (int)floor(sys->box[d] / rc);
        if (g->nc[d] < 3) return;
    }
    g->mode = FORCE_CELLS;
    int64_t ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    g->cell_start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    g->cell_atoms = (int64_t *)malloc((size_t)(sys->n > 0 ? sys->n : 1) * sizeof(int64_t));
    int64_t *cid = (int64_t *)malloc((size_t)(sys->n > 0 ? sys->n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < sys->n; ++i) {
        int64_t cx = cell_coord(x[3 * i + 0], sys->box[0], g->nc[0]);
        int64_t cy = cell_coord(x[3 * i + 1], sys->box[1], g->nc[1]);
        int64_t cz = cell_coord(x[3 * i + 2], sys->box[2], g->nc[2]);
        cid[i] = (cx * g->nc[1] + cy) * g->nc[2] + cz;
        g->cell_start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) g->cell_start[c + 1] += g->cell_start[c];
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    memcpy(fill, g->cell_start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < sys->n; ++i) g->cell_atoms[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
}

static void grid_free(ora_grid *g) {
    free(g->cell_start);
    free(g->cell_atoms);
    memset(g, 0, sizeof(*g));
}

/* Fills cand[] with candidate j (ascending, j != i); returns the count. */
static int64_t grid_candidates(const ora_grid *g, const ora_sys *sys, const double *x,
                               int64_t i, int64_t *cand) {
    int64_t m = 0;
    if (g->mode == FORCE_BRUTE) {
        for (int64_t j = 0; j < g->n; ++j)
            if (j != i) cand[m++] = j;
        return m;
    }
    int64_t c[3];
    for (int d = 0; d < 3; ++d) c[d] = cell_coord(x[3 * i + d], sys->box[d], g->nc[d]);
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int64_t cx = (c[0] + dx + g->nc[0]) % g->nc[0];
                int64_t cy = (c[1] + dy + g->nc[1]) % g->nc[1];
                int64_t cz = (c[2] + dz + g->nc[2]) % g->nc[2];
                int64_t cc = (cx * g->nc[1] + cy) * g->nc[2] + cz;
                for (int64_t k = g->cell_start[cc]; k < g->cell_start[cc + 1]; ++k)
                    if (g->cell_atoms[k] != i) cand[m++] = g->cell_atoms[k];
            }
    qsort(cand, (size_t)m, sizeof(int64_t), cmp_i64);
    return m;
}

static int64_t grid_max_candidates(const ora_grid *g) {
    if (g->mode == FORCE_BRUTE) return g->n;
    int64_t ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2], mx = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t k = g->cell_start[c + 1] - g->cell_start[c];
        if (k > mx) mx = k;
    }
    return 27 * mx;
}

/* ------------------------------------------------------------------------ */
/* Energy and forces.  F = -grad E (Sec. 2.1).                               */

static int check_box(const ora_sys *sys, const ora_pot *pot) {
    if (sys->n < 0) return -1;
    if (pot->kind == POT_QUAD || pot->kind == POT_DWELL) return 0;
    double rc = pot_cutoff(pot);
    for (int d = 0; d < 3; ++d)
        if (sys->periodic[d] && sys->box[d] < 2.0 * rc) return -2;
    return 0;
}

/* Stillinger-Weber energy and forces (all atoms), written plainly: the pair
 * sum over j > i, then for every centre i every pair j < k of its neighbours
 * within a sigma, with the gradient of each term added to i, j and k.
 * F = -grad E (Sec. 2.1). */
static void sw_phi2(const ora_pot *pot, double r, double *e, double *de) {
    const double s = pot->sigma, rc = pot->sw_a * s;
    const double sr = s / r, bp = pot->sw_B * pow(sr, pot->sw_p), bq = pow(sr, pot->sw_q);
    const double ex = exp(s / (r - rc));
    *e = pot->sw_A * pot->eps * (bp - bq) * ex;
    /* d/dr: A eps ex [(-p bp + q bq) / r - (bp - bq) s / (r - rc)^2] */
    *de = pot->sw_A * pot->eps * ex *
          ((-pot->sw_p * bp + pot->sw_q * bq) / r - (bp - bq) * s / ((r - rc) * (r - rc)));
}

static int sw_energy_forces(const ora_sys *sys, const ora_pot *pot, const double *x, double *f,
                            double *energy, int mode) {
    const int64_t n = sys->n;
    const double rc = pot_cutoff(pot), rc2 = rc * rc, s = pot->sigma;
    ora_grid g;
    grid_build(&g, sys, x, rc, mode);
    const int64_t cap = grid_max_candidates(&g) + 1;
    int64_t *cand = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    int64_t *nb = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    double *dv = (double *)malloc((size_t)cap * 3 * sizeof(double));
    double *rv = (double *)malloc((size_t)cap * sizeof(double));
    if (f)
        for (int64_t k = 0; k < 3 * n; ++k) f[k] = 0.0;
    double etot = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t m = grid_candidates(&g, sys, x, i, cand);
        int64_t cnt = 0;
        for (int64_t c = 0; c < m; ++c) {
            const int64_t j = cand[c];
            double d[3];
            for (int a = 0; a < 3; ++a)
                d[a] = min_image(x[3 * j + a] - x[3 * i + a], sys->box[a], sys->periodic[a]);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= rc2) continue;
            const double r = sqrt(r2);
            nb[cnt] = j;
            rv[cnt] = r;
            for (int a = 0; a < 3; ++a) dv[3 * cnt + a] = d[a];
            ++cnt;
            if (j > i) {   /* pair term once per pair */
                double e2, de2;
                sw_phi2(pot, r, &e2, &de2);
                etot += e2;
                if (f)
                    for (int a = 0; a < 3; ++a) {   /* dE/dx_j = de2 d/r */
                        f[3 * j + a] -= de2 * d[a] / r;
                        f[3 * i + a] += de2 * d[a] / r;
                    }
            }
        }
        /* three-body terms centred on i */
        for (int64_t p = 0; p < cnt; ++p)
            for (int64_t q = p + 1; q < cnt; ++q) {
                const double rj = rv[p], rk = rv[q];
                const double *dj = dv + 3 * p, *dk = dv + 3 * q;
                const double cs = (dj[0] * dk[0] + dj[1] * dk[1] + dj[2] * dk[2]) / (rj * rk);
                const double ej = exp(pot->sw_gamma * s / (rj - rc));
                const double ek = exp(pot->sw_gamma * s / (rk - rc));
                const double w = cs + 1.0 / 3.0;
                const double h = pot->sw_lambda * pot->eps * w * w * ej * ek;
                etot += h;
                if (!f) continue;
                const double dh_dc = 2.0 * pot->sw_lambda * pot->eps * w * ej * ek;
                const double dh_drj = -h * pot->sw_gamma * s / ((rj - rc) * (rj - rc));
                const double dh_drk = -h * pot->sw_gamma * s / ((rk - rc) * (rk - rc));
                for (int a = 0; a < 3; ++a) {
                    const double uj = dj[a] / rj, uk = dk[a] / rk;
                    const double gj = dh_drj * uj + dh_dc * (uk - cs * uj) / rj;   /* dh/dx_j */
                    const double gk = dh_drk * uk + dh_dc * (uj - cs * uk) / rk;   /* dh/dx_k */
                    f[3 * nb[p] + a] -= gj;
                    f[3 * nb[q] + a] -= gk;
                    f[3 * i + a] += gj + gk;
                }
            }
    }
    free(cand);
    free(nb);
    free(dv);
    free(rv);
    grid_free(&g);
    *energy = etot;
    return 0;
}

/* Evaluates E and (if f != NULL) F for the atoms listed in `which` (or all
 * atoms when which == NULL).  E is always the total energy. */
static int energy_forces_impl(const ora_sys *sys, const ora_pot *pot, const double *x,
                              double *f, double *energy, int mode,
                              const int64_t *which, int64_t nwhich) {
    int rc_ok = check_box(sys, pot);
    if (rc_ok) return rc_ok;
    const int64_t n = sys->n;
    if (pot->kind == POT_QUAD) {
        double e = 0.0;
        for (int64_t k = 0; k < 3 * n; ++k) {
            double d = x[k] - pot->quad_x0[k];
            e += 0.5 * pot->quad_k[k] * d * d;
            if (f) f[k] = -pot->quad_k[k] * d;
        }
        *energy = e;
        return 0;
    }
    if (pot->kind == POT_DWELL) {
        const double h = pot->dwell[0], a = pot->dwell[1], c = pot->dwell[2];
        const double ky = pot->dwell[3], kz = pot->dwell[4];
        double e = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double X = x[3 * i], Y = x[3 * i + 1], Z = x[3 * i + 2];
            const double w = X * X / (a * a) - 1.0, y = Y - c * X * X;
            e += h * w * w + ky * y * y + kz * Z * Z;
            if (f) {
                f[3 * i] = -(4.0 * h * w * X / (a * a) - 4.0 * ky * c * X * y);
                f[3 * i + 1] = -2.0 * ky * y;
                f[3 * i + 2] = -2.0 * kz * Z;
            }
        }
        *energy = e;
        return 0;
    }
    if (pot->kind == POT_SW) {
        if (which) return -1;   /* all atoms only */
        return sw_energy_forces(sys, pot, x, f, energy, mode);
    }
    const double rc = pot_cutoff(pot), rc2 = rc * rc;
    ora_grid g;
    grid_build(&g, sys, x, rc, mode);
    const int64_t cap = grid_max_candidates(&g) + 1;

    if (pot->kind == POT_LJ) {
        const double shift = lj_phi(pot, rc);
        double etot = 0.0;
        double *ei = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel
        {
            int64_t *cand = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < n; ++i) {
                double fi[3] = {0.0, 0.0, 0.0}, e = 0.0;
                int64_t m = grid_candidates(&g, sys, x, i, cand);
                for (int64_t k = 0; k < m; ++k) {
                    int64_t j = cand[k];
                    double d[3];
                    for (int a = 0; a < 3; ++a)
                        d[a] = min_image(x[3 * i + a] - x[3 * j + a], sys->box[a], sys->periodic[a]);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 >= rc2) continue;
                    double r = sqrt(r2);
                    e += 0.5 * (lj_phi(pot, r) - shift);
                    /* -dphi/dr / r = 24 eps [2 (s/r)^12 - (s/r)^6] / r^2 */
                    double sr6 = pow(pot->sigma / r, 6.0);
                    double fpair = 24.0 * pot->eps * (2.0 * sr6 * sr6 - sr6) / r2;
                    for (int a = 0; a < 3; ++a) fi[a] += fpair * d[a];
                }
                ei[i] = e;
                if (f) for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];
            }
            free(cand);
        }
        for (int64_t i = 0; i < n; ++i) etot += ei[i];
        free(ei);
        *energy = etot;
        grid_free(&g);
        return 0;
    }

    /* RGL: pass 1 -- density rho_i and repulsive energy per atom. */
    double *rho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *erep = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *dF = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel
    {
        int64_t *cand = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            double rh = 0.0, er = 0.0;
            int64_t m = grid_candidates(&g, sys, x, i, cand);
            for (int64_t k = 0; k < m; ++k) {
                int64_t j = cand[k];
                double d[3];
                for (int a = 0; a < 3; ++a)
                    d[a] = min_image(x[3 * i + a] - x[3 * j + a], sys->box[a], sys->periodic[a]);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 >= rc2) continue;
                double phi, dphi, gg, dg;
                rgl_pair(pot, sqrt(r2), &phi, &dphi, &gg, &dg);
                er += phi;
                rh += gg;
            }
            rho[i] = rh;
            erep[i] = er;
            /* embedding F(rho) = -sqrt(rho); F'(rho) = -1 / (2 sqrt(rho)).
             * An atom with rho = 0 has no pair inside rc, so F' is never used. */
            dF[i] = rh > 0.0 ? -0.5 / sqrt(rh) : 0.0;
        }
        free(cand);
    }
    double etot = 0.0;
    for (int64_t i = 0; i < n; ++i) etot += erep[i] - sqrt(rho[i]);
    *energy = etot;

    /* pass 2 -- forces: F_k = -sum_j [2 phi'(r) + (F'_k + F'_j) g'(r)] (x_k - x_j)/r */
    if (f) {
        int64_t cnt = which ? nwhich : n;
#pragma omp parallel
        {
            int64_t *cand = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
#pragma omp for schedule(dynamic, 64)
            for (int64_t w = 0; w < cnt; ++w) {
                int64_t i = which ? which[w] : w;
                double fi[3] = {0.0, 0.0, 0.0};
                int64_t m = grid_candidates(&g, sys, x, i, cand);
                for (int64_t k = 0; k < m; ++k) {
                    int64_t j = cand[k];
                    double d[3];
                    for (int a = 0; a < 3; ++a)
                        d[a] = min_image(x[3 * i + a] - x[3 * j + a], sys->box[a], sys->periodic[a]);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 >= rc2) continue;
                    double r = sqrt(r2);
                    double phi, dphi, gg, dg;
                    rgl_pair(pot, r, &phi, &dphi, &gg, &dg);
                    double dEdr = 2.0 * dphi + (dF[i] + dF[j]) * dg;
                    for (int a = 0; a < 3; ++a) fi[a] -= dEdr * d[a] / r;
                }
                for (int a = 0; a < 3; ++a) f[3 * w + a] = fi[a];
            }
            free(cand);
        }
    }
    free(rho);
    free(erep);
    free(dF);
    grid_free(&g);
    return 0;
}

int ora_energy_forces(const ora_sys *sys, const ora_pot *pot, const double *x,
                      double *f, double *energy, int mode) {
    return energy_forces_impl(sys, pot, x, f, energy, mode, NULL, 0);
}

/* Forces of a subset of atoms (rows of f follow `which`), total energy. */
int ora_energy_forces_subset(const ora_sys *sys, const ora_pot *pot, const double *x,
                             const int64_t *which, int64_t nwhich, double *f,
                             double *energy, int mode) {
    return energy_forces_impl(sys, pot, x, f, energy, mode, which, nwhich);
}

/* Per-atom densities rho_i (RGL only) -- used by tests on vacancy boxes. */
int ora_densities(const ora_sys *sys, const ora_pot *pot, const double *x, double *rho) {
    int rc_ok = check_box(sys, pot);
    if (rc_ok) return rc_ok;
    if (pot->kind != POT_RGL) return -1;
    const double rc2 = pot->rc * pot->rc;
    for (int64_t i = 0; i < sys->n; ++i) {
        double rh = 0.0;
        for (int64_t j = 0; j < sys->n; ++j) {
            if (j == i) continue;
            double d[3];
            for (int a = 0; a < 3; ++a)
                d[a] = min_image(x[3 * i + a] - x[3 * j + a], sys->box[a], sys->periodic[a]);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= rc2) continue;
            double phi, dphi, gg, dg;
            rgl_pair(pot, sqrt(r2), &phi, &dphi, &gg, &dg);
            rh += gg;
        }
        rho[i] = rh;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Derivatives for the differentiable form (RGL only).                       */
/*                                                                          */
/* theta = (A, xi, p, q).  With d = x_j - x_i, r = |d|, s = r/r0 - 1,       */
/* e_p = exp(-p s), e_q = exp(-2 q s) and the taper S(r):                    */
/*   phi  = A e_p S,  phi'  = A e_p (-(p/r0) S + S'),                        */
/*   phi''= A e_p ((p/r0)^2 S - 2 (p/r0) S' + S''),                          */
/*   g    = xi^2 e_q S, g' and g'' likewise with 2q in place of p,           */
/*   rho_i = sum_j g,  F'_i = -1/(2 sqrt(rho_i)),  F''_i = 1/(4 rho_i^1.5),  */
/*   F_i = sum_j [2 phi' + (F'_i + F'_j) g'] d / r.                          */

static void taper2(const ora_pot *pot, double r, double *S, double *dS, double *d2S) {
    if (r <= pot->rs) { *S = 1.0; *dS = 0.0; *d2S = 0.0; return; }
    if (r >= pot->rc) { *S = 0.0; *dS = 0.0; *d2S = 0.0; return; }
    double w = pot->rc - pot->rs;
    double t = (r - pot->rs) / w;
    *S = 1.0 - 10.0 * t * t * t + 15.0 * t * t * t * t - 6.0 * t * t * t * t * t;
    *dS = (-30.0 * t * t + 60.0 * t * t * t - 30.0 * t * t * t * t) / w;
    *d2S = (-60.0 * t + 180.0 * t * t - 120.0 * t * t * t) / (w * w);
}

typedef struct {
    double r, s, ep, eq, S, dS, d2S;
    double phi, dphi, d2phi, g, dg, d2g;
} ora_pair2;

static void rgl_pair2(const ora_pot *pot, double r, ora_pair2 *q) {
    q->r = r;
    q->s = r / pot->r0 - 1.0;
    taper2(pot, r, &q->S, &q->dS, &q->d2S);
    double a = pot->p / pot->r0, b = 2.0 * pot->q / pot->r0;
    q->ep = exp(-pot->p * q->s);
    q->eq = exp(-2.0 * pot->q * q->s);
    q->phi = pot->A * q->ep * q->S;
    q->dphi = pot->A * q->ep * (-a * q->S + q->dS);
    q->d2phi = pot->A * q->ep * (a * a * q->S - 2.0 * a * q->dS + q->d2S);
    double xi2 = pot->xi * pot->xi;
    q->g = xi2 * q->eq * q->S;
    q->dg = xi2 * q->eq * (-b * q->S + q->dS);
    q->d2g = xi2 * q->eq * (b * b * q->S - 2.0 * b * q->dS + q->d2S);
}

/* Neighbour lists within rc in CSR form (ascending j per atom), from the
 * same candidate enumeration as the force routines. */
typedef struct {
    int64_t *start, *nbr;
} ora_csr;

static void csr_build(const ora_sys *sys, const ora_pot *pot, const double *x, int mode,
                      ora_csr *L) {
    const int64_t n = sys->n;
    const double rc2 = pot->rc * pot->rc;
    ora_grid g;
    grid_build(&g, sys, x, pot->rc, mode);
    const int64_t cap = grid_max_candidates(&g) + 1;
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t **tmp = (int64_t **)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t *));
#pragma omp parallel
    {
        int64_t *cand = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            int64_t m = grid_candidates(&g, sys, x, i, cand), k = 0;
            tmp[i] = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
            for (int64_t c = 0; c < m; ++c) {
                int64_t j = cand[c];
                double d[3];
                for (int a = 0; a < 3; ++a)
                    d[a] = min_image(x[3 * j + a] - x[3 * i + a], sys->box[a], sys->periodic[a]);
                if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2) tmp[i][k++] = j;
            }
            cnt[i + 1] = k;
        }
        free(cand);
    }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    L->start = cnt;
    L->nbr = (int64_t *)malloc((size_t)(cnt[n] > 0 ? cnt[n] : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        memcpy(L->nbr + cnt[i], tmp[i], (size_t)(cnt[i + 1] - cnt[i]) * sizeof(int64_t));
        free(tmp[i]);
    }
    free(tmp);
    grid_free(&g);
}

static void csr_free(ora_csr *L) {
    free(L->start);
    free(L->nbr);
}

/* Minimum-image d = x_j - x_i, r and the pair functions of pair (i, j). */
static void pair_geom(const ora_sys *sys, const ora_pot *pot, const double *x, int64_t i,
                      int64_t j, double d[3], ora_pair2 *q) {
    for (int a = 0; a < 3; ++a)
        d[a] = min_image(x[3 * j + a] - x[3 * i + a], sys->box[a], sys->periodic[a]);
    rgl_pair2(pot, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), q);
}

/* Per-atom rho_i, F'_i, F''_i and drho_i/dq. */
static void rgl_atom_terms(const ora_sys *sys, const ora_pot *pot, const double *x,
                           const ora_csr *L, double *rho, double *F1, double *F2,
                           double *drho_dq) {
    const int64_t n = sys->n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double rh = 0.0, dq = 0.0, d[3];
        for (int64_t k = L->start[i]; k < L->start[i + 1]; ++k) {
            ora_pair2 q;
            pair_geom(sys, pot, x, i, L->nbr[k], d, &q);
            rh += q.g;
            dq += -2.0 * q.s * q.g;
        }
        rho[i] = rh;
        F1[i] = rh > 0.0 ? -0.5 / sqrt(rh) : 0.0;
        F2[i] = rh > 0.0 ? 0.25 / (rh * sqrt(rh)) : 0.0;
        if (drho_dq) drho_dq[i] = dq;
    }
}

/* dE/dtheta (4 values) and, if dF != NULL, dF/dtheta laid out as
 * dF[k * 3N + 3 i + a] for theta_k = (A, xi, p, q). */
int ora_rgl_param_derivs(const ora_sys *sys, const ora_pot *pot, const double *x, double *dE,
                         double *dF, int mode) {
    int rc_ok = check_box(sys, pot);
    if (rc_ok) return rc_ok;
    if (pot->kind != POT_RGL) return -1;
    const int64_t n = sys->n, n1 = n > 0 ? n : 1;
    ora_csr L;
    csr_build(sys, pot, x, mode, &L);
    double *rho = (double *)calloc((size_t)n1, sizeof(double));
    double *F1 = (double *)calloc((size_t)n1, sizeof(double));
    double *F2 = (double *)calloc((size_t)n1, sizeof(double));
    double *dq = (double *)calloc((size_t)n1, sizeof(double));
    double *eAi = (double *)calloc((size_t)n1, sizeof(double));
    double *ePi = (double *)calloc((size_t)n1, sizeof(double));
    rgl_atom_terms(sys, pot, x, &L, rho, F1, F2, dq);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double fA[3] = {0, 0, 0}, fX[3] = {0, 0, 0}, fP[3] = {0, 0, 0}, fQ[3] = {0, 0, 0};
        double sA = 0.0, sP = 0.0, d[3];
        for (int64_t k = L.start[i]; k < L.start[i + 1]; ++k) {
            const int64_t j = L.nbr[k];
            ora_pair2 q;
            pair_geom(sys, pot, x, i, j, d, &q);
            sA += q.ep * q.S;
            sP += -q.s * q.phi;
            double c = F1[i] + F1[j];
            double dphi_dp = -q.s * q.dphi - pot->A * q.ep * q.S / pot->r0;
            double dg_dq = -2.0 * q.s * q.dg - 2.0 * pot->xi * pot->xi * q.eq * q.S / pot->r0;
            double dc_dq = F2[i] * dq[i] + F2[j] * dq[j];
            double wA = 2.0 * q.dphi / pot->A / q.r;
            double wX = c * q.dg / pot->xi / q.r;
            double wP = 2.0 * dphi_dp / q.r;
            double wQ = (dc_dq * q.dg + c * dg_dq) / q.r;
            for (int a = 0; a < 3; ++a) {
                fA[a] += wA * d[a];
                fX[a] += wX * d[a];
                fP[a] += wP * d[a];
                fQ[a] += wQ * d[a];
            }
        }
        eAi[i] = sA;
        ePi[i] = sP;
        if (dF) {
            for (int a = 0; a < 3; ++a) {
                dF[0 * 3 * n + 3 * i + a] = fA[a];
                dF[1 * 3 * n + 3 * i + a] = fX[a];
                dF[2 * 3 * n + 3 * i + a] = fP[a];
                dF[3 * 3 * n + 3 * i + a] = fQ[a];
            }
        }
    }
    /* dE/dA = sum_i sum_j e_p S; dE/dxi = sum_i F'_i 2 rho_i / xi;
     * dE/dp = sum_i sum_j (-s) phi; dE/dq = sum_i F'_i drho_i/dq */
    double eA = 0.0, eXi = 0.0, eP = 0.0, eQ = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        eA += eAi[i];
        eP += ePi[i];
        eXi += F1[i] * 2.0 * rho[i] / pot->xi;
        eQ += F1[i] * dq[i];
    }
    dE[0] = eA;
    dE[1] = eXi;
    dE[2] = eP;
    dE[3] = eQ;
    free(rho); free(F1); free(F2); free(dq); free(eAi); free(ePi);
    csr_free(&L);
    return 0;
}

/* Hu = -(d/de) F(x + e u) at e = 0, the directional derivative of the
 * two-pass force written out (L: lists at x, F1/F2: F'(rho), F''(rho)). */
static void hvp_apply(const ora_sys *sys, const ora_pot *pot, const double *x, const ora_csr *L,
                      const double *F1, const double *F2, double *drho, const double *u,
                      double *Hu) {
    const int64_t n = sys->n;
    /* d rho_i = sum_j g'(r_ij) dr_ij,  dr_ij = d . (u_j - u_i) / r */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0, d[3];
        for (int64_t k = L->start[i]; k < L->start[i + 1]; ++k) {
            const int64_t j = L->nbr[k];
            ora_pair2 q;
            pair_geom(sys, pot, x, i, j, d, &q);
            double dr = 0.0;
            for (int a = 0; a < 3; ++a) dr += d[a] * (u[3 * j + a] - u[3 * i + a]);
            acc += q.dg * dr / q.r;
        }
        drho[i] = acc;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double dF[3] = {0, 0, 0}, d[3], du[3];
        for (int64_t k = L->start[i]; k < L->start[i + 1]; ++k) {
            const int64_t j = L->nbr[k];
            ora_pair2 q;
            pair_geom(sys, pot, x, i, j, d, &q);
            for (int a = 0; a < 3; ++a) du[a] = u[3 * j + a] - u[3 * i + a];
            double c = F1[i] + F1[j];
            double fs = (2.0 * q.dphi + c * q.dg) / q.r;
            double dr = (d[0] * du[0] + d[1] * du[1] + d[2] * du[2]) / q.r;
            double dc = F2[i] * drho[i] + F2[j] * drho[j];
            double dfs = ((2.0 * q.d2phi + c * q.d2g) / q.r - fs / q.r) * dr + dc * q.dg / q.r;
            for (int a = 0; a < 3; ++a) dF[a] += dfs * d[a] + fs * du[a];
        }
        for (int a = 0; a < 3; ++a) Hu[3 * i + a] = -dF[a];
    }
}

int ora_rgl_hvp(const ora_sys *sys, const ora_pot *pot, const double *x, const double *u,
                double *Hu, int mode) {
    int rc_ok = check_box(sys, pot);
    if (rc_ok) return rc_ok;
    if (pot->kind != POT_RGL) return -1;
    const int64_t n1 = sys->n > 0 ? sys->n : 1;
    ora_csr L;
    csr_build(sys, pot, x, mode, &L);
    double *rho = (double *)calloc((size_t)n1, sizeof(double));
    double *F1 = (double *)calloc((size_t)n1, sizeof(double));
    double *F2 = (double *)calloc((size_t)n1, sizeof(double));
    double *drho = (double *)calloc((size_t)n1, sizeof(double));
    rgl_atom_terms(sys, pot, x, &L, rho, F1, F2, NULL);
    hvp_apply(sys, pot, x, &L, F1, F2, drho, u, Hu);
    free(rho); free(F1); free(F2); free(drho);
    csr_free(&L);
    return 0;
}

/* Removes the mean of each Cartesian component (the translation modes). */
static void project_translations(double *v, int64_t n) {
    for (int a = 0; a < 3; ++a) {
        double m = 0.0;
        for (int64_t i = 0; i < n; ++i) m += v[3 * i + a];
        m /= (double)(n > 0 ? n : 1);
        for (int64_t i = 0; i < n; ++i) v[3 * i + a] -= m;
    }
}

/* Conjugate gradients for H lambda = b in the subspace orthogonal to the
 * three translations (H is singular along them under periodic boundaries).
 * Stops when |r| <= tol |b|.  Returns the iteration count (or -1). */
int64_t ora_rgl_cg(const ora_sys *sys, const ora_pot *pot, const double *x, const double *b_in,
                   double tol, int64_t maxit, double *lambda, int mode) {
    int rc_ok = check_box(sys, pot);
    if (rc_ok || pot->kind != POT_RGL) return -1;
    const int64_t n = sys->n, m = 3 * n, n1 = n > 0 ? n : 1;
    ora_csr L;
    csr_build(sys, pot, x, mode, &L);
    double *rho = (double *)calloc((size_t)n1, sizeof(double));
    double *F1 = (double *)calloc((size_t)n1, sizeof(double));
    double *F2 = (double *)calloc((size_t)n1, sizeof(double));
    double *drho = (double *)calloc((size_t)n1, sizeof(double));
    rgl_atom_terms(sys, pot, x, &L, rho, F1, F2, NULL);
    double *b = (double *)malloc((size_t)3 * n1 * sizeof(double));
    double *r = (double *)malloc((size_t)3 * n1 * sizeof(double));
    double *p = (double *)malloc((size_t)3 * n1 * sizeof(double));
    double *Ap = (double *)malloc((size_t)3 * n1 * sizeof(double));
    memcpy(b, b_in, (size_t)m * sizeof(double));
    project_translations(b, n);
    for (int64_t k = 0; k < m; ++k) { lambda[k] = 0.0; r[k] = b[k]; p[k] = b[k]; }
    double rr = dot3n(r, r, m);
    const double stop2 = tol * tol * rr;
    int64_t it = 0;
    while (it < maxit && rr > stop2 && rr > 0.0) {
        hvp_apply(sys, pot, x, &L, F1, F2, drho, p, Ap);
        project_translations(Ap, n);
        double pAp = dot3n(p, Ap, m);
        if (!(pAp > 0.0)) break;
        double alpha = rr / pAp;
        for (int64_t k = 0; k < m; ++k) {
            lambda[k] += alpha * p[k];
            r[k] -= alpha * Ap[k];
        }
        double rr_new = dot3n(r, r, m);
        double beta = rr_new / rr;
        for (int64_t k = 0; k < m; ++k) p[k] = r[k] + beta * p[k];
        rr = rr_new;
        ++it;
    }
    free(rho); free(F1); free(F2); free(drho); free(b); free(r); free(p); free(Ap);
    csr_free(&L);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Force norms of Sec. 3.4.                                                   */

static void force_norms(const double *f, int64_t n, double *fmax_atom, double *f2, double *finf) {
    double m = 0.0, s = 0.0, mi = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double a2 = f[3 * i] * f[3 * i] + f[3 * i + 1] * f[3 * i + 1] + f[3 * i + 2] * f[3 * i + 2];
        s += a2;
        double a = sqrt(a2);
        if (a > m) m = a;
        for (int d = 0; d < 3; ++d)
            if (fabs(f[3 * i + d]) > mi) mi = fabs(f[3 * i + d]);
    }
    *fmax_atom = m;
    *f2 = sqrt(s);
    *finf = mi;
}

static double pick_norm(int norm, double fmax_atom, double f2, double finf) {
    if (norm == NORM_TWO) return f2;
    if (norm == NORM_INF) return finf;
    return fmax_atom;
}

static double dot3n(const double *a, const double *b, int64_t n3) {
    double s = 0.0;
    for (int64_t k = 0; k < n3; ++k) s += a[k] * b[k];
    return s;
}

/* ------------------------------------------------------------------------ */
/* FIRE 2.0 (Algorithm 2) or FIRE (Algorithm 1), with the integrators of      */
/* Algorithms 3-6.                                                            */

/* Zero the frozen force components (see ora_params.frozen). */
static void apply_frozen(double *f, int64_t n, const uint8_t *frozen) {
    if (!frozen) return;
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            if (frozen[i] & (1u << d)) f[3 * i + d] = 0.0;
}

/* x += dt_eff v with dt_eff = dt, or dmax / max_i |v_i| when that is smaller
 * (see ora_params.dmax). */
static void drift(double *x, const double *v, int64_t n, double dt, double dmax) {
    double dt_eff = dt;
    if (dmax > 0.0) {
        double vmax2 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double a2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                        v[3 * i + 2] * v[3 * i + 2];
            if (a2 > vmax2) vmax2 = a2;
        }
        double vmax = sqrt(vmax2);
        if (dt * vmax > dmax) dt_eff = dmax / vmax;
    }
    for (int64_t k = 0; k < 3 * n; ++k) x[k] += dt_eff * v[k];
}

/* v = (1 - alpha) v + alpha |v| F / |F| (the mixing of Algs. 1 and 3-6). */
static void mix_velocity(double *v, const double *f, int64_t n3, double alpha) {
    double vn = sqrt(dot3n(v, v, n3)), fn = sqrt(dot3n(f, f, n3));
    if (fn > 0.0)
        for (int64_t k = 0; k < n3; ++k) v[k] = (1.0 - alpha) * v[k] + alpha * vn * f[k] / fn;
}

/* The force of the system being relaxed: E and F at x (3 n values); returns
 * 0 or an error code.  Plain relaxations evaluate the potential (with the
 * frozen components zeroed); the nudged elastic band evaluates every image
 * and projects. */
typedef int (*ora_force_fn)(void *ctx, const double *x, double *f, double *E);

typedef struct {
    const ora_sys *sys;
    const ora_pot *pot;
    const uint8_t *frozen;
    int mode;
} plain_ctx;

static int plain_force(void *ctx, const double *x, double *f, double *E) {
    plain_ctx *c = (plain_ctx *)ctx;
    int rc_ok = ora_energy_forces(c->sys, c->pot, x, f, E, c->mode);
    if (rc_ok == 0) apply_frozen(f, c->sys->n, c->frozen);
    return rc_ok;
}

static int fire_loop(int64_t n, double m, ora_force_fn force, void *ctx, const ora_params *par,
                     double *x, double ftol, int64_t maxiter, ora_result *out,
                     ora_trace *trace, int64_t trace_cap);

int ora_fire2(const ora_sys *sys, const ora_pot *pot, const ora_params *par, double *x,
              double ftol, int64_t maxiter, int mode, ora_result *out,
              ora_trace *trace, int64_t trace_cap) {
    plain_ctx c = {sys, pot, par->frozen, mode};
    int rc_ok = check_box(sys, pot);
    if (rc_ok) return rc_ok;
    return fire_loop(sys->n, sys->mass, plain_force, &c, par, x, ftol, maxiter, out, trace,
                     trace_cap);
}

/* FIRE 2.0 (Algorithm 2) or FIRE (Algorithm 1) on n atoms of mass m under
 * `force`, with the integrators of Algorithms 3-6. */
static int fire_loop(int64_t n, double m, ora_force_fn force, void *ctx, const ora_params *par,
                     double *x, double ftol, int64_t maxiter, ora_result *out,
                     ora_trace *trace, int64_t trace_cap) {
    if (par->integrator < INT_EULER_IMPLICIT || par->integrator > INT_LEAPFROG) return -3;
    if (par->variant != VAR_FIRE2 && par->variant != VAR_FIRE1) return -3;
    if (maxiter < 0 || !(ftol >= 0.0) || !(par->dt_start > 0.0) || !(m > 0.0)) return -1;
    if (!(par->dmax >= 0.0)) return -1;
    const int64_t n3 = 3 * n;
    double *v = (double *)calloc((size_t)(n3 > 0 ? n3 : 1), sizeof(double));
    double *f = (double *)calloc((size_t)(n3 > 0 ? n3 : 1), sizeof(double));
    double E = 0.0;
    int rc_ok = force(ctx, x, f, &E);
    if (rc_ok) { free(v); free(f); return rc_ok; }

    /* initialisation: v = 0, alpha = alpha_start, dt = dt_start, counters 0 */
    double alpha = par->alpha0, dt = par->dt_start;
    const double dtmax = par->tmax * par->dt_start, dtmin = par->tmin * par->dt_start;
    int64_t npos = 0, nneg = 0, evals = 1, iters = 0;
    int stop = STOP_MAXITER;
    /* Leapfrog initialisation (Algorithm 5): v(-dt/2) = -dt/2 F(x) / m */
    if (par->integrator == INT_LEAPFROG)
        for (int64_t k = 0; k < n3; ++k) v[k] = -0.5 * dt * f[k] / m;
    double fmax_atom, f2, finf;
    force_norms(f, n, &fmax_atom, &f2, &finf);

    if (pick_norm(par->norm, fmax_atom, f2, finf) < ftol) {
        stop = STOP_FTOL;
    } else {
        for (int64_t i = 1; i <= maxiter; ++i) {
            double P = dot3n(f, v, n3);
            int mix_in_integrator = 0;
            if (par->variant == VAR_FIRE1) {
                /* Algorithm 1: mixing at the start of the step when P > 0 */
                if (P > 0.0) {
                    npos += 1;
                    mix_velocity(v, f, n3, alpha);
                    if (npos > par->delaystep) {
                        dt = fmin(dt * par->dtgrow, dtmax);
                        alpha *= par->alphashrink;
                    }
                } else {
                    npos = 0;
                    for (int64_t k = 0; k < n3; ++k) v[k] = 0.0;
                    dt *= par->dtshrink;
                    alpha = par->alpha0;
                }
            } else {
                /* Algorithm 2 */
                if (P > 0.0) {
                    npos += 1;
                    nneg = 0;
                    if (npos > par->delaystep) {
                        dt = fmin(dt * par->dtgrow, dtmax);
                        alpha *= par->alphashrink;
                    }
                    mix_in_integrator = 1;
                } else {
                    npos = 0;
                    nneg += 1;
                    if (nneg > par->vdfmax) { stop = STOP_MAXVDOTF; iters = i - 1; break; }
                    if (!(par->initialdelay && i < par->delaystep)) {
                        if (dt * par->dtshrink >= dtmin) dt *= par->dtshrink;
                        alpha = par->alpha0;
                    }
                    if (par->halfstepback)
                        for (int64_t k = 0; k < n3; ++k) x[k] -= 0.5 * dt * v[k];
                    for (int64_t k = 0; k < n3; ++k) v[k] = 0.0;
                }
            }
            /* MD integration (Algorithms 3-6); the FIRE 2.0 mixing sits inside */
            if (par->integrator == INT_EULER_EXPLICIT) {
                /* Algorithm 3: mix v(t), x += dt v(t), v += dt F(x(t)) / m */
                if (mix_in_integrator) mix_velocity(v, f, n3, alpha);
                drift(x, v, n, dt, par->dmax);
                for (int64_t k = 0; k < n3; ++k) v[k] += dt * f[k] / m;
                rc_ok = force(ctx, x, f, &E);
            } else if (par->integrator == INT_VERLET) {
                /* Algorithm 6: half kick, mix, drift, new force, half kick */
                for (int64_t k = 0; k < n3; ++k) v[k] += 0.5 * dt * f[k] / m;
                if (mix_in_integrator) mix_velocity(v, f, n3, alpha);
                drift(x, v, n, dt, par->dmax);
                rc_ok = force(ctx, x, f, &E);
                for (int64_t k = 0; k < n3; ++k) v[k] += 0.5 * dt * f[k] / m;
            } else {
                /* Algorithms 4 and 5: kick, mix (of the kicked v), drift, new force */
                for (int64_t k = 0; k < n3; ++k) v[k] += dt * f[k] / m;
                if (mix_in_integrator) mix_velocity(v, f, n3, alpha);
                drift(x, v, n, dt, par->dmax);
                rc_ok = force(ctx, x, f, &E);
            }
            if (rc_ok) { free(v); free(f); return rc_ok; }
            evals += 1;
            iters = i;
            force_norms(f, n, &fmax_atom, &f2, &finf);
            double fn_conv = pick_norm(par->norm, fmax_atom, f2, finf);
            if (trace && i - 1 < trace_cap) {
                ora_trace *t = &trace[i - 1];
                t->i = i; t->npos = npos; t->nneg = nneg;
                t->P = P; t->dt = dt; t->alpha = alpha; t->energy = E; t->fnorm = fn_conv;
            }
            if (fn_conv < ftol) { stop = STOP_FTOL; break; }
        }
    }
    force_norms(f, n, &fmax_atom, &f2, &finf);
    out->energy = E;
    out->iterations = iters;
    out->force_evals = evals;
    out->stop = stop;
    out->pad = 0;
    out->fmax_atom = fmax_atom;
    out->f2norm = f2;
    out->finf = finf;
    out->dt_final = dt;
    out->alpha_final = alpha;
    free(v);
    free(f);
    return 0;
}

void ora_set_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

int ora_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Nudged elastic band.  The paper's cases 7 and 8 relax, with FIRE 2.0, an   */
/* ensemble of images between two fixed end states under modified forces     */
/* (Sec. 4); it states no formulas and cites Sheppard et al. (2008), whose    */
/* standard method is written out here:                                      */
/*   tangent t_i (improved estimate of Henkelman and Jonsson, 2000) from the  */
/*   neighbour separations t+ = R_{i+1} - R_i, t- = R_i - R_{i-1} (minimum    */
/*   image) and the energies: t+ if E_{i+1} > E_i > E_{i-1}, t- if            */
/*   E_{i+1} < E_i < E_{i-1}, else dEmax t+ + dEmin t- (E_{i+1} > E_{i-1}) or */
/*   dEmin t+ + dEmax t- with dEmax/min = max/min(|E_{i+1}-E_i|,              */
/*   |E_{i-1}-E_i|); normalised;                                             */
/*   F_i^NEB = F_i - (F_i.t) t + k (|t+| - |t-|) t, or, for the climbing      */
/*   image (the movable image of highest energy, when enabled),               */
/*   F_i - 2 (F_i.t) t.                                                       */
/* The m movable images form one system of m n atoms for FIRE: one dt, one    */
/* alpha and one P over the whole band, and the stopping norm is taken over   */
/* all images -- a simultaneous minimisation of the ensemble.  Frozen         */
/* components (if any) are zeroed in the true force, the tangent and the     */
/* NEB force.  If the tangent vanishes (equal energies on both sides), t+ + t- */
/* is used; if that vanishes too, the force is left unprojected.             */

typedef struct {
    const ora_sys *sys;
    const ora_pot *pot;
    const uint8_t *frozen;
    int mode;
    int64_t m;
    const double *end0, *end1;
    double e_end0, e_end1;
    double k;
    int climb;
    double *E;          /* m + 2 energies */
    int64_t climber;    /* 1..m, or 0 */
} neb_ctx;

static const double *neb_image(const neb_ctx *c, const double *x, int64_t i) {
    if (i == 0) return c->end0;
    if (i == c->m + 1) return c->end1;
    return x + 3 * c->sys->n * (i - 1);
}

static int neb_force(void *ctx, const double *x, double *f, double *Etot) {
    neb_ctx *c = (neb_ctx *)ctx;
    const ora_sys *sys = c->sys;
    const int64_t n = sys->n, n3 = 3 * n, M = c->m;
    c->E[0] = c->e_end0;
    c->E[M + 1] = c->e_end1;
    for (int64_t i = 1; i <= M; ++i) {
        int rc_ok = ora_energy_forces(sys, c->pot, neb_image(c, x, i), f + n3 * (i - 1), &c->E[i],
                                      c->mode);
        if (rc_ok) return rc_ok;
        apply_frozen(f + n3 * (i - 1), n, c->frozen);
    }
    c->climber = 0;
    if (c->climb) {
        c->climber = 1;
        for (int64_t i = 2; i <= M; ++i)
            if (c->E[i] > c->E[c->climber]) c->climber = i;
    }
    double tot = 0.0;
    for (int64_t i = 1; i <= M; ++i) tot += c->E[i];
    *Etot = tot;
    const size_t bytes = (size_t)(n3 > 0 ? n3 : 1) * sizeof(double);
    double *tp = (double *)malloc(bytes), *tm = (double *)malloc(bytes);
    double *t = (double *)malloc(bytes);
    for (int64_t i = 1; i <= M; ++i) {
        const double *R = neb_image(c, x, i), *Rp = neb_image(c, x, i + 1);
        const double *Rm = neb_image(c, x, i - 1);
        for (int64_t q = 0; q < n3; ++q) {
            const int a = (int)(q % 3);
            tp[q] = min_image(Rp[q] - R[q], sys->box[a], sys->periodic[a]);
            tm[q] = min_image(R[q] - Rm[q], sys->box[a], sys->periodic[a]);
        }
        const double Ep = c->E[i + 1], Ei = c->E[i], Em = c->E[i - 1];
        double wp, wm;
        if (Ep > Ei && Ei > Em) {
            wp = 1.0;
            wm = 0.0;
        } else if (Ep < Ei && Ei < Em) {
            wp = 0.0;
            wm = 1.0;
        } else {
            const double dmx = fmax(fabs(Ep - Ei), fabs(Em - Ei));
            const double dmn = fmin(fabs(Ep - Ei), fabs(Em - Ei));
            if (Ep > Em) {
                wp = dmx;
                wm = dmn;
            } else {
                wp = dmn;
                wm = dmx;
            }
        }
        for (int64_t q = 0; q < n3; ++q) t[q] = wp * tp[q] + wm * tm[q];
        apply_frozen(t, n, c->frozen);
        double tn = sqrt(dot3n(t, t, n3));
        if (!(tn > 0.0)) {
            for (int64_t q = 0; q < n3; ++q) t[q] = tp[q] + tm[q];
            apply_frozen(t, n, c->frozen);
            tn = sqrt(dot3n(t, t, n3));
        }
        double *fi = f + n3 * (i - 1);
        if (tn > 0.0) {
            for (int64_t q = 0; q < n3; ++q) t[q] /= tn;
            const double ft = dot3n(fi, t, n3);
            if (i == c->climber) {
                for (int64_t q = 0; q < n3; ++q) fi[q] -= 2.0 * ft * t[q];
            } else {
                const double sp = c->k * (sqrt(dot3n(tp, tp, n3)) - sqrt(dot3n(tm, tm, n3)));
                for (int64_t q = 0; q < n3; ++q) fi[q] += (sp - ft) * t[q];
            }
        }
        apply_frozen(fi, n, c->frozen);
    }
    free(tp);
    free(tm);
    free(t);
    return 0;
}

/* path: (m + 2) images of n atoms (x, y, z), image 0 and m + 1 the fixed end
 * states; the m movable images are relaxed in place.  energies: m + 2
 * values out; climber: index of the climbing image at the end (0 = none).
 * out->energy is the sum of the movable images' energies. */
int ora_neb(const ora_sys *sys, const ora_pot *pot, const ora_params *par, int64_t m,
            double *path, double k, int climb, double ftol, int64_t maxiter, int mode,
            ora_result *out, double *energies, int64_t *climber) {
    if (m < 1 || !(k >= 0.0)) return -1;
    int rc_ok = check_box(sys, pot);
    if (rc_ok) return rc_ok;
    const int64_t n3 = 3 * sys->n;
    neb_ctx c;
    c.sys = sys;
    c.pot = pot;
    c.frozen = par->frozen;
    c.mode = mode;
    c.m = m;
    c.end0 = path;
    c.end1 = path + n3 * (m + 1);
    c.k = k;
    c.climb = climb;
    c.E = energies;
    c.climber = 0;
    double *fw = (double *)malloc((size_t)(n3 > 0 ? n3 : 1) * sizeof(double));
    rc_ok = ora_energy_forces(sys, pot, c.end0, fw, &c.e_end0, mode);
    if (!rc_ok) rc_ok = ora_energy_forces(sys, pot, c.end1, fw, &c.e_end1, mode);
    free(fw);
    if (rc_ok) return rc_ok;
    rc_ok = fire_loop(sys->n * m, sys->mass, neb_force, &c, par, path + n3, ftol, maxiter, out,
                      NULL, 0);
    *climber = c.climber;
    return rc_ok;
}
