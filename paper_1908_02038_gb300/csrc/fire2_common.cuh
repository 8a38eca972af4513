// Device definitions shared by the single-system kernels (fire2_device.cuh)
// and the batched persistent kernel (fire2_batch.cu): data types, launch
// constants, block reductions, geometry helpers and the RGL pair functions.
// Only inline functions and types live here, so several translation units
// may include it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fire2_math.cuh"

namespace fire2 {

// Per-atom 3-vectors live in 32-byte aligned, zero-padded double quads so a
// load or store of one atom is a single aligned 32-byte sector.
using dvec4 = double4_32a;
__host__ __device__ __forceinline__ dvec4 make_dvec4(double x, double y, double z, double w) {
    return make_double4_32a(x, y, z, w);
}

constexpr uint32_t kIdxBits = 25;
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1u;
constexpr int kCodeZero = 62;  // image code of the zero shift, (2 + 5*2 + 25*2)
constexpr int kForceBlock = 128;
constexpr int kTabBlock = 256;    // FP32 table kernels (more warps per shared table copy)
constexpr int kTabBlock64 = 512;  // FP64 table kernel (both tables, ~112 KB, in shared memory)
constexpr int kElemBlock = 256;
constexpr int kDensFF1Block = 512;   // double-float density pass, one thread per atom
constexpr int kCtlThreads = 512;
constexpr int kRedRows = 6;   // rows of the per-block partials: P, |F|^2, |v|^2, max |F_i|^2,
                              // max |F_i,d|, energy (red_write)

enum { ST_OK = 0, ST_NONFINITE = 4, ST_NBR_OVERFLOW = 5, ST_TIMEOUT = 6, ST_RANGE = 8,
       ST_CROWDED = 9 };
enum { STOP_FTOL = 0, STOP_MAXITER = 1, STOP_MAXVDOTF = 2 };
enum { POT_LJ = 0, POT_RGL = 1 };
enum { CTL_INITIAL = 0, CTL_LOOP = 1, CTL_EVAL = 2 };

// Knots of the tabulated RGL pair functions (built in fire2_table.cuh):
// region A covers [u_lo, u_rs] with spacing 1/hA_inv and a knot at u = 0,
// region B covers [u_rs, rc^2 - r0^2] with spacing 1/hB_inv.
struct TabMeta {
    int nA0;                    // intervals of region A below u = 0
    int nA;                     // intervals of region A
    int nB;                     // intervals of region B
    int pad;
    double hA_inv, hB_inv, u_lo, u_rs;
    float hA_inv_f, hB_inv_f, u_lo_f, u_rs_f;
};

// Potential constants, passed by value.
struct PotC {
    int kind;
    double rc2;            // interaction cut-off squared
    // LJ
    double eps, sigma2, lj_shift;
    // SW (eps above): sigma, a sigma, and the published dimensionless set
    double sw_sigma, sw_rc, sw_A, sw_B, sw_p, sw_q, sw_lambda, sw_gamma;
    int sw_pi, sw_qi;      // sw_p, sw_q as small non-negative integers, or -1
    // RGL
    double A, xi2, p, q2, r0inv, p_r0, q2_r0, rs, rc, winv;
    ExpC ex;               // constants of the table-driven exponential
    // FP32-pair form: FP32 copies of the constants; r^2 tests in fixed point
    Exp32C ex32;
    float A_f, xi2_f, p_f, q2_f, r0_f, p_r0_f, q2_r0_f, rs_f, winv_f;
    long long rc2q, r0sq_q;   // rc^2 and r0^2 in (fixed-point unit)^2
    float qinv, qinv2;        // 1 / qscale, 1 / qscale^2
    double xi_inv;            // 1 / xi (theta-derivatives)
    double r0sq;              // r0^2 (table variable u = r^2 - r0^2)
    float r0sq_f, rc2_f;      // FP32 copies (table index and cut-off test of the FP64 pass)
    TabMeta tab;              // knots of the tabulated pair functions (FP64)
    TabMeta tab32;            // knots of the FP32 tables
};

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// max(a, b) of non-negative doubles (NaN propagates: its pattern is larger
// than that of +inf) and |x|, both on the integer pipes.
__device__ __forceinline__ double max_nonneg(double a, double b) {
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ double abs_bits(double x) {
    return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffll);
}

// FP64 instructions issue at 1/58 of the FP32 rate on this part and a warp
// pays for all 32 lanes of each, so the reductions below keep them few.
//
// Four sums over the warp with 6 FP64 additions in place of 4 x 5: the first
// two butterfly steps halve the set of quantities each lane carries (lanes
// 0-15 go on with q0, q1 and lanes 16-31 with q2, q3; then lanes with bit 3
// clear keep the first of the two), the last three add one value.  On return
// lanes 8k .. 8k + 7 hold the total of q_k (fixed order: deterministic).
__device__ __forceinline__ double warp_sum4(double q0, double q1, double q2, double q3) {
    const unsigned lane = threadIdx.x & 31u;
    const bool b4 = (lane & 16u) != 0u, b3 = (lane & 8u) != 0u;
    const double r0 = __shfl_xor_sync(0xffffffffu, b4 ? q0 : q2, 16);
    const double r1 = __shfl_xor_sync(0xffffffffu, b4 ? q1 : q3, 16);
    const double a0 = (b4 ? q2 : q0) + r0, a1 = (b4 ? q3 : q1) + r1;
    double v = (b3 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, b3 ? a0 : a1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Maximum over the warp of non-negative doubles (NaN propagates) on the
// integer pipes: their IEEE patterns order like the values; every lane
// receives it.
__device__ __forceinline__ double warp_max_nonneg(double v) {
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    return __longlong_as_double(b);
}

// Sum over the TPA consecutive lanes that share one atom in the pair passes
// (TPA = 1, 2, 4, 8, 16 or 32 threads per atom); every lane of the group receives
// the total.  Only the group's own lanes are named in the mask, so groups
// whose atom index is past the end may have left the kernel.
template <int TPA>
__device__ __forceinline__ double group_sum(double v) {
    static_assert(TPA == 1 || TPA == 2 || TPA == 4 || TPA == 8 || TPA == 16 || TPA == 32,
                  "threads per atom");
    if (TPA > 1) {
        const unsigned lane = threadIdx.x & 31u;
        const unsigned gmask = TPA == 32 ? 0xffffffffu
                                         : ((1u << (TPA & 31)) - 1u) << (lane & ~(unsigned)(TPA - 1));
#pragma unroll
        for (int o = TPA / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o, TPA);
    }
    return v;
}

// Block-wide sum; result valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}
// Block-wide maximum of non-negative doubles on the integer pipes; result
// valid in thread 0.
__device__ __forceinline__ double block_max_nonneg(double v, double* sh) {
    v = warp_max_nonneg(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) r = warp_max_nonneg((lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0);
    return r;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
    v = warp_max(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        r = warp_max(r);
    }
    return r;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Cell index of coordinate x on an axis of nc cells over [0, L): wrapped into
// the box on a periodic axis, clamped to the edge cells on an open one (an
// atom outside the box shares the edge cell; with cells at least the list
// radius wide, any two atoms within that radius still lie in the same or
// adjacent cells).
__device__ __forceinline__ int cell_coord(double x, double Linv, int nc, int per) {
    double u = x * Linv;
    if (per) u -= floor(u);
    const double c = floor(u * nc);
    if (!(c >= 0.0)) return 0;   // also NaN
    return c >= nc ? nc - 1 : (int)c;
}

// Neighbour cell cx + o on an axis: wrapped on a periodic axis; -1 when it
// falls outside an open one.
__device__ __forceinline__ int cell_step(int cx, int o, int nc, int per) {
    const int a = cx + o;
    if (per) return (a + nc) % nc;
    return (a < 0 || a >= nc) ? -1 : a;
}

// Fixed-point coordinate (units of 1/qscale) modulo 2^32.  Differences of two
// such values, taken in 32-bit wrap-around arithmetic, are exact whenever the
// true separation is below 2^31 / qscale (qscale is chosen so that every list
// pair qualifies), whatever periodic image the raw coordinates sit in.
// round(x qscale) modulo 2^32 for qscale = 2^k, rounding half to even, with
// integer operations on the IEEE-754 fields (FP64 conversions issue at 1/58
// of the FP32 rate on this part): x = M 2^(E - 1075) with the 53-bit
// significand M, so x qscale = M 2^-sh with sh = 1075 - k - E.
__device__ __forceinline__ int to_fixed(double x, double qscale) {
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    const int k = (int)(((unsigned long long)__double_as_longlong(qscale) >> 52) & 0x7ffull) - 1023;
    const int E = (int)((bx >> 52) & 0x7ffull);
    if (E == 0) return 0;                       // zero (positions are never subnormal)
    const unsigned long long M = (bx & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1075 - k - E;
    unsigned long long q;
    if (sh <= 0) {
        q = M << (-sh < 63 ? -sh : 63);         // |x qscale| >= 2^52: wraps
    } else if (sh >= 64) {
        q = 0ull;
    } else {
        q = M >> sh;
        const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1ull))) ++q;
    }
    unsigned r = (unsigned)q;
    if ((long long)bx < 0) r = 0u - r;
    return (int)r;
}

// round(x 2^k) as a 64-bit integer (|x 2^k| < 2^62), half to even, by the
// same integer operations as to_fixed.
__device__ __forceinline__ long long to_fixed64(double x, int k) {
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((bx >> 52) & 0x7ffull);
    if (E == 0) return 0ll;
    const unsigned long long M = (bx & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1075 - k - E;
    unsigned long long q;
    if (sh <= 0) {
        q = M << (-sh < 63 ? -sh : 63);
    } else if (sh >= 64) {
        q = 0ull;
    } else {
        q = M >> sh;
        const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1ull))) ++q;
    }
    return (long long)bx < 0 ? -(long long)q : (long long)q;
}

struct __align__(32) lvec4 {   // fixed-point position (x, y, z, unused)
    long long x, y, z, w;
};

__device__ __forceinline__ int wrap_sub(int a, int b) { return (int)((unsigned)a - (unsigned)b); }

// Upper half-space test on the minimum-image vector d = x_j - x_i: exactly
// one of (i, j) and (j, i) passes because IEEE subtraction, rounding to the
// nearest integer and the squares are all symmetric under d -> -d.
__device__ __forceinline__ bool upper_half(float dx, float dy, float dz) {
    return dz > 0.f || (dz == 0.f && (dy > 0.f || (dy == 0.f && dx > 0.f)));
}

// RGL pair terms in FP64 (Sec. 5.2 EAM family, second-moment form):
// phi = A e^{-p s} S(r), g = xi^2 e^{-2q s} S(r), s = r/r0 - 1, with the
// quintic taper S on [rs, rc).  Returns 1/r and the derivatives.
__device__ __forceinline__ void rgl_pair64(const PotC& P, double r2, const double* etab,
                                           double& rinv, double& phi, double& dphi, double& g,
                                           double& dg) {
    rinv = rsqrt(r2);
    const double r = r2 * rinv;
    const double s = r * P.r0inv - 1.0;
    const double ep = P.A * exp_tang(-P.p * s, P.ex, etab);
    const double eq = P.xi2 * exp_tang(-P.q2 * s, P.ex, etab);
    double S = 1.0, dS = 0.0;
    if (r > P.rs) {
        const double t = (r - P.rs) * P.winv;
        const double t2 = t * t, t3 = t2 * t;
        S = 1.0 - 10.0 * t3 + 15.0 * t3 * t - 6.0 * t3 * t2;
        dS = (-30.0 * t2 + 60.0 * t3 - 30.0 * t3 * t) * P.winv;
    }
    phi = ep * S;
    g = eq * S;
    dphi = ep * (-P.p_r0 * S + dS);
    dg = eq * (-P.q2_r0 * S + dS);
}

// int64 -> float through two exact 32-bit halves (the 64-bit conversion
// would occupy the FP64 pipe, 1/58 of the FP32 rate on this part).
__device__ __forceinline__ float ll_to_float(long long v) {
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)(v & 0xffffffffll);
    return fmaf((float)hi, 4294967296.0f, (float)lo);
}

// RGL pair terms in FP32 from the exact fixed-point r^2.
__device__ __forceinline__ void rgl_pair32(const PotC& P, long long r2q, const float* et,
                                           float& rinv, float& phi, float& dphi, float& g,
                                           float& dg) {
    const float r2 = ll_to_float(r2q) * P.qinv2;
    const float u = ll_to_float(r2q - P.r0sq_q) * P.qinv2;   // r^2 - r0^2
    rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float s = u / (P.r0_f * (r + P.r0_f));                // r/r0 - 1
    const float ep = P.A_f * exp32_tang(-P.p_f * s, P.ex32, et);
    const float eq = P.xi2_f * exp32_tang(-P.q2_f * s, P.ex32, et);
    float S = 1.f, dS = 0.f;
    if (r > P.rs_f) {
        const float t = (r - P.rs_f) * P.winv_f;
        const float t2 = t * t, t3 = t2 * t;
        S = 1.f - 10.f * t3 + 15.f * t3 * t - 6.f * t3 * t2;
        dS = (-30.f * t2 + 60.f * t3 - 30.f * t3 * t) * P.winv_f;
    }
    phi = ep * S;
    g = eq * S;
    dphi = ep * (-P.p_r0_f * S + dS);
    dg = eq * (-P.q2_r0_f * S + dS);
}

// ---------------------------------------------------------------------------
// FIRE 2.0 scalar control (Algorithm 2) and the element-wise update
// (Algorithm 4), shared by the single-system and the batched kernels.

enum { INT_EULER_IMPLICIT = 0, INT_EULER_EXPLICIT = 1, INT_VERLET = 2, INT_LEAPFROG = 3 };
enum { VAR_FIRE2 = 0, VAR_FIRE1 = 1 };

// Parameters of Table 1 and the call arguments, device copy.
struct FireParamsD {
    double ftol;
    long long maxiter;
    double dt_start, dtmax, dtmin, dtgrow, dtshrink, alpha0, alphashrink, mass;
    int delaystep, vdfmax, halfstepback, initialdelay, norm, integrator, variant, pad;
    double dmax;           // maximum displacement per step, 0 = no cap
};

// Scalar state of Algorithms 1/2 plus the coefficients the next element-wise
// update applies (see fire_update_pre and fire_update_drift_k).
struct FireScal {
    double dt, alpha;
    long long npos, nneg, iter, evals;
    int stop, zero_v, premix, postmix, lf_init, vv, pad0, pad1;
    double dtm;                  // dt / m
    double halfstep;             // x -= halfstep v before v = 0
    double kick_pre;             // v += kick_pre F before the drift
    double kick_after;           // v += kick_after F after the drift (explicit Euler)
    double vv_half;              // v += vv_half F_new after the force (velocity Verlet)
    double lf_c;                 // v(-dt/2) = lf_c F (Leapfrog initialisation)
    double dt_cur;               // drift x += dt_cur v
    double mix_a, mix_fv_pre, mix_fv_post;   // mixing coefficients
    // kick and mixing of the kicked velocity as one step (Algs. 4-6 when
    // P > 0): v <- (1 - a) (v + c F) + a fv F = post_v v + post_f F
    double post_v, post_f;
};

__host__ __device__ inline void fire_scal_init(const FireParamsD& p, FireScal& s) {
    s.dt = p.dt_start;
    s.alpha = p.alpha0;
    s.npos = s.nneg = s.iter = s.evals = 0;
    s.stop = STOP_MAXITER;
    s.zero_v = s.premix = s.postmix = s.lf_init = s.vv = s.pad0 = s.pad1 = 0;
    s.dtm = s.halfstep = s.kick_pre = s.kick_after = s.vv_half = s.lf_c = s.dt_cur = 0.0;
    s.mix_a = s.mix_fv_pre = s.mix_fv_post = 0.0;
    s.post_v = s.post_f = 0.0;
}

// Called after every force evaluation with the FP64 reductions of the
// current (F, v) (for velocity Verlet after its second half kick).  Tests
// convergence (after the integration, Alg. 2) and the iteration budget,
// then prepares the next iteration:
//  * FIRE 2.0 (Algorithm 2): the P > 0 / P <= 0 branch with its counters,
//    dt growth capped at dt_max after N_delay positive steps, alpha decay,
//    the N_P<=0 cap (MAXVDOTF, before any correction), the initial delay,
//    the dt_min guard and the half step back with the shrunk dt; mixing
//    inside the integrator when P > 0 (of the kicked velocity for
//    Algorithms 4-6, of v(t) for Algorithm 3);
//  * FIRE (Algorithm 1): mixing of v(t) at the start of the step when
//    P > 0, plain dt * f_dec, alpha reset and v = 0 when P <= 0;
//  * the integrator coefficients of Algorithms 3-6 with the new dt; the
//    Leapfrog initialisation v(-dt/2) = -dt/2 F / m at the first iteration.
// Norms of mixed velocities come from the reductions:
// |v + c F|^2 = |v|^2 + 2 c P + c^2 |F|^2.  Returns true to stop.
// The stopping norm of Sec. 3.4 (fire_norm) from the reductions.
__device__ __forceinline__ double force_norm(int norm, double F2, double fa2, double fin) {
    return norm == 1 ? sqrt(F2) : (norm == 2 ? fin : sqrt(fa2));
}

__device__ inline bool fire_control_step(const FireParamsD& p, FireScal& s, double P, double F2,
                                         double V2, double fa2, double fin) {
    s.evals += 1;
    const double fn = force_norm(p.norm, F2, fa2, fin);
    if (fn < p.ftol) {
        s.stop = STOP_FTOL;
        return true;
    }
    if (s.iter >= p.maxiter) {
        s.stop = STOP_MAXITER;
        return true;
    }
    const long long i = ++s.iter;
    s.lf_init = 0;
    if (p.integrator == INT_LEAPFROG && i == 1) {
        s.lf_init = 1;
        s.lf_c = -0.5 * p.dt_start / p.mass;
        P = s.lf_c * F2;                 // F . v(-dt/2)
        V2 = s.lf_c * s.lf_c * F2;
    }
    const double fnorm = sqrt(F2);
    s.zero_v = 0;
    s.halfstep = 0.0;
    s.premix = 0;
    s.postmix = 0;
    bool mix_in_integrator = false;
    if (p.variant == VAR_FIRE1) {
        if (P > 0.0) {
            s.npos += 1;
            s.premix = fnorm > 0.0;
            s.mix_a = s.alpha;
            s.mix_fv_pre = fnorm > 0.0 ? sqrt(V2) / fnorm : 0.0;
            if (s.npos > p.delaystep) {
                s.dt = fmin(s.dt * p.dtgrow, p.dtmax);
                s.alpha *= p.alphashrink;
            }
        } else {
            s.npos = 0;
            s.zero_v = 1;
            s.dt *= p.dtshrink;
            s.alpha = p.alpha0;
        }
    } else if (P > 0.0) {
        s.npos += 1;
        s.nneg = 0;
        if (s.npos > p.delaystep) {
            s.dt = fmin(s.dt * p.dtgrow, p.dtmax);
            s.alpha *= p.alphashrink;
        }
        mix_in_integrator = true;
    } else {
        s.npos = 0;
        s.nneg += 1;
        if (s.nneg > p.vdfmax) {
            s.stop = STOP_MAXVDOTF;
            s.iter = i - 1;
            return true;
        }
        if (!(p.initialdelay && i < p.delaystep)) {
            if (s.dt * p.dtshrink >= p.dtmin) s.dt *= p.dtshrink;
            s.alpha = p.alpha0;
        }
        s.zero_v = 1;
        s.halfstep = p.halfstepback ? 0.5 * s.dt : 0.0;
    }
    const double dtm = s.dt / p.mass;
    s.dtm = dtm;
    s.dt_cur = s.dt;
    s.kick_pre = p.integrator == INT_EULER_EXPLICIT ? 0.0
                 : (p.integrator == INT_VERLET ? 0.5 * dtm : dtm);
    s.kick_after = p.integrator == INT_EULER_EXPLICIT ? dtm : 0.0;
    s.vv = p.integrator == INT_VERLET;
    s.vv_half = p.integrator == INT_VERLET ? 0.5 * dtm : 0.0;
    if (mix_in_integrator && fnorm > 0.0) {
        s.mix_a = s.alpha;
        if (p.integrator == INT_EULER_EXPLICIT) {
            s.premix = 1;
            s.mix_fv_pre = sqrt(V2) / fnorm;
        } else {
            const double c = s.kick_pre;
            s.postmix = 1;
            s.mix_fv_post = sqrt(fmax(V2 + 2.0 * c * P + c * c * F2, 0.0)) / fnorm;
            s.post_v = 1.0 - s.alpha;
            s.post_f = s.post_v * c + s.alpha * s.mix_fv_post;
        }
    }
    return false;
}

// One atom of the element-wise step, in the order of the algorithms: the
// Leapfrog initial velocity, the half step back and v = 0 after P <= 0
// (Alg. 2, or v = 0 only for Alg. 1), mixing of v(t) (Algs. 1 and 3), the
// kick before the drift, mixing of the kicked velocity (Algs. 4-6), the
// drift x += dt v, and the explicit-Euler kick with the force at x(t).
// The part before the drift (everything the maximum-displacement cap needs
// to know the drift velocity), then the drift with a given dt and the
// explicit-Euler kick (fire_update_drift_k); the update passes chain the
// two with the FIRE dt.
__device__ __forceinline__ void fire_update_pre(const FireScal& s, dvec4& x, dvec4& v,
                                                const dvec4& f) {
    if (s.lf_init) v = make_dvec4(s.lf_c * f.x, s.lf_c * f.y, s.lf_c * f.z, 0.0);
    if (s.zero_v) {
        x.x -= s.halfstep * v.x;
        x.y -= s.halfstep * v.y;
        x.z -= s.halfstep * v.z;
        v = make_dvec4(0.0, 0.0, 0.0, 0.0);
    }
    if (s.premix) {
        const double a = s.mix_a, afv = s.mix_a * s.mix_fv_pre;
        v.x = (1.0 - a) * v.x + afv * f.x;
        v.y = (1.0 - a) * v.y + afv * f.y;
        v.z = (1.0 - a) * v.z + afv * f.z;
    }
    if (s.postmix) {
        // the kick and the mixing of the kicked velocity together: one FP64
        // multiply and one multiply-add per component in place of three
        // (FP64 issues at 1/58 of the FP32 rate on this part)
        v.x = fma(s.post_f, f.x, s.post_v * v.x);
        v.y = fma(s.post_f, f.y, s.post_v * v.y);
        v.z = fma(s.post_f, f.z, s.post_v * v.z);
    } else {
        v.x += s.kick_pre * f.x;
        v.y += s.kick_pre * f.y;
        v.z += s.kick_pre * f.z;
    }
}

// KICK: the kick after the drift (explicit Euler, s.kick_after != 0), a
// choice the caller makes once per pass rather than once per atom
template <bool KICK>
__device__ __forceinline__ void fire_update_drift_k(const FireScal& s, double dt, dvec4& x,
                                                    dvec4& v, const dvec4& f) {
    x.x += dt * v.x;
    x.y += dt * v.y;
    x.z += dt * v.z;
    if (KICK) {
        v.x += s.kick_after * f.x;
        v.y += s.kick_after * f.y;
        v.z += s.kick_after * f.z;
    }
}
// Drift timestep under the maximum-displacement cap: dmax / max_i |v_i| when
// dt max_i |v_i| exceeds dmax > 0, else dt.
__host__ __device__ inline double fire_capped_dt(double dt, double dmax, double vmax2) {
    if (dmax > 0.0) {
        const double vmax = sqrt(vmax2);
        if (dt * vmax > dmax) return dmax / vmax;
    }
    return dt;
}

// Velocity Verlet's second half kick with the new force (Algorithm 6).
__device__ __forceinline__ void fire_vv_kick(const FireScal& s, dvec4& v, const dvec4& f) {
    v.x += s.vv_half * f.x;
    v.y += s.vv_half * f.y;
    v.z += s.vv_half * f.z;
}

}  // namespace fire2
