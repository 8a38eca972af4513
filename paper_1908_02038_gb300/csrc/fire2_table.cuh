// Tabulated RGL pair functions.
//
// The two exponentials, the square root and the taper of every pair are
// replaced by piecewise quintic Hermite polynomials in u = r^2 - r0^2:
//   density table: phi(u), g(u)               (6 coefficients each)
//   force table:   phi_u(u), g_u(u) = d/du    (6 coefficients each)
// with phi = A e^{-p(r/r0-1)} S(r) and g = xi^2 e^{-2q(r/r0-1)} S(r).  Since
// (dE/dr)/r = 2 dE/du, the force pass needs neither r nor 1/r.
//
// Knots: region A covers [u_lo, u_rs] with spacing hA, and u = 0 and
// u_rs = rs^2 - r0^2 are knots; region B covers the taper [u_rs, u_rc] with
// spacing hB (u_rc = rc^2 - r0^2 a knot), so the jumps of S''' at rs and rc
// fall on knots.  u_lo = -0.75 r0^2 (r = r0/2); closer pairs fall back to the
// analytic functions.  Each interval's quintic matches the function and its
// first two u-derivatives at both ends: for the density table f, f_u, f_uu
// and for the force table f_u, f_uu, f_uuu, with (primes = d/dr)
//   f_u = f'/(2r),  f_uu = (f'' - f'/r)/(4 r^2),
//   f_uuu = (f''' - 3 f''/r + 3 f'/r^2)/(8 r^3).
// With spacings near 0.04 A^2 (FP64 tables) the interpolation error is
// ~1e-11 relative or better on the Cu parameters (largest for pairs
// compressed towards r0/2, ~1e-12 above 0.8 r0); the FP32 tables use
// 0.12 A^2, still far below float rounding.
//
// Index arithmetic: region A uses x = u / hA (so pairs near r0, where the
// forces are stiffest, keep the full precision of u even in FP32), region B
// x = (u - u_rs) / hB.
#pragma once

#include <cmath>
#include <cstring>
#include <vector>

#include "fire2_common.cuh"

namespace fire2 {

constexpr int kTabDens = 12;    // coefficients per interval, density table
constexpr int kTabForce = 12;   // coefficients per interval, force table

struct RglTables {
    TabMeta meta;
    std::vector<double> dens64, force64;
    std::vector<float> dens32, force32;
};

// Analytic phi, g and their first three r-derivatives (host):
// out = (phi, phi', phi'', phi''', g, g', g'', g''').  taper < 0: decide from
// r; taper = 0: S = 1 (inside region A); taper = 1: the taper polynomial
// with t clamped to [0, 1] (inside region B) -- the table builder passes the
// region so that the one-sided limits at rs and rc are used (S''' jumps there).
inline void rgl_analytic(double A, double xi, double p, double q, double r0, double rs,
                         double rc, double r, double out[8], int taper = -1) {
    double S = 1.0, dS = 0.0, d2S = 0.0, d3S = 0.0;
    if (taper < 0) taper = (r >= rc) ? 2 : (r > rs ? 1 : 0);
    if (taper == 2) {
        S = 0.0;
    } else if (taper == 1) {
        const double w = rc - rs;
        double t = (r - rs) / w;
        t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
        S = 1.0 - 10.0 * t * t * t + 15.0 * t * t * t * t - 6.0 * t * t * t * t * t;
        dS = (-30.0 * t * t + 60.0 * t * t * t - 30.0 * t * t * t * t) / w;
        d2S = (-60.0 * t + 180.0 * t * t - 120.0 * t * t * t) / (w * w);
        d3S = (-60.0 + 360.0 * t - 360.0 * t * t) / (w * w * w);
    }
    const double s = r / r0 - 1.0;
    const double pre[2] = {A * std::exp(-p * s), xi * xi * std::exp(-2.0 * q * s)};
    const double rate[2] = {p / r0, 2.0 * q / r0};
    for (int k = 0; k < 2; ++k) {
        const double e = pre[k], a = rate[k];
        out[4 * k] = e * S;
        out[4 * k + 1] = e * (-a * S + dS);
        out[4 * k + 2] = e * (a * a * S - 2.0 * a * dS + d2S);
        out[4 * k + 3] = e * (-a * a * a * S + 3.0 * a * a * dS - 3.0 * a * d2S + d3S);
    }
}

// Quintic Hermite coefficients on [0, 1] from values F, scaled first
// derivatives D = h f_u and scaled second derivatives S = h^2 f_uu at both ends.
inline void quintic_hermite(double F0, double D0, double S0, double F1, double D1, double S1,
                            double c[6]) {
    const double dF = F1 - F0;
    c[0] = F0;
    c[1] = D0;
    c[2] = 0.5 * S0;
    c[3] = 10.0 * dF - 6.0 * D0 - 4.0 * D1 - 1.5 * S0 + 0.5 * S1;
    c[4] = -15.0 * dF + 8.0 * D0 + 7.0 * D1 + 1.5 * S0 - S1;
    c[5] = 6.0 * dF - 3.0 * D0 - 3.0 * D1 - 0.5 * S0 + 0.5 * S1;
}

// target: knot spacing in A^2 (0.04 for the FP64 tables, 0.12 for FP32).
inline RglTables build_rgl_tables(double A, double xi, double p, double q, double r0, double rs,
                                  double rc, double target = 0.04) {
    RglTables T;
    const double r02 = r0 * r0;
    const double u_rs = rs * rs - r02, u_rc = rc * rc - r02, u_min = -0.75 * r02;
    const int nAp = std::max(1, (int)std::ceil(u_rs / target));            // knots 0..u_rs
    const double hA = u_rs / nAp;
    const int nA0 = (int)std::ceil(-u_min / hA);                           // below u = 0
    const int nB = std::max(1, (int)std::ceil((u_rc - u_rs) / target));
    const double hB = (u_rc - u_rs) / nB;
    TabMeta& m = T.meta;
    m.nA0 = nA0;
    m.nA = nA0 + nAp;
    m.nB = nB;
    m.hA_inv = 1.0 / hA;
    m.hB_inv = 1.0 / hB;
    m.u_lo = -nA0 * hA;
    m.u_rs = u_rs;
    m.hA_inv_f = (float)m.hA_inv;
    m.hB_inv_f = (float)m.hB_inv;
    m.u_lo_f = (float)m.u_lo;
    m.u_rs_f = (float)u_rs;
    const int nint = m.nA + m.nB;
    T.dens64.resize((size_t)nint * kTabDens);
    T.force64.resize((size_t)nint * kTabForce);
    // f, f_u, f_uu, f_uuu in u for phi (k = 0) and g (k = 1)
    auto derivs_u = [&](double u, int taper, double f[2][4]) {
        const double r = std::sqrt(r02 + u);
        double a[8];
        rgl_analytic(A, xi, p, q, r0, rs, rc, r, a, taper);
        for (int k = 0; k < 2; ++k) {
            const double f0 = a[4 * k], f1 = a[4 * k + 1], f2 = a[4 * k + 2], f3 = a[4 * k + 3];
            f[k][0] = f0;
            f[k][1] = f1 / (2.0 * r);
            f[k][2] = (f2 - f1 / r) / (4.0 * r * r);
            f[k][3] = (f3 - 3.0 * f2 / r + 3.0 * f1 / (r * r)) / (8.0 * r * r * r);
        }
    };
    for (int i = 0; i < nint; ++i) {
        double ua, h;
        if (i < m.nA) {
            h = hA;
            ua = (i - nA0) * hA;
        } else {
            h = hB;
            ua = u_rs + (i - m.nA) * hB;
        }
        const double ub = (i == m.nA - 1) ? u_rs : ((i == nint - 1) ? u_rc : ua + h);
        double fa[2][4], fb[2][4];
        const int taper = i < m.nA ? 0 : 1;
        derivs_u(ua, taper, fa);
        derivs_u(ub, taper, fb);
        for (int k = 0; k < 2; ++k) {
            double c[6];
            quintic_hermite(fa[k][0], h * fa[k][1], h * h * fa[k][2], fb[k][0], h * fb[k][1],
                            h * h * fb[k][2], c);
            for (int j = 0; j < 6; ++j) T.dens64[(size_t)i * kTabDens + 6 * k + j] = c[j];
            quintic_hermite(fa[k][1], h * fa[k][2], h * h * fa[k][3], fb[k][1], h * fb[k][2],
                            h * h * fb[k][3], c);
            for (int j = 0; j < 6; ++j) T.force64[(size_t)i * kTabForce + 6 * k + j] = c[j];
        }
    }
    T.dens32.assign(T.dens64.begin(), T.dens64.end());
    T.force32.assign(T.force64.begin(), T.force64.end());
    return T;
}

// Interval index and local coordinate t in [0, 1]; false outside the table
// (u < u_lo; u >= u_rc never reaches here because of the cut-off test).
__host__ __device__ __forceinline__ bool tab_locate(const TabMeta& m, double u, int& k, double& t) {
    if (u < m.u_lo) return false;
    double x;
    if (u < m.u_rs) {
        x = u * m.hA_inv;
        const double fl = floor(x);
        k = (int)fl + m.nA0;
        t = x - fl;
        if (k >= m.nA) {   // rounding at u_rs
            k = m.nA - 1;
            t = 1.0;
        }
    } else {
        x = (u - m.u_rs) * m.hB_inv;
        const double fl = floor(x);
        k = (int)fl;
        t = x - fl;
        if (k >= m.nB) {
            k = m.nB - 1;
            t = 1.0;
        }
        k += m.nA;
    }
    if (k < 0) {
        k = 0;
        t = 0.0;
    }
    return true;
}

__device__ __forceinline__ bool tab_locate_f(const TabMeta& m, float u, int& k, float& t) {
    if (u < m.u_lo_f) return false;
    if (u < m.u_rs_f) {
        const float x = u * m.hA_inv_f;
        const float fl = floorf(x);
        k = (int)fl + m.nA0;
        t = x - fl;
        if (k >= m.nA) {
            k = m.nA - 1;
            t = 1.f;
        }
    } else {
        const float x = (u - m.u_rs_f) * m.hB_inv_f;
        const float fl = floorf(x);
        k = (int)fl;
        t = x - fl;
        if (k >= m.nB) {
            k = m.nB - 1;
            t = 1.f;
        }
        k += m.nA;
    }
    if (k < 0) {
        k = 0;
        t = 0.f;
    }
    return true;
}

template <typename T>
__host__ __device__ __forceinline__ T poly5(const T* c, T t) {
    return ((((c[5] * t + c[4]) * t + c[3]) * t + c[2]) * t + c[1]) * t + c[0];
}
template <typename T>
__host__ __device__ __forceinline__ T poly4(const T* c, T t) {
    return (((c[4] * t + c[3]) * t + c[2]) * t + c[1]) * t + c[0];
}

}  // namespace fire2

namespace fire2 {

// ---------------------------------------------------------------------------
// FP64-accurate pair terms without FP64 instructions.
//
// FP64 instructions issue at 1/58 of the FP32 rate on this part, so the FP64
// form's pair passes use no FP64 instruction per pair:
//   * separations are exact: positions in 64-bit fixed point (2^44 units per
//     A, i.e. a grid finer than the last bit of a double coordinate beyond
//     ~2 A), differences in integers, then split exactly into two floats;
//   * everything else is double-float arithmetic: each value is an
//     unevaluated sum hi + lo of two floats (Dekker 1971; Knuth's TwoSum),
//     good to ~2^-44 relative, in FP32 instructions only:
//       r^2 = dx^2 + dy^2 + dz^2,  s = r^2 - (u_k + r0^2),
//       f = c0 + s (c1 + s (c2 + s q)),   q = c3 + s (c4 + s c5)
//     with c0..c2 and s as float pairs and q in plain FP32: on these tables
//     |s c_{j+1} / c_j| < ~0.07, so s^3 q is < ~1e-4 of f and its FP32
//     rounding enters at ~1e-11 relative or less;
//   * the cut-off test and the interval index use the FP32 high part of r^2:
//     the taper makes phi, g and their first two derivatives vanish at rc,
//     so a pair within FP32 rounding of rc contributes nothing either way,
//     and an index one off at an interval edge only moves s by ~1e-6 of the
//     interval outside [0, h], where the quintic is still accurate.
// Float/double crossings (per atom only) are integer operations on the
// IEEE-754 fields.
//
// Rows (kFFRow floats = 80 bytes, 16-byte aligned): [0], [1] u_k + r0^2 as
// hi, lo; then two polynomials of 9 floats each: c0 hi, c0 lo, c1 hi, c1 lo,
// c2 hi, c2 lo, c3, c4, c5 (coefficients in s, i.e. divided by h^j).
// Density rows: phi, g.  Force rows: 4 phi_u = 2 phi'/r, 2 g_u = g'/r.

constexpr int kFFRow = 20;
constexpr int kFixedBits64 = 44;   // fixed-point positions of the FP64 form: 2^44 per A


__host__ __device__ __forceinline__ void dbl_words(double d, unsigned& hi, unsigned& lo) {
#ifdef __CUDA_ARCH__
    hi = (unsigned)__double2hiint(d);
    lo = (unsigned)__double2loint(d);
#else
    unsigned long long b;
    std::memcpy(&b, &d, sizeof b);
    hi = (unsigned)(b >> 32);
    lo = (unsigned)b;
#endif
}

__host__ __device__ __forceinline__ double dbl_from_words(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)hi, (int)lo);
#else
    const unsigned long long b = ((unsigned long long)hi << 32) | lo;
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
#endif
}

__host__ __device__ __forceinline__ float flt_from_bits(unsigned b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    std::memcpy(&f, &b, sizeof f);
    return f;
#endif
}

__host__ __device__ __forceinline__ unsigned flt_bits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    unsigned b;
    std::memcpy(&b, &f, sizeof b);
    return b;
#endif
}

// double -> float by truncating the significand (exponent rebiased by
// 1023 - 127 = 896); magnitudes below 2^-126 give +-0, none here exceed 2^127.
__host__ __device__ __forceinline__ float f64_to_f32_trunc(double d) {
    unsigned hi, lo;
    dbl_words(d, hi, lo);
    const unsigned sgn = hi & 0x80000000u, ahi = hi & 0x7fffffffu;
    if (ahi < (897u << 20)) return flt_from_bits(sgn);
    return flt_from_bits(sgn | ((ahi - (896u << 20)) << 3) | (lo >> 29));
}

// float -> double, exact for normal floats (zero and subnormals give +-0).
__host__ __device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned b = flt_bits(f), a = b & 0x7fffffffu;
    if (a < 0x00800000u) return dbl_from_words(b & 0x80000000u, 0u);
    return dbl_from_words((b & 0x80000000u) | ((a >> 3) + (896u << 20)), a << 29);
}

// Rounded FP32 operations the compiler may not fuse into FMAs (the error
// terms below depend on the exact rounding of each step).
__host__ __device__ __forceinline__ float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ __forceinline__ float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}

struct ffloat {
    float hi, lo;
};

// a + b = s + e exactly (Knuth's TwoSum)
__host__ __device__ __forceinline__ ffloat two_sum(float a, float b) {
    const float s = add_rn(a, b);
    const float bb = add_rn(s, -a);
    const float e = add_rn(add_rn(a, -add_rn(s, -bb)), add_rn(b, -bb));
    return {s, e};
}
// a + b = s + e exactly when |a| >= |b| (Dekker's Fast2Sum)
__host__ __device__ __forceinline__ ffloat fast_two_sum(float a, float b) {
    const float s = add_rn(a, b);
    return {s, add_rn(b, -add_rn(s, -a))};
}
__host__ __device__ __forceinline__ ffloat ff_add(ffloat a, ffloat b) {
    const ffloat s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, add_rn(s.lo, add_rn(a.lo, b.lo)));
}
// (a.hi + a.lo)(b.hi + b.lo) without the lo*lo term
__host__ __device__ __forceinline__ ffloat ff_mul(ffloat a, ffloat b) {
    const float p = mul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);
    return fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
// a b as an unnormalised pair (p, t): p = fl(a.hi b.hi), t its error plus
// the cross terms, |t| ~ 2^-23 |p|; exact input for ff_acc, ff_to_f64 and
// the TwoSum of ff_madd, which take any pair
__host__ __device__ __forceinline__ ffloat ff_mul_nn(ffloat a, ffloat b) {
    const float p = mul_rn(a.hi, b.hi);
    return {p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)))};
}
// c + a b with one renormalisation: the product's error and cross terms
// join the low part of the TwoSum of c.hi and fl(a.hi b.hi) (a.lo b.lo
// dropped, as in ff_mul); 15 FP32 instructions against 18 for
// ff_add(c, ff_mul(a, b)), the same error bound
__host__ __device__ __forceinline__ ffloat ff_madd(ffloat a, ffloat b, ffloat c) {
    const ffloat p = ff_mul_nn(a, b);
    const ffloat s = two_sum(c.hi, p.hi);
    return fast_two_sum(s.hi, add_rn(s.lo, add_rn(c.lo, p.lo)));
}
// c + a b for a float b
__host__ __device__ __forceinline__ ffloat ff_madd_f(ffloat a, float b, ffloat c) {
    const float p = mul_rn(a.hi, b);
    const ffloat s = two_sum(c.hi, p);
    return fast_two_sum(s.hi, add_rn(s.lo, add_rn(c.lo, fmaf(a.lo, b, fmaf(a.hi, b, -p)))));
}
__host__ __device__ __forceinline__ double ff_to_f64(ffloat a) {
    return f32_to_f64(a.hi) + f32_to_f64(a.lo);
}
// Running sum of double-float terms: TwoSum on the high parts, the low
// parts and the TwoSum errors added in plain FP32, no renormalisation
// (ff_to_f64 takes the pair as it is).  Over the few dozen terms of one
// atom's list the low sum stays below ~2^-48 of the largest term.
__host__ __device__ __forceinline__ ffloat ff_acc(ffloat acc, ffloat t) {
    const ffloat s = two_sum(acc.hi, t.hi);
    return {s.hi, add_rn(acc.lo, add_rn(s.lo, t.lo))};
}
// d (|d| < 2^127) as hi + lo, both truncated: |d - hi - lo| < 2^-46 |d|
__host__ __device__ __forceinline__ ffloat f64_to_ff(double d) {
    const float hi = f64_to_f32_trunc(d);
    return {hi, f64_to_f32_trunc(d - f32_to_f64(hi))};
}

// RGL embedding of the double-float form: sqrt(rho) and F'(rho) =
// -1/(2 sqrt(rho)) as float pairs from one reciprocal square root y.  The
// FP32 estimate y0 (relative error e0 ~ 2^-22) takes one Newton step on
// 1/y^2 - rho, y1 = y0 + y0 (1 - rho y0^2) / 2, with 1 - rho y0^2 formed in
// float pairs; y1 is then off by 1.5 e0^2 ~ 1e-13 (relative, from below),
// the precision of the pair terms.  FP32 and integer instructions only (FP64
// issues at 1/58 of the FP32 rate on this part).  Valid for rho in the
// normal FP32 range; the caller takes the FP64 routine outside it.
__device__ __forceinline__ void rgl_embed_ff(ffloat r, ffloat& sq, ffloat& fp) {
    const float y0 = rsqrtf(r.hi);
    const float p = y0 * y0;
    const ffloat y0sq = {p, fmaf(y0, y0, -p)};              // exact square
    const ffloat t = ff_mul(r, y0sq);                       // rho y0^2 ~ 1
    const ffloat e = ff_add({1.f, 0.f}, {-t.hi, -t.lo});     // ~2^-22
    const ffloat y1 = fast_two_sum(y0, 0.5f * y0 * e.hi);
    sq = ff_mul(r, y1);
    fp = {-0.5f * y1.hi, -0.5f * y1.lo};                    // exact scaling
}

// Whether 2^-60 < d < 2^60, on the integer pipes (positive doubles order
// like their bit patterns; negative values and NaN fail).
__device__ __forceinline__ bool ff_range(double d) {
    const long long bits = __double_as_longlong(d);
    return bits > 0x3C30000000000000ll && bits < 0x43B0000000000000ll;
}

// d with ff_range(d) as a float pair without an FP64 instruction: hi is d
// truncated to 24 significant bits (f64_to_f32_trunc), lo the remaining 29
// bits of the significand, rem 2^(e - 52), rounded to 24 bits
// (|d - hi - lo| <= 2^-48 |d|).
__device__ __forceinline__ ffloat f64_to_ff_int(double d) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((bits >> 52) & 0x7ffull) - 1023;               // -60 <= e < 60
    const float scale = __int_as_float((e - 52 + 127) << 23);          // 2^(e - 52)
    const float lo = __uint2float_rn((unsigned)(bits & 0x1fffffffull)) * scale;
    return {f64_to_f32_trunc(d), lo};
}

// The embedding of the double-float form at an FP64 density: sqrt(rho) and
// F'(rho) in FP64, and F' as the float pair the force pass reads.
__device__ __forceinline__ void rgl_embed_dd(double rho, double& sq, double& fp, ffloat& fpf) {
    if (ff_range(rho)) {
        ffloat sqf;
        rgl_embed_ff(f64_to_ff_int(rho), sqf, fpf);
        sq = ff_to_f64(sqf);
        fp = ff_to_f64(fpf);
    } else {
        rgl_embed(rho, sq, fp);
        fpf = f64_to_ff(fp);
    }
}

// One quintic of a row: c = 9 floats (see the layout above), s as a float pair.
// Horner steps c_k + s r as fused double-float multiply-adds.
__host__ __device__ __forceinline__ ffloat ff_poly(const float* c, ffloat s) {
    const float q = fmaf(fmaf(c[8], s.hi, c[7]), s.hi, c[6]);
    ffloat r = ff_madd_f(s, q, {c[4], c[5]});
    r = ff_madd(s, r, {c[2], c[3]});
    return ff_madd(s, r, {c[0], c[1]});
}

__host__ __device__ __forceinline__ ffloat ff_neg(ffloat a) { return {-a.hi, -a.lo}; }

// Interval of u (from its FP32 copy uf), clamped to the table.
__host__ __device__ __forceinline__ int ff_index(const TabMeta& m, float uf) {
    int k = uf < m.u_rs_f ? m.nA0 + (int)floorf(uf * m.hA_inv_f)
                          : m.nA + (int)floorf((uf - m.u_rs_f) * m.hB_inv_f);
    const int last = m.nA + m.nB - 1;
    return k < 0 ? 0 : (k > last ? last : k);
}

// Row k of a table in global memory (80 bytes, 16-byte aligned), through L1.
__device__ __forceinline__ void load_row(const float* tab, int k, float row[kFFRow]) {
    const float4* src = reinterpret_cast<const float4*>(tab + (size_t)k * kFFRow);
#pragma unroll
    for (int q = 0; q < kFFRow / 4; ++q) {
        const float4 v = __ldg(src + q);
        row[4 * q] = v.x;
        row[4 * q + 1] = v.y;
        row[4 * q + 2] = v.z;
        row[4 * q + 3] = v.w;
    }
}

// The two polynomials of `row` at r^2 (float pair): out[0], out[1].
__host__ __device__ __forceinline__ void ff_row_eval(const float* row, ffloat r2, ffloat out[2]) {
    // s = r^2 - (u_k + r0^2): r2.hi and the knot's high part row[0] lie
    // within a factor 2 of each other (r^2 falls in the knot's interval,
    // ~0.04 A^2 wide, above 0.25 r0^2), so their difference is exact
    // (Sterbenz); the low parts' difference joins it in one Fast2Sum (where
    // that difference exceeds the first, both are below 2^-20 A^2 and the
    // pair is off by far less than 2^-40 A^2)
    const ffloat s = fast_two_sum(add_rn(r2.hi, -row[0]), add_rn(r2.lo, -row[1]));
    out[0] = ff_poly(row + 2, s);
    out[1] = ff_poly(row + 11, s);
}

// Exact split of a 64-bit integer |n| < 2^47 times 2^-kFixedBits64 into a
// float pair (both parts exact: 24 + 23 bits).
__host__ __device__ __forceinline__ ffloat fixed_to_ff(long long n) {
    const long long a = n >> 23;                          // floor(n / 2^23)
    const unsigned b = (unsigned)n & 0x7fffffu;           // n - a 2^23, 0 <= b < 2^23
    const float hi = (float)(int)a * 0x1p-21f;            // 2^(23 - 44)
    // b 2^-44 without an integer-to-float conversion: the float with
    // exponent -21 and significand bits b is 2^-21 (1 + b 2^-23), and taking
    // 2^-21 from it is exact (Sterbenz)
    const float lo = add_rn(flt_from_bits((106u << 23) | b), -0x1p-21f);
    return fast_two_sum(hi, lo);   // |hi| >= 2^-21 > lo >= 0, or hi = 0
}

// x^2 + y^2 + z^2 of normalised float pairs: exact products of the high
// parts, the cross terms 2 hi lo added to their errors (lo^2 < 2^-48 hi^2 is
// dropped), one renormalisation at the end.
__host__ __device__ __forceinline__ ffloat ff_norm2(ffloat x, ffloat y, ffloat z) {
    const float px = mul_rn(x.hi, x.hi), py = mul_rn(y.hi, y.hi), pz = mul_rn(z.hi, z.hi);
    const float ex = fmaf(2.f * x.hi, x.lo, fmaf(x.hi, x.hi, -px));
    const float ey = fmaf(2.f * y.hi, y.lo, fmaf(y.hi, y.hi, -py));
    const float ez = fmaf(2.f * z.hi, z.lo, fmaf(z.hi, z.hi, -pz));
    const ffloat s1 = two_sum(px, py);
    const ffloat s2 = two_sum(s1.hi, pz);
    return fast_two_sum(s2.hi, add_rn(add_rn(s1.lo, s2.lo), add_rn(add_rn(ex, ey), ez)));
}

// Host evaluation with the kernels' arithmetic (diagnostic): row of the
// table of u = r^2 - r0^2, or NULL below the table (u < u_lo, where the
// kernels use the exponentials).
inline const float* ff_row(const TabMeta& m, const std::vector<float>& tab, float uf) {
    if (uf < m.u_lo_f) return nullptr;
    return tab.data() + (size_t)ff_index(m, uf) * kFFRow;
}

// Density rows (phi, g) and force rows (2 phi'/r, g'/r) from the Hermite
// coefficients of build_rgl_tables (in t = s / h).
inline void build_ff_tables(const RglTables& T, double r0, std::vector<float>& dens,
                            std::vector<float>& force) {
    const TabMeta& m = T.meta;
    const int nint = m.nA + m.nB;
    dens.assign((size_t)nint * kFFRow, 0.f);
    force.assign((size_t)nint * kFFRow, 0.f);
    const double hA = 1.0 / m.hA_inv, hB = 1.0 / m.hB_inv;
    const double scale[4] = {1.0, 1.0, 4.0, 2.0};
    auto split = [](double v, float* o) {
        const float hi = (float)v;
        o[0] = hi;
        o[1] = (float)(v - (double)hi);
    };
    for (int i = 0; i < nint; ++i) {
        const double h = i < m.nA ? hA : hB;
        const double uk = i < m.nA ? (i - m.nA0) * hA : m.u_rs + (i - m.nA) * hB;
        float* rows[2] = {dens.data() + (size_t)i * kFFRow, force.data() + (size_t)i * kFFRow};
        split(uk + r0 * r0, rows[0]);
        split(uk + r0 * r0, rows[1]);
        for (int p = 0; p < 4; ++p) {
            const double* src = (p < 2 ? T.dens64.data() + (size_t)i * kTabDens + 6 * p
                                       : T.force64.data() + (size_t)i * kTabForce + 6 * (p - 2));
            double hp = 1.0;
            double cs[6];
            for (int j = 0; j < 6; ++j) {
                cs[j] = scale[p] * src[j] / hp;
                hp *= h;
            }
            float* o = rows[p / 2] + 2 + 9 * (p % 2);
            for (int j = 0; j < 3; ++j) split(cs[j], o + 2 * j);
            for (int j = 0; j < 3; ++j) o[6 + j] = (float)cs[3 + j];
        }
    }
}

}  // namespace fire2
