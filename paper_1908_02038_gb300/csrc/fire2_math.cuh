// FP64 exponential for the pair functions of the RGL potential.
//
// GB300 issues FP64 at about 1/58 of its FP32 rate, so the two exponentials
// per pair dominate the density pass.  Their arguments, -p (r/r0 - 1) and
// -2q (r/r0 - 1), lie in a bounded interval (|x| < 80 is checked when the
// potential is set up), so no overflow, underflow or special-value handling
// is needed.  The method is P. T. P. Tang's table-driven exponential
// ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989):
//
//   x = k ln2/N + r,  k = m N + j,  |r| <= ln2/(2N),  e^x = 2^m 2^(j/N) e^r,
//
// with N = 256, the Cody-Waite two-part constant ln2/N = c_hi + c_lo (c_hi
// has 32 significant bits so k c_hi is exact), the table T[j] = 2^(j/N) in
// shared memory, and e^r - 1 by its Taylor series to r^4/24 (truncation
// below 4e-17 relative for |r| <= 1.36e-3).  The scaling by 2^m adds m to the
// exponent field with integer instructions.
#pragma once

#include <cmath>
#include <cuda_runtime.h>

namespace fire2 {

constexpr int kExpTableBits = 8;
constexpr int kExpTableSize = 1 << kExpTableBits;

struct ExpC {
    double inv_c;     // N / ln2
    double c_hi;      // ln2 / N, 32 significant bits
    double c_lo;      // ln2 / N - c_hi
};

// Host-side set-up of the constants and the table (2^(j/N), correctly
// rounded up to the host libm's exp2 accuracy).
inline ExpC make_exp_constants(double* table) {
    // ln 2 = LN2_HI + LN2_LO (the double nearest ln 2 and the remainder)
    const double LN2_HI = 0x1.62e42fefa39efp-1;
    const double LN2_LO = 0x1.abc9e3b39803fp-56;
    ExpC c;
    const double cn = LN2_HI / kExpTableSize;
    int e = 0;
    std::frexp(cn, &e);
    c.c_hi = std::ldexp(std::trunc(std::ldexp(cn, 32 - e)), e - 32);
    c.c_lo = ((LN2_HI - kExpTableSize * c.c_hi) + LN2_LO) / kExpTableSize;
    c.inv_c = kExpTableSize / LN2_HI;
    for (int j = 0; j < kExpTableSize; ++j) table[j] = std::exp2((double)j / kExpTableSize);
    return c;
}

// e^x for |x| < 700 (see above).  `tbl` is the 2^(j/N) table in shared memory.
__device__ __forceinline__ double exp_tang(double x, const ExpC& c, const double* tbl) {
    const double magic = 0x1.8p52;               // 1.5 * 2^52: rounds to an integer
    const double t = fma(x, c.inv_c, magic);
    const double kd = t - magic;
    const int k = __double2loint(t);              // the same integer, two's complement
    double r = fma(-kd, c.c_hi, x);               // exact (Cody-Waite)
    r = fma(-kd, c.c_lo, r);
    // e^r - 1 = r (1 + r (1/2 + r (1/6 + r/24)))
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p *= r;
    const double tj = tbl[k & (kExpTableSize - 1)];
    const double y = fma(tj, p, tj);
    const int m = k >> kExpTableBits;             // arithmetic shift = floor(k / N)
    return __hiloint2double(__double2hiint(y) + (m << 20), __double2loint(y));
}

// ---------------------------------------------------------------------------
// FP32 version for the FP32-pair form: the same method with N = 64 and
// e^r - 1 to r^3/6 (truncation below 4e-11 for |r| <= 5.5e-3), valid for
// |x| < 87.  The table holds 2^(j/64) rounded to float; the result is within
// about one float ulp.

constexpr int kExp32TableBits = 6;
constexpr int kExp32TableSize = 1 << kExp32TableBits;

struct Exp32C {
    float inv_c;      // 64 / ln2
    float c_hi;       // ln2 / 64 with 12 significant bits (k c_hi exact for |k| < 2^11)
    float c_lo;       // ln2 / 64 - c_hi
};

inline Exp32C make_exp32_constants(float* table) {
    const double LN2_HI = 0x1.62e42fefa39efp-1;
    Exp32C c;
    const double cn = LN2_HI / kExp32TableSize;
    int e = 0;
    std::frexp(cn, &e);
    const double hi = std::ldexp(std::trunc(std::ldexp(cn, 12 - e)), e - 12);
    c.c_hi = (float)hi;
    c.c_lo = (float)(cn - hi);
    c.inv_c = (float)(kExp32TableSize / LN2_HI);
    for (int j = 0; j < kExp32TableSize; ++j) table[j] = (float)std::exp2((double)j / kExp32TableSize);
    return c;
}

__device__ __forceinline__ float exp32_tang(float x, const Exp32C& c, const float* tbl) {
    const float magic = 0x1.8p23f;                // 1.5 * 2^23
    const float t = fmaf(x, c.inv_c, magic);
    const float kd = t - magic;
    const int k = __float_as_int(t) - 0x4B400000;  // the integer kd
    float r = fmaf(-kd, c.c_hi, x);
    r = fmaf(-kd, c.c_lo, r);
    float q = fmaf(r, 1.0f / 6.0f, 0.5f);
    q = fmaf(q, r, 1.0f);
    const float p = q * r;
    const float tj = tbl[k & (kExp32TableSize - 1)];
    const float y = fmaf(tj, p, tj);
    const int m = k >> kExp32TableBits;
    return __int_as_float(__float_as_int(y) + (m << 23));
}

// RGL embedding F(rho) = -sqrt(rho) at density rho: sqrt(rho) and
// F'(rho) = -1/(2 sqrt(rho)) from one reciprocal square root y.  Newton's
// method on f(y) = 1/y^2 - rho gives y <- y + y (1 - rho y^2) / 2, which
// squares the relative error of y at each step: from the FP32 estimate
// (~2e-7) two steps land below the FP64 rounding, so sqrt(rho) = rho y and
// F' = -y/2 are within a few FP64 ulps -- about ten FP64 instructions in
// place of an IEEE square root and an IEEE division (FP64 issues at 1/58 of
// FP32 on this part).  Densities outside the FP32 range take the IEEE
// operations; rho <= 0 (no pair inside rc) gives sqrt = 0, F' = 0.
__device__ __forceinline__ double rsqrt_newton(double x) {
    double y = (double)rsqrtf((float)x);
    for (int k = 0; k < 2; ++k) {
        const double e = fma(-x * y, y, 1.0);
        y = fma(0.5 * y, e, y);
    }
    return y;
}

__device__ __forceinline__ void rgl_embed(double rho, double& sq, double& fp) {
    if (rho > 1e-30 && rho < 1e30) {
        const double y = rsqrt_newton(rho);
        sq = rho * y;
        fp = -0.5 * y;
    } else {
        sq = sqrt(rho);
        fp = rho > 0.0 ? -0.5 / sq : 0.0;
    }
}

// Compensated (Kahan) accumulation in FP32: sum + c carries the running
// total to about one float ulp of the sum.
struct Kahan32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

}  // namespace fire2
