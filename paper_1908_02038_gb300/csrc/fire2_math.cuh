// FP64 exponential for the pair functions of the RGL potential.
//
// GB300 issues FP64 at about 1/58 of its FP32 rate, so the two exponentials
// per pair dominate the density pass.  Their arguments, -p (r/r0 - 1) and
// -2q (r/r0 - 1), lie in a bounded interval (|x| < 700 is checked when the
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

}  // namespace fire2
