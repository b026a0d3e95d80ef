// Correctly rounded division by 6 for the 3D update (rbgs3d.cu), in three FP64 operations.
// __host__ __device__ so that the host test harness checks it against IEEE division.
#pragma once

#include <cmath>
#include <cstdint>

#include "fp64.cuh"

namespace rbgs {

// s / 6 correctly rounded, in three FP64 operations: Markstein's correction step for division
// by a constant (P. Markstein, "Computation of elementary functions on the IBM RISC
// System/6000 processor", IBM J. Res. Dev. 34, 1990; N. Brisebarre, J.-M. Muller,
// S. K. Raina, "Accelerating correctly rounded floating-point division when the divisor is
// known in advance", IEEE Trans. Computers 53, 2004): with y = RN(1/6), q0 = RN(s y) is within
// an ulp of s/6, the remainder r = s - 6 q0 is exact in one fused multiply-add, and
// RN(q0 + r y) is the correctly rounded quotient.  Host-checked against IEEE division on
// structured and random operands over the whole normal range.  Outside biased exponents
// 7..2043 (tiny operands whose quotient or remainder nears the subnormal range, huge ones,
// Inf and NaN) the division instruction sequence takes over: on the device behind a vote of
// the active lanes, so that it is not issued for the common case.
__host__ __device__ __forceinline__ double div6(double s) {
    const double y6 = 0x1.5555555555555p-3;  // RN(1/3) / 2 = RN(1/6)
#if defined(__CUDA_ARCH__)
    const double q0 = __dmul_rn(s, y6);
    const double r = __fma_rn(-6.0, q0, s);
    double q = __fma_rn(r, y6, q0);
    const unsigned e = ((unsigned)__double2hiint(s) >> 20) & 0x7FFu;
    const bool ok = e - 7u <= 2036u;
    if (__any_sync(__activemask(), !ok)) {
        if (!ok) q = __ddiv_rn(s, 6.0);
    }
    return q;
#else
    const unsigned e = (unsigned)(dbits(s) >> 52) & 0x7FFu;
    if (e - 7u > 2036u) return s / 6.0;
    volatile double q0 = s * y6;
    const double r = fma(-6.0, (double)q0, s);
    return fma(r, y6, (double)q0);
#endif
}

}  // namespace rbgs
