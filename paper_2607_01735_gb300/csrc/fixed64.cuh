// 64-bit fixed-point helpers of the fused FP64 update (rbgs_opts.fma = 1).
//
// The fused update forms h2f + N + S + W + E exactly and rounds once:
//
//     u = RN( (T(h2f) + T(N) + T(S) + T(W) + T(E)) * 2^-(e+2) )
//
// where T(t) = trunc(t * 2^e) is a term on the fixed-point grid of step 2^-e (an int64),
// the five-term sum is exact integer arithmetic, the factor 2^-2 is the division by 4,
// and RN rounds to the nearest binary64, ties to even.  The scale e is chosen so that
// no term and no sum reaches 2^61 (scale_exponent below), and e <= kFixedMaxE keeps every
// nonzero result a normal number, so the rounding never meets the subnormal range.
//
// Everything is integer work (shifts, logic, adds, count-leading-zeros): on GB300 the
// update leaves the FP64 pipe, which bounds the bit-exact four-add form.
//
// The functions are __host__ __device__ so that the host test harness checks them against
// the C library's own conversions.
#pragma once

#include <cstdint>

#include "fp64.cuh"

namespace rbgs {

constexpr int kFixedMaxE = 1020;
constexpr int kFixedLimitBits = 61;  // |term|, |sum| < 2^61

// trunc(t * 2^e) for a finite t with |t| 2^e < 2^61 and e <= kFixedMaxE.  t = m 2^(E-1075)
// with m the 53-bit significand; m is placed at bits 10..62 and shifted right by
// r = 1085 - e - E (>= 2 for any t in range).  Zeros and subnormals (E = 0) give r >= 65
// for e <= 1020 and so 0, which is also their truncated value (|t| 2^e < 2^-2).
__host__ __device__ __forceinline__ int64_t to_fixed(double t, int e) {
    const uint64_t u = dbits(t);
    const int E = (int)((u >> 52) & 0x7FFu);
    const uint64_t M = ((u & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull) << 10;
    int r = 1085 - e - E;
    r = r < 63 ? r : 63;  // M < 2^63, so a shift by 63 leaves 0
    const int64_t mag = (int64_t)(M >> r);
    const int64_t neg = (int64_t)u >> 63;  // 0 or -1
    return (mag ^ neg) - neg;
}

// RN(s * 2^-(e+2)) as a binary64, for |s| < 2^63 and e <= kFixedMaxE (the result is then
// zero or normal).  |s| = an 2^-lz with an in [2^63, 2^64): the result's biased exponent is
// 1084 - lz - e, its significand the top 53 bits of an, rounded half to even on the 11 bits
// below; a carry out of the significand moves into the exponent field.
__host__ __device__ __forceinline__ double fixed_quarter_to_double(int64_t s, int e) {
    const uint64_t sign = (uint64_t)s & 0x8000000000000000ull;
    const uint64_t a = s < 0 ? (uint64_t)0 - (uint64_t)s : (uint64_t)s;
    const int lz = clz64(a);
    const uint64_t an = a << (lz & 63);
    const uint64_t mant = an >> 11;
    const uint64_t rem = an & 0x7FFull;
    const uint64_t inc = (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
    const uint64_t eb = (uint64_t)(int64_t)(1084 - lz - e);
    const uint64_t bits = (((eb - 1ull) << 52) + mant + inc) | sign;
    return a ? bitsd(bits) : 0.0;
}

// Scale of one block of nsweeps fused sweeps.  B = max |u| over the whole grid (ring
// included) and Q = max |h2 f| when the block starts.  An update changes no value by more
// than Q/4 beyond the largest neighbour, so after t sweeps every |u| <= B + t Q / 2 and
// every sum (before the division by 4) is at most S = 4 B + (2 nsweeps + 1) Q.  With
// S = m 2^k, 0.5 <= m < 1, e = 61 - k gives S 2^e < 2^61; e is capped at kFixedMaxE and
// is 0 when S = 0.  Returns false when B, Q or S is not finite (the caller then runs the
// bit-exact update instead).  S is formed as (4 B) + ((2 nsweeps + 1) Q), each operation
// correctly rounded, so that every implementation picks the same e.
__host__ __device__ __forceinline__ bool scale_exponent(double B, double Q, long long nsweeps, int *e) {
#if defined(__CUDA_ARCH__)
    const double S = __dadd_rn(__dmul_rn(4.0, B), __dmul_rn((double)(2 * nsweeps + 1), Q));
#else
    volatile double t1 = 4.0 * B;
    volatile double t2 = (double)(2 * nsweeps + 1) * Q;
    volatile double S = t1 + t2;
#endif
    if (!(S <= 1.7976931348623157e308)) return false;  // Inf or NaN
    if (S == 0.0) {
        *e = 0;
        return true;
    }
    int k = 0;
    frexp((double)S, &k);
    const int ee = kFixedLimitBits - k;
    *e = ee < kFixedMaxE ? ee : kFixedMaxE;
    return true;
}

// The fused update of one point from its five terms, already on the fixed-point grid.
__host__ __device__ __forceinline__ double fused_update(int64_t hf, int64_t vn, int64_t vs, int64_t vw, int64_t ve,
                                                        int e) {
    return fixed_quarter_to_double(hf + vn + vs + vw + ve, e);
}

}  // namespace rbgs
