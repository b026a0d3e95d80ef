// Exact binary64 helpers for the RBGS update on GB300.
//
// GB300 issues FP64 arithmetic at a small fraction of its FP32 and INT32 rates, so
// the bit-exact update (((h2f + N) + S) + W) + E, times 0.25, is limited by the FP64
// pipe long before HBM.  These helpers move work to the integer pipe without changing
// a single result bit:
//
//  * quarter(s): s * 0.25 by subtracting 2 from the biased exponent whenever the result
//    stays a normal number (biased exponent of s in 3..2046), which is exact; zeros,
//    subnormal results, Inf and NaN go through an integer rounding of the significand
//    (quarter_bits_small), so the multiply never reaches the FP64 pipe.
//  * add_int(a, b): IEEE 754 binary64 addition with round-to-nearest-even, written from
//    the standard's definition (align, add or subtract the 53-bit significands with
//    guard bits and a sticky bit, normalise, round half to even).  It handles finite
//    normal operands whose sum is normal; any other case (a zero or subnormal operand,
//    Inf/NaN, an exactly cancelling or subnormal sum, overflow past the largest
//    exponent before rounding) falls back to the hardware add.
//  * add_fma(a, b, one): a + b computed as fma(a, one, b) with one == 1.0: one rounding
//    of the exact sum, the same value as the add instruction.
//
// The functions are __host__ __device__ so that the host test harness can check them
// against the CPU's own IEEE addition.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rbgs {

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(uint64_t u) { return __longlong_as_double((long long)u); }
__device__ __forceinline__ int clz64(uint64_t x) { return __clzll((long long)x); }
__device__ __forceinline__ double hw_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double hw_mul(double a, double b) { return __dmul_rn(a, b); }
#else
inline uint64_t dbits(double x) { uint64_t u; __builtin_memcpy(&u, &x, 8); return u; }
inline double bitsd(uint64_t u) { double x; __builtin_memcpy(&x, &u, 8); return x; }
inline int clz64(uint64_t x) { return x ? __builtin_clzll(x) : 64; }
inline double hw_add(double a, double b) { volatile double s = a + b; return s; }
inline double hw_mul(double a, double b) { volatile double p = a * b; return p; }
#endif

// s * 0.25, exactly as the multiply would round it.  On the device the multiply of the
// rare path sits behind a warp vote and an opaque instruction, so that the compiler can
// neither evaluate it speculatively nor predicate it into the common path (either would
// put an FP64 instruction back on the pipe for every update).  All 32 lanes of the warp
// must call it together.
// s * 0.25 for the cases the exponent decrement cannot take (biased exponent 0, 1, 2 or
// 2047), from the definition of the binary64 format: Inf and NaN are returned unchanged;
// otherwise s = m 2^(max(e, 1) - 1075) with m the significand (implicit bit included when
// e > 0), so s / 4 = (m / 2^k) 2^-1074 with k = 1 for e = 2 and k = 2 for e = 0, 1: a
// subnormal (or zero) whose significand is m / 2^k rounded half to even.  A carry to 2^52
// is the encoding of the smallest normal number, so sign | q is the result in every case.
// Integer operations only: the FP64 pipe never sees this path.
__host__ __device__ __forceinline__ uint64_t quarter_bits_small(uint64_t u) {
    const unsigned e = (unsigned)(u >> 52) & 0x7FFu;
    if (e == 0x7FFu) return u;
    const uint64_t sign = u & 0x8000000000000000ull;
    const uint64_t m = (u & 0x000FFFFFFFFFFFFFull) | (e ? 0x0010000000000000ull : 0ull);
    const unsigned k = e == 2u ? 1u : 2u;
    uint64_t q = m >> k;
    const uint64_t rem = m & ((1ull << k) - 1ull), half = 1ull << (k - 1u);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    return sign | q;
}

__host__ __device__ __forceinline__ double quarter(double s) {
#if defined(__CUDA_ARCH__)
    const int hi = __double2hiint(s);
    const int lo = __double2loint(s);
    const unsigned e = ((unsigned)hi >> 20) & 0x7FFu;
    const bool fast = e - 3u <= 2043u;
    double r = __hiloint2double(hi - (2 << 20), lo);
    if (__any_sync(0xffffffffu, !fast)) {
        if (!fast) r = bitsd(quarter_bits_small(dbits(s)));
    }
    return r;
#else
    uint64_t u = dbits(s);
    unsigned e = (unsigned)(u >> 52) & 0x7FFu;
    if (e - 3u <= 2043u) return bitsd(u - (2ull << 52));
    return bitsd(quarter_bits_small(u));
#endif
}

// a + b computed as fma(a, one, b) with one == 1.0: one rounding of the exact sum, the
// same value as the add instruction.  `one` must come from run-time data (a kernel
// argument) so that the compiler keeps the fused multiply-add, which GB300 issues at a
// higher rate than the add.
__host__ __device__ __forceinline__ double add_fma(double a, double b, double one) {
#if defined(__CUDA_ARCH__)
    return __fma_rn(a, one, b);
#else
    (void)one;
    return hw_add(a, b);
#endif
}

// a + b on the integer pipe, round to nearest even.  Sets ok = false (result undefined)
// outside the domain given in the file comment.
__host__ __device__ __forceinline__ double add_int_core(double a, double b, bool &ok) {
    const uint64_t SIGN = 0x8000000000000000ull;
    const uint64_t FRAC = 0x000FFFFFFFFFFFFFull;
    const uint64_t HID = 0x0010000000000000ull;
    uint64_t A = dbits(a), B = dbits(b);
    uint64_t ma = A & ~SIGN, mb = B & ~SIGN;
    bool a_big = ma >= mb;
    uint64_t big = a_big ? A : B;
    uint64_t mbig = a_big ? ma : mb;
    uint64_t msml = a_big ? mb : ma;
    unsigned eb = (unsigned)(mbig >> 52);
    unsigned es = (unsigned)(msml >> 52);
    // significands with the leading one at bit 62 and 10 guard bits below
    uint64_t Mb = ((mbig & FRAC) | HID) << 10;
    uint64_t Ms = ((msml & FRAC) | HID) << 10;
    unsigned d = eb - es;
    uint64_t Msh, lost;
    if (d < 64u) {
        Msh = Ms >> d;
        lost = d ? (Ms << (64u - d)) : 0ull;
    } else {
        Msh = 0ull;
        lost = Ms;
    }
    Msh |= (lost != 0ull) ? 1ull : 0ull;  // sticky bit
    bool sub = ((A ^ B) & SIGN) != 0ull;
    uint64_t S = sub ? (Mb - Msh) : (Mb + Msh);
    int lz = clz64(S);
    int e = (int)eb + 1 - lz;
    uint64_t Nn = (lz == 0) ? ((S >> 1) | (S & 1ull)) : (S << ((lz - 1) & 63));
    uint64_t mant = Nn >> 10;
    unsigned rb = (unsigned)(Nn & 0x3FFull);
    uint64_t inc = (rb > 0x200u || (rb == 0x200u && (mant & 1ull))) ? 1ull : 0ull;
    uint64_t res = ((((uint64_t)(int64_t)(e - 1)) << 52) + mant + inc) | (big & SIGN);
    ok = (eb - 1u < 2046u) && (es >= 1u) && (S != 0ull) && (e >= 1) && (e <= 2046);
    return bitsd(res);
}

// a + b, exactly rounded: the integer-pipe add where it applies, else the hardware add
// (behind a warp vote and an opaque instruction on the device, as in quarter(); all 32
// lanes must call it together).
__host__ __device__ __forceinline__ double add_int(double a, double b) {
    bool ok;
    double r = add_int_core(a, b, ok);
#if defined(__CUDA_ARCH__)
    if (__any_sync(0xffffffffu, !ok)) {
        if (!ok) asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
    }
    return r;
#else
    return ok ? r : hw_add(a, b);
#endif
}

}  // namespace rbgs
