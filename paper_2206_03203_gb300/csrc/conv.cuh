// Conversions between binary64 and binary32 by integer operations.
//
// On this GPU a conversion between FP64 and FP32 issues on the FP64 unit,
// whose rate is that of the FP64 arithmetic; a streaming kernel that
// converts every element it moves (the FP32 copy of each new Krylov basis
// vector, the FP64 result of the mixed V-cycle) then spends as much of that
// unit on conversions as on its arithmetic.  These functions compute the same
// results from the IEEE 754 encodings with integer operations only:
//  - narrowing rounds to nearest, ties to even, including results in the
//    binary32 subnormal range, overflow to infinity, and signed zeros; a NaN
//    stays a NaN (quiet, sign and the leading payload bits kept);
//  - widening is exact, binary32 subnormals included.
// The same source builds for the host (the CPU tests compare it with the
// host's own conversions on random and boundary encodings).
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define MDS_HD __host__ __device__ __forceinline__
#else
#define MDS_HD inline
#endif

namespace mds {

// binary64 encoding -> binary32 encoding, round to nearest even
MDS_HD uint32_t f64_to_f32_bits(uint64_t u) {
    const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
    const int e = (int)((u >> 52) & 0x7FF);
    const uint64_t m = u & 0xFFFFFFFFFFFFFull;  // 52 fraction bits
    if (e == 0x7FF) return m ? (sign | 0x7FC00000u | (uint32_t)(m >> 29)) : (sign | 0x7F800000u);
    const int E = e - 1023 + 127;  // biased binary32 exponent of a normal result
    if (E >= 0xFF) return sign | 0x7F800000u;
    if (E <= 0) {
        // below the binary32 normal range: the result is k 2^-149 with k an
        // integer below 2^23 (or exactly 2^23, the least normal, after rounding)
        if (e == 0) return sign;  // a binary64 subnormal or zero is far below 2^-150
        const int shift = 926 - e;  // value = M 2^(e - 1075) = (M >> shift) 2^-149
        if (shift >= 54) return sign;  // below half of 2^-149
        const uint64_t M = m | (1ull << 52);
        uint64_t k = M >> shift;
        const uint64_t rem = M & ((1ull << shift) - 1), half = 1ull << (shift - 1);
        if (rem > half || (rem == half && (k & 1))) k++;
        return sign | (uint32_t)k;
    }
    uint32_t bits = ((uint32_t)E << 23) | (uint32_t)(m >> 29);
    const uint64_t rem = m & 0x1FFFFFFFull, half = 1ull << 28;
    if (rem > half || (rem == half && (bits & 1))) bits++;  // a carry raises the exponent (to infinity at the top)
    return sign | bits;
}

// binary32 encoding -> binary64 encoding (exact)
MDS_HD uint64_t f32_to_f64_bits(uint32_t u) {
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xFF, m = u & 0x7FFFFFu;
    if (e == 0xFF) return sign | 0x7FF0000000000000ull | ((uint64_t)m << 29);
    if (e == 0) {
        if (m == 0) return sign;
        // subnormal m 2^-149: normalise on its leading bit p
        int p = 22;
        while (!((m >> p) & 1u)) p--;
        const uint64_t frac = ((uint64_t)m << (52 - p)) & 0xFFFFFFFFFFFFFull;
        return sign | ((uint64_t)(p + 874) << 52) | frac;
    }
    return sign | ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)m << 29);
}

#if defined(__CUDACC__)
__device__ __forceinline__ float d2f_int(double x) {
    return __uint_as_float(f64_to_f32_bits((uint64_t)__double_as_longlong(x)));
}
__device__ __forceinline__ double f2d_int(float x) {
    return __longlong_as_double((long long)f32_to_f64_bits(__float_as_uint(x)));
}
#endif

}  // namespace mds
