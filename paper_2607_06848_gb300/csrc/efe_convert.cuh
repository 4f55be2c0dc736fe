// The binary64 -> binary32 conversion done with integer operations.  On this
// GPU the FP64 pipe is narrow, and a conversion through it costs more than
// the FP64 arithmetic around it; the filter's start pass narrows every
// element of an FP64 block, so it builds the result bit by bit from the IEEE
// 754 encodings instead.
//
// f64_to_f32_rn: round to nearest, ties to even, with gradual underflow into
// the binary32 subnormals, overflow to +-inf, NaN kept a (quiet) NaN -- the
// IEEE 754 conversion.
#pragma once
#include <cstdint>

__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long mant = b & 0xfffffffffffffull;
    if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (mant ? 0x400000u : 0u));
    const int ef = e - 1023 + 127;                       // binary32 biased exponent
    if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
    if (ef <= 0) {
        // binary32 subnormal (or zero): significand units of 2^-149
        if (e == 0) return __uint_as_float(sign);        // binary64 subnormals are far below 2^-149
        const int sh = 30 - ef;                           // >= 30
        if (sh >= 64) return __uint_as_float(sign);
        const unsigned long long M = mant | (1ull << 52);
        uint32_t m = (uint32_t)(M >> sh);
        const unsigned long long rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1u))) ++m;   // may carry into the smallest normal
        return __uint_as_float(sign | m);
    }
    const uint32_t m = (uint32_t)(mant >> 29);
    const uint32_t rem = (uint32_t)(mant & 0x1fffffffu);
    uint32_t r = ((uint32_t)ef << 23) + m;
    if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ++r;   // a carry raises the exponent
    return __uint_as_float(sign | r);
}
