// binary64 -> binary32 conversion and splitting done with integer operations,
// and a double-single product difference.  On this GPU the FP64 pipe is
// narrow, and a conversion through it costs more than the FP64 arithmetic
// around it; the filter's start pass reads every element of two FP64 blocks,
// so it splits them bit by bit from the IEEE 754 encodings and does its
// arithmetic on the FP32 pipe.
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

// x = hi + lo with hi = f64_to_f32_rn(x) and lo the rest to 22 bits
// (|x - hi - lo| < 2^-45 |x| where hi and lo are binary32 normals, i.e.
// 2^-100 <= |x| < 2^128), by integer operations only: the rest is the low 29
// bits of the significand (less 2^29 when hi rounded up); its top 22 bits
// become a binary32 by the 1.5 * 2^23 bias (no integer-to-float instruction,
// which takes the narrow FP64 pipe on this part), then take the exponent.
// For |x| below 2^-126 (hi subnormal or zero) lo is 0.
__device__ __noinline__ float f64_to_f32_rn_call(double x) { return f64_to_f32_rn(x); }
__device__ __forceinline__ void f64_split(double x, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 897 || e > 1150) {                        // hi not a binary32 normal (rare: out of line)
        hi = f64_to_f32_rn_call(x);
        lo = 0.f;
        return;
    }
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const uint32_t m = (uint32_t)(b >> 29) & 0x7fffffu;          // hi's fraction, truncated
    const int rem = (int)((uint32_t)b & 0x1fffffffu);
    const bool up = rem > 0x10000000 || (rem == 0x10000000 && (m & 1u));
    // the carry of a round-up runs into the exponent field: the IEEE 754 rounding
    hi = __uint_as_float(sign | ((((uint32_t)(e - 896)) << 23) + m + (up ? 1u : 0u)));
    const int d = (up ? rem - 0x20000000 : rem) >> 7;             // |d| <= 2^21
    const float fd = __int_as_float(0x4B400000 + d) - 12582912.0f;  // exact: |d| < 2^22
    // lo = +-fd 2^(e - 1068), in two exact power-of-two steps below 2^-126
    const float sl = sign ? -fd : fd;
    if (e >= 942) lo = sl * __uint_as_float((uint32_t)(e - 941) << 23);
    else lo = (sl * __uint_as_float((uint32_t)(e - 841) << 23)) * 0x1p-100f;
}

// a b - c d for binary64 inputs given as (hi, lo) pairs, in binary32
// arithmetic (double-single): the exact products of the high parts (FMA),
// their rounded cross terms, and an error-free difference of the high
// products; the result is within one unit in the last place of the exact
// a b - c d plus about 2^-44 (|a b| + |c d|) with operands split to 2^-45, so
// a difference that cancels to a residual-sized value keeps ~2^-44 / residual
// of relative accuracy.
__device__ __forceinline__ float ds_mul_sub(float ah, float al, float bh, float bl, float ch, float cl, float dh,
                                            float dl) {
    const float p1 = ah * bh, e1 = fmaf(ah, bh, -p1);
    const float p2 = ch * dh, e2 = fmaf(ch, dh, -p2);
    const float t1 = fmaf(ah, bl, fmaf(al, bh, e1));
    const float t2 = fmaf(ch, dl, fmaf(cl, dh, e2));
    const float s = p1 - p2;
    const float bb = s - p1;
    const float err = (p1 - (s - bb)) + (-p2 - bb);
    return s + (err + (t1 - t2));
}
