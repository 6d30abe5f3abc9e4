// Double-FP32 ("df") primitives: a value is an unevaluated sum hi + lo of two binary32 numbers.
// The steps are the error-free transformations of Knuth (two-sum), Dekker (fast two-sum, valid
// when |a| >= |b|) and the FMA-based exact product; each operation is written with explicit
// round-to-nearest intrinsics so that the compiler cannot contract or reassociate it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fx {

__device__ __forceinline__ void split_df(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Compensated dot-product step with an exact FP32 input x (no input low word): S + E += (ch + cl) x
// (Ogita, Rump & Oishi 2005, algorithm Dot2).
__device__ __forceinline__ void dot2_step_x(float ch, float cl, float x, float &S, float &E)
{
    const float p = __fmul_rn(ch, x);
    const float e = __fmaf_rn(ch, x, -p);
    const float s = __fadd_rn(S, p);
    const float bv = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    S = s;
    E = __fmaf_rn(cl, x, __fadd_rn(E, __fadd_rn(err, e)));
}

// (h, l) <- (s + t) renormalised so that |l| <= ulp(h) / 2 (Dekker's fast two-sum, |s| >= |t|).
__device__ __forceinline__ void df_renorm(float s, float t, float &h, float &l)
{
    h = __fadd_rn(s, t);
    l = __fsub_rn(t, __fsub_rn(h, s));
}

// (h, l) <- (h, l) + (bh, bl), renormalised.
__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl)
{
    const float s = __fadd_rn(h, bh);
    const float bv = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(bh, bv));   // h + bh = s + err
    df_renorm(s, __fadd_rn(__fadd_rn(l, bl), err), h, l);
}

// One Horner step (h, l) <- (h, l) j + (eh, el) for an exact FP32 multiplier j.
__device__ __forceinline__ void df_horner(float &h, float &l, float j, float eh, float el)
{
    const float p = __fmul_rn(h, j);
    const float pl = __fmaf_rn(l, j, __fmaf_rn(h, j, -p));   // h j = p + (h j - p) exactly
    h = p;
    l = pl;
    df_add(h, l, eh, el);
}

// binary32 -> binary64 from the IEEE 754 encodings: sign kept, exponent rebiased by
// 1023 - 127 = 896, significand shifted into the top of the 52-bit field. Exact for normal
// numbers and zeros; subnormals, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double f32_to_f64_bits(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) {
        if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((uint64_t)(b >> 31) << 63));
        return (double)f;
    }
    const uint64_t d = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// binary64 -> binary32 rounded to nearest even, from the encodings: for results in binary32's
// normal range the exponent is rebiased by -896 and the 52-bit significand cut to 23 bits, adding
// one unit when the 29 dropped bits exceed half a unit or equal it with an odd kept part (a carry
// into the exponent is the correct rounded value, up to infinity). Other inputs (zeros,
// binary32 subnormal results, overflow, infinities, NaNs) take the hardware conversion. Used where
// FP64 conversions would occupy the FP64 pipe, which on this GPU is the bottleneck.
__device__ __forceinline__ float f64_to_f32_bits(double v)
{
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
    if (e < 897u || e > 1150u) return (float)v;
    const uint64_t m = b & 0xfffffffffffffull;
    uint32_t r = ((e - 896u) << 23) | (uint32_t)(m >> 29);
    const uint64_t rem = m & 0x1fffffffull, half = 0x10000000ull;
    if (rem > half || (rem == half && (r & 1u))) r += 1u;
    return __uint_as_float((uint32_t)(b >> 63) << 31 | r);
}

// Conversion between FP32 and FP64 with the hardware's result (exact widening, round-to-nearest-
// even narrowing) but, for FP32 <-> FP64, from the encodings on the integer pipe.
template <typename To, typename From>
__device__ __forceinline__ To convert_bits(From v)
{
    if constexpr (sizeof(To) == 8 && sizeof(From) == 4) return f32_to_f64_bits(v);
    else if constexpr (sizeof(To) == 4 && sizeof(From) == 8) return f64_to_f32_bits(v);
    else return (To)v;
}

}  // namespace fx
