// Double-FP32 ("df") primitives: a value is an unevaluated sum hi + lo of two binary32 numbers.
// The steps are the error-free transformations of Knuth (two-sum), Dekker (fast two-sum, valid
// when |a| >= |b|) and the FMA-based exact product; each operation is written with explicit
// round-to-nearest intrinsics so that the compiler cannot contract or reassociate it.
#pragma once
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

}  // namespace fx
