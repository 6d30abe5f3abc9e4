// Evaluation of the Legendre templates and of W applied to them, shared by the template kernels
// and by the double-FP32 right-hand-side kernel that folds the template correction in.
//
// For a polynomial p of degree <= 3 and a symmetric band of half-width halo whose full width fits
// around sample t,
//   sum_k c_|k| p(tau_t + h k) = mu0 p(tau_t) + (mu2 h^2 / 2) p''(tau_t),
// (mu0 = sum_k c_|k|, mu2 = sum_k k^2 c_|k|, h = 2/(ns-1); odd moments of a symmetric band vanish
// and the fourth derivative of p is zero). Within a half-width of either end of the stream the
// truncated sum is taken term by term.
#pragma once
#include "internal.cuh"

namespace fx {

// P_0..P_3 at tau (closed forms).
template <typename T>
__device__ __forceinline__ void legendre4(T tau, T (&L)[4])
{
    L[0] = T(1);
    L[1] = tau;
    L[2] = T(1.5) * tau * tau - T(0.5);
    L[3] = tau * (T(2.5) * tau * tau - T(1.5));
}

template <typename T>
__device__ __forceinline__ T tpl_tap(const NoiseView &nv, int64_t gdet, int k)
{
    if (nv.kind == FURAX_NOISE_WHITE) {
        if (k != 0) return T(0);
        if constexpr (sizeof(T) == 4) return nv.p32[gdet];
        else return nv.p64[gdet];
    }
    if constexpr (sizeof(T) == 4) return nv.p32[gdet * nv.ntaps + k];
    else return nv.p64[gdet * nv.ntaps + k];
}

template <typename T>
__device__ __forceinline__ T tpl_tau(int64_t t, int64_t ns, T h)
{
    return ns > 1 ? T(t) * h - T(1) : T(0);
}

// w[l] = (W P_l)(t) for one detector stream of ns samples.
template <typename T>
__device__ __forceinline__ void wt_eval(const NoiseView &nv, const TplView &tv, int64_t gdet, int64_t ns, int64_t t,
                                        T (&w)[4])
{
    const T h = ns > 1 ? T(2) / T(ns - 1) : T(0);
    if (t >= tv.halo && t + tv.halo < ns) {
        const double2 m = tv.mom[gdet];
        const T mu0 = T(m.x);
        const T k2 = T(m.y) * h * h * T(0.5);
        const T tau = tpl_tau<T>(t, ns, h);
        T L[4];
        legendre4(tau, L);
        w[0] = mu0;
        w[1] = mu0 * tau;
        w[2] = mu0 * L[2] + T(3) * k2;
        w[3] = mu0 * L[3] + T(15) * k2 * tau;
        return;
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) w[l] = T(0);
    for (int k = -tv.halo; k <= tv.halo; ++k) {
        const int64_t s = t + k;
        if (s < 0 || s >= ns) continue;
        const T c = tpl_tap<T>(nv, gdet, k < 0 ? -k : k);
        T L[4];
        legendre4(tpl_tau<T>(s, ns, h), L);
#pragma unroll
        for (int l = 0; l < 4; ++l) w[l] += c * L[l];
    }
}

// Coefficients of sum_l b_l (W P_l)(tau) = c0 + c1 tau + c2 tau^2 + c3 tau^3, valid in the
// interior of a stream (the closed form above with P_0..P_3 written out).
__device__ __forceinline__ void tpl_cubic(double mu0, double k2, const double (&b)[4], double (&c)[4])
{
    c[0] = mu0 * (b[0] - 0.5 * b[2]) + 3.0 * k2 * b[2];
    c[1] = mu0 * (b[1] - 1.5 * b[3]) + 15.0 * k2 * b[3];
    c[2] = 1.5 * mu0 * b[2];
    c[3] = 2.5 * mu0 * b[3];
}

// The same cubic re-expanded in the offset j of a sample from a reference sample of scaled time
// tc (tau = tc + h j): e0 + e1 j + e2 j^2 + e3 j^3.
__device__ __forceinline__ void cubic_shift(const double (&c)[4], double tc, double h, double (&e)[4])
{
    e[0] = ((c[3] * tc + c[2]) * tc + c[1]) * tc + c[0];
    e[1] = h * ((3.0 * c[3] * tc + 2.0 * c[2]) * tc + c[1]);
    e[2] = h * h * (3.0 * c[3] * tc + c[2]);
    e[3] = h * h * h * c[3];
}

// Scaled time of sample t (0 for a one-sample stream), as a reference point for cubic_shift.
__device__ __forceinline__ double tpl_tau_ref(int64_t t, int64_t ns)
{
    return ns > 1 ? (double)t * (2.0 / (double)(ns - 1)) - 1.0 : 0.0;
}

// True when sample t of a stream of ns samples has the band's full width inside the stream.
__device__ __forceinline__ bool tpl_interior(const TplView &tv, int64_t t, int64_t ns)
{
    return t >= tv.halo && t + tv.halo < ns;
}

}  // namespace fx
