// Per-sample pointing in FP64: detector quaternion, line of sight, HEALPix RING pixel and
// polarisation weights (PointingOperator, "Map-making classes" of the Furax paper; HEALPix
// landscape, "Landscape types").
//
// Every floating-point step is an explicit round-to-nearest intrinsic (__dmul_rn, __dadd_rn,
// __dsub_rn, __ddiv_rn, __dsqrt_rn, __fma_rn), so the compiler cannot contract or reorder
// them: the result is a function of the inputs alone, and any implementation that follows
// the same written recipe in IEEE FP64 gets the same pixel.
#pragma once
#include "dfloat.cuh"
#include <cstdint>

namespace fx {

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// atan(k/8), k = 0..8, each the nearest double.
__device__ __forceinline__ double atan_k8(int k)
{
    switch (k) {
    case 0: return 0.0;
    case 1: return 0x1.fd5ba9aac2f6ep-4;
    case 2: return 0x1.f5b75f92c80ddp-3;
    case 3: return 0x1.6f61941e4def1p-2;
    case 4: return 0x1.dac670561bb4fp-2;
    case 5: return 0x1.1e00babdefeb4p-1;
    case 6: return 0x1.4978fa3269ee1p-1;
    case 7: return 0x1.700a7c5784634p-1;
    default: return 0x1.921fb54442d18p-1;
    }
}
constexpr double kPi2 = 0x1.921fb54442d18p+0;   // pi/2
constexpr double kPi = 0x1.921fb54442d18p+1;    // pi
constexpr double k2Pi = 0x1.921fb54442d18p+2;   // 2 pi
constexpr double k2OverPi = 0x1.45f306dc9c883p-1;

// atan(t) for t in [0, 1]: nearest k/8 (k = floor(8t + 1/2)), reduced argument
// r = (t - k/8)/(1 + t k/8) with |r| <= 1/16, then the Taylor series of atan to r^15
// evaluated by Horner's rule in s = r^2 with fused multiply-adds.
__device__ __forceinline__ double atan_unit(double t)
{
    int k = (int)dadd(dmul(t, 8.0), 0.5);
    double c = dmul((double)k, 0.125);
    double r = ddiv(dsub(t, c), dadd(1.0, dmul(t, c)));
    double s = dmul(r, r);
    double p = -1.0 / 15.0;
    p = __fma_rn(p, s, 1.0 / 13.0);
    p = __fma_rn(p, s, -1.0 / 11.0);
    p = __fma_rn(p, s, 1.0 / 9.0);
    p = __fma_rn(p, s, -1.0 / 7.0);
    p = __fma_rn(p, s, 1.0 / 5.0);
    p = __fma_rn(p, s, -1.0 / 3.0);
    p = dmul(p, s);
    return dadd(atan_k8(k), __fma_rn(r, p, r));
}

// Azimuth of (x, y) in [0, 2 pi): octant reduction to atan on [0, 1], then the
// quadrant from the signs. (0, 0) -> 0.
__device__ __forceinline__ double azimuth(double x, double y)
{
    double ax = fabs(x), ay = fabs(y), a;
    if (ax == 0.0 && ay == 0.0) return 0.0;
    if (ax >= ay) a = atan_unit(ddiv(ay, ax));
    else a = dsub(kPi2, atan_unit(ddiv(ax, ay)));
    if (x < 0.0) a = dsub(kPi, a);
    if (y < 0.0) a = dsub(k2Pi, a);
    if (a >= k2Pi) a = 0.0;
    return a;
}

// HEALPix RING index from z = cos(theta), |z|, tt = 2 phi / pi in [0, 4] and 1 - |z|.
// Equatorial belt (|z| <= 2/3): the pixel lies between edge lines of the two families
// N (1/2 + tt - 3z/4) and N (1/2 + tt + 3z/4) = integer; their integer parts give the
// ring (counted from z = 2/3) and the position within the ring's 4N pixels.
// Polar caps: with tp = frac(tt) and s = N sqrt(3 (1 - |z|)), the integer parts of
// tp s and (1 - tp) s give the ring counted from the pole (ring i has 4i pixels) and
// floor(tt i) the position within it.
__device__ __forceinline__ int64_t ring_pixel(int64_t nside, double z, double za, double tt, double one_minus_za)
{
    const double n = (double)nside;
    if (za <= 2.0 / 3.0) {
        double temp1 = dmul(n, dadd(0.5, tt));
        double temp2 = dmul(n, dmul(z, 0.75));
        int64_t jp = (int64_t)floor(dsub(temp1, temp2));
        int64_t jm = (int64_t)floor(dadd(temp1, temp2));
        int64_t ir = nside + 1 + jp - jm;            // 1 .. 2N+1
        int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - nside + kshift) / 2;
        int64_t nl4 = 4 * nside;
        ip %= nl4;
        if (ip < 0) ip += nl4;
        return 2 * nside * (nside - 1) + (ir - 1) * nl4 + ip;
    }
    double tp = dsub(tt, floor(tt));
    double tmp = dmul(n, __dsqrt_rn(dmul(3.0, one_minus_za)));
    int64_t jp = (int64_t)floor(dmul(tp, tmp));
    int64_t jm = (int64_t)floor(dmul(dsub(1.0, tp), tmp));
    int64_t ir = jp + jm + 1;
    int64_t ip = (int64_t)floor(dmul(tt, (double)ir));
    int64_t nl = 4 * ir;
    ip %= nl;
    if (ip < 0) ip += nl;
    if (z > 0.0) return 2 * ir * (ir - 1) + ip;
    return 12 * nside * nside - 2 * ir * (ir + 1) + ip;
}

struct Quat {
    double w, x, y, z;
};

struct SampleF64 {
    int32_t pix;   // -1 if the quaternion product is not finite
    double c, s;   // cos 2psi, sin 2psi (before any detector offset)
};

// q = qb (x) qd (Hamilton, scalar first, summed left to right); line of sight d = R(q) z^,
// orientation o = R(q) x^; pixel of d; psi from local north (-e_theta) through east (e_phi):
// a = rho (o . north) = -d_z (o_x d_x + o_y d_y) + rho^2 o_z, b = rho (o . east) = -o_x d_y + o_y d_x,
// cos 2psi = (a^2 - b^2)/(a^2 + b^2), sin 2psi = 2ab/(a^2 + b^2), (1, 0) at a pole.
__device__ __forceinline__ SampleF64 point_f64(Quat qb, Quat qd, int64_t nside)
{
    const double a0 = qb.w, a1 = qb.x, a2 = qb.y, a3 = qb.z;
    const double b0 = qd.w, b1 = qd.x, b2 = qd.y, b3 = qd.z;
    double w = dsub(dsub(dsub(dmul(a0, b0), dmul(a1, b1)), dmul(a2, b2)), dmul(a3, b3));
    double x = dsub(dadd(dadd(dmul(a0, b1), dmul(a1, b0)), dmul(a2, b3)), dmul(a3, b2));
    double y = dadd(dadd(dsub(dmul(a0, b2), dmul(a1, b3)), dmul(a2, b0)), dmul(a3, b1));
    double z = dadd(dsub(dadd(dmul(a0, b3), dmul(a1, b2)), dmul(a2, b1)), dmul(a3, b0));
    SampleF64 out;
    if (!(isfinite(w) && isfinite(x) && isfinite(y) && isfinite(z))) {
        out.pix = -1; out.c = 0.0; out.s = 0.0;
        return out;
    }
    double xx = dmul(x, x), yy = dmul(y, y), zz = dmul(z, z);
    double xy = dmul(x, y), xz = dmul(x, z), yz = dmul(y, z);
    double wx = dmul(w, x), wy = dmul(w, y), wz = dmul(w, z);
    double d0 = dmul(2.0, dadd(xz, wy));
    double d1 = dmul(2.0, dsub(yz, wx));
    double d2 = dsub(1.0, dmul(2.0, dadd(xx, yy)));
    double o0 = dsub(1.0, dmul(2.0, dadd(yy, zz)));
    double o1 = dmul(2.0, dadd(xy, wz));
    double o2 = dmul(2.0, dsub(xz, wy));

    double za = fabs(d2);
    double rho2 = dadd(dmul(d0, d0), dmul(d1, d1));
    double tt = dmul(azimuth(d0, d1), k2OverPi);
    const int64_t pix = ring_pixel(nside, d2, za, tt, ddiv(rho2, dadd(1.0, za)));
    // a quaternion far from unit norm can send the ring index past the last ring: no pixel
    if (pix < 0 || pix >= 12 * nside * nside) {
        out.pix = -1; out.c = 0.0; out.s = 0.0;
        return out;
    }
    out.pix = (int32_t)pix;

    double a = dadd(dmul(-d2, dadd(dmul(o0, d0), dmul(o1, d1))), dmul(rho2, o2));
    double b = dadd(dmul(-o0, d1), dmul(o1, d0));
    double aa = dmul(a, a), bb = dmul(b, b), n2 = dadd(aa, bb);
    if (n2 > 0.0) {
        out.c = ddiv(dsub(aa, bb), n2);
        out.s = ddiv(dmul(dmul(2.0, a), b), n2);
    } else {
        out.c = 1.0; out.s = 0.0;
    }
    return out;
}

__device__ __forceinline__ Quat load_quat(const double *q, int64_t i)
{
    const double2 *p = reinterpret_cast<const double2 *>(q + 4 * i);
    double2 lo = __ldg(p), hi = __ldg(p + 1);
    return Quat{lo.x, lo.y, hi.x, hi.y};
}

// FP32 rotation with explicit roundings, so that every kernel performs the same operations
// whatever the compiler's contraction choices: c' = fma(c, c2, -(s s2)), s' = fma(s, c2, c s2).
__device__ __forceinline__ void rotate_psi_f(float &c, float &s, float c2, float s2)
{
    const float c1 = __fmaf_rn(c, c2, -__fmul_rn(s, s2));
    const float s1 = __fmaf_rn(s, c2, __fmul_rn(c, s2));
    c = c1; s = s1;
}

// Rotate (c, s) = (cos 2psi, sin 2psi) by the detector offset: (cos 2(psi+delta), sin 2(psi+delta)).
template <typename T>
__device__ __forceinline__ void rotate_psi(T &c, T &s, double2 cs)
{
    if constexpr (sizeof(T) == 4) {
        rotate_psi_f(c, s, (float)cs.x, (float)cs.y);
    } else {
        T c2 = (T)cs.x, s2 = (T)cs.y;
        T c1 = c * c2 - s * s2;
        T s1 = s * c2 + c * s2;
        c = c1; s = s1;
    }
}

// Ideal half-wave plate at angle w in front of the detector (HWPOperator, Table 3 of the Furax
// paper): the detector's angle enters the weights as 4w - 2psi, i.e. (cos 2psi, sin 2psi) is
// reflected into (cos 4w c + sin 4w s, sin 4w c - cos 4w s). An offset rotation by 2 delta applied
// before the plate equals a rotation by -2 delta after it ("Algebraic reductions":
// R(theta) o HWP = HWP o R(-theta)), which is how per-detector offsets are applied to weights
// that already carry the plate (see launch_set_psi).
template <typename T>
__device__ __forceinline__ void apply_hwp(T &c, T &s, double2 h)
{
    const T c4 = (T)h.x, s4 = (T)h.y;
    if constexpr (sizeof(T) == 4) {   // explicit roundings, as in rotate_psi_f
        const float c1 = __fmaf_rn(c4, c, __fmul_rn(s4, s));
        const float s1 = __fmaf_rn(s4, c, -__fmul_rn(c4, s));
        c = c1; s = s1;
    } else {
        const T c1 = c4 * c + s4 * s;
        const T s1 = s4 * c - c4 * s;
        c = c1; s = s1;
    }
}

// Per-sample pointing from a PointingView, for each storage mode.
// MODE 0: on the fly (FP64); 1: FP32 cache; 2: FP64 cache; 3: FP32 hi + lo cache (FP32 readers see
// hi, FP64 readers hi + lo). Returns the pixel local to the
// observation (-1 if invalid) and the weights in precision T, offset included.
template <int MODE, typename T>
__device__ __forceinline__ int32_t get_sample(const PointingView &pv, const ObsInfo &ob, int32_t det, int64_t t,
                                              T &c, T &s)
{
    int32_t pix;
    const int64_t gdet = ob.det_off + det;
    if constexpr (MODE == 0) {
        SampleF64 r = point_f64(load_quat(pv.q_bore, ob.bore_off + t), load_quat(pv.q_det, gdet), ob.nside);
        pix = r.pix;
        double cc = r.c, ss = r.s;
        if (pix >= 0) {
            if (pv.hwp_cs) apply_hwp<double>(cc, ss, pv.hwp_cs[ob.bore_off + t]);
            if (pv.psi_cs) rotate_psi<double>(cc, ss, pv.psi_cs[gdet]);
        }
        c = (T)cc; s = (T)ss;
        return pix;
    } else {
        const int64_t i = ob.tod_off + det * ob.nsamp + t;
        pix = pv.pix[i];
        // FP32 words widen exactly from their encodings on the integer pipe (the FP64 pipe, which a
        // conversion instruction would occupy, runs ~70x below FP32 on this GPU)
        if constexpr (MODE == 1) {
            if constexpr (sizeof(T) == 4) { c = pv.c32[i]; s = pv.s32[i]; }
            else { c = f32_to_f64_bits(pv.c32[i]); s = f32_to_f64_bits(pv.s32[i]); }
        } else if constexpr (MODE == 3) {
            if constexpr (sizeof(T) == 4) { c = pv.c32[i]; s = pv.s32[i]; }
            else {
                c = f32_to_f64_bits(pv.c32[i]) + f32_to_f64_bits(pv.c32lo[i]);
                s = f32_to_f64_bits(pv.s32[i]) + f32_to_f64_bits(pv.s32lo[i]);
            }
        }
        else { c = (T)pv.c64[i]; s = (T)pv.s64[i]; }
        if (pv.psi_cs && pix >= 0) rotate_psi<T>(c, s, pv.psi_cs[gdet]);
        return pix;
    }
}

}  // namespace fx
