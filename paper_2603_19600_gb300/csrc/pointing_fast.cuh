// Certified FP32 evaluation of the pointing (PointingOperator, "Map-making classes"; HEALPix RING
// pixels, "Landscape types"), shared by the cache fill (pointing_fast.cu) and the on-the-fly FP32
// operator (fused_f32.cu). The design, the error budget and the margins are described at the top
// of pointing_fast.cu: a sample whose FP32 decisions the margins cannot certify returns false and
// is recomputed by the caller with the exact FP64 recipe, so pixels equal the recipe's.
#pragma once
#include "pointing_math.cuh"

namespace fx {

constexpr float kU = 5.9604645e-8f;   // 2^-24

// Row . vector in double-FP32 (exact products of the hi parts, two-sums), rounded to FP32.
__device__ __forceinline__ float dot3_df(const float *mh, const float *ml, const float (&vh)[3], const float (&vl)[3])
{
    float s = 0.f, err = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float p = __fmul_rn(mh[j], vh[j]);
        const float e = __fmaf_rn(mh[j], vh[j], -p);
        const float t = __fadd_rn(s, p);
        const float bv = __fsub_rn(t, s);
        const float te = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
        s = t;
        err = __fmaf_rn(mh[j], vl[j], __fmaf_rn(ml[j], vh[j], __fadd_rn(err, __fadd_rn(te, e))));
    }
    return __fadd_rn(s, err);
}

__device__ __forceinline__ float frac_dist(float v)
{
    const float f = v - floorf(v);
    return fminf(f, 1.f - f);
}

// FP32 RING lookup with certified floors; false if any decision is within its error bound.
// Integer work is 32-bit (every index stays below 12 * 8192^2 < 2^31): conversions between FP32
// and 64-bit integers would run on the FP64 pipe.
__device__ __forceinline__ bool fast_ring_pixel(float dx, float dy, float dz, int32_t nside, int32_t &pix)
{
    const float rho2 = fmaf(dx, dx, dy * dy);
    if (!(rho2 >= 0.0025f)) return false;              // within ~3 deg of a pole (or NaN)
    const float rho = sqrtf(rho2);
    const float za = fabsf(dz);
    if (fabsf(za - 0.6666667f) <= 64.f * kU) return false;   // zone decision
    const float N = (float)nside;
    float phi = atan2f(dy, dx);
    if (phi < 0.f) phi += 6.2831855f;
    const float tt = phi * 0.63661977f;
    if (za <= 0.6666667f) {
        const float t1 = N * (0.5f + tt), t2 = N * (dz * 0.75f);
        const float a1 = t1 - t2, a2 = t1 + t2;
        const float m = 96.f * N * kU + 16.f * kU;
        if (frac_dist(a1) <= m || frac_dist(a2) <= m) return false;
        const int32_t jp = (int32_t)floorf(a1), jm = (int32_t)floorf(a2);
        const int32_t ir = nside + 1 + jp - jm;
        const int32_t kshift = 1 - (ir & 1);
        int32_t ip = (jp + jm - nside + kshift) / 2;
        const int32_t nl4 = 4 * nside;
        ip %= nl4;
        if (ip < 0) ip += nl4;
        const int32_t p = 2 * nside * (nside - 1) + (ir - 1) * nl4 + ip;
        if (p < 0 || p >= 12 * nside * nside) return false;
        pix = p;
        return true;
    }
    const float ft = tt - floorf(tt);
    if (fminf(ft, 1.f - ft) <= 16.f * kU / rho + 64.f * kU) return false;   // facet edge
    const float tmp = N * sqrtf(3.f * (rho2 / (1.f + za)));
    const float b1 = ft * tmp, b2 = (1.f - ft) * tmp;
    const float mc = 112.f * N * kU + 16.f * kU;
    if (frac_dist(b1) <= mc || frac_dist(b2) <= mc) return false;
    const int32_t jp = (int32_t)floorf(b1), jm = (int32_t)floorf(b2);
    const int32_t ir = jp + jm + 1;
    const float b3 = tt * (float)ir;
    if (frac_dist(b3) <= 96.f * N * kU + 16.f * kU / rho + 64.f * kU) return false;
    int32_t ip = (int32_t)floorf(b3);
    const int32_t nl = 4 * ir;
    ip %= nl;
    if (ip < 0) ip += nl;
    const int32_t p = dz > 0.f ? 2 * ir * (ir - 1) + ip : 12 * nside * nside - 2 * ir * (ir + 1) + ip;
    if (p < 0 || p >= 12 * nside * nside) return false;
    pix = p;
    return true;
}

// Third and first columns of R(q_det) (line of sight and orientation of the detector) in
// double-FP32: out = d hi[3], d lo[3], o hi[3], o lo[3]. False if |q_det|^2 is not within 4u of 1
// (every sample of that detector then takes the exact recipe). FP64: call once per detector.
__device__ __forceinline__ bool det_axes_df(const Quat &qd, float *out)
{
    const double n2 = qd.w * qd.w + qd.x * qd.x + qd.y * qd.y + qd.z * qd.z;
    const double xx = qd.x * qd.x, yy = qd.y * qd.y, zz = qd.z * qd.z;
    const double xy = qd.x * qd.y, xz = qd.x * qd.z, yz = qd.y * qd.z;
    const double wx = qd.w * qd.x, wy = qd.w * qd.y, wz = qd.w * qd.z;
    const double dv[3] = {2.0 * (xz + wy), 2.0 * (yz - wx), 1.0 - 2.0 * (xx + yy)};
    const double ov[3] = {1.0 - 2.0 * (yy + zz), 2.0 * (xy + wz), 2.0 * (xz - wy)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float h = (float)dv[k], g = (float)ov[k];
        out[k] = h;
        out[3 + k] = (float)(dv[k] - (double)h);
        out[6 + k] = g;
        out[9 + k] = (float)(ov[k] - (double)g);
    }
    return fabs(n2 - 1.0) <= 4.0 * 5.9604644775390625e-8;
}

// Pixel and FP32 weights (cos 2psi, sin 2psi) of one sample from its boresight matrix m (18
// floats: hi[9], lo[9]; hi[0] NaN marks a boresight quaternion for the exact path) and the
// detector axes; false if the exact recipe must decide. No half-wave plate or offset rotation.
__device__ __forceinline__ bool certified_sample(const float *m, const float (&dh)[3], const float (&dl)[3],
                                                 const float (&oh)[3], const float (&ol)[3], int32_t nside,
                                                 int32_t &pix, float &c, float &s)
{
    float mh[9], ml[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) { mh[j] = m[j]; ml[j] = m[9 + j]; }
    if (isnan(mh[0])) return false;
    const float dx = dot3_df(mh + 0, ml + 0, dh, dl), dy = dot3_df(mh + 3, ml + 3, dh, dl),
                dz = dot3_df(mh + 6, ml + 6, dh, dl);
    const float ox = dot3_df(mh + 0, ml + 0, oh, ol), oy = dot3_df(mh + 3, ml + 3, oh, ol),
                oz = dot3_df(mh + 6, ml + 6, oh, ol);
    if (!fast_ring_pixel(dx, dy, dz, nside, pix)) return false;
    // psi from local north through east (same convention as the exact recipe)
    const float rho2 = fmaf(dx, dx, dy * dy);
    const float a = fmaf(-dz, fmaf(ox, dx, oy * dy), rho2 * oz);
    const float b = fmaf(oy, dx, -ox * dy);
    const float n2 = fmaf(a, a, b * b);
    const float inv = 1.f / n2;
    c = (a * a - b * b) * inv;
    s = 2.f * a * b * inv;
    return true;
}

// Boresight rotation matrices for certified_sample ([n][18], pointing_fast.cu).
__global__ void bore_matrix_kernel(const double *__restrict__ q_bore, int64_t n, float *__restrict__ m);

}  // namespace fx
