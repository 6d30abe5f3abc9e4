/*
 * FP64 CPU oracle for linear-operator CMB map-making (Furax, arXiv 2603.19600).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the CUDA
 * path is checked against. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it. It shares no code with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off (no fused multiply-add except where fma() is
 * written out), so every floating-point step below is one IEEE operation in the
 * order written.
 *
 * What the paper fixes (Statement of Need, Software Design):
 *   d = P m + n                                   (linear data model, H = P)
 *   m^ = (P^T N^-1 P)^-1 P^T N^-1 d               (GLS / maximum likelihood estimator)
 *   P  : PointingOperator, projection computed on the fly (Table 3, "Map-making classes")
 *   P^T: its transpose (Table 1, A.T), a scatter-add of samples into pixels
 *   N^-1: HomothetyOperator (white) or SymmetricBandToeplitzOperator (Table 2)
 *   M  : block-Jacobi preconditioner (BJPreconditioner), inverse via a solver (A.I(...))
 * Below the operator level the paper is silent; the conventions written here are
 * the ones the CUDA path states independently:
 *   - quaternions (w,x,y,z), Hamilton product, q = q_bore (x) q_det;
 *   - direction = third column of R(q), orientation = first column;
 *   - HEALPix RING ang2pix (Gorski et al. 2005), 1-|z| = rho^2/(1+|z|) in the caps;
 *   - phi = a deterministic two-argument arctangent (below), in [0, 2 pi);
 *   - weights (1, cos 2psi, sin 2psi), psi from local north through east;
 *   - N^-1 banded: y_t = sum_{|k|<K} c_|k| x_{t+k} over 0 <= t+k < n (finite section);
 *   - block-Jacobi uses the diagonal of N^-1; a pixel is solved for iff
 *     hits >= 3 and rcond >= rcond_min.
 * Parity is pinned by the tests against closed forms, a second projection-plane
 * pixel lookup, scipy rotations, dense linear algebra and finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Quaternions                                                              */
/* ------------------------------------------------------------------------ */

/* Hamilton product out = a (x) b, scalar first, each component summed left to right. */
void orc_quat_mul(const double *a, const double *b, double *out)
{
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    out[0] = w; out[1] = x; out[2] = y; out[3] = z;
}

/* Line of sight d = R(q) z^ and orientation o = R(q) x^ for a unit quaternion q. */
void orc_quat_axes(const double *q, double *d, double *o)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double xx = x * x, yy = y * y, zz = z * z;
    double xy = x * y, xz = x * z, yz = y * z;
    double wx = w * x, wy = w * y, wz = w * z;
    d[0] = 2.0 * (xz + wy);
    d[1] = 2.0 * (yz - wx);
    d[2] = 1.0 - 2.0 * (xx + yy);
    o[0] = 1.0 - 2.0 * (yy + zz);
    o[1] = 2.0 * (xy + wz);
    o[2] = 2.0 * (xz - wy);
}

/* ------------------------------------------------------------------------ */
/* Azimuth phi = atan2(y, x) in [0, 2 pi), deterministic                    */
/* ------------------------------------------------------------------------ */
/*
 * A two-argument arctangent built only from IEEE-exact basic operations and
 * explicit fma(), so that any implementation following the same recipe gets the
 * same bits. Recipe (table-based argument reduction + Taylor series):
 *   t = min(|x|,|y|) / max(|x|,|y|) in [0, 1];
 *   k = (int)(8 t + 0.5), c = k/8;  r = (t - c) / (1 + t c), |r| <= 1/16;
 *   atan(t) = atan(k/8) + r (1 + s(-1/3 + s(1/5 + ... + s(-1/15)))), s = r^2
 *   (Taylor series of atan to r^15; truncation < 1e-20 relative);
 *   octant and quadrant fix-ups with pi/2, pi, 2 pi rounded to nearest.
 * atan(k/8) for k = 0..8 are the nearest doubles (a mathematical table).
 */
static const double ORC_ATAN_K8[9] = {
    0.0,
    0x1.fd5ba9aac2f6ep-4,
    0x1.f5b75f92c80ddp-3,
    0x1.6f61941e4def1p-2,
    0x1.dac670561bb4fp-2,
    0x1.1e00babdefeb4p-1,
    0x1.4978fa3269ee1p-1,
    0x1.700a7c5784634p-1,
    0x1.921fb54442d18p-1,
};
static const double ORC_PI_2 = 0x1.921fb54442d18p+0;
static const double ORC_PI = 0x1.921fb54442d18p+1;
static const double ORC_2PI = 0x1.921fb54442d18p+2;
static const double ORC_2_OVER_PI = 0x1.45f306dc9c883p-1;

static double orc_atan_unit(double t) /* t in [0, 1] */
{
    int k = (int)(t * 8.0 + 0.5);
    double c = (double)k * 0.125;
    double r = (t - c) / (1.0 + t * c);
    double s = r * r;
    double p = -1.0 / 15.0;
    p = fma(p, s, 1.0 / 13.0);
    p = fma(p, s, -1.0 / 11.0);
    p = fma(p, s, 1.0 / 9.0);
    p = fma(p, s, -1.0 / 7.0);
    p = fma(p, s, 1.0 / 5.0);
    p = fma(p, s, -1.0 / 3.0);
    p = p * s;
    return ORC_ATAN_K8[k] + fma(r, p, r);
}

double orc_phi(double x, double y)
{
    double ax = fabs(x), ay = fabs(y), a;
    if (ax == 0.0 && ay == 0.0) return 0.0;
    if (ax >= ay) a = orc_atan_unit(ay / ax);
    else a = ORC_PI_2 - orc_atan_unit(ax / ay);
    if (x < 0.0) a = ORC_PI - a;
    if (y < 0.0) a = ORC_2PI - a;
    if (a >= ORC_2PI) a = 0.0;
    return a;
}

/* ------------------------------------------------------------------------ */
/* HEALPix RING pixelisation (Gorski et al. 2005, ApJ 622:759)              */
/* ------------------------------------------------------------------------ */
/*
 * Npix = 12 N^2. North cap rings i = 1..N-1 hold 4i pixels at z = 1 - i^2/(3N^2);
 * equatorial rings i = N..3N hold 4N pixels at z = 4/3 - 2i/(3N); the south cap
 * mirrors the north. Pixels are numbered ring by ring from the north pole,
 * eastwards from phi = 0 within a ring.
 *
 * Lookup: with tt = 2 phi/pi in [0,4), the pixel edges are two families of
 * lines. In the belt (|z| <= 2/3) they are N(1/2 + tt -/+ 3z/4) = integer:
 *   jp = floor(N(1/2 + tt - 3z/4)), jm = floor(N(1/2 + tt + 3z/4)),
 *   ring counted from z = 2/3: ir = N + 1 + jp - jm  (1..2N+1),
 *   in-ring index (jp + jm - N + [ir even]) / 2 modulo 4N.
 * In a cap (|z| > 2/3), with tp = tt - floor(tt) and s = N sqrt(3(1-|z|)):
 *   jp = floor(tp s), jm = floor((1 - tp) s), ring from the pole ir = jp + jm + 1,
 *   in-ring index floor(tt ir) modulo 4 ir.
 * one_minus_za is supplied by the caller (computed without cancellation).
 */
static int64_t orc_ring_lookup(int64_t nside, double z, double za, double tt, double one_minus_za)
{
    double n = (double)nside;
    if (za <= 2.0 / 3.0) {
        double temp1 = n * (0.5 + tt);
        double temp2 = n * (z * 0.75);
        int64_t jp = (int64_t)floor(temp1 - temp2);
        int64_t jm = (int64_t)floor(temp1 + temp2);
        int64_t ir = nside + 1 + jp - jm;
        int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - nside + kshift) / 2;
        int64_t nl4 = 4 * nside;
        ip = ((ip % nl4) + nl4) % nl4;
        return 2 * nside * (nside - 1) + (ir - 1) * nl4 + ip;
    } else {
        double tp = tt - floor(tt);
        double tmp = n * sqrt(3.0 * one_minus_za);
        int64_t jp = (int64_t)floor(tp * tmp);
        int64_t jm = (int64_t)floor((1.0 - tp) * tmp);
        int64_t ir = jp + jm + 1;
        int64_t ip = (int64_t)floor(tt * (double)ir);
        int64_t nl = 4 * ir;
        ip = ((ip % nl) + nl) % nl;
        if (z > 0.0) return 2 * ir * (ir - 1) + ip;
        return 12 * nside * nside - 2 * ir * (ir + 1) + ip;
    }
}

/* ang2pix from (z = cos theta, phi in [0, 2 pi)). */
int64_t orc_ang2pix_ring(int64_t nside, double z, double phi)
{
    double za = fabs(z);
    double tt = phi * ORC_2_OVER_PI;
    return orc_ring_lookup(nside, z, za, tt, 1.0 - za);
}

/* ang2pix from a unit direction vector; 1 - |z| = (x^2 + y^2) / (1 + |z|). */
int64_t orc_vec2pix_ring(int64_t nside, const double *d)
{
    double z = d[2], za = fabs(z);
    double rho2 = d[0] * d[0] + d[1] * d[1];
    double tt = orc_phi(d[0], d[1]) * ORC_2_OVER_PI;
    return orc_ring_lookup(nside, z, za, tt, rho2 / (1.0 + za));
}

static int64_t orc_isqrt(int64_t v)
{
    int64_t r = (int64_t)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

/* Pixel centre (z, phi) of RING pixel p. */
void orc_pix2ang_ring(int64_t nside, int64_t p, double *z, double *phi)
{
    int64_t npix = 12 * nside * nside, ncap = 2 * nside * (nside - 1);
    double n = (double)nside;
    if (p < ncap) {
        /* largest i with 2 i (i-1) <= p */
        int64_t i = (1 + orc_isqrt(1 + 2 * p)) / 2;
        while (2 * i * (i - 1) > p) --i;
        while (2 * (i + 1) * i <= p) ++i;
        int64_t k = p - 2 * i * (i - 1);
        *z = 1.0 - (double)(i * i) / (3.0 * n * n);
        *phi = (ORC_PI / (2.0 * (double)i)) * ((double)k + 0.5);
    } else if (p < npix - ncap) {
        int64_t q = p - ncap;
        int64_t i = q / (4 * nside) + nside;
        int64_t k = q % (4 * nside);
        double shift = ((i - nside) % 2 == 0) ? 0.5 : 0.0;
        *z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * n);
        *phi = (ORC_PI / (2.0 * n)) * ((double)k + shift);
    } else {
        int64_t q = npix - 1 - p;
        int64_t i = (1 + orc_isqrt(1 + 2 * q)) / 2;
        while (2 * i * (i - 1) > q) --i;
        while (2 * (i + 1) * i <= q) ++i;
        int64_t k = 4 * i - 1 - (q - 2 * i * (i - 1));
        *z = -(1.0 - (double)(i * i) / (3.0 * n * n));
        *phi = (ORC_PI / (2.0 * (double)i)) * ((double)k + 0.5);
    }
}

/* Batch helpers for the tests. */
void orc_ang2pix_ring_batch(int64_t nside, int64_t n, const double *z, const double *phi, int64_t *pix)
{
    for (int64_t i = 0; i < n; ++i) pix[i] = orc_ang2pix_ring(nside, z[i], phi[i]);
}
void orc_vec2pix_ring_batch(int64_t nside, int64_t n, const double *v, int64_t *pix)
{
    for (int64_t i = 0; i < n; ++i) pix[i] = orc_vec2pix_ring(nside, v + 3 * i);
}
void orc_pix2ang_ring_batch(int64_t nside, int64_t n, const int64_t *pix, double *z, double *phi)
{
    for (int64_t i = 0; i < n; ++i) orc_pix2ang_ring(nside, pix[i], z + i, phi + i);
}
void orc_phi_batch(int64_t n, const double *x, const double *y, double *phi)
{
    for (int64_t i = 0; i < n; ++i) phi[i] = orc_phi(x[i], y[i]);
}
void orc_quat_mul_batch(int64_t n, const double *a, const double *b, double *out)
{
    for (int64_t i = 0; i < n; ++i) orc_quat_mul(a + 4 * i, b + 4 * i, out + 4 * i);
}
void orc_quat_axes_batch(int64_t n, const double *q, double *d, double *o)
{
    for (int64_t i = 0; i < n; ++i) orc_quat_axes(q + 4 * i, d + 3 * i, o + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Pointing: pixel and polarisation weights per sample                      */
/* ------------------------------------------------------------------------ */
/*
 * For sample (det, t): q = q_bore[t] (x) q_det[det]; d, o = axes(q);
 * pixel = vec2pix(d); with a = rho (o . north), b = rho (o . east):
 *   a = -d_z (o_x d_x + o_y d_y) + (d_x^2 + d_y^2) o_z,   b = -o_x d_y + o_y d_x,
 *   cos 2psi = (a^2 - b^2)/(a^2 + b^2), sin 2psi = 2ab/(a^2 + b^2)  (1, 0 at a pole);
 * an angle offset delta rotates (cos 2psi, sin 2psi) by 2 delta.
 * A non-finite quaternion gives pixel -1 and weights 0. Returns the number of such samples.
 */
int64_t orc_pointing(int64_t nside, int64_t nsamp, const double *q_bore, int64_t ndet,
                     const double *q_det, const double *psi_offset, const double *hwp,
                     int32_t *pix, double *cw, double *sw)
{
    int64_t bad = 0;
    for (int64_t j = 0; j < ndet; ++j) {
        double c2d = 1.0, s2d = 0.0;
        if (psi_offset) { c2d = cos(2.0 * psi_offset[j]); s2d = sin(2.0 * psi_offset[j]); }
        for (int64_t t = 0; t < nsamp; ++t) {
            double q[4], d[3], o[3];
            int64_t i = j * nsamp + t;
            orc_quat_mul(q_bore + 4 * t, q_det + 4 * j, q);
            if (!(isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]))) {
                pix[i] = -1; cw[i] = 0.0; sw[i] = 0.0; ++bad; continue;
            }
            orc_quat_axes(q, d, o);
            /* A quaternion far from unit norm can send the ring index past the last ring: no pixel. */
            int64_t pp = orc_vec2pix_ring(nside, d);
            if (pp < 0 || pp >= 12 * nside * nside) { pix[i] = -1; cw[i] = 0.0; sw[i] = 0.0; ++bad; continue; }
            pix[i] = (int32_t)pp;
            double rho2 = d[0] * d[0] + d[1] * d[1];
            double a = -d[2] * (o[0] * d[0] + o[1] * d[1]) + rho2 * o[2];
            double b = -o[0] * d[1] + o[1] * d[0];
            double aa = a * a, bb = b * b, n2 = aa + bb;
            double c = 1.0, s = 0.0;
            if (n2 > 0.0) { c = (aa - bb) / n2; s = (2.0 * a * b) / n2; }
            if (psi_offset) {
                double c1 = c * c2d - s * s2d;
                double s1 = s * c2d + c * s2d;
                c = c1; s = s1;
            }
            if (hwp) {
                /* Ideal half-wave plate at angle w in front of the detector (HWPOperator, Table 3):
                 * the detector's angle 2psi' enters as 4w - 2psi', i.e.
                 * (cos(4w - 2psi'), sin(4w - 2psi')) = (cos4w c + sin4w s, sin4w c - cos4w s). */
                double c4 = cos(4.0 * hwp[t]), s4 = sin(4.0 * hwp[t]);
                double c1 = c4 * c + s4 * s;
                double s1 = s4 * c - c4 * s;
                c = c1; s = s1;
            }
            cw[i] = c; sw[i] = s;
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* P and P^T                                                                */
/* ------------------------------------------------------------------------ */

/* tod[i] = I_p + Q_p c_i + U_p s_i (0 where the pixel is -1). map is [npix][3]. */
void orc_P(int64_t nsamp_total, const int32_t *pix, const double *cw, const double *sw,
           const double *map, double *tod)
{
    for (int64_t i = 0; i < nsamp_total; ++i) {
        int32_t p = pix[i];
        if (p < 0) { tod[i] = 0.0; continue; }
        const double *m = map + 3 * (int64_t)p;
        tod[i] = m[0] + m[1] * cw[i] + m[2] * sw[i];
    }
}

/* Neumaier-compensated accumulation of v into (sum, comp). */
static inline void orc_neumaier(double *sum, double *comp, double v)
{
    double s = *sum, t = s + v;
    if (fabs(s) >= fabs(v)) *comp += (s - t) + v;
    else *comp += (v - t) + s;
    *sum = t;
}

/*
 * map[p] = sum over samples i with pix[i] = p of tod[i] (1, c_i, s_i); hits[p] = count.
 * Sums are Neumaier-compensated. map and hits are overwritten; hits may be NULL.
 */
void orc_PT(int64_t npix, int64_t nsamp_total, const int32_t *pix, const double *cw, const double *sw,
            const double *tod, double *map, int32_t *hits)
{
    double *comp = (double *)calloc((size_t)npix * 3, sizeof(double));
    memset(map, 0, sizeof(double) * 3 * (size_t)npix);
    if (hits) memset(hits, 0, sizeof(int32_t) * (size_t)npix);
    for (int64_t i = 0; i < nsamp_total; ++i) {
        int32_t p = pix[i];
        if (p < 0) continue;
        double y = tod[i];
        orc_neumaier(map + 3 * (int64_t)p + 0, comp + 3 * (int64_t)p + 0, y);
        orc_neumaier(map + 3 * (int64_t)p + 1, comp + 3 * (int64_t)p + 1, y * cw[i]);
        orc_neumaier(map + 3 * (int64_t)p + 2, comp + 3 * (int64_t)p + 2, y * sw[i]);
        if (hits) hits[p] += 1;
    }
    for (int64_t k = 0; k < 3 * npix; ++k) map[k] += comp[k];
    free(comp);
}

/* ------------------------------------------------------------------------ */
/* N^-1: white and symmetric banded Toeplitz                                */
/* ------------------------------------------------------------------------ */

/* y[j][t] = x[j][t] / sigma2[j] */
void orc_ninv_white(int64_t ndet, int64_t nsamp, const double *sigma2, const double *x, double *y)
{
    for (int64_t j = 0; j < ndet; ++j)
        for (int64_t t = 0; t < nsamp; ++t) y[j * nsamp + t] = x[j * nsamp + t] / sigma2[j];
}

/*
 * y[j][t] = sum_{k=-(K-1)}^{K-1} taps[j][|k|] x[j][t+k], terms with t+k outside [0, nsamp)
 * dropped (the finite section of the infinite symmetric Toeplitz matrix), summed in
 * increasing k. in and out must not alias.
 */
void orc_ninv_band(int64_t ndet, int64_t nsamp, int64_t ntaps, const double *taps,
                   const double *x, double *y)
{
    for (int64_t j = 0; j < ndet; ++j) {
        const double *c = taps + j * ntaps;
        const double *xj = x + j * nsamp;
        double *yj = y + j * nsamp;
        for (int64_t t = 0; t < nsamp; ++t) {
            double acc = 0.0;
            for (int64_t k = -(ntaps - 1); k <= ntaps - 1; ++k) {
                int64_t u = t + k;
                if (u < 0 || u >= nsamp) continue;
                acc += c[k < 0 ? -k : k] * xj[u];
            }
            yj[t] = acc;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Block-Jacobi preconditioner                                              */
/* ------------------------------------------------------------------------ */
/*
 * M_p = sum_{i: pix[i]=p} w_i ninv[det(i)] w_i^T with w = (1, c, s): the 3x3 diagonal
 * blocks of P^T diag(N^-1) P. Stored as 6 unique entries (00,01,02,11,12,22).
 * Inverse via the Cholesky factor M = L L^T (backward stable for symmetric positive definite
 * matrices): M^-1 = L^-T L^-1; rcond = 1 / (||M||_1 ||M^-1||_1).
 * valid[p] = hits >= 3, every Cholesky pivot > 0 and rcond >= rcond_min; inv = 0 where invalid.
 * (A block that is singular in exact arithmetic - e.g. a pixel crossed several times with the
 * same angle - fails a pivot or yields a tiny rcond; an adjugate/determinant inverse of such a
 * block is rounding noise and can pass an rcond test with an indefinite "inverse".)
 */
static double orc_norm1_sym(const double *m)
{
    double c0 = fabs(m[0]) + fabs(m[1]) + fabs(m[2]);
    double c1 = fabs(m[1]) + fabs(m[3]) + fabs(m[4]);
    double c2 = fabs(m[2]) + fabs(m[4]) + fabs(m[5]);
    double r = c0 > c1 ? c0 : c1;
    return r > c2 ? r : c2;
}

/* Inverse of the symmetric 3x3 matrix m = (00,01,02,11,12,22) through its Cholesky factor
 * L (lower): l11 = sqrt(m00), l21 = m01/l11, l31 = m02/l11, l22 = sqrt(m11 - l21^2),
 * l32 = (m12 - l31 l21)/l22, l33 = sqrt(m22 - l31^2 - l32^2); W = L^-1 by forward substitution;
 * m^-1 = W^T W. Returns 0 (and leaves inv untouched) if a pivot is not positive. */
static int orc_bj_invert(const double *m, double *inv)
{
    if (!(m[0] > 0.0)) return 0;
    const double l11 = sqrt(m[0]);
    const double l21 = m[1] / l11, l31 = m[2] / l11;
    const double p2 = m[3] - l21 * l21;
    if (!(p2 > 0.0)) return 0;
    const double l22 = sqrt(p2);
    const double l32 = (m[4] - l31 * l21) / l22;
    const double p3 = (m[5] - l31 * l31) - l32 * l32;
    if (!(p3 > 0.0)) return 0;
    const double l33 = sqrt(p3);
    const double w11 = 1.0 / l11, w22 = 1.0 / l22, w33 = 1.0 / l33;
    const double w21 = -(l21 * w11) / l22;
    const double w32 = -(l32 * w22) / l33;
    const double w31 = -(l31 * w11 + l32 * w21) / l33;
    inv[0] = (w11 * w11 + w21 * w21) + w31 * w31;
    inv[1] = w21 * w22 + w31 * w32;
    inv[2] = w31 * w33;
    inv[3] = w22 * w22 + w32 * w32;
    inv[4] = w32 * w33;
    inv[5] = w33 * w33;
    return 1;
}

void orc_bj(int64_t npix, int64_t ndet, int64_t nsamp, const int32_t *pix, const double *cw,
            const double *sw, const double *ninv_diag, double rcond_min,
            double *blocks, double *inv, uint8_t *valid, int32_t *hits, double *rcond)
{
    double *comp = (double *)calloc((size_t)npix * 6, sizeof(double));
    memset(blocks, 0, sizeof(double) * 6 * (size_t)npix);
    memset(hits, 0, sizeof(int32_t) * (size_t)npix);
    for (int64_t j = 0; j < ndet; ++j) {
        double w0 = ninv_diag[j];
        for (int64_t t = 0; t < nsamp; ++t) {
            int64_t i = j * nsamp + t;
            int32_t p = pix[i];
            if (p < 0) continue;
            double c = cw[i], s = sw[i];
            double *b = blocks + 6 * (int64_t)p, *e = comp + 6 * (int64_t)p;
            orc_neumaier(b + 0, e + 0, w0);
            orc_neumaier(b + 1, e + 1, w0 * c);
            orc_neumaier(b + 2, e + 2, w0 * s);
            orc_neumaier(b + 3, e + 3, w0 * c * c);
            orc_neumaier(b + 4, e + 4, w0 * c * s);
            orc_neumaier(b + 5, e + 5, w0 * s * s);
            hits[p] += 1;
        }
    }
    for (int64_t k = 0; k < 6 * npix; ++k) blocks[k] += comp[k];
    free(comp);
    for (int64_t p = 0; p < npix; ++p) {
        const double *m = blocks + 6 * p;
        double *v = inv + 6 * p;
        double rc = 0.0;
        int ok = hits[p] >= 3 && orc_bj_invert(m, v);
        if (ok) {
            rc = 1.0 / (orc_norm1_sym(m) * orc_norm1_sym(v));
            ok = rc >= rcond_min;
        }
        if (!ok) for (int k = 0; k < 6; ++k) v[k] = 0.0;
        valid[p] = (uint8_t)ok;
        if (rcond) rcond[p] = rc;
    }
}

/* z_p = Minv_p r_p (symmetric 3x3 from 6 entries); zero where invalid. */
void orc_bj_apply(int64_t npix, const double *inv, const uint8_t *valid, const double *r, double *z)
{
    for (int64_t p = 0; p < npix; ++p) {
        const double *v = inv + 6 * p, *x = r + 3 * p;
        double *o = z + 3 * p;
        if (!valid[p]) { o[0] = o[1] = o[2] = 0.0; continue; }
        o[0] = v[0] * x[0] + v[1] * x[1] + v[2] * x[2];
        o[1] = v[1] * x[0] + v[3] * x[1] + v[4] * x[2];
        o[2] = v[2] * x[0] + v[4] * x[1] + v[5] * x[2];
    }
}

/* ------------------------------------------------------------------------ */
/* The normal-equations operator and PCG                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t npix, ndet, nsamp;
    const int32_t *pix;
    const double *cw, *sw;
    int noise_kind;          /* 0 white (sigma2[ndet]), 1 banded (taps[ndet][ntaps]) */
    const double *sigma2;
    const double *taps;
    int64_t ntaps;
    const uint8_t *valid;    /* may be NULL: no mask */
    double *tod, *tod2;      /* workspace [ndet*nsamp] */
} orc_problem;

static void orc_apply_ninv(const orc_problem *pb, const double *x, double *y)
{
    if (pb->noise_kind == 0) orc_ninv_white(pb->ndet, pb->nsamp, pb->sigma2, x, y);
    else orc_ninv_band(pb->ndet, pb->nsamp, pb->ntaps, pb->taps, x, y);
}

/* out = S P^T N^-1 P S^T x : the map-making operator restricted to valid pixels. */
static void orc_apply_A(const orc_problem *pb, const double *x, double *out)
{
    int64_t ns = pb->ndet * pb->nsamp;
    double *xs = NULL;
    if (pb->valid) {
        /* S^T x: unknowns exist only on valid pixels */
        xs = (double *)malloc(sizeof(double) * 3 * (size_t)pb->npix);
        for (int64_t p = 0; p < pb->npix; ++p)
            for (int k = 0; k < 3; ++k) xs[3 * p + k] = pb->valid[p] ? x[3 * p + k] : 0.0;
        x = xs;
    }
    orc_P(ns, pb->pix, pb->cw, pb->sw, x, pb->tod);
    free(xs);
    orc_apply_ninv(pb, pb->tod, pb->tod2);
    orc_PT(pb->npix, ns, pb->pix, pb->cw, pb->sw, pb->tod2, out, NULL);
    if (pb->valid)
        for (int64_t p = 0; p < pb->npix; ++p)
            if (!pb->valid[p]) out[3 * p] = out[3 * p + 1] = out[3 * p + 2] = 0.0;
}

static double orc_dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) orc_neumaier(&s, &c, a[i] * b[i]);
    return s + c;
}

/* rhs = S P^T N^-1 d */
void orc_rhs(int64_t npix, int64_t ndet, int64_t nsamp, const int32_t *pix, const double *cw,
             const double *sw, int noise_kind, const double *sigma2, const double *taps,
             int64_t ntaps, const uint8_t *valid, const double *d, double *rhs)
{
    int64_t ns = ndet * nsamp;
    double *tod = (double *)malloc(sizeof(double) * (size_t)ns);
    orc_problem pb = {npix, ndet, nsamp, pix, cw, sw, noise_kind, sigma2, taps, ntaps, valid, NULL, NULL};
    orc_apply_ninv(&pb, d, tod);
    orc_PT(npix, ns, pix, cw, sw, tod, rhs, NULL);
    if (valid)
        for (int64_t p = 0; p < npix; ++p)
            if (!valid[p]) rhs[3 * p] = rhs[3 * p + 1] = rhs[3 * p + 2] = 0.0;
    free(tod);
}

/* out = S P^T N^-1 P S^T x */
void orc_apply_ata(int64_t npix, int64_t ndet, int64_t nsamp, const int32_t *pix, const double *cw,
                   const double *sw, int noise_kind, const double *sigma2, const double *taps,
                   int64_t ntaps, const uint8_t *valid, const double *x, double *out)
{
    int64_t ns = ndet * nsamp;
    orc_problem pb = {npix, ndet, nsamp, pix, cw, sw, noise_kind, sigma2, taps, ntaps, valid, NULL, NULL};
    pb.tod = (double *)malloc(sizeof(double) * (size_t)ns);
    pb.tod2 = (double *)malloc(sizeof(double) * (size_t)ns);
    orc_apply_A(&pb, x, out);
    free(pb.tod); free(pb.tod2);
}

/*
 * Preconditioned conjugate gradient (Hestenes-Stiefel) on S P^T N^-1 P S^T x = b,
 * block-Jacobi preconditioner Minv, x0 = 0:
 *   r0 = b, z0 = M^-1 r0, p0 = z0;
 *   alpha = <r,z>/<p,Ap>; x += alpha p; r -= alpha Ap; z = M^-1 r;
 *   beta = <r',z'>/<r,z>; p = z + beta p.
 * Stops when ||r_k|| / ||b|| <= tol (recursive residual) or after maxiter steps.
 * hist[k] = ||r_k||/||b|| for k = 0..iters (needs maxiter+1 entries). Returns iters.
 */
int64_t orc_pcg(int64_t npix, int64_t ndet, int64_t nsamp, const int32_t *pix, const double *cw,
                const double *sw, int noise_kind, const double *sigma2, const double *taps,
                int64_t ntaps, const uint8_t *valid, const double *minv, const double *b,
                double *x, int64_t maxiter, double tol, double *hist)
{
    int64_t n = 3 * npix, ns = ndet * nsamp;
    orc_problem pb = {npix, ndet, nsamp, pix, cw, sw, noise_kind, sigma2, taps, ntaps, valid, NULL, NULL};
    pb.tod = (double *)malloc(sizeof(double) * (size_t)ns);
    pb.tod2 = (double *)malloc(sizeof(double) * (size_t)ns);
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    memset(x, 0, sizeof(double) * (size_t)n);
    memcpy(r, b, sizeof(double) * (size_t)n);
    orc_bj_apply(npix, minv, valid, r, z);
    memcpy(p, z, sizeof(double) * (size_t)n);
    double bnorm = sqrt(orc_dot(n, b, b));
    double rz = orc_dot(n, r, z);
    int64_t k = 0;
    if (hist) hist[0] = bnorm > 0 ? 1.0 : 0.0;
    while (k < maxiter) {
        if (bnorm == 0.0) break;
        orc_apply_A(&pb, p, q);
        double pq = orc_dot(n, p, q);
        double alpha = rz / pq;
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        orc_bj_apply(npix, minv, valid, r, z);
        double rz_new = orc_dot(n, r, z);
        double rel = sqrt(orc_dot(n, r, r)) / bnorm;
        ++k;
        if (hist) hist[k] = rel;
        if (rel <= tol) break;
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    free(pb.tod); free(pb.tod2); free(r); free(z); free(p); free(q);
    return k;
}

/* ------------------------------------------------------------------------ */
/* chi^2 and its gradients                                                  */
/* ------------------------------------------------------------------------ */
/*
 * r = d - P(delta) m,  chi2 = r^T N^-1 r,
 * dchi2/dm = -2 P^T N^-1 r,
 * dchi2/ddelta_j = -2 sum_t (N^-1 r)_{j,t} * 2 (U_p c_{j,t} - Q_p s_{j,t}),
 * with (c, s) already including the offsets delta (from orc_pointing). grad_map and
 * grad_psi may be NULL. Returns chi2 (Neumaier-summed).
 */
double orc_chi2_grad(int64_t npix, int64_t ndet, int64_t nsamp, const int32_t *pix, const double *cw,
                     const double *sw, int noise_kind, const double *sigma2, const double *taps,
                     int64_t ntaps, const double *map, const double *d, double *grad_map,
                     double *grad_psi)
{
    int64_t ns = ndet * nsamp;
    orc_problem pb = {npix, ndet, nsamp, pix, cw, sw, noise_kind, sigma2, taps, ntaps, NULL, NULL, NULL};
    double *r = (double *)malloc(sizeof(double) * (size_t)ns);
    double *nr = (double *)malloc(sizeof(double) * (size_t)ns);
    orc_P(ns, pix, cw, sw, map, r);
    for (int64_t i = 0; i < ns; ++i) r[i] = d[i] - r[i];
    orc_apply_ninv(&pb, r, nr);
    double chi2 = orc_dot(ns, r, nr);
    if (grad_map) {
        orc_PT(npix, ns, pix, cw, sw, nr, grad_map, NULL);
        for (int64_t k = 0; k < 3 * npix; ++k) grad_map[k] *= -2.0;
    }
    if (grad_psi) {
        for (int64_t j = 0; j < ndet; ++j) {
            double s = 0.0, c = 0.0;
            for (int64_t t = 0; t < nsamp; ++t) {
                int64_t i = j * nsamp + t;
                int32_t p = pix[i];
                if (p < 0) continue;
                const double *m = map + 3 * (int64_t)p;
                double dt = 2.0 * (m[2] * cw[i] - m[1] * sw[i]);
                orc_neumaier(&s, &c, nr[i] * dt);
            }
            grad_psi[j] = -2.0 * (s + c);
        }
    }
    free(r); free(nr);
    return chi2;
}
