// Template deprojection: the weighting-and-deprojection operator
//   F_T = W - W T (T^T W T)^-1 T^T W
// of the Furax paper (Statement of Need, the generalised least-squares estimator with
// templates; TemplateOperator, Table 3), with W = N^-1 and, for each detector, the Legendre
// polynomials P_0 .. P_K (K <= 3) of the scaled time tau_t = 2t/(ns-1) - 1 as templates.
//
// The deprojected normal operator is the plain one minus a correction of rank K+1 per detector
// (W is symmetric, so T^T W u = (W T)^T u):
//   P^T F_T P x = P^T W P x - P^T (W T) b,   b = G^-1 (W T)^T P x,   G = T^T W T.
// The fused kernels of P^T N^-1 P are used unchanged; three small kernels add the rest:
//   project  a_det = (W T)^T u over the detector's stream (u = P x, or a TOD),
//   solve    b_det = G_det^-1 a_det,
//   scatter  acc -= P^T (W T) b   (or, for a TOD, y -= (W T) b).
// For the right-hand side of FP32 data in the mixed-precision solver the scatter is not a pass of
// its own: the double-FP32 pass that forms P^T W d subtracts (W T) b from W d per sample.
//
// (W T)(t) needs no band product. For a polynomial p of degree <= 3 and a symmetric band whose
// full width fits around t,
//   sum_k c_|k| p(tau_t + h k) = mu0 p(tau_t) + (mu2 h^2 / 2) p''(tau_t),
// with mu0 = sum_k c_|k|, mu2 = sum_k k^2 c_|k| over k = -halo..halo and h = 2/(ns-1): the odd
// moments of a symmetric band vanish and the fourth derivative of p is zero. Within a half-width
// of either end of the stream the truncated sum is taken term by term.
#include "tile.cuh"
#include "tpl_eval.cuh"
#include "dfloat.cuh"

namespace fx {

// Sum of v[0..N) over the CTA (FT threads); the result is valid in thread 0.
template <int N, typename T>
__device__ __forceinline__ void cta_sum(T (&v)[N])
{
    __shared__ T red[FT / 32][N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) red[warp][i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            T s = T(0);
            for (int w = 0; w < FT / 32; ++w) s += red[w][i];
            v[i] = s;
        }
    }
}

// ------------------------------------------------------------------------------------ setup
// (mu0, mu2) per detector from its band (white noise: mu0 = 1/sigma^2, mu2 = 0).
__global__ void tpl_moments_kernel(int64_t ndet, NoiseView nv, int halo, double2 *mom)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet) return;
    double m0 = tpl_tap<double>(nv, i, 0), m2 = 0.0;
    for (int k = 1; k <= halo; ++k) {
        const double c = tpl_tap<double>(nv, i, k);
        m0 += 2.0 * c;
        m2 += 2.0 * (double)k * (double)k * c;
    }
    mom[i] = make_double2(m0, m2);
}

// gram[det] += sum over the tile of P_k(tau_t) (W P_l)(t), k, l < 4 (FP64). Interior samples enter
// through the power sums S_m = sum tau^m (m <= 6): there (W P_l) = mu0 P_l + k2 P_l'' with
// k2 = mu2 h^2 / 2, so the entry is sum_{m,n} A_km (mu0 A_ln + k2 B_ln) S_{m+n} with A the
// Legendre coefficients in powers of tau and B those of P_l''. Samples within a half-band of
// either end are summed term by term.
__global__ void __launch_bounds__(FT) tpl_gram_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                      NoiseView nv, TplView tv, double *__restrict__ gram)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    const double h = ob.nsamp > 1 ? 2.0 / (double)(ob.nsamp - 1) : 0.0;
    double S[7], g[16];
#pragma unroll
    for (int i = 0; i < 7; ++i) S[i] = 0.0;
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = 0.0;
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t t = tl.t0 + u;
        const double tau = tpl_tau<double>(t, ob.nsamp, h);
        if (tpl_interior(tv, t, ob.nsamp)) {
            double v = 1.0;
#pragma unroll
            for (int m = 0; m < 7; ++m) {
                S[m] += v;
                v *= tau;
            }
        } else {
            double w[4], L[4];
            wt_eval<double>(nv, tv, gdet, ob.nsamp, t, w);
            legendre4(tau, L);
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int l = 0; l < 4; ++l) g[4 * k + l] += L[k] * w[l];
        }
    }
    const bool has_edge = tl.t0 < tv.halo || tl.t0 + tl.len + tv.halo > ob.nsamp;   // CTA-uniform
    cta_sum<7, double>(S);
    if (has_edge) cta_sum<16, double>(g);
    if (threadIdx.x != 0) return;
    constexpr double A[4][4] = {{1.0, 0.0, 0.0, 0.0}, {0.0, 1.0, 0.0, 0.0}, {-0.5, 0.0, 1.5, 0.0}, {0.0, -1.5, 0.0, 2.5}};
    constexpr double B[4][2] = {{0.0, 0.0}, {0.0, 0.0}, {3.0, 0.0}, {0.0, 15.0}};   // P_l'' = B_l0 + B_l1 tau
    const double2 mo = tv.mom[gdet];
    const double mu0 = mo.x, k2 = mo.y * h * h * 0.5;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (k > tv.order || l > tv.order) continue;
            double v = 0.0;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (A[k][m] == 0.0) continue;
                double c = 0.0;
#pragma unroll
                for (int n = 0; n < 4; ++n)
                    if (A[l][n] != 0.0) c += mu0 * A[l][n] * S[m + n];
#pragma unroll
                for (int n = 0; n < 2; ++n)
                    if (B[l][n] != 0.0) c += k2 * B[l][n] * S[m + n];
                v += A[k][m] * c;
            }
            red_add_f64(gram + 16 * gdet + 4 * k + l, v + (has_edge ? g[4 * k + l] : 0.0));
        }
}

// ginv[det] = G^-1 by Cholesky (K+1 <= 4, FP64). A pivot that loses all but 1e-13 of its
// diagonal entry marks the Gram matrix as not positive definite (bad[0] = 1 + det).
__global__ void tpl_invert_kernel(int64_t ndet, int order, const double *__restrict__ gram, double *__restrict__ ginv,
                                  unsigned long long *bad)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet) return;
    const int n = order + 1;
    double G[4][4], L[4][4], Li[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) { G[r][c] = 0.5 * (gram[16 * i + 4 * r + c] + gram[16 * i + 4 * c + r]); L[r][c] = 0.0; Li[r][c] = 0.0; }
    bool ok = true;
    for (int j = 0; j < n; ++j) {
        double d = G[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 1e-13 * G[j][j]) || !(G[j][j] > 0.0)) { ok = false; break; }
        L[j][j] = sqrt(d);
        for (int r = j + 1; r < n; ++r) {
            double v = G[r][j];
            for (int k = 0; k < j; ++k) v -= L[r][k] * L[j][k];
            L[r][j] = v / L[j][j];
        }
    }
    if (!ok) {
        atomicCAS(bad, 0ull, (unsigned long long)(i + 1));
        for (int k = 0; k < 16; ++k) ginv[16 * i + k] = 0.0;
        return;
    }
    // L^-1 by forward substitution, then G^-1 = L^-T L^-1.
    for (int c = 0; c < n; ++c) {
        for (int r = c; r < n; ++r) {
            double v = r == c ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) v -= L[r][k] * Li[k][c];
            Li[r][c] = v / L[r][r];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double v = 0.0;
            if (r < n && c < n)
                for (int k = 0; k < n; ++k) v += Li[k][r] * Li[k][c];
            ginv[16 * i + 4 * r + c] = v;
        }
}

// ------------------------------------------------------------------------------------ apply
template <typename T>
__device__ __forceinline__ T map_value(const float4 *x, int64_t gp, T c, T s)
{
    const float4 m = __ldg(x + gp);
    return T(m.x) + T(m.y) * c + T(m.z) * s;
}

template <typename T>
__device__ __forceinline__ T map_value(const double *x, int64_t gp, T c, T s)
{
    return T(x[3 * gp]) + T(x[3 * gp + 1]) * c + T(x[3 * gp + 2]) * s;
}

// a[det] += scale sum_t (W T)(t) u_t, u = P x (map x: FP32 float4 or FP64 [np][3]) or a TOD d.
template <int MODE, typename T, typename XT, bool FROM_TOD, typename DT>
__global__ void __launch_bounds__(FT) tpl_project_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                         TplView tv, const XT *__restrict__ x,
                                                         const DT *__restrict__ d, double scale, double *__restrict__ a)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    const T h = ob.nsamp > 1 ? T(2) / T(ob.nsamp - 1) : T(0);
    // interior samples: power sums pw[m] = sum u tau^m, combined with the band's moments at the end
    T acc[4] = {T(0), T(0), T(0), T(0)}, pw[4] = {T(0), T(0), T(0), T(0)};
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t t = tl.t0 + u;
        T val;
        if constexpr (FROM_TOD) {
            val = T(d[ob.tod_off + (int64_t)tl.det * ob.nsamp + t]);
        } else {
            T c, s;
            const int32_t pix = get_sample<MODE, T>(pv, ob, tl.det, t, c, s);
            if (pix < 0) continue;
            val = map_value<T>(x, ob.map_off + pix, c, s);
        }
        if (t >= tv.halo && t + tv.halo < ob.nsamp) {
            const T tau = tpl_tau<T>(t, ob.nsamp, h);
            T v = val;
            pw[0] += v; v *= tau;
            pw[1] += v; v *= tau;
            pw[2] += v; v *= tau;
            pw[3] += v;
        } else {
            T w[4];
            wt_eval<T>(nv, tv, gdet, ob.nsamp, t, w);
#pragma unroll
            for (int l = 0; l < 4; ++l) acc[l] += w[l] * val;
        }
    }
    {   // interior (W P_l)(tau) = mu0 P_l(tau) + (mu2 h^2 / 2) P_l''(tau)
        const double2 m = tv.mom[gdet];
        const T mu0 = T(m.x), k2 = T(m.y) * h * h * T(0.5);
        acc[0] += mu0 * pw[0];
        acc[1] += mu0 * pw[1];
        acc[2] += mu0 * (T(1.5) * pw[2] - T(0.5) * pw[0]) + T(3) * k2 * pw[0];
        acc[3] += mu0 * (T(2.5) * pw[3] - T(1.5) * pw[1]) + T(15) * k2 * pw[1];
    }
    cta_sum<4, T>(acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int l = 0; l < 4; ++l)
            if (l <= tv.order) red_add_f64(a + 4 * gdet + l, scale * (double)acc[l]);
}

// a[det] += scale sum_t (W T)(t) d_t for FP32 data d, FP64-accurate on FP32 units. Interior samples
// (band fully inside the stream) contribute through the power sums Q_i = sum d_t j^i (i <= 3) of
// the offset j = t - t_c from the middle sample t_c of the tile (so that |tau_c| <= 1 and the
// re-expansion does not extrapolate), accumulated as double-FP32 compensated
// dot products with exact multipliers (j and j^2 are exact in binary32 for |j| <= 2048; j^3 is
// split exactly into two words); the CTA combines them in FP64 with tau = tau_c + h j and the
// band's moments. Samples near the ends of the stream take the FP64 term-by-term sum.
__global__ void __launch_bounds__(FT) tpl_project_tod_df_kernel(const Tile *__restrict__ tiles,
                                                                const ObsInfo *__restrict__ obs, NoiseView nv,
                                                                TplView tv, const float *__restrict__ d, double scale,
                                                                double *__restrict__ a)
{
    static_assert(TILE / 2 <= 2048, "offsets and their squares must be exact in binary32");
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    const float *row = d + ob.tod_off + (int64_t)tl.det * ob.nsamp;
    float S[4] = {0.f, 0.f, 0.f, 0.f}, E[4] = {0.f, 0.f, 0.f, 0.f};
    double edge[4] = {0.0, 0.0, 0.0, 0.0};
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t t = tl.t0 + u;
        const float x = row[t];
        if (tpl_interior(tv, t, ob.nsamp)) {
            const float j = (float)(u - (tl.len >> 1));
            const float j2 = __fmul_rn(j, j);
            const float j3 = __fmul_rn(j2, j), j3l = __fmaf_rn(j2, j, -j3);
            dot2_step_x(1.f, 0.f, x, S[0], E[0]);
            dot2_step_x(j, 0.f, x, S[1], E[1]);
            dot2_step_x(j2, 0.f, x, S[2], E[2]);
            dot2_step_x(j3, j3l, x, S[3], E[3]);
        } else {
            double w[4];
            wt_eval<double>(nv, tv, gdet, ob.nsamp, t, w);
#pragma unroll
            for (int l = 0; l < 4; ++l) edge[l] += w[l] * (double)x;
        }
    }
    // warp sums in double-FP32, then FP64 across the warps
    __shared__ double red[FT / 32][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float h, l;
        df_renorm(S[i], E[i], h, l);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, h, o), ol = __shfl_down_sync(0xffffffffu, l, o);
            df_add(h, l, oh, ol);
        }
        S[i] = h;
        E[i] = l;
    }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) red[threadIdx.x >> 5][i] = (double)S[i] + (double)E[i];
    // edge samples only occur in a stream's first and last tiles
    const bool has_edge = tl.t0 < tv.halo || tl.t0 + tl.len + tv.halo > ob.nsamp;
    if (has_edge) cta_sum<4, double>(edge);
    else __syncthreads();
    if (threadIdx.x != 0) return;
    double Q[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Q[i] = 0.0;
        for (int w = 0; w < FT / 32; ++w) Q[i] += red[w][i];
    }
    const double h = ob.nsamp > 1 ? 2.0 / (double)(ob.nsamp - 1) : 0.0;
    const double tc = tpl_tau_ref(tl.t0 + (tl.len >> 1), ob.nsamp);
    const double hq1 = h * Q[1], h2q2 = h * h * Q[2], h3q3 = h * h * h * Q[3];
    // pw[m] = sum d tau^m over the interior samples, tau = tc + h j
    const double pw0 = Q[0];
    const double pw1 = tc * Q[0] + hq1;
    const double pw2 = tc * (tc * Q[0] + 2.0 * hq1) + h2q2;
    const double pw3 = tc * (tc * (tc * Q[0] + 3.0 * hq1) + 3.0 * h2q2) + h3q3;
    const double2 m = tv.mom[gdet];
    const double mu0 = m.x, k2 = m.y * h * h * 0.5;
    const double v[4] = {mu0 * pw0, mu0 * pw1, mu0 * (1.5 * pw2 - 0.5 * pw0) + 3.0 * k2 * pw0,
                         mu0 * (2.5 * pw3 - 1.5 * pw1) + 15.0 * k2 * pw1};
#pragma unroll
    for (int l = 0; l < 4; ++l)
        if (l <= tv.order) red_add_f64(a + 4 * gdet + l, scale * (v[l] + (has_edge ? edge[l] : 0.0)));
}

// b[det] = G^-1 a[det]; a[det] = 0 for the next projection.
__global__ void tpl_solve_kernel(int64_t ndet, const double *__restrict__ ginv, double *__restrict__ a,
                                 double *__restrict__ b)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet) return;
    double av[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) { av[l] = a[4 * i + l]; a[4 * i + l] = 0.0; }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = 0.0;
#pragma unroll
        for (int l = 0; l < 4; ++l) v += ginv[16 * i + 4 * k + l] * av[l];
        b[4 * i + k] = v;
    }
}

// sum_l b_l (W P_l)(t) for one detector stream: in the interior the cubic c0 + c1 tau + c2 tau^2 + c3 tau^3,
// whose coefficients are fixed per detector; term by term within a half-band of either end.
template <typename T>
struct TplPoly {
    T h, c[4];
    __device__ __forceinline__ TplPoly(const TplView &tv, int64_t gdet, int64_t ns, const T (&bv)[4])
    {
        h = ns > 1 ? T(2) / T(ns - 1) : T(0);
        const double2 m = tv.mom[gdet];
        const T mu0 = T(m.x), k2 = T(m.y) * h * h * T(0.5);
        c[0] = mu0 * (bv[0] - T(0.5) * bv[2]) + T(3) * k2 * bv[2];
        c[1] = mu0 * (bv[1] - T(1.5) * bv[3]) + T(15) * k2 * bv[3];
        c[2] = T(1.5) * mu0 * bv[2];
        c[3] = T(2.5) * mu0 * bv[3];
    }
};

template <typename T>
__device__ __forceinline__ T tpl_value(const NoiseView &nv, const TplView &tv, int64_t gdet, int64_t ns, int64_t t,
                                       const T (&bv)[4], const TplPoly<T> &pl)
{
    if (t >= tv.halo && t + tv.halo < ns) {
        const T tau = tpl_tau<T>(t, ns, pl.h);
        return ((pl.c[3] * tau + pl.c[2]) * tau + pl.c[1]) * tau + pl.c[0];
    }
    T w[4];
    wt_eval<T>(nv, tv, gdet, ns, t, w);
    return bv[0] * w[0] + bv[1] * w[1] + bv[2] * w[2] + bv[3] * w[3];
}

// acc[pix] -= v (1, c, s) with v = sum_l b_l (W P_l)(t): subtracts P^T (W T) b.
template <int MODE, typename T, int ACC>
__global__ void __launch_bounds__(FT) tpl_scatter_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                         TplView tv, float4 *__restrict__ hi, float4 *__restrict__ lo,
                                                         double *__restrict__ acc64)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    T bv[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) bv[l] = T(tv.b[4 * gdet + l]);
    const TplPoly<T> pl(tv, gdet, ob.nsamp, bv);
    if constexpr (ACC == FURAX_ACC_F64) {
        // three FP64 sums per sample, issued as whole pixel records by the warp (values of type
        // T, widened after the exchange); warp-uniform trip count
        __shared__ T stage[FT / 32][96];
        __shared__ int32_t spx[FT / 32][32];
        double *base = acc64 + 3 * ob.map_off;
        for (int uw = threadIdx.x & ~31; uw < tl.len; uw += FT) {
            const int u = uw + (threadIdx.x & 31);
            int32_t pix = -1;
            T v3[3] = {T(0), T(0), T(0)};
            if (u < tl.len) {
                const int64_t t = tl.t0 + u;
                T c, s;
                pix = get_sample<MODE, T>(pv, ob, tl.det, t, c, s);
                if (pix >= 0) {
                    const T v = -tpl_value<T>(nv, tv, gdet, ob.nsamp, t, bv, pl);
                    v3[0] = v;
                    v3[1] = v * c;
                    v3[2] = v * s;
                }
            }
            red_add_f64_records_warp<3, T>(base, pix, v3, stage[threadIdx.x >> 5], spx[threadIdx.x >> 5]);
        }
        return;
    }
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t t = tl.t0 + u;
        T c, s;
        const int32_t pix = get_sample<MODE, T>(pv, ob, tl.det, t, c, s);
        if (pix < 0) continue;
        const T v = -tpl_value<T>(nv, tv, gdet, ob.nsamp, t, bv, pl);
        const int64_t gp = ob.map_off + pix;
        if constexpr (ACC == FURAX_ACC_F32) {
            red_add_v4(hi + gp, make_float4(float(v), float(v * c), float(v * s), 0.f));
        } else {
            kahan_add_v4(hi + kKahanStride * gp, lo + kKahanStride * gp,
                         make_float4(float(v), float(v * c), float(v * s), 0.f));
        }
    }
}

// y[t] -= sum_l b_l (W P_l)(t) over a TOD.
template <typename T>
__global__ void __launch_bounds__(FT) tpl_tod_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                     NoiseView nv, TplView tv, T *__restrict__ y)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    T bv[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) bv[l] = T(tv.b[4 * gdet + l]);
    const TplPoly<T> pl(tv, gdet, ob.nsamp, bv);
    T *row = y + ob.tod_off + (int64_t)tl.det * ob.nsamp;
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t t = tl.t0 + u;
        row[t] -= tpl_value<T>(nv, tv, gdet, ob.nsamp, t, bv, pl);
    }
}

// ------------------------------------------------------------------------------------ launchers
static unsigned det_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 127) / 128); }

template <typename T, typename XT, bool FROM_TOD, typename DT>
static void project_mode(const furax_templates *tp, const XT *x, const DT *d, cudaStream_t st, double scale = 1.0)
{
    const furax_pointing *p = tp->p;
    const unsigned g = (unsigned)p->n_tiles;
    if constexpr (FROM_TOD && sizeof(T) == 8 && sizeof(DT) == 4) {   // FP64-accurate from FP32 data
        tpl_project_tod_df_kernel<<<g, FT, 0, st>>>(p->d_tiles, p->d_obs, tp->n->view(), tp->view(), d, scale, tp->a);
    } else {
        const PointingView pv = p->view();
        const NoiseView nv = tp->n->view();
        const TplView tv = tp->view();
        switch (FROM_TOD ? 2 : p->mode) {
        case FURAX_POINTING_ON_THE_FLY: tpl_project_kernel<0, T, XT, FROM_TOD, DT><<<g, FT, 0, st>>>(p->d_tiles, pv, nv, tv, x, d, scale, tp->a); break;
        case FURAX_POINTING_CACHE_F32: tpl_project_kernel<1, T, XT, FROM_TOD, DT><<<g, FT, 0, st>>>(p->d_tiles, pv, nv, tv, x, d, scale, tp->a); break;
        case FURAX_POINTING_CACHE_MIXED: tpl_project_kernel<3, T, XT, FROM_TOD, DT><<<g, FT, 0, st>>>(p->d_tiles, pv, nv, tv, x, d, scale, tp->a); break;
        default: tpl_project_kernel<2, T, XT, FROM_TOD, DT><<<g, FT, 0, st>>>(p->d_tiles, pv, nv, tv, x, d, scale, tp->a); break;
        }
    }
}

template <typename T, int ACC>
static void scatter_mode(const furax_templates *tp, float4 *hi, float4 *lo, double *a64, cudaStream_t st)
{
    const furax_pointing *p = tp->p;
    const unsigned g = (unsigned)p->n_tiles;
    const PointingView pv = p->view();
    const NoiseView nv = tp->n->view();
    const TplView tv = tp->view();
    switch (p->mode) {
    case FURAX_POINTING_ON_THE_FLY: tpl_scatter_kernel<0, T, ACC><<<g, FT, 0, st>>>(p->d_tiles, pv, nv, tv, hi, lo, a64); break;
    case FURAX_POINTING_CACHE_F32: tpl_scatter_kernel<1, T, ACC><<<g, FT, 0, st>>>(p->d_tiles, pv, nv, tv, hi, lo, a64); break;
    case FURAX_POINTING_CACHE_MIXED: tpl_scatter_kernel<3, T, ACC><<<g, FT, 0, st>>>(p->d_tiles, pv, nv, tv, hi, lo, a64); break;
    default: tpl_scatter_kernel<2, T, ACC><<<g, FT, 0, st>>>(p->d_tiles, pv, nv, tv, hi, lo, a64); break;
    }
}

static void solve(const furax_templates *tp, cudaStream_t st)
{
    tpl_solve_kernel<<<det_grid(tp->ndet), 128, 0, st>>>(tp->ndet, tp->ginv, tp->a, tp->b);
}

double *tpl_fused_target(const furax_templates *tp, const furax_pointing *p)
{
    return tp && !long_band(tp->n) && fused_f32_projects_templates(p) ? tp->a : nullptr;
}

furax_status launch_tpl_map(const furax_templates *tp, int precision, int acc, const float4 *x32, const double *x64,
                            float4 *hi, float4 *lo, double *acc64, cudaStream_t st, bool projected)
{
    if (tp->p->n_tiles == 0) return FURAX_OK;
    if (precision == FURAX_F32) {
        if (!projected) project_mode<float, float4, false, float>(tp, x32, nullptr, st);
        solve(tp, st);
        if (acc == FURAX_ACC_F32) scatter_mode<float, FURAX_ACC_F32>(tp, hi, lo, acc64, st);
        else if (acc == FURAX_ACC_F32_KAHAN) scatter_mode<float, FURAX_ACC_F32_KAHAN>(tp, hi, lo, acc64, st);
        else scatter_mode<float, FURAX_ACC_F64>(tp, hi, lo, acc64, st);
    } else {
        project_mode<double, double, false, float>(tp, x64, nullptr, st);
        solve(tp, st);
        scatter_mode<double, FURAX_ACC_F64>(tp, hi, lo, acc64, st);
    }
    count_launches(projected && precision == FURAX_F32 ? 2 : 3);
    return check_launch("template deprojection (map)");
}

furax_status launch_tpl_rhs_amplitudes(const furax_templates *tp, const void *d, int d_t, cudaStream_t st)
{
    if (tp->p->n_tiles > 0) {
        if (d_t == FURAX_F64) project_mode<double, double, true, double>(tp, nullptr, (const double *)d, st);
        else project_mode<double, double, true, float>(tp, nullptr, (const float *)d, st);
    }
    solve(tp, st);
    count_launches(2);
    return check_launch("template amplitudes of the right-hand side");
}

furax_status launch_tpl_rhs(const furax_templates *tp, const void *d, int d_t, double *acc64, cudaStream_t st)
{
    if (tp->p->n_tiles == 0) return FURAX_OK;
    if (d_t == FURAX_F64) project_mode<double, double, true, double>(tp, nullptr, (const double *)d, st);
    else project_mode<double, double, true, float>(tp, nullptr, (const float *)d, st);
    solve(tp, st);
    scatter_mode<double, FURAX_ACC_F64>(tp, nullptr, nullptr, acc64, st);
    count_launches(3);
    return check_launch("template deprojection (right-hand side)");
}

furax_status deproject_apply(const furax_templates *tp, const void *in, void *out, int dtype, cudaStream_t st)
{
    furax_status rc = launch_ninv(tp->n, in, out, dtype, st);   // out = W x
    if (rc || tp->p->n_tiles == 0) return rc;
    const furax_pointing *p = tp->p;
    const unsigned g = (unsigned)p->n_tiles;
    if (dtype == FURAX_F64) {
        project_mode<double, double, true, double>(tp, nullptr, (const double *)in, st);
        solve(tp, st);
        tpl_tod_kernel<double><<<g, FT, 0, st>>>(p->d_tiles, p->d_obs, tp->n->view(), tp->view(), (double *)out);
    } else {
        project_mode<float, double, true, float>(tp, nullptr, (const float *)in, st);
        solve(tp, st);
        tpl_tod_kernel<float><<<g, FT, 0, st>>>(p->d_tiles, p->d_obs, tp->n->view(), tp->view(), (float *)out);
    }
    count_launches(3);
    return check_launch("template deprojection (TOD)");
}

// ------------------------------------------------------------------------------------ augmented
// The inner FP32 solve of the mixed-precision PCG runs on the augmented normal equations
//   [P^T W P   P^T W T] [e]   [r]
//   [T^T W P   T^T W T] [f] = [0],
// whose map part e solves (P^T F_T P) e = r (eliminate f: f = -G^-1 T^T W P e). Its operator is
// one fused pass (the amplitudes are one pseudo-pixel per detector that every sample of the
// detector reads with weights (P_0, P_1, P_2)(tau)), and its block-Jacobi block for a pseudo-
// pixel is G^-1.
bool tpl_augmented(const furax_templates *tp, int precision)
{
    return tp && precision == FURAX_F32 && tp->order <= 2 && tp->d_aug_ptiles && !long_band(tp->n) &&
           fused_f32_projects_templates(tp->p);
}

__global__ void tpl_aug_precond_kernel(int64_t ndet, int64_t base, const double *__restrict__ ginv,
                                       double *__restrict__ minv, uint8_t *__restrict__ valid)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet) return;
    const double *g = ginv + 16 * i;   // zero beyond the order
    double *m = minv + 6 * (base + i);
    m[0] = g[0]; m[1] = g[1]; m[2] = g[2]; m[3] = g[5]; m[4] = g[6]; m[5] = g[10];
    valid[base + i] = 1;
}

furax_status launch_tpl_aug_precond(const furax_templates *tp, double *minv, uint8_t *valid, cudaStream_t st)
{
    if (tp->ndet == 0) return FURAX_OK;
    tpl_aug_precond_kernel<<<det_grid(tp->ndet), 128, 0, st>>>(tp->ndet, tp->p->npix_total, tp->ginv, minv, valid);
    count_launches(1);
    return check_launch("amplitude preconditioner");
}

// Pixel tiles of the augmented system: every map's pixel tiles, then the amplitude pseudo-pixels
// of all detectors of its observations; observations carry their map's range.
static furax_status build_aug_layout(furax_templates *tp, cudaStream_t st)
{
    const furax_pointing *p = tp->p;
    const int64_t base = p->npix_total;
    std::vector<PTile> pt;
    std::vector<ObsInfo> ob = p->obs;
    std::vector<int> owner(p->obs.size());
    for (size_t i = 0; i < p->obs.size(); ++i) {
        owner[i] = (int)i;
        for (size_t j = 0; j < i; ++j)
            if (p->obs[j].map_off == p->obs[i].map_off) { owner[i] = (int)j; break; }
    }
    for (size_t k = 0; k < p->obs.size(); ++k) {
        if (owner[k] != (int)k) continue;
        const int64_t first = (int64_t)pt.size();
        for (int64_t t = 0; t < p->obs[k].nptile; ++t) pt.push_back(p->ptiles[p->obs[k].ptile0 + t]);
        for (size_t i = k; i < p->obs.size(); ++i) {
            if (owner[i] != (int)k) continue;
            for (int32_t d0 = 0; d0 < p->obs[i].ndet; d0 += PTILE) {
                PTile t;
                t.p0 = base + p->obs[i].det_off + d0;
                t.obs = (int32_t)k;
                t.len = std::min<int32_t>(PTILE, p->obs[i].ndet - d0);
                pt.push_back(t);
            }
        }
        for (size_t i = k; i < p->obs.size(); ++i)
            if (owner[i] == (int)k) { ob[i].ptile0 = first; ob[i].nptile = (int32_t)((int64_t)pt.size() - first); }
    }
    tp->n_aug_ptiles = (int64_t)pt.size();
    furax_status rc = check_cuda(cudaMalloc((void **)&tp->d_aug_ptiles, sizeof(PTile) * std::max<size_t>(1, pt.size())),
                                 "template workspace");
    if (!rc) rc = check_cuda(cudaMalloc((void **)&tp->d_aug_obs, sizeof(ObsInfo) * ob.size()), "template workspace");
    if (!rc && !pt.empty())
        rc = check_cuda(cudaMemcpyAsync(tp->d_aug_ptiles, pt.data(), sizeof(PTile) * pt.size(), cudaMemcpyHostToDevice, st),
                        "copy layout");
    if (!rc)
        rc = check_cuda(cudaMemcpyAsync(tp->d_aug_obs, ob.data(), sizeof(ObsInfo) * ob.size(), cudaMemcpyHostToDevice, st),
                        "copy layout");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "copy layout");   // the host vectors go out of scope
    return rc;
}

// amp[det][l] (l <= K) = G^-1 (W T)^T (d - P m): the template amplitudes of the map m.
furax_status tpl_amplitudes(const furax_templates *tp, const void *d, int d_t, const double *m, double *amp,
                            cudaStream_t st)
{
    if (tp->ndet == 0) return FURAX_OK;
    if (tp->p->n_tiles > 0) {
        if (d_t == FURAX_F64) project_mode<double, double, true, double>(tp, nullptr, (const double *)d, st);
        else project_mode<double, double, true, float>(tp, nullptr, (const float *)d, st);
        project_mode<double, double, false, float>(tp, m, nullptr, st, -1.0);
    }
    solve(tp, st);
    count_launches(3);
    furax_status rc = check_launch("template amplitudes");
    if (rc) return rc;
    const int k1 = tp->order + 1;
    return check_cuda(cudaMemcpy2DAsync(amp, sizeof(double) * k1, tp->b, sizeof(double) * 4, sizeof(double) * k1,
                                        (size_t)tp->ndet, cudaMemcpyDeviceToDevice, st),
                      "copy amplitudes");
}

__global__ void tpl_gram_out_kernel(int64_t ndet, int k1, const double *__restrict__ gram, double *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet * k1 * k1) return;
    const int64_t det = i / (k1 * k1);
    const int r = (int)(i / k1 % k1), c = (int)(i % k1);
    out[i] = gram[16 * det + 4 * r + c];
}

furax_status tpl_gram_out(const furax_templates *tp, double *out, cudaStream_t st)
{
    const int k1 = tp->order + 1;
    const int64_t n = tp->ndet * k1 * k1;
    if (n == 0) return FURAX_OK;
    tpl_gram_out_kernel<<<det_grid(n), 128, 0, st>>>(tp->ndet, k1, tp->gram, out);
    count_launches(1);
    return check_launch("template Gram matrices");
}

void templates_destroy(furax_templates *tp)
{
    if (!tp) return;
    cudaFree(tp->mom); cudaFree(tp->gram); cudaFree(tp->ginv); cudaFree(tp->a); cudaFree(tp->b); cudaFree(tp->bad);
    cudaFree(tp->d_aug_ptiles); cudaFree(tp->d_aug_obs);
    delete tp;
}

furax_status templates_create(const furax_pointing *p, const furax_noise *n, int order, cudaStream_t st,
                              furax_templates **out)
{
    for (const ObsInfo &o : p->obs)
        if (o.ndet > 0 && o.nsamp < order + 1)
            return set_error(FURAX_EBADINPUT, "a stream of %lld samples cannot carry %d templates", (long long)o.nsamp,
                             order + 1);
    furax_templates *tp = new furax_templates();
    tp->p = p;
    tp->n = n;
    tp->order = order;
    tp->halo = n->kind == FURAX_NOISE_BANDED ? n->ntaps - 1 : 0;
    tp->ndet = p->ndet_total;
    const size_t nd = (size_t)std::max<int64_t>(1, tp->ndet);
    furax_status rc = FURAX_OK;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (rc) return;
        rc = check_cuda(cudaMalloc(ptr, bytes), "template workspace");
    };
    alloc((void **)&tp->mom, sizeof(double2) * nd);
    alloc((void **)&tp->gram, sizeof(double) * 16 * nd);
    alloc((void **)&tp->ginv, sizeof(double) * 16 * nd);
    alloc((void **)&tp->a, sizeof(double) * 4 * nd);
    alloc((void **)&tp->b, sizeof(double) * 4 * nd);
    alloc((void **)&tp->bad, sizeof(unsigned long long));
    if (!rc) rc = check_cuda(cudaMemsetAsync(tp->gram, 0, sizeof(double) * 16 * nd, st), "memset");
    if (!rc) rc = check_cuda(cudaMemsetAsync(tp->a, 0, sizeof(double) * 4 * nd, st), "memset");
    if (!rc) rc = check_cuda(cudaMemsetAsync(tp->b, 0, sizeof(double) * 4 * nd, st), "memset");
    if (!rc) rc = check_cuda(cudaMemsetAsync(tp->bad, 0, sizeof(unsigned long long), st), "memset");
    if (!rc && tp->ndet > 0) {
        tpl_moments_kernel<<<det_grid(tp->ndet), 128, 0, st>>>(tp->ndet, n->view(), tp->halo, tp->mom);
        if (p->n_tiles > 0)
            tpl_gram_kernel<<<(unsigned)p->n_tiles, FT, 0, st>>>(p->d_tiles, p->d_obs, n->view(), tp->view(), tp->gram);
        tpl_invert_kernel<<<det_grid(tp->ndet), 128, 0, st>>>(tp->ndet, order, tp->gram, tp->ginv, tp->bad);
        count_launches(3);
        rc = check_launch("template setup");
    }
    unsigned long long bad = 0;
    if (!rc) rc = check_cuda(cudaMemcpyAsync(&bad, tp->bad, sizeof bad, cudaMemcpyDeviceToHost, st), "read status");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "template setup");
    if (!rc && bad)
        rc = set_error(FURAX_EBADINPUT, "T^T W T is not positive definite for detector %llu", bad - 1);
    if (!rc && order <= 2) rc = build_aug_layout(tp, st);
    if (rc) { templates_destroy(tp); return rc; }
    *out = tp;
    return FURAX_OK;
}

}  // namespace fx
