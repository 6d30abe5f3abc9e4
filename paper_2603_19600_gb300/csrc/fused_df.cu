// FP64-accurate normal-equations operator on FP32 units (FURAX_PREC_F32X2).
//
// Same tile skeleton as the FP32/FP64 fused kernels (Furax paper: A = (H.T @ N.I @ H).I @
// H.T @ N.I, Software Design listing). On GB300 the FP64 pipe runs ~70x below the FP32 pipe,
// so the 127-term band product — the only per-sample arithmetic of real size — is computed in
// double-FP32 with a compensated dot product (Ogita, Rump & Oishi 2005, "Accurate sum and dot
// product", algorithm Dot2): every product c_hi x_hi is split exactly into p + e by an FMA,
// the p are summed with Knuth's two-sum (exact error term), and errors, the e and the cross
// terms c_hi x_lo + c_lo x_hi are gathered in a second FP32 word. The result is as accurate as
// an evaluation in twice the FP32 precision (~2^-48) followed by rounding. The projection and
// the per-pixel sums stay in FP64 (a few FP64 operations per sample).
#include "tile.cuh"

namespace fx {

// Exact-error steps: explicit round-to-nearest operations, never contracted.
__device__ __forceinline__ void dot2_step(float ch, float cl, float xh, float xl, float &S, float &E)
{
    const float p = __fmul_rn(ch, xh);
    const float e = __fmaf_rn(ch, xh, -p);             // ch*xh = p + e exactly
    const float s = __fadd_rn(S, p);
    const float bv = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bv)), __fsub_rn(p, bv));   // S + p = s + err exactly
    S = s;
    E = __fmaf_rn(ch, xl, __fmaf_rn(cl, xh, __fadd_rn(E, __fadd_rn(err, e))));
}

// y_t = sum_j c_|j-63| x_{t+j-63} for R consecutive outputs, in double-FP32 (S + E).
template <int R>
__device__ __forceinline__ void band_product_df(const float *__restrict__ xh, const float *__restrict__ xl,
                                                const float *__restrict__ th, const float *__restrict__ tl, int base,
                                                float (&S)[R], float (&E)[R])
{
    float wh[R], wl[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        wh[r] = xh[spos(base + r)];
        wl[r] = xl[spos(base + r)];
        S[r] = 0.f;
        E[r] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < kBand; ++j) {
        const int k = j < kHalo ? kHalo - j : j - kHalo;
        const float ch = th[k], cl = tl[k];
#pragma unroll
        for (int r = 0; r < R; ++r) dot2_step(ch, cl, wh[r], wl[r], S[r], E[r]);
        if (j < kBand - 1) {
#pragma unroll
            for (int r = 0; r < R - 1; ++r) { wh[r] = wh[r + 1]; wl[r] = wl[r + 1]; }
            wh[R - 1] = xh[spos(base + R + j)];
            wl[R - 1] = xl[spos(base + R + j)];
        }
    }
}

__device__ __forceinline__ void split_df(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

constexpr size_t kDfSmem = sizeof(float) * (2 * XS + 2 * MAXTAPS) + sizeof(float2) * 2 * CS + sizeof(int32_t) * CS;

// acc64 += P^T N^-1 P x  (x: FP64 [npix][3], zero on masked pixels), or acc64 += P^T N^-1 d (FROM_TOD).
template <int MODE, bool BANDED, bool FROM_TOD, typename DT>
__global__ void __launch_bounds__(FT, 1) fused_df_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                         const double *__restrict__ x, const DT *__restrict__ d,
                                                         double *__restrict__ acc64)
{
    extern __shared__ __align__(16) float dfsm[];
    float *xh = dfsm;                                  // [XS]
    float *xl = xh + XS;                               // [XS]
    float *th = xl + XS;                               // [MAXTAPS]
    float *tl = th + MAXTAPS;                          // [MAXTAPS]
    float2 *sc = reinterpret_cast<float2 *>(tl + MAXTAPS);   // [CS] (hi, lo) of cos 2psi
    float2 *ss = sc + CS;                              // [CS] (hi, lo) of sin 2psi
    int32_t *spix = reinterpret_cast<int32_t *>(ss + CS);    // [CS]

    const Tile tile = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tile.obs];
    const int64_t gdet = ob.det_off + tile.det;
    constexpr int halo = BANDED ? kHalo : 0;
    if (threadIdx.x < MAXTAPS) {
        double c = 0.0;
        if constexpr (BANDED) c = threadIdx.x < nv.ntaps ? nv.p64[gdet * nv.ntaps + threadIdx.x] : 0.0;
        else c = threadIdx.x == 0 ? nv.p64[gdet] : 0.0;   // white: the single tap 1/sigma^2
        split_df(c, th[threadIdx.x], tl[threadIdx.x]);
    }
    const int nload = tile.len + 2 * halo;
    for (int u = threadIdx.x; u < nload; u += FT) {
        const int64_t t = tile.t0 - halo + u;
        double v = 0.0, c = 0.0, s = 0.0;
        int32_t pix = -1;
        if (t >= 0 && t < ob.nsamp) {
            pix = get_sample<MODE, double>(pv, ob, tile.det, t, c, s);
            if constexpr (FROM_TOD) {
                v = (double)d[ob.tod_off + tile.det * ob.nsamp + t];
            } else if (pix >= 0) {
                const double *m = x + 3 * (ob.map_off + pix);
                v = fma(m[2], s, fma(m[1], c, m[0]));
            }
        }
        split_df(v, xh[spos(u)], xl[spos(u)]);
        const int core = u - halo;
        if (core >= 0 && core < tile.len) {
            float2 cc, sv;
            split_df(c, cc.x, cc.y);
            split_df(s, sv.x, sv.y);
            spix[spos(core)] = pix;
            sc[spos(core)] = cc;
            ss[spos(core)] = sv;
        }
    }
    __syncthreads();

    const int base = threadIdx.x * FR;
    if (base >= tile.len) return;
    float S[FR], E[FR];
    if constexpr (BANDED) {
        band_product_df<FR>(xh, xl, th, tl, base, S, E);
    } else {
#pragma unroll
        for (int r = 0; r < FR; ++r) {
            S[r] = 0.f;
            E[r] = 0.f;
            dot2_step(th[0], tl[0], xh[spos(base + r)], xl[spos(base + r)], S[r], E[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        const int k = base + r;
        if (k >= tile.len) break;
        const int32_t pix = spix[spos(k)];
        if (pix < 0) continue;
        const double y = (double)S[r] + (double)E[r];
        const float2 cc = sc[spos(k)], sv = ss[spos(k)];
        const double c = (double)cc.x + (double)cc.y, s = (double)sv.x + (double)sv.y;
        const int64_t gp = ob.map_off + pix;
        red_add_f64(acc64 + 3 * gp + 0, y);
        red_add_f64(acc64 + 3 * gp + 1, y * c);
        red_add_f64(acc64 + 3 * gp + 2, y * s);
    }
}

template <int MODE, bool BANDED, bool FROM_TOD, typename DT>
static furax_status run_df(const furax_pointing *p, const furax_noise *n, const double *x, const DT *d, double *a64,
                           cudaStream_t st)
{
    return launch_dyn(fused_df_kernel<MODE, BANDED, FROM_TOD, DT>, (unsigned)p->n_tiles, FT, kDfSmem, st, p->d_tiles,
                      p->view(), n->view(), x, d, a64);
}

template <bool FROM_TOD, typename DT>
static furax_status dispatch_df(const furax_pointing *p, const furax_noise *n, const double *x, const DT *d,
                                double *a64, cudaStream_t st)
{
    const bool b = n->kind == FURAX_NOISE_BANDED;
    switch (p->mode) {
    case FURAX_POINTING_ON_THE_FLY:
        return b ? run_df<0, true, FROM_TOD, DT>(p, n, x, d, a64, st) : run_df<0, false, FROM_TOD, DT>(p, n, x, d, a64, st);
    case FURAX_POINTING_CACHE_F32:
        return b ? run_df<1, true, FROM_TOD, DT>(p, n, x, d, a64, st) : run_df<1, false, FROM_TOD, DT>(p, n, x, d, a64, st);
    case FURAX_POINTING_CACHE_MIXED:
        return b ? run_df<3, true, FROM_TOD, DT>(p, n, x, d, a64, st) : run_df<3, false, FROM_TOD, DT>(p, n, x, d, a64, st);
    default:
        return b ? run_df<2, true, FROM_TOD, DT>(p, n, x, d, a64, st) : run_df<2, false, FROM_TOD, DT>(p, n, x, d, a64, st);
    }
}

furax_status launch_fused_df(const furax_pointing *p, const furax_noise *n, const double *x, const void *d, int d_t,
                             double *acc64, cudaStream_t st)
{
    if (p->n_tiles == 0) return FURAX_OK;
    furax_status rc;
    if (!d) rc = dispatch_df<false, double>(p, n, x, (const double *)nullptr, acc64, st);
    else if (d_t == FURAX_F64) rc = dispatch_df<true, double>(p, n, nullptr, (const double *)d, acc64, st);
    else rc = dispatch_df<true, float>(p, n, nullptr, (const float *)d, acc64, st);
    if (rc) return rc;
    count_launches(1);
    return check_launch("double-FP32 P^T N^-1 P");
}

template <int MODE, bool B>
static furax_status prep_df_mode_band()
{
    furax_status rc = FURAX_OK;
    if (!rc) rc = allow_smem((const void *)fused_df_kernel<MODE, B, false, double>, kDfSmem);
    if (!rc) rc = allow_smem((const void *)fused_df_kernel<MODE, B, true, double>, kDfSmem);
    if (!rc) rc = allow_smem((const void *)fused_df_kernel<MODE, B, true, float>, kDfSmem);
    return rc;
}

furax_status prepare_fused_df()
{
    furax_status rc = FURAX_OK;
    if (!rc) rc = prep_df_mode_band<0, true>();
    if (!rc) rc = prep_df_mode_band<0, false>();
    if (!rc) rc = prep_df_mode_band<1, true>();
    if (!rc) rc = prep_df_mode_band<1, false>();
    if (!rc) rc = prep_df_mode_band<2, true>();
    if (!rc) rc = prep_df_mode_band<2, false>();
    if (!rc) rc = prep_df_mode_band<3, true>();
    if (!rc) rc = prep_df_mode_band<3, false>();
    return rc;
}

}  // namespace fx
