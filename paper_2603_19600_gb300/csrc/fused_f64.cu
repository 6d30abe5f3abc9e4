// Fused tile kernels of the map-making operator (Furax paper: the estimator
// A = (H.T @ N.I @ H).I @ H.T @ N.I in the Software Design listing, with the block
// decomposition P^T N^-1 P = sum_i P_i^T N_i^-1 P_i of "Algebraic reductions").
//
// One CTA owns one tile: one detector, TILE consecutive samples. It
//   1. gathers the projected map P x for the tile plus a 63-sample halo on each side into
//      shared memory (samples outside the detector stream are zeros: finite section),
//   2. applies N^-1 (white scale, or the 127-term symmetric band, register-blocked),
//   3. scatters y (1, cos 2psi, sin 2psi) into per-pixel accumulators with L2 reductions.
// The time-ordered data never leaves the SM. The same skeleton gives the standalone N^-1,
// the right-hand side P^T N^-1 d and chi^2 with its gradients.
#include "tile.cuh"

namespace fx {

// ------------------------------------------------------------------------------------
// FP64 fused apply: acc64 += P^T N^-1 P x  (x: FP64 [npix][3], zero on masked pixels).
// Also the FP64 right-hand side when FROM_TOD: acc64 += P^T N^-1 d.
// ------------------------------------------------------------------------------------
template <int MODE, bool BANDED, bool FROM_TOD, typename DT>
__global__ void __launch_bounds__(FT) fused_f64_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                       const double *__restrict__ x, const DT *__restrict__ d,
                                                       double *__restrict__ acc64)
{
    extern __shared__ double dsm[];
    double *xs = dsm;                         // [XS]
    double *taps = xs + XS;                   // [MAXTAPS]
    double *sc = taps + MAXTAPS;              // [CS]
    double *ss = sc + CS;                     // [CS]
    int32_t *spix = reinterpret_cast<int32_t *>(ss + CS);   // [CS]

    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    constexpr int halo = BANDED ? kHalo : 0;
    if constexpr (BANDED) load_taps<double>(nv, gdet, taps);

    const int nload = tl.len + 2 * halo;
    for (int u = threadIdx.x; u < nload; u += FT) {
        const int64_t t = tl.t0 - halo + u;
        double v = 0.0, c = 0.0, s = 0.0;
        int32_t pix = -1;
        if (t >= 0 && t < ob.nsamp) {
            pix = get_sample<MODE, double>(pv, ob, tl.det, t, c, s);
            if constexpr (FROM_TOD) {
                v = (double)d[ob.tod_off + tl.det * ob.nsamp + t];
            } else if (pix >= 0) {
                const double *m = x + 3 * (ob.map_off + pix);
                v = fma(m[2], s, fma(m[1], c, m[0]));
            }
        }
        xs[spos(u)] = v;
        const int core = u - halo;
        if (core >= 0 && core < tl.len) { spix[spos(core)] = pix; sc[spos(core)] = c; ss[spos(core)] = s; }
    }
    __syncthreads();

    const int base = threadIdx.x * FR;
    if (base >= tl.len) return;
    double y[FR];
    if constexpr (BANDED) {
        band_product<double, FR>(xs, taps, base, y);
    } else {
        const double w = white_scale<double>(nv, gdet);
#pragma unroll
        for (int r = 0; r < FR; ++r) y[r] = xs[spos(base + r)] * w;
    }
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        const int k = base + r;
        if (k >= tl.len) break;
        const int32_t pix = spix[spos(k)];
        if (pix < 0) continue;
        const int64_t gp = ob.map_off + pix;
        red_add_f64(acc64 + 3 * gp + 0, y[r]);
        red_add_f64(acc64 + 3 * gp + 1, y[r] * sc[spos(k)]);
        red_add_f64(acc64 + 3 * gp + 2, y[r] * ss[spos(k)]);
    }
}

template <int MODE, bool BANDED, bool FROM_TOD, typename DT>
static furax_status run_f64(const furax_pointing *p, const furax_noise *n, const double *x, const DT *d, double *a64,
                            cudaStream_t st)
{
    return launch_dyn(fused_f64_kernel<MODE, BANDED, FROM_TOD, DT>, (unsigned)p->n_tiles, FT, kF64Smem, st, p->d_tiles,
                      p->view(), n->view(), x, d, a64);
}

template <bool FROM_TOD, typename DT>
static furax_status dispatch_f64(const furax_pointing *p, const furax_noise *n, const double *x, const DT *d,
                                 double *a64, cudaStream_t st)
{
    const bool b = n->kind == FURAX_NOISE_BANDED;
    if (p->mode == FURAX_POINTING_ON_THE_FLY)
        return b ? run_f64<0, true, FROM_TOD, DT>(p, n, x, d, a64, st) : run_f64<0, false, FROM_TOD, DT>(p, n, x, d, a64, st);
    if (p->mode == FURAX_POINTING_CACHE_F32)
        return b ? run_f64<1, true, FROM_TOD, DT>(p, n, x, d, a64, st) : run_f64<1, false, FROM_TOD, DT>(p, n, x, d, a64, st);
    if (p->mode == FURAX_POINTING_CACHE_MIXED)
        return b ? run_f64<3, true, FROM_TOD, DT>(p, n, x, d, a64, st) : run_f64<3, false, FROM_TOD, DT>(p, n, x, d, a64, st);
    return b ? run_f64<2, true, FROM_TOD, DT>(p, n, x, d, a64, st) : run_f64<2, false, FROM_TOD, DT>(p, n, x, d, a64, st);
}

furax_status launch_fused_f64(const furax_pointing *p, const furax_noise *n, const double *x, double *a64,
                              cudaStream_t st)
{
    if (p->n_tiles == 0) return FURAX_OK;
    furax_status rc = dispatch_f64<false, double>(p, n, x, (const double *)nullptr, a64, st);
    if (rc) return rc;
    count_launches(1);
    return check_launch("fused P^T N^-1 P (FP64)");
}

furax_status launch_rhs_f64(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, double *a64,
                            cudaStream_t st)
{
    if (p->n_tiles == 0) return FURAX_OK;
    furax_status rc = d_t == FURAX_F64 ? dispatch_f64<true, double>(p, n, nullptr, (const double *)d, a64, st)
                                       : dispatch_f64<true, float>(p, n, nullptr, (const float *)d, a64, st);
    if (rc) return rc;
    count_launches(1);
    return check_launch("right-hand side P^T N^-1 d");
}

template <int MODE, bool B>
static furax_status prep_f64_mode_band()
{
    furax_status rc = FURAX_OK;
    if (!rc) rc = allow_smem((const void *)fused_f64_kernel<MODE, B, false, double>, kF64Smem);
    if (!rc) rc = allow_smem((const void *)fused_f64_kernel<MODE, B, true, double>, kF64Smem);
    if (!rc) rc = allow_smem((const void *)fused_f64_kernel<MODE, B, true, float>, kF64Smem);
    return rc;
}

furax_status prepare_fused_f64()
{
    furax_status rc = FURAX_OK;
    if (!rc) rc = prep_f64_mode_band<0, true>();
    if (!rc) rc = prep_f64_mode_band<0, false>();
    if (!rc) rc = prep_f64_mode_band<1, true>();
    if (!rc) rc = prep_f64_mode_band<1, false>();
    if (!rc) rc = prep_f64_mode_band<2, true>();
    if (!rc) rc = prep_f64_mode_band<2, false>();
    if (!rc) rc = prep_f64_mode_band<3, true>();
    if (!rc) rc = prep_f64_mode_band<3, false>();
    if (!rc) rc = prepare_fused_df();
    return rc;
}

furax_status prepare_kernels()
{
    static furax_status done = 1;
    if (done == FURAX_OK) return FURAX_OK;
    furax_status rc = prepare_fused_f32();
    if (!rc) rc = prepare_fused_f64();
    done = rc;
    return rc;
}

}  // namespace fx
