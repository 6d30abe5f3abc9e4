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
#include "pointing_fast.cuh"

namespace fx {

// ------------------------------------------------------------------------------------
// FP32 fused apply: acc += P^T N^-1 P x32  (x32: padded FP32 map, zero on masked pixels)
// ------------------------------------------------------------------------------------
// Samples of one tile (with halos) handled by each thread in the gather phases.
constexpr int kPerThread = (TILE + 2 * kHalo + FT - 1) / FT;

// bm (on the fly): boresight matrices of the certified FP32 pointing (pointing_fast.cuh).
template <int MODE, int ACC, bool BANDED>
__global__ void __launch_bounds__(FT, 3) fused_f32_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                          const float4 *__restrict__ x32, float4 *__restrict__ acc_hi,
                                                          float4 *__restrict__ acc_lo, double *__restrict__ acc64,
                                                          const float *__restrict__ bm)
{
    extern __shared__ float fsm[];
    float *xs = fsm;                           // [XS] projected map P x over the tile and its halos
    float *taps = xs + XS;                     // [MAXTAPS]
    float *sc = taps + MAXTAPS;                // [XS] cos 2psi of the same samples
    float *ss = sc + XS;                       // [XS] sin 2psi
    int32_t *spix = reinterpret_cast<int32_t *>(ss + XS);   // [XS] pixel (-1: none)

    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    constexpr int halo = BANDED ? kHalo : 0;
    if constexpr (BANDED) load_taps<float>(nv, gdet, taps);
    const int nload = tl.len + 2 * halo;
    const int64_t t_first = tl.t0 - halo;

    if constexpr (MODE == FURAX_POINTING_CACHE_F32) {
        // Phase A: every load of the thread's samples is issued before any is used, so each
        // thread keeps ~50 loads in flight (the pointing stream is read once: evict-first).
        const int64_t row = ob.tod_off + tl.det * ob.nsamp;
        int32_t pk[kPerThread];
        float ck[kPerThread], sk[kPerThread];
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int u = threadIdx.x + k * FT;
            const int64_t t = t_first + u;
            pk[k] = -1; ck[k] = 0.f; sk[k] = 0.f;
            if (u < nload && t >= 0 && t < ob.nsamp) {
                pk[k] = __ldcs(pv.pix + row + t);
                ck[k] = __ldcs(pv.c32 + row + t);
                sk[k] = __ldcs(pv.s32 + row + t);
            }
        }
        if (pv.psi_cs) {
            const double2 cs = pv.psi_cs[gdet];
#pragma unroll
            for (int k = 0; k < kPerThread; ++k) rotate_psi<float>(ck[k], sk[k], cs);
        }
        // Phase B: the map gathers (L2), again all issued before use.
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int u = threadIdx.x + k * FT;
            if (u < nload) {
                float v = 0.f;
                if (pk[k] >= 0) {
                    const float4 m = __ldg(x32 + ob.map_off + pk[k]);
                    v = fmaf(m.z, sk[k], fmaf(m.y, ck[k], m.x));
                }
                xs[spos(u)] = v;
                spix[spos(u)] = pk[k];
                sc[spos(u)] = ck[k];
                ss[spos(u)] = sk[k];
            }
        }
    } else if constexpr (MODE == FURAX_POINTING_ON_THE_FLY) {
        // The pointing of the tile and its halos on the FP32 units, certified (pointing_fast.cuh);
        // the samples the margins cannot certify take the exact FP64 recipe densely afterwards;
        // then the map gathers. Pixels equal the recipe's; weights are FP32 (as in the FP32 cache).
        __shared__ float sdet[12];
        __shared__ int sdet_ok, qn;
        if (threadIdx.x == 0) {
            sdet_ok = det_axes_df(load_quat(pv.q_det, gdet), sdet);
            qn = 0;
        }
        __syncthreads();
        float dh[3], dl[3], oh[3], ol[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) { dh[k] = sdet[k]; dl[k] = sdet[3 + k]; oh[k] = sdet[6 + k]; ol[k] = sdet[9 + k]; }
        float2 psf = make_float2(1.f, 0.f);   // the detector's offset rotation, rounded once
        if (pv.psi_cs) psf = make_float2((float)pv.psi_cs[gdet].x, (float)pv.psi_cs[gdet].y);
        int32_t *queue = reinterpret_cast<int32_t *>(xs);   // xs is written only after the pointing
        for (int u = threadIdx.x; u < nload; u += FT) {
            const int64_t t = t_first + u;
            float c = 0.f, s = 0.f;
            int32_t pix = -1;
            if (t >= 0 && t < ob.nsamp) {
                if (sdet_ok &&
                    certified_sample(bm + 18 * (ob.bore_off + t), dh, dl, oh, ol, (int32_t)ob.nside, pix, c, s)) {
                    if (pv.hwp_cs) apply_hwp<float>(c, s, pv.hwp_cs[ob.bore_off + t]);
                    if (pv.psi_cs) rotate_psi_f(c, s, psf.x, psf.y);
                } else {
                    pix = -1;
                    queue[atomicAdd(&qn, 1)] = u;
                }
            }
            spix[spos(u)] = pix;
            sc[spos(u)] = c;
            ss[spos(u)] = s;
        }
        __syncthreads();
        // the exact recipe as in the cache fill: FP64 weights (half-wave plate in FP64) rounded to
        // FP32, then the offset rotation in FP32 like every other sample
        const int nq = qn;
        const Quat qd = load_quat(pv.q_det, gdet);
        for (int j = threadIdx.x; j < nq; j += FT) {
            const int u = queue[j];
            const int64_t t = t_first + u;
            const SampleF64 r = point_f64(load_quat(pv.q_bore, ob.bore_off + t), qd, ob.nside);
            double cd = r.c, sd = r.s;
            if (pv.hwp_cs && r.pix >= 0) apply_hwp<double>(cd, sd, pv.hwp_cs[ob.bore_off + t]);
            float c = (float)cd, s = (float)sd;
            if (pv.psi_cs && r.pix >= 0) rotate_psi_f(c, s, psf.x, psf.y);
            spix[spos(u)] = r.pix;
            sc[spos(u)] = c;
            ss[spos(u)] = s;
        }
        __syncthreads();
        for (int u = threadIdx.x; u < nload; u += FT) {
            const int32_t pix = spix[spos(u)];
            float v = 0.f;
            if (pix >= 0) {
                const float4 m = __ldg(x32 + ob.map_off + pix);
                v = fmaf(m.z, ss[spos(u)], fmaf(m.y, sc[spos(u)], m.x));
            }
            xs[spos(u)] = v;
        }
    } else {
        for (int u = threadIdx.x; u < nload; u += FT) {
            const int64_t t = t_first + u;
            float v = 0.f, c = 0.f, s = 0.f;
            int32_t pix = -1;
            if (t >= 0 && t < ob.nsamp) {
                pix = get_sample<MODE, float>(pv, ob, tl.det, t, c, s);
                if (pix >= 0) {
                    const float4 m = __ldg(x32 + ob.map_off + pix);
                    v = fmaf(m.z, s, fmaf(m.y, c, m.x));
                }
            }
            xs[spos(u)] = v;
            spix[spos(u)] = pix;
            sc[spos(u)] = c;
            ss[spos(u)] = s;
        }
    }
    __syncthreads();

    // Phase C: N^-1 on the tile, then the scatter of y (1, c, s).
    const int base = threadIdx.x * FR;
    if (base >= tl.len) return;
    float y[FR];
    if constexpr (BANDED) {
        band_product<float, FR>(xs, taps, base, y);
    } else {
        const float w = white_scale<float>(nv, gdet);
#pragma unroll
        for (int r = 0; r < FR; ++r) y[r] = xs[spos(base + r)] * w;
    }
#pragma unroll
    for (int r = 0; r < FR; ++r) {
        const int k = base + r;
        if (k >= tl.len) break;
        const int u = k + halo;
        const int32_t pix = spix[spos(u)];
        if (pix < 0) continue;
        const float c = sc[spos(u)], s = ss[spos(u)];
        const int64_t gp = ob.map_off + pix;
        const float4 v = make_float4(y[r], y[r] * c, y[r] * s, 0.f);
        if constexpr (ACC == FURAX_ACC_F32) red_add_v4(acc_hi + gp, v);
        else if constexpr (ACC == FURAX_ACC_F32_KAHAN)
            kahan_add_v4(acc_hi + kKahanStride * gp, acc_lo + kKahanStride * gp, v);
        else {
            red_add_f64(acc64 + 3 * gp + 0, (double)v.x);
            red_add_f64(acc64 + 3 * gp + 1, (double)v.y);
            red_add_f64(acc64 + 3 * gp + 2, (double)v.z);
        }
    }
}

template <int MODE, bool BANDED>
static furax_status dispatch_fused_f32_acc(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc,
                                           float4 *hi, float4 *lo, double *a64, cudaStream_t st)
{
    const unsigned g = (unsigned)p->n_tiles;
    const PointingView pv = p->view();
    const NoiseView nv = n->view();
    const float *bm = MODE == FURAX_POINTING_ON_THE_FLY ? p->ws_bore_m : nullptr;
    if (acc == FURAX_ACC_F32)
        return launch_dyn(fused_f32_kernel<MODE, FURAX_ACC_F32, BANDED>, g, FT, kF32Smem, st, p->d_tiles, pv, nv, x32,
                          hi, lo, a64, bm);
    if (acc == FURAX_ACC_F32_KAHAN)
        return launch_dyn(fused_f32_kernel<MODE, FURAX_ACC_F32_KAHAN, BANDED>, g, FT, kF32Smem, st, p->d_tiles, pv, nv,
                          x32, hi, lo, a64, bm);
    return launch_dyn(fused_f32_kernel<MODE, FURAX_ACC_F64, BANDED>, g, FT, kF32Smem, st, p->d_tiles, pv, nv, x32, hi,
                      lo, a64, bm);
}

template <int MODE>
static furax_status dispatch_fused_f32(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc,
                                       float4 *hi, float4 *lo, double *a64, cudaStream_t st)
{
    if (n->kind == FURAX_NOISE_BANDED) return dispatch_fused_f32_acc<MODE, true>(p, n, x32, acc, hi, lo, a64, st);
    return dispatch_fused_f32_acc<MODE, false>(p, n, x32, acc, hi, lo, a64, st);
}

bool fused_f32_projects_templates(const furax_pointing *p)
{
    return p->mode == FURAX_POINTING_CACHE_F32 || p->mode == FURAX_POINTING_CACHE_MIXED;
}

furax_status launch_fused_f32(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc, float4 *hi,
                              float4 *lo, double *a64, cudaStream_t st, const FusedTpl *ft)
{
    if (p->n_tiles == 0) return FURAX_OK;
    furax_status rc;
    if (ft && !fused_f32_projects_templates(p))
        return set_error(FURAX_EINVAL, "template work is fused only for the cached FP32 pointing");
    if (p->mode == FURAX_POINTING_ON_THE_FLY) {
        // the boresight matrices of the certified pointing, from the handle's current quaternions
        furax_pointing *pm = const_cast<furax_pointing *>(p);
        if ((rc = ensure_ws(pm, (void **)&pm->ws_bore_m, sizeof(float) * 18 * std::max<int64_t>(1, p->nbore_total))))
            return rc;
        const unsigned bg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p->nbore_total + 255) / 256, 16LL * p->n_sm));
        bore_matrix_kernel<<<bg, 256, 0, st>>>(p->q_bore, p->nbore_total, pm->ws_bore_m);
        count_launches(1);
        if ((rc = check_launch("boresight matrices"))) return rc;
        rc = dispatch_fused_f32<0>(p, n, x32, acc, hi, lo, a64, st);
    }
    else if ((p->mode == FURAX_POINTING_CACHE_F32 || p->mode == FURAX_POINTING_CACHE_MIXED) && !ft &&
             sorted_active(p) && !long_band(n))
        rc = launch_fused_sorted(p, n, x32, acc, hi, lo, a64, st);   // pixel-sorted schedule
    else if (p->mode == FURAX_POINTING_CACHE_F32 || p->mode == FURAX_POINTING_CACHE_MIXED)  // FP32 weights: hi
        rc = launch_fused_tma(p, n, x32, acc, hi, lo, a64, st, ft);
    else rc = dispatch_fused_f32<2>(p, n, x32, acc, hi, lo, a64, st);
    if (rc) return rc;
    count_launches(1);
    return check_launch("fused P^T N^-1 P (FP32)");
}

template <int MODE, bool B>
static furax_status prep_f32_mode_band()
{
    furax_status rc = FURAX_OK;
    if (!rc) rc = allow_smem((const void *)fused_f32_kernel<MODE, FURAX_ACC_F32, B>, kF32Smem);
    if (!rc) rc = allow_smem((const void *)fused_f32_kernel<MODE, FURAX_ACC_F32_KAHAN, B>, kF32Smem);
    if (!rc) rc = allow_smem((const void *)fused_f32_kernel<MODE, FURAX_ACC_F64, B>, kF32Smem);
    return rc;
}

furax_status prepare_fused_f32()
{
    furax_status rc = prepare_fused_tma();
    if (!rc) rc = prepare_fused_sorted();
    if (!rc) rc = prep_f32_mode_band<0, true>();
    if (!rc) rc = prep_f32_mode_band<0, false>();
    if (!rc) rc = prep_f32_mode_band<1, true>();
    if (!rc) rc = prep_f32_mode_band<1, false>();
    if (!rc) rc = prep_f32_mode_band<2, true>();
    if (!rc) rc = prep_f32_mode_band<2, false>();
    return rc;
}

}  // namespace fx
