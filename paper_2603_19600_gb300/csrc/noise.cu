// Standalone noise weighting N^-1 (HomothetyOperator / SymmetricBandToeplitzOperator,
// Table 2 of the Furax paper) and chi^2 = (d - P m)^T N^-1 (d - P m) with its gradients
// with respect to the map and the per-detector polarisation-angle offsets (the paper's
// differentiability, "Summary"). Same tile skeleton as the fused operator.
#include "tile.cuh"
#include "dfloat.cuh"

namespace fx {

// ------------------------------------------------------------------------------------
// Standalone N^-1 on a TOD (white or banded), FP32 or FP64.
// ------------------------------------------------------------------------------------
template <typename T, bool BANDED>
__global__ void __launch_bounds__(FT) ninv_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                  NoiseView nv, const T *__restrict__ in, T *__restrict__ out)
{
    __shared__ T xs[BANDED ? XS : 1];
    __shared__ T taps[MAXTAPS];
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    const int64_t row = ob.tod_off + tl.det * ob.nsamp;
    if constexpr (!BANDED) {
        const T w = white_scale<T>(nv, gdet);
        for (int k = threadIdx.x; k < tl.len; k += FT) out[row + tl.t0 + k] = in[row + tl.t0 + k] * w;
        return;
    } else {
        load_taps<T>(nv, gdet, taps);
        const int nload = tl.len + 2 * kHalo;
        for (int u = threadIdx.x; u < nload; u += FT) {
            const int64_t t = tl.t0 - kHalo + u;
            xs[spos(u)] = (t >= 0 && t < ob.nsamp) ? in[row + t] : T(0);
        }
        __syncthreads();
        const int base = threadIdx.x * FR;
        if (base >= tl.len) return;
        T y[FR];
        band_product<T, FR>(xs, taps, base, y);
#pragma unroll
        for (int r = 0; r < FR; ++r)
            if (base + r < tl.len) out[row + tl.t0 + base + r] = y[r];
    }
}

furax_status launch_ninv(const furax_noise *n, const void *in, void *out, int dtype, cudaStream_t st)
{
    if (long_band(n)) return launch_ninv_fft(n, in, out, dtype, st);
    if (n->n_tiles == 0) return FURAX_OK;
    const unsigned g = (unsigned)n->n_tiles;
    const NoiseView nv = n->view();
    const bool b = n->kind == FURAX_NOISE_BANDED;
    if (dtype == FURAX_F64) {
        if (b) ninv_kernel<double, true><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, nv, (const double *)in, (double *)out);
        else ninv_kernel<double, false><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, nv, (const double *)in, (double *)out);
    } else {
        if (b) ninv_kernel<float, true><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, nv, (const float *)in, (float *)out);
        else ninv_kernel<float, false><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, nv, (const float *)in, (float *)out);
    }
    count_launches(1);
    return check_launch("N^-1 apply");
}

// ------------------------------------------------------------------------------------
// chi^2 = r^T N^-1 r, r = d - P m; grad_map -= 2 P^T N^-1 r; grad_psi -= 2 sum (N^-1 r) 2 (U c - Q s).
// T is the precision of r and N^-1 r; all sums are FP64.
// ------------------------------------------------------------------------------------
template <int MODE, typename T, bool BANDED, typename DT>
__global__ void __launch_bounds__(FT) chi2_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                  const DT *__restrict__ d, const double *__restrict__ m,
                                                  double *__restrict__ chi2, double *__restrict__ grad_map,
                                                  double *__restrict__ grad_psi)
{
    extern __shared__ double csm[];
    double *red = csm;                         // [2][FT/32]
    T *xs = reinterpret_cast<T *>(red + 2 * (FT / 32));   // [XS]
    T *taps = xs + XS;                         // [MAXTAPS]
    T *sc = taps + MAXTAPS;                    // [CS]
    T *ss = sc + CS;                           // [CS]
    int32_t *spix = reinterpret_cast<int32_t *>(ss + CS);   // [CS]

    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    const int64_t row = ob.tod_off + tl.det * ob.nsamp;
    constexpr int halo = BANDED ? kHalo : 0;
    if constexpr (BANDED) load_taps<T>(nv, gdet, taps);
    const int nload = tl.len + 2 * halo;
    for (int u = threadIdx.x; u < nload; u += FT) {
        const int64_t t = tl.t0 - halo + u;
        T v = T(0), c = T(0), s = T(0);
        int32_t pix = -1;
        if (t >= 0 && t < ob.nsamp) {
            pix = get_sample<MODE, T>(pv, ob, tl.det, t, c, s);
            T model = T(0);
            if (pix >= 0) {
                const double *mm = m + 3 * (ob.map_off + pix);
                model = (T)mm[0] + (T)mm[1] * c + (T)mm[2] * s;
            }
            v = (T)d[row + t] - model;
        }
        xs[spos(u)] = v;
        const int core = u - halo;
        if (core >= 0 && core < tl.len) { spix[spos(core)] = pix; sc[spos(core)] = c; ss[spos(core)] = s; }
    }
    __syncthreads();

    double part_chi2 = 0.0, part_psi = 0.0;
    // d(weights)/d delta = 2 (-s, c), or its opposite when a half-wave plate reflects the weights
    const double psi_sign = ob.hwp ? -1.0 : 1.0;
    const int base = threadIdx.x * FR;
    if (base < tl.len) {
        T y[FR];
        if constexpr (BANDED) {
            band_product<T, FR>(xs, taps, base, y);
        } else {
            const T w = white_scale<T>(nv, gdet);
#pragma unroll
            for (int r = 0; r < FR; ++r) y[r] = xs[spos(base + r)] * w;
        }
#pragma unroll
        for (int r = 0; r < FR; ++r) {
            const int k = base + r;
            if (k >= tl.len) break;
            const double nr = (double)y[r];
            part_chi2 += (double)xs[spos(k + halo)] * nr;
            const int32_t pix = spix[spos(k)];
            if (pix < 0) continue;
            const double c = (double)sc[spos(k)], s = (double)ss[spos(k)];
            const int64_t gp = ob.map_off + pix;
            const double *mm = m + 3 * gp;
            part_psi += nr * 2.0 * (mm[2] * c - mm[1] * s) * psi_sign;
            if (grad_map) {
                red_add_f64(grad_map + 3 * gp + 0, -2.0 * nr);
                red_add_f64(grad_map + 3 * gp + 1, -2.0 * nr * c);
                red_add_f64(grad_map + 3 * gp + 2, -2.0 * nr * s);
            }
        }
    }
    // block reduction (fixed order within the block)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        part_chi2 += __shfl_down_sync(0xffffffffu, part_chi2, o);
        part_psi += __shfl_down_sync(0xffffffffu, part_psi, o);
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = part_chi2; red[FT / 32 + (threadIdx.x >> 5)] = part_psi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < FT / 32; ++w) { a += red[w]; b += red[FT / 32 + w]; }
        red_add_f64(chi2 + tl.obs, a);
        if (grad_psi) red_add_f64(grad_psi + gdet, -2.0 * b);
    }
}

// ------------------------------------------------------------------------------------
// The same in FP32 (precision FURAX_F32) with no FP64 instruction per sample in the cached modes:
// the map is read as FP32 (packed once per call), FP64 weights and data are rounded from their
// encodings, each thread's partial sums of chi^2 and of the angle gradient are FP32 over its
// samples and FP64 across threads, and the map gradient's three FP64 sums per sample are issued
// as whole pixel records by the warp (FP32 values widened by cvt).
// ------------------------------------------------------------------------------------
__global__ void pack_map_f32_kernel(const double *__restrict__ m, float4 *__restrict__ m32, int64_t np)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x)
        m32[i] = make_float4((float)m[3 * i], (float)m[3 * i + 1], (float)m[3 * i + 2], 0.f);
}

template <int MODE>
__device__ __forceinline__ int32_t sample_f32(const PointingView &pv, const ObsInfo &ob, int32_t det, int64_t t,
                                              float2 csf, float &c, float &s)
{
    if constexpr (MODE == 0) {
        return get_sample<0, float>(pv, ob, det, t, c, s);   // the exact recipe runs in FP64 anyway
    } else {
        const int64_t i = ob.tod_off + det * ob.nsamp + t;
        const int32_t pix = pv.pix[i];
        if constexpr (MODE == 2) { c = f64_to_f32_bits(pv.c64[i]); s = f64_to_f32_bits(pv.s64[i]); }
        else { c = pv.c32[i]; s = pv.s32[i]; }
        if (pv.psi_cs && pix >= 0) rotate_psi_f(c, s, csf.x, csf.y);
        return pix;
    }
}

template <typename DT>
__device__ __forceinline__ float data_f32(DT v)
{
    if constexpr (sizeof(DT) == 8) return f64_to_f32_bits(v);
    else return v;
}

template <int MODE, bool BANDED, typename DT>
__global__ void __launch_bounds__(FT) chi2_f32_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                      const DT *__restrict__ d, const float4 *__restrict__ m32,
                                                      double *__restrict__ chi2, double *__restrict__ grad_map,
                                                      double *__restrict__ grad_psi)
{
    extern __shared__ float fsm[];
    float *xs = fsm;                      // [XS] r = d - P m over the tile and halos
    float *taps = xs + XS;                // [MAXTAPS]
    float *ys = taps + MAXTAPS;           // [CS] N^-1 r of the core samples
    __shared__ double red[2][FT / 32];
    __shared__ float xv[FT / 32][96];
    __shared__ int32_t xp[FT / 32][32];

    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    const int64_t row = ob.tod_off + tl.det * ob.nsamp;
    constexpr int halo = BANDED ? kHalo : 0;
    if constexpr (BANDED) load_taps<float>(nv, gdet, taps);
    float2 csf = make_float2(1.f, 0.f);
    if (pv.psi_cs) csf = make_float2((float)pv.psi_cs[gdet].x, (float)pv.psi_cs[gdet].y);
    const int nload = tl.len + 2 * halo;
    for (int u = threadIdx.x; u < nload; u += FT) {
        const int64_t t = tl.t0 - halo + u;
        float v = 0.f;
        if (t >= 0 && t < ob.nsamp) {
            float c = 0.f, s = 0.f;
            const int32_t pix = sample_f32<MODE>(pv, ob, tl.det, t, csf, c, s);
            float model = 0.f;
            if (pix >= 0) {
                const float4 mm = m32[ob.map_off + pix];
                model = mm.x + mm.y * c + mm.z * s;
            }
            v = data_f32(d[row + t]) - model;
        }
        xs[spos(u)] = v;
    }
    __syncthreads();

    float part_chi2 = 0.f;
    const int base = threadIdx.x * FR;
    if (base < tl.len) {
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
            if (base + r >= tl.len) break;
            part_chi2 += xs[spos(base + r + halo)] * y[r];
            ys[spos(base + r)] = y[r];
        }
    }
    __syncthreads();

    // d(weights)/d delta = 2 (-s, c), or its opposite when a half-wave plate reflects the weights
    float part_psi = 0.f;
    double *rec = grad_map ? grad_map + 3 * ob.map_off : nullptr;
    for (int kw = threadIdx.x & ~31; kw < tl.len; kw += FT) {   // warp-uniform trip count
        const int k = kw + (threadIdx.x & 31);
        float c = 0.f, s = 0.f, nr = 0.f;
        const int32_t pix = k < tl.len ? sample_f32<MODE>(pv, ob, tl.det, tl.t0 + k, csf, c, s) : -1;
        if (pix >= 0) {
            nr = ys[spos(k)];
            const float4 mm = m32[ob.map_off + pix];
            part_psi += nr * (mm.z * c - mm.y * s);
        }
        if (rec) {
            const float g = -2.f * nr;
            const float v[3] = {g, g * c, g * s};
            red_add_f64_records_warp<3, float>(rec, pix, v, xv[threadIdx.x >> 5], xp[threadIdx.x >> 5]);
        }
    }
    // block reduction (fixed order within the block), in FP64 across threads
    double a = part_chi2, b = (ob.hwp ? -2.0 : 2.0) * (double)part_psi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < FT / 32; ++w) { sa += red[0][w]; sb += red[1][w]; }
        red_add_f64(chi2 + tl.obs, sa);
        if (grad_psi) red_add_f64(grad_psi + gdet, -2.0 * sb);
    }
}

template <int MODE, typename DT>
static furax_status dispatch_chi2_f32(const furax_pointing *p, const furax_noise *n, const DT *d, const double *m,
                                      double *chi2, double *gm, double *gp, cudaStream_t st)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    furax_status rc;
    const int64_t np = p->npix_total;
    if ((rc = ensure_ws(pm, (void **)&pm->ws_map32, sizeof(float4) * np))) return rc;
    const unsigned pg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, 8LL * p->n_sm));
    pack_map_f32_kernel<<<pg, 256, 0, st>>>(m, pm->ws_map32, np);
    count_launches(1);
    if ((rc = check_launch("FP32 copy of the map"))) return rc;
    const unsigned g = (unsigned)p->n_tiles;
    const size_t smem = sizeof(float) * (XS + MAXTAPS + CS);
    if (n->kind == FURAX_NOISE_BANDED)
        return launch_dyn(chi2_f32_kernel<MODE, true, DT>, g, FT, smem, st, p->d_tiles, p->view(), n->view(), d,
                          pm->ws_map32, chi2, gm, gp);
    return launch_dyn(chi2_f32_kernel<MODE, false, DT>, g, FT, smem, st, p->d_tiles, p->view(), n->view(), d,
                      pm->ws_map32, chi2, gm, gp);
}

template <int MODE, typename T, typename DT>
static furax_status dispatch_chi2_t(const furax_pointing *p, const furax_noise *n, const DT *d, const double *m,
                                    double *chi2, double *gm, double *gp, cudaStream_t st)
{
    const unsigned g = (unsigned)p->n_tiles;
    const size_t smem = sizeof(double) * 2 * (FT / 32) + sizeof(T) * (XS + MAXTAPS + 2 * CS) + sizeof(int32_t) * CS;
    if (n->kind == FURAX_NOISE_BANDED)
        return launch_dyn(chi2_kernel<MODE, T, true, DT>, g, FT, smem, st, p->d_tiles, p->view(), n->view(), d, m, chi2,
                          gm, gp);
    return launch_dyn(chi2_kernel<MODE, T, false, DT>, g, FT, smem, st, p->d_tiles, p->view(), n->view(), d, m, chi2, gm,
                      gp);
}

template <int MODE>
static furax_status dispatch_chi2(const furax_pointing *p, const furax_noise *n, const void *d, int d_t,
                                  const double *m, double *chi2, double *gm, double *gp, int precision, cudaStream_t st)
{
    if (precision == FURAX_F64) {
        if (d_t == FURAX_F64) return dispatch_chi2_t<MODE, double, double>(p, n, (const double *)d, m, chi2, gm, gp, st);
        return dispatch_chi2_t<MODE, double, float>(p, n, (const float *)d, m, chi2, gm, gp, st);
    }
    if (d_t == FURAX_F64) return dispatch_chi2_f32<MODE, double>(p, n, (const double *)d, m, chi2, gm, gp, st);
    return dispatch_chi2_f32<MODE, float>(p, n, (const float *)d, m, chi2, gm, gp, st);
}

furax_status launch_chi2_grad(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, const double *m,
                              double *chi2, double *grad_map, double *grad_psi, int precision, cudaStream_t st)
{
    furax_status rc;
    if ((rc = check_cuda(cudaMemsetAsync(chi2, 0, sizeof(double) * p->n_obs, st), "memset"))) return rc;
    if (grad_map && (rc = check_cuda(cudaMemsetAsync(grad_map, 0, sizeof(double) * 3 * p->npix_total, st), "memset")))
        return rc;
    if (grad_psi && (rc = check_cuda(cudaMemsetAsync(grad_psi, 0, sizeof(double) * p->ndet_total, st), "memset")))
        return rc;
    if (p->n_tiles == 0) return FURAX_OK;
    if (precision == FURAX_PREC_F32X2) return launch_chi2_df(p, n, d, d_t, m, chi2, grad_map, grad_psi, st);
    if (p->mode == FURAX_POINTING_ON_THE_FLY) rc = dispatch_chi2<0>(p, n, d, d_t, m, chi2, grad_map, grad_psi, precision, st);
    else if (p->mode == FURAX_POINTING_CACHE_F32)
        rc = dispatch_chi2<1>(p, n, d, d_t, m, chi2, grad_map, grad_psi, precision, st);
    else if (p->mode == FURAX_POINTING_CACHE_MIXED)
        rc = dispatch_chi2<3>(p, n, d, d_t, m, chi2, grad_map, grad_psi, precision, st);
    else rc = dispatch_chi2<2>(p, n, d, d_t, m, chi2, grad_map, grad_psi, precision, st);
    if (rc) return rc;
    count_launches(1);
    return check_launch("chi2 and gradients");
}

}  // namespace fx
