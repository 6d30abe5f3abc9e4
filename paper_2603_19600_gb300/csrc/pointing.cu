// Pointing operator kernels: expansion (pixel + weights), P (gather), P^T (scatter-add)
// and the block-Jacobi preconditioner (Furax paper: PointingOperator, Table 3 and
// "Map-making classes"; transpose, Table 1; BJPreconditioner).
//
// Work is cut into tiles of one detector x up to TILE consecutive samples, listed per
// observation, so one launch covers a whole batch of ragged observations.
#include "internal.cuh"
#include "pointing_math.cuh"
#include "atomics.cuh"

namespace fx {

// ------------------------------------------------------------------------------------
// Expansion: pixel and weights for every sample (FP64 recipe), cached or returned.
// ------------------------------------------------------------------------------------
template <typename WT>
__global__ void __launch_bounds__(256) expand_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                     const double *__restrict__ q_bore, const double *__restrict__ q_det,
                                                     const double2 *__restrict__ psi_cs, const double2 *__restrict__ hwp_cs,
                                                     int32_t *__restrict__ pix_out,
                                                     WT *__restrict__ c_out, WT *__restrict__ s_out,
                                                     unsigned long long *__restrict__ n_invalid,
                                                     float *__restrict__ c_lo, float *__restrict__ s_lo)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    const Quat qd = load_quat(q_det, gdet);
    const double2 cs = psi_cs ? psi_cs[gdet] : make_double2(1.0, 0.0);
    int bad = 0;
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
        const int64_t t = tl.t0 + k;
        SampleF64 r = point_f64(load_quat(q_bore, ob.bore_off + t), qd, ob.nside);
        double c = r.c, s = r.s;
        if (hwp_cs && r.pix >= 0) apply_hwp<double>(c, s, hwp_cs[ob.bore_off + t]);
        if (psi_cs && r.pix >= 0) rotate_psi<double>(c, s, cs);
        const int64_t i = ob.tod_off + tl.det * ob.nsamp + t;
        pix_out[i] = r.pix;
        if (c_out) { c_out[i] = (WT)c; s_out[i] = (WT)s; }
        if (c_lo) {  // FP32 correction words: (double)hi + (double)lo == c to ~2^-48
            c_lo[i] = (float)(c - (double)(float)c);
            s_lo[i] = (float)(s - (double)(float)s);
        }
        bad += (r.pix < 0);
    }
    if (n_invalid) {
        bad = __reduce_add_sync(0xffffffffu, bad);
        if ((threadIdx.x & 31) == 0 && bad) atomicAdd(n_invalid, (unsigned long long)bad);
    }
}

furax_status launch_expand(const furax_pointing *p, int32_t *pix, float *c32, float *s32, double *c64, double *s64,
                           unsigned long long *n_invalid, cudaStream_t st, bool, float *c32lo, float *s32lo)
{
    if (p->n_tiles == 0) return FURAX_OK;
    const double2 *cs = p->has_psi ? p->d_psi_cs : nullptr;
    const double2 *hw = p->has_hwp ? p->d_hwp_cs : nullptr;
    if (c64 || (!c32 && !c64))
        expand_kernel<double><<<(unsigned)p->n_tiles, 256, 0, st>>>(p->d_tiles, p->d_obs, p->q_bore, p->q_det, cs, hw,
                                                                    pix, c64, s64, n_invalid, nullptr, nullptr);
    else
        expand_kernel<float><<<(unsigned)p->n_tiles, 256, 0, st>>>(p->d_tiles, p->d_obs, p->q_bore, p->q_det, cs, hw,
                                                                   pix, c32, s32, n_invalid, c32lo, s32lo);
    count_launches(1);
    return check_launch("pointing expansion");
}

// (cos 2 delta, sin 2 delta) per detector; with a half-wave plate the rotation is applied to
// weights that already carry the plate, where it acts with the opposite sign (see apply_hwp).
__global__ void psi_kernel(const double *__restrict__ psi, double2 *__restrict__ cs, int64_t n, int through_hwp)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        double s, c;
        sincos(2.0 * psi[i], &s, &c);
        cs[i] = make_double2(c, through_hwp ? -s : s);
    }
}

// (cos 4w, sin 4w) per boresight sample of the half-wave plate angle w.
__global__ void hwp_kernel(const double *__restrict__ w, double2 *__restrict__ cs, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincos(4.0 * w[i], &s, &c);
        cs[i] = make_double2(c, s);
    }
}

furax_status launch_set_hwp(furax_pointing *p, const double *hwp, cudaStream_t st)
{
    if (!hwp) { p->has_hwp = false; return FURAX_OK; }
    furax_status rc = ensure_ws(p, (void **)&p->d_hwp_cs, sizeof(double2) * std::max<int64_t>(1, p->nbore_total));
    if (rc) return rc;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p->nbore_total + 255) / 256, 16LL * p->n_sm));
    hwp_kernel<<<g, 256, 0, st>>>(hwp, p->d_hwp_cs, p->nbore_total);
    count_launches(1);
    p->has_hwp = true;
    return check_launch("half-wave plate angles");
}

furax_status launch_set_psi(furax_pointing *p, const double *psi, cudaStream_t st)
{
    if (!psi) { p->has_psi = false; return FURAX_OK; }
    int64_t n = p->ndet_total;
    psi_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(psi, p->d_psi_cs, n, p->has_hwp ? 1 : 0);
    count_launches(1);
    p->has_psi = true;
    return check_launch("psi offsets");
}

// ------------------------------------------------------------------------------------
// P: tod = I + Q c + U s
// ------------------------------------------------------------------------------------
template <int MODE, typename T, typename MT, typename TT>
__global__ void __launch_bounds__(256) P_kernel(const Tile *__restrict__ tiles, PointingView pv,
                                                const MT *__restrict__ map, TT *__restrict__ tod)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
        const int64_t t = tl.t0 + k;
        T c, s;
        const int32_t pix = get_sample<MODE, T>(pv, ob, tl.det, t, c, s);
        T v = (T)0;
        if (pix >= 0) {
            const MT *m = map + 3 * (ob.map_off + pix);
            v = (T)m[0] + (T)m[1] * c + (T)m[2] * s;
        }
        tod[ob.tod_off + tl.det * ob.nsamp + t] = convert_bits<TT>(v);
    }
}

template <int MODE>
static void dispatch_P(const furax_pointing *p, const void *map, int map_t, void *tod, int tod_t, cudaStream_t st)
{
    const unsigned g = (unsigned)p->n_tiles;
    const PointingView pv = p->view();
    if (map_t == FURAX_F64 && tod_t == FURAX_F64)
        P_kernel<MODE, double, double, double><<<g, 256, 0, st>>>(p->d_tiles, pv, (const double *)map, (double *)tod);
    else if (map_t == FURAX_F64)
        P_kernel<MODE, double, double, float><<<g, 256, 0, st>>>(p->d_tiles, pv, (const double *)map, (float *)tod);
    else if (tod_t == FURAX_F64)
        P_kernel<MODE, double, float, double><<<g, 256, 0, st>>>(p->d_tiles, pv, (const float *)map, (double *)tod);
    else
        P_kernel<MODE, float, float, float><<<g, 256, 0, st>>>(p->d_tiles, pv, (const float *)map, (float *)tod);
}

furax_status launch_P(const furax_pointing *p, const void *map, int map_t, void *tod, int tod_t, cudaStream_t st)
{
    if (p->n_tiles == 0) return FURAX_OK;
    if (p->mode == FURAX_POINTING_ON_THE_FLY) dispatch_P<0>(p, map, map_t, tod, tod_t, st);
    else if (p->mode == FURAX_POINTING_CACHE_F32) dispatch_P<1>(p, map, map_t, tod, tod_t, st);
    else if (p->mode == FURAX_POINTING_CACHE_MIXED) dispatch_P<3>(p, map, map_t, tod, tod_t, st);
    else dispatch_P<2>(p, map, map_t, tod, tod_t, st);
    count_launches(1);
    return check_launch("pointing apply");
}

// ------------------------------------------------------------------------------------
// P^T: accumulate tod * (1, c, s) per pixel into a workspace, then finalise into the map.
// ------------------------------------------------------------------------------------
template <int MODE, int ACC, typename T, typename TT>
__global__ void __launch_bounds__(256) PT_kernel(const Tile *__restrict__ tiles, PointingView pv,
                                                 const TT *__restrict__ tod, float4 *__restrict__ hi,
                                                 float4 *__restrict__ lo, double *__restrict__ acc64,
                                                 int32_t *__restrict__ hits)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    if constexpr (ACC == FURAX_ACC_F64) {
        // three FP64 sums per sample, issued as whole pixel records by the warp (launched with
        // 256 threads: eight staging areas); warp-uniform trip count
        __shared__ double stage[8][96];
        __shared__ int32_t spx[8][32];
        const int warp = threadIdx.x >> 5;
        double *base = acc64 + 3 * ob.map_off;
        for (int kw = threadIdx.x & ~31; kw < tl.len; kw += blockDim.x) {
            const int k = kw + (threadIdx.x & 31);
            int32_t pix = -1;
            double v[3] = {0.0, 0.0, 0.0};
            if (k < tl.len) {
                const int64_t t = tl.t0 + k;
                T c, s;
                pix = get_sample<MODE, T>(pv, ob, tl.det, t, c, s);
                if (pix >= 0) {
                    const T y = convert_bits<T>(tod[ob.tod_off + tl.det * ob.nsamp + t]);
                    v[0] = (double)y;
                    v[1] = (double)(y * c);
                    v[2] = (double)(y * s);
                }
            }
            red_add_f64_records_warp<3, double>(base, pix, v, stage[warp], spx[warp]);
            if (hits && pix >= 0) red_add_s32(hits + ob.map_off + pix, 1);
        }
        return;
    }
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
        const int64_t t = tl.t0 + k;
        T c, s;
        const int32_t pix = get_sample<MODE, T>(pv, ob, tl.det, t, c, s);
        if (pix < 0) continue;
        const int64_t gp = ob.map_off + pix;
        const T y = convert_bits<T>(tod[ob.tod_off + tl.det * ob.nsamp + t]);
        if constexpr (ACC == FURAX_ACC_F32) {
            red_add_v4(hi + gp, make_float4((float)y, (float)(y * c), (float)(y * s), 0.f));
        } else {
            kahan_add_v4(hi + kKahanStride * gp, lo + kKahanStride * gp,
                         make_float4((float)y, (float)(y * c), (float)(y * s), 0.f));
        }
        if (hits) red_add_s32(hits + gp, 1);
    }
}

// map (+)= accumulator, in the map's dtype.
template <typename MT>
__global__ void PT_finalize_kernel(int acc, const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                                   const double *__restrict__ acc64, MT *__restrict__ map, int64_t npix, int accumulate)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        double v0, v1, v2;
        if (acc == FURAX_ACC_F64) { v0 = acc64[3 * p]; v1 = acc64[3 * p + 1]; v2 = acc64[3 * p + 2]; }
        else {
            const bool k = acc == FURAX_ACC_F32_KAHAN;
            float4 h = hi[k ? kKahanStride * p : p];
            v0 = h.x; v1 = h.y; v2 = h.z;
            if (k) { float4 l = lo[kKahanStride * p]; v0 += l.x; v1 += l.y; v2 += l.z; }
        }
        if (accumulate) { v0 += (double)map[3 * p]; v1 += (double)map[3 * p + 1]; v2 += (double)map[3 * p + 2]; }
        map[3 * p] = (MT)v0; map[3 * p + 1] = (MT)v1; map[3 * p + 2] = (MT)v2;
    }
}

template <int MODE, int ACC>
static void dispatch_PT_acc(const furax_pointing *p, const void *tod, int tod_t, float4 *hi, float4 *lo, double *a64,
                            int32_t *hits, cudaStream_t st)
{
    const unsigned g = (unsigned)p->n_tiles;
    const PointingView pv = p->view();
    if (tod_t == FURAX_F64)
        PT_kernel<MODE, ACC, double, double><<<g, 256, 0, st>>>(p->d_tiles, pv, (const double *)tod, hi, lo, a64, hits);
    else if (ACC == FURAX_ACC_F64)
        PT_kernel<MODE, ACC, double, float><<<g, 256, 0, st>>>(p->d_tiles, pv, (const float *)tod, hi, lo, a64, hits);
    else
        PT_kernel<MODE, ACC, float, float><<<g, 256, 0, st>>>(p->d_tiles, pv, (const float *)tod, hi, lo, a64, hits);
}

template <int MODE>
static void dispatch_PT(const furax_pointing *p, const void *tod, int tod_t, int acc, float4 *hi, float4 *lo,
                        double *a64, int32_t *hits, cudaStream_t st)
{
    if (acc == FURAX_ACC_F64) dispatch_PT_acc<MODE, FURAX_ACC_F64>(p, tod, tod_t, hi, lo, a64, hits, st);
    else if (acc == FURAX_ACC_F32) dispatch_PT_acc<MODE, FURAX_ACC_F32>(p, tod, tod_t, hi, lo, a64, hits, st);
    else dispatch_PT_acc<MODE, FURAX_ACC_F32_KAHAN>(p, tod, tod_t, hi, lo, a64, hits, st);
}

furax_status launch_PT_acc64(const furax_pointing *p, const void *tod, int tod_t, double *acc64, cudaStream_t st)
{
    if (p->n_tiles == 0) return FURAX_OK;
    if (p->mode == FURAX_POINTING_ON_THE_FLY) dispatch_PT<0>(p, tod, tod_t, FURAX_ACC_F64, nullptr, nullptr, acc64, nullptr, st);
    else if (p->mode == FURAX_POINTING_CACHE_F32) dispatch_PT<1>(p, tod, tod_t, FURAX_ACC_F64, nullptr, nullptr, acc64, nullptr, st);
    else if (p->mode == FURAX_POINTING_CACHE_MIXED) dispatch_PT<3>(p, tod, tod_t, FURAX_ACC_F64, nullptr, nullptr, acc64, nullptr, st);
    else dispatch_PT<2>(p, tod, tod_t, FURAX_ACC_F64, nullptr, nullptr, acc64, nullptr, st);
    count_launches(1);
    return check_launch("pointing transpose");
}

furax_status launch_PT(const furax_pointing *p, const void *tod, int tod_t, void *map, int map_t, int acc,
                       int32_t *hits, int accumulate, cudaStream_t st)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    const int64_t np = p->npix_total;
    furax_status rc;
    float4 *hi = nullptr, *lo = nullptr;
    double *a64 = nullptr;
    if (acc == FURAX_ACC_F64) {
        if ((rc = ensure_ws(pm, (void **)&pm->ws_acc64, sizeof(double) * 3 * np))) return rc;
        a64 = pm->ws_acc64;
        if ((rc = check_cuda(cudaMemsetAsync(a64, 0, sizeof(double) * 3 * np, st), "memset"))) return rc;
    } else {
        // room for the interleaved compensated layout (hi[2i], lo[2i] = hi[2i + 1])
        if ((rc = ensure_ws(pm, (void **)&pm->ws_acc_hi, sizeof(float4) * kKahanStride * np))) return rc;
        hi = pm->ws_acc_hi;
        if (acc == FURAX_ACC_F32_KAHAN) lo = hi + 1;
        const size_t words = (acc == FURAX_ACC_F32_KAHAN ? kKahanStride : 1) * (size_t)np;
        if ((rc = check_cuda(cudaMemsetAsync(hi, 0, sizeof(float4) * words, st), "memset"))) return rc;
    }
    if (hits && !accumulate)
        if ((rc = check_cuda(cudaMemsetAsync(hits, 0, sizeof(int32_t) * np, st), "memset"))) return rc;
    if (p->n_tiles > 0) {
        if (p->mode == FURAX_POINTING_ON_THE_FLY) dispatch_PT<0>(p, tod, tod_t, acc, hi, lo, a64, hits, st);
        else if (p->mode == FURAX_POINTING_CACHE_F32) dispatch_PT<1>(p, tod, tod_t, acc, hi, lo, a64, hits, st);
        else if (p->mode == FURAX_POINTING_CACHE_MIXED) dispatch_PT<3>(p, tod, tod_t, acc, hi, lo, a64, hits, st);
        else dispatch_PT<2>(p, tod, tod_t, acc, hi, lo, a64, hits, st);
        count_launches(1);
        if ((rc = check_launch("pointing transpose"))) return rc;
    }
    const unsigned fg = (unsigned)std::min<int64_t>((np + 255) / 256, 16LL * p->n_sm);
    if (map_t == FURAX_F64)
        PT_finalize_kernel<double><<<fg, 256, 0, st>>>(acc, hi, lo, a64, (double *)map, np, accumulate);
    else
        PT_finalize_kernel<float><<<fg, 256, 0, st>>>(acc, hi, lo, a64, (float *)map, np, accumulate);
    count_launches(1);
    return check_launch("pointing transpose finalise");
}

// ------------------------------------------------------------------------------------
// Block-Jacobi: M_p = sum ninv w w^T (6 unique entries), hits; then invert in FP64.
// ------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) bj_accum_kernel(const Tile *__restrict__ tiles, PointingView pv,
                                                       const double *__restrict__ ninv_diag, double *__restrict__ m6,
                                                       int32_t *__restrict__ hits)
{
    // per-warp staging of the six block entries: the warp issues them as whole 48-byte records
    __shared__ double stage[8][32 * 6];
    __shared__ int32_t spix[8][32];
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tl.obs];
    const double w0 = ninv_diag[ob.det_off + tl.det];
    const int warp = threadIdx.x >> 5;
    double *base = m6 + 6 * ob.map_off;
    for (int kw = threadIdx.x & ~31; kw < tl.len; kw += 256) {   // warp-uniform trip count
        const int k = kw + (threadIdx.x & 31);
        double c = 0.0, s = 0.0;
        const int32_t pix = k < tl.len ? get_sample<MODE, double>(pv, ob, tl.det, tl.t0 + k, c, s) : -1;
        const double wc = w0 * c, ws = w0 * s;
        const double v[6] = {w0, wc, ws, wc * c, wc * s, ws * s};
        red_add_f64_records_warp<6, double>(base, pix, v, stage[warp], spix[warp]);
        if (pix >= 0) red_add_s32(hits + ob.map_off + pix, 1);
    }
}

__device__ __forceinline__ double norm1_sym(double a, double b, double c, double d, double e, double f)
{
    double c0 = fabs(a) + fabs(b) + fabs(c);
    double c1 = fabs(b) + fabs(d) + fabs(e);
    double c2 = fabs(c) + fabs(e) + fabs(f);
    return fmax(c0, fmax(c1, c2));
}

// Inverse of the symmetric 3x3 block m = (00,01,02,11,12,22) through its Cholesky factor
// M = L L^T, W = L^-1 by forward substitution, M^-1 = W^T W (explicit round-to-nearest FP64
// operations, no contraction). Returns false if a pivot is not positive: such a block is not
// positive definite to working precision (e.g. a pixel crossed only at one angle), and an
// adjugate/determinant inverse of it would be rounding noise.
__device__ __forceinline__ bool bj_invert3(const double *m, double *inv)
{
    if (!(m[0] > 0.0)) return false;
    const double l11 = __dsqrt_rn(m[0]);
    const double l21 = __ddiv_rn(m[1], l11), l31 = __ddiv_rn(m[2], l11);
    const double p2 = __dsub_rn(m[3], __dmul_rn(l21, l21));
    if (!(p2 > 0.0)) return false;
    const double l22 = __dsqrt_rn(p2);
    const double l32 = __ddiv_rn(__dsub_rn(m[4], __dmul_rn(l31, l21)), l22);
    const double p3 = __dsub_rn(__dsub_rn(m[5], __dmul_rn(l31, l31)), __dmul_rn(l32, l32));
    if (!(p3 > 0.0)) return false;
    const double l33 = __dsqrt_rn(p3);
    const double w11 = __ddiv_rn(1.0, l11), w22 = __ddiv_rn(1.0, l22), w33 = __ddiv_rn(1.0, l33);
    const double w21 = -__ddiv_rn(__dmul_rn(l21, w11), l22);
    const double w32 = -__ddiv_rn(__dmul_rn(l32, w22), l33);
    const double w31 = -__ddiv_rn(__dadd_rn(__dmul_rn(l31, w11), __dmul_rn(l32, w21)), l33);
    inv[0] = __dadd_rn(__dadd_rn(__dmul_rn(w11, w11), __dmul_rn(w21, w21)), __dmul_rn(w31, w31));
    inv[1] = __dadd_rn(__dmul_rn(w21, w22), __dmul_rn(w31, w32));
    inv[2] = __dmul_rn(w31, w33);
    inv[3] = __dadd_rn(__dmul_rn(w22, w22), __dmul_rn(w32, w32));
    inv[4] = __dmul_rn(w32, w33);
    inv[5] = __dmul_rn(w33, w33);
    return true;
}

// In place: m6 holds M on entry and M^-1 (0 where invalid) on exit. Valid iff hits >= 3, the
// block is positive definite (Cholesky pivots > 0) and rcond = 1/(|M|_1 |M^-1|_1) >= rcond_min.
__global__ void bj_invert_kernel(double *__restrict__ m6, const int32_t *__restrict__ hits, uint8_t *__restrict__ valid,
                                 double *__restrict__ rcond, int64_t npix, double rcond_min)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        double *m = m6 + 6 * p;
        double mm[6] = {m[0], m[1], m[2], m[3], m[4], m[5]};
        double rc = 0.0, v[6] = {0, 0, 0, 0, 0, 0};
        bool ok = hits[p] >= 3 && bj_invert3(mm, v);
        if (ok) {
            rc = 1.0 / (norm1_sym(mm[0], mm[1], mm[2], mm[3], mm[4], mm[5]) * norm1_sym(v[0], v[1], v[2], v[3], v[4], v[5]));
            ok = rc >= rcond_min;
        }
        for (int k = 0; k < 6; ++k) m[k] = ok ? v[k] : 0.0;
        valid[p] = ok ? 1 : 0;
        if (rcond) rcond[p] = rc;
    }
}

furax_status launch_bj(const furax_pointing *p, const furax_noise *n, double rcond_min, double *blocks_inv,
                       uint8_t *valid, int32_t *hits, double *rcond, cudaStream_t st, const AllReduce &ar)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    const int64_t np = p->npix_total;
    furax_status rc;
    int32_t *h = hits;
    if (!h) {
        if ((rc = ensure_ws(pm, (void **)&pm->ws_hits, sizeof(int32_t) * np))) return rc;
        h = pm->ws_hits;
    }
    if ((rc = check_cuda(cudaMemsetAsync(blocks_inv, 0, sizeof(double) * 6 * np, st), "memset"))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(h, 0, sizeof(int32_t) * np, st), "memset"))) return rc;
    if (p->n_tiles > 0) {
        const unsigned g = (unsigned)p->n_tiles;
        const PointingView pv = p->view();
        if (p->mode == FURAX_POINTING_ON_THE_FLY)
            bj_accum_kernel<0><<<g, 256, 0, st>>>(p->d_tiles, pv, n->diag, blocks_inv, h);
        else if (p->mode == FURAX_POINTING_CACHE_F32)
            bj_accum_kernel<1><<<g, 256, 0, st>>>(p->d_tiles, pv, n->diag, blocks_inv, h);
        else if (p->mode == FURAX_POINTING_CACHE_MIXED)
            bj_accum_kernel<3><<<g, 256, 0, st>>>(p->d_tiles, pv, n->diag, blocks_inv, h);
        else
            bj_accum_kernel<2><<<g, 256, 0, st>>>(p->d_tiles, pv, n->diag, blocks_inv, h);
        count_launches(1);
        if ((rc = check_launch("preconditioner accumulation"))) return rc;
    }
    // detector sharding: the blocks and hits of every process's detectors, before the inversion
    if (ar.on() && ((rc = ar(blocks_inv, 6 * np, FURAX_REDUCE_F64, st)) || (rc = ar(h, np, FURAX_REDUCE_I32, st))))
        return rc;
    const unsigned fg = (unsigned)std::min<int64_t>((np + 255) / 256, 16LL * p->n_sm);
    bj_invert_kernel<<<fg, 256, 0, st>>>(blocks_inv, h, valid, rcond, np, rcond_min);
    count_launches(1);
    return check_launch("preconditioner inversion");
}

}  // namespace fx
