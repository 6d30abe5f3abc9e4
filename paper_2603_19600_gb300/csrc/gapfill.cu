// Gap filling by constrained Gaussian realisation, the use the Furax paper gives its symmetric
// band Toeplitz operator besides noise weighting (SymmetricBandToeplitzOperator, Table 2). With N
// the noise covariance (a symmetric band per detector), d the data, v the observed samples, g the
// gaps and n an unconstrained realisation of covariance N (supplied by the caller: the random
// draws of the method),
//     d_g <- n_g + N_gv N_vv^-1 (d_v - n_v),    d_v unchanged.
// N_vv^-1 is applied by conjugate gradients run for every detector at once: the operator is the
// band product (direct, or overlap-save for long bands) between two applications of the mask,
// and each detector keeps its own scalars (per-CTA partial sums reduced into them).
#include "tile.cuh"
#include "dfloat.cuh"

namespace fx {

struct GfDet {
    double rr, rr0, pq, rr_new, alpha, beta;
    int32_t done, iters;
};

__device__ __forceinline__ double cta_sum_d(double v)
{
    __shared__ double red[FT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < FT / 32; ++w) s += red[w];
    return s;
}

__device__ __forceinline__ int64_t tod_index(const ObsInfo &ob, const Tile &tl, int u)
{
    return ob.tod_off + (int64_t)tl.det * ob.nsamp + tl.t0 + u;
}

// r = S (d - n), p = r, y = 0; rr[det] += |r|^2.
template <typename DT>
__global__ void __launch_bounds__(FT) gf_init_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                     const DT *__restrict__ d, const DT *__restrict__ nr,
                                                     const uint8_t *__restrict__ valid, double *__restrict__ y,
                                                     double *__restrict__ r, double *__restrict__ p,
                                                     GfDet *__restrict__ sc)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    double acc = 0.0;
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t i = tod_index(ob, tl, u);
        const double rv = valid[i] ? (double)d[i] - (double)nr[i] : 0.0;
        r[i] = rv;
        p[i] = rv;
        y[i] = 0.0;
        acc += rv * rv;
    }
    acc = cta_sum_d(acc);
    if (threadIdx.x == 0) red_add_f64(&sc[ob.det_off + tl.det].rr, acc);
}

__global__ void gf_start_kernel(int64_t ndet, GfDet *__restrict__ sc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet) return;
    GfDet &s = sc[i];
    s.rr0 = s.rr;
    s.done = s.rr0 > 0.0 ? 0 : 1;
    s.iters = 0;
    s.pq = 0.0;
    s.rr_new = 0.0;
}

// FP32 copy of an FP64 TOD (the operand of the FP32 band product).
__global__ void __launch_bounds__(FT) gf_to_f32_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                       const double *__restrict__ x, float *__restrict__ x32)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t i = tod_index(ob, tl, u);
        x32[i] = f64_to_f32_bits(x[i]);
    }
}

// q = S (N p) (the band product nq, FP64 or FP32); pq[det] += p . q. The FP64 q is stored (in
// place over nq); the FP32 one is recomputed from nq by the update, which saves a stored vector.
template <typename QT>
__global__ void __launch_bounds__(FT) gf_pq_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                   const uint8_t *__restrict__ valid, const double *__restrict__ p,
                                                   const QT *__restrict__ nq, double *__restrict__ q,
                                                   GfDet *__restrict__ sc)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    if (sc[ob.det_off + tl.det].done) return;
    double acc = 0.0;
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t i = tod_index(ob, tl, u);
        double qv = 0.0;
        if (valid[i]) {
            if constexpr (sizeof(QT) == 8) qv = nq[i];
            else qv = f32_to_f64_bits(nq[i]);   // exact, and no FP64 conversion issued
        }
        if constexpr (sizeof(QT) == 8) q[i] = qv;
        acc += p[i] * qv;
    }
    acc = cta_sum_d(acc);
    if (threadIdx.x == 0) red_add_f64(&sc[ob.det_off + tl.det].pq, acc);
}

__global__ void gf_alpha_kernel(int64_t ndet, GfDet *__restrict__ sc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet) return;
    GfDet &s = sc[i];
    s.alpha = (!s.done && s.pq > 0.0) ? s.rr / s.pq : 0.0;
    s.rr_new = 0.0;
}

// y += alpha p; r -= alpha q; rr_new[det] += |r|^2. q is the stored FP64 S N p, or S applied to the
// FP32 band product.
template <typename QT>
__global__ void __launch_bounds__(FT) gf_update_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                       const uint8_t *__restrict__ valid, const double *__restrict__ p,
                                                       const QT *__restrict__ q, double *__restrict__ y,
                                                       double *__restrict__ r, GfDet *__restrict__ sc)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    const GfDet s = sc[ob.det_off + tl.det];
    if (s.done) return;
    double acc = 0.0;
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t i = tod_index(ob, tl, u);
        y[i] += s.alpha * p[i];
        double qv;
        if constexpr (sizeof(QT) == 8) qv = q[i];
        else qv = valid[i] ? f32_to_f64_bits(q[i]) : 0.0;
        const double rv = r[i] - s.alpha * qv;
        r[i] = rv;
        acc += rv * rv;
    }
    acc = cta_sum_d(acc);
    if (threadIdx.x == 0) red_add_f64(&sc[ob.det_off + tl.det].rr_new, acc);
}

__global__ void gf_beta_kernel(int64_t ndet, double tol2, GfDet *__restrict__ sc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet) return;
    GfDet &s = sc[i];
    s.pq = 0.0;
    if (s.done) { s.beta = 0.0; return; }
    s.beta = s.rr > 0.0 ? s.rr_new / s.rr : 0.0;
    s.rr = s.rr_new;
    s.iters += 1;
    if (s.rr <= tol2 * s.rr0) s.done = 1;
}

// p = r + beta p (detectors still iterating), and its FP32 copy for the next FP32 band product.
__global__ void __launch_bounds__(FT) gf_dir_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                    const double *__restrict__ r, double *__restrict__ p,
                                                    float *__restrict__ x32, const GfDet *__restrict__ sc)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    const GfDet s = sc[ob.det_off + tl.det];
    if (s.done) return;
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t i = tod_index(ob, tl, u);
        const double pv = r[i] + s.beta * p[i];
        p[i] = pv;
        if (x32) x32[i] = f64_to_f32_bits(pv);
    }
}

// out = d on observed samples, n + (N y) in the gaps. out may be d (documented in-place use), so
// neither carries __restrict__.
template <typename DT, typename QT>
__global__ void __launch_bounds__(FT) gf_fill_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                     const DT *d, const DT *__restrict__ nr,
                                                     const uint8_t *__restrict__ valid, const QT *__restrict__ ny,
                                                     DT *out)
{
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    for (int u = threadIdx.x; u < tl.len; u += FT) {
        const int64_t i = tod_index(ob, tl, u);
        out[i] = valid[i] ? d[i] : (DT)((double)nr[i] + (double)ny[i]);
    }
}

furax_status gapfill(const furax_noise *n, const void *d, const uint8_t *valid, const void *nr, void *out, int dtype,
                     int maxiter, double tol, int precision, int32_t *iters_out, cudaStream_t st)
{
    const bool f32 = precision == FURAX_F32;   // band product in FP32, vectors and scalars in FP64
    // FURAX_PREC_F32X2: the FP64 path with its band products in double-FP32 (short bands; a long
    // band keeps the FP64 overlap-save product)
    const bool df = precision == FURAX_PREC_F32X2 && !long_band(n);
    auto ninv64 = [&](const double *in, double *o) {
        return df ? launch_ninv_df(n, in, o, st) : launch_ninv(n, in, o, FURAX_F64, st);
    };
    const int64_t ns = n->nsamp_total, nd = n->ndet_total;
    if (ns == 0 || nd == 0) return FURAX_OK;
    const unsigned g = (unsigned)n->n_tiles;
    const unsigned dg = (unsigned)((nd + 127) / 128);
    furax_noise *nm = const_cast<furax_noise *>(n);   // workspaces live in the handle
    furax_status rc = FURAX_OK;
    auto ensure = [&](void **ptr, size_t bytes) {
        if (!rc && !*ptr && (rc = check_cuda(cudaMalloc(ptr, bytes), "gap-filling workspace"))) *ptr = nullptr;
    };
    ensure((void **)&nm->gf_y, sizeof(double) * ns);
    ensure((void **)&nm->gf_r, sizeof(double) * ns);
    ensure((void **)&nm->gf_p, sizeof(double) * ns);
    if (!f32) ensure((void **)&nm->gf_q, sizeof(double) * ns);   // FP32 band product: q is not stored
    ensure(&nm->gf_sc, sizeof(GfDet) * nd);
    if (f32) {
        ensure((void **)&nm->gf_x32, sizeof(float) * ns);
        ensure((void **)&nm->gf_n32, sizeof(float) * ns);
    }
    double *y = nm->gf_y, *r = nm->gf_r, *p = nm->gf_p, *q = nm->gf_q;
    GfDet *sc = (GfDet *)nm->gf_sc;
    float *x32 = nm->gf_x32, *n32 = nm->gf_n32;
    std::vector<GfDet> h(nd);
    bool all_done = false;
    if (!rc) rc = check_cuda(cudaMemsetAsync(sc, 0, sizeof(GfDet) * nd, st), "memset");
    if (!rc) {
        if (dtype == FURAX_F64)
            gf_init_kernel<double><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, (const double *)d, (const double *)nr, valid,
                                                      y, r, p, sc);
        else
            gf_init_kernel<float><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, (const float *)d, (const float *)nr, valid,
                                                     y, r, p, sc);
        gf_start_kernel<<<dg, 128, 0, st>>>(nd, sc);
        count_launches(2);
        if (f32) {   // the first direction's FP32 copy; later ones come from gf_dir
            gf_to_f32_kernel<<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, p, x32);
            count_launches(1);
        }
        rc = check_launch("gap filling (start)");
    }
    for (int it = 0; !rc && it < maxiter && !all_done; ++it) {
        if (f32) {   // N p in FP32
            if ((rc = launch_ninv(n, x32, n32, FURAX_F32, st))) break;
            gf_pq_kernel<float><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, valid, p, n32, nullptr, sc);
            gf_alpha_kernel<<<dg, 128, 0, st>>>(nd, sc);
            gf_update_kernel<float><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, valid, p, n32, y, r, sc);
        } else {
            if ((rc = ninv64(p, q))) break;
            gf_pq_kernel<double><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, valid, p, q, q, sc);
            gf_alpha_kernel<<<dg, 128, 0, st>>>(nd, sc);
            gf_update_kernel<double><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, valid, p, q, y, r, sc);
        }
        gf_beta_kernel<<<dg, 128, 0, st>>>(nd, tol * tol, sc);
        gf_dir_kernel<<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, r, p, f32 ? x32 : nullptr, sc);
        count_launches(5);
        if ((rc = check_launch("gap filling (iteration)"))) break;
        if ((it + 1) % 16 == 0 || it + 1 == maxiter) {
            if ((rc = check_cuda(cudaMemcpyAsync(h.data(), sc, sizeof(GfDet) * nd, cudaMemcpyDeviceToHost, st), "read")))
                break;
            if ((rc = check_cuda(cudaStreamSynchronize(st), "gap filling"))) break;
            all_done = true;
            for (const GfDet &s : h) all_done = all_done && s.done;
        }
    }
    if (!rc && f32) {   // N y
        gf_to_f32_kernel<<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, y, x32);
        count_launches(1);
        rc = launch_ninv(n, x32, n32, FURAX_F32, st);
    } else if (!rc) {
        rc = ninv64(y, q);
    }
    if (!rc) {
        if (dtype == FURAX_F64 && f32)
            gf_fill_kernel<double, float><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, (const double *)d, (const double *)nr,
                                                             valid, n32, (double *)out);
        else if (dtype == FURAX_F64)
            gf_fill_kernel<double, double><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, (const double *)d, (const double *)nr,
                                                              valid, q, (double *)out);
        else if (f32)
            gf_fill_kernel<float, float><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, (const float *)d, (const float *)nr,
                                                            valid, n32, (float *)out);
        else
            gf_fill_kernel<float, double><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, (const float *)d, (const float *)nr,
                                                             valid, q, (float *)out);
        count_launches(1);
        rc = check_launch("gap filling (fill)");
    }
    if (!rc) rc = check_cuda(cudaMemcpyAsync(h.data(), sc, sizeof(GfDet) * nd, cudaMemcpyDeviceToHost, st), "read");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "gap filling");
    if (rc) return rc;
    all_done = true;
    for (int64_t i = 0; i < nd; ++i) {
        all_done = all_done && h[i].done;
        if (iters_out) iters_out[i] = h[i].iters;
    }
    return all_done ? FURAX_OK : FURAX_ENOTCONVERGED;
}

}  // namespace fx
