// Map-making solver: the normal-equations operator, right-hand side and preconditioned
// conjugate gradient (Furax paper: "A.I(solver=..., preconditioner=...)", Table 1; the
// maximum-likelihood and binned estimators and BJPreconditioner, "Map-making classes";
// GLS estimator, Statement of Need).
//
// Each observation is an independent problem with its own PCG scalars (alpha, beta,
// <r,z>, convergence flag). Dot products are reduced deterministically: a fixed-order
// block reduction per pixel tile, then a fixed-order sum of the tiles of one observation.
// The iteration body is a fixed sequence of launches on one stream, captured once into a
// CUDA graph and replayed; the host reads the convergence flags every few iterations.
//
// Precision: FP64 runs the plain FP64 operator. F32 solves with the FP32 operator inside
// an FP64 defect-correction loop: r = b - A64 x is recomputed with the FP64 operator, the
// inner PCG solves A32 e = r to a modest tolerance, x += e. The vectors and every scalar
// stay FP64 throughout.
#include "internal.cuh"
#include "atomics.cuh"

namespace fx {

constexpr int VT = 256;   // threads per vector-kernel block
constexpr int KD = 3;     // dot slots per pixel tile

struct CgScalars {
    double bb, rz, rr, pq, alpha, beta;
    int32_t done, iters;
};

struct CgWs {
    int64_t np = 0;
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    double *minv = nullptr;       // [np][6]
    uint8_t *valid = nullptr;     // [np]
    double *bfull = nullptr, *e = nullptr, *acc64 = nullptr;
    float4 *p32 = nullptr, *hi = nullptr, *lo = nullptr;
    double *partial = nullptr;    // [n_ptiles][KD]
    CgScalars *sc = nullptr;      // [n_obs]
    CgScalars *h_sc = nullptr;    // pinned host mirror
    unsigned *h_err = nullptr;    // pinned copy of the handle's device error word
    double *hist = nullptr;       // [hist_cap] device
    int32_t hist_cap = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0, graph_prec = -1, graph_acc = -1;
    const void *graph_noise = nullptr;
    const void *graph_tpl = nullptr;
    const void *graph_pt = nullptr;
    const double *graph_x = nullptr;
    double graph_tol2 = -1.0;
    bool graph_prof = false;
    std::vector<cudaEvent_t> ev;  // timing events baked into the graph (2 per iteration)
};

// Run f() between two timing events when kernel timing is on (eager launches only).
template <class F>
static furax_status timed(int kind, cudaStream_t st, F &&f)
{
    if (!prof_on()) return f();
    cudaEvent_t a = nullptr, b = nullptr;
    prof_pair(&a, &b);
    if (a) cudaEventRecord(a, st);
    furax_status rc = f();
    if (b) cudaEventRecord(b, st);
    prof_push(rc ? 0 : kind, rc ? nullptr : a, b);
    return rc;
}

static void free_cg(CgWs *w)
{
    if (!w) return;
    cudaFree(w->r); cudaFree(w->z); cudaFree(w->p); cudaFree(w->q); cudaFree(w->minv); cudaFree(w->valid);
    cudaFree(w->bfull); cudaFree(w->e); cudaFree(w->acc64); cudaFree(w->p32); cudaFree(w->hi);   // lo = hi + 1
    cudaFree(w->partial); cudaFree(w->sc); cudaFree(w->hist);
    for (cudaEvent_t e : w->ev) cudaEventDestroy(e);
    if (w->h_sc) cudaFreeHost(w->h_sc);
    if (w->h_err) cudaFreeHost(w->h_err);
    if (w->graph) cudaGraphExecDestroy(w->graph);
    delete w;
}

void destroy_cg_ws(furax_pointing *p)
{
    free_cg(p->cg);
    p->cg = nullptr;
}

// ------------------------------------------------------------------------------------
// Elementwise helpers
// ------------------------------------------------------------------------------------

// Clear pixel i of the FP32 accumulators: plain (za[i]) or compensated (zb = za + 1: za[2i], zb[2i]).
__device__ __forceinline__ void zero_acc(float4 *za, float4 *zb, int64_t i)
{
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (zb) { za[kKahanStride * i] = z; zb[kKahanStride * i] = z; }
    else if (za) za[i] = z;
}

// x32[p] = (float)x[p] on valid pixels (0 elsewhere); zero the FP32 accumulators.
__global__ void pack_x32_kernel(const double *__restrict__ x, const uint8_t *__restrict__ valid, float4 *__restrict__ x32,
                                float4 *__restrict__ za, float4 *__restrict__ zb, int64_t np)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = !valid || valid[i];
        x32[i] = ok ? make_float4((float)x[3 * i], (float)x[3 * i + 1], (float)x[3 * i + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        zero_acc(za, zb, i);
    }
}

__device__ __forceinline__ void acc_value(int acc, const float4 *hi, const float4 *lo, const double *a64, int64_t i,
                                          double &v0, double &v1, double &v2)
{
    if (acc == FURAX_ACC_F64) { v0 = a64[3 * i]; v1 = a64[3 * i + 1]; v2 = a64[3 * i + 2]; return; }
    const bool k = acc == FURAX_ACC_F32_KAHAN;   // interleaved: hi[2i], lo[2i] (atomics.cuh)
    const float4 h = hi[k ? kKahanStride * i : i];
    v0 = h.x; v1 = h.y; v2 = h.z;
    if (k) { const float4 l = lo[kKahanStride * i]; v0 += l.x; v1 += l.y; v2 += l.z; }
}

__global__ void finalize_acc_kernel(int acc, const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                                    const double *__restrict__ a64, const uint8_t *__restrict__ valid,
                                    double *__restrict__ out, int64_t np)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        double v0, v1, v2;
        acc_value(acc, hi, lo, a64, i, v0, v1, v2);
        const bool ok = !valid || valid[i];
        out[3 * i] = ok ? v0 : 0.0; out[3 * i + 1] = ok ? v1 : 0.0; out[3 * i + 2] = ok ? v2 : 0.0;
    }
}

__global__ void mask_copy_kernel(const double *__restrict__ x, const uint8_t *__restrict__ valid, double *__restrict__ out,
                                 int64_t np)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = !valid || valid[i];
        out[3 * i] = ok ? x[3 * i] : 0.0; out[3 * i + 1] = ok ? x[3 * i + 1] : 0.0; out[3 * i + 2] = ok ? x[3 * i + 2] : 0.0;
    }
}

// Grid-stride vector kernels: at most eight VT-thread blocks per SM of the handle's device.
static unsigned vgrid(const furax_pointing *p, int64_t np)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((np + VT - 1) / VT, 8LL * p->n_sm));
}

furax_status launch_pack_x32(const furax_pointing *p, const double *x, const uint8_t *valid, float4 *x32, float4 *za,
                             float4 *zb, cudaStream_t st)
{
    pack_x32_kernel<<<vgrid(p, p->npix_total), VT, 0, st>>>(x, valid, x32, za, zb, p->npix_total);
    count_launches(1);
    return check_launch("pack FP32 map");
}

furax_status launch_finalize_acc(const furax_pointing *p, int acc, const float4 *hi, const float4 *lo,
                                 const double *a64, const uint8_t *valid, double *out, cudaStream_t st)
{
    finalize_acc_kernel<<<vgrid(p, p->npix_total), VT, 0, st>>>(acc, hi, lo, a64, valid, out, p->npix_total);
    count_launches(1);
    return check_launch("finalise accumulator");
}

furax_status launch_mask_copy(const furax_pointing *p, const double *x, const uint8_t *valid, double *out,
                              cudaStream_t st)
{
    mask_copy_kernel<<<vgrid(p, p->npix_total), VT, 0, st>>>(x, valid, out, p->npix_total);
    count_launches(1);
    return check_launch("mask copy");
}

__global__ void tod_to_f64_kernel(const float *__restrict__ in, double *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

furax_status tod_ws(const furax_pointing *p)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    const size_t bytes = sizeof(double) * (size_t)std::max<int64_t>(1, p->nsamp_total);
    furax_status rc = ensure_ws(pm, &pm->ws_tod, bytes);
    if (!rc) rc = ensure_ws(pm, &pm->ws_tod2, bytes);
    return rc;
}

furax_status launch_ata_chain(const furax_pointing *p, const furax_noise *n, const double *x, int tod_t,
                              double *acc64, cudaStream_t st)
{
    furax_status rc;
    if ((rc = launch_P(p, x, FURAX_F64, p->ws_tod, tod_t, st))) return rc;
    if ((rc = launch_ninv(n, p->ws_tod, p->ws_tod2, tod_t, st))) return rc;
    return launch_PT_acc64(p, p->ws_tod2, tod_t, acc64, st);
}

furax_status launch_rhs_chain(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, double *acc64,
                              cudaStream_t st)
{
    furax_status rc;
    const void *d64 = d;
    if (d_t == FURAX_F32) {
        tod_to_f64_kernel<<<vgrid(p, p->nsamp_total), VT, 0, st>>>((const float *)d, (double *)p->ws_tod, p->nsamp_total);
        count_launches(1);
        if ((rc = check_launch("TOD to FP64"))) return rc;
        d64 = p->ws_tod;
    }
    if ((rc = launch_ninv(n, d64, p->ws_tod2, FURAX_F64, st))) return rc;
    return launch_PT_acc64(p, p->ws_tod2, FURAX_F64, acc64, st);
}

// out = S P^T N^-1 P S^T x
furax_status ptnp_apply(const furax_pointing *p, const furax_noise *n, const double *x, double *out,
                        const uint8_t *valid, int precision, int acc, cudaStream_t st, const furax_templates *tp)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    const int64_t np = p->npix_total;
    furax_status rc;
    if (long_band(n)) {
        // the band does not fit the fused kernels: P, overlap-save N^-1 and P^T with the TOD in HBM,
        // FP64 accumulation (FP32 TOD for precision FURAX_F32)
        if ((rc = tod_ws(p))) return rc;
        if ((rc = ensure_ws(pm, (void **)&pm->ws_acc64, sizeof(double) * 3 * np))) return rc;
        const double *xin = x;
        if (valid) {
            if ((rc = ensure_ws(pm, (void **)&pm->ws_x64, sizeof(double) * 3 * np))) return rc;
            if ((rc = launch_mask_copy(p, x, valid, pm->ws_x64, st))) return rc;
            xin = pm->ws_x64;
        }
        if ((rc = check_cuda(cudaMemsetAsync(pm->ws_acc64, 0, sizeof(double) * 3 * np, st), "memset"))) return rc;
        const int tod_t = precision == FURAX_F32 ? FURAX_F32 : FURAX_F64;
        if ((rc = launch_ata_chain(p, n, xin, tod_t, pm->ws_acc64, st))) return rc;
        if (tp && (rc = launch_tpl_map(tp, FURAX_F64, FURAX_ACC_F64, nullptr, xin, nullptr, nullptr, pm->ws_acc64, st)))
            return rc;
        return launch_finalize_acc(p, FURAX_ACC_F64, nullptr, nullptr, pm->ws_acc64, valid, out, st);
    }
    if (precision == FURAX_F64 || precision == FURAX_PREC_F32X2) {
        if ((rc = ensure_ws(pm, (void **)&pm->ws_acc64, sizeof(double) * 3 * np))) return rc;
        const double *xin = x;
        if (valid) {
            if ((rc = ensure_ws(pm, (void **)&pm->ws_x64, sizeof(double) * 3 * np))) return rc;
            if ((rc = launch_mask_copy(p, x, valid, pm->ws_x64, st))) return rc;
            xin = pm->ws_x64;
        }
        if ((rc = check_cuda(cudaMemsetAsync(pm->ws_acc64, 0, sizeof(double) * 3 * np, st), "memset"))) return rc;
        if (precision == FURAX_F64) {
            if ((rc = timed(1, st, [&] { return launch_fused_f64(p, n, xin, pm->ws_acc64, st); }))) return rc;
        } else {
            if ((rc = timed(2, st, [&] { return launch_fused_df(p, n, xin, nullptr, 0, pm->ws_acc64, st); }))) return rc;
        }
        if (tp && (rc = launch_tpl_map(tp, FURAX_F64, FURAX_ACC_F64, nullptr, xin, nullptr, nullptr, pm->ws_acc64, st)))
            return rc;
        return launch_finalize_acc(p, FURAX_ACC_F64, nullptr, nullptr, pm->ws_acc64, valid, out, st);
    }
    if ((rc = ensure_ws(pm, (void **)&pm->ws_map32, sizeof(float4) * np))) return rc;
    float4 *hi = nullptr, *lo = nullptr;
    double *a64 = nullptr;
    if (acc == FURAX_ACC_F64) {
        if ((rc = ensure_ws(pm, (void **)&pm->ws_acc64, sizeof(double) * 3 * np))) return rc;
        a64 = pm->ws_acc64;
        if ((rc = check_cuda(cudaMemsetAsync(a64, 0, sizeof(double) * 3 * np, st), "memset"))) return rc;
    } else {
        if ((rc = ensure_ws(pm, (void **)&pm->ws_acc_hi, sizeof(float4) * kKahanStride * np))) return rc;
        hi = pm->ws_acc_hi;
        if (acc == FURAX_ACC_F32_KAHAN) lo = hi + 1;   // interleaved compensated layout
    }
    if ((rc = launch_pack_x32(p, x, valid, pm->ws_map32, hi, lo, st))) return rc;
    double *tpl_a = tpl_fused_target(tp, p);
    const FusedTpl ft{1, tpl_a, 0, tp ? tp->order : 0};
    if ((rc = timed(0, st, [&] { return launch_fused_f32(p, n, pm->ws_map32, acc, hi, lo, a64, st,
                                                         tpl_a ? &ft : nullptr); })))
        return rc;
    if (tp && (rc = launch_tpl_map(tp, FURAX_F32, acc, pm->ws_map32, nullptr, hi, lo, a64, st, tpl_a != nullptr)))
        return rc;
    return launch_finalize_acc(p, acc, hi, lo, a64, valid, out, st);
}

// ------------------------------------------------------------------------------------
// PCG kernels (per-observation scalars)
// ------------------------------------------------------------------------------------

template <int K>
__device__ __forceinline__ void block_store_partials(double (&v)[K], double *__restrict__ out)
{
    __shared__ double red[K][VT / 32];
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[k][threadIdx.x >> 5] = v[k];
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < VT / 32; ++w) s += red[threadIdx.x][w];
        out[threadIdx.x] = s;
    }
}

// Sum the partials of each observation's tiles in order (one block per observation).
__device__ __forceinline__ double obs_sum(const ObsInfo &ob, const double *__restrict__ partial, int slot)
{
    __shared__ double red[VT / 32];
    double s = 0.0;
    for (int t = threadIdx.x; t < ob.nptile; t += VT) s += partial[(ob.ptile0 + t) * KD + slot];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < VT / 32; ++w) tot += red[w];
    __syncthreads();
    return tot;
}

__device__ __forceinline__ void apply_minv(const double *__restrict__ m, const double *__restrict__ r, double *z)
{
    z[0] = m[0] * r[0] + m[1] * r[1] + m[2] * r[2];
    z[1] = m[1] * r[0] + m[3] * r[1] + m[4] * r[2];
    z[2] = m[2] * r[0] + m[4] * r[1] + m[5] * r[2];
}

// Start: r = b (masked), z = M^-1 r, p = z, x = 0; partials <b,b>, <r,z>.
__global__ void cg_init_kernel(const PTile *__restrict__ pt, const double *__restrict__ b, const double *__restrict__ minv,
                               const uint8_t *__restrict__ valid, double *__restrict__ x, double *__restrict__ r,
                               double *__restrict__ z, double *__restrict__ p, double *__restrict__ partial)
{
    const PTile t = pt[blockIdx.x];
    double v[2] = {0.0, 0.0};
    for (int k = threadIdx.x; k < t.len; k += VT) {
        const int64_t i = t.p0 + k;
        double rr[3], zz[3] = {0.0, 0.0, 0.0};
        const bool ok = valid[i];
        for (int c = 0; c < 3; ++c) rr[c] = ok ? b[3 * i + c] : 0.0;
        if (ok) apply_minv(minv + 6 * i, rr, zz);
        for (int c = 0; c < 3; ++c) {
            r[3 * i + c] = rr[c]; z[3 * i + c] = zz[c]; p[3 * i + c] = zz[c]; x[3 * i + c] = 0.0;
            v[0] += rr[c] * rr[c]; v[1] += rr[c] * zz[c];
        }
    }
    block_store_partials<2>(v, partial + (int64_t)blockIdx.x * KD);
}

__global__ void cg_init_scalars_kernel(const ObsInfo *__restrict__ obs, const double *__restrict__ partial,
                                       CgScalars *__restrict__ sc, double *__restrict__ hist)
{
    const ObsInfo ob = obs[blockIdx.x];
    const double bb = obs_sum(ob, partial, 0);
    const double rz = obs_sum(ob, partial, 1);
    if (threadIdx.x == 0) {
        CgScalars s;
        s.bb = bb; s.rz = rz; s.rr = bb; s.pq = 0.0; s.alpha = 0.0; s.beta = 0.0;
        s.done = bb > 0.0 ? 0 : 1;
        s.iters = 0;
        sc[blockIdx.x] = s;
        if (blockIdx.x == 0 && hist) hist[0] = bb > 0.0 ? 1.0 : 0.0;
    }
}

// p32 = (float)p, zero accumulators (start of an FP32 operator application).
__global__ void cg_pack_kernel(const double *__restrict__ p, float4 *__restrict__ p32, float4 *__restrict__ za,
                               float4 *__restrict__ zb, double *__restrict__ z64, int64_t np)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        if (p32) p32[i] = make_float4((float)p[3 * i], (float)p[3 * i + 1], (float)p[3 * i + 2], 0.f);
        zero_acc(za, zb, i);
        if (z64) { z64[3 * i] = 0.0; z64[3 * i + 1] = 0.0; z64[3 * i + 2] = 0.0; }
    }
}

// q = S (accumulator); partial <p, q>.
__global__ void cg_q_kernel(const PTile *__restrict__ pt, int acc, const float4 *__restrict__ hi,
                            const float4 *__restrict__ lo, const double *__restrict__ a64,
                            const uint8_t *__restrict__ valid, const double *__restrict__ p, double *__restrict__ q,
                            double *__restrict__ partial)
{
    const PTile t = pt[blockIdx.x];
    double v[1] = {0.0};
    for (int k = threadIdx.x; k < t.len; k += VT) {
        const int64_t i = t.p0 + k;
        double a[3];
        acc_value(acc, hi, lo, a64, i, a[0], a[1], a[2]);
        const bool ok = valid[i];
        for (int c = 0; c < 3; ++c) {
            const double qq = ok ? a[c] : 0.0;
            q[3 * i + c] = qq;
            v[0] += p[3 * i + c] * qq;
        }
    }
    block_store_partials<1>(v, partial + (int64_t)blockIdx.x * KD);
}

__global__ void cg_alpha_kernel(const ObsInfo *__restrict__ obs, const double *__restrict__ partial,
                                CgScalars *__restrict__ sc)
{
    const ObsInfo ob = obs[blockIdx.x];
    const double pq = obs_sum(ob, partial, 0);
    if (threadIdx.x == 0) {
        CgScalars &s = sc[blockIdx.x];
        s.pq = pq;
        s.alpha = (s.done || pq <= 0.0) ? 0.0 : s.rz / pq;
        if (!s.done && pq <= 0.0) s.done = 2;   // breakdown: operator not positive on p
    }
}

// x += alpha p; r -= alpha q; z = M^-1 r; partials <r,z>, <r,r>.
__global__ void cg_update_kernel(const PTile *__restrict__ pt, const CgScalars *__restrict__ sc,
                                 const double *__restrict__ minv, const uint8_t *__restrict__ valid,
                                 double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
                                 const double *__restrict__ p, const double *__restrict__ q, double *__restrict__ partial)
{
    const PTile t = pt[blockIdx.x];
    const double alpha = sc[t.obs].alpha;
    double v[2] = {0.0, 0.0};
    for (int k = threadIdx.x; k < t.len; k += VT) {
        const int64_t i = t.p0 + k;
        double rr[3], zz[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 3; ++c) {
            x[3 * i + c] += alpha * p[3 * i + c];
            rr[c] = r[3 * i + c] - alpha * q[3 * i + c];
            r[3 * i + c] = rr[c];
        }
        if (valid[i]) apply_minv(minv + 6 * i, rr, zz);
        for (int c = 0; c < 3; ++c) {
            z[3 * i + c] = zz[c];
            v[0] += rr[c] * zz[c];
            v[1] += rr[c] * rr[c];
        }
    }
    block_store_partials<2>(v, partial + (int64_t)blockIdx.x * KD);
}

__global__ void cg_beta_kernel(const ObsInfo *__restrict__ obs, const double *__restrict__ partial,
                               CgScalars *__restrict__ sc, double tol2, double *__restrict__ hist, int hist_cap)
{
    const ObsInfo ob = obs[blockIdx.x];
    const double rz = obs_sum(ob, partial, 0);
    const double rr = obs_sum(ob, partial, 1);
    if (threadIdx.x == 0) {
        CgScalars &s = sc[blockIdx.x];
        if (s.done) { s.beta = 0.0; return; }
        s.iters += 1;
        s.rr = rr;
        s.beta = rz / s.rz;
        s.rz = rz;
        if (blockIdx.x == 0 && hist && s.iters < hist_cap) hist[s.iters] = sqrt(rr / s.bb);
        if (rr <= tol2 * s.bb) s.done = 1;
    }
}

// p = z + beta p (frozen when the observation is done); then prepare the next application.
__global__ void cg_dir_kernel(const PTile *__restrict__ pt, const CgScalars *__restrict__ sc,
                              const double *__restrict__ z, double *__restrict__ p, float4 *__restrict__ p32,
                              float4 *__restrict__ za, float4 *__restrict__ zb, double *__restrict__ z64)
{
    const PTile t = pt[blockIdx.x];
    const CgScalars s = sc[t.obs];
    for (int k = threadIdx.x; k < t.len; k += VT) {
        const int64_t i = t.p0 + k;
        double pp[3];
        for (int c = 0; c < 3; ++c) {
            pp[c] = s.done ? p[3 * i + c] : z[3 * i + c] + s.beta * p[3 * i + c];
            p[3 * i + c] = pp[c];
        }
        if (p32) p32[i] = make_float4((float)pp[0], (float)pp[1], (float)pp[2], 0.f);
        zero_acc(za, zb, i);
        if (z64) { z64[3 * i] = 0.0; z64[3 * i + 1] = 0.0; z64[3 * i + 2] = 0.0; }
    }
}

// rtrue = S (b - acc64); partial ||rtrue||^2 ; also used for final residual norms.
__global__ void residual_kernel(const PTile *__restrict__ pt, const double *__restrict__ b,
                                const double *__restrict__ a64, const uint8_t *__restrict__ valid,
                                double *__restrict__ rout, double *__restrict__ partial)
{
    const PTile t = pt[blockIdx.x];
    double v[2] = {0.0, 0.0};
    for (int k = threadIdx.x; k < t.len; k += VT) {
        const int64_t i = t.p0 + k;
        const bool ok = valid[i];
        for (int c = 0; c < 3; ++c) {
            const double rr = ok ? b[3 * i + c] - a64[3 * i + c] : 0.0;
            if (rout) rout[3 * i + c] = rr;
            v[0] += rr * rr;
            v[1] += ok ? b[3 * i + c] * b[3 * i + c] : 0.0;
        }
    }
    block_store_partials<2>(v, partial + (int64_t)blockIdx.x * KD);
}

__global__ void obs_norms_kernel(const ObsInfo *__restrict__ obs, const double *__restrict__ partial,
                                 double *__restrict__ out /* [n_obs][2] */)
{
    const ObsInfo ob = obs[blockIdx.x];
    const double a = obs_sum(ob, partial, 0);
    const double b = obs_sum(ob, partial, 1);
    if (threadIdx.x == 0) { out[2 * blockIdx.x] = a; out[2 * blockIdx.x + 1] = b; }
}

// x += e on valid pixels
__global__ void axpy_kernel(double *__restrict__ x, const double *__restrict__ e, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += e[i];
}

// ------------------------------------------------------------------------------------
// Driver
// ------------------------------------------------------------------------------------

static furax_status alloc(void **ptr, size_t bytes)
{
    if (cudaMalloc(ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_error(FURAX_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    return FURAX_OK;
}

static furax_status get_ws(furax_pointing *p, int hist_cap, CgWs **out)
{
    if (p->cg && p->cg->hist_cap >= hist_cap) { *out = p->cg; return FURAX_OK; }
    if (p->cg) destroy_cg_ws(p);
    CgWs *w = new CgWs();
    // room for one amplitude pseudo-pixel per detector (the augmented system of template deprojection)
    const int64_t np = p->npix_total + p->ndet_total;
    w->np = np;
    furax_status rc = FURAX_OK;
    const size_t v3 = sizeof(double) * 3 * (size_t)np;
    if (!rc) rc = alloc((void **)&w->r, v3);
    if (!rc) rc = alloc((void **)&w->z, v3);
    if (!rc) rc = alloc((void **)&w->p, v3);
    if (!rc) rc = alloc((void **)&w->q, v3);
    if (!rc) rc = alloc((void **)&w->bfull, v3);
    if (!rc) rc = alloc((void **)&w->e, v3);
    if (!rc) rc = alloc((void **)&w->acc64, v3);
    if (!rc) rc = alloc((void **)&w->minv, sizeof(double) * 6 * (size_t)np);
    if (!rc) rc = alloc((void **)&w->valid, (size_t)np);
    if (!rc) rc = alloc((void **)&w->p32, sizeof(float4) * (size_t)np);
    // FP32 accumulators: plain hi[i], or compensated interleaved hi[2i], lo[2i] with lo = hi + 1
    if (!rc) rc = alloc((void **)&w->hi, sizeof(float4) * kKahanStride * (size_t)np);
    if (!rc) w->lo = w->hi + 1;
    const int64_t nparts = p->n_ptiles + p->n_obs + p->ndet_total / PTILE + 1;   // also the augmented tiles
    if (!rc) rc = alloc((void **)&w->partial, sizeof(double) * KD * (size_t)nparts);
    if (!rc) rc = alloc((void **)&w->sc, sizeof(CgScalars) * p->n_obs);
    w->hist_cap = std::max(hist_cap, 1);
    if (!rc) rc = alloc((void **)&w->hist, sizeof(double) * w->hist_cap);
    if (!rc && (cudaMallocHost((void **)&w->h_sc, sizeof(CgScalars) * p->n_obs) != cudaSuccess ||
                cudaMallocHost((void **)&w->h_err, sizeof(unsigned)) != cudaSuccess)) {
        cudaGetLastError();
        rc = set_error(FURAX_ENOMEM, "pinned host allocation failed");
    }
    if (rc) { free_cg(w); return rc; }
    p->cg = w;
    *out = w;
    return FURAX_OK;
}

struct Body {
    const furax_pointing *p;
    const furax_noise *n;
    CgWs *w;
    int precision, acc;
    double tol2;
    double *x;
    unsigned pg;   // pixel-tile grid
    const furax_templates *tp;   // template deprojection, or nullptr
    // layout of the solved vector: the pointing's pixel tiles and observations, or the augmented
    // ones of the templates (the map plus one amplitude pseudo-pixel per detector)
    const PTile *pt;
    const ObsInfo *cobs;
    int64_t np_cg;
    bool aug;
    AllReduce ar;                // detector sharding: sum of the operator's output over processes
};

// One PCG iteration: q = A p, alpha, x/r/z update, beta, new direction (+ accumulator reset).
static furax_status body(const Body &b, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    CgWs *w = b.w;
    const furax_pointing *p = b.p;
    furax_status rc;
    int acc = b.acc;
    if (e0) cudaEventRecordWithFlags(e0, st, cudaEventRecordExternal);  // a timing node inside a captured graph
    const bool lb = long_band(b.n);
    if (lb) {
        // TOD in HBM; FP32 TOD for the inner solve of the mixed precision, FP64 accumulation
        if ((rc = launch_ata_chain(p, b.n, w->p, b.precision == FURAX_F64 ? FURAX_F64 : FURAX_F32, w->acc64, st)))
            return rc;
        acc = FURAX_ACC_F64;
    } else if (b.precision == FURAX_F64) {
        if ((rc = launch_fused_f64(p, b.n, w->p, w->acc64, st))) return rc;
        acc = FURAX_ACC_F64;
    } else {
        FusedTpl ft{0, nullptr, 0, 0};
        if (b.aug) ft = FusedTpl{2, nullptr, p->npix_total, b.tp->order};
        else if (double *pa = tpl_fused_target(b.tp, p)) ft = FusedTpl{1, pa, 0, b.tp->order};
        if ((rc = launch_fused_f32(p, b.n, w->p32, acc, w->hi, w->lo, w->acc64, st, ft.mode ? &ft : nullptr)))
            return rc;
    }
    if (e1) cudaEventRecordWithFlags(e1, st, cudaEventRecordExternal);
    int acc_q = acc;   // where cg_q reads the operator's output
    if (b.ar.on()) {
        // detector sharding: this process's partial P^T N^-1 P p, in FP64, summed over processes
        // (the FP32 accumulators are still cleared for the next application below)
        if (acc != FURAX_ACC_F64) {
            if ((rc = launch_finalize_acc(p, acc, w->hi, w->lo, nullptr, nullptr, w->acc64, st))) return rc;
            acc_q = FURAX_ACC_F64;
        }
        if ((rc = b.ar(w->acc64, 3 * p->npix_total, FURAX_REDUCE_F64, st))) return rc;
    }
    if (b.tp && !b.aug) {
        const bool f64 = b.precision == FURAX_F64 || lb;
        if ((rc = launch_tpl_map(b.tp, f64 ? FURAX_F64 : FURAX_F32, acc, w->p32, w->p, w->hi, w->lo, w->acc64, st,
                                 !f64 && tpl_fused_target(b.tp, p) != nullptr)))
            return rc;
    }
    cg_q_kernel<<<b.pg, VT, 0, st>>>(b.pt, acc_q, w->hi, w->lo, w->acc64, w->valid, w->p, w->q, w->partial);
    cg_alpha_kernel<<<p->n_obs, VT, 0, st>>>(b.cobs, w->partial, w->sc);
    cg_update_kernel<<<b.pg, VT, 0, st>>>(b.pt, w->sc, w->minv, w->valid, b.x, w->r, w->z, w->p, w->q, w->partial);
    cg_beta_kernel<<<p->n_obs, VT, 0, st>>>(b.cobs, w->partial, w->sc, b.tol2, w->hist, w->hist_cap);
    const bool f32 = b.precision != FURAX_F64;
    cg_dir_kernel<<<b.pg, VT, 0, st>>>(b.pt, w->sc, w->z, w->p, f32 ? w->p32 : nullptr,
                                       (f32 && acc != FURAX_ACC_F64) ? w->hi : nullptr,
                                       (f32 && acc == FURAX_ACC_F32_KAHAN) ? w->lo : nullptr,
                                       (!f32 || acc == FURAX_ACC_F64) ? w->acc64 : nullptr);
    count_launches(5);
    return check_launch("PCG iteration");
}

// Prepare the first application after cg_init (pack p, zero accumulators).
static furax_status body_prologue(const Body &b, cudaStream_t st)
{
    CgWs *w = b.w;
    const bool f32 = b.precision != FURAX_F64;
    const int acc = f32 ? b.acc : FURAX_ACC_F64;
    cg_pack_kernel<<<vgrid(b.p, b.np_cg), VT, 0, st>>>(w->p, f32 ? w->p32 : nullptr,
                                                          (f32 && acc != FURAX_ACC_F64) ? w->hi : nullptr,
                                                          (f32 && acc == FURAX_ACC_F32_KAHAN) ? w->lo : nullptr,
                                                          (acc == FURAX_ACC_F64) ? w->acc64 : nullptr, b.np_cg);
    count_launches(1);
    return check_launch("PCG prologue");
}

static int64_t graph_nodes_per_iter(const Body &b)
{
    if (b.aug) return 6;
    const bool lb = long_band(b.n);
    int64_t k = 5 + (lb ? 3 : 1);
    if (b.tp) k += (!lb && b.precision != FURAX_F64 && tpl_fused_target(b.tp, b.p)) ? 2 : 3;
    return k;
}

// Run PCG from b (in w->bfull or a given rhs) into x. Returns iterations used (max over obs).
static furax_status pcg(const Body &b, const double *rhs, int maxiter, int use_graph, int check_every,
                        cudaStream_t st, int *iters_out, bool *all_done)
{
    CgWs *w = b.w;
    const furax_pointing *p = b.p;
    furax_status rc;
    cg_init_kernel<<<b.pg, VT, 0, st>>>(b.pt, rhs, w->minv, w->valid, b.x, w->r, w->z, w->p, w->partial);
    cg_init_scalars_kernel<<<p->n_obs, VT, 0, st>>>(b.cobs, w->partial, w->sc, w->hist);
    count_launches(2);
    if ((rc = check_launch("PCG init"))) return rc;
    if ((rc = body_prologue(b, st))) return rc;
    check_every = std::max(1, check_every);
    // Stream capture is not possible on the legacy default stream, nor around the caller's
    // sharding sum (host code).
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread || b.ar.on()) use_graph = 0;
    int done_iters = 0;
    *all_done = false;
    while (done_iters < maxiter) {
        const int n = std::min(check_every, maxiter - done_iters);
        int graph_timed = 0;
        if (use_graph && n == check_every) {
            const bool prof = prof_on();
            const bool rebuild = !w->graph || w->graph_iters != n || w->graph_prec != b.precision ||
                                 w->graph_acc != b.acc || w->graph_noise != (const void *)b.n || w->graph_x != b.x ||
                                 w->graph_tol2 != b.tol2 || w->graph_prof != prof || w->graph_tpl != (const void *)b.tp ||
                                 w->graph_pt != (const void *)b.pt;
            if (rebuild) {
                if (w->graph) { cudaGraphExecDestroy(w->graph); w->graph = nullptr; }
                while (prof && (int)w->ev.size() < 2 * n) {
                    cudaEvent_t e;
                    if ((rc = check_cuda(cudaEventCreate(&e), "timing event"))) return rc;
                    w->ev.push_back(e);
                }
                cudaGraph_t g;
                if ((rc = check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture")))
                    return rc;
                furax_status brc = FURAX_OK;
                const int64_t before = furax_launch_count();
                for (int i = 0; i < n && !brc; ++i)
                    brc = body(b, st, prof ? w->ev[2 * i] : nullptr, prof ? w->ev[2 * i + 1] : nullptr);
                count_launches(before - furax_launch_count());   // capture is not execution
                cudaError_t e = cudaStreamEndCapture(st, &g);
                if (brc) { if (e == cudaSuccess) cudaGraphDestroy(g); return brc; }
                if ((rc = check_cuda(e, "end capture"))) return rc;
                e = cudaGraphInstantiate(&w->graph, g, 0);
                cudaGraphDestroy(g);
                if ((rc = check_cuda(e, "graph instantiate"))) return rc;
                w->graph_iters = n; w->graph_prec = b.precision; w->graph_acc = b.acc; w->graph_noise = b.n;
                w->graph_x = b.x; w->graph_tol2 = b.tol2; w->graph_prof = prof; w->graph_tpl = b.tp;
                w->graph_pt = b.pt;
            }
            if ((rc = check_cuda(cudaGraphLaunch(w->graph, st), "graph launch"))) return rc;
            count_launches(graph_nodes_per_iter(b) * n);
            graph_timed = w->graph_prof ? n : 0;
        } else {
            const int kind = b.precision == FURAX_F64 ? 1 : 0;
            for (int i = 0; i < n; ++i) {
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (prof_on()) prof_pair(&e0, &e1);
                if ((rc = body(b, st, e0, e1))) return rc;
                prof_push(kind, e0, e1);
            }
        }
        done_iters += n;
        if ((rc = check_cuda(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(CgScalars) * p->n_obs, cudaMemcpyDeviceToHost, st),
                             "read PCG state")))
            return rc;
        if ((rc = check_cuda(cudaMemcpyAsync(w->h_err, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                             "read device status")))
            return rc;
        if ((rc = check_cuda(cudaStreamSynchronize(st), "PCG sync"))) return rc;
        if (*w->h_err) return set_error(FURAX_ETIMEOUT, "a bounded device-side wait gave up during PCG");
        for (int i = 0; i < graph_timed; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, w->ev[2 * i], w->ev[2 * i + 1]) == cudaSuccess)
                prof_add(b.precision == FURAX_F64 ? 1 : 0, ms);
            else
                cudaGetLastError();
        }
        prof_flush();
        bool all = true;
        for (int o = 0; o < p->n_obs; ++o) all = all && w->h_sc[o].done;
        if (all) { *all_done = true; break; }
    }
    int it = 0;
    for (int o = 0; o < p->n_obs; ++o) it = std::max(it, (int)w->h_sc[o].iters);
    *iters_out = it;
    return FURAX_OK;
}

// rtrue = S(b - A64 x), per-observation ||rtrue||/||b|| -> host max.
static furax_status true_residual(const Body &b, const double *x, double *rtrue, double *max_rel, cudaStream_t st)
{
    CgWs *w = b.w;
    const furax_pointing *p = b.p;
    furax_status rc;
    if ((rc = check_cuda(cudaMemsetAsync(w->acc64, 0, sizeof(double) * 3 * p->npix_total, st), "memset"))) return rc;
    // The plain FP64 solve checks itself with the FP64 operator; the mixed solve with the
    // FP64-accurate double-FP32 operator (same system, ~2^-48 arithmetic, FP32 pipes).
    if (long_band(b.n)) {
        if ((rc = launch_ata_chain(p, b.n, x, FURAX_F64, w->acc64, st))) return rc;
    } else if (b.precision == FURAX_F64) {
        if ((rc = timed(1, st, [&] { return launch_fused_f64(p, b.n, x, w->acc64, st); }))) return rc;
    } else {
        if ((rc = timed(2, st, [&] { return launch_fused_df(p, b.n, x, nullptr, 0, w->acc64, st); }))) return rc;
    }
    if (b.tp && (rc = launch_tpl_map(b.tp, FURAX_F64, FURAX_ACC_F64, nullptr, x, nullptr, nullptr, w->acc64, st)))
        return rc;
    if (b.ar.on() && (rc = b.ar(w->acc64, 3 * p->npix_total, FURAX_REDUCE_F64, st))) return rc;
    residual_kernel<<<b.pg, VT, 0, st>>>(p->d_ptiles, w->bfull, w->acc64, w->valid, rtrue, w->partial);
    double *norms = w->q;   // scratch [n_obs][2] (q is free here)
    obs_norms_kernel<<<p->n_obs, VT, 0, st>>>(p->d_obs, w->partial, norms);
    count_launches(2);
    if ((rc = check_launch("true residual"))) return rc;
    std::vector<double> h(2 * p->n_obs);
    if ((rc = check_cuda(cudaMemcpyAsync(h.data(), norms, sizeof(double) * 2 * p->n_obs, cudaMemcpyDeviceToHost, st),
                         "read residual")))
        return rc;
    if ((rc = check_cuda(cudaStreamSynchronize(st), "residual sync"))) return rc;
    double m = 0.0;
    for (int o = 0; o < p->n_obs; ++o) m = std::max(m, h[2 * o + 1] > 0 ? std::sqrt(h[2 * o] / h[2 * o + 1]) : 0.0);
    *max_rel = m;
    return FURAX_OK;
}

furax_status mapmaker_cg(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, double *x,
                         uint8_t *valid_out, const furax_cg_opts *o, furax_cg_result *res, cudaStream_t st,
                         const furax_templates *tp, double *amplitudes)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    CgWs *w = nullptr;
    furax_status rc;
    if ((rc = get_ws(pm, o->maxiter + 1, &w))) return rc;
    const int64_t np = p->npix_total;
    const unsigned pg = (unsigned)std::max<int64_t>(1, p->n_ptiles);

    const AllReduce ar{o->allreduce, o->allreduce_user};
    if (ar.on() && tp) return set_error(FURAX_EINVAL, "detector sharding (allreduce) is not available with templates");
    // Preconditioner and mask (FP64 blocks from the handle's pointing; summed over the processes
    // of a sharded map before the inversion).
    if ((rc = launch_bj(p, n, o->rcond_min, w->minv, w->valid, nullptr, nullptr, st, ar))) return rc;
    // Right-hand side b = S P^T N^-1 d in FP64 (the first read of d).
    if (o->d_ready && (rc = check_cuda(cudaStreamWaitEvent(st, (cudaEvent_t)o->d_ready, 0), "wait for d")))
        return rc;
    if ((rc = check_cuda(cudaMemsetAsync(w->acc64, 0, sizeof(double) * 3 * np, st), "memset"))) return rc;
    // the double-FP32 pass from FP32 data subtracts the template correction itself, with the
    // amplitudes solved beforehand
    const bool tpl_folded = tp && !long_band(n) && o->precision != FURAX_F64 && d_t == FURAX_F32;
    if (tpl_folded && (rc = launch_tpl_rhs_amplitudes(tp, d, d_t, st))) return rc;
    if (long_band(n)) {
        // TOD workspaces exist before any stream capture of the iteration
        if ((rc = tod_ws(p))) return rc;
        if ((rc = launch_rhs_chain(p, n, d, d_t, w->acc64, st))) return rc;
    } else if (o->precision == FURAX_F64) {
        if ((rc = timed(1, st, [&] { return launch_rhs_f64(p, n, d, d_t, w->acc64, st); }))) return rc;
    } else {
        if ((rc = timed(2, st, [&] { return launch_fused_df(p, n, nullptr, d, d_t, w->acc64, st, tpl_folded ? tp : nullptr); })))
            return rc;
    }
    if (tp && !tpl_folded && (rc = launch_tpl_rhs(tp, d, d_t, w->acc64, st))) return rc;
    if (ar.on() && (rc = ar(w->acc64, 3 * np, FURAX_REDUCE_F64, st))) return rc;
    if ((rc = launch_finalize_acc(p, FURAX_ACC_F64, nullptr, nullptr, w->acc64, w->valid, w->bfull, st))) return rc;
    if (valid_out && (rc = check_cuda(cudaMemcpyAsync(valid_out, w->valid, np, cudaMemcpyDeviceToDevice, st), "copy mask")))
        return rc;

    // a long band accumulates in FP64 (its operator goes through the TOD in HBM)
    Body b{p, n, w, o->precision, long_band(n) ? FURAX_ACC_F64 : o->acc, o->tol * o->tol, x, pg, tp,
           p->d_ptiles, p->d_obs, np, false, ar};
    int total_iters = 0, outer = 0;
    bool converged = false;
    double rel = 0.0, true_rel = 0.0;

    if (o->binned_only) {
        // x = M^-1 b (the binned map): one cg_init gives z = M^-1 b.
        cg_init_kernel<<<pg, VT, 0, st>>>(p->d_ptiles, w->bfull, w->minv, w->valid, w->e, w->r, x, w->p, w->partial);
        count_launches(1);
        if ((rc = check_launch("binned map"))) return rc;
        if ((rc = true_residual(b, x, nullptr, &true_rel, st))) return rc;
        converged = true;
        rel = true_rel;
    } else if (o->precision == FURAX_F64) {
        bool all = false;
        if ((rc = pcg(b, w->bfull, o->maxiter, o->use_graph, o->check_every, st, &total_iters, &all))) return rc;
        double mr = 0.0;
        for (int i = 0; i < p->n_obs; ++i) mr = std::max(mr, w->h_sc[i].bb > 0 ? std::sqrt(w->h_sc[i].rr / w->h_sc[i].bb) : 0.0);
        rel = mr;
        if (o->true_residual) {
            if ((rc = true_residual(b, x, nullptr, &true_rel, st))) return rc;
        } else {
            true_rel = -1.0;
        }
        converged = all;
        outer = 0;
    } else {
        // Defect correction: x = 0, r = b; repeat { inner PCG on A32 e = r; x += e; r = S(b - A64 x) }.
        // The inner solve reads its right-hand side once (cg_init, in place when it is w->r).
        if ((rc = check_cuda(cudaMemsetAsync(x, 0, sizeof(double) * 3 * np, st), "memset"))) return rc;
        true_rel = 1.0;
        Body bi = b;
        bi.x = w->e;
        bi.tol2 = o->inner_tol * o->inner_tol;
        const int64_t npseudo = 3 * p->ndet_total;   // amplitude entries of the augmented system
        if (tpl_augmented(tp, o->precision)) {
            bi.aug = true;
            bi.pt = tp->d_aug_ptiles;
            bi.cobs = tp->d_aug_obs;
            bi.pg = (unsigned)std::max<int64_t>(1, tp->n_aug_ptiles);
            bi.np_cg = np + p->ndet_total;
            if ((rc = launch_tpl_aug_precond(tp, w->minv, w->valid, st))) return rc;
            if ((rc = check_cuda(cudaMemsetAsync(w->bfull + 3 * np, 0, sizeof(double) * npseudo, st), "memset")))
                return rc;
        }
        while (outer < o->max_outer && total_iters < o->maxiter) {
            const double *rhs_in = outer == 0 ? w->bfull : w->r;
            // the augmented right-hand side is [r; 0]: r's amplitude part holds the last inner residual
            if (bi.aug && outer > 0 &&
                (rc = check_cuda(cudaMemsetAsync(w->r + 3 * np, 0, sizeof(double) * npseudo, st), "memset")))
                return rc;
            int it = 0;
            bool all = false;
            if ((rc = pcg(bi, rhs_in, o->maxiter - total_iters, o->use_graph, o->check_every, st, &it, &all))) return rc;
            total_iters += it;
            double mr = 0.0;
            for (int i = 0; i < p->n_obs; ++i)
                mr = std::max(mr, w->h_sc[i].bb > 0 ? std::sqrt(w->h_sc[i].rr / w->h_sc[i].bb) : 0.0);
            axpy_kernel<<<vgrid(p, 3 * np), VT, 0, st>>>(x, w->e, 3 * np);
            count_launches(1);
            if ((rc = check_launch("defect correction update"))) return rc;
            ++outer;
            if (!o->true_residual && (outer >= o->max_outer || total_iters >= o->maxiter)) {
                // last pass and no residual requested: report the inner recursive residual
                true_rel = -1.0;
                rel = mr;
                break;
            }
            if ((rc = true_residual(b, x, w->r, &true_rel, st))) return rc;
            rel = true_rel;
            if (true_rel <= o->tol) { converged = true; break; }
            if (it == 0) break;
        }
    }
    if (tp && amplitudes && (rc = tpl_amplitudes(tp, d, d_t, x, amplitudes, st))) return rc;
    res->iters = total_iters;
    res->outer = outer;
    res->rel_res = rel;
    res->true_rel_res = true_rel;
    // valid count and history
    {
        std::vector<uint8_t> hv(np);
        if ((rc = check_cuda(cudaMemcpyAsync(hv.data(), w->valid, np, cudaMemcpyDeviceToHost, st), "read mask"))) return rc;
        if (res->hist && res->hist_len > 0) {
            const int nh = std::min<int>(res->hist_len, std::min(w->hist_cap, total_iters + 1));
            if ((rc = check_cuda(cudaMemcpyAsync(res->hist, w->hist, sizeof(double) * nh, cudaMemcpyDeviceToHost, st),
                                 "read history")))
                return rc;
            res->hist_written = nh;
        } else {
            res->hist_written = 0;
        }
        if ((rc = check_cuda(cudaMemcpyAsync(w->h_err, p->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                             "read device status")))
            return rc;
        if ((rc = check_cuda(cudaStreamSynchronize(st), "final sync"))) return rc;
        if (*w->h_err) return set_error(FURAX_ETIMEOUT, "a bounded device-side wait gave up");
        int64_t nv = 0;
        for (int64_t i = 0; i < np; ++i) nv += hv[i];
        res->n_valid = nv;
        if (nv == 0) return set_error(FURAX_EBADINPUT, "no pixel passes the preconditioner validity test");
    }
    return converged ? FURAX_OK : FURAX_ENOTCONVERGED;
}

}  // namespace fx
