// Persistent, TMA-pipelined FP32 operator acc += P^T N^-1 P x32 for the cached FP32
// pointing (the hot path of the map-making PCG: the estimator A = (H.T @ N.I @ H).I @ H.T @ N.I
// of the Furax paper's Software Design listing, with the per-detector block decomposition of
// "Algebraic reductions").
//
// One CTA per SM walks the tile list (one detector x up to TILE samples per tile) with stride
// gridDim.x. Three warp roles hand tiles to each other through shared-memory rings guarded by
// mbarriers:
//   loader (1 warp, 1 thread): bulk-copies (cp.async.bulk, completion counted in bytes on an
//     mbarrier) the cached pixel index and FP32 weights of the tile and its 63-sample halos
//     into one of kRawStages stages, up to kRawStages - 1 tiles ahead of the consumers;
//   gather (7 warps): reads a landed stage, gathers the map values of the tile's pixels from
//     the FP32 map in L2 (all loads of a thread issued before any is used) and writes the
//     projected samples P x into one of kXsStages stages;
//   consumer (8 or 16 warps): applies N^-1 (the 127-term symmetric band, consecutive outputs per
//     thread from a sliding register window), writes y over the consumed stage and scatters
//     y (1, cos 2psi, sin 2psi), lane-consecutive in time: one 16-byte FP32 L2 reduction per
//     sample, the compensated pair of ACC_F32_KAHAN, or, for ACC_F64, three FP64 reductions per
//     sample that the warp issues as whole 24-byte pixel records (red_add_f64_records_warp).
// Shared memory is kept near 138 KB: the rest of the SM's L1/shared array is L1, where the
// gathers' misses in flight are staged.
// The pointing stream is read from HBM exactly once (plus 126 halo samples per tile); the map
// and the accumulators stay in L2. Every wait is bounded: a wait that gives up sets the error
// word and the role leaves its loop; the loader waits (bounded) for its own copies in flight
// before it exits.
#include "tile.cuh"
#include "mbarrier.cuh"

namespace fx {

constexpr int kTmaGather = 7;                      // gather warps
// Consumer warps KC (a template parameter: 8 or 16, chosen by the schedule): each consumer thread
// owns TILE / (32 KC) consecutive outputs of the band; with 16 the scatter has twice the
// threads (and returning atomics) in flight and the band product half the outputs per thread.
template <int KC> constexpr int cons_out() { return TILE / (32 * KC); }
template <int KC> constexpr int tma_threads() { return 32 * (kTmaGather + KC + 1); }
constexpr int kRawStages = 2;
constexpr int kXsStages = 2;
// Elements of one pointing stream copied per tile: tile + halos, widened to 16-byte boundaries.
constexpr int kRawN = 4232;
static_assert(kRawN % 4 == 0 && kRawN >= TILE + 2 * kHalo + 6, "raw stage must hold an aligned tile + halos");
constexpr int kGatherPer = (TILE + 2 * kHalo + 32 * kTmaGather - 1) / (32 * kTmaGather);
constexpr int kKahanBatch = 4;                     // returning atomics in flight per consumer thread
static_assert(cons_out<16>() % kKahanBatch == 0 && cons_out<8>() % kKahanBatch == 0,
              "Kahan batches tile a thread's outputs");

struct TmaSmem {
    int32_t pix[kRawStages][kRawN];
    float c[kRawStages][kRawN];
    float s[kRawStages][kRawN];
    float xs[kXsStages][XS];
    alignas(16) float taps[kXsStages][2 * kBandPad];   // band in tap order as (c_|j-63|, c_|j-63|) pairs
    alignas(16) float4 amp[kRawStages];                // TPL 2: the tile detector's template amplitudes
    uint64_t raw_full[kRawStages], raw_empty[kRawStages], xs_full[kXsStages], xs_empty[kXsStages];
};
constexpr size_t kTmaSmem = sizeof(TmaSmem);
// ACC_F64: behind the ring, one staging area per consumer warp for the record-wise FP64
// reductions (96 values + 32 pixel indices).
constexpr int kXchWords = 128;
template <int ACC, int KC> constexpr size_t tma_smem()
{
    return kTmaSmem + (ACC == FURAX_ACC_F64 ? sizeof(float) * kXchWords * KC : 0);
}
// The SM's L1 cache and shared memory share one array, and global-load misses in flight are
// staged in L1: the map gathers need at most ~150 KB of shared memory per SM to keep their
// full rate (measured: a 206 KB reservation halves it).
static_assert(tma_smem<FURAX_ACC_F64, 16>() <= 150 * 1024, "leave L1 room for the gathers in flight");
static_assert(sizeof(int32_t) * kRawN % 16 == 0, "stage arrays stay 16-byte aligned");

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy; completion is signalled on `bar` as transferred bytes.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// AND of `ok` over the 32 KC consumer threads (named barrier 1); every consumer thread must call it.
template <int KC>
__device__ __forceinline__ bool consumers_all(bool ok)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)ok), "n"(32 * KC)
        : "memory");
    return r != 0;
}

template <int KC>
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(32 * KC) : "memory");
}

// Tile geometry in the flat cache: the copied range [g0, g0 + n) covers every in-stream sample
// of the tile and its halos; sample t of the detector sits at stage index row + t - g0.
struct TileSpan {
    int64_t row, g0;
    int32_t n;
};

__device__ __forceinline__ TileSpan tile_span(const Tile &tl, const ObsInfo &ob, int halo)
{
    TileSpan sp;
    sp.row = ob.tod_off + (int64_t)tl.det * ob.nsamp;
    const int64_t t_lo = tl.t0 - halo > 0 ? tl.t0 - halo : 0;
    const int64_t t_hi = tl.t0 + tl.len + halo < ob.nsamp ? tl.t0 + tl.len + halo : ob.nsamp;
    sp.g0 = (sp.row + t_lo) & ~int64_t(3);
    const int64_t g1 = (sp.row + t_hi + 3) & ~int64_t(3);
    sp.n = (int32_t)(g1 - sp.g0);
    return sp;
}

// Template work (T = Legendre P_0.. of tau_t = 2t/(ns-1) - 1 per detector, z = N^-1 u of the
// tile's samples):
//   TPL 1: the consumers add T^T z (P_0..P_3) to tpl.proj[det][4], the projection of the
//          template-deprojected operator, which then needs no pass of its own;
//   TPL 2: the augmented system [m; a]: u_t = (P m)_t + sum_l a_l P_l(tau_t) with the detector's
//          amplitudes a (l <= 2) read from x32[tpl.base + det], and T^T z (l <= tpl.order)
//          accumulated into the amplitude pseudo-pixel tpl.base + det like a pixel.
template <int ACC, bool BANDED, int TPL, int KC>
__global__ void __launch_bounds__(tma_threads<KC>(), 1)
    fused_tma_kernel(const Tile *__restrict__ tiles, int64_t n_tiles, PointingView pv, NoiseView nv,
                     const float4 *__restrict__ x32, float4 *__restrict__ acc_hi, float4 *__restrict__ acc_lo,
                     double *__restrict__ acc64, unsigned *__restrict__ err, FusedTpl tpl, int l2_hint)
{
    constexpr int kTmaConsumer = KC;
    constexpr int kConsOut = cons_out<KC>();
    extern __shared__ __align__(128) unsigned char tsm[];
    TmaSmem &S = *reinterpret_cast<TmaSmem *>(tsm);
    constexpr int halo = BANDED ? kHalo : 0;
    const int warp = threadIdx.x >> 5;
    const long long budget = wait_budget(err);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kRawStages; ++i) { mbar_init(&S.raw_full[i], 1); mbar_init(&S.raw_empty[i], 32 * kTmaConsumer); }
        for (int i = 0; i < kXsStages; ++i) { mbar_init(&S.xs_full[i], 32 * kTmaGather); mbar_init(&S.xs_empty[i], 32 * kTmaConsumer); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kTmaGather + kTmaConsumer) {
        // ---------------- loader
        if ((threadIdx.x & 31) != 0) return;
        // held (test hook): issue nothing; the gather and consumer waits then run out
        if (loader_held(err)) return;
        const bool hint = l2_hint != 0;   // the pointing stream is read once: evict it first
        const uint64_t pol = hint ? evict_first_policy() : 0ull;
        int64_t it = 0;
        for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x, ++it) {
            const int r = (int)(it % kRawStages);
            const uint32_t par = (uint32_t)((it / kRawStages) & 1);
            if (!mbar_wait(&S.raw_empty[r], par ^ 1u, err, budget)) break;
            const Tile tl = tiles[ti];
            const ObsInfo ob = pv.obs[tl.obs];
            const TileSpan sp = tile_span(tl, ob, halo);
            const uint32_t bytes = (uint32_t)sp.n * 4u;
            mbar_expect_tx(&S.raw_full[r], 3u * bytes + (TPL == 2 ? (uint32_t)sizeof(float4) : 0u));
            bulk_copy_g2s(S.pix[r], pv.pix + sp.g0, bytes, &S.raw_full[r], hint, pol);
            bulk_copy_g2s(S.c[r], pv.c32 + sp.g0, bytes, &S.raw_full[r], hint, pol);
            bulk_copy_g2s(S.s[r], pv.s32 + sp.g0, bytes, &S.raw_full[r], hint, pol);
            // the tile detector's amplitudes ride on the same barrier (16 bytes, 16-byte aligned)
            if constexpr (TPL == 2)
                bulk_g2s(&S.amp[r], x32 + tpl.base + ob.det_off + tl.det, (uint32_t)sizeof(float4), &S.raw_full[r]);
        }
        // Copies into a stage complete its current phase; wait for the last one issued into each
        // stage so that no copy is still writing when the CTA exits.
        for (int64_t j = it - 1; j >= 0 && j >= it - kRawStages; --j)
            mbar_wait(&S.raw_full[j % kRawStages], (uint32_t)((j / kRawStages) & 1), err, budget);
        return;
    }

    if (warp < kTmaGather) {
        // ---------------- gather: xs = P x over the tile and its halos
        const int tid = threadIdx.x;
        int64_t it = 0;
        for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x, ++it) {
            const int r = (int)(it % kRawStages);
            const int q = (int)(it % kXsStages);
            if (!mbar_wait(&S.xs_empty[q], (uint32_t)(((it / kXsStages) & 1) ^ 1), err, budget)) break;
            if (!mbar_wait(&S.raw_full[r], (uint32_t)((it / kRawStages) & 1), err, budget)) break;
            const Tile tl = tiles[ti];
            const ObsInfo ob = pv.obs[tl.obs];
            const int64_t gdet = ob.det_off + tl.det;
            const TileSpan sp = tile_span(tl, ob, halo);
            if (BANDED && tid < kBandPad) {
                const int k = tid < kHalo ? kHalo - tid : tid - kHalo;
                const float c = (tid < kBand && k < nv.ntaps) ? nv.p32[gdet * nv.ntaps + k] : 0.f;
                reinterpret_cast<float2 *>(S.taps[q])[tid] = make_float2(c, c);
            }
            const int nload = tl.len + 2 * halo;
            const int64_t t_first = tl.t0 - halo;
            const int64_t shift = sp.row + t_first - sp.g0;   // stage index of u is u + shift
            const int32_t *spix = S.pix[r];
            float4 m[kGatherPer];
#pragma unroll
            for (int k = 0; k < kGatherPer; ++k) {
                const int u = tid + k * 32 * kTmaGather;
                const int64_t t = t_first + u;
                const int32_t pix = (u < nload && t >= 0 && t < ob.nsamp) ? spix[u + shift] : -1;
                m[k] = pix >= 0 ? __ldg(x32 + ob.map_off + pix) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            double2 cs = make_double2(1.0, 0.0);
            if (pv.psi_cs) cs = pv.psi_cs[gdet];
#pragma unroll
            for (int k = 0; k < kGatherPer; ++k) {
                const int u = tid + k * 32 * kTmaGather;
                const int64_t t = t_first + u;
                if (u < nload) {
                    float v = 0.f;
                    if (t >= 0 && t < ob.nsamp && spix[u + shift] >= 0) {
                        float c = S.c[r][u + shift], s = S.s[r][u + shift];
                        if (pv.psi_cs) rotate_psi<float>(c, s, cs);
                        v = fmaf(m[k].z, s, fmaf(m[k].y, c, m[k].x));
                    }
                    S.xs[q][spos(u)] = v;
                }
            }
            if constexpr (TPL == 2) {
                // the templates act on every sample of the stream; a second pass over this
                // thread's own slots keeps the loads above free of extra live registers
                const float4 amp = S.amp[r];
                const float h = ob.nsamp > 1 ? 2.f / (float)(ob.nsamp - 1) : 0.f;
                const float tau0 = ob.nsamp > 1 ? (float)t_first * h - 1.f : 0.f;
                // (float)u without a conversion per sample: tid and the loop's strides convert
                // exactly (integers below 2^24), so their FP32 sum is (float)u exactly
                const float tidf = (float)tid;
#pragma unroll 4
                for (int k = 0; k < kGatherPer; ++k) {
                    const int u = tid + k * 32 * kTmaGather;
                    const int64_t t = t_first + u;
                    if (u < nload && t >= 0 && t < ob.nsamp) {
                        const float tau = fmaf(tidf + (float)(k * 32 * kTmaGather), h, tau0);
                        S.xs[q][spos(u)] += fmaf(amp.z, 1.5f * tau * tau - 0.5f, fmaf(amp.y, tau, amp.x));
                    }
                }
            }
            mbar_arrive(&S.xs_full[q]);
        }
        return;
    }

    // ---------------- consumer: y = N^-1 xs, then acc[pix] += y (1, c, s)
    const int tid = threadIdx.x - 32 * kTmaGather;
    int64_t it = 0;
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x, ++it) {
        const int r = (int)(it % kRawStages);
        const int q = (int)(it % kXsStages);
        const bool ok = mbar_wait(&S.xs_full[q], (uint32_t)((it / kXsStages) & 1), err, budget);
        const Tile tl = tiles[ti];
        const ObsInfo ob = pv.obs[tl.obs];
        const int64_t gdet = ob.det_off + tl.det;
        const int base = tid * kConsOut;
        float y[kConsOut];
        if (ok && base < tl.len) {
            if constexpr (BANDED) {
                band_product_x2<kConsOut>(S.xs[q], S.taps[q], base, y);
            } else {
                const float w = white_scale<float>(nv, gdet);
#pragma unroll
                for (int i = 0; i < kConsOut; ++i) y[i] = S.xs[q][spos(base + i)] * w;
            }
        }
        // Every consumer has read its stencil inputs: y overwrites the stage in place (core
        // sample u at slot spos(u)), which is released to the gathers after the scatter.
        if (!consumers_all<KC>(ok)) break;
        if constexpr (TPL != 0) {
            float a[4] = {0.f, 0.f, 0.f, 0.f};
            if (base < tl.len) {
                const float h = ob.nsamp > 1 ? 2.f / (float)(ob.nsamp - 1) : 0.f;
                // one 64-bit conversion per thread instead of one per output (64-bit integer
                // conversions run on the FP64 pipe); for t < 2^24 tb + i is (float)t exactly
                const float tb = (float)(tl.t0 + base);
#pragma unroll
                for (int i = 0; i < kConsOut; ++i) {
                    if (base + i >= tl.len) break;
                    const float tau = ob.nsamp > 1 ? (tb + (float)i) * h - 1.f : 0.f;
                    a[0] += y[i];
                    a[1] += tau * y[i];
                    a[2] += (1.5f * tau * tau - 0.5f) * y[i];
                    a[3] += tau * (2.5f * tau * tau - 1.5f) * y[i];
                }
            }
#pragma unroll
            for (int l = 0; l < 4; ++l)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a[l] += __shfl_down_sync(0xffffffffu, a[l], o);
            if ((threadIdx.x & 31) == 0) {
                if constexpr (TPL == 1) {
#pragma unroll
                    for (int l = 0; l < 4; ++l) red_add_f64(tpl.proj + 4 * gdet + l, (double)a[l]);
                } else {
                    const float4 v = make_float4(a[0], tpl.order >= 1 ? a[1] : 0.f, tpl.order >= 2 ? a[2] : 0.f, 0.f);
                    const int64_t gp = tpl.base + gdet;
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
        }
        float *ys = S.xs[q];
#pragma unroll
        for (int i = 0; i < kConsOut; ++i)
            if (base + i < tl.len) ys[spos(base + i)] = y[i];
        consumers_sync<KC>();
        const TileSpan sp = tile_span(tl, ob, halo);
        const int64_t shift = sp.row + tl.t0 - sp.g0;   // stage index of core sample u
        double2 cs = make_double2(1.0, 0.0);
        if (pv.psi_cs) cs = pv.psi_cs[gdet];
        if constexpr (ACC == FURAX_ACC_F32_KAHAN) {
            // The compensation needs each atomic's old value: issue kKahanBatch returning atomics
            // back to back, then their error reductions, so that a thread has a batch in flight
            // instead of one round trip per sample.
#pragma unroll
            for (int k0 = 0; k0 < kConsOut; k0 += kKahanBatch) {
                float4 old[kKahanBatch];
                float3 v[kKahanBatch];
                int32_t px[kKahanBatch];
#pragma unroll
                for (int b = 0; b < kKahanBatch; ++b) {
                    const int u = tid + (k0 + b) * 32 * kTmaConsumer;
                    px[b] = u < tl.len ? S.pix[r][u + shift] : -1;
                    if (px[b] >= 0) {
                        float c = S.c[r][u + shift], s = S.s[r][u + shift];
                        if (pv.psi_cs) rotate_psi<float>(c, s, cs);
                        const float yv = ys[spos(u)];
                        v[b] = make_float3(yv, yv * c, yv * s);
                        old[b] = atom_add_v4(acc_hi + kKahanStride * (ob.map_off + px[b]),
                                             make_float4(v[b].x, v[b].y, v[b].z, 0.f));
                    }
                }
#pragma unroll
                for (int b = 0; b < kKahanBatch; ++b)
                    if (px[b] >= 0)
                        red_add_v4(acc_lo + kKahanStride * (ob.map_off + px[b]),
                                   kahan_error_v4(old[b], make_float4(v[b].x, v[b].y, v[b].z, 0.f)));
            }
        } else if constexpr (ACC == FURAX_ACC_F64) {
            // three FP64 reductions per sample, issued as whole pixel records by the warp through
            // its staging area behind the ring (lanes past the tile offer pix = -1; the stage
            // entries they read are in bounds and unused)
            double *base = acc64 + 3 * ob.map_off;
            float *xv = reinterpret_cast<float *>(tsm + kTmaSmem) + (tid >> 5) * kXchWords;
            int32_t *xp = reinterpret_cast<int32_t *>(xv + 96);
#pragma unroll 4
            for (int k = 0; k < kConsOut; ++k) {
                const int u = tid + k * 32 * kTmaConsumer;
                const bool in = u < tl.len;
                const int32_t pix = in ? S.pix[r][u + shift] : -1;
                float c = S.c[r][u + shift], s = S.s[r][u + shift];
                if (pv.psi_cs) rotate_psi<float>(c, s, cs);
                const float y0 = in ? ys[spos(u)] : 0.f;
                const float v[3] = {y0, y0 * c, y0 * s};
                red_add_f64_records_warp<3, float>(base, pix, v, xv, xp);
            }
        } else {
#pragma unroll 4
            for (int k = 0; k < kConsOut; ++k) {
                const int u = tid + k * 32 * kTmaConsumer;
                if (u >= tl.len) break;
                const int32_t pix = S.pix[r][u + shift];
                if (pix < 0) continue;
                float c = S.c[r][u + shift], s = S.s[r][u + shift];
                if (pv.psi_cs) rotate_psi<float>(c, s, cs);
                const float yv = ys[spos(u)];
                red_add_v4(acc_hi + ob.map_off + pix, make_float4(yv, yv * c, yv * s, 0.f));
            }
        }
        mbar_arrive(&S.xs_empty[q]);
        mbar_arrive(&S.raw_empty[r]);
    }
}

template <int ACC, bool BANDED, int TPL, int KC>
static furax_status run_tma_kc(const furax_pointing *p, const furax_noise *n, const float4 *x32, float4 *hi,
                               float4 *lo, double *a64, const FusedTpl &ft, cudaStream_t st)
{
    const unsigned g = (unsigned)std::min<int64_t>(p->n_tiles, p->n_sm);
    return launch_dyn(fused_tma_kernel<ACC, BANDED, TPL, KC>, g, tma_threads<KC>(), tma_smem<ACC, KC>(), st, p->d_tiles,
                      p->n_tiles, p->view(), n->view(), x32, hi, lo, a64, p->d_err, ft, (int)p->sched.l2_evict_first);
}

// 16 consumer warps when the schedule asks for them (plain operator only; the template modes keep 8).
template <int ACC, bool BANDED, int TPL>
static furax_status run_tma(const furax_pointing *p, const furax_noise *n, const float4 *x32, float4 *hi, float4 *lo,
                            double *a64, const FusedTpl &ft, cudaStream_t st)
{
    if constexpr (TPL == 0)
        if (p->sched.consumer_warps == 16) return run_tma_kc<ACC, BANDED, TPL, 16>(p, n, x32, hi, lo, a64, ft, st);
    return run_tma_kc<ACC, BANDED, TPL, 8>(p, n, x32, hi, lo, a64, ft, st);
}

template <bool BANDED, int TPL>
static furax_status dispatch_tma(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc, float4 *hi,
                                 float4 *lo, double *a64, const FusedTpl &ft, cudaStream_t st)
{
    if (acc == FURAX_ACC_F32) return run_tma<FURAX_ACC_F32, BANDED, TPL>(p, n, x32, hi, lo, a64, ft, st);
    if (acc == FURAX_ACC_F32_KAHAN) return run_tma<FURAX_ACC_F32_KAHAN, BANDED, TPL>(p, n, x32, hi, lo, a64, ft, st);
    return run_tma<FURAX_ACC_F64, BANDED, TPL>(p, n, x32, hi, lo, a64, ft, st);
}

template <int TPL>
static furax_status dispatch_tma_band(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc,
                                      float4 *hi, float4 *lo, double *a64, const FusedTpl &ft, cudaStream_t st)
{
    return n->kind == FURAX_NOISE_BANDED ? dispatch_tma<true, TPL>(p, n, x32, acc, hi, lo, a64, ft, st)
                                         : dispatch_tma<false, TPL>(p, n, x32, acc, hi, lo, a64, ft, st);
}

furax_status launch_fused_tma(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc, float4 *hi,
                              float4 *lo, double *a64, cudaStream_t st, const FusedTpl *ft)
{
    const FusedTpl none{0, nullptr, 0, 0};
    if (!ft || ft->mode == 0) return dispatch_tma_band<0>(p, n, x32, acc, hi, lo, a64, none, st);
    if (ft->mode == 1) return dispatch_tma_band<1>(p, n, x32, acc, hi, lo, a64, *ft, st);
    return dispatch_tma_band<2>(p, n, x32, acc, hi, lo, a64, *ft, st);
}

template <bool BANDED, int TPL, int KC>
static furax_status prepare_tma_band()
{
    furax_status rc = FURAX_OK;
    if (!rc) rc = allow_smem((const void *)fused_tma_kernel<FURAX_ACC_F32, BANDED, TPL, KC>, tma_smem<FURAX_ACC_F32, KC>());
    if (!rc) rc = allow_smem((const void *)fused_tma_kernel<FURAX_ACC_F32_KAHAN, BANDED, TPL, KC>, tma_smem<FURAX_ACC_F32_KAHAN, KC>());
    if (!rc) rc = allow_smem((const void *)fused_tma_kernel<FURAX_ACC_F64, BANDED, TPL, KC>, tma_smem<FURAX_ACC_F64, KC>());
    return rc;
}

furax_status prepare_fused_tma()
{
    furax_status rc = FURAX_OK;
    if (!rc) rc = prepare_tma_band<true, 0, 8>();
    if (!rc) rc = prepare_tma_band<false, 0, 8>();
    if (!rc) rc = prepare_tma_band<true, 0, 16>();
    if (!rc) rc = prepare_tma_band<false, 0, 16>();
    if (!rc) rc = prepare_tma_band<true, 1, 8>();
    if (!rc) rc = prepare_tma_band<false, 1, 8>();
    if (!rc) rc = prepare_tma_band<true, 2, 8>();
    if (!rc) rc = prepare_tma_band<false, 2, 8>();
    return rc;
}

}  // namespace fx
