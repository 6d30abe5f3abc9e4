// Pixel-sorted FP32 operator acc += P^T N^-1 P x32 for the cached FP32 pointing.
//
// The block decomposition P^T N^-1 P = sum_i P_i^T N_i^-1 P_i of the Furax paper ("Algebraic
// reductions") is taken over tiles chosen so that their samples share pixels: the detectors of a
// tile lie on one circle about the instantaneous rotation axis of the scan (for a spinning
// satellite, one column of the focal plane along the scan), so they follow the same track on the
// sky a few samples apart, and a tile covers tile_len consecutive samples of each. Once per
// pointing refresh the gathered samples of every tile (core samples and the band's halos) are
// sorted by pixel (sort_tiles_kernel). The operator then
//   gathers x[pix] in sorted order: lanes of a warp that hold the same pixel issue the same address,
//     which the memory system serves with one request;
//   applies N^-1 per detector row in time order (the 127-term band, taps read from global memory);
//   accumulates in sorted order: the first sample of each run of equal pixels sums the run's
//     core contributions (compensated in FURAX_ACC_F32_KAHAN and FURAX_ACC_F64) and issues one
//     reduction (one compensated pair) for the whole run.
// On the 256-detector scan this halves the random L2 reductions per sample and cuts the random
// gathers by about 30 %; the pointing stream is read once (halos of neighbouring tiles hit in L2).
//
// Pipeline (one persistent CTA per SM, roles joined by mbarrier rings with bounded waits, as in
// fused_tma.cu): a loader thread bulk-copies each row's cached pixels and weights (with halos,
// widened to 16-byte boundaries) and the tile's permutation; 7 gather warps build P x; 8 consumer
// warps run the band and the run-wise scatter.
#include <cmath>
#include <algorithm>
#include <numeric>

#include "tile.cuh"
#include "mbarrier.cuh"
#include "dfloat.cuh"

namespace fx {

constexpr int kSGather = 7;
constexpr int kSConsumer = 8;
constexpr int kSThreads = 32 * (kSGather + kSConsumer + 1);
constexpr int kSXS = spos(kSNE + 32) + 1;                              // band reads run up to 16 past a row
constexpr int kSGatherPer = (kSNE + 32 * kSGather - 1) / (32 * kSGather);
constexpr int kSConsPer = kSNE / (32 * kSConsumer);                    // permutation entries per consumer thread
constexpr int kSKahanBatch = 4;                                        // returning atomics in flight per thread
constexpr int kSCore0 = 3 + 63;                                        // stage position of a row's first core sample
constexpr int kSortThreads = 512;
static_assert(kSNE == 4096 && kSRowMax <= 16, "permutation entries hold a 12-bit position and a 4-bit row");
static_assert(kSConsPer % kSKahanBatch == 0, "Kahan batches tile a thread's entries");

struct SRow {
    int32_t delta;   // raw stage position - band stage position of the row's samples
    int32_t gdet;    // global detector index
};

struct SortedSmem {
    int32_t pix[2][kSNE];
    float c[2][kSNE];
    float s[2][kSNE];
    uint16_t perm[2][kSNE];
    float xs[2][kSXS];
    SRow row[2][kSRowMax];
    int32_t nperm[2];
    uint64_t raw_full[2], raw_empty[2], xs_full[2], xs_empty[2];
};
constexpr size_t kSortedSmem = sizeof(SortedSmem);
static_assert(kSortedSmem <= 150 * 1024, "leave L1 room for the gathers in flight");

__device__ __forceinline__ void smbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool sconsumers_all(bool ok)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)ok), "n"(32 * kSConsumer)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void sconsumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kSConsumer) : "memory"); }
__device__ __forceinline__ void sgathers_sync() { asm volatile("bar.sync 2, %0;" ::"n"(32 * kSGather) : "memory"); }

// AND of `ok` over the gather threads (named barrier 3): a thread whose bounded wait gave up leaves
// together with the others, so none is left at the gathers' own barrier.
__device__ __forceinline__ bool sgathers_all(bool ok)
{
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 3, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)ok), "n"(32 * kSGather)
        : "memory");
    return r != 0;
}

// The copied range of one row: global cache indices [g0, g0 + n), 16-byte aligned, covering the
// in-stream samples of [t0 - 63, t0 + len + 63).
struct SRowSpan {
    int64_t g0;
    int32_t n;
    int32_t delta;
};

__device__ __forceinline__ SRowSpan srow_span(const STile &tl, const ObsInfo &ob, int32_t det)
{
    const int64_t row_start = ob.tod_off + (int64_t)det * ob.nsamp;
    const int64_t t_lo = tl.t0 - 63 > 0 ? tl.t0 - 63 : 0;
    const int64_t t_hi = tl.t0 + tl.len + 63 < ob.nsamp ? tl.t0 + tl.len + 63 : ob.nsamp;
    SRowSpan sp;
    sp.g0 = (row_start + t_lo) & ~int64_t(3);
    sp.n = (int32_t)(((row_start + t_hi + 3) & ~int64_t(3)) - sp.g0);
    // band position of time t: 3 + t - t0 + 63; raw position: row_start + t - g0
    sp.delta = (int32_t)(row_start + tl.t0 - kSCore0 - sp.g0);
    return sp;
}

// One CTA per tile: the tile's gathered samples with a valid pixel, sorted by (pixel, row, position).
__global__ void __launch_bounds__(kSortThreads) sort_tiles_kernel(const STile *__restrict__ tiles,
                                                                  const ObsInfo *__restrict__ obs,
                                                                  const int32_t *__restrict__ sdet,
                                                                  const int32_t *__restrict__ pix,
                                                                  uint16_t *__restrict__ perm, int32_t *__restrict__ perm_n)
{
    __shared__ unsigned long long key[kSNE];
    __shared__ int cnt;
    const STile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const int64_t t_lo = tl.t0 - 63 > 0 ? tl.t0 - 63 : 0;
    const int64_t t_hi = tl.t0 + tl.len + 63 < ob.nsamp ? tl.t0 + tl.len + 63 : ob.nsamp;
    const int span = (int)(t_hi - t_lo);
    for (int r = 0; r < tl.nrow; ++r) {
        const int64_t row_start = ob.tod_off + (int64_t)sdet[tl.det0 + r] * ob.nsamp;
        for (int k = threadIdx.x; k < span; k += kSortThreads) {
            const int64_t t = t_lo + k;
            const int32_t p = pix[row_start + t];
            if (p >= 0) {
                const int slot = atomicAdd(&cnt, 1);
                const unsigned pos = (unsigned)(3 + t - tl.t0 + 63);   // < row stride <= 4096
                key[slot] = ((unsigned long long)(unsigned)p << 16) | ((unsigned long long)r << 12) | pos;
            }
        }
    }
    __syncthreads();
    const int n = cnt;   // <= nrow (len + 126) < kSNE
    for (int k = n + threadIdx.x; k < kSNE; k += kSortThreads) key[k] = ~0ull;
    __syncthreads();
    // bitonic sort of kSNE keys, ascending
    for (int k = 2; k <= kSNE; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < kSNE; i += kSortThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = key[i], b = key[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { key[i] = b; key[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < n; k += kSortThreads) perm[tl.perm_off + k] = (uint16_t)(key[k] & 0xffffu);
    if (threadIdx.x == 0) perm_n[blockIdx.x] = n;
}

// Decoded permutation entry: band position X (xs), raw position R (pix, c, s), row.
struct SEntry {
    int X, R, row;
};

__device__ __forceinline__ SEntry sdecode(const SortedSmem &S, int st, int rs, uint16_t e)
{
    SEntry d;
    d.row = e >> 12;
    d.X = d.row * rs + (e & 0xfff);
    d.R = d.X + S.row[st][d.row].delta;
    return d;
}

template <int ACC, bool BANDED>
__global__ void __launch_bounds__(kSThreads, 1)
    fused_sorted_kernel(const STile *__restrict__ tiles, int64_t n_tiles, const int32_t *__restrict__ sdet,
                        const uint16_t *__restrict__ perm, const int32_t *__restrict__ perm_n, PointingView pv,
                        NoiseView nv, const float4 *__restrict__ x32, float4 *__restrict__ acc_hi,
                        float4 *__restrict__ acc_lo, double *__restrict__ acc64, unsigned *__restrict__ err,
                        int l2_hint)
{
    extern __shared__ __align__(128) unsigned char ssm[];
    SortedSmem &S = *reinterpret_cast<SortedSmem *>(ssm);
    const int warp = threadIdx.x >> 5;
    const long long budget = wait_budget(err);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&S.raw_full[i], 1);
            mbar_init(&S.raw_empty[i], 32 * kSConsumer);
            mbar_init(&S.xs_full[i], 32 * kSGather);
            mbar_init(&S.xs_empty[i], 32 * kSConsumer);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kSGather + kSConsumer) {
        // ---------------- loader: rows' pixels and weights (with halos) and the tile's permutation
        if ((threadIdx.x & 31) != 0) return;
        if (loader_held(err)) return;
        const bool hint = l2_hint != 0;   // the pointing stream and permutation are read once
        const uint64_t pol = hint ? evict_first_policy() : 0ull;
        int64_t it = 0;
        for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x, ++it) {
            const int r = (int)(it & 1);
            if (!mbar_wait(&S.raw_empty[r], (uint32_t)(((it >> 1) & 1) ^ 1), err, budget)) break;
            const STile tl = tiles[ti];
            const ObsInfo ob = pv.obs[tl.obs];
            const int rs = srow_stride(tl.len);
            uint32_t bytes = 0;
            for (int row = 0; row < tl.nrow; ++row) {
                const int32_t det = sdet[tl.det0 + row];
                const SRowSpan sp = srow_span(tl, ob, det);
                S.row[r][row] = SRow{sp.delta, (int32_t)(ob.det_off + det)};
                bytes += 3u * 4u * (uint32_t)sp.n;
            }
            const int32_t np = perm_n[ti];
            S.nperm[r] = np;
            const uint32_t pbytes = ((uint32_t)np * 2u + 15u) & ~15u;
            smbar_expect_tx(&S.raw_full[r], bytes + pbytes);   // release: the row table above is visible
            for (int row = 0; row < tl.nrow; ++row) {
                const SRowSpan sp = srow_span(tl, ob, sdet[tl.det0 + row]);
                const uint32_t nb = 4u * (uint32_t)sp.n;
                bulk_copy_g2s(&S.pix[r][row * rs], pv.pix + sp.g0, nb, &S.raw_full[r], hint, pol);
                bulk_copy_g2s(&S.c[r][row * rs], pv.c32 + sp.g0, nb, &S.raw_full[r], hint, pol);
                bulk_copy_g2s(&S.s[r][row * rs], pv.s32 + sp.g0, nb, &S.raw_full[r], hint, pol);
            }
            if (pbytes) bulk_copy_g2s(S.perm[r], perm + tl.perm_off, pbytes, &S.raw_full[r], hint, pol);
        }
        for (int64_t j = it - 1; j >= 0 && j >= it - 2; --j)
            mbar_wait(&S.raw_full[j & 1], (uint32_t)((j >> 1) & 1), err, budget);
        return;
    }

    if (warp < kSGather) {
        // ---------------- gather: xs = P x at every gathered sample, in pixel order
        const int tid = threadIdx.x;
        int64_t it = 0;
        for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x, ++it) {
            const int q = (int)(it & 1);
            const uint32_t par = (uint32_t)((it >> 1) & 1);
            bool okg = mbar_wait(&S.xs_empty[q], par ^ 1u, err, budget);
            okg = okg && mbar_wait(&S.raw_full[q], par, err, budget);
            if (!sgathers_all(okg)) break;
            const STile tl = tiles[ti];
            const ObsInfo ob = pv.obs[tl.obs];
            const int rs = srow_stride(tl.len);
            float *xs = S.xs[q];
            // out-of-stream halos and invalid samples read as zero in the band
            const int nz = min(tl.nrow * rs + 32, kSNE + 32);
            for (int X = tid; X < nz; X += 32 * kSGather) xs[spos(X)] = 0.f;
            sgathers_sync();
            const int np = S.nperm[q];
            float4 m[kSGatherPer];
#pragma unroll
            for (int k = 0; k < kSGatherPer; ++k) {
                const int j = tid + k * 32 * kSGather;
                m[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < np) {
                    const SEntry d = sdecode(S, q, rs, S.perm[q][j]);
                    m[k] = __ldg(x32 + ob.map_off + S.pix[q][d.R]);
                }
            }
#pragma unroll
            for (int k = 0; k < kSGatherPer; ++k) {
                const int j = tid + k * 32 * kSGather;
                if (j < np) {
                    const SEntry d = sdecode(S, q, rs, S.perm[q][j]);
                    float c = S.c[q][d.R], s = S.s[q][d.R];
                    if (pv.psi_cs) rotate_psi<float>(c, s, pv.psi_cs[S.row[q][d.row].gdet]);
                    xs[spos(d.X)] = fmaf(m[k].z, s, fmaf(m[k].y, c, m[k].x));
                }
            }
            mbar_arrive(&S.xs_full[q]);
        }
        return;
    }

    // ---------------- consumer: y = N^-1 xs per row, then one reduction per run of equal pixels
    const int tid = threadIdx.x - 32 * kSGather;
    int64_t it = 0;
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x, ++it) {
        const int q = (int)(it & 1);
        const bool ok = mbar_wait(&S.xs_full[q], (uint32_t)((it >> 1) & 1), err, budget);
        const STile tl = tiles[ti];
        const ObsInfo ob = pv.obs[tl.obs];
        const int rs = srow_stride(tl.len);
        const int tpr = (tl.len + 15) >> 4;                // consumer threads per row (16 outputs each)
        const int row = tid / tpr;
        const int o = (tid - row * tpr) * 16;
        const bool active = ok && row < tl.nrow;
        float *xs = S.xs[q];
        const int base = row * rs + 3 + o;                 // band position of input t0 + o - 63
        float y[16];
        if (active) {
            const int32_t gdet = S.row[q][row].gdet;
            if constexpr (BANDED) {
                band_product_x2<16, true>(xs, nv.band2 + (int64_t)gdet * 2 * kBandPad, base, y);
            } else {
                const float w = nv.p32[gdet];
#pragma unroll
                for (int i = 0; i < 16; ++i) y[i] = xs[spos(base + 63 + i)] * w;
            }
        }
        if (!sconsumers_all(ok)) break;
        if (active) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (o + i < tl.len) xs[spos(base + 63 + i)] = y[i];
        }
        sconsumers_sync();
        const int np = S.nperm[q];
        const int32_t *spx = S.pix[q];
        // Run sums: the first entry of each run of equal pixels adds up the run's core samples.
        auto run_head = [&](int j, int32_t &pixj) -> bool {
            const SEntry d = sdecode(S, q, rs, S.perm[q][j]);
            pixj = spx[d.R];
            return j == 0 || spx[sdecode(S, q, rs, S.perm[q][j - 1]).R] != pixj;
        };
        auto run_sum = [&](int j, int32_t pixj, float3 &h, float3 &l) -> bool {
            bool any = false;
            h = make_float3(0.f, 0.f, 0.f);
            l = make_float3(0.f, 0.f, 0.f);
            for (int mm = j; mm < np; ++mm) {
                const uint16_t e = S.perm[q][mm];
                const SEntry d = sdecode(S, q, rs, e);
                if (spx[d.R] != pixj) break;
                if ((unsigned)((e & 0xfff) - kSCore0) >= (unsigned)tl.len) continue;   // halo sample
                float c = S.c[q][d.R], s = S.s[q][d.R];
                if (pv.psi_cs) rotate_psi<float>(c, s, pv.psi_cs[S.row[q][d.row].gdet]);
                const float yv = xs[spos(d.X)];
                const float v0 = yv, v1 = yv * c, v2 = yv * s;
                if constexpr (ACC == FURAX_ACC_F32) {
                    h.x += v0; h.y += v1; h.z += v2;
                } else {
                    const float t0 = h.x + v0, t1 = h.y + v1, t2 = h.z + v2;
                    l.x += two_sum_err(h.x, v0, t0);
                    l.y += two_sum_err(h.y, v1, t1);
                    l.z += two_sum_err(h.z, v2, t2);
                    h = make_float3(t0, t1, t2);
                }
                any = true;
            }
            return any;
        };
        if constexpr (ACC == FURAX_ACC_F32_KAHAN) {
#pragma unroll
            for (int k0 = 0; k0 < kSConsPer; k0 += kSKahanBatch) {
                float4 old[kSKahanBatch];
                float3 hh[kSKahanBatch], ll[kSKahanBatch];
                int32_t px[kSKahanBatch];
#pragma unroll
                for (int b = 0; b < kSKahanBatch; ++b) {
                    const int j = tid + (k0 + b) * 32 * kSConsumer;
                    px[b] = -1;
                    int32_t pj;
                    if (j < np && run_head(j, pj) && run_sum(j, pj, hh[b], ll[b])) {
                        px[b] = pj;
                        old[b] = atom_add_v4(acc_hi + kKahanStride * (ob.map_off + pj),
                                             make_float4(hh[b].x, hh[b].y, hh[b].z, 0.f));
                    }
                }
#pragma unroll
                for (int b = 0; b < kSKahanBatch; ++b)
                    if (px[b] >= 0) {
                        float4 e = kahan_error_v4(old[b], make_float4(hh[b].x, hh[b].y, hh[b].z, 0.f));
                        e.x += ll[b].x; e.y += ll[b].y; e.z += ll[b].z;
                        red_add_v4(acc_lo + kKahanStride * (ob.map_off + px[b]), e);
                    }
            }
        } else {
            for (int j = tid; j < np; j += 32 * kSConsumer) {
                int32_t pj;
                float3 h, l;
                if (!run_head(j, pj) || !run_sum(j, pj, h, l)) continue;
                const int64_t gp = ob.map_off + pj;
                if constexpr (ACC == FURAX_ACC_F32) {
                    red_add_v4(acc_hi + gp, make_float4(h.x, h.y, h.z, 0.f));
                } else {
                    // FP64 accumulation of the compensated run sum, converted on the integer pipe
                    red_add_f64(acc64 + 3 * gp + 0, f32_to_f64_bits(h.x));
                    red_add_f64(acc64 + 3 * gp + 1, f32_to_f64_bits(h.y));
                    red_add_f64(acc64 + 3 * gp + 2, f32_to_f64_bits(h.z));
                    if (l.x != 0.f) red_add_f64(acc64 + 3 * gp + 0, f32_to_f64_bits(l.x));
                    if (l.y != 0.f) red_add_f64(acc64 + 3 * gp + 1, f32_to_f64_bits(l.y));
                    if (l.z != 0.f) red_add_f64(acc64 + 3 * gp + 2, f32_to_f64_bits(l.z));
                }
            }
        }
        mbar_arrive(&S.xs_empty[q]);
        mbar_arrive(&S.raw_empty[q]);
    }
}

// ------------------------------------------------------------------------------------
// Host: schedule, tiles, permutation
// ------------------------------------------------------------------------------------

// v' = R(q) v for a unit quaternion q = (w, x, y, z).
static void qrot(const double *q, const double *v, double *out)
{
    const double w = q[0], ux = q[1], uy = q[2], uz = q[3];
    const double cx = uy * v[2] - uz * v[1], cy = uz * v[0] - ux * v[2], cz = ux * v[1] - uy * v[0];
    const double ccx = uy * cz - uz * cy, ccy = uz * cx - ux * cz, ccz = ux * cy - uy * cx;
    out[0] = v[0] + 2.0 * (w * cx + ccx);
    out[1] = v[1] + 2.0 * (w * cy + ccy);
    out[2] = v[2] + 2.0 * (w * cz + ccz);
}

// Axis of the boresight frame's rotation from sample t to t + 1, in the frame at t (q1* (x) q2).
static bool rotation_axis(const double *q1, const double *q2, double *axis)
{
    const double w1 = q1[0], x1 = -q1[1], y1 = -q1[2], z1 = -q1[3];
    const double w2 = q2[0], x2 = q2[1], y2 = q2[2], z2 = q2[3];
    const double x = w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2;
    const double y = w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2;
    const double z = w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2;
    const double w = w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2;
    const double nv = std::sqrt(x * x + y * y + z * z);
    if (!(nv > 0.0) || !std::isfinite(nv)) return false;
    const double sg = w < 0.0 ? -1.0 : 1.0;   // the rotation by the smaller angle
    axis[0] = sg * x / nv; axis[1] = sg * y / nv; axis[2] = sg * z / nv;
    return true;
}

void free_sorted(furax_pointing *p)
{
    cudaFree(p->d_stiles); cudaFree(p->d_sdet); cudaFree(p->d_perm); cudaFree(p->d_perm_n);
    p->d_stiles = nullptr; p->d_sdet = nullptr; p->d_perm = nullptr; p->d_perm_n = nullptr;
    p->n_stiles = 0;
    p->perm_cap = 0;
}

bool sorted_active(const furax_pointing *p)
{
    return p->sched.kernel == FURAX_SCHED_PIXEL_SORTED && p->n_stiles > 0;
}

furax_status sort_sorted_tiles(const furax_pointing *p, cudaStream_t st)
{
    if (!sorted_active(p)) return FURAX_OK;
    sort_tiles_kernel<<<(unsigned)p->n_stiles, kSortThreads, 0, st>>>(p->d_stiles, p->d_obs, p->d_sdet, p->pix,
                                                                       p->d_perm, p->d_perm_n);
    count_launches(1);
    return check_launch("pixel sort of the tiles");
}

furax_status set_schedule(furax_pointing *p, const furax_schedule &s, cudaStream_t st)
{
    if (s.kernel != FURAX_SCHED_TIME_ORDERED && s.kernel != FURAX_SCHED_PIXEL_SORTED)
        return set_error(FURAX_EINVAL, "unknown schedule kernel %d", s.kernel);
    if (s.l2_evict_first != 0 && s.l2_evict_first != 1) return set_error(FURAX_EINVAL, "l2_evict_first must be 0 or 1");
    if (s.consumer_warps != 0 && s.consumer_warps != 8 && s.consumer_warps != 16)
        return set_error(FURAX_EINVAL, "consumer_warps must be 0, 8 or 16");
    if (s.kernel == FURAX_SCHED_PIXEL_SORTED) {
        if (p->mode != FURAX_POINTING_CACHE_F32 && p->mode != FURAX_POINTING_CACHE_MIXED)
            return set_error(FURAX_EINVAL, "the pixel-sorted schedule needs the FP32 pointing cache");
        if (s.tile_len != 0 && (s.tile_len < 16 || s.tile_len > 4096 || s.tile_len % 16 != 0))
            return set_error(FURAX_EINVAL, "tile_len must be 0 or a multiple of 16 in [16, 4096]");
        if (s.max_rows < 1 || s.max_rows > kSRowMax)
            return set_error(FURAX_EINVAL, "max_rows must be in [1, %d]", kSRowMax);
        if (!(s.group_tol > 0.0) || !std::isfinite(s.group_tol))
            return set_error(FURAX_EINVAL, "group_tol must be a positive number of pixel widths");
    }
    furax_status rc = check_cuda(cudaStreamSynchronize(st), "schedule sync");
    if (rc) return rc;
    free_sorted(p);
    p->sched = s;
    if (s.kernel == FURAX_SCHED_TIME_ORDERED) return FURAX_OK;

    // detector lines of sight in the boresight frame
    std::vector<double> qd(4 * (size_t)p->ndet_total);
    if ((rc = check_cuda(cudaMemcpy(qd.data(), p->q_det, sizeof(double) * qd.size(), cudaMemcpyDeviceToHost),
                         "read detector quaternions")))
        return rc;
    std::vector<STile> tiles;
    std::vector<int32_t> sdet;
    int64_t cap = 0;
    const double zhat[3] = {0.0, 0.0, 1.0};
    for (int32_t oi = 0; oi < p->n_obs; ++oi) {
        const ObsInfo &ob = p->obs[oi];
        if (ob.nsamp < 1 || ob.ndet < 1) continue;
        // mean rotation axis of the scan over 16 sample pairs spread over the observation
        double ax[3] = {0.0, 0.0, 0.0};
        if (ob.nsamp >= 2) {
            std::vector<double> qb(8);
            for (int k = 0; k < 16; ++k) {
                const int64_t t = std::min<int64_t>(ob.nsamp - 2, (int64_t)((k + 0.5) * (double)ob.nsamp / 16.0));
                if ((rc = check_cuda(cudaMemcpy(qb.data(), p->q_bore + 4 * (ob.bore_off + t), sizeof(double) * 8,
                                                cudaMemcpyDeviceToHost), "read boresight")))
                    return rc;
                double a[3];
                if (rotation_axis(qb.data(), qb.data() + 4, a)) {
                    const double sg = (a[0] * ax[0] + a[1] * ax[1] + a[2] * ax[2]) < 0.0 ? -1.0 : 1.0;
                    for (int c = 0; c < 3; ++c) ax[c] += sg * a[c];
                }
            }
        }
        const double an = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
        // angle of each detector's line of sight to the axis: equal angles, equal tracks
        std::vector<double> ang(ob.ndet, 0.0);
        for (int32_t d = 0; d < ob.ndet; ++d) {
            double v[3];
            qrot(&qd[4 * (ob.det_off + d)], zhat, v);
            if (an > 0.0) {
                const double cth = (v[0] * ax[0] + v[1] * ax[1] + v[2] * ax[2]) / an;
                ang[d] = std::acos(std::max(-1.0, std::min(1.0, cth)));
            } else {
                ang[d] = (double)d;   // no motion: every detector alone
            }
        }
        std::vector<int32_t> order(ob.ndet);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return ang[a] < ang[b]; });
        const double tol = s.group_tol * std::sqrt(4.0 * M_PI / (double)ob.npix);
        // groups of consecutive detectors within tol of the group's first, at most max_rows
        std::vector<std::pair<int32_t, int32_t>> groups;   // (first index into sdet, rows)
        for (int32_t k = 0; k < ob.ndet;) {
            int32_t e = k + 1;
            while (e < ob.ndet && e - k < s.max_rows && ang[order[e]] - ang[order[k]] <= tol) ++e;
            groups.push_back({(int32_t)sdet.size(), e - k});
            for (int32_t m = k; m < e; ++m) sdet.push_back(order[m]);
            k = e;
        }
        // time blocks per group: as long as the stage holds (nrow rows of srow_stride(len) entries,
        // nrow ceil(len / 16) consumer threads), at most tile_len; tiles in time-major order
        struct Run { int32_t det0, nrow, len; };
        std::vector<Run> runs;
        for (auto &g : groups) {
            int32_t L = std::min<int32_t>(4096, (kSNE / g.second) / 16 * 16);
            while (L > 16 && g.second * srow_stride(L) > kSNE) L -= 16;
            if (s.tile_len > 0) L = std::min(L, s.tile_len);
            runs.push_back({g.first, g.second, L});
        }
        std::vector<STile> obs_tiles;
        for (const Run &r : runs)
            for (int64_t t0 = 0; t0 < ob.nsamp; t0 += r.len) {
                STile tl;
                tl.t0 = t0;
                tl.obs = oi;
                tl.len = (int32_t)std::min<int64_t>(r.len, ob.nsamp - t0);
                tl.nrow = r.nrow;
                tl.det0 = r.det0;
                tl.perm_off = 0;
                obs_tiles.push_back(tl);
            }
        std::stable_sort(obs_tiles.begin(), obs_tiles.end(), [](const STile &a, const STile &b) { return a.t0 < b.t0; });
        for (STile &tl : obs_tiles) {
            tl.perm_off = cap;
            cap += ((int64_t)tl.nrow * (tl.len + 126) + 7) & ~int64_t(7);
            tiles.push_back(tl);
        }
    }
    if (tiles.empty()) { p->sched.kernel = FURAX_SCHED_TIME_ORDERED; return FURAX_OK; }
    // Every index the kernels form from a tile stays inside its stage, its permutation slot and
    // the (4-element padded) cache; checked here for each tile and row before anything runs.
    const int64_t tod4 = (p->nsamp_total + 3) & ~int64_t(3);
    for (const STile &tl : tiles) {
        const ObsInfo &ob = p->obs[tl.obs];
        const int rs = srow_stride(tl.len);
        const int64_t cap_t = ((int64_t)tl.nrow * (tl.len + 126) + 7) & ~int64_t(7);
        bool ok = tl.len >= 1 && tl.nrow >= 1 && tl.nrow <= kSRowMax && (int64_t)tl.nrow * rs <= kSNE &&
                  (int64_t)tl.nrow * ((tl.len + 15) / 16) <= 32 * kSConsumer && tl.len + 129 <= rs &&
                  tl.perm_off % 8 == 0 && tl.perm_off + cap_t <= cap && tl.t0 >= 0 && tl.t0 + tl.len <= ob.nsamp;
        for (int r = 0; ok && r < tl.nrow; ++r) {
            const int32_t det = sdet[tl.det0 + r];
            const int64_t row_start = ob.tod_off + (int64_t)det * ob.nsamp;
            const int64_t t_lo = std::max<int64_t>(tl.t0 - 63, 0), t_hi = std::min<int64_t>(tl.t0 + tl.len + 63, ob.nsamp);
            const int64_t g0 = (row_start + t_lo) & ~int64_t(3), g1 = (row_start + t_hi + 3) & ~int64_t(3);
            const int64_t delta = row_start + tl.t0 - kSCore0 - g0;
            ok = det >= 0 && det < ob.ndet && g0 >= 0 && g1 <= tod4 && g1 - g0 <= rs && (g1 - g0) % 4 == 0 &&
                 delta > -rs && delta < rs &&
                 // first and last in-stream sample land inside the copied range
                 3 + t_lo - tl.t0 + 63 + delta >= 0 && 3 + (t_hi - 1) - tl.t0 + 63 + delta < g1 - g0;
        }
        if (!ok) {
            free_sorted(p);
            p->sched.kernel = FURAX_SCHED_TIME_ORDERED;
            return set_error(FURAX_EINVAL, "pixel-sorted schedule: tile at t0 %lld of observation %d fails its layout "
                             "checks", (long long)tl.t0, tl.obs);
        }
    }
    if ((int64_t)tiles.size() >= (1LL << 31)) return set_error(FURAX_EINVAL, "too many sorted tiles for one grid");
    cudaError_t e = cudaMalloc((void **)&p->d_stiles, sizeof(STile) * tiles.size());
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_sdet, sizeof(int32_t) * sdet.size());
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_perm, sizeof(uint16_t) * (size_t)cap + 16);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_perm_n, sizeof(int32_t) * tiles.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_sorted(p);
        p->sched.kernel = FURAX_SCHED_TIME_ORDERED;
        return set_error(FURAX_ENOMEM, "pixel-sorted schedule: allocation of %lld permutation entries failed",
                         (long long)cap);
    }
    p->n_stiles = (int64_t)tiles.size();
    p->perm_cap = cap;
    if ((rc = check_cuda(cudaMemcpy(p->d_stiles, tiles.data(), sizeof(STile) * tiles.size(), cudaMemcpyHostToDevice),
                         "upload sorted tiles")) ||
        (rc = check_cuda(cudaMemcpy(p->d_sdet, sdet.data(), sizeof(int32_t) * sdet.size(), cudaMemcpyHostToDevice),
                         "upload tile rows"))) {
        free_sorted(p);
        p->sched.kernel = FURAX_SCHED_TIME_ORDERED;
        return rc;
    }
    if ((rc = sort_sorted_tiles(p, st))) return rc;
    return check_cuda(cudaStreamSynchronize(st), "schedule sort sync");
}

template <int ACC, bool BANDED>
static furax_status run_sorted(const furax_pointing *p, const furax_noise *n, const float4 *x32, float4 *hi, float4 *lo,
                               double *a64, cudaStream_t st)
{
    const unsigned g = (unsigned)std::min<int64_t>(p->n_stiles, p->n_sm);
    return launch_dyn(fused_sorted_kernel<ACC, BANDED>, g, kSThreads, kSortedSmem, st, p->d_stiles, p->n_stiles,
                      p->d_sdet, p->d_perm, p->d_perm_n, p->view(), n->view(), x32, hi, lo, a64, p->d_err,
                      (int)p->sched.l2_evict_first);
}

template <bool BANDED>
static furax_status dispatch_sorted(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc,
                                    float4 *hi, float4 *lo, double *a64, cudaStream_t st)
{
    if (acc == FURAX_ACC_F32) return run_sorted<FURAX_ACC_F32, BANDED>(p, n, x32, hi, lo, a64, st);
    if (acc == FURAX_ACC_F32_KAHAN) return run_sorted<FURAX_ACC_F32_KAHAN, BANDED>(p, n, x32, hi, lo, a64, st);
    return run_sorted<FURAX_ACC_F64, BANDED>(p, n, x32, hi, lo, a64, st);
}

furax_status launch_fused_sorted(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc, float4 *hi,
                                 float4 *lo, double *a64, cudaStream_t st)
{
    if (n->kind == FURAX_NOISE_BANDED) {
        if (!n->band2) return set_error(FURAX_EINVAL, "the pixel-sorted operator needs a band of at most %d taps", MAXTAPS);
        return dispatch_sorted<true>(p, n, x32, acc, hi, lo, a64, st);
    }
    return dispatch_sorted<false>(p, n, x32, acc, hi, lo, a64, st);
}

template <bool BANDED>
static furax_status prepare_sorted_band()
{
    furax_status rc = allow_smem((const void *)fused_sorted_kernel<FURAX_ACC_F32, BANDED>, kSortedSmem);
    if (!rc) rc = allow_smem((const void *)fused_sorted_kernel<FURAX_ACC_F32_KAHAN, BANDED>, kSortedSmem);
    if (!rc) rc = allow_smem((const void *)fused_sorted_kernel<FURAX_ACC_F64, BANDED>, kSortedSmem);
    return rc;
}

furax_status prepare_fused_sorted()
{
    furax_status rc = prepare_sorted_band<true>();
    if (!rc) rc = prepare_sorted_band<false>();
    return rc;
}

}  // namespace fx
