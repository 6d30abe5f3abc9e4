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
#include "dfloat.cuh"
#include "tpl_eval.cuh"

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
// Taps are walked in rolled blocks of 8, each unrolled over 8 taps x R outputs from register
// windows of R + 7 inputs (a fully unrolled 127 x R body overflows the instruction cache).
template <int R>
__device__ __forceinline__ void band_product_df(const float *__restrict__ xh, const float *__restrict__ xl,
                                                const float *__restrict__ th, const float *__restrict__ tl, int base,
                                                float (&S)[R], float (&E)[R])
{
    constexpr int JB = 8;
#pragma unroll
    for (int r = 0; r < R; ++r) { S[r] = 0.f; E[r] = 0.f; }
#pragma unroll 1
    for (int j0 = 0; j0 < kBand; j0 += JB) {
        float wh[R + JB - 1], wl[R + JB - 1];
#pragma unroll
        for (int i = 0; i < R + JB - 1; ++i) {
            wh[i] = xh[spos(base + j0 + i)];
            wl[i] = xl[spos(base + j0 + i)];
        }
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
            const int j = j0 + jj;
            if (j < kBand) {
                const int k = j < kHalo ? kHalo - j : j - kHalo;
                const float ch = th[k], cl = tl[k];
#pragma unroll
                for (int r = 0; r < R; ++r) dot2_step(ch, cl, wh[r + jj], wl[r + jj], S[r], E[r]);
            }
        }
    }
}

constexpr size_t kDfSmem = sizeof(float) * (2 * XS + 2 * MAXTAPS) + sizeof(float2) * 2 * CS + sizeof(int32_t) * CS;

// acc64 += P^T N^-1 d (FROM_TOD: the right-hand side from FP64 data, the form launched), or
// acc64 += P^T N^-1 P x (x: FP64 [npix][3]); the map form is served by df_apply_kernel below, which
// issues no FP64 arithmetic per sample.
template <int MODE, bool BANDED, bool FROM_TOD, typename DT>
__global__ void __launch_bounds__(FT, 2) fused_df_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
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

// ------------------------------------------------------------------------------------
// Standalone N^-1 on an FP64 TOD, FP64-accurate on FP32 units: the input and the taps are split
// into double-FP32 pairs and the band product is the compensated dot product above; the result
// S + E is returned in FP64. For the band products of the FP64-accurate gap filling.
// ------------------------------------------------------------------------------------
template <bool BANDED>
__global__ void __launch_bounds__(FT) ninv_df_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                     NoiseView nv, const double *__restrict__ in,
                                                     double *__restrict__ out)
{
    __shared__ float xh[XS], xl[XS], th[MAXTAPS], tl[MAXTAPS];
    const Tile tile = tiles[blockIdx.x];
    const ObsInfo ob = obs[tile.obs];
    const int64_t gdet = ob.det_off + tile.det;
    const int64_t row = ob.tod_off + tile.det * ob.nsamp;
    constexpr int halo = BANDED ? kHalo : 0;
    if (threadIdx.x < MAXTAPS) {
        double c = 0.0;
        if constexpr (BANDED) c = threadIdx.x < nv.ntaps ? nv.p64[gdet * nv.ntaps + threadIdx.x] : 0.0;
        else c = threadIdx.x == 0 ? nv.p64[gdet] : 0.0;
        split_df(c, th[threadIdx.x], tl[threadIdx.x]);
    }
    const int nload = tile.len + 2 * halo;
    for (int u = threadIdx.x; u < nload; u += FT) {
        const int64_t t = tile.t0 - halo + u;
        split_df((t >= 0 && t < ob.nsamp) ? in[row + t] : 0.0, xh[spos(u)], xl[spos(u)]);
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
    for (int r = 0; r < FR; ++r)
        if (base + r < tile.len) out[row + tile.t0 + base + r] = (double)S[r] + (double)E[r];
}

furax_status launch_ninv_df(const furax_noise *n, const double *in, double *out, cudaStream_t st)
{
    if (long_band(n)) return set_error(FURAX_EINVAL, "internal: the double-FP32 N^-1 takes bands of up to %d taps", MAXTAPS);
    if (n->n_tiles == 0) return FURAX_OK;
    const unsigned g = (unsigned)n->n_tiles;
    if (n->kind == FURAX_NOISE_BANDED)
        ninv_df_kernel<true><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, n->view(), in, out);
    else
        ninv_df_kernel<false><<<g, FT, 0, st>>>(n->d_tiles, n->d_obs, n->view(), in, out);
    count_launches(1);
    return check_launch("double-FP32 N^-1 apply");
}

// ------------------------------------------------------------------------------------
// Right-hand side from FP32 time-ordered data: acc64 + lo += P^T N^-1 d.
// The input word is exact in FP32, so the compensated band product carries no input low word.
// The output y = S + E is renormalised to (y_hi, y_lo); each weighted term y w (w = 1, cos, sin)
// is formed as an exact FP32 product head plus a tail. Heads are accumulated in FP64 (their
// binary64 value is built from the binary32 encoding, so no FP64 arithmetic is issued); tails,
// which are ~2^-24 of the heads, are accumulated in FP32 and folded in afterwards.
// ------------------------------------------------------------------------------------

// The taps are walked in blocks of JB (a rolled loop), each block unrolled over JB taps x R
// outputs from a register window of R + JB - 1 inputs: a fully unrolled 127 x R body does not fit
// the instruction cache (measured: warps then mostly wait for instructions). The last block is
// partial (127 = 15 x 8 + 7); its extra window slots read initialised tile slots and are unused.
constexpr int kDfJB = 8;

template <int R>
__device__ __forceinline__ void band_product_dfx(const float *__restrict__ xs, const float *__restrict__ th,
                                                 const float *__restrict__ tl, int base, float (&S)[R], float (&E)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r) { S[r] = 0.f; E[r] = 0.f; }
#pragma unroll 1
    for (int j0 = 0; j0 < kBand; j0 += kDfJB) {
        float w[R + kDfJB - 1];
#pragma unroll
        for (int i = 0; i < R + kDfJB - 1; ++i) w[i] = xs[spos(base + j0 + i)];
#pragma unroll
        for (int jj = 0; jj < kDfJB; ++jj) {
            const int j = j0 + jj;
            if (j < kBand) {
                const int k = j < kHalo ? kHalo - j : j - kHalo;
                const float ch = th[k], cl = tl[k];
#pragma unroll
                for (int r = 0; r < R; ++r) dot2_step_x(ch, cl, w[r + jj], S[r], E[r]);
            }
        }
    }
}

// Packed form of the same compensated sum on output pairs (y_i, y_{i+8}): every step is the
// lane-wise f32x2 version of dot2_step_x, with the product negated once so that no packed
// negation is needed (fl(-ch x) = -fl(ch x), S - (-p) = S + p, -((-p) + b) = p - b exactly), so
// the results are bit-identical with half the instructions. C4[j] = (c_hi, c_hi, -c_hi, -c_hi) and
// CL2[j] = (c_lo, c_lo) hold the band in tap order (j < 127; zero for j = 127).
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ void dot2_step_x2(unsigned long long ch, unsigned long long nch, unsigned long long cl,
                                             unsigned long long x, unsigned long long &S, unsigned long long &E)
{
    const unsigned long long np = f2_mul(nch, x);          // -p
    const unsigned long long e = f2_fma(ch, x, np);        // ch x - p exactly
    const unsigned long long s = f2_sub(S, np);            // S + p
    const unsigned long long bv = f2_sub(s, S);
    const unsigned long long t2 = f2_sub(S, f2_sub(s, bv));
    const unsigned long long err = f2_sub(t2, f2_add(np, bv));   // (S - (s - bv)) + (p - bv)
    S = s;
    E = f2_fma(cl, x, f2_add(E, f2_add(err, e)));
}

// LO: the input is double-FP32 too (low words in xl), and each step adds the cross term
// c_hi x_lo to the error word after c_lo x_hi, as dot2_step does.
template <int R, bool LO = false>
__device__ __forceinline__ void band_product_dfx2(const float *__restrict__ xs, const float4 *__restrict__ C4,
                                                  const float2 *__restrict__ CL2, int base, float (&S)[R], float (&E)[R],
                                                  const float *__restrict__ xl = nullptr)
{
    constexpr int H = R / 2;
    unsigned long long W[H], WL[LO ? H : 1], SS[H], EE[H];   // W[i] = (x[base+i+j], x[base+i+H+j]) at tap j
#pragma unroll
    for (int i = 0; i < H; ++i) {
        W[i] = pack_f32x2(xs[spos(base + i)], xs[spos(base + i + H)]);
        if constexpr (LO) WL[i] = pack_f32x2(xl[spos(base + i)], xl[spos(base + i + H)]);
        SS[i] = 0ull;
        EE[i] = 0ull;
    }
#pragma unroll 1
    for (int j0 = 0; j0 < kBandPad; j0 += kDfJB) {
#pragma unroll
        for (int jj = 0; jj < kDfJB; ++jj) {
            const int j = j0 + jj;
            if (j < kBand) {
                const float4 c4 = C4[j];
                const float2 c2 = CL2[j];
                const unsigned long long ch = pack_f32x2(c4.x, c4.y), nch = pack_f32x2(c4.z, c4.w);
                const unsigned long long cl = pack_f32x2(c2.x, c2.y);
#pragma unroll
                for (int i = 0; i < H; ++i) {
                    dot2_step_x2(ch, nch, cl, W[i], SS[i], EE[i]);
                    if constexpr (LO) EE[i] = f2_fma(ch, WL[i], EE[i]);
                }
                if (j < kBand - 1) {
                    float lo0, hi0;
                    unpack_f32x2(W[0], lo0, hi0);
                    const unsigned long long wl = pack_f32x2(hi0, xs[spos(base + R + j)]);
#pragma unroll
                    for (int i = 0; i < H - 1; ++i) W[i] = W[i + 1];
                    W[H - 1] = wl;
                    if constexpr (LO) {
                        unpack_f32x2(WL[0], lo0, hi0);
                        const unsigned long long wll = pack_f32x2(hi0, xl[spos(base + R + j)]);
#pragma unroll
                        for (int i = 0; i < H - 1; ++i) WL[i] = WL[i + 1];
                        WL[H - 1] = wll;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        unpack_f32x2(SS[i], S[i], S[i + H]);
        unpack_f32x2(EE[i], E[i], E[i + H]);
    }
}

// Pixel and weights of one sample as double-FP32 pairs (offset rotation included).
template <int MODE>
__device__ __forceinline__ int32_t sample_df(const PointingView &pv, const ObsInfo &ob, int32_t det, int64_t t,
                                             float &ch, float &cl, float &sh, float &sl)
{
    if constexpr (MODE == 1 || MODE == 3) {
        if (!pv.psi_cs) {   // cached FP32 weights (plus the cached low words in mode 3): no FP64
            const int64_t i = ob.tod_off + det * ob.nsamp + t;
            const int32_t pix = pv.pix[i];
            ch = pv.c32[i]; sh = pv.s32[i];
            if constexpr (MODE == 3) { cl = pv.c32lo[i]; sl = pv.s32lo[i]; }
            else { cl = 0.f; sl = 0.f; }
            return pix;
        }
    }
    double c = 0.0, s = 0.0;
    const int32_t pix = get_sample<MODE, double>(pv, ob, det, t, c, s);
    split_df(c, ch, cl);
    split_df(s, sh, sl);
    return pix;
}

constexpr size_t kDfRhsSmem = sizeof(float4) * kBandPad + sizeof(float2) * kBandPad + sizeof(float) * (XS + CS + 2 * MAXTAPS);
static_assert(sizeof(float4) * kBandPad % 16 == 0 && sizeof(float2) * kBandPad % 16 == 0, "coefficient arrays stay 16-byte aligned");

// TPL: the template correction of the deprojected right-hand side is folded in, y -= (W T) b for
// amplitudes b already solved from d: in the interior of a stream (W T b)(t) is a cubic in the
// offset j of t from the middle sample of the tile's own samples (no extrapolation in tau), evaluated by Horner's rule in double-FP32 from
// coefficients the CTA forms once in FP64; near the ends of the stream it is summed term by term
// in FP64.
template <int MODE, bool BANDED, bool TPL>
__global__ void __launch_bounds__(FT, 2) df_rhs_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                       const float *__restrict__ d, double *__restrict__ acc64,
                                                       float4 *__restrict__ acc_lo, TplView tv)
{
    extern __shared__ __align__(16) float rsm[];
    float4 *C4 = reinterpret_cast<float4 *>(rsm);            // [kBandPad] (c_hi, c_hi, -c_hi, -c_hi), tap order
    float2 *CL2 = reinterpret_cast<float2 *>(C4 + kBandPad); // [kBandPad] (c_lo, c_lo)
    float *xs = reinterpret_cast<float *>(CL2 + kBandPad);   // [XS] d over the tile and halos; then y_hi of the core
    float *yl = xs + XS;        // [CS] y_lo of the core samples
    float *th = yl + CS;        // [MAXTAPS]
    float *tl = th + MAXTAPS;   // [MAXTAPS]

    const Tile tile = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tile.obs];
    const int64_t gdet = ob.det_off + tile.det;
    constexpr int halo = BANDED ? kHalo : 0;
    if (threadIdx.x < MAXTAPS) {
        double c = 0.0;
        if constexpr (BANDED) c = threadIdx.x < nv.ntaps ? nv.p64[gdet * nv.ntaps + threadIdx.x] : 0.0;
        else c = threadIdx.x == 0 ? nv.p64[gdet] : 0.0;
        split_df(c, th[threadIdx.x], tl[threadIdx.x]);
    }
    if (BANDED && threadIdx.x < kBandPad) {
        const int j = threadIdx.x, k = j < kHalo ? kHalo - j : j - kHalo;
        float h = 0.f, l = 0.f;
        if (j < kBand && k < nv.ntaps) split_df(nv.p64[gdet * nv.ntaps + k], h, l);
        C4[j] = make_float4(h, h, -h, -h);
        CL2[j] = make_float2(l, l);
    }
    __shared__ float2 ecoef[4];   // TPL: coefficients of the tile's cubic in j, double-FP32
    if constexpr (TPL) {
        if (threadIdx.x == 0) {
            const double h = ob.nsamp > 1 ? 2.0 / (double)(ob.nsamp - 1) : 0.0;
            const double2 m = tv.mom[gdet];
            const double bv[4] = {tv.b[4 * gdet], tv.b[4 * gdet + 1], tv.b[4 * gdet + 2], tv.b[4 * gdet + 3]};
            double c[4], e[4];
            tpl_cubic(m.x, m.y * h * h * 0.5, bv, c);
            cubic_shift(c, tpl_tau_ref(tile.t0 + (tile.len >> 1), ob.nsamp), h, e);
#pragma unroll
            for (int i = 0; i < 4; ++i) split_df(e[i], ecoef[i].x, ecoef[i].y);
        }
    }
    const int nload = tile.len + 2 * halo;
    const int64_t row = ob.tod_off + tile.det * ob.nsamp;
    for (int u = threadIdx.x; u < nload; u += FT) {
        const int64_t t = tile.t0 - halo + u;
        xs[spos(u)] = (t >= 0 && t < ob.nsamp) ? d[row + t] : 0.f;
    }
    __syncthreads();

    const int base = threadIdx.x * FR;
    float S[FR], E[FR];
    if (base < tile.len) {
        if constexpr (BANDED) {
            band_product_dfx2<FR>(xs, C4, CL2, base, S, E);
        } else {
#pragma unroll
            for (int r = 0; r < FR; ++r) {
                S[r] = 0.f;
                E[r] = 0.f;
                dot2_step_x(th[0], tl[0], xs[spos(base + r)], S[r], E[r]);
            }
        }
    }
    __syncthreads();   // every stencil input has been read: y overwrites the tile in place
    if (base < tile.len) {
#pragma unroll
        for (int r = 0; r < FR; ++r) {
            if (base + r < tile.len) {
                const float h = __fadd_rn(S[r], E[r]);          // |S| >= |E|: fast two-sum
                xs[spos(base + r)] = h;
                yl[spos(base + r)] = __fsub_rn(E[r], __fsub_rn(h, S[r]));
            }
        }
    }
    __syncthreads();

    // Warp-uniform trip count: the FP64 head of each sample's contribution leaves through the
    // warp's record-wise reductions (staging area below), which every lane joins; lanes past the
    // tile or on masked samples offer pix = -1.
    __shared__ float xv[FT / 32][96];
    __shared__ int32_t xp[FT / 32][32];
    double *rec = acc64 + 3 * ob.map_off;
    for (int kw = threadIdx.x & ~31; kw < tile.len; kw += FT) {
        const int k = kw + (threadIdx.x & 31);
        float ch = 0.f, cl = 0.f, sh = 0.f, sl = 0.f;
        const int32_t pix = k < tile.len ? sample_df<MODE>(pv, ob, tile.det, tile.t0 + k, ch, cl, sh, sl) : -1;
        float yh = 0.f, qc = 0.f, qs = 0.f;
        if (pix >= 0) {
            yh = xs[spos(k)];
            float ylo = yl[spos(k)];
            if constexpr (TPL) {
                const int64_t t = tile.t0 + k;
                if (tpl_interior(tv, t, ob.nsamp)) {
                    const float j = (float)(k - (tile.len >> 1));
                    float vh = ecoef[3].x, vl = ecoef[3].y;
                    df_horner(vh, vl, j, ecoef[2].x, ecoef[2].y);
                    df_horner(vh, vl, j, ecoef[1].x, ecoef[1].y);
                    df_horner(vh, vl, j, ecoef[0].x, ecoef[0].y);
                    df_add(yh, ylo, -vh, -vl);
                } else {
                    double w[4];
                    wt_eval<double>(nv, tv, gdet, ob.nsamp, t, w);
                    double v = (double)yh + (double)ylo;
#pragma unroll
                    for (int l = 0; l < 4; ++l) v -= tv.b[4 * gdet + l] * w[l];
                    split_df(v, yh, ylo);
                }
            }
            qc = __fmul_rn(yh, ch);
            qs = __fmul_rn(yh, sh);
            const float ec = __fmaf_rn(yh, ch, -qc), es = __fmaf_rn(yh, sh, -qs);
            const float lc = __fadd_rn(ec, __fmaf_rn(ylo, ch, __fmul_rn(yh, cl)));
            const float ls = __fadd_rn(es, __fmaf_rn(ylo, sh, __fmul_rn(yh, sl)));
            red_add_v4(acc_lo + ob.map_off + pix, make_float4(ylo, lc, ls, 0.f));
        }
        const float v[3] = {yh, qc, qs};
        red_add_f64_records_warp<3, float>(rec, pix, v, xv[threadIdx.x >> 5], xp[threadIdx.x >> 5]);
    }
}

// ------------------------------------------------------------------------------------
// FP64-accurate normal operator on a map, acc64 + lo += P^T N^-1 P x, with no FP64 arithmetic
// per sample (FP64 runs ~70x below FP32 on this GPU). x is split once per pixel into double-FP32
// pairs; each sample's P x is formed in double-FP32 from those and the double-FP32 weights; N^-1
// is the packed compensated band product with the input's low words; the scatter splits each
// weighted term into an FP32 head, accumulated in FP64 as whole pixel records, and a tail,
// accumulated in FP32 and folded in afterwards, as for the right-hand side.
// ------------------------------------------------------------------------------------

// x2[2 i] = high words (I, Q, U, 0) of x[i], x2[2 i + 1] = low words.
__global__ void split_map_df_kernel(const double *__restrict__ x, float4 *__restrict__ x2, int64_t np)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        float h[3], l[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) split_df(x[3 * i + c], h[c], l[c]);
        x2[2 * i] = make_float4(h[0], h[1], h[2], 0.f);
        x2[2 * i + 1] = make_float4(l[0], l[1], l[2], 0.f);
    }
}

// v = m0 + m1 c + m2 s in double-FP32 (m = mh + ml, c = ch + cl, s = sh + sl) as vh + vl: exact
// products of the heads, two-sums of the head terms, and the remaining first-order terms in the
// low word (the dropped ml cl, ml sl are ~2^-48 of the terms).
__device__ __forceinline__ void df_weighted_sum(const float4 &mh, const float4 &ml, float ch, float cl, float sh,
                                                float sl, float &vh, float &vl)
{
    const float p1 = __fmul_rn(mh.y, ch), e1 = __fmaf_rn(mh.y, ch, -p1);
    const float p2 = __fmul_rn(mh.z, sh), e2 = __fmaf_rn(mh.z, sh, -p2);
    const float s1 = __fadd_rn(mh.x, p1), t1 = two_sum_err(mh.x, p1, s1);
    const float s2 = __fadd_rn(s1, p2), t2 = two_sum_err(s1, p2, s2);
    float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(t1, t2));
    lo = __fmaf_rn(mh.y, cl, lo);
    lo = __fmaf_rn(ml.y, ch, lo);
    lo = __fmaf_rn(mh.z, sl, lo);
    lo = __fmaf_rn(ml.z, sh, lo);
    lo = __fadd_rn(lo, ml.x);
    vh = __fadd_rn(s2, lo);
    vl = two_sum_err(s2, lo, vh);
}

constexpr size_t kDfApplySmem = sizeof(float4) * kBandPad + sizeof(float2) * kBandPad + sizeof(float) * (2 * XS + 2 * MAXTAPS);

template <int MODE, bool BANDED>
__global__ void __launch_bounds__(FT, 2) df_apply_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                         const float4 *__restrict__ x2, double *__restrict__ acc64,
                                                         float4 *__restrict__ acc_lo)
{
    extern __shared__ __align__(16) float dsm_[];
    float4 *C4 = reinterpret_cast<float4 *>(dsm_);           // [kBandPad] (c_hi, c_hi, -c_hi, -c_hi), tap order
    float2 *CL2 = reinterpret_cast<float2 *>(C4 + kBandPad); // [kBandPad] (c_lo, c_lo)
    float *xh = reinterpret_cast<float *>(CL2 + kBandPad);   // [XS] (P x)_hi over the tile and halos; then y_hi
    float *xl = xh + XS;                                     // [XS] (P x)_lo; then y_lo
    float *th = xl + XS;                                     // [MAXTAPS]
    float *tl = th + MAXTAPS;                                // [MAXTAPS]
    __shared__ float xv[FT / 32][96];
    __shared__ int32_t xp[FT / 32][32];

    const Tile tile = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tile.obs];
    const int64_t gdet = ob.det_off + tile.det;
    constexpr int halo = BANDED ? kHalo : 0;
    if (threadIdx.x < MAXTAPS) {
        double c = 0.0;
        if constexpr (BANDED) c = threadIdx.x < nv.ntaps ? nv.p64[gdet * nv.ntaps + threadIdx.x] : 0.0;
        else c = threadIdx.x == 0 ? nv.p64[gdet] : 0.0;
        split_df(c, th[threadIdx.x], tl[threadIdx.x]);
    }
    if (BANDED && threadIdx.x < kBandPad) {
        const int j = threadIdx.x, k = j < kHalo ? kHalo - j : j - kHalo;
        float h = 0.f, l = 0.f;
        if (j < kBand && k < nv.ntaps) split_df(nv.p64[gdet * nv.ntaps + k], h, l);
        C4[j] = make_float4(h, h, -h, -h);
        CL2[j] = make_float2(l, l);
    }
    const int nload = tile.len + 2 * halo;
    for (int u = threadIdx.x; u < nload; u += FT) {
        const int64_t t = tile.t0 - halo + u;
        float vh = 0.f, vl = 0.f;
        if (t >= 0 && t < ob.nsamp) {
            float ch, cl, sh, sl;
            const int32_t pix = sample_df<MODE>(pv, ob, tile.det, t, ch, cl, sh, sl);
            if (pix >= 0) {
                const int64_t gp = ob.map_off + pix;
                df_weighted_sum(x2[2 * gp], x2[2 * gp + 1], ch, cl, sh, sl, vh, vl);
            }
        }
        xh[spos(u)] = vh;
        xl[spos(u)] = vl;
    }
    __syncthreads();

    const int base = threadIdx.x * FR;
    float S[FR], E[FR];
    if (base < tile.len) {
        if constexpr (BANDED) {
            band_product_dfx2<FR, true>(xh, C4, CL2, base, S, E, xl);
        } else {
#pragma unroll
            for (int r = 0; r < FR; ++r) {
                S[r] = 0.f;
                E[r] = 0.f;
                dot2_step(th[0], tl[0], xh[spos(base + r)], xl[spos(base + r)], S[r], E[r]);
            }
        }
    }
    __syncthreads();   // every stencil input has been read: y overwrites the tile in place
    if (base < tile.len) {
#pragma unroll
        for (int r = 0; r < FR; ++r) {
            if (base + r < tile.len) {
                const float h = __fadd_rn(S[r], E[r]);          // |S| >= |E|: fast two-sum
                xh[spos(base + r)] = h;
                xl[spos(base + r)] = __fsub_rn(E[r], __fsub_rn(h, S[r]));
            }
        }
    }
    __syncthreads();

    // Warp-uniform trip count for the warp's record-wise reductions (lanes past the tile or on
    // masked samples offer pix = -1); the weights are read again (the tile's stretch of the
    // pointing stream is in L2 from the gather above).
    double *rec = acc64 + 3 * ob.map_off;
    for (int kw = threadIdx.x & ~31; kw < tile.len; kw += FT) {
        const int k = kw + (threadIdx.x & 31);
        float ch = 0.f, cl = 0.f, sh = 0.f, sl = 0.f;
        const int32_t pix = k < tile.len ? sample_df<MODE>(pv, ob, tile.det, tile.t0 + k, ch, cl, sh, sl) : -1;
        float yh = 0.f, qc = 0.f, qs = 0.f;
        if (pix >= 0) {
            yh = xh[spos(k)];
            const float ylo = xl[spos(k)];
            qc = __fmul_rn(yh, ch);
            qs = __fmul_rn(yh, sh);
            const float ec = __fmaf_rn(yh, ch, -qc), es = __fmaf_rn(yh, sh, -qs);
            const float lc = __fadd_rn(ec, __fmaf_rn(ylo, ch, __fmul_rn(yh, cl)));
            const float ls = __fadd_rn(es, __fmaf_rn(ylo, sh, __fmul_rn(yh, sl)));
            red_add_v4(acc_lo + ob.map_off + pix, make_float4(ylo, lc, ls, 0.f));
        }
        const float v[3] = {yh, qc, qs};
        red_add_f64_records_warp<3, float>(rec, pix, v, xv[threadIdx.x >> 5], xp[threadIdx.x >> 5]);
    }
}

// ------------------------------------------------------------------------------------
// chi^2 = r^T N^-1 r, r = d - P m, with grad_map = -2 P^T N^-1 r and
// grad_psi = -2 sum (N^-1 r) 2 (U c - Q s), FP64-accurate on the FP32 units (precision
// FURAX_PREC_F32X2): r in double-FP32 from the split map and double-FP32 weights, N^-1 r by the
// packed compensated band product, each thread's sums as double-FP32 pairs (FP64 across threads),
// and the map gradient as FP32 heads reduced in FP64 records plus FP32 tails folded afterwards.
// ------------------------------------------------------------------------------------

// (ah, al) += (xh + xl)(yh + yl), the product's head exact by FMA, its tail and the cross terms
// in the low word.
__device__ __forceinline__ void df_mac(float xh, float xl, float yh, float yl, float &ah, float &al)
{
    const float p = __fmul_rn(xh, yh), e = __fmaf_rn(xh, yh, -p);
    const float s = __fadd_rn(ah, p), t = two_sum_err(ah, p, s);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(t, __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, e))));
}

template <typename DT>
__device__ __forceinline__ void data_df(DT v, float &h, float &l)
{
    if constexpr (sizeof(DT) == 8) {
        h = f64_to_f32_bits(v);
        l = f64_to_f32_bits(v - f32_to_f64_bits(h));   // exact difference, one FP64 subtraction
    } else {
        h = v;
        l = 0.f;
    }
}

template <int MODE, bool BANDED, typename DT>
__global__ void __launch_bounds__(FT, 2) chi2_df_kernel(const Tile *__restrict__ tiles, PointingView pv, NoiseView nv,
                                                        const DT *__restrict__ d, const float4 *__restrict__ m2,
                                                        double *__restrict__ chi2, double *__restrict__ grad_map,
                                                        float4 *__restrict__ gm_lo, double *__restrict__ grad_psi)
{
    extern __shared__ __align__(16) float csm_[];
    float4 *C4 = reinterpret_cast<float4 *>(csm_);           // [kBandPad] (c_hi, c_hi, -c_hi, -c_hi), tap order
    float2 *CL2 = reinterpret_cast<float2 *>(C4 + kBandPad); // [kBandPad] (c_lo, c_lo)
    float *xh = reinterpret_cast<float *>(CL2 + kBandPad);   // [XS] r_hi over the tile and halos; then y_hi
    float *xl = xh + XS;                                     // [XS] r_lo; then y_lo
    float *th = xl + XS;                                     // [MAXTAPS]
    float *tl = th + MAXTAPS;                                // [MAXTAPS]
    __shared__ float xv[FT / 32][96];
    __shared__ int32_t xp[FT / 32][32];
    __shared__ double red[2][FT / 32];

    const Tile tile = tiles[blockIdx.x];
    const ObsInfo ob = pv.obs[tile.obs];
    const int64_t gdet = ob.det_off + tile.det;
    const int64_t row = ob.tod_off + tile.det * ob.nsamp;
    constexpr int halo = BANDED ? kHalo : 0;
    if (threadIdx.x < MAXTAPS) {
        double c = 0.0;
        if constexpr (BANDED) c = threadIdx.x < nv.ntaps ? nv.p64[gdet * nv.ntaps + threadIdx.x] : 0.0;
        else c = threadIdx.x == 0 ? nv.p64[gdet] : 0.0;
        split_df(c, th[threadIdx.x], tl[threadIdx.x]);
    }
    if (BANDED && threadIdx.x < kBandPad) {
        const int j = threadIdx.x, k = j < kHalo ? kHalo - j : j - kHalo;
        float h = 0.f, l = 0.f;
        if (j < kBand && k < nv.ntaps) split_df(nv.p64[gdet * nv.ntaps + k], h, l);
        C4[j] = make_float4(h, h, -h, -h);
        CL2[j] = make_float2(l, l);
    }
    const int nload = tile.len + 2 * halo;
    for (int u = threadIdx.x; u < nload; u += FT) {
        const int64_t t = tile.t0 - halo + u;
        float rh = 0.f, rl = 0.f;
        if (t >= 0 && t < ob.nsamp) {
            float ch, cl, sh, sl, vh = 0.f, vl = 0.f, dh, dl;
            const int32_t pix = sample_df<MODE>(pv, ob, tile.det, t, ch, cl, sh, sl);
            if (pix >= 0) {
                const int64_t gp = ob.map_off + pix;
                df_weighted_sum(m2[2 * gp], m2[2 * gp + 1], ch, cl, sh, sl, vh, vl);
            }
            data_df(d[row + t], dh, dl);
            // r = d - model: two-sum of the heads, the low words in the tail
            const float sdiff = __fsub_rn(dh, vh), e = two_sum_err(dh, -vh, sdiff);
            const float lo = __fadd_rn(e, __fsub_rn(dl, vl));
            rh = __fadd_rn(sdiff, lo);
            rl = two_sum_err(sdiff, lo, rh);
        }
        xh[spos(u)] = rh;
        xl[spos(u)] = rl;
    }
    __syncthreads();

    const int base = threadIdx.x * FR;
    float S[FR], E[FR];
    float ah = 0.f, al = 0.f;   // this thread's part of r^T N^-1 r
    if (base < tile.len) {
        if constexpr (BANDED) {
            band_product_dfx2<FR, true>(xh, C4, CL2, base, S, E, xl);
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
            if (base + r >= tile.len) break;
            const float h = __fadd_rn(S[r], E[r]);              // |S| >= |E|: fast two-sum
            const float l = __fsub_rn(E[r], __fsub_rn(h, S[r]));
            S[r] = h;
            E[r] = l;
            df_mac(xh[spos(base + r + halo)], xl[spos(base + r + halo)], h, l, ah, al);
        }
    }
    __syncthreads();   // every stencil input has been read: y overwrites the tile in place
    if (base < tile.len) {
#pragma unroll
        for (int r = 0; r < FR; ++r) {
            if (base + r < tile.len) {
                xh[spos(base + r)] = S[r];
                xl[spos(base + r)] = E[r];
            }
        }
    }
    __syncthreads();

    float bh = 0.f, bl = 0.f;   // this thread's part of sum y (U c - Q s)
    double *rec = grad_map ? grad_map + 3 * ob.map_off : nullptr;
    for (int kw = threadIdx.x & ~31; kw < tile.len; kw += FT) {   // warp-uniform trip count
        const int k = kw + (threadIdx.x & 31);
        float ch = 0.f, cl = 0.f, sh = 0.f, sl = 0.f;
        const int32_t pix = k < tile.len ? sample_df<MODE>(pv, ob, tile.det, tile.t0 + k, ch, cl, sh, sl) : -1;
        float gh = 0.f, qc = 0.f, qs = 0.f;
        if (pix >= 0) {
            const float yh = xh[spos(k)], yl = xl[spos(k)];
            const int64_t gp = ob.map_off + pix;
            const float4 mh = m2[2 * gp], ml = m2[2 * gp + 1];
            // w = U c - Q s in double-FP32, then (bh, bl) += y w
            float uh = 0.f, ul = 0.f;
            df_mac(mh.z, ml.z, ch, cl, uh, ul);
            df_mac(-mh.y, -ml.y, sh, sl, uh, ul);
            const float wh = __fadd_rn(uh, ul), wl = two_sum_err(uh, ul, wh);
            df_mac(yh, yl, wh, wl, bh, bl);
            if (rec) {
                gh = -2.f * yh;   // exact
                const float gl = -2.f * yl;
                qc = __fmul_rn(gh, ch);
                qs = __fmul_rn(gh, sh);
                const float ec = __fmaf_rn(gh, ch, -qc), es = __fmaf_rn(gh, sh, -qs);
                const float lc = __fadd_rn(ec, __fmaf_rn(gl, ch, __fmul_rn(gh, cl)));
                const float ls = __fadd_rn(es, __fmaf_rn(gl, sh, __fmul_rn(gh, sl)));
                red_add_v4(gm_lo + gp, make_float4(gl, lc, ls, 0.f));
            }
        }
        if (rec) {
            const float v[3] = {gh, qc, qs};
            red_add_f64_records_warp<3, float>(rec, pix, v, xv[threadIdx.x >> 5], xp[threadIdx.x >> 5]);
        }
    }
    // block reduction (fixed order within the block), in FP64 across threads
    double a = (double)ah + (double)al;
    double b = (ob.hwp ? -2.0 : 2.0) * ((double)bh + (double)bl);
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
        red_add_f64(chi2 + tile.obs, sa);
        if (grad_psi) red_add_f64(grad_psi + gdet, -2.0 * sb);
    }
}

// acc64 += lo (per pixel, then lo is no longer needed).
__global__ void fold_lo_kernel(const float4 *__restrict__ lo, double *__restrict__ acc64, int64_t np)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 l = lo[i];
        acc64[3 * i + 0] += (double)l.x;
        acc64[3 * i + 1] += (double)l.y;
        acc64[3 * i + 2] += (double)l.z;
    }
}

template <int MODE, bool B>
static furax_status run_df_rhs(const furax_pointing *p, const furax_noise *n, const float *d, double *a64, float4 *lo,
                               cudaStream_t st, const TplView *tv)
{
    if (tv)
        return launch_dyn(df_rhs_kernel<MODE, B, true>, (unsigned)p->n_tiles, FT, kDfRhsSmem, st, p->d_tiles, p->view(),
                          n->view(), d, a64, lo, *tv);
    return launch_dyn(df_rhs_kernel<MODE, B, false>, (unsigned)p->n_tiles, FT, kDfRhsSmem, st, p->d_tiles, p->view(),
                      n->view(), d, a64, lo, TplView{});
}

static furax_status launch_df_rhs_f32(const furax_pointing *p, const furax_noise *n, const float *d, double *a64,
                                      cudaStream_t st, const TplView *tv)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    furax_status rc;
    const int64_t np = p->npix_total;
    if ((rc = ensure_ws(pm, (void **)&pm->ws_df_lo, sizeof(float4) * np))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(pm->ws_df_lo, 0, sizeof(float4) * np, st), "memset"))) return rc;
    const bool b = n->kind == FURAX_NOISE_BANDED;
    switch (p->mode) {
    case FURAX_POINTING_ON_THE_FLY:
        rc = b ? run_df_rhs<0, true>(p, n, d, a64, pm->ws_df_lo, st, tv) : run_df_rhs<0, false>(p, n, d, a64, pm->ws_df_lo, st, tv);
        break;
    case FURAX_POINTING_CACHE_F32:
        rc = b ? run_df_rhs<1, true>(p, n, d, a64, pm->ws_df_lo, st, tv) : run_df_rhs<1, false>(p, n, d, a64, pm->ws_df_lo, st, tv);
        break;
    case FURAX_POINTING_CACHE_MIXED:
        rc = b ? run_df_rhs<3, true>(p, n, d, a64, pm->ws_df_lo, st, tv) : run_df_rhs<3, false>(p, n, d, a64, pm->ws_df_lo, st, tv);
        break;
    default:
        rc = b ? run_df_rhs<2, true>(p, n, d, a64, pm->ws_df_lo, st, tv) : run_df_rhs<2, false>(p, n, d, a64, pm->ws_df_lo, st, tv);
    }
    if (rc) return rc;
    if ((rc = check_launch("double-FP32 P^T N^-1 d"))) return rc;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, (int64_t)p->n_sm * 8));
    fold_lo_kernel<<<g, 256, 0, st>>>(pm->ws_df_lo, a64, np);
    count_launches(2);
    return check_launch("fold low words");
}

template <int MODE, bool B>
static furax_status run_df_apply(const furax_pointing *p, const furax_noise *n, const float4 *x2, double *a64,
                                 float4 *lo, cudaStream_t st)
{
    return launch_dyn(df_apply_kernel<MODE, B>, (unsigned)p->n_tiles, FT, kDfApplySmem, st, p->d_tiles, p->view(),
                      n->view(), x2, a64, lo);
}

// acc64 += P^T N^-1 P x on the FP32 units: split x, apply, fold the low words.
static furax_status launch_df_apply(const furax_pointing *p, const furax_noise *n, const double *x, double *a64,
                                    cudaStream_t st)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    furax_status rc;
    const int64_t np = p->npix_total;
    if ((rc = ensure_ws(pm, (void **)&pm->ws_x2, sizeof(float4) * 2 * np))) return rc;
    if ((rc = ensure_ws(pm, (void **)&pm->ws_df_lo, sizeof(float4) * np))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(pm->ws_df_lo, 0, sizeof(float4) * np, st), "memset"))) return rc;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, (int64_t)p->n_sm * 8));
    split_map_df_kernel<<<g, 256, 0, st>>>(x, pm->ws_x2, np);
    count_launches(1);
    if ((rc = check_launch("double-FP32 split of the map"))) return rc;
    const bool b = n->kind == FURAX_NOISE_BANDED;
    switch (p->mode) {
    case FURAX_POINTING_ON_THE_FLY:
        rc = b ? run_df_apply<0, true>(p, n, pm->ws_x2, a64, pm->ws_df_lo, st) : run_df_apply<0, false>(p, n, pm->ws_x2, a64, pm->ws_df_lo, st);
        break;
    case FURAX_POINTING_CACHE_F32:
        rc = b ? run_df_apply<1, true>(p, n, pm->ws_x2, a64, pm->ws_df_lo, st) : run_df_apply<1, false>(p, n, pm->ws_x2, a64, pm->ws_df_lo, st);
        break;
    case FURAX_POINTING_CACHE_MIXED:
        rc = b ? run_df_apply<3, true>(p, n, pm->ws_x2, a64, pm->ws_df_lo, st) : run_df_apply<3, false>(p, n, pm->ws_x2, a64, pm->ws_df_lo, st);
        break;
    default:
        rc = b ? run_df_apply<2, true>(p, n, pm->ws_x2, a64, pm->ws_df_lo, st) : run_df_apply<2, false>(p, n, pm->ws_x2, a64, pm->ws_df_lo, st);
    }
    if (rc) return rc;
    count_launches(1);
    if ((rc = check_launch("double-FP32 P^T N^-1 P"))) return rc;
    fold_lo_kernel<<<g, 256, 0, st>>>(pm->ws_df_lo, a64, np);
    count_launches(1);
    return check_launch("fold low words");
}

template <int MODE, typename DT>
static furax_status run_chi2_df(const furax_pointing *p, const furax_noise *n, const DT *d, const float4 *m2,
                                double *chi2, double *gm, float4 *lo, double *gp, cudaStream_t st)
{
    if (n->kind == FURAX_NOISE_BANDED)
        return launch_dyn(chi2_df_kernel<MODE, true, DT>, (unsigned)p->n_tiles, FT, kDfApplySmem, st, p->d_tiles,
                          p->view(), n->view(), d, m2, chi2, gm, lo, gp);
    return launch_dyn(chi2_df_kernel<MODE, false, DT>, (unsigned)p->n_tiles, FT, kDfApplySmem, st, p->d_tiles,
                      p->view(), n->view(), d, m2, chi2, gm, lo, gp);
}

template <typename DT>
static furax_status dispatch_chi2_df(const furax_pointing *p, const furax_noise *n, const DT *d, const float4 *m2,
                                     double *chi2, double *gm, float4 *lo, double *gp, cudaStream_t st)
{
    switch (p->mode) {
    case FURAX_POINTING_ON_THE_FLY: return run_chi2_df<0, DT>(p, n, d, m2, chi2, gm, lo, gp, st);
    case FURAX_POINTING_CACHE_F32: return run_chi2_df<1, DT>(p, n, d, m2, chi2, gm, lo, gp, st);
    case FURAX_POINTING_CACHE_MIXED: return run_chi2_df<3, DT>(p, n, d, m2, chi2, gm, lo, gp, st);
    default: return run_chi2_df<2, DT>(p, n, d, m2, chi2, gm, lo, gp, st);
    }
}

// chi^2 and gradients in double-FP32 (the outputs are cleared by the caller): split m, run,
// fold the map gradient's low words.
furax_status launch_chi2_df(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, const double *m,
                            double *chi2, double *grad_map, double *grad_psi, cudaStream_t st)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    furax_status rc;
    const int64_t np = p->npix_total;
    if ((rc = ensure_ws(pm, (void **)&pm->ws_x2, sizeof(float4) * 2 * np))) return rc;
    if ((rc = ensure_ws(pm, (void **)&pm->ws_df_lo, sizeof(float4) * np))) return rc;
    if (grad_map && (rc = check_cuda(cudaMemsetAsync(pm->ws_df_lo, 0, sizeof(float4) * np, st), "memset"))) return rc;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((np + 255) / 256, (int64_t)p->n_sm * 8));
    split_map_df_kernel<<<g, 256, 0, st>>>(m, pm->ws_x2, np);
    count_launches(1);
    if ((rc = check_launch("double-FP32 split of the map"))) return rc;
    rc = d_t == FURAX_F64
             ? dispatch_chi2_df<double>(p, n, (const double *)d, pm->ws_x2, chi2, grad_map, pm->ws_df_lo, grad_psi, st)
             : dispatch_chi2_df<float>(p, n, (const float *)d, pm->ws_x2, chi2, grad_map, pm->ws_df_lo, grad_psi, st);
    if (rc) return rc;
    count_launches(1);
    if ((rc = check_launch("double-FP32 chi2 and gradients"))) return rc;
    if (!grad_map) return FURAX_OK;
    fold_lo_kernel<<<g, 256, 0, st>>>(pm->ws_df_lo, grad_map, np);
    count_launches(1);
    return check_launch("fold low words");
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
                             double *acc64, cudaStream_t st, const furax_templates *tp)
{
    if (p->n_tiles == 0) return FURAX_OK;
    furax_status rc;
    if (tp && !(d && d_t == FURAX_F32))
        return set_error(FURAX_EINVAL, "internal: the template correction is folded only into the FP32-data right-hand side");
    if (d && d_t == FURAX_F32) {
        const TplView tv = tp ? tp->view() : TplView{};
        return launch_df_rhs_f32(p, n, (const float *)d, acc64, st, tp ? &tv : nullptr);
    }
    if (!d) return launch_df_apply(p, n, x, acc64, st);
    if (d_t == FURAX_F64) rc = dispatch_df<true, double>(p, n, nullptr, (const double *)d, acc64, st);
    else rc = dispatch_df<true, float>(p, n, nullptr, (const float *)d, acc64, st);
    if (rc) return rc;
    count_launches(1);
    return check_launch("double-FP32 P^T N^-1 P");
}

template <int MODE, bool B>
static furax_status prep_df_mode_band()
{
    furax_status rc = FURAX_OK;
    if (!rc) rc = allow_smem((const void *)fused_df_kernel<MODE, B, true, double>, kDfSmem);
    if (!rc) rc = allow_smem((const void *)fused_df_kernel<MODE, B, true, float>, kDfSmem);
    if (!rc && kDfRhsSmem > 48 * 1024) rc = allow_smem((const void *)df_rhs_kernel<MODE, B, false>, kDfRhsSmem);
    if (!rc && kDfRhsSmem > 48 * 1024) rc = allow_smem((const void *)df_rhs_kernel<MODE, B, true>, kDfRhsSmem);
    if (!rc && kDfApplySmem > 48 * 1024) rc = allow_smem((const void *)df_apply_kernel<MODE, B>, kDfApplySmem);
    if (!rc && kDfApplySmem > 48 * 1024) rc = allow_smem((const void *)chi2_df_kernel<MODE, B, double>, kDfApplySmem);
    if (!rc && kDfApplySmem > 48 * 1024) rc = allow_smem((const void *)chi2_df_kernel<MODE, B, float>, kDfApplySmem);
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
