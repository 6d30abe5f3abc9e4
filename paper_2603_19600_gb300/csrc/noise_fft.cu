// N^-1 for long symmetric bands by overlap-save (SymmetricBandToeplitzOperator, Table 2, offers a
// direct, an FFT and an overlap-save evaluation; the paper uses the operator for correlated noise).
//
// y_t = sum_{k=-H}^{H} c_|k| x_{t+k} over 0 <= t+k < ns (the same finite section as the direct
// band) is computed block by block: a block of L = 8192 input samples [s - H, s - H + L) (zeros
// outside the stream) is transformed, multiplied by the spectrum of the band arranged circularly,
// and transformed back; its outputs [H, L - H) are free of wrap-around and give y over
// [s, s + L - 2H). The band is real and symmetric, so its spectrum is real and the transform of
// x1 + i x2 carries two blocks of one detector at once (real part: first block, imaginary part:
// second block).
//
// The transform: one CTA per pair of blocks, L complex values in shared memory. Spans of 32 and
// more go in radix-4 passes (two radix-2 stages each, a synchronisation between passes); the
// spans below 32, whose shared-memory patterns conflict, run in registers with one warp per 32
// consecutive values. The forward transform is decimation in frequency (natural order in,
// bit-reversed order out), the spectrum is stored in that bit-reversed order, and the inverse is
// decimation in time (bit-reversed in, natural out), so no permutation is done.
#include "tile.cuh"

namespace fx {

constexpr int kFftLog = 13;
constexpr int kFftL = 1 << kFftLog;
constexpr int kFftThreads = 512;
static_assert(2 * (kLongTaps - 1) < kFftL, "a block must hold the band on both sides of its outputs");

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    return T2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// (-i) z and (+i) z
template <typename T2>
__device__ __forceinline__ T2 mul_neg_i(T2 z) { return T2{z.y, -z.x}; }
template <typename T2>
__device__ __forceinline__ T2 mul_pos_i(T2 z) { return T2{-z.y, z.x}; }

// Two consecutive decimation-in-frequency radix-2 stages (spans h = 2^LH, then h/2) fused into one
// pass of 4-point butterflies on z[i], z[i + h/2], z[i + h], z[i + 3h/2]. LH is a compile-time
// constant so that, for spans of 1024 and less, a thread's butterflies share their twiddles.
template <int LH, typename T2>
__device__ __forceinline__ void dif_radix4(T2 *z, const T2 *__restrict__ tw)
{
    constexpr int lh = LH;
    constexpr int hh = 1 << (lh - 1);
    constexpr int sh = kFftLog - 1 - lh;   // W_2h^p = tw[p << sh], W_h^p = tw[p << (sh + 1)]
#pragma unroll
    for (int g = threadIdx.x; g < kFftL / 4; g += kFftThreads) {
        const int pos = g & (hh - 1);
        const int i = ((g >> (lh - 1)) << (lh + 1)) + pos;
        const T2 a0 = z[i], a1 = z[i + hh], a2 = z[i + 2 * hh], a3 = z[i + 3 * hh];
        const T2 w1 = tw[pos << sh], w2 = tw[pos << (sh + 1)];
        const T2 b0 = T2{a0.x + a2.x, a0.y + a2.y}, b1 = T2{a1.x + a3.x, a1.y + a3.y};
        const T2 c0 = cmul(T2{a0.x - a2.x, a0.y - a2.y}, w1);
        const T2 c1 = mul_neg_i(cmul(T2{a1.x - a3.x, a1.y - a3.y}, w1));
        z[i] = T2{b0.x + b1.x, b0.y + b1.y};
        z[i + hh] = cmul(T2{b0.x - b1.x, b0.y - b1.y}, w2);
        z[i + 2 * hh] = T2{c0.x + c1.x, c0.y + c1.y};
        z[i + 3 * hh] = cmul(T2{c0.x - c1.x, c0.y - c1.y}, w2);
    }
    __syncthreads();
}

// Two consecutive decimation-in-time radix-2 stages of the inverse (spans h/2, then h = 2^LH).
template <int LH, typename T2>
__device__ __forceinline__ void dit_radix4_inv(T2 *z, const T2 *__restrict__ tw)
{
    constexpr int lh = LH;
    constexpr int hh = 1 << (lh - 1);
    constexpr int sh = kFftLog - 1 - lh;
#pragma unroll
    for (int g = threadIdx.x; g < kFftL / 4; g += kFftThreads) {
        const int pos = g & (hh - 1);
        const int i = ((g >> (lh - 1)) << (lh + 1)) + pos;
        const T2 a0 = z[i], a1 = z[i + hh], a2 = z[i + 2 * hh], a3 = z[i + 3 * hh];
        T2 w1 = tw[pos << sh], w2 = tw[pos << (sh + 1)];
        w1.y = -w1.y;
        w2.y = -w2.y;
        T2 v = cmul(a1, w2);
        const T2 b0 = T2{a0.x + v.x, a0.y + v.y}, b1 = T2{a0.x - v.x, a0.y - v.y};
        v = cmul(a3, w2);
        const T2 b2 = T2{a2.x + v.x, a2.y + v.y}, b3 = T2{a2.x - v.x, a2.y - v.y};
        v = cmul(b2, w1);
        z[i] = T2{b0.x + v.x, b0.y + v.y};
        z[i + 2 * hh] = T2{b0.x - v.x, b0.y - v.y};
        v = mul_pos_i(cmul(b3, w1));
        z[i + hh] = T2{b1.x + v.x, b1.y + v.y};
        z[i + 3 * hh] = T2{b1.x - v.x, b1.y - v.y};
    }
    __syncthreads();
}

// Forward transform (exp(-2 pi i jk/L)), natural order in, bit-reversed order out: six radix-4
// passes (spans 4096 and 2048, ..., 4 and 2), then the radix-2 stage of span 1.
template <typename T2>
__device__ __forceinline__ void fft_forward_dif(T2 *z, const T2 *__restrict__ tw)
{
    static_assert(kFftLog == 13, "pass schedule written for L = 8192");
    dif_radix4<12>(z, tw);
    dif_radix4<10>(z, tw);
    dif_radix4<8>(z, tw);
    dif_radix4<6>(z, tw);
    dif_radix4<4>(z, tw);
    dif_radix4<2>(z, tw);
    for (int b = threadIdx.x; b < kFftL / 2; b += kFftThreads) {   // span 1: pairs (2b, 2b + 1)
        const T2 u = z[2 * b], v = z[2 * b + 1];
        z[2 * b] = T2{u.x + v.x, u.y + v.y};
        z[2 * b + 1] = T2{u.x - v.x, u.y - v.y};
    }
    __syncthreads();
}

template <typename T2>
__device__ __forceinline__ T2 shfl_xor2(T2 v, int m)
{
    return T2{__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}

// Spans 16 .. 1 of the forward transform, the spectrum multiply and spans 1 .. 16 of the inverse,
// on 32 consecutive values held one per lane (butterfly partners by xor shuffles): the stages
// whose shared-memory access patterns conflict, done without shared memory.
template <typename T, typename T2>
__device__ __forceinline__ void fft_tail_in_warps(T2 *z, const T2 *__restrict__ tw, const T *__restrict__ sp)
{
    const int lane = threadIdx.x & 31;
    T2 w[5];   // this lane's twiddle at spans 1, 2, 4, 8, 16 (the same for every block)
#pragma unroll
    for (int ls = 0; ls <= 4; ++ls) w[ls] = tw[(lane & ((1 << ls) - 1)) << (kFftLog - 1 - ls)];
    for (int base = threadIdx.x & ~31; base < kFftL; base += kFftThreads) {
        T2 x = z[base + lane];
#pragma unroll
        for (int ls = 4; ls >= 0; --ls) {
            const int s = 1 << ls;
            const T2 p = shfl_xor2(x, s);
            x = (lane & s) ? cmul(T2{p.x - x.x, p.y - x.y}, w[ls]) : T2{x.x + p.x, x.y + p.y};
        }
        const T f = sp[base + lane];
        x.x *= f;
        x.y *= f;
#pragma unroll
        for (int ls = 0; ls <= 4; ++ls) {
            const int s = 1 << ls;
            const T2 p = shfl_xor2(x, s);
            const T2 wc = T2{w[ls].x, -w[ls].y};
            if (lane & s) {
                const T2 t = cmul(x, wc);
                x = T2{p.x - t.x, p.y - t.y};
            } else {
                const T2 t = cmul(p, wc);
                x = T2{x.x + t.x, x.y + t.y};
            }
        }
        z[base + lane] = x;
    }
    __syncthreads();
}

// tw[m] = exp(-2 pi i m / L), m < L/2.
__global__ void fft_twiddle_kernel(double2 *__restrict__ tw64, float2 *__restrict__ tw32)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= kFftL / 2) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)kFftL, &s, &c);
    tw64[m] = make_double2(c, -s);
    tw32[m] = make_float2((float)c, (float)-s);
}

// Spectrum of each detector's band, arranged circularly (h[k] = c_|k| at k mod L), in the
// bit-reversed order of the forward transform. It is real: the imaginary part is dropped.
__global__ void __launch_bounds__(kFftThreads) fft_spectrum_kernel(const double *__restrict__ taps, int ntaps,
                                                                   const double2 *__restrict__ tw64,
                                                                   double *__restrict__ spec64,
                                                                   float *__restrict__ spec32)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    double2 *z = reinterpret_cast<double2 *>(fsm);
    const int64_t det = blockIdx.x;
    const double *c = taps + det * ntaps;
    for (int j = threadIdx.x; j < kFftL; j += kFftThreads) {
        const int k = j <= kFftL / 2 ? j : kFftL - j;
        z[j] = make_double2(k < ntaps ? c[k] : 0.0, 0.0);
    }
    __syncthreads();
    fft_forward_dif<double2>(z, tw64);
    for (int j = threadIdx.x; j < kFftL; j += kFftThreads) {
        spec64[det * kFftL + j] = z[j].x;
        spec32[det * kFftL + j] = (float)z[j].x;
    }
}

template <typename T, typename DT>
__global__ void __launch_bounds__(kFftThreads) ninv_fft_kernel(const FftItem *__restrict__ items,
                                                               const ObsInfo *__restrict__ obs, int halo,
                                                               const T *__restrict__ spec,
                                                               const typename Cplx<T>::type *__restrict__ tw,
                                                               const DT *__restrict__ in, DT *__restrict__ out)
{
    using T2 = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char fsm[];
    T2 *z = reinterpret_cast<T2 *>(fsm);
    const FftItem it = items[blockIdx.x];
    const ObsInfo ob = obs[it.obs];
    const int64_t gdet = ob.det_off + it.det;
    const int m = kFftL - 2 * halo;         // outputs per block
    const int64_t ns = ob.nsamp;
    const int64_t b1 = it.q0 * m, b2 = b1 + m;   // first outputs of the two blocks
    const bool two = b2 < ns;
    const DT *row = in + ob.tod_off + (int64_t)it.det * ns;
    for (int j = threadIdx.x; j < kFftL; j += kFftThreads) {
        const int64_t t1 = b1 - halo + j, t2 = b2 - halo + j;
        const T re = (t1 >= 0 && t1 < ns) ? T(row[t1]) : T(0);
        const T im = (two && t2 >= 0 && t2 < ns) ? T(row[t2]) : T(0);
        z[j] = T2{re, im};
    }
    __syncthreads();
    // forward spans 4096 .. 32 (radix-4 passes), then spans 16 .. 1, the spectrum and the inverse
    // spans 1 .. 16 in registers, then the inverse spans 32 .. 4096
    dif_radix4<12>(z, tw);
    dif_radix4<10>(z, tw);
    dif_radix4<8>(z, tw);
    dif_radix4<6>(z, tw);
    fft_tail_in_warps<T, T2>(z, tw, spec + gdet * kFftL);
    dit_radix4_inv<6>(z, tw);
    dit_radix4_inv<8>(z, tw);
    dit_radix4_inv<10>(z, tw);
    dit_radix4_inv<12>(z, tw);
    const T scale = T(1) / T(kFftL);
    DT *orow = out + ob.tod_off + (int64_t)it.det * ns;
    for (int j = threadIdx.x; j < m; j += kFftThreads) {
        const int64_t t1 = b1 + j, t2 = b2 + j;
        if (t1 < ns) orow[t1] = DT(z[halo + j].x * scale);
        if (two && t2 < ns) orow[t2] = DT(z[halo + j].y * scale);
    }
}

constexpr size_t kFftSmem32 = sizeof(float2) * kFftL;
constexpr size_t kFftSmem64 = sizeof(double2) * kFftL;

furax_status prepare_noise_fft(furax_noise *n, const std::vector<ObsInfo> &obs, cudaStream_t st)
{
    const int halo = n->ntaps - 1;
    const int64_t m = kFftL - 2 * halo;
    std::vector<FftItem> items;
    for (int32_t o = 0; o < (int32_t)obs.size(); ++o) {
        const int64_t nb = (obs[o].nsamp + m - 1) / m;   // blocks per detector stream
        for (int32_t d = 0; d < obs[o].ndet; ++d)
            for (int64_t q = 0; q < nb; q += 2) items.push_back(FftItem{q, o, d});
    }
    n->n_fft_items = (int64_t)items.size();
    if (n->n_fft_items >= (1LL << 31)) return set_error(FURAX_EINVAL, "too many transform blocks");
    const int64_t nd = n->ndet_total;
    furax_status rc = FURAX_OK;
    auto alloc = [&](void **p, size_t bytes) {
        if (!rc) rc = check_cuda(cudaMalloc(p, std::max<size_t>(bytes, 16)), "long-band noise workspace");
    };
    alloc((void **)&n->fft_items, sizeof(FftItem) * items.size());
    alloc((void **)&n->tw64, sizeof(double2) * kFftL / 2);
    alloc((void **)&n->tw32, sizeof(float2) * kFftL / 2);
    alloc((void **)&n->spec64, sizeof(double) * kFftL * nd);
    alloc((void **)&n->spec32, sizeof(float) * kFftL * nd);
    if (rc) return rc;
    if (!items.empty() &&
        (rc = check_cuda(cudaMemcpyAsync(n->fft_items, items.data(), sizeof(FftItem) * items.size(),
                                         cudaMemcpyHostToDevice, st), "copy transform blocks")))
        return rc;
    // kernel attributes are set here, outside any stream capture of a later solve
    if ((rc = allow_smem((const void *)fft_spectrum_kernel, kFftSmem64))) return rc;
    if ((rc = allow_smem((const void *)ninv_fft_kernel<double, double>, kFftSmem64))) return rc;
    if ((rc = allow_smem((const void *)ninv_fft_kernel<float, float>, kFftSmem32))) return rc;
    fft_twiddle_kernel<<<(kFftL / 2 + 255) / 256, 256, 0, st>>>(n->tw64, n->tw32);
    if (nd > 0) fft_spectrum_kernel<<<(unsigned)nd, kFftThreads, kFftSmem64, st>>>(n->p64, n->ntaps, n->tw64, n->spec64, n->spec32);
    count_launches(2);
    if ((rc = check_launch("long-band noise setup"))) return rc;
    // the items vector is read by the copy above: wait before it goes out of scope
    return check_cuda(cudaStreamSynchronize(st), "long-band noise setup");
}

furax_status launch_ninv_fft(const furax_noise *n, const void *in, void *out, int dtype, cudaStream_t st)
{
    if (n->n_fft_items == 0) return FURAX_OK;
    const unsigned g = (unsigned)n->n_fft_items;
    const int halo = n->ntaps - 1;
    furax_status rc;
    if (dtype == FURAX_F64) {
        if ((rc = launch_dyn(ninv_fft_kernel<double, double>, g, kFftThreads, kFftSmem64, st, n->fft_items, n->d_obs,
                             halo, (const double *)n->spec64, (const double2 *)n->tw64, (const double *)in,
                             (double *)out)))
            return rc;
    } else {
        if ((rc = launch_dyn(ninv_fft_kernel<float, float>, g, kFftThreads, kFftSmem32, st, n->fft_items, n->d_obs,
                             halo, (const float *)n->spec32, (const float2 *)n->tw32, (const float *)in,
                             (float *)out)))
            return rc;
    }
    count_launches(1);
    return check_launch("N^-1 apply (overlap-save)");
}

}  // namespace fx
