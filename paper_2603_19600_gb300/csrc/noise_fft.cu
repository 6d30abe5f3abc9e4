// N^-1 for long symmetric bands by overlap-save (SymmetricBandToeplitzOperator, Table 2: "direct
// convolution, FFT, overlap and save"; the operator "central to correlated noise modeling").
//
// y_t = sum_{k=-H}^{H} c_|k| x_{t+k} over 0 <= t+k < ns (the same finite section as the direct
// band) is computed block by block: a block of L = 8192 input samples [s - H, s - H + L) (zeros
// outside the stream) is transformed, multiplied by the spectrum of the band arranged circularly,
// and transformed back; its outputs [H, L - H) are free of wrap-around and give y over
// [s, s + L - 2H). The band is real and symmetric, so its spectrum is real and the transform of
// x1 + i x2 carries two blocks of one detector at once (real part: first block, imaginary part:
// second block).
//
// The transform: one CTA per pair of blocks, L complex values in shared memory, radix-2 stages
// with a synchronisation between stages; the forward pass is decimation in frequency (natural
// order in, bit-reversed order out), the spectrum is stored in that bit-reversed order, and the
// inverse pass is decimation in time (bit-reversed in, natural out), so no permutation is done.
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

// Forward transform (exp(-2 pi i jk/L)), natural order in, bit-reversed order out.
template <typename T2>
__device__ __forceinline__ void fft_forward_dif(T2 *z, const T2 *__restrict__ tw)
{
    for (int s = 0; s < kFftLog; ++s) {
        const int lh = kFftLog - 1 - s;   // log2 of the butterfly span
        const int half = 1 << lh;
        for (int b = threadIdx.x; b < kFftL / 2; b += kFftThreads) {
            const int pos = b & (half - 1);
            const int i = ((b >> lh) << (lh + 1)) + pos;
            const T2 u = z[i], v = z[i + half];
            z[i] = T2{u.x + v.x, u.y + v.y};
            z[i + half] = cmul(T2{u.x - v.x, u.y - v.y}, tw[pos << s]);
        }
        __syncthreads();
    }
}

// Inverse transform without the 1/L (exp(+2 pi i jk/L)), bit-reversed order in, natural out.
template <typename T2>
__device__ __forceinline__ void fft_inverse_dit(T2 *z, const T2 *__restrict__ tw)
{
    for (int s = kFftLog - 1; s >= 0; --s) {
        const int lh = kFftLog - 1 - s;
        const int half = 1 << lh;
        for (int b = threadIdx.x; b < kFftL / 2; b += kFftThreads) {
            const int pos = b & (half - 1);
            const int i = ((b >> lh) << (lh + 1)) + pos;
            T2 w = tw[pos << s];
            w.y = -w.y;
            const T2 u = z[i], v = cmul(z[i + half], w);
            z[i] = T2{u.x + v.x, u.y + v.y};
            z[i + half] = T2{u.x - v.x, u.y - v.y};
        }
        __syncthreads();
    }
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
    fft_forward_dif<T2>(z, tw);
    const T *sp = spec + gdet * kFftL;
    for (int j = threadIdx.x; j < kFftL; j += kFftThreads) {
        const T f = sp[j];
        z[j].x *= f;
        z[j].y *= f;
    }
    __syncthreads();
    fft_inverse_dit<T2>(z, tw);
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
