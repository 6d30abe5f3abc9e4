// furax_ptnp_apply_noalloc: the FP32 normal-equations operator for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a memory budget fixed
// up front (an embedding framework's pre-sized pool, a plugin that must not grow the
// process's device footprint), or code that must not synchronise the device, which
// cudaMalloc and cudaFree may do. This entry point takes every input and output from the
// caller and allocates nothing. Its two scratch maps (the FP32 copy of x and the FP32
// accumulator) live in one file-scope __device__ array of fixed size, which every GPU that
// loads the library holds until the process exits.
//
// Limits and behaviour:
//   * at most kNoAllocMaxPix pixels (nside <= 256); larger problems return FURAX_EINVAL;
//   * the first call on a device looks up the array's device address (cudaGetSymbolAddress)
//     with that device current; make that first call before any stream capture;
//   * all calls share the one array and it keeps the last call's contents: the kernels clear
//     what must start at zero, but calls that overlap on the GPU (different streams, or
//     threads, without ordering between them) race on it and give wrong results.
#include <mutex>

#include "internal.cuh"
#include "atomics.cuh"
#include "stencil.cuh"

namespace fx {

constexpr int64_t kNoAllocMaxPix = 12LL * 256 * 256;   // 786,432 pixels: 2 x 12.6 MB of scratch
constexpr int kNoAllocMaxDevices = 64;
constexpr int NT = 256;                                 // threads per tile CTA
constexpr int NR = TILE / NT;                           // outputs per thread
constexpr int NXS = spos(TILE + 2 * kHalo) + 1;

// [0, kNoAllocMaxPix): FP32 copy of x (I, Q, U, 0); [kNoAllocMaxPix, 2 kNoAllocMaxPix): accumulator.
static __device__ __align__(256) float4 g_noalloc_scratch[2 * kNoAllocMaxPix];

// x32 = (float)x on valid pixels (0 elsewhere); accumulator = 0.
__global__ void noalloc_pack_kernel(const double *__restrict__ x, const uint8_t *__restrict__ valid,
                                    float4 *__restrict__ scratch, int64_t npix)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = !valid || valid[i];
        scratch[i] = ok ? make_float4((float)x[3 * i], (float)x[3 * i + 1], (float)x[3 * i + 2], 0.f)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        scratch[kNoAllocMaxPix + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// One CTA per (time chunk, detector) tile: gather P x into shared memory with halos, apply the
// band, scatter y (1, c, s) into the accumulator with one 16-byte reduction per sample.
__global__ void __launch_bounds__(NT) noalloc_tile_kernel(const int32_t *__restrict__ pix, const float *__restrict__ cw,
                                                          const float *__restrict__ sw, int32_t ndet, int64_t nsamp,
                                                          int64_t npix, const float *__restrict__ taps_g, int32_t ntaps,
                                                          float4 *__restrict__ scratch)
{
    __shared__ float xs[NXS];
    __shared__ float taps[MAXTAPS];
    const int64_t chunk = blockIdx.x / ndet;
    const int32_t det = (int32_t)(blockIdx.x % ndet);
    const int64_t t0 = chunk * TILE;
    const int len = (int)std::min<int64_t>(TILE, nsamp - t0);
    const bool banded = ntaps > 1;
    const int halo = banded ? kHalo : 0;
    const int64_t row = (int64_t)det * nsamp;
    const float4 *x32 = scratch;
    float4 *acc = scratch + kNoAllocMaxPix;
    if (threadIdx.x < MAXTAPS) taps[threadIdx.x] = threadIdx.x < ntaps ? taps_g[(int64_t)det * ntaps + threadIdx.x] : 0.f;
    const int nload = len + 2 * halo;
    for (int u = threadIdx.x; u < nload; u += NT) {
        const int64_t t = t0 - halo + u;
        float v = 0.f;
        if (t >= 0 && t < nsamp) {
            const int32_t p = pix[row + t];
            if (p >= 0 && p < npix) {
                const float4 m = x32[p];
                v = fmaf(m.z, sw[row + t], fmaf(m.y, cw[row + t], m.x));
            }
        }
        xs[spos(u)] = v;
    }
    __syncthreads();
    const int base = threadIdx.x * NR;
    if (base >= len) return;
    float y[NR];
    if (banded) {
        band_product<float, NR>(xs, taps, base, y);
    } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) y[r] = xs[spos(base + r)] * taps[0];
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int k = base + r;
        if (k >= len) break;
        const int64_t t = t0 + k;
        const int32_t p = pix[row + t];
        if (p < 0 || p >= npix) continue;
        red_add_v4(acc + p, make_float4(y[r], y[r] * cw[row + t], y[r] * sw[row + t], 0.f));
    }
}

__global__ void noalloc_finalize_kernel(const float4 *__restrict__ scratch, const uint8_t *__restrict__ valid,
                                        double *__restrict__ out, int64_t npix)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = scratch[kNoAllocMaxPix + i];
        const bool ok = !valid || valid[i];
        out[3 * i] = ok ? (double)a.x : 0.0;
        out[3 * i + 1] = ok ? (double)a.y : 0.0;
        out[3 * i + 2] = ok ? (double)a.z : 0.0;
    }
}

// Device address of the scratch array on the current device and the device's SM count, looked
// up once per device (neither lookup allocates).
static furax_status noalloc_scratch(float4 **out, int *n_sm)
{
    static std::mutex mu;
    static float4 *addr[kNoAllocMaxDevices] = {};
    static int sms[kNoAllocMaxDevices] = {};
    int dev = 0;
    furax_status rc = check_cuda(cudaGetDevice(&dev), "current device");
    if (rc) return rc;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(FURAX_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        int n = 0;
        if ((rc = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "scratch symbol address"))) return rc;
        if ((rc = check_cuda(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev), "SM count"))) return rc;
        sms[dev] = n > 0 ? n : 1;
        addr[dev] = static_cast<float4 *>(p);
    }
    *out = addr[dev];
    *n_sm = sms[dev];
    return FURAX_OK;
}

}  // namespace fx

using namespace fx;

extern "C" furax_status furax_ptnp_apply_noalloc(const int32_t *pix, const float *c, const float *s, int32_t ndet,
                                                 int64_t nsamp, int32_t nside, const float *taps, int32_t ntaps,
                                                 const uint8_t *valid, const double *x, double *out, void *stream)
{
    if (!pix || !c || !s || !taps || !x || !out)
        return set_error(FURAX_EINVAL, "pix, c, s, taps, x and out must be device pointers");
    if (x == out) return set_error(FURAX_EINVAL, "x and out must not alias");
    if (ndet < 1 || nsamp < 1) return set_error(FURAX_EINVAL, "ndet and nsamp must be >= 1");
    if (nside < 1) return set_error(FURAX_EINVAL, "nside must be >= 1");
    const int64_t npix = 12LL * nside * nside;
    if (npix > kNoAllocMaxPix)
        return set_error(FURAX_EINVAL, "nside %d needs %lld pixels; this entry point holds scratch for at most %lld "
                         "(nside 256)", nside, (long long)npix, (long long)kNoAllocMaxPix);
    if (ntaps < 1 || ntaps > MAXTAPS) return set_error(FURAX_EINVAL, "ntaps must be in [1, %d]", MAXTAPS);
    const int64_t nchunk = (nsamp + TILE - 1) / TILE;
    if (nchunk * ndet >= (1LL << 31)) return set_error(FURAX_EINVAL, "problem too large for one launch grid");
    float4 *scratch = nullptr;
    int n_sm = 1;
    furax_status rc = noalloc_scratch(&scratch, &n_sm);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // grid-stride vector passes: eight 256-thread blocks per SM at most
    const unsigned vg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((npix + 255) / 256, 8LL * n_sm));
    noalloc_pack_kernel<<<vg, 256, 0, st>>>(x, valid, scratch, npix);
    noalloc_tile_kernel<<<(unsigned)(nchunk * ndet), NT, 0, st>>>(pix, c, s, ndet, nsamp, npix, taps, ntaps, scratch);
    noalloc_finalize_kernel<<<vg, 256, 0, st>>>(scratch, valid, out, npix);
    count_launches(3);
    return check_launch("P^T N^-1 P without allocation");
}
