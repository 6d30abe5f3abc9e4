// Device probes: the per-unit rates that bound the map-making kernels (FP64 and FP32 FMA issue,
// L2-resident random gathers and reductions), measured on the GPU at hand, and a bit-exact check
// of the encoding-level FP32/FP64 conversions (dfloat.cuh) against the hardware conversions.
// None of this has a counterpart in the paper: these are measurement instruments for the roofline
// denominators of kernels that are not HBM-bound.
#include "internal.cuh"
#include "atomics.cuh"
#include "dfloat.cuh"
#include "stencil.cuh"

namespace fx {

constexpr int PB = 256;      // threads per probe block
constexpr int kChains = 8;   // independent FMA chains per thread

__global__ void probe_convert_kernel(const double *__restrict__ in64, float *__restrict__ out32,
                                     const float *__restrict__ in32, double *__restrict__ out64, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (in64) out32[i] = f64_to_f32_bits(in64[i]);
        if (in32) out64[i] = f32_to_f64_bits(in32[i]);
    }
}

// kChains independent chains a <- a * b + c per thread; the sum is stored only if it is exactly
// zero (never, for these operands), so the work cannot be removed.
template <typename T>
__global__ void __launch_bounds__(PB) probe_fma_kernel(int64_t iters, T b, T c, T *__restrict__ sink)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(1) + T(threadIdx.x) * T(1e-3) + T(k);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if constexpr (sizeof(T) == 8) a[k] = __fma_rn(a[k], b, c);
            else a[k] = __fmaf_rn(a[k], b, c);
        }
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == T(0)) sink[0] = s;
}

// The same with packed fma.rn.f32x2 (two FP32 FMAs per instruction).
__global__ void __launch_bounds__(PB) probe_fma_x2_kernel(int64_t iters, float b, float c, float *__restrict__ sink)
{
    unsigned long long a[kChains];
    const unsigned long long bb = pack_f32x2(b, b), cc = pack_f32x2(c, c);
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = pack_f32x2(1.f + threadIdx.x * 1e-3f + k, 2.f + k);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        unpack_f32x2(a[k], lo, hi);
        s += lo + hi;
    }
    if (s == 0.f) sink[0] = s;
}

// Random L2 operations at the indices idx[0..n): kind 0 gathers a float4, 1 issues one
// red.add.v4.f32, 2 the compensated pair (atom.add.v4.f32 returning the old value, red.add.v4.f32
// of the rounding error into the second half of the table), 3 three red.add.f64 (one FP64 map
// entry per Stokes component, [ntab][3] records), 4 the same into 32-byte records [ntab][4],
// 5 the same three reductions issued by three consecutive lanes of one instruction (lane 3k + c
// adds component c of index k), so that one warp instruction covers a pixel's whole record;
// 6 kind 5 and 7 kind 0 with kProbeBatch operations per thread in flight (all index loads, then
// all gathers or reductions), so that the L2, not the latency of a thread's index load, sets the
// rate; 8 kind 5 with 64-bit integer reductions (red.add.u64) instead of FP64 ones.
constexpr int kProbeBatch = 8;
__global__ void __launch_bounds__(PB) probe_l2_kernel(int kind, const int32_t *__restrict__ idx, int64_t n,
                                                      float4 *__restrict__ t4, double *__restrict__ t64, int64_t ntab,
                                                      float *__restrict__ sink)
{
    float acc = 0.f;
    const float4 v = make_float4(1e-3f, 2e-3f, 3e-3f, 0.f);
    if (kind == 6 || kind == 7) {
        const int64_t total = kind == 6 ? 3 * n : n;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t f0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f0 < total; f0 += kProbeBatch * stride) {
            int32_t p[kProbeBatch];
#pragma unroll
            for (int b = 0; b < kProbeBatch; ++b) {
                const int64_t f = f0 + b * stride;
                p[b] = f < total ? idx[kind == 6 ? f / 3 : f] : -1;
            }
            if (kind == 6) {
#pragma unroll
                for (int b = 0; b < kProbeBatch; ++b) {
                    const int64_t f = f0 + b * stride;
                    const int c = (int)(f % 3);
                    if (p[b] >= 0) red_add_f64(t64 + 3 * (int64_t)p[b] + c, 1e-3 * (c + 1));
                }
            } else {
                float4 m[kProbeBatch];
#pragma unroll
                for (int b = 0; b < kProbeBatch; ++b) m[b] = p[b] >= 0 ? __ldg(t4 + p[b]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int b = 0; b < kProbeBatch; ++b) acc += m[b].x + m[b].y + m[b].z;
            }
        }
        if (acc == 12345.f) sink[0] = acc;
        return;
    }
    if (kind == 8) {
        unsigned long long *t = reinterpret_cast<unsigned long long *>(t64);
        for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < 3 * n; f += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = f / 3;
            const int c = (int)(f - 3 * i);
            asm volatile("red.global.add.u64 [%0], %1;" ::"l"(t + 3 * (int64_t)idx[i] + c), "l"((unsigned long long)(c + 1))
                         : "memory");
        }
        return;
    }
    if (kind == 5) {
        for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < 3 * n; f += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = f / 3;
            const int c = (int)(f - 3 * i);
            red_add_f64(t64 + 3 * (int64_t)idx[i] + c, 1e-3 * (c + 1));
        }
        return;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = idx[i];
        if (kind == 0) {
            const float4 m = __ldg(t4 + p);
            acc += m.x + m.y + m.z;
        } else if (kind == 1) {
            red_add_v4(t4 + p, v);
        } else if (kind == 2) {
            kahan_add_v4(t4 + p, t4 + ntab + p, v);
        } else {
            const int64_t stride = kind == 3 ? 3 : 4;
            red_add_f64(t64 + stride * p, 1e-3);
            red_add_f64(t64 + stride * p + 1, 2e-3);
            red_add_f64(t64 + stride * p + 2, 3e-3);
        }
    }
    if (acc == 12345.f) sink[0] = acc;
}

}  // namespace fx

using namespace fx;

extern "C" furax_status furax_probe_convert(const double *in64, float *out32, const float *in32, double *out64,
                                            int64_t n, void *stream)
{
    if (n < 0) return set_error(FURAX_EINVAL, "n must be >= 0");
    if ((in64 && !out32) || (in32 && !out64)) return set_error(FURAX_EINVAL, "each input needs its output");
    if (n == 0 || (!in64 && !in32)) return FURAX_OK;
    const unsigned g = (unsigned)std::min<int64_t>((n + PB - 1) / PB, 4096);
    probe_convert_kernel<<<g, PB, 0, (cudaStream_t)stream>>>(in64, out32, in32, out64, n);
    count_launches(1);
    return check_launch("conversion probe");
}

extern "C" furax_status furax_probe_fma(int32_t kind, int64_t iters, void *sink, double *flops, void *stream)
{
    if (kind < 0 || kind > 2) return set_error(FURAX_EINVAL, "kind must be 0 (FP64), 1 (FP32) or 2 (packed FP32)");
    if (iters < 1 || !sink || !flops) return set_error(FURAX_EINVAL, "iters >= 1, sink and flops are required");
    int dev = 0, sms = 1;
    furax_status rc = check_cuda(cudaGetDevice(&dev), "device");
    if (!rc) rc = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (rc) return rc;
    const unsigned g = (unsigned)(8 * sms);   // 8 x 256 threads per SM: enough warps to cover the latency
    cudaStream_t st = (cudaStream_t)stream;
    const double per_thread = 2.0 * kChains * (double)iters * (kind == 2 ? 2.0 : 1.0);
    *flops = per_thread * g * PB;
    if (kind == 0) probe_fma_kernel<double><<<g, PB, 0, st>>>(iters, 0.9999999, 1e-9, (double *)sink);
    else if (kind == 1) probe_fma_kernel<float><<<g, PB, 0, st>>>(iters, 0.9999f, 1e-6f, (float *)sink);
    else probe_fma_x2_kernel<<<g, PB, 0, st>>>(iters, 0.9999f, 1e-6f, (float *)sink);
    count_launches(1);
    return check_launch("FMA probe");
}

extern "C" furax_status furax_probe_l2(int32_t kind, const int32_t *idx, int64_t n, void *table, int64_t ntable,
                                       void *sink, void *stream)
{
    if (kind < 0 || kind > 8) return set_error(FURAX_EINVAL, "kind must be in [0, 8]");
    if (!idx || !table || !sink || n < 0 || ntable < 1) return set_error(FURAX_EINVAL, "invalid probe arguments");
    if (n == 0) return FURAX_OK;
    int dev = 0, sms = 1;
    furax_status rc = check_cuda(cudaGetDevice(&dev), "device");
    if (!rc) rc = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (rc) return rc;
    // indices are the caller's: each must lie in [0, ntable) (float4 kinds: table holds 2 ntable
    // float4 for kind 2; kinds 3, 5, 6: 3 ntable doubles, kind 8 3 ntable 64-bit integers; kind 4: 4
    // ntable doubles)
    const unsigned g = (unsigned)std::min<int64_t>((n + PB - 1) / PB, 8LL * sms);
    probe_l2_kernel<<<g, PB, 0, (cudaStream_t)stream>>>(kind, idx, n, (float4 *)table, (double *)table, ntable,
                                                         (float *)sink);
    count_launches(1);
    return check_launch("L2 probe");
}
