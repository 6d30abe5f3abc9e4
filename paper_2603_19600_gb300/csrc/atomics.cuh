// Fire-and-forget reductions into global memory (resolved in L2) and the compensated
// FP32 accumulation used by FURAX_ACC_F32_KAHAN.
#pragma once
#include <cstdint>

namespace fx {

__device__ __forceinline__ void red_add_f64(double *a, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(a), "d"(v) : "memory");
}

__device__ __forceinline__ void red_add_s32(int32_t *a, int32_t v)
{
    asm volatile("red.global.add.s32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// One 16-byte vector reduction: four FP32 adds at the cost of one L2 atomic operation.
__device__ __forceinline__ void red_add_v4(float4 *a, float4 v)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ float4 atom_add_v4(float4 *a, float4 v)
{
    float4 r;
    asm volatile("atom.global.v4.f32.add {%0, %1, %2, %3}, [%4], {%5, %6, %7, %8};"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
    return r;
}

// Rounding error of s = fl(a + b) (Knuth's two-sum): a + b = s + err exactly in
// round-to-nearest FP32.
__device__ __forceinline__ float two_sum_err(float a, float b, float s)
{
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    return __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// Rounding error of each component of the FP32 addition old + v that an atomic performed.
__device__ __forceinline__ float4 kahan_error_v4(float4 old, float4 v)
{
    float4 e;
    e.x = two_sum_err(old.x, v.x, __fadd_rn(old.x, v.x));
    e.y = two_sum_err(old.y, v.y, __fadd_rn(old.y, v.y));
    e.z = two_sum_err(old.z, v.z, __fadd_rn(old.z, v.z));
    e.w = 0.f;
    return e;
}

// Warp-cooperative FP64 reductions into pixel records of NC doubles, base[NC pix + c]: every lane
// offers one sample (pix < 0: none) and its NC values, and the warp's 32 NC reductions leave as NC
// instructions in which lane L of instruction i adds component (32 i + L) mod NC of the sample of
// lane (32 i + L) / NC. Consecutive lanes then address the consecutive doubles of one record, which
// the L2 serves together: for NC = 3, 31 % more reductions per second on this GPU than one lane
// issuing a record's three (furax_probe_l2 kinds 5 and 3). The samples are exchanged through a
// warp-private staging area (buf: 32 NC values, ibuf: 32 ints), which costs fewer instructions than
// NC shuffles per instruction; FP32 values are widened to FP64 after the exchange. All 32 lanes of
// the warp call it, with the same base.
template <int NC, typename T>
__device__ __forceinline__ void red_add_f64_records_warp(double *base, int32_t pix, const T (&v)[NC], T *buf,
                                                         int32_t *ibuf)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < NC; ++c) buf[NC * lane + c] = v[c];
    ibuf[lane] = pix;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        const int f = 32 * i + lane;
        const int src = f / NC, comp = f - NC * src;
        const int32_t p = ibuf[src];
        if (p >= 0) red_add_f64(base + (int64_t)NC * p + comp, (double)buf[f]);
    }
    __syncwarp();   // the staging area is free again
}

// Compensated FP32 accumulators are interleaved: pixel i's sum is hi[2i] and its compensation
// lo[2i], with lo = hi + 1, so both words of a pixel share one 32-byte sector and the reduction of
// the rounding error hits the sector that the returning atomic just brought into L2. Plain FP32
// accumulators are hi[i].
constexpr int kKahanStride = 2;

// Compensated accumulation: the atomic returns the value it added to, so the exact
// rounding error of that addition can be recomputed here and accumulated in `lo`.
// hi + lo then equals the exact sum up to second-order terms, whatever the order in
// which the atomics were applied.
__device__ __forceinline__ void kahan_add_v4(float4 *hi, float4 *lo, float4 v)
{
    float4 old = atom_add_v4(hi, v);
    float4 e;
    e.x = two_sum_err(old.x, v.x, __fadd_rn(old.x, v.x));
    e.y = two_sum_err(old.y, v.y, __fadd_rn(old.y, v.y));
    e.z = two_sum_err(old.z, v.z, __fadd_rn(old.z, v.z));
    e.w = 0.f;
    red_add_v4(lo, e);
}

}  // namespace fx
