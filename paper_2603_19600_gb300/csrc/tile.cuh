// Tile geometry and helpers shared by the fused tile kernels (one detector x TILE samples
// per CTA; 16 consecutive outputs per thread).
#pragma once
#include "internal.cuh"
#include "pointing_math.cuh"
#include "atomics.cuh"
#include "stencil.cuh"

namespace fx {

constexpr int FT = 256;            // threads per tile CTA
constexpr int FR = TILE / FT;      // 16 outputs per thread
static_assert(FR == 16, "tile geometry");
constexpr int XS = spos(TILE + 2 * kHalo) + 1;   // shared slots for the tile + halos
constexpr int CS = spos(TILE) + 1;               // shared slots for per-sample stash

template <typename T>
__device__ __forceinline__ void load_taps(const NoiseView &nv, int64_t gdet, T *taps)
{
    if (threadIdx.x < MAXTAPS) {
        T v = T(0);
        if (threadIdx.x < nv.ntaps) {
            if constexpr (sizeof(T) == 4) v = nv.p32[gdet * nv.ntaps + threadIdx.x];
            else v = nv.p64[gdet * nv.ntaps + threadIdx.x];
        }
        taps[threadIdx.x] = v;
    }
}

template <typename T>
__device__ __forceinline__ T white_scale(const NoiseView &nv, int64_t gdet)
{
    if constexpr (sizeof(T) == 4) return nv.p32[gdet];
    else return nv.p64[gdet];
}

constexpr size_t kF32Smem = sizeof(float) * (XS + MAXTAPS + 2 * XS) + sizeof(int32_t) * XS;
constexpr size_t kF64Smem = sizeof(double) * (XS + MAXTAPS + 2 * CS) + sizeof(int32_t) * CS;

// Kernel shared-memory setup for each translation unit (called once, outside stream capture).
furax_status prepare_fused_f32();
furax_status prepare_fused_f64();
furax_status prepare_fused_df();
furax_status prepare_fused_tma();

// Cached FP32 pointing: persistent TMA-pipelined operator (cache rows must be readable up to the
// next 16-byte boundary past the last sample).
// With ft, also does the template work of ft->mode (projection, or the augmented system).
furax_status launch_fused_tma(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc, float4 *hi,
                              float4 *lo, double *a64, cudaStream_t st, const FusedTpl *ft = nullptr);

}  // namespace fx
