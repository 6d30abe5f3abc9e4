// Symmetric banded Toeplitz product on a tile held in shared memory
// (SymmetricBandToeplitzOperator, direct convolution: Table 2 of the Furax paper):
//   y_t = sum_{k=-(K-1)}^{K-1} c_|k| x_{t+k},  K = 64 (shorter bands are zero-padded).
// Values outside the detector stream are stored as zeros, which gives the finite section.
#pragma once
#include <cstdint>

namespace fx {

constexpr int kHalo = 63;          // K - 1
constexpr int kBand = 2 * kHalo + 1;

// Shared-memory position of tile element u: one pad word every 16 words, so threads that
// each own 16 consecutive outputs (stride 16) hit 32 distinct banks.
__host__ __device__ constexpr int spos(int u) { return u + (u >> 4); }

// y[r] = sum_j taps[|j - 63|] * xs[spos(base + r + j)], j = 0..126, for R consecutive outputs.
// A register window of R inputs slides one element per tap: one shared load per tap per thread.
template <typename T, int R>
__device__ __forceinline__ void band_product(const T *__restrict__ xs, const T *__restrict__ taps, int base, T (&y)[R])
{
    T w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { w[r] = xs[spos(base + r)]; y[r] = T(0); }
#pragma unroll
    for (int j = 0; j < kBand; ++j) {
        const T c = taps[j < kHalo ? kHalo - j : j - kHalo];
#pragma unroll
        for (int r = 0; r < R; ++r) y[r] = fma(c, w[r], y[r]);
        if (j < kBand - 1) {
#pragma unroll
            for (int r = 0; r < R - 1; ++r) w[r] = w[r + 1];
            w[R - 1] = xs[spos(base + R + j)];
        }
    }
}

// The same sum with packed FP32 pairs: output pairs (y_i, y_{i+8}), i < 8, are accumulated with
// fma.rn.f32x2 (each lane one single-rounded FMA, same tap order as band_product, so the results
// are identical) - half the FMA instructions of the scalar form, which leaves issue slots to the
// warps that share the SM. T2 holds the band in tap order as duplicated pairs,
// T2[2j] = T2[2j+1] = c_|j-63| for j < 127 and 0 for j = 127 (16-byte aligned, 256 floats).
constexpr int kBandPad = 128;

__device__ __forceinline__ unsigned long long pack_f32x2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack_f32x2(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ void fma_f32x2(unsigned long long &d, unsigned long long a, unsigned long long b)
{
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// R consecutive outputs per thread (R even): y[r] = sum_j c_|j-63| x[base + r + j] (x in skewed
// slots), accumulated as pairs (y_i, y_{i+R/2}).
// GTAPS: T2 lives in global memory (read through the read-only cache) rather than shared memory.
template <int R, bool GTAPS = false>
__device__ __forceinline__ void band_product_x2(const float *__restrict__ xs, const float *__restrict__ T2, int base,
                                                float (&y)[R])
{
    constexpr int H = R / 2;
    unsigned long long W[H], Y[H];   // W[i] = (x[base+i+j], x[base+i+H+j]) at tap j
#pragma unroll
    for (int i = 0; i < H; ++i) {
        W[i] = pack_f32x2(xs[spos(base + i)], xs[spos(base + i + H)]);
        Y[i] = 0ull;
    }
#pragma unroll
    for (int j2 = 0; j2 < kBandPad; j2 += 2) {
        unsigned long long cpair[2];
        if constexpr (GTAPS) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(T2 + 2 * j2));
            cpair[0] = pack_f32x2(f.x, f.y);
            cpair[1] = pack_f32x2(f.z, f.w);
        } else {
            const ulonglong2 cc = *reinterpret_cast<const ulonglong2 *>(T2 + 2 * j2);
            cpair[0] = cc.x;
            cpair[1] = cc.y;
        }
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int j = j2 + jj;
            if (j < kBand) {
#pragma unroll
                for (int i = 0; i < H; ++i) fma_f32x2(Y[i], W[i], cpair[jj]);
                if (j < kBand - 1) {
                    float lo0, hi0;
                    unpack_f32x2(W[0], lo0, hi0);
                    const unsigned long long wl = pack_f32x2(hi0, xs[spos(base + R + j)]);
#pragma unroll
                    for (int i = 0; i < H - 1; ++i) W[i] = W[i + 1];
                    W[H - 1] = wl;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < H; ++i) unpack_f32x2(Y[i], y[i], y[i + H]);
}

}  // namespace fx
