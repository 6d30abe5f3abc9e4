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

// The same sum with the band stored expanded in tap order, T[j] = c_|j-63| for j < 127 and
// T[127] = 0 (16-byte aligned): four coefficients per 16-byte broadcast load instead of one
// shared load per tap.
constexpr int kBandPad = 128;

template <int R>
__device__ __forceinline__ void band_product_x4(const float *__restrict__ xs, const float *__restrict__ T, int base,
                                                float (&y)[R])
{
    float w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { w[r] = xs[spos(base + r)]; y[r] = 0.f; }
#pragma unroll
    for (int j4 = 0; j4 < kBandPad; j4 += 4) {
        const float4 t4 = *reinterpret_cast<const float4 *>(T + j4);
        const float tc[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = j4 + jj;
            if (j < kBand) {
#pragma unroll
                for (int r = 0; r < R; ++r) y[r] = fmaf(tc[jj], w[r], y[r]);
                if (j < kBand - 1) {
#pragma unroll
                    for (int r = 0; r < R - 1; ++r) w[r] = w[r + 1];
                    w[R - 1] = xs[spos(base + R + j)];
                }
            }
        }
    }
}

}  // namespace fx
