// Fast pointing expansion for the FP32 cache (PointingOperator, "Map-making classes": the
// pointing is expanded from the quaternions; HEALPix RING pixels, "Landscape types").
//
// GB300 runs FP64 ~70x slower than FP32, and the exact FP64 recipe of pointing_math.cuh costs
// ~150 FP64 operations per sample. Here each sample is computed on the FP32 pipes and the
// exact recipe runs only where the FP32 result could differ from it:
//   * R(q_bore(t)) is formed once per boresight sample in FP64 and stored as double-FP32
//     (hi + lo, 18 floats); the detector axes R(q_det) z^, R(q_det) x^ once per tile.
//     d = R(q_bore) d_det and o = R(q_bore) o_det are then evaluated with exact FP32 products
//     and two-sums, so the FP32 line of sight and orientation are within ~1 ulp of the exact
//     values (R(a (x) b) = R(a) R(b) for unit quaternions).
//   * The RING lookup is done in FP32 (atan2f: at most 3 ulp). Every floor() argument is
//     accepted only if it lies farther from an integer than a bound on its FP32 error
//     (derived below); the zone test, facet edges and the neighbourhood of the poles likewise.
//     An accepted floor equals the floor of the exact value, hence the FP64 recipe's floor.
//   * Samples that fail any test are queued in shared memory and recomputed with the exact
//     FP64 recipe by the whole CTA (dense, no divergence). Non-unit or non-finite quaternions
//     always take the exact path, which gives them pixel -1 where the recipe does.
// Pixels are therefore identical to the FP64 recipe's; weights are FP32 (relative error a few
// 1e-7 away from the poles).
//
// Error budget (u = 2^-24): |d - d_exact|, |o - o_exact| <= 6u per component (rounding of the
// double-FP32 result plus |q|^2 within 4u of 1). phi: <= 8.5u/rho + 24u (atan2f) + 8u (2 pi
// wrap); tt = 2 phi/pi: <= 5.4u/rho + 24.4u. Belt arguments N(1/2 + tt -/+ 3z/4): <= 44 N u;
// cap arguments tp s, (1 - tp) s with s = N sqrt(3 (1-|z|)): <= 51 N u; cap in-ring argument
// tt * ir: <= 47 N u + 5.4u/rho. The margins used are about twice these.
#include "internal.cuh"
#include "pointing_math.cuh"
#include "pointing_fast.cuh"

namespace fx {

// Bore matrices: M_t = R(q_bore(t)) row-major, hi[9] then lo[9]; hi[0] = NaN marks a
// boresight quaternion that must take the exact path (not finite, or |q|^2 not within 4u of 1).
__global__ void bore_matrix_kernel(const double *__restrict__ q_bore, int64_t n, float *__restrict__ m)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const Quat q = load_quat(q_bore, t);
        const double n2 = q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z;
        float *o = m + 18 * t;
        if (!(fabs(n2 - 1.0) <= 4.0 * 5.9604644775390625e-8)) {
            o[0] = __int_as_float(0x7fc00000);
            continue;
        }
        const double xx = q.x * q.x, yy = q.y * q.y, zz = q.z * q.z;
        const double xy = q.x * q.y, xz = q.x * q.z, yz = q.y * q.z;
        const double wx = q.w * q.x, wy = q.w * q.y, wz = q.w * q.z;
        const double r[9] = {1.0 - 2.0 * (yy + zz), 2.0 * (xy - wz), 2.0 * (xz + wy),
                             2.0 * (xy + wz), 1.0 - 2.0 * (xx + zz), 2.0 * (yz - wx),
                             2.0 * (xz - wy), 2.0 * (yz + wx), 1.0 - 2.0 * (xx + yy)};
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float h = (float)r[k];
            o[k] = h;
            o[9 + k] = (float)(r[k] - (double)h);
        }
    }
}

__global__ void __launch_bounds__(256) expand_fast_kernel(const Tile *__restrict__ tiles, const ObsInfo *__restrict__ obs,
                                                          const double *__restrict__ q_bore, const double *__restrict__ q_det,
                                                          const float *__restrict__ bm, const double2 *__restrict__ hwp_cs,
                                                          int32_t *__restrict__ pix_out,
                                                          float *__restrict__ c_out, float *__restrict__ s_out,
                                                          unsigned long long *__restrict__ n_invalid)
{
    __shared__ int qn, sdet_ok;
    __shared__ float sdet[12];   // detector axes: d hi, d lo, o hi, o lo
    __shared__ int32_t queue[TILE];
    const Tile tl = tiles[blockIdx.x];
    const ObsInfo ob = obs[tl.obs];
    const int64_t gdet = ob.det_off + tl.det;
    const Quat qd = load_quat(q_det, gdet);
    // detector axes in double-FP32, formed once per tile (FP64 work: one thread, not every thread)
    if (threadIdx.x == 0) {
        sdet_ok = det_axes_df(qd, sdet);
        qn = 0;
    }
    __syncthreads();
    float dh[3], dl[3], oh[3], ol[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { dh[k] = sdet[k]; dl[k] = sdet[3 + k]; oh[k] = sdet[6 + k]; ol[k] = sdet[9 + k]; }
    const bool det_ok = sdet_ok != 0;
    const int64_t row = ob.tod_off + tl.det * ob.nsamp;
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
        const int64_t t = tl.t0 + k;
        int32_t p = -1;
        float c = 1.f, s = 0.f;
        bool ok = det_ok && certified_sample(bm + 18 * (ob.bore_off + t), dh, dl, oh, ol, (int32_t)ob.nside, p, c, s);
        if (ok && hwp_cs) apply_hwp<float>(c, s, hwp_cs[ob.bore_off + t]);
        if (ok) {
            pix_out[row + t] = p;
            c_out[row + t] = c;
            s_out[row + t] = s;
        } else {
            queue[atomicAdd(&qn, 1)] = k;
        }
    }
    __syncthreads();
    // exact FP64 recipe for the queued samples, densely
    const int nq = qn;
    int bad = 0;
    for (int j = threadIdx.x; j < nq; j += blockDim.x) {
        const int64_t t = tl.t0 + queue[j];
        const SampleF64 r = point_f64(load_quat(q_bore, ob.bore_off + t), qd, ob.nside);
        double c = r.c, s = r.s;
        if (hwp_cs && r.pix >= 0) apply_hwp<double>(c, s, hwp_cs[ob.bore_off + t]);
        pix_out[row + t] = r.pix;
        c_out[row + t] = (float)c;
        s_out[row + t] = (float)s;
        bad += r.pix < 0;
    }
    if (n_invalid) {
        bad = __reduce_add_sync(0xffffffffu, bad);
        if ((threadIdx.x & 31) == 0 && bad) atomicAdd(n_invalid, (unsigned long long)bad);
    }
}

furax_status launch_expand_fast(const furax_pointing *p, unsigned long long *n_invalid, cudaStream_t st)
{
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    furax_status rc;
    if ((rc = ensure_ws(pm, (void **)&pm->ws_bore_m, sizeof(float) * 18 * std::max<int64_t>(1, p->nbore_total))))
        return rc;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p->nbore_total + 255) / 256, 16LL * p->n_sm));
    bore_matrix_kernel<<<g, 256, 0, st>>>(p->q_bore, p->nbore_total, pm->ws_bore_m);
    count_launches(1);
    if ((rc = check_launch("boresight matrices"))) return rc;
    if (p->n_tiles == 0) return FURAX_OK;
    expand_fast_kernel<<<(unsigned)p->n_tiles, 256, 0, st>>>(p->d_tiles, p->d_obs, p->q_bore, p->q_det, pm->ws_bore_m,
                                                             p->has_hwp ? p->d_hwp_cs : nullptr, p->pix, p->c32,
                                                             p->s32, n_invalid);
    count_launches(1);
    return check_launch("fast pointing expansion");
}

}  // namespace fx
