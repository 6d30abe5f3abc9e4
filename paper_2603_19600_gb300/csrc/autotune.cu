// Schedule autotuner of the cached FP32 normal operator: times each candidate schedule
// (furax_schedule) on the handle's own pointing, noise and accumulation mode and keeps the fastest.
// The accumulation mode is an input and is never changed: candidates differ only in the order in
// which the operator walks the samples. The paper has no counterpart (its operators are compiled by
// XLA); this picks, per workload, among the tile and sort strategies of fused_tma.cu and
// fused_sorted.cu.
#include <cfloat>

#include "internal.cuh"
#include "atomics.cuh"

namespace fx {

// The built-in search space, with and without the L2 evict-first policy on the pointing stream:
// the time-ordered kernel with 8 or 16 consumer warps, then the pixel-sorted kernel over tile
// length (0 = the largest the stage holds for the tile's rows), detectors per tile and the
// cross-scan grouping tolerance in pixel widths.
static std::vector<furax_schedule> default_space()
{
    std::vector<furax_schedule> v;
    for (int hint : {0, 1}) {
        for (int kc : {8, 16}) v.push_back(furax_schedule{FURAX_SCHED_TIME_ORDERED, 0, 1, 1.0, hint, kc});
        for (int tl : {0, 256, 512})
            for (int rows : {8, 12})
                for (double tol : {1.0, 2.0})
                    v.push_back(furax_schedule{FURAX_SCHED_PIXEL_SORTED, tl, rows, tol, hint, 0});
    }
    return v;
}

// Mean duration of one launch of the fused FP32 operator under the handle's current schedule
// (accumulators cleared before each launch, outside the timed interval).
static furax_status time_operator(furax_pointing *p, const furax_noise *n, int acc, int reps, cudaStream_t st,
                                  double *ms)
{
    const int64_t np = p->npix_total;
    furax_status rc;
    if ((rc = ensure_ws(p, (void **)&p->ws_map32, sizeof(float4) * np))) return rc;
    float4 *hi = nullptr, *lo = nullptr;
    double *a64 = nullptr;
    if (acc == FURAX_ACC_F64) {
        if ((rc = ensure_ws(p, (void **)&p->ws_acc64, sizeof(double) * 3 * np))) return rc;
        a64 = p->ws_acc64;
    } else {
        if ((rc = ensure_ws(p, (void **)&p->ws_acc_hi, sizeof(float4) * kKahanStride * np))) return rc;
        hi = p->ws_acc_hi;
        if (acc == FURAX_ACC_F32_KAHAN) lo = hi + 1;   // interleaved compensated layout
    }
    // the input's values do not change the work: a zero map
    if ((rc = check_cuda(cudaMemsetAsync(p->ws_map32, 0, sizeof(float4) * np, st), "autotune input"))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((rc = check_cuda(cudaEventCreate(&e0), "event")) || (rc = check_cuda(cudaEventCreate(&e1), "event"))) {
        if (e0) cudaEventDestroy(e0);
        return rc;
    }
    double total = 0.0;
    for (int r = -1; r < reps && !rc; ++r) {   // r = -1: warm-up
        if (hi) rc = check_cuda(cudaMemsetAsync(hi, 0, sizeof(float4) * (lo ? kKahanStride : 1) * np, st), "clear");
        if (!rc && a64) rc = check_cuda(cudaMemsetAsync(a64, 0, sizeof(double) * 3 * np, st), "clear");
        if (!rc) rc = check_cuda(cudaEventRecord(e0, st), "event");
        if (!rc) rc = launch_fused_f32(p, n, p->ws_map32, acc, hi, lo, a64, st);
        if (!rc) rc = check_cuda(cudaEventRecord(e1, st), "event");
        if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "event sync");
        float t = 0.f;
        if (!rc) rc = check_cuda(cudaEventElapsedTime(&t, e0, e1), "elapsed");
        if (!rc && r >= 0) total += t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *ms = total / reps;
    return FURAX_OK;
}

}  // namespace fx

using namespace fx;

extern "C" int32_t furax_autotune_space(furax_schedule *out, int32_t cap)
{
    const std::vector<furax_schedule> v = default_space();
    for (int32_t i = 0; out && i < cap && i < (int32_t)v.size(); ++i) out[i] = v[i];
    return (int32_t)v.size();
}

extern "C" furax_status furax_autotune(furax_pointing_t *p, const furax_noise_t *n, int32_t acc,
                                       const furax_schedule *cand, int32_t ncand, int32_t reps, double *ms_out,
                                       int32_t *best_out, void *stream)
{
    if (!p || !n) return set_error(FURAX_EINVAL, "pointing and noise handles are required");
    if (n->ndet_total != p->ndet_total) return set_error(FURAX_EINVAL, "noise and pointing detector counts differ");
    if (p->mode != FURAX_POINTING_CACHE_F32 && p->mode != FURAX_POINTING_CACHE_MIXED)
        return set_error(FURAX_EINVAL, "the autotuner schedules the cached FP32 operator (FP32 or mixed cache)");
    if (acc != FURAX_ACC_F64 && acc != FURAX_ACC_F32 && acc != FURAX_ACC_F32_KAHAN)
        return set_error(FURAX_EINVAL, "unknown accumulation %d", acc);
    if (!cand || ncand < 1 || reps < 1 || !ms_out || !best_out)
        return set_error(FURAX_EINVAL, "candidates (ncand >= 1), reps >= 1, ms_out and best_out are required");
    if (p->n_tiles == 0) return set_error(FURAX_EINVAL, "the pointing has no samples");
    if (long_band(n)) return set_error(FURAX_EINVAL, "bands longer than %d taps do not use the fused operator", MAXTAPS);
    cudaStream_t st = (cudaStream_t)stream;
    const furax_schedule before = p->sched;
    int32_t best = -1;
    double best_ms = DBL_MAX;
    for (int32_t k = 0; k < ncand; ++k) {
        ms_out[k] = -1.0;   // a candidate the handle rejects (e.g. its fields) stays at -1
        if (set_schedule(p, cand[k], st) != FURAX_OK) continue;
        double ms = 0.0;
        furax_status rc = time_operator(p, n, acc, reps, st, &ms);
        if (rc) {   // a device or allocation error ends the search with the handle's previous schedule
            set_schedule(p, before, st);
            return rc;
        }
        ms_out[k] = ms;
        if (ms < best_ms) { best_ms = ms; best = k; }
    }
    if (best < 0) {
        set_schedule(p, before, st);
        return set_error(FURAX_EINVAL, "no candidate schedule is valid for this handle");
    }
    *best_out = best;
    return set_schedule(p, cand[best], st);
}
