// C-ABI entry points of libfurax: argument checks, handle lifetime, dispatch to the kernels.
#include <cstdarg>
#include <cmath>
#include <mutex>
#include <atomic>
#include <unordered_map>
#include <unordered_set>

#include "internal.cuh"

namespace fx {

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

furax_status set_error(furax_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

furax_status check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return FURAX_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(FURAX_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(FURAX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

furax_status check_launch(const char *what) { return check_cuda(cudaGetLastError(), what); }

furax_status AllReduce::operator()(void *buf, int64_t n, int32_t dtype, cudaStream_t st) const
{
    if (!fn || n <= 0) return FURAX_OK;
    furax_status rc = check_launch("before the sharding sum");
    if (rc) return rc;
    rc = fn(buf, n, dtype, (void *)st, user);
    if (rc) return set_error(rc < 0 ? rc : FURAX_EINVAL, "the sharding sum (allreduce) returned %d", rc);
    return FURAX_OK;
}

void count_launches(int64_t n) { g_launches += n; }

furax_status allow_smem(const void *kern, size_t bytes)
{
    static std::mutex mu;
    static std::unordered_set<const void *> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(kern)) return FURAX_OK;
    furax_status rc = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
                                 "shared-memory limit");
    if (!rc) done.insert(kern);
    return rc;
}

furax_status ensure_ws(furax_pointing *p, void **ptr, size_t bytes)
{
    if (*ptr) return FURAX_OK;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return set_error(FURAX_ENOMEM, "workspace allocation of %zu bytes failed", bytes);
    }
    return FURAX_OK;
}

void destroy_cg_ws(furax_pointing *p);

// ---- kernel timing
static std::atomic<bool> g_prof_on{false};
static std::mutex g_prof_mu;
static double g_prof_ms[3] = {0.0, 0.0, 0.0};
static int64_t g_prof_cnt[3] = {0, 0, 0};
struct PendingPair { int kind; cudaEvent_t a, b; };
static std::vector<PendingPair> g_pending;
static std::vector<cudaEvent_t> g_pool;

bool prof_on() { return g_prof_on.load(); }

void prof_pair(cudaEvent_t *a, cudaEvent_t *b)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (cudaEvent_t *e : {a, b}) {
        if (!g_pool.empty()) { *e = g_pool.back(); g_pool.pop_back(); }
        else if (cudaEventCreate(e) != cudaSuccess) { cudaGetLastError(); *e = nullptr; }
    }
}

void prof_push(int kind, cudaEvent_t a, cudaEvent_t b)
{
    if (!a || !b) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending.push_back({kind, a, b});
}

void prof_add(int kind, double ms)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_ms[kind] += ms;
    g_prof_cnt[kind] += 1;
}

void prof_flush()
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const PendingPair &pp : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(pp.b) == cudaSuccess && cudaEventElapsedTime(&ms, pp.a, pp.b) == cudaSuccess) {
            g_prof_ms[pp.kind] += ms;
            g_prof_cnt[pp.kind] += 1;
        } else {
            cudaGetLastError();
        }
        g_pool.push_back(pp.a);
        g_pool.push_back(pp.b);
    }
    g_pending.clear();
}

}  // namespace fx

using namespace fx;

namespace fx {
// Observations sharing a map_id share one map (and its pixel tiles): they carry the offset and
// pixel-tile range of the map, whose tiles name the first of them. The PCG's per-observation
// scalars are then the per-map scalars, computed identically for each observation of the map.
void build_layout(const furax_obs_desc *desc, Layout &L)
{
    int64_t det = 0, bore = 0, tod = 0, map = 0, ptile = 0;
    std::unordered_map<int32_t, int> first_of;   // map_id -> first observation with it
    for (int i = 0; i < desc->n_obs; ++i) {
        ObsInfo o{};
        o.nsamp = desc->nsamp[i];
        o.ndet = desc->ndet[i];
        o.nside = desc->nside[i];
        o.npix = 12LL * o.nside * o.nside;
        o.det_off = det; o.bore_off = bore; o.tod_off = tod;
        int owner = i;
        if (desc->map_id) owner = first_of.emplace(desc->map_id[i], i).first->second;
        if (owner != i) {
            o.map_off = L.obs[owner].map_off;
            o.ptile0 = L.obs[owner].ptile0;
            o.nptile = L.obs[owner].nptile;
        } else {
            o.map_off = map;
            o.ptile0 = ptile;
            o.nptile = (int32_t)((o.npix + PTILE - 1) / PTILE);
            for (int64_t k = 0; k < o.nptile; ++k) {
                PTile t;
                t.p0 = map + k * PTILE;
                t.obs = i;
                t.len = (int32_t)std::min<int64_t>(PTILE, o.npix - k * PTILE);
                L.ptiles.push_back(t);
            }
            map += o.npix;
            ptile += o.nptile;
        }
        // Time-major order: the CTAs resident at any moment process every detector over the
        // same stretch of time, i.e. one compact swath of sky, so the map gathers and the
        // per-pixel reductions stay in L2 instead of spanning the whole map.
        for (int64_t t0 = 0; t0 < o.nsamp; t0 += TILE)
            for (int32_t j = 0; j < o.ndet; ++j) {
                Tile t;
                t.t0 = t0; t.obs = i; t.det = j;
                t.len = (int32_t)std::min<int64_t>(TILE, o.nsamp - t0);
                t.pad = 0;
                L.tiles.push_back(t);
            }
        det += o.ndet; bore += o.nsamp; tod += o.ndet * o.nsamp;
        L.max_ndet = std::max(L.max_ndet, o.ndet);
        L.obs.push_back(o);
    }
    L.ndet = det; L.nbore = bore; L.nsamp = tod; L.npix = map;
}
}  // namespace fx

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
static bool valid_dtype(int32_t t) { return t == FURAX_F32 || t == FURAX_F64; }
static bool valid_acc(int32_t a) { return a == FURAX_ACC_F64 || a == FURAX_ACC_F32 || a == FURAX_ACC_F32_KAHAN; }

#define REQUIRE(cond, ...) \
    do { if (!(cond)) return set_error(FURAX_EINVAL, __VA_ARGS__); } while (0)

extern "C" {

const char *furax_last_error(void) { return g_err.c_str(); }
int64_t furax_launch_count(void) { return g_launches.load(); }
const char *furax_version(void) { return "furax-gb300 0.1 (sm_103a)"; }

void furax_profile_enable(int32_t on) { g_prof_on = on != 0; }

furax_status furax_profile_read(int32_t kernel, double *total_ms, int64_t *count)
{
    REQUIRE(kernel >= 0 && kernel <= 2, "kernel must be 0 (FP32 fused), 1 (FP64 fused) or 2 (double-FP32 fused)");
    prof_flush();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (total_ms) *total_ms = g_prof_ms[kernel];
    if (count) *count = g_prof_cnt[kernel];
    return FURAX_OK;
}

void furax_profile_reset(void)
{
    prof_flush();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_ms[0] = g_prof_ms[1] = g_prof_ms[2] = 0.0;
    g_prof_cnt[0] = g_prof_cnt[1] = g_prof_cnt[2] = 0;
}

furax_status furax_device_status(furax_pointing_t *p, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    furax_status rc = check_cuda(cudaMemcpyAsync(&h, p->d_err, sizeof h, cudaMemcpyDeviceToHost, st), "read status");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "status sync");
    if (rc) return rc;
    if (h) {
        cudaMemsetAsync(p->d_err, 0, sizeof(unsigned), st);
        cudaStreamSynchronize(st);
        return set_error(FURAX_ETIMEOUT, "a bounded device-side wait gave up (error word %u)", h);
    }
    return FURAX_OK;
}

furax_status furax_set_wait_budget(furax_pointing_t *p, int64_t cycles, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(cycles >= 0, "the wait budget must be >= 0 cycles (0 selects the default)");
    cudaStream_t st = (cudaStream_t)stream;
    // a kernel reads the budget at its start: the write is ordered on the stream like a launch
    furax_status rc = check_cuda(cudaMemcpyAsync(p->d_err + 2, &cycles, sizeof cycles, cudaMemcpyHostToDevice, st),
                                 "set wait budget");
    return rc ? rc : check_cuda(cudaStreamSynchronize(st), "wait budget sync");
}

furax_status furax_debug_hold_loader(furax_pointing_t *p, int32_t hold, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned h = hold ? 1u : 0u;
    furax_status rc = check_cuda(cudaMemcpyAsync(p->d_err + 1, &h, sizeof h, cudaMemcpyHostToDevice, st), "hold loader");
    return rc ? rc : check_cuda(cudaStreamSynchronize(st), "hold loader sync");
}

furax_status furax_pointing_cache(const furax_pointing_t *p, int32_t *pix, float *c, float *s, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(pix && c && s, "pix, c and s must be device pointers");
    REQUIRE(p->mode == FURAX_POINTING_CACHE_F32 || p->mode == FURAX_POINTING_CACHE_MIXED,
            "only the FP32 and mixed caches hold FP32 weights");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)p->nsamp_total;
    furax_status rc = check_cuda(cudaMemcpyAsync(pix, p->pix, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st), "copy");
    if (!rc) rc = check_cuda(cudaMemcpyAsync(c, p->c32, sizeof(float) * n, cudaMemcpyDeviceToDevice, st), "copy");
    if (!rc) rc = check_cuda(cudaMemcpyAsync(s, p->s32, sizeof(float) * n, cudaMemcpyDeviceToDevice, st), "copy");
    return rc;
}

furax_status furax_pointing_refresh(furax_pointing_t *p, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->mode == FURAX_POINTING_ON_THE_FLY) return FURAX_OK;
    const bool had = p->has_psi;
    p->has_psi = false;
    furax_status rc;
    if (p->mode == FURAX_POINTING_CACHE_F32) rc = launch_expand_fast(p, nullptr, st);
    else if (p->mode == FURAX_POINTING_CACHE_MIXED)
        rc = launch_expand(p, p->pix, p->c32, p->s32, nullptr, nullptr, nullptr, st, false, p->c32lo, p->s32lo);
    else rc = launch_expand(p, p->pix, nullptr, nullptr, p->c64, p->s64, nullptr, st, false);
    p->has_psi = had;
    if (!rc) rc = sort_sorted_tiles(p, st);   // the pixel-sorted tiles follow the new cache
    return rc;
}

furax_status furax_pointing_set_schedule(furax_pointing_t *p, const furax_schedule *s, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(s, "schedule is NULL");
    return set_schedule(p, *s, (cudaStream_t)stream);
}

furax_status furax_pointing_get_schedule(const furax_pointing_t *p, furax_schedule *s)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(s, "schedule is NULL");
    *s = p->sched;
    return FURAX_OK;
}

static void pointing_free(furax_pointing *p)
{
    if (!p) return;
    destroy_cg_ws(p);
    free_sorted(p);
    cudaFree(p->d_obs); cudaFree(p->d_tiles); cudaFree(p->d_ptiles); cudaFree(p->d_psi_cs); cudaFree(p->d_hwp_cs);
    cudaFree(p->pix); cudaFree(p->c32); cudaFree(p->s32); cudaFree(p->c64); cudaFree(p->s64);
    cudaFree(p->c32lo); cudaFree(p->s32lo); cudaFree(p->ws_bore_m);
    cudaFree(p->ws_map32); cudaFree(p->ws_acc_hi); cudaFree(p->ws_acc64); cudaFree(p->ws_df_lo); cudaFree(p->ws_x64);
    cudaFree(p->ws_x2);
    cudaFree(p->ws_tod); cudaFree(p->ws_tod2); cudaFree(p->ws_hits); cudaFree(p->d_err);
    delete p;
}

static furax_status check_desc(const furax_obs_desc *d)
{
    REQUIRE(d, "desc is NULL");
    REQUIRE(d->n_obs >= 1, "n_obs must be >= 1 (got %d)", d->n_obs);
    REQUIRE(d->ndet && d->nsamp && d->nside, "ndet, nsamp and nside must be host arrays");
    for (int i = 0; i < d->n_obs; ++i) {
        REQUIRE(d->ndet[i] >= 1, "ndet[%d] = %d must be >= 1", i, d->ndet[i]);
        REQUIRE(d->nsamp[i] >= 1, "nsamp[%d] = %lld must be >= 1", i, (long long)d->nsamp[i]);
        REQUIRE(d->nside[i] >= 1 && d->nside[i] <= 8192, "nside[%d] = %d must be in [1, 8192]", i, d->nside[i]);
    }
    if (d->map_id) {
        std::unordered_map<int32_t, int> first_of;
        for (int i = 0; i < d->n_obs; ++i) {
            const int j = first_of.emplace(d->map_id[i], i).first->second;
            REQUIRE(d->nside[j] == d->nside[i], "observations %d and %d share map %d but have nside %d and %d", j, i,
                    d->map_id[i], d->nside[j], d->nside[i]);
        }
    }
    return FURAX_OK;
}

furax_status furax_pointing_create(const furax_obs_desc *desc, int32_t mode, void *stream, furax_pointing_t **out)
{
    REQUIRE(out, "out is NULL");
    *out = nullptr;
    furax_status rc = check_desc(desc);
    if (rc) return rc;
    REQUIRE(mode == FURAX_POINTING_ON_THE_FLY || mode == FURAX_POINTING_CACHE_F32 || mode == FURAX_POINTING_CACHE_F64 ||
                mode == FURAX_POINTING_CACHE_MIXED,
            "unknown pointing mode %d", mode);
    REQUIRE(desc->q_bore && desc->q_det, "q_bore and q_det must be device pointers");
    REQUIRE(aligned16(desc->q_bore) && aligned16(desc->q_det), "quaternion arrays must be 16-byte aligned");
    REQUIRE(is_device_ptr(desc->q_bore) && is_device_ptr(desc->q_det), "quaternion arrays must be device memory");
    if ((rc = prepare_kernels())) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    furax_pointing *p = new furax_pointing();
    p->mode = mode;
    {
        int dev = 0, sms = 1;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            p->n_sm = std::max(1, sms);
        cudaGetLastError();
    }
    p->n_obs = desc->n_obs;
    p->q_bore = desc->q_bore;
    p->q_det = desc->q_det;
    Layout L;
    build_layout(desc, L);
    if (desc->hwp_angle)
        for (auto &o : L.obs) o.hwp = 1;
    p->obs = L.obs; p->tiles = L.tiles; p->ptiles = L.ptiles;
    p->ndet_total = L.ndet; p->nbore_total = L.nbore; p->nsamp_total = L.nsamp; p->npix_total = L.npix;
    p->max_ndet = L.max_ndet;
    const int64_t det = L.ndet, tod = L.nsamp;
    p->n_tiles = (int64_t)p->tiles.size();
    p->n_ptiles = (int64_t)p->ptiles.size();
    if (p->n_tiles >= (1LL << 31) || p->n_ptiles >= (1LL << 31)) {
        pointing_free(p);
        return set_error(FURAX_EINVAL, "problem too large for one launch grid");
    }
    auto up = [&](void **dst, const void *src, size_t bytes) -> furax_status {
        furax_status r = ensure_ws(p, dst, bytes);
        if (r) return r;
        return check_cuda(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st), "upload");
    };
    if ((rc = up((void **)&p->d_obs, p->obs.data(), sizeof(ObsInfo) * p->obs.size())) ||
        (rc = up((void **)&p->d_tiles, p->tiles.data(), sizeof(Tile) * p->tiles.size())) ||
        (rc = up((void **)&p->d_ptiles, p->ptiles.data(), sizeof(PTile) * p->ptiles.size())) ||
        (rc = ensure_ws(p, (void **)&p->d_psi_cs, sizeof(double2) * det)) ||
        (rc = ensure_ws(p, (void **)&p->d_err, sizeof(unsigned) * kCtlWords)) ||
        (rc = check_cuda(cudaMemsetAsync(p->d_err, 0, sizeof(unsigned) * kCtlWords, st), "memset"))) {
        pointing_free(p);
        return rc;
    }
    if (desc->hwp_angle) {   // before the offsets: they pass through the plate
        if (!is_device_ptr(desc->hwp_angle)) {
            pointing_free(p);
            return set_error(FURAX_EINVAL, "hwp_angle must be device memory");
        }
        if ((rc = launch_set_hwp(p, desc->hwp_angle, st))) { pointing_free(p); return rc; }
    }
    if (desc->psi_offset) {
        REQUIRE(is_device_ptr(desc->psi_offset), "psi_offset must be device memory");
        if ((rc = launch_set_psi(p, desc->psi_offset, st))) { pointing_free(p); return rc; }
    }
    unsigned long long *d_bad = nullptr;
    if ((rc = ensure_ws(p, (void **)&d_bad, sizeof(unsigned long long))) ||
        (rc = check_cuda(cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st), "memset"))) {
        pointing_free(p);
        return rc;
    }
    // Expansion: caches pixel + weights, or (on the fly) only validates the quaternions.
    int32_t *pix = nullptr;
    if (mode == FURAX_POINTING_CACHE_F32 || mode == FURAX_POINTING_CACHE_MIXED) {
        const bool mixed = mode == FURAX_POINTING_CACHE_MIXED;
        // padded to a 16-byte multiple: the operator bulk-copies rows on 16-byte boundaries
        const int64_t tod4 = (tod + 3) & ~int64_t(3);
        if ((rc = ensure_ws(p, (void **)&p->pix, sizeof(int32_t) * tod4)) ||
            (rc = ensure_ws(p, (void **)&p->c32, sizeof(float) * tod4)) ||
            (rc = ensure_ws(p, (void **)&p->s32, sizeof(float) * tod4)) ||
            (mixed && (rc = ensure_ws(p, (void **)&p->c32lo, sizeof(float) * tod))) ||
            (mixed && (rc = ensure_ws(p, (void **)&p->s32lo, sizeof(float) * tod)))) {
            cudaFree(d_bad); pointing_free(p); return rc;
        }
        pix = p->pix;
        // weights are cached without the offsets; kernels rotate them per detector
        const bool had = p->has_psi; p->has_psi = false;
        if (mixed) rc = launch_expand(p, p->pix, p->c32, p->s32, nullptr, nullptr, d_bad, st, false, p->c32lo, p->s32lo);
        else rc = launch_expand_fast(p, d_bad, st);
        p->has_psi = had;
    } else if (mode == FURAX_POINTING_CACHE_F64) {
        if ((rc = ensure_ws(p, (void **)&p->pix, sizeof(int32_t) * tod)) ||
            (rc = ensure_ws(p, (void **)&p->c64, sizeof(double) * tod)) ||
            (rc = ensure_ws(p, (void **)&p->s64, sizeof(double) * tod))) {
            cudaFree(d_bad); pointing_free(p); return rc;
        }
        pix = p->pix;
        const bool had = p->has_psi; p->has_psi = false;
        rc = launch_expand(p, p->pix, nullptr, nullptr, p->c64, p->s64, d_bad, st, false);
        p->has_psi = had;
    } else {
        // validation pass into a temporary pixel buffer
        int32_t *tmp = nullptr;
        if ((rc = ensure_ws(p, (void **)&tmp, sizeof(int32_t) * tod))) { cudaFree(d_bad); pointing_free(p); return rc; }
        const bool had = p->has_psi; p->has_psi = false;
        rc = launch_expand(p, tmp, nullptr, nullptr, nullptr, nullptr, d_bad, st, false);
        p->has_psi = had;
        if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "pointing validation");
        cudaFree(tmp);
    }
    (void)pix;
    unsigned long long bad = 0;
    if (!rc) rc = check_cuda(cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, st), "read count");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st), "pointing create");
    cudaFree(d_bad);
    if (rc) { pointing_free(p); return rc; }
    p->n_invalid = (int64_t)bad;
    *out = p;
    return FURAX_OK;
}

furax_status furax_pointing_destroy(furax_pointing_t *p)
{
    if (!p) return FURAX_OK;
    cudaDeviceSynchronize();
    pointing_free(p);
    return check_launch("pointing destroy");
}

furax_status furax_pointing_info(const furax_pointing_t *p, int64_t *nsamp_total, int64_t *npix_total,
                                 int64_t *ndet_total, int64_t *n_invalid)
{
    REQUIRE(p, "pointing handle is NULL");
    if (nsamp_total) *nsamp_total = p->nsamp_total;
    if (npix_total) *npix_total = p->npix_total;
    if (ndet_total) *ndet_total = p->ndet_total;
    if (n_invalid) *n_invalid = p->n_invalid;
    return FURAX_OK;
}

furax_status furax_pointing_set_psi_offset(furax_pointing_t *p, const double *psi_offset, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(!psi_offset || is_device_ptr(psi_offset), "psi_offset must be device memory");
    return launch_set_psi(p, psi_offset, (cudaStream_t)stream);
}

furax_status furax_pointing_expand(const furax_pointing_t *p, int32_t *pix, void *c, void *s, int32_t w_t, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(pix && c && s, "pix, c and s must be device pointers");
    REQUIRE(valid_dtype(w_t), "unknown weight dtype %d", w_t);
    cudaStream_t st = (cudaStream_t)stream;
    if (w_t == FURAX_F64) return launch_expand(p, pix, nullptr, nullptr, (double *)c, (double *)s, nullptr, st, true);
    return launch_expand(p, pix, (float *)c, (float *)s, nullptr, nullptr, nullptr, st, true);
}

furax_status furax_pointing_apply(const furax_pointing_t *p, const void *map, int32_t map_t, void *tod, int32_t tod_t,
                                  void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(map && tod, "map and tod must be device pointers");
    REQUIRE(valid_dtype(map_t) && valid_dtype(tod_t), "unknown dtype");
    return launch_P(p, map, map_t, tod, tod_t, (cudaStream_t)stream);
}

furax_status furax_pointing_transpose(const furax_pointing_t *p, const void *tod, int32_t tod_t, void *map, int32_t map_t,
                                      int32_t acc, int32_t *hits, int32_t accumulate, void *stream)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(map && tod, "map and tod must be device pointers");
    REQUIRE(valid_dtype(map_t) && valid_dtype(tod_t), "unknown dtype");
    REQUIRE(valid_acc(acc), "unknown accumulation mode %d", acc);
    return launch_PT(p, tod, tod_t, map, map_t, acc, hits, accumulate ? 1 : 0, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------- noise
__global__ void noise_prep_kernel(int kind, const double *__restrict__ in, int64_t n, int ntaps, double *__restrict__ p64,
                                  float *__restrict__ p32, double *__restrict__ diag, int64_t ndet)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (kind == FURAX_NOISE_WHITE) {
        if (i < ndet) {
            const double w = 1.0 / in[i];
            p64[i] = w; p32[i] = (float)w; diag[i] = w;
        }
    } else {
        if (i < n) { p64[i] = in[i]; p32[i] = (float)in[i]; }
        if (i < ndet) diag[i] = in[i * ntaps];
    }
}

// Band in tap order as duplicated pairs for the pixel-sorted operator: out[d][2j] = out[d][2j+1] =
// c_|j-63| (zero past the band and for j = 127).
__global__ void band_pairs_kernel(const float *__restrict__ p32, int32_t ntaps, int64_t ndet, float *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ndet * kBandPairs) return;
    const int64_t d = i / kBandPairs;
    const int j = (int)(i % kBandPairs);
    const int k = j < 63 ? 63 - j : j - 63;
    const float c = (j < 127 && k < ntaps) ? p32[d * ntaps + k] : 0.f;
    out[2 * i] = c;
    out[2 * i + 1] = c;
}

furax_status furax_noise_create(int32_t kind, const double *params, int32_t ntaps, const furax_obs_desc *desc,
                                void *stream, furax_noise_t **out)
{
    REQUIRE(out, "out is NULL");
    *out = nullptr;
    furax_status rc = check_desc(desc);
    if (rc) return rc;
    REQUIRE(kind == FURAX_NOISE_WHITE || kind == FURAX_NOISE_BANDED, "unknown noise kind %d", kind);
    REQUIRE(params && is_device_ptr(params), "params must be device memory");
    if (kind == FURAX_NOISE_BANDED)
        REQUIRE(ntaps >= 1 && ntaps <= kLongTaps, "ntaps = %d must be in [1, %d]", ntaps, kLongTaps);
    else
        ntaps = 1;
    Layout L;
    build_layout(desc, L);
    const int64_t ndet = L.ndet;
    furax_noise *n = new furax_noise();
    n->kind = kind;
    n->ntaps = ntaps;
    n->ndet_total = ndet;
    n->nsamp_total = L.nsamp;
    n->n_tiles = (int64_t)L.tiles.size();
    if (cudaMalloc((void **)&n->d_obs, sizeof(ObsInfo) * L.obs.size()) != cudaSuccess ||
        cudaMalloc((void **)&n->d_tiles, sizeof(Tile) * std::max<size_t>(1, L.tiles.size())) != cudaSuccess ||
        cudaMemcpyAsync(n->d_obs, L.obs.data(), sizeof(ObsInfo) * L.obs.size(), cudaMemcpyHostToDevice,
                        (cudaStream_t)stream) != cudaSuccess ||
        cudaMemcpyAsync(n->d_tiles, L.tiles.data(), sizeof(Tile) * L.tiles.size(), cudaMemcpyHostToDevice,
                        (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(n->d_obs); cudaFree(n->d_tiles);
        delete n;
        return set_error(FURAX_ENOMEM, "noise layout allocation failed");
    }
    const int64_t cnt = kind == FURAX_NOISE_WHITE ? ndet : ndet * ntaps;
    if (cudaMalloc((void **)&n->p64, sizeof(double) * cnt) != cudaSuccess ||
        cudaMalloc((void **)&n->p32, sizeof(float) * cnt) != cudaSuccess ||
        cudaMalloc((void **)&n->diag, sizeof(double) * ndet) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(n->p64); cudaFree(n->p32); cudaFree(n->diag); cudaFree(n->d_obs); cudaFree(n->d_tiles);
        delete n;
        return set_error(FURAX_ENOMEM, "noise allocation failed");
    }
    const int64_t m = std::max(cnt, ndet);
    noise_prep_kernel<<<(unsigned)((m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(kind, params, cnt, ntaps, n->p64,
                                                                                    n->p32, n->diag, ndet);
    count_launches(1);
    if (!(rc = check_launch("noise create")) && long_band(n)) rc = prepare_noise_fft(n, L.obs, (cudaStream_t)stream);
    if (!rc && kind == FURAX_NOISE_BANDED && !long_band(n)) {
        if (cudaMalloc((void **)&n->band2, sizeof(float) * kBandPairs * 2 * (size_t)ndet) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(FURAX_ENOMEM, "noise band table allocation failed");
        } else {
            const int64_t nb = ndet * kBandPairs;
            band_pairs_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n->p32, ntaps, ndet,
                                                                                              n->band2);
            count_launches(1);
            rc = check_launch("noise band table");
        }
    }
    if (rc) {
        furax_noise_destroy(n);
        return rc;
    }
    *out = n;
    return FURAX_OK;
}

furax_status furax_noise_destroy(furax_noise_t *n)
{
    if (!n) return FURAX_OK;
    cudaDeviceSynchronize();
    cudaFree(n->p64); cudaFree(n->p32); cudaFree(n->diag); cudaFree(n->d_obs); cudaFree(n->d_tiles); cudaFree(n->band2);
    cudaFree(n->fft_items); cudaFree(n->tw64); cudaFree(n->tw32); cudaFree(n->spec64); cudaFree(n->spec32);
    cudaFree(n->gf_y); cudaFree(n->gf_r); cudaFree(n->gf_p); cudaFree(n->gf_q); cudaFree(n->gf_x32); cudaFree(n->gf_n32);
    cudaFree(n->gf_sc);
    delete n;
    return check_launch("noise destroy");
}

static furax_status check_pair(const furax_pointing_t *p, const furax_noise_t *n)
{
    REQUIRE(p, "pointing handle is NULL");
    REQUIRE(n, "noise handle is NULL");
    REQUIRE(n->ndet_total == p->ndet_total, "noise has %lld detectors, pointing %lld", (long long)n->ndet_total,
            (long long)p->ndet_total);
    return FURAX_OK;
}

furax_status furax_noise_inv_apply(const furax_noise_t *n, const void *in, void *out, int32_t dtype, void *stream)
{
    REQUIRE(n, "noise handle is NULL");
    REQUIRE(in && out, "in and out must be device pointers");
    REQUIRE(in != out, "in and out must not alias");
    REQUIRE(valid_dtype(dtype), "unknown dtype %d", dtype);
    return launch_ninv(n, in, out, dtype, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------- operators
furax_status furax_blockdiag_precond(const furax_pointing_t *p, const furax_noise_t *n, double rcond_min,
                                     double *blocks_inv, uint8_t *valid, int32_t *hits, double *rcond, void *stream)
{
    furax_status rc = check_pair(p, n);
    if (rc) return rc;
    REQUIRE(blocks_inv && valid, "blocks_inv and valid must be device pointers");
    REQUIRE(rcond_min >= 0.0 && rcond_min <= 1.0, "rcond_min must be in [0, 1]");
    return launch_bj(p, n, rcond_min, blocks_inv, valid, hits, rcond, (cudaStream_t)stream);
}

furax_status furax_ptnp_apply(const furax_pointing_t *p, const furax_noise_t *n, const double *x, double *out,
                              const uint8_t *valid, int32_t precision, int32_t acc, void *stream)
{
    furax_status rc = check_pair(p, n);
    if (rc) return rc;
    REQUIRE(x && out, "x and out must be device pointers");
    REQUIRE(x != out, "x and out must not alias");
    REQUIRE(valid_dtype(precision) || precision == FURAX_PREC_F32X2, "unknown precision %d", precision);
    REQUIRE(valid_acc(acc), "unknown accumulation mode %d", acc);
    return ptnp_apply(p, n, x, out, valid, precision, acc, (cudaStream_t)stream);
}

furax_status furax_rhs(const furax_pointing_t *p, const furax_noise_t *n, const void *d, int32_t d_t,
                       const uint8_t *valid, double *b, void *stream)
{
    furax_status rc = check_pair(p, n);
    if (rc) return rc;
    REQUIRE(d && b, "d and b must be device pointers");
    REQUIRE(valid_dtype(d_t), "unknown dtype %d", d_t);
    furax_pointing *pm = const_cast<furax_pointing *>(p);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_ws(pm, (void **)&pm->ws_acc64, sizeof(double) * 3 * p->npix_total))) return rc;
    if ((rc = check_cuda(cudaMemsetAsync(pm->ws_acc64, 0, sizeof(double) * 3 * p->npix_total, st), "memset"))) return rc;
    const bool prof = prof_on();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) { prof_pair(&e0, &e1); if (e0) cudaEventRecord(e0, st); }
    // FP64-accurate on FP32 pipes (double-FP32 band product); FP64 arithmetic would be ~5x slower here.
    // A band longer than the fused kernels hold: overlap-save N^-1 in FP64 with the TOD in HBM.
    if (long_band(n)) {
        if ((rc = tod_ws(p)) || (rc = launch_rhs_chain(p, n, d, d_t, pm->ws_acc64, st))) return rc;
    } else if ((rc = launch_fused_df(p, n, nullptr, d, d_t, pm->ws_acc64, st))) {
        return rc;
    }
    if (prof) { if (e1) cudaEventRecord(e1, st); prof_push(2, e0, e1); }
    return launch_finalize_acc(p, FURAX_ACC_F64, nullptr, nullptr, pm->ws_acc64, valid, b, st);
}

void furax_cg_default_opts(furax_cg_opts *o)
{
    if (!o) return;
    o->maxiter = 50;
    o->tol = 1e-8;
    o->precision = FURAX_F64;
    o->acc = FURAX_ACC_F32;
    o->inner_tol = 1e-5;
    o->max_outer = 8;
    o->use_graph = 1;
    o->check_every = 10;
    o->rcond_min = 1e-3;
    o->binned_only = 0;
    o->true_residual = 1;
    o->d_ready = nullptr;
    o->allreduce = nullptr;
    o->allreduce_user = nullptr;
}

furax_status furax_mapmaker_cg(const furax_pointing_t *p, const furax_noise_t *n, const void *d, int32_t d_t, double *x,
                               uint8_t *valid, const furax_cg_opts *o, furax_cg_result *res, void *stream)
{
    furax_status rc = check_pair(p, n);
    if (rc) return rc;
    REQUIRE(d && x, "d and x must be device pointers");
    REQUIRE(o && res, "opts and result must be host pointers");
    REQUIRE(valid_dtype(d_t), "unknown dtype %d", d_t);
    REQUIRE(o->maxiter >= 0 && o->maxiter <= 1000000, "maxiter out of range");
    REQUIRE(o->tol >= 0.0, "tol must be >= 0");
    REQUIRE(valid_dtype(o->precision), "unknown precision %d", o->precision);
    REQUIRE(valid_acc(o->acc), "unknown accumulation mode %d", o->acc);
    REQUIRE(o->precision == FURAX_F64 || (o->inner_tol >= 0.0 && o->inner_tol < 1.0 && o->max_outer >= 1),
            "mixed precision needs 0 <= inner_tol < 1 and max_outer >= 1");
    REQUIRE(o->check_every >= 1, "check_every must be >= 1");
    REQUIRE(!res->hist || res->hist_len >= 0, "hist_len must be >= 0");
    return mapmaker_cg(p, n, d, d_t, x, valid, o, res, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------- gap filling
furax_status furax_gapfill(const furax_noise_t *cov, const void *d, const uint8_t *valid, const void *n_real,
                           void *out, int32_t dtype, int32_t maxiter, double tol, int32_t precision, int32_t *iters_out,
                           void *stream)
{
    REQUIRE(cov, "covariance handle is NULL");
    REQUIRE(cov->kind == FURAX_NOISE_BANDED, "the covariance must be a banded noise handle");
    REQUIRE(d && valid && n_real && out, "d, valid, n_real and out must be device pointers");
    REQUIRE(valid_dtype(dtype), "unknown dtype %d", dtype);
    REQUIRE(maxiter >= 0 && maxiter <= 1000000, "maxiter out of range");
    REQUIRE(tol >= 0.0, "tol must be >= 0");
    REQUIRE(valid_dtype(precision) || precision == FURAX_PREC_F32X2, "unknown precision %d", precision);
    return gapfill(cov, d, valid, n_real, out, dtype, maxiter, tol, precision, iters_out, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------- templates
furax_status furax_templates_create(const furax_pointing_t *p, const furax_noise_t *n, int32_t order, void *stream,
                                    furax_templates_t **out)
{
    REQUIRE(out, "out must be a host pointer");
    *out = nullptr;
    furax_status rc = check_pair(p, n);
    if (rc) return rc;
    REQUIRE(n->nsamp_total == p->nsamp_total, "noise streams hold %lld samples, pointing %lld",
            (long long)n->nsamp_total, (long long)p->nsamp_total);
    REQUIRE(order >= 0 && order <= 3, "template order %d outside [0, 3]", order);
    return templates_create(p, n, order, (cudaStream_t)stream, out);
}

furax_status furax_templates_destroy(furax_templates_t *t)
{
    templates_destroy(t);
    return FURAX_OK;
}

furax_status furax_templates_gram(const furax_templates_t *t, double *gram, void *stream)
{
    REQUIRE(t, "templates handle is NULL");
    REQUIRE(gram, "gram must be a device pointer");
    return tpl_gram_out(t, gram, (cudaStream_t)stream);
}

furax_status furax_deproject_apply(const furax_templates_t *t, const void *in, void *out, int32_t dtype, void *stream)
{
    REQUIRE(t, "templates handle is NULL");
    REQUIRE(in && out, "in and out must be device pointers");
    REQUIRE(in != out, "in and out must not alias");
    REQUIRE(valid_dtype(dtype), "unknown dtype %d", dtype);
    return deproject_apply(t, in, out, dtype, (cudaStream_t)stream);
}

furax_status furax_ptfp_apply(const furax_templates_t *t, const double *x, double *out, const uint8_t *valid,
                              int32_t precision, int32_t acc, void *stream)
{
    REQUIRE(t, "templates handle is NULL");
    REQUIRE(x && out, "x and out must be device pointers");
    REQUIRE(x != out, "x and out must not alias");
    REQUIRE(valid_dtype(precision) || precision == FURAX_PREC_F32X2, "unknown precision %d", precision);
    REQUIRE(valid_acc(acc), "unknown accumulation mode %d", acc);
    return ptnp_apply(t->p, t->n, x, out, valid, precision, acc, (cudaStream_t)stream, t);
}

furax_status furax_mapmaker_cg_deproject(const furax_templates_t *t, const void *d, int32_t d_t, double *x,
                                         uint8_t *valid, const furax_cg_opts *o, furax_cg_result *res,
                                         double *amplitudes, void *stream)
{
    REQUIRE(t, "templates handle is NULL");
    REQUIRE(d && x, "d and x must be device pointers");
    REQUIRE(o && res, "opts and result must be host pointers");
    REQUIRE(valid_dtype(d_t), "unknown dtype %d", d_t);
    REQUIRE(o->maxiter >= 0 && o->maxiter <= 1000000, "maxiter out of range");
    REQUIRE(o->tol >= 0.0, "tol must be >= 0");
    REQUIRE(valid_dtype(o->precision), "unknown precision %d", o->precision);
    REQUIRE(valid_acc(o->acc), "unknown accumulation mode %d", o->acc);
    REQUIRE(o->precision == FURAX_F64 || (o->inner_tol >= 0.0 && o->inner_tol < 1.0 && o->max_outer >= 1),
            "mixed precision needs 0 <= inner_tol < 1 and max_outer >= 1");
    REQUIRE(o->check_every >= 1, "check_every must be >= 1");
    REQUIRE(!res->hist || res->hist_len >= 0, "hist_len must be >= 0");
    REQUIRE(!o->allreduce, "detector sharding (allreduce) is not available with templates");
    return mapmaker_cg(t->p, t->n, d, d_t, x, valid, o, res, (cudaStream_t)stream, t, amplitudes);
}

furax_status furax_chi2_grad(const furax_pointing_t *p, const furax_noise_t *n, const void *d, int32_t d_t,
                             const double *m, double *chi2, double *grad_map, double *grad_psi, int32_t precision,
                             void *stream)
{
    furax_status rc = check_pair(p, n);
    if (rc) return rc;
    REQUIRE(d && m && chi2, "d, m and chi2 must be device pointers");
    REQUIRE(valid_dtype(d_t) && (valid_dtype(precision) || precision == FURAX_PREC_F32X2), "unknown dtype or precision");
    REQUIRE(!long_band(n), "chi2 and its gradients take bands of at most %d taps", MAXTAPS);
    return launch_chi2_grad(p, n, d, d_t, m, chi2, grad_map, grad_psi, precision, (cudaStream_t)stream);
}

}  // extern "C"
