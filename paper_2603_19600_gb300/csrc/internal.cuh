// Internal declarations shared by the CUDA translation units of libfurax.
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "furax.h"

namespace fx {

constexpr int TILE = 4096;      // samples per work tile (one detector, contiguous in time)
constexpr int PTILE = 4096;     // pixels per pixel tile (vector kernels, per-observation reductions)
constexpr int MAXTAPS = 64;     // longest band of the fused kernels (c_0..c_63)
constexpr int kLongTaps = 2048; // longest band of the overlap-save N^-1 (TOD in HBM)
constexpr int kCtlWords = 4;    // device control block of a pointing handle (error, hold, wait budget)
constexpr int kBandPairs = 128; // band of the fused kernels in tap order (127 taps + one zero), as FP32 pairs

struct ObsInfo {
    int64_t nsamp;     // samples per detector
    int64_t det_off;   // first detector (global index into q_det / noise parameters)
    int64_t bore_off;  // first boresight sample (global index into q_bore)
    int64_t tod_off;   // first TOD element
    int64_t map_off;   // first pixel of this observation's map
    int64_t npix;      // 12 nside^2
    int64_t ptile0;    // first pixel tile of this observation
    int32_t nptile;    // number of pixel tiles
    int32_t ndet;
    int32_t nside;
    int32_t hwp;       // 1 if the batch has a half-wave plate (weights reflected per sample)
};

struct Tile {          // one detector, samples [t0, t0+len)
    int64_t t0;
    int32_t obs;
    int32_t det;       // local detector index within the observation
    int32_t len;
    int32_t pad;
};

struct FftItem {       // two consecutive overlap-save blocks of one detector stream
    int64_t q0;        // first block index
    int32_t obs;
    int32_t det;       // local detector index within the observation
};

// A pixel-sorted tile (fused_sorted.cu): nrow detectors of one observation whose tracks on the sky
// coincide (one column of the focal plane along the scan), over the core samples [t0, t0 + len)
// of each, with the band's halos. Its gathered samples, sorted by pixel once per pointing refresh,
// are perm[perm_off .. perm_off + perm_n[tile]) (entries: row << 12 | stage position in the row).
struct STile {
    int64_t t0;
    int64_t perm_off;  // first uint16 entry (a multiple of 8: 16-byte aligned)
    int32_t obs;
    int32_t len;       // core samples per row
    int32_t nrow;      // detectors (rows), <= kSRowMax
    int32_t det0;      // first entry of the tile's rows in the sorted-detector list (local indices)
};
constexpr int kSNE = 4096;     // stage entries of a pixel-sorted tile (all rows, halos included)
constexpr int kSRowMax = 16;   // rows per pixel-sorted tile (4 bits of a permutation entry)
// Row stride of a pixel-sorted tile in stage entries: core + two band halos + up to 3 + 3 entries
// of 16-byte alignment of the copied range, rounded to 4.
__host__ __device__ constexpr int srow_stride(int len) { return (len + 2 * 63 + 6 + 3) & ~3; }

struct PTile {         // pixels [p0, p0+len) of one observation (global map indices)
    int64_t p0;
    int32_t obs;
    int32_t len;
};

// Everything a kernel needs to know about the pointing; passed by value.
struct PointingView {
    const ObsInfo *obs;
    const double *q_bore;
    const double *q_det;
    const double2 *psi_cs;  // per global detector (cos 2 delta, sin 2 delta), or nullptr
    const int32_t *pix;     // cache (modes 1, 2)
    const float *c32, *s32; // cache modes 1 and 3 (weights rounded to FP32)
    const float *c32lo, *s32lo; // cache mode 3: FP64 weight - FP32 weight
    const double *c64, *s64;// cache mode 2
    const double2 *hwp_cs;  // per boresight sample (cos 4w, sin 4w) of the half-wave plate, or nullptr
};

struct NoiseView {
    int32_t kind;           // FURAX_NOISE_WHITE / BANDED
    int32_t ntaps;
    const double *p64;      // white: inverse variance [ndet]; banded: taps [ndet][ntaps]
    const float *p32;
    const double *diag;     // diagonal of N^-1 per detector [ndet] (FP64)
    const float *band2;     // banded (<= MAXTAPS taps): [ndet][2 kBandPad] band in tap order as duplicated pairs
};

// Template work folded into the fused FP32 operator (see fused_tma.cu).
struct FusedTpl {
    int mode;        // 1: add T^T N^-1 P x to proj[det][4]; 2: augmented system, amplitudes at base + det
    double *proj;    // mode 1
    int64_t base;    // mode 2: index of detector 0's amplitude pseudo-pixel (npix_total)
    int order;       // highest Legendre degree
};

// Template deprojection (per-detector Legendre templates, W = N^-1).
struct TplView {
    int32_t order;          // highest Legendre degree K (<= 3)
    int32_t halo;           // band half-width of W (0 for white noise)
    const double2 *mom;     // [ndet] (mu0, mu2): zeroth and second moments of the band
    const double *ginv;     // [ndet][4][4] (T^T W T)^-1, zero beyond K
    const double *b;        // [ndet][4] template amplitudes of the last solve
};

// The caller's detector-sharding sum (furax_cg_opts.allreduce), or nothing.
struct AllReduce {
    furax_allreduce_fn fn = nullptr;
    void *user = nullptr;
    bool on() const { return fn != nullptr; }
    furax_status operator()(void *buf, int64_t n, int32_t dtype, cudaStream_t st) const;
};

// Status helpers (thread-local message).
furax_status set_error(furax_status code, const char *fmt, ...);
furax_status check_cuda(cudaError_t e, const char *what);
furax_status check_launch(const char *what);
void count_launches(int64_t n);

// Kernel timing (furax_profile_*): kind 0 = FP32 fused apply, 1 = FP64 fused apply.
bool prof_on();
void prof_pair(cudaEvent_t *a, cudaEvent_t *b);          // two events from the pool
void prof_push(int kind, cudaEvent_t a, cudaEvent_t b);  // recorded pair, read later
void prof_add(int kind, double ms);
void prof_flush();                                       // wait for pending pairs, accumulate

// Raise a kernel's dynamic shared-memory limit once (per process, per kernel), then launch.
furax_status allow_smem(const void *kern, size_t bytes);
template <typename... KArgs, typename... Args>
furax_status launch_dyn(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                        Args... args)
{
    if (smem > 48 * 1024) {
        furax_status rc = allow_smem((const void *)kern, smem);
        if (rc) return rc;
    }
    kern<<<grid, block, smem, st>>>(args...);
    return FURAX_OK;
}

struct CgWs;

}  // namespace fx

// Handles (opaque to the C API).
struct furax_pointing {
    int32_t mode = 0;
    int32_t n_obs = 0;
    std::vector<fx::ObsInfo> obs;     // host copy
    fx::ObsInfo *d_obs = nullptr;
    std::vector<fx::Tile> tiles;      // host copy
    fx::Tile *d_tiles = nullptr;
    int64_t n_tiles = 0;
    std::vector<fx::PTile> ptiles;
    fx::PTile *d_ptiles = nullptr;
    int64_t n_ptiles = 0;
    const double *q_bore = nullptr, *q_det = nullptr;
    double2 *d_psi_cs = nullptr;
    bool has_psi = false;
    double2 *d_hwp_cs = nullptr;      // [nbore] (cos 4w, sin 4w), with a half-wave plate
    bool has_hwp = false;
    int32_t *pix = nullptr;
    float *c32 = nullptr, *s32 = nullptr;
    float *c32lo = nullptr, *s32lo = nullptr;
    double *c64 = nullptr, *s64 = nullptr;
    int64_t nsamp_total = 0, npix_total = 0, ndet_total = 0, nbore_total = 0, n_invalid = 0;
    int32_t max_ndet = 0;
    int32_t n_sm = 1;                 // SMs of the device (persistent grids)
    unsigned *d_err = nullptr;        // device control block (kCtlWords): error word of the bounded waits,
                                      // loader hold flag, wait budget (mbarrier.cuh)
    // workspaces, allocated on first use and freed by destroy
    float4 *ws_map32 = nullptr;       // [npix] padded FP32 copy of a map for the gather
    float4 *ws_acc_hi = nullptr;      // [2 npix] FP32 accumulator (I,Q,U,-): plain hi[i], or compensated
                                      // hi[2i] with its compensation at hi[2i + 1] (atomics.cuh)
    double *ws_acc64 = nullptr;       // [npix][3] FP64 accumulator
    float4 *ws_df_lo = nullptr;       // [npix] FP32 low-word accumulator of the double-FP32 RHS and operator
    float4 *ws_x2 = nullptr;          // [npix][2] double-FP32 split (high, low words) of an FP64 map
    double *ws_x64 = nullptr;         // [npix][3] masked FP64 copy
    void *ws_tod = nullptr;           // [nsamp] scratch TOD (FP64 size)
    void *ws_tod2 = nullptr;
    int32_t *ws_hits = nullptr;       // [npix] hit counts when the caller passes none
    float *ws_bore_m = nullptr;       // [nbore][18] boresight rotation matrices (double-FP32)
    fx::CgWs *cg = nullptr;           // solver workspace (allocated by the first solve)
    // operator schedule (furax_pointing_set_schedule); pixel-sorted tiles and their permutation
    furax_schedule sched{};
    fx::STile *d_stiles = nullptr;
    int64_t n_stiles = 0;
    int32_t *d_sdet = nullptr;        // detectors of the sorted tiles' rows, grouped (local indices)
    uint16_t *d_perm = nullptr;       // per tile: gathered samples sorted by pixel
    int32_t *d_perm_n = nullptr;      // per tile: entries of its permutation
    int64_t perm_cap = 0;
    fx::PointingView view() const {
        return fx::PointingView{d_obs, q_bore, q_det, has_psi ? d_psi_cs : nullptr, pix, c32, s32, c32lo, s32lo, c64, s64,
                                has_hwp ? d_hwp_cs : nullptr};
    }
};

struct furax_templates {
    const furax_pointing *p = nullptr;   // layout and pointing (caller-owned, outlives the handle)
    const furax_noise *n = nullptr;      // W = N^-1 (caller-owned, outlives the handle)
    int32_t order = 0;
    int32_t halo = 0;
    int64_t ndet = 0;
    double2 *mom = nullptr;
    double *gram = nullptr;              // [ndet][4][4] T^T W T
    double *ginv = nullptr;              // [ndet][4][4]
    double *a = nullptr;                 // [ndet][4] projections (kept zero between uses)
    double *b = nullptr;                 // [ndet][4]
    unsigned long long *bad = nullptr;   // setup status (1 + first detector with a singular Gram matrix)
    // Augmented layout of the inner FP32 solve (order <= 2): one amplitude pseudo-pixel per
    // detector at npix_total + det; each map's pixel tiles followed by its detectors' pseudo tiles.
    fx::PTile *d_aug_ptiles = nullptr;
    fx::ObsInfo *d_aug_obs = nullptr;
    int64_t n_aug_ptiles = 0;
    fx::TplView view() const { return fx::TplView{order, halo, mom, ginv, b}; }
};

struct furax_noise {
    int32_t kind = 0;
    int32_t ntaps = 0;
    int64_t ndet_total = 0;
    int64_t nsamp_total = 0;
    double *p64 = nullptr;
    float *p32 = nullptr;
    double *diag = nullptr;
    fx::ObsInfo *d_obs = nullptr;     // TOD layout for the standalone N^-1
    fx::Tile *d_tiles = nullptr;
    int64_t n_tiles = 0;
    // bands longer than MAXTAPS: overlap-save blocks, twiddles, spectra (bit-reversed order)
    fx::FftItem *fft_items = nullptr;
    int64_t n_fft_items = 0;
    double2 *tw64 = nullptr;
    float2 *tw32 = nullptr;
    double *spec64 = nullptr;   // [ndet][8192]
    float *spec32 = nullptr;
    // gap-filling workspaces (TOD-sized), allocated by the first furax_gapfill that needs them and
    // reused by later calls; freed with the handle
    double *gf_y = nullptr, *gf_r = nullptr, *gf_p = nullptr, *gf_q = nullptr;
    float *gf_x32 = nullptr, *gf_n32 = nullptr;
    void *gf_sc = nullptr;
    float *band2 = nullptr;     // banded, <= MAXTAPS taps: [ndet][256] band in tap order as duplicated pairs
    fx::NoiseView view() const { return fx::NoiseView{kind, ntaps, p64, p32, diag, band2}; }
};

namespace fx {

furax_status ensure_ws(furax_pointing *p, void **ptr, size_t bytes);

// ---- launchers (pointing.cu)
furax_status launch_expand(const furax_pointing *p, int32_t *pix, float *c32, float *s32, double *c64,
                           double *s64, unsigned long long *n_invalid, cudaStream_t st, bool all_mode,
                           float *c32lo = nullptr, float *s32lo = nullptr);
furax_status launch_set_psi(furax_pointing *p, const double *psi, cudaStream_t st);
furax_status launch_set_hwp(furax_pointing *p, const double *hwp, cudaStream_t st);
// FP32 cache fill with certified FP32 pixels and exact FP64 fallback (pointing_fast.cu)
furax_status launch_expand_fast(const furax_pointing *p, unsigned long long *n_invalid, cudaStream_t st);
furax_status launch_P(const furax_pointing *p, const void *map, int map_t, void *tod, int tod_t, cudaStream_t st);
furax_status launch_PT(const furax_pointing *p, const void *tod, int tod_t, void *map, int map_t, int acc,
                       int32_t *hits, int accumulate, cudaStream_t st);
furax_status launch_bj(const furax_pointing *p, const furax_noise *n, double rcond_min, double *blocks_inv,
                       uint8_t *valid, int32_t *hits, double *rcond, cudaStream_t st, const AllReduce &ar = AllReduce{});

// ---- launchers (noise.cu)
furax_status launch_ninv(const furax_noise *n, const void *in, void *out, int dtype, cudaStream_t st);
// FP64 in, FP64 out, band product in double-FP32 (bands of up to MAXTAPS taps; fused_df.cu)
furax_status launch_ninv_df(const furax_noise *n, const double *in, double *out, cudaStream_t st);
// Bands longer than the fused kernels hold go through the TOD in HBM (overlap-save N^-1).
inline bool long_band(const furax_noise *n) { return n->kind == FURAX_NOISE_BANDED && n->ntaps > MAXTAPS; }
// noise_fft.cu: blocks, twiddles and spectra of a long band (synchronises st); the N^-1 apply.
furax_status prepare_noise_fft(furax_noise *n, const std::vector<ObsInfo> &obs, cudaStream_t st);
furax_status launch_ninv_fft(const furax_noise *n, const void *in, void *out, int dtype, cudaStream_t st);
// acc64 += P^T tod (FP64 accumulation into the caller's [npix][3] accumulator; pointing.cu).
furax_status launch_PT_acc64(const furax_pointing *p, const void *tod, int tod_t, double *acc64, cudaStream_t st);
// The normal operator and right-hand side with the TOD in HBM (solver.cu): acc64 += P^T N^-1 P x
// (TOD in tod_t) and acc64 += P^T N^-1 d (FP64 TOD). The TOD workspaces must exist (tod_ws).
furax_status tod_ws(const furax_pointing *p);
furax_status launch_ata_chain(const furax_pointing *p, const furax_noise *n, const double *x, int tod_t,
                              double *acc64, cudaStream_t st);
furax_status launch_rhs_chain(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, double *acc64,
                              cudaStream_t st);
// Observation table, time tiles and pixel tiles of a batch.
struct Layout {
    std::vector<ObsInfo> obs;
    std::vector<Tile> tiles;
    std::vector<PTile> ptiles;
    int64_t ndet = 0, nbore = 0, nsamp = 0, npix = 0;
    int32_t max_ndet = 0;
};
void build_layout(const furax_obs_desc *d, Layout &L);
furax_status prepare_kernels();
// r_out = N^-1 (d - P m) in FP64 or FP32; also per-detector psi gradient partials
furax_status launch_chi2_grad(const furax_pointing *p, const furax_noise *n, const void *d, int d_t,
                              const double *m, double *chi2, double *grad_map, double *grad_psi, int precision,
                              cudaStream_t st);

// ---- pixel-sorted operator (fused_sorted.cu)
// Build (or drop, for the time-ordered kernel) the pixel-sorted tiles of a cached FP32 pointing and
// sort them; synchronises st. The permutation follows the cache: sort_sorted_tiles after a refresh.
furax_status set_schedule(furax_pointing *p, const furax_schedule &s, cudaStream_t st);
furax_status sort_sorted_tiles(const furax_pointing *p, cudaStream_t st);
bool sorted_active(const furax_pointing *p);
void free_sorted(furax_pointing *p);
furax_status launch_fused_sorted(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc, float4 *hi,
                                 float4 *lo, double *a64, cudaStream_t st);
furax_status prepare_fused_sorted();

// ---- launchers (fused.cu)
// acc_* workspaces must be zeroed by the caller; x32 is the padded FP32 copy of the (masked) input.
// With ft (cached FP32 pointing only: see fused_f32_projects_templates), the kernel also does
// the template work of ft->mode.
furax_status launch_fused_f32(const furax_pointing *p, const furax_noise *n, const float4 *x32, int acc,
                              float4 *acc_hi, float4 *acc_lo, double *acc64, cudaStream_t st,
                              const FusedTpl *ft = nullptr);
bool fused_f32_projects_templates(const furax_pointing *p);
furax_status launch_fused_f64(const furax_pointing *p, const furax_noise *n, const double *x, double *acc64,
                              cudaStream_t st);
// FP64-accurate operator on FP32 units (double-FP32 band product): acc64 += P^T N^-1 P x, or
// acc64 += P^T N^-1 d when d != nullptr.
// tp (FP32 d only): fold the template correction -P^T (W T) b of the deprojected right-hand side into
// the same pass, with b already solved by launch_tpl_rhs_amplitudes.
furax_status launch_chi2_df(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, const double *m,
                            double *chi2, double *grad_map, double *grad_psi, cudaStream_t st);
furax_status launch_fused_df(const furax_pointing *p, const furax_noise *n, const double *x, const void *d, int d_t,
                             double *acc64, cudaStream_t st, const furax_templates *tp = nullptr);
// b = P^T N^-1 d accumulated into acc64 (FP64 stencil)
furax_status launch_rhs_f64(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, double *acc64,
                            cudaStream_t st);

// ---- vector helpers (solver.cu)
furax_status launch_pack_x32(const furax_pointing *p, const double *x, const uint8_t *valid, float4 *x32,
                             float4 *zero_a, float4 *zero_b, cudaStream_t st);
furax_status launch_finalize_acc(const furax_pointing *p, int acc, const float4 *hi, const float4 *lo,
                                 const double *acc64, const uint8_t *valid, double *out, cudaStream_t st);
furax_status launch_mask_copy(const furax_pointing *p, const double *x, const uint8_t *valid, double *out,
                              cudaStream_t st);
furax_status ptnp_apply(const furax_pointing *p, const furax_noise *n, const double *x, double *out,
                        const uint8_t *valid, int precision, int acc, cudaStream_t st,
                        const furax_templates *tp = nullptr);
furax_status mapmaker_cg(const furax_pointing *p, const furax_noise *n, const void *d, int d_t, double *x,
                         uint8_t *valid, const furax_cg_opts *o, furax_cg_result *res, cudaStream_t st,
                         const furax_templates *tp = nullptr, double *amplitudes = nullptr);

// ---- template deprojection (templates.cu)
furax_status templates_create(const furax_pointing *p, const furax_noise *n, int order, cudaStream_t st,
                              furax_templates **out);
void templates_destroy(furax_templates *tp);
// acc -= P^T (W T) G^-1 (W T)^T P x; FP32 (x32, acc mode) or FP64 (x64, acc64) arithmetic.
// projected: the projection is already in tp->a (accumulated by the fused FP32 kernel).
furax_status launch_tpl_map(const furax_templates *tp, int precision, int acc, const float4 *x32, const double *x64,
                            float4 *hi, float4 *lo, double *acc64, cudaStream_t st, bool projected = false);
// The tp->a the fused FP32 operator should accumulate into, or nullptr (no templates, or a
// pointing mode whose FP32 kernel does not project).
double *tpl_fused_target(const furax_templates *tp, const furax_pointing *p);
// acc64 -= P^T (W T) G^-1 (W T)^T d (FP64 arithmetic).
furax_status launch_tpl_rhs(const furax_templates *tp, const void *d, int d_t, double *acc64, cudaStream_t st);
// b = G^-1 (W T)^T d only (the first half of launch_tpl_rhs), for a right-hand side that folds the
// correction into its own pass.
furax_status launch_tpl_rhs_amplitudes(const furax_templates *tp, const void *d, int d_t, cudaStream_t st);
// The inner FP32 solve runs on the augmented system [m; amplitudes] (one fused pass per iteration).
bool tpl_augmented(const furax_templates *tp, int precision);
// minv and valid of the amplitude pseudo-pixels: the 3x3 leading block of G^-1.
furax_status launch_tpl_aug_precond(const furax_templates *tp, double *minv, uint8_t *valid, cudaStream_t st);
// amp [ndet][K+1] = G^-1 (W T)^T (d - P m) (m: FP64 map, zero on masked pixels).
furax_status tpl_amplitudes(const furax_templates *tp, const void *d, int d_t, const double *m, double *amp,
                            cudaStream_t st);
// out [ndet][K+1][K+1] = T^T W T.
furax_status tpl_gram_out(const furax_templates *tp, double *out, cudaStream_t st);
// out = F_T in for a TOD (in != out).
// Gap filling by constrained realisation (gapfill.cu); n holds the covariance band.
furax_status gapfill(const furax_noise *n, const void *d, const uint8_t *valid, const void *nr, void *out, int dtype,
                     int maxiter, double tol, int precision, int32_t *iters_out, cudaStream_t st);
furax_status deproject_apply(const furax_templates *tp, const void *in, void *out, int dtype, cudaStream_t st);

}  // namespace fx
