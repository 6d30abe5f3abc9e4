/*
 * furax.h — C-ABI of the GB300 map-making hot path (libfurax.so).
 *
 * The library implements the operators of linear-operator CMB map-making as
 * stated in the Furax paper (arXiv 2603.19600):
 *   data model d = P m + n and the estimator m^ = (P^T N^-1 P)^-1 P^T N^-1 d
 *     (Statement of Need; the Software Design listing "A = (H.T @ N.I @ H).I @ H.T @ N.I"),
 *   PointingOperator: sky-to-TOD projection with the pointing expanded on the
 *     fly (Table 3; "Map-making classes"),
 *   its transpose (Table 1, "A.T"),
 *   HomothetyOperator / SymmetricBandToeplitzOperator noise weighting (Table 2),
 *   BJPreconditioner and the solver-backed inverse "A.I(solver=..., preconditioner=...)"
 *     (Table 1; "Map-making classes"),
 *   the block decomposition P^T N^-1 P = sum_i P_i^T N_i^-1 P_i over observations
 *     ("Algebraic reductions"; MultiObservationMapMaker).
 * Conventions below the operator level (the paper states none) are fixed here:
 *   quaternions (w, x, y, z), Hamilton product, detector quaternion q_bore (x) q_det;
 *   line of sight = R(q) z^, orientation = R(q) x^; HEALPix RING pixels;
 *   weights (1, cos 2psi, sin 2psi) with psi measured from north through east;
 *   banded N^-1: y_t = sum_{|k|<K} c_|k| x_{t+k} over 0 <= t+k < nsamp.
 *
 * Layouts (all row-major, caller-owned):
 *   observation i has ndet_i detectors, nsamp_i samples, nside_i; npix_i = 12 nside_i^2.
 *   TOD: observations concatenated, each [ndet_i][nsamp_i]   (sum_i ndet_i*nsamp_i elements)
 *   map: observations concatenated, each [npix_i][3] = (I,Q,U) (sum_i npix_i pixels)
 *   q_bore: [sum_i nsamp_i][4] FP64; q_det: [sum_i ndet_i][4] FP64.
 * Pointers named "device" must be CUDA device pointers (or managed memory) on the
 * current device; "host" pointers are ordinary host memory. Every call is
 * asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream) unless
 * it says it synchronises. Handles are not thread-safe: one stream at a time.
 *
 * Errors: every function returns a furax_status. Negative values are errors and
 * leave outputs unspecified; furax_last_error() returns a thread-local message.
 * No function aborts, traps or exits on bad input.
 */
#ifndef FURAX_H
#define FURAX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t furax_status;
#define FURAX_OK 0
#define FURAX_ENOTCONVERGED 1 /* solver stopped at maxiter above tolerance (not an error) */
#define FURAX_EINVAL (-1)      /* bad argument: null pointer, size, enum, mismatch */
#define FURAX_ENOMEM (-2)      /* device allocation failed */
#define FURAX_ECUDA (-3)       /* a CUDA call failed; message has the CUDA error string */
#define FURAX_EBADINPUT (-4)   /* data unusable (e.g. no valid pixel to solve for) */
#define FURAX_ETIMEOUT (-5)    /* a bounded device-side wait gave up */

typedef enum { FURAX_F32 = 0, FURAX_F64 = 1 } furax_dtype;

/* Arithmetic of an operator application (furax_ptnp_apply): FURAX_F32, FURAX_F64, or
 * FURAX_PREC_F32X2 = FP64-accurate results computed on FP32 units (double-FP32 "Dot2" band
 * product with exact FP32 products and two-sums; FP64 gather and per-pixel sums). */
#define FURAX_PREC_F32X2 2

/* Accumulation of P^T into pixels. */
typedef enum {
    FURAX_ACC_F64 = 0,       /* FP64 atomic sums per pixel component */
    FURAX_ACC_F32_KAHAN = 1, /* FP32 sums with every rounding error captured exactly
                                (atomic two-sum) and summed in a second FP32 word */
    FURAX_ACC_F32 = 2        /* plain FP32 atomic sums (fastest, least accurate) */
} furax_acc;

/* How the pointing is held between operator applications. */
typedef enum {
    FURAX_POINTING_ON_THE_FLY = 0, /* recompute pixel and weights from quaternions each call */
    FURAX_POINTING_CACHE_F32 = 1,  /* cache int32 pixel + FP32 (cos 2psi, sin 2psi): 12 B/sample */
    FURAX_POINTING_CACHE_F64 = 2,  /* cache int32 pixel + FP64 weights: 20 B/sample */
    FURAX_POINTING_CACHE_MIXED = 3 /* cache int32 pixel + FP32 weights (hi) + FP32 corrections (lo),
                                      hi + lo = the FP64 weight to ~2^-48: FP32 operators stream
                                      12 B/sample, FP64-accurate ones 20 B/sample */
} furax_pointing_mode;

typedef enum { FURAX_NOISE_WHITE = 0, FURAX_NOISE_BANDED = 1 } furax_noise_kind;

typedef struct furax_pointing furax_pointing_t;
typedef struct furax_noise furax_noise_t;
typedef struct furax_templates furax_templates_t;

/* How the cached FP32 normal operator walks the samples (furax_pointing_set_schedule). It changes
 * the order of the floating-point additions only, never the operator or the accumulation mode.
 *   FURAX_SCHED_TIME_ORDERED: tiles of one detector x 4096 consecutive samples; every sample does
 *     one gather of its pixel and one reduction into it.
 *   FURAX_SCHED_PIXEL_SORTED: tiles of the detectors whose tracks on the sky coincide (one column
 *     of the focal plane along the scan: equal cross-scan offsets within group_tol pixel widths,
 *     at most max_rows of them) over tile_len samples each; the samples of a tile, sorted by pixel
 *     once per pointing refresh, gather each pixel once and accumulate each pixel's run of samples
 *     with one reduction (the block decomposition P^T N^-1 P = sum_i P_i^T N_i^-1 P_i of
 *     "Algebraic reductions", taken over such tiles). Templates keep the time-ordered kernel. */
#define FURAX_SCHED_TIME_ORDERED 0
#define FURAX_SCHED_PIXEL_SORTED 1
typedef struct {
    int32_t kernel;     /* FURAX_SCHED_TIME_ORDERED or FURAX_SCHED_PIXEL_SORTED */
    int32_t tile_len;   /* pixel-sorted: samples per detector row, a multiple of 16 in [16, 4096]; 0 = as
                           many as the tile's stage holds for its rows */
    int32_t max_rows;   /* pixel-sorted: detectors per tile, 1..16 */
    double group_tol;   /* pixel-sorted: cross-scan grouping tolerance in pixel widths (> 0) */
    int32_t l2_evict_first; /* both kernels: 1 reads the pointing stream (read once per application)
                               with an L2 evict-first policy, so that it does not evict the map and
                               the accumulators; 0 uses the default policy */
    int32_t consumer_warps; /* time-ordered kernel: warps that run the band and the scatter, 8 or 16
                               (0 = 8); with 16 twice the reductions are in flight (templates keep 8) */
} furax_schedule;

/* A batch of observations: each with its own map, or sharing maps by map_id. */
typedef struct {
    int32_t n_obs;            /* >= 1 */
    const int32_t *ndet;      /* host [n_obs], each >= 1 */
    const int64_t *nsamp;     /* host [n_obs], each >= 1 */
    const int32_t *nside;     /* host [n_obs], each in [1, 8192] */
    const double *q_bore;     /* device [sum nsamp][4], unit quaternions (not renormalised) */
    const double *q_det;      /* device [sum ndet][4], unit quaternions */
    const double *psi_offset; /* device [sum ndet] polarisation-angle offsets (rad), or NULL */
    const double *hwp_angle;  /* device [sum nsamp] angle w (rad) of an ideal half-wave plate in front
                                 of every detector, one value per boresight sample, or NULL (no plate).
                                 With a plate (HWPOperator, Table 3) the weights become
                                 (1, cos(4w - 2psi), sin(4w - 2psi)); pixels do not change. Read once
                                 at creation (kept as cos 4w, sin 4w). */
    const int32_t *map_id;    /* host [n_obs] or NULL (one map per observation). Observations with
                                 equal map_id share one map and are solved jointly ("Algebraic
                                 reductions": P^T N^-1 P = sum_i P_i^T N_i^-1 P_i over the
                                 observations i of the map); they must have equal nside. Maps are
                                 laid out in order of the first observation of each, and every
                                 map-sized array ([npix_total][...]) follows that layout. */
} furax_obs_desc;

/* ---------------------------------------------------------------------------------------
 * Pointing operator P (PointingOperator, Table 3; IndexOperator "projecting skies onto
 * time-ordered series", Table 2; QU rotation + ideal polariser folded into the weights).
 * ------------------------------------------------------------------------------------- */

/* Create a pointing operator over `desc`. The quaternion arrays are referenced, not copied:
 * they must stay valid and unchanged while the handle lives. psi_offset is copied.
 * Cache modes run the pointing expansion once here. Samples whose quaternion product is
 * not finite get pixel -1 and are skipped by every operator; their count is available
 * from furax_pointing_info. Synchronises `stream` once (to read that count).
 * Errors: EINVAL (bad sizes/pointers/mode), ENOMEM, ECUDA. *out is NULL on error. */
furax_status furax_pointing_create(const furax_obs_desc *desc, int32_t mode, void *stream,
                                   furax_pointing_t **out);
furax_status furax_pointing_destroy(furax_pointing_t *p);

/* Host query: total samples, total pixels, total detectors, number of invalid samples. */
furax_status furax_pointing_info(const furax_pointing_t *p, int64_t *nsamp_total, int64_t *npix_total,
                                 int64_t *ndet_total, int64_t *n_invalid);

/* Recompute the cached pixels and weights from the quaternion arrays given at creation (their
 * contents may have changed, their shapes may not). No-op for FURAX_POINTING_ON_THE_FLY. */
furax_status furax_pointing_refresh(furax_pointing_t *p, void *stream);

/* Choose how the cached FP32 normal operator of this handle walks its samples (see
 * furax_schedule). A pixel-sorted schedule builds its tiles from the detectors' focal-plane
 * offsets and the direction of the boresight's motion (read from q_det and a few q_bore samples),
 * allocates its permutation (about 3 bytes per sample, owned by the handle) and sorts it;
 * furax_pointing_refresh re-sorts it. Synchronises `stream`. Errors: FURAX_EINVAL for a pointing
 * without an FP32 cache (modes FURAX_POINTING_CACHE_F32 / _MIXED) or out-of-range fields,
 * FURAX_ENOMEM. The default is FURAX_SCHED_TIME_ORDERED. */
furax_status furax_pointing_set_schedule(furax_pointing_t *p, const furax_schedule *s, void *stream);
/* The handle's current schedule. */
furax_status furax_pointing_get_schedule(const furax_pointing_t *p, furax_schedule *s);

/* Autotuner of the schedule: for each of the ncand candidate schedules (host array), set it on
 * the handle, run the fused FP32 normal operator once untimed and `reps` times timed (CUDA events
 * on `stream` around each launch, a zero input map, accumulators cleared outside the timed
 * interval) with the given accumulation (FURAX_ACC_*, never changed by the search), and write the
 * mean milliseconds per launch to ms_out[k] (host, -1 for a candidate the handle rejects). The
 * fastest is left set on the handle and its index written to *best_out. Synchronises `stream`
 * repeatedly; allocates the handle's operator workspaces. Errors: FURAX_EINVAL for a pointing
 * without an FP32 cache, a band longer than 64 taps, bad arguments or no valid candidate (the
 * previous schedule is then restored); a device error ends the search the same way. The paper has
 * no counterpart: its operators are compiled by XLA. */
furax_status furax_autotune(furax_pointing_t *p, const furax_noise_t *n, int32_t acc, const furax_schedule *cand,
                            int32_t ncand, int32_t reps, double *ms_out, int32_t *best_out, void *stream);
/* The built-in search space: copies up to cap candidates into out (may be NULL) and returns how
 * many there are: for l2_evict_first 0 and 1, the time-ordered kernel with 8 and 16 consumer
 * warps, then the pixel-sorted kernel over tile_len {0, 256, 512} x max_rows {8, 12} x
 * group_tol {1, 2}. */
int32_t furax_autotune_space(furax_schedule *out, int32_t cap);

/* Replace the per-detector polarisation-angle offsets (device [sum ndet] rad, or NULL for none).
 * Weights become (cos 2(psi+delta), sin 2(psi+delta)), or with a half-wave plate
 * (cos(4w - 2(psi+delta)), sin(4w - 2(psi+delta))) - the offset rotation passes through the plate
 * with its sign reversed ("Algebraic reductions": R(theta) o HWP = HWP o R(-theta)); pixels do
 * not change. */
furax_status furax_pointing_set_psi_offset(furax_pointing_t *p, const double *psi_offset, void *stream);

/* Expand the pointing: per sample its pixel within its observation's map (int32, -1 if
 * invalid) and weights (cos 2psi, sin 2psi) including offsets, in the TOD layout.
 * pix: device int32 [nsamp_total]; c, s: device [nsamp_total] of dtype w_t. */
furax_status furax_pointing_expand(const furax_pointing_t *p, int32_t *pix, void *c, void *s,
                                   int32_t w_t, void *stream);

/* furax_pointing_expand recomputes with the exact FP64 recipe. This copies out what the FP32
 * operators actually read from an FP32 or mixed cache: pixels (identical to the FP64 recipe's)
 * and FP32 weights without offsets (FURAX_POINTING_CACHE_F32 fills them from FP32 arithmetic,
 * relative error a few 1e-7 away from the poles; FURAX_POINTING_CACHE_MIXED rounds the FP64 values).
 * pix, c, s: device [nsamp_total]. Errors: EINVAL for other modes. */
furax_status furax_pointing_cache(const furax_pointing_t *p, int32_t *pix, float *c, float *s, void *stream);

/* tod = P map: tod[i] = I_p + Q_p cos 2psi_i + U_p sin 2psi_i (0 for invalid samples).
 * map: device [npix_total][3] of map_t; tod: device [nsamp_total] of tod_t (overwritten).
 * Arithmetic is FP64 if either dtype is FP64, else FP32. */
furax_status furax_pointing_apply(const furax_pointing_t *p, const void *map, int32_t map_t,
                                  void *tod, int32_t tod_t, void *stream);

/* map (+)= P^T tod: map[p] += sum_{i: pix_i = p} tod[i] (1, cos 2psi_i, sin 2psi_i).
 * accumulate = 0 overwrites map (and hits), 1 adds to it. hits (device int32 [npix_total])
 * may be NULL; when given it counts samples per pixel. acc selects the accumulation. */
furax_status furax_pointing_transpose(const furax_pointing_t *p, const void *tod, int32_t tod_t,
                                      void *map, int32_t map_t, int32_t acc, int32_t *hits,
                                      int32_t accumulate, void *stream);

/* ---------------------------------------------------------------------------------------
 * Noise weighting N^-1 (HomothetyOperator sigma^2, Software Design listing; DiagonalOperator;
 * SymmetricBandToeplitzOperator with direct convolution, Table 2).
 * ------------------------------------------------------------------------------------- */

/* kind WHITE: params = device FP64 [sum ndet] variances sigma^2 (N^-1 = 1/sigma^2 per detector).
 * kind BANDED: params = device FP64 [sum ndet][ntaps] taps c_0..c_{K-1} of the symmetric band
 * (1 <= ntaps <= 64); the band must be positive definite for the solver to converge.
 * The taps are copied (an FP32 copy is kept for the FP32 path). */
furax_status furax_noise_create(int32_t kind, const double *params, int32_t ntaps,
                                const furax_obs_desc *desc, void *stream, furax_noise_t **out);
furax_status furax_noise_destroy(furax_noise_t *n);

/* out = N^-1 in, per detector, finite section at the ends of each detector stream.
 * in, out: device [nsamp_total] of dtype; in and out must not overlap. */
furax_status furax_noise_inv_apply(const furax_noise_t *n, const void *in, void *out, int32_t dtype,
                                   void *stream);

/* ---------------------------------------------------------------------------------------
 * Block-Jacobi preconditioner (BJPreconditioner, "Map-making classes").
 * ------------------------------------------------------------------------------------- */

/* M_p = sum_{i: pix_i = p} ninv_det(i) w_i w_i^T with w = (1, cos 2psi, sin 2psi) and ninv the
 * diagonal of N^-1 (1/sigma^2, or tap c_0). Inverted in FP64 per pixel through its Cholesky
 * factor; pixel p is valid iff hits >= 3, every Cholesky pivot is positive (the block is positive
 * definite to working precision) and rcond = 1/(|M|_1 |M^-1|_1) >= rcond_min.
 * blocks_inv: device FP64 [npix_total][6] = (00,01,02,11,12,22) of M^-1, 0 where invalid;
 * valid: device uint8 [npix_total]; hits: device int32 [npix_total] (may be NULL);
 * rcond: device FP64 [npix_total] (may be NULL). */
furax_status furax_blockdiag_precond(const furax_pointing_t *p, const furax_noise_t *n, double rcond_min,
                                     double *blocks_inv, uint8_t *valid, int32_t *hits, double *rcond,
                                     void *stream);

/* ---------------------------------------------------------------------------------------
 * Normal-equations operator and right-hand side ("A = (H.T @ N.I @ H).I @ H.T @ N.I",
 * Software Design listing; block decomposition P^T N^-1 P = sum_i P_i^T N_i^-1 P_i).
 * ------------------------------------------------------------------------------------- */

/* out = S P^T N^-1 P S^T x with S the valid-pixel selector (valid may be NULL: all pixels).
 * x, out: device FP64 [npix_total][3], must not overlap. precision FURAX_F32 runs the
 * projection, the noise stencil and the weights in FP32 (x rounded to FP32 once) with
 * accumulation `acc`; FURAX_F64 runs everything in FP64 (acc ignored). One fused pass:
 * the time-ordered data never reaches device memory. */
furax_status furax_ptnp_apply(const furax_pointing_t *p, const furax_noise_t *n, const double *x,
                              double *out, const uint8_t *valid, int32_t precision, int32_t acc,
                              void *stream);

/* The FP32 normal-equations operator of furax_ptnp_apply (precision FURAX_F32, FURAX_ACC_F32) for
 * callers that cannot allocate device memory: code running inside a memory budget fixed up front
 * (a pre-sized pool of a host framework, a plugin that must not grow the process's footprint) or
 * code that must not synchronise the device, as cudaMalloc/cudaFree may. It takes one observation's
 * expanded pointing directly and allocates nothing; the paper has no counterpart (a deployment
 * variant). Its scratch (an FP32 copy of x and the FP32 accumulator) is one file-scope device array
 * sized for nside <= 256 (786,432 pixels, 25 MB), held by every GPU that loads the library until
 * the process exits.
 *   pix, c, s: device [ndet][nsamp] int32 / FP32 / FP32 (as furax_pointing_expand gives them; pixel
 *   -1 or outside the map = skipped); taps: device FP32 [ndet][ntaps], the symmetric band
 *   c_0..c_{K-1} (ntaps = 1: white noise, taps = 1/sigma^2); valid: device uint8 [12 nside^2] or
 *   NULL; x, out: device FP64 [12 nside^2][3], must not overlap.
 * Errors: FURAX_EINVAL for null pointers, bad sizes, or nside > 256. The first call on a device
 * looks up the scratch address (cudaGetSymbolAddress) with that device current: make it before
 * any stream capture. Every call shares the scratch and it keeps the last call's contents (the
 * kernels clear what must start at zero); calls that overlap on the GPU race on it. */
furax_status furax_ptnp_apply_noalloc(const int32_t *pix, const float *c, const float *s, int32_t ndet,
                                      int64_t nsamp, int32_t nside, const float *taps, int32_t ntaps,
                                      const uint8_t *valid, const double *x, double *out, void *stream);

/* b = S P^T N^-1 d in FP64 (d of dtype d_t, device [nsamp_total]; b device FP64 [npix_total][3]). */
furax_status furax_rhs(const furax_pointing_t *p, const furax_noise_t *n, const void *d, int32_t d_t,
                       const uint8_t *valid, double *b, void *stream);

/* ---------------------------------------------------------------------------------------
 * Map-maker: preconditioned conjugate gradient ("A.I(solver=..., preconditioner=...)",
 * Table 1; maximum-likelihood and binned estimators, "Map-making classes").
 * ------------------------------------------------------------------------------------- */

/* Sum over processes, for a map shared by processes that each hold a subset of its detectors
 * (detector sharding of P^T N^-1 P = sum_i P_i^T N_i^-1 P_i, "Algebraic reductions"). The solver
 * calls it with a device buffer of n elements (dtype FURAX_REDUCE_F64 or FURAX_REDUCE_I32) after
 * enqueueing the work that produced it on `stream`; on return, or for every operation enqueued
 * later on `stream`, buf must hold the elementwise sum over all processes (e.g. a collective
 * enqueued on the stream, or a synchronisation, a host-side sum and a copy back). Every process
 * must make the same sequence of calls with the same pointing layout (observations, nside, map
 * ids). A non-zero return ends the solve with that status. */
#define FURAX_REDUCE_F64 0
#define FURAX_REDUCE_I32 1
typedef furax_status (*furax_allreduce_fn)(void *buf, int64_t n, int32_t dtype, void *stream, void *user);

typedef struct {
    int32_t maxiter;       /* cap on PCG iterations per observation (all outer steps together) */
    double tol;            /* stop when ||b - A x||/||b|| <= tol */
    int32_t precision;     /* FURAX_F64: plain FP64 PCG. FURAX_F32: mixed precision — inner PCG
                              with the FP32 operator, outer defect correction with the FP64 operator */
    int32_t acc;           /* accumulation of the inner operator (FURAX_F32 only) */
    double inner_tol;      /* FURAX_F32: relative reduction asked of each inner solve (e.g. 1e-5);
                              0 runs the inner solve to the iteration cap */
    int32_t max_outer;     /* FURAX_F32: cap on outer corrections */
    int32_t use_graph;     /* capture the iteration in a CUDA graph and replay it */
    int32_t check_every;   /* iterations between host convergence checks (>= 1) */
    double rcond_min;      /* preconditioner validity threshold (e.g. 1e-3) */
    int32_t binned_only;   /* 1: return the binned map M^-1 b (no iterations) */
    int32_t true_residual; /* 1 computes ||b - A64 x||/||b|| at exit (one more application of the
                              FP64 operator); 0 skips it where it is not needed to continue
                              (true_rel_res = -1; FURAX_F32 then stops after its last inner solve) */
    void *d_ready;         /* cudaEvent_t recorded once d is written (e.g. after its host-to-device
                              copy on another stream), or NULL: the solver waits for it only before
                              it reads d, so the copy overlaps the preconditioner set-up */
    furax_allreduce_fn allreduce; /* NULL, or the detector-sharding sum: called on the
                              preconditioner blocks and hit counts before their inversion, the
                              right-hand side, every application of the normal operator (summed in
                              FP64) and the true residual's operator; all vectors, dot products
                              and scalars are then the same on every process. Disables graph
                              capture; not available with templates */
    void *allreduce_user;  /* passed to allreduce */
} furax_cg_opts;

typedef struct {
    int32_t iters;          /* PCG iterations performed (max over observations) */
    int32_t outer;          /* outer corrections performed (FURAX_F32) */
    double rel_res;         /* final recursive ||r||/||b|| (max over observations) */
    double true_rel_res;    /* final ||b - A64 x||/||b|| with the FP64 operator (max over observations) */
    int64_t n_valid;        /* number of solved pixels */
    double *hist;           /* host, caller-owned, [hist_len] recursive residual of observation 0
                               per iteration (entry 0 = 1), or NULL */
    int32_t hist_len;
    int32_t hist_written;   /* entries written to hist */
} furax_cg_result;

/* Fill `opts` with defaults: maxiter 50, tol 1e-8, FP64, ACC_F32, inner_tol 1e-5, max_outer 8,
 * graph on, check_every 10, rcond_min 1e-3, true_residual 1. */
void furax_cg_default_opts(furax_cg_opts *opts);

/* Solve (S P^T N^-1 P S^T) x = S P^T N^-1 d for every observation independently (per-observation
 * PCG scalars), x0 = 0, block-Jacobi preconditioner. x: device FP64 [npix_total][3], overwritten,
 * zero on unsolved pixels. valid (device uint8 [npix_total], may be NULL) receives the mask.
 * Allocates its workspace, synchronises `stream`, fills `res` (host). Returns FURAX_OK when every
 * observation reached tol, FURAX_ENOTCONVERGED when the iteration cap was hit first. */
furax_status furax_mapmaker_cg(const furax_pointing_t *p, const furax_noise_t *n, const void *d, int32_t d_t,
                               double *x, uint8_t *valid, const furax_cg_opts *opts, furax_cg_result *res,
                               void *stream);

/* ---------------------------------------------------------------------------------------
 * Template deprojection: the weighting-and-deprojection operator
 *   F_T = W - W T (T^T W T)^-1 T^T W
 * of the generalised least-squares estimator m = (P^T F_T P)^-1 P^T F_T d (Statement of Need;
 * TemplateOperator, Table 3). W = N^-1 of a noise handle. T, per detector: the Legendre
 * polynomials P_0 .. P_order (order <= 3) of the scaled time tau_t = 2t/(ns-1) - 1 over the
 * detector's whole stream (tau = 0 when ns = 1). F_T acts on each detector separately.
 * With P_0 among the templates, a constant I map is deprojected with the offsets: the I
 * monopole of the observed pixels is not constrained by the data.
 * ------------------------------------------------------------------------------------- */

/* Build the per-detector Gram matrices G = T^T W T (FP64, on the device) and their inverses.
 * p and n (same detectors and streams) are kept by reference and must outlive the handle.
 * Synchronises `stream`. FURAX_EINVAL: order outside [0, 3] or mismatched handles.
 * FURAX_EBADINPUT: a stream shorter than order + 1 samples, or a G that is not positive
 * definite (the message names the detector). */
furax_status furax_templates_create(const furax_pointing_t *p, const furax_noise_t *n, int32_t order, void *stream,
                                    furax_templates_t **out);
furax_status furax_templates_destroy(furax_templates_t *t);

/* gram: device FP64 [sum ndet][order+1][order+1] <- T^T W T per detector. */
furax_status furax_templates_gram(const furax_templates_t *t, double *gram, void *stream);

/* out = F_T in over the whole TOD (device, [nsamp_total] of dtype; in and out must not alias). */
furax_status furax_deproject_apply(const furax_templates_t *t, const void *in, void *out, int32_t dtype, void *stream);

/* out = S P^T F_T P S^T x: the deprojected normal operator (precision and acc as for
 * furax_ptnp_apply). x, out: device FP64 [npix_total][3]; valid: device uint8 or NULL. */
furax_status furax_ptfp_apply(const furax_templates_t *t, const double *x, double *out, const uint8_t *valid,
                              int32_t precision, int32_t acc, void *stream);

/* furax_mapmaker_cg for the deprojected system (S P^T F_T P S^T) x = S P^T F_T d (same options,
 * preconditioner, mask and result). amplitudes: device FP64 [sum ndet][order+1] receiving
 * G^-1 (W T)^T (d - P x) of the solved map, or NULL. */
furax_status furax_mapmaker_cg_deproject(const furax_templates_t *t, const void *d, int32_t d_t, double *x,
                                         uint8_t *valid, const furax_cg_opts *opts, furax_cg_result *res,
                                         double *amplitudes, void *stream);

/* ---------------------------------------------------------------------------------------
 * Gap filling by constrained Gaussian realisation (the use the paper gives the symmetric band
 * Toeplitz operator besides noise weighting; SymmetricBandToeplitzOperator, Table 2). The paper
 * does not state the construction; this is the standard conditional one: with N the noise
 * covariance, v the observed samples, g the gaps and n a realisation of covariance N,
 *   d_g <- n_g + N_gv N_vv^-1 (d_v - n_v),   d_v unchanged,
 * with N_vv^-1 applied by conjugate gradients for every detector at once.
 * ------------------------------------------------------------------------------------- */

/* cov: a banded noise handle whose taps hold the covariance band N (lags 0..ntaps-1, up to
 * 2048; bands above 64 taps use the overlap-save product). d, n_real, out: device
 * [nsamp_total] of dtype (out may be d); valid: device uint8 [nsamp_total], 1 = observed. n_real
 * is the unconstrained realisation (the caller's random draws). Per detector, CG from 0 until
 * ||r|| <= tol ||r_0|| or maxiter iterations; precision FURAX_F64 applies N in FP64, FURAX_F32 in
 * FP32 (vectors and scalars stay FP64; the filled values are then good to ~1e-7 relative),
 * FURAX_PREC_F32X2 FP64-accurate in double-FP32 on the FP32 units (bands of up to 64 taps; a
 * longer band is applied as for FURAX_F64);
 * iters_out: host int32 [sum ndet] or NULL. The first call allocates TOD-sized workspaces in the
 * handle (3 FP64, plus 1 FP64 for FURAX_F64 / FURAX_PREC_F32X2 or 2 FP32 for FURAX_F32) that later calls reuse and
 * furax_noise_destroy frees, so calls on one handle must not run concurrently; synchronises
 * stream. FURAX_ENOTCONVERGED when a detector stopped at maxiter (out is still written). */
furax_status furax_gapfill(const furax_noise_t *cov, const void *d, const uint8_t *valid, const void *n_real,
                           void *out, int32_t dtype, int32_t maxiter, double tol, int32_t precision,
                           int32_t *iters_out, void *stream);

/* ---------------------------------------------------------------------------------------
 * chi^2 and its gradients (differentiability, "Summary"; "Research Impact Statement").
 * ------------------------------------------------------------------------------------- */

/* r = d - P(delta) m; chi2 = r^T N^-1 r; grad_map = -2 P^T N^-1 r;
 * grad_psi[j] = -2 sum_t (N^-1 r)_{j,t} * 2 (U_p cos 2psi - Q_p sin 2psi) (offsets included).
 * d device [nsamp_total] of d_t; m device FP64 [npix_total][3]; chi2 device FP64 [n_obs]
 * (per observation); grad_map device FP64 [npix_total][3] or NULL; grad_psi device FP64
 * [sum ndet] or NULL. precision FURAX_F64: everything in FP64; FURAX_F32: residual, N^-1 and
 * each thread's partial sums in FP32, sums across threads and the map gradient in FP64;
 * FURAX_PREC_F32X2: FP64-accurate in double-FP32 on the FP32 units (residual, compensated band
 * product, partial sums), sums across threads and the map gradient in FP64. */
furax_status furax_chi2_grad(const furax_pointing_t *p, const furax_noise_t *n, const void *d, int32_t d_t,
                             const double *m, double *chi2, double *grad_map, double *grad_psi,
                             int32_t precision, void *stream);

/* ---------------------------------------------------------------------------------------
 * Diagnostics.
 * ------------------------------------------------------------------------------------- */

/* Synchronise `stream` and report whether any bounded device-side wait of this handle's kernels
 * gave up since the last check (FURAX_ETIMEOUT, and the error word is cleared) or not (FURAX_OK).
 * furax_mapmaker_cg checks this itself at its synchronisation points. */
furax_status furax_device_status(furax_pointing_t *p, void *stream);

/* Budget of every bounded device-side wait of this handle's pipelined kernels (the mbarrier
 * hand-offs between the roles of the cached FP32 operator), in SM clock cycles; 0 restores the
 * default of 2^32 cycles (about 2 s). A wait that runs out sets the error word that
 * furax_device_status reports (FURAX_ETIMEOUT) and its role leaves its loop, so the kernel
 * returns; the output of that launch is then incomplete. Ordered on `stream`; synchronises it.
 * Errors: FURAX_EINVAL for a NULL handle or a negative budget. The paper has no counterpart:
 * this is a property of the GPU pipeline. */
furax_status furax_set_wait_budget(furax_pointing_t *p, int64_t cycles, void *stream);

/* Test hook for the bounded waits: with hold != 0 the loader role of the cached FP32 operator
 * issues no copies in this handle's later launches, so the other roles' waits run out after the
 * wait budget (no copy is ever left in flight). hold = 0 restores normal operation. Ordered on
 * `stream`; synchronises it. The paper has no counterpart. */
furax_status furax_debug_hold_loader(furax_pointing_t *p, int32_t hold, void *stream);

/* ---------------------------------------------------------------------------------------
 * Device probes (measurement instruments; the paper has no counterpart). They give the
 * per-unit rates of this GPU that bound the kernels that are not HBM-bound, for their roofline
 * fractions, and check the encoding-level FP32/FP64 conversions against the hardware ones.
 * ------------------------------------------------------------------------------------- */

/* out32[i] = in64[i] rounded to binary32 (nearest even) and out64[i] = in32[i] widened, both by
 * the library's own encoding arithmetic (the conversions the gap-filling vector passes and the
 * FP64 accumulation of the double-FP32 path use). Either pair may be NULL. Device arrays of n
 * elements; asynchronous on `stream`. FURAX_EINVAL for n < 0 or an input without its output. */
furax_status furax_probe_convert(const double *in64, float *out32, const float *in32, double *out64, int64_t n,
                                 void *stream);

/* Launch one FMA throughput kernel (kind 0: FP64 FMA, 1: FP32 FMA, 2: packed FP32x2 FMA) that
 * issues `iters` iterations of 8 independent chains per thread on 8 x 256 threads per SM;
 * *flops receives the kernel's floating-point operation count (2 per FMA). The caller times the
 * launch on `stream` with events. sink: device scratch of one element (never written in
 * practice). FURAX_EINVAL for a bad kind, iters < 1 or NULL pointers. */
furax_status furax_probe_fma(int32_t kind, int64_t iters, void *sink, double *flops, void *stream);

/* Random L2 operations at the n device indices idx[i] (each in [0, ntable)): kind 0 gathers a
 * float4 from table (ntable float4), 1 issues one red.add.v4.f32 into it, 2 the compensated
 * pair of FURAX_ACC_F32_KAHAN (atomic add returning the old value + a reduction of its rounding
 * error into table[ntable + idx], so table holds 2 ntable float4), 3 three FP64 reductions
 * (table holds [ntable][3] doubles), 4 the same into 32-byte records ([ntable][4] doubles), 5 the
 * kind-3 reductions issued by three consecutive lanes of one instruction per index ([ntable][3]),
 * 6 kind 5 and 7 kind 0 with 8 operations per thread in flight (index loads first), 8 kind 5 with
 * 64-bit integer reductions (table: 3 ntable 64-bit words).
 * Grid of 8 x 256 threads per SM; the caller times it. The indices are not checked on the device.
 * sink: one float of device scratch. */
furax_status furax_probe_l2(int32_t kind, const int32_t *idx, int64_t n, void *table, int64_t ntable, void *sink,
                            void *stream);

/* Thread-local message describing the last error ("" if none). Never NULL. */
const char *furax_last_error(void);
/* Number of kernels this library has launched in this process (graph replays count their
 * kernel nodes). */
int64_t furax_launch_count(void);
/* Library version string. */
const char *furax_version(void);

/* Kernel timing: when enabled, the library brackets every launch of the fused P^T N^-1 P
 * kernels (FP32 and FP64) with CUDA events on the launching stream (also inside captured
 * graphs) and accumulates their durations, read at the solver's synchronisation points and
 * at furax_profile_read. kernel: 0 = FP32 fused apply, 1 = FP64 fused apply (incl. the FP64
 * right-hand side), 2 = double-FP32 fused apply (incl. its right-hand side). Writes the total milliseconds and the number of timed launches. */
void furax_profile_enable(int32_t on);
furax_status furax_profile_read(int32_t kernel, double *total_ms, int64_t *count);
void furax_profile_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* FURAX_H */
