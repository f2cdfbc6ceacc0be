/*
 * stab.h -- C ABI of the GB300 (sm_103a) video-stabilisation hot path of
 * "Real-Time Optical flow-based Video Stabilization for Unmanned Aerial
 * Vehicles" (Lim et al., arXiv 1701.03572).
 *
 * The path per frame (Sec. 3-5): Gaussian pyramid, Shi-Tomasi corners on a
 * reduced region of interest, pyramidal Lucas-Kanade tracking with a
 * forward-backward check, robust rigid / similarity fit, averaging-window
 * trajectory smoothing, bilinear compensating warp.  Every step runs in
 * hand-written CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *  - Images are uint8, row-major with a pitch in bytes; gray (1 channel) or
 *    interleaved RGB (3 channels).  Pixel (x, y) is column x, row y.
 *  - Points are float pairs (x, y) in pixel coordinates, packed xyxy...
 *  - A motion m = (tx, ty, theta, log s) is a similarity acting on centred
 *    coordinates p~ = p - ((w-1)/2, (h-1)/2): p~' = s R(theta) p~ + t.  The
 *    motion of frame t maps points of frame t-1 onto frame t (Eq. 7: src =
 *    previous frame, dst = current frame).
 *  - A warp matrix Minv = [a00 a01 b0 a10 a11 b1] maps an OUTPUT pixel p to the
 *    source position q = (a00 x + a01 y + b0, a10 x + a11 y + b1).
 *  - "_dev" pointers are device memory, "_host" pointers host memory (pinned
 *    for asynchronous copies).  The caller owns every buffer it passes; a
 *    context owns its internal buffers.  No entry point keeps a caller pointer
 *    after it returns, except where stated.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued asynchronously; argument errors are returned synchronously,
 *    device-side errors are latched in the context and returned by
 *    stab_sync().  A context or batch is not thread-safe.
 */
#ifndef STAB_H
#define STAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STAB_OK = 0,
    STAB_WARN_SKIPPED = 1,        /* too few tracks: identity motion (Sec. 4.1, skip rule) */
    STAB_ERR_INVALID_ARG = -1,
    STAB_ERR_CUDA = -2,
    STAB_ERR_OOM = -3,
    STAB_ERR_DEGENERATE = -4,
    STAB_ERR_TIMEOUT = -5,
    STAB_ERR_CAPACITY = -6        /* a device buffer would have overflowed */
} stab_status;

/* Sec. 4: rigid (3 DOF), similarity (4 DOF), or the hybrid mechanism of
 * Sec. 4.1 that fits both every `dwell` transitions and keeps the one with the
 * lower RMS distance for the next `dwell` transitions. */
typedef enum { STAB_RIGID = 0, STAB_SIMILARITY = 1, STAB_HYBRID = 2 } stab_model;
typedef enum { STAB_FP32 = 0, STAB_FP16_STORAGE = 1 } stab_precision;  /* storage of I, Ix, Iy planes */

/* Flag bits of stab_motion.flags */
#define STAB_FLAG_SKIPPED 1       /* fewer than min_fit pairs or no valid hypothesis */
#define STAB_FLAG_DETECTED 2      /* corners were re-detected on the previous frame */
#define STAB_FLAG_RIGID 4         /* the motion was fitted with the rigid model */
#define STAB_FLAG_DECISION 8      /* hybrid mechanism: a decision transition ((t - 1) % dwell == 0) */

typedef struct {
    int max_corners;      /* K: corners kept per detection (Sec. 3.1 fixes a count; <= 2048) */
    int levels;           /* pyramid levels (Sec. 3.2; 1..8) */
    int win_radius;       /* LK window (2r+1)^2 (r = 10: 21x21; 1..12) */
    int max_iters;        /* LK iterations per level */
    float eps;            /* LK stop when |eta| < eps (px); 0 = always max_iters */
    float min_eig;        /* lost if min eigenvalue of G / window area < min_eig */
    float quality;        /* corner threshold: q * max response (0.01) */
    int roi_margin_x;     /* reduced ROI (Sec. 3.1); -1 = max(w/10, r+2) */
    int roi_margin_y;     /* -1 = max(h/10, r+2) */
    int redetect_period;  /* detect on frame t-1 when (t-1 + redetect_phase) % period == 0
                             (Sec. 3.2: 5) */
    int min_tracks;       /* also re-detect when fewer live tracks */
    float fb_thresh;      /* forward-backward round-trip limit (px) */
    float inlier_thresh;  /* robust fit inlier radius (px) */
    int hypotheses;       /* sampled two-point hypotheses per frame */
    uint64_t seed;        /* hypothesis sampling seed (SplitMix64 counter hash) */
    int min_fit;          /* skip rule: fewer pairs => identity (Sec. 4.1) */
    int smooth_window;    /* averaging window W (Sec. 5.1; 1..63) */
    int model;            /* stab_model */
    int precision;        /* stab_precision */
    int dwell;            /* hybrid mechanism: transitions between decisions (Sec. 4.1: 20) */
    float crop_zoom;      /* composition crop (Sec. 5.1): output = centre region of the warped
                             frame magnified by crop_zoom about the image centre; 1 = no crop,
                             range [1, 4] */
    int redetect_phase;   /* place of the stream in its detection cycle, 0 .. period-1: besides
                             the first transition, detect on frame t-1 when
                             (t-1 + phase) % period == 0.  Streams of a batch with different
                             phases spread their detection frames over the cycle (default 0) */
} stab_params;

typedef struct {
    float tx, ty, theta, log_scale;  /* motion of this frame (centred coordinates) */
    int inliers;                     /* inliers of the refit */
    int n_tracks;                    /* pairs that passed the forward-backward check */
    float rms;                       /* RMS residual of the refit over its inliers (px) */
    int flags;                       /* STAB_FLAG_* */
    float e_rigid;                   /* RMS of the rigid fit made at this transition (px), -1 if none */
    float e_similarity;              /* RMS of the similarity fit made at this transition, -1 if none */
} stab_motion;

/* Result of the 6-DOF affine fit (Eq. 7-8): dst = A src + t in centred
 * coordinates (pixel minus ((w-1)/2, (h-1)/2)), A = [a00 a01; a10 a11]. */
typedef struct {
    float a00, a01, a10, a11, tx, ty;
    int inliers;                     /* inliers of the refit */
    int n_tracks;                    /* pairs given */
    float rms;                       /* RMS residual of the refit over its inliers (px) */
    int flags;                       /* STAB_FLAG_SKIPPED when no fit: identity */
} stab_affine;

typedef struct stab_ctx stab_ctx;
typedef struct stab_batch stab_batch;

/* Library version string. */
const char *stab_version(void);

/* Default parameters: K = 200, 3 levels, r = 10, 30 iterations, eps = 0.01,
 * min_eig = 0.01, q = 0.01, auto ROI, period 5, min_tracks 10, fb 1 px,
 * inliers 1 px, 100 hypotheses, seed 0, min_fit 10, W = 15, similarity, FP32. */
stab_status stab_default_params(stab_params *out);

/* Create a single-stream context for w x h frames (w, h in [16, 8192]).
 * Allocates all device buffers on the current device.  *out is NULL on error. */
stab_status stab_create(int w, int h, const stab_params *p, stab_ctx **out);
void stab_destroy(stab_ctx *ctx);

/* Drain the context's last stream; return the latched device error status
 * (STAB_OK if none) and clear it. */
stab_status stab_sync(stab_ctx *ctx);
/* Text of the last error of this context ("" if none).  Owned by ctx. */
const char *stab_last_error(const stab_ctx *ctx);

/* Gaussian pyramid of one frame (Sec. 3.2, Burt-Adelson REDUCE with
 * [1 4 6 4 1]/16, reflect-101 border, round half up).  channels = 1 or 3 (RGB
 * is converted to luma first: (77R + 150G + 29B + 128) >> 8).  Writes the
 * levels packed one after another (level l is w_l * h_l bytes, w_l =
 * (w_{l-1}+1)/2) into levels_out_dev.  Test hook; also fills the context's
 * pyramid slot 0. */
stab_status stab_pyramid(stab_ctx *ctx, const uint8_t *frame_dev, int pitch, int channels,
                         uint8_t *levels_out_dev, void *stream);

/* Copy the I, Ix, Iy planes of pyramid level `level` of the frame last passed
 * to stab_pyramid, as float32 (w_l * h_l each; NULL to skip).  Ix = (I(x+1) -
 * I(x-1)) / 2 with replicated borders, likewise Iy.  Test hook. */
stab_status stab_planes(stab_ctx *ctx, int level, float *I_dev, float *Ix_dev, float *Iy_dev, void *stream);

/* Shi-Tomasi corners (Sec. 3.1, Eq. 2) on the ROI of a gray frame: response
 * min(lambda1, lambda2) of the Sobel structure tensor summed over 3x3, 3x3
 * non-maximum suppression, threshold q * max, strongest max_corners first
 * (ties: lower raster index).  Writes pts_dev (2 * max_corners floats),
 * optional lam_dev (max_corners scores), n_dev (count), optional
 * ncand_dev (NMS survivors above the threshold, before the top-K cut).
 * Counts are device ints.  Also replaces the context's feature set. */
stab_status stab_detect(stab_ctx *ctx, const uint8_t *gray_dev, int pitch, float *pts_dev, float *lam_dev,
                        int *n_dev, int *ncand_dev, void *stream);

/* Corner detection that allocates nothing, for callers that cannot call
 * cudaMalloc: code whose device memory belongs to a host application's own
 * pool allocator, or a real-time loop that must not call cudaMalloc / cudaFree
 * (they can synchronise the device and stall the frame cadence).  The paper has
 * no counterpart; this is a deployment variant of stab_detect.
 * Same result as stab_detect for the same frame, ROI [roi_x0, roi_x1) x
 * [roi_y0, roi_y1) (at least 3 px from every border), quality and
 * max_corners, without a context: all scratch lives in one fixed device array
 * of about 5.4 MB inside the library, held by every GPU that loads it until
 * the process exits.  Limits: ROI at most 1536 x 864 pixels, max_corners at
 * most 2048; larger requests return STAB_ERR_CAPACITY (with a message on
 * stderr).  The caller passes the gray frame and the outputs (as for
 * stab_detect).  The first call on a device looks up the array's device
 * address; make that first call before any stream capture.  Every call
 * shares the one array: calls whose work overlaps on the GPU (different
 * streams, different host threads) race and must be serialised by the
 * caller. */
stab_status stab_detect_noalloc(const uint8_t *gray_dev, int w, int h, int pitch, int roi_x0, int roi_y0,
                                int roi_x1, int roi_y1, float quality, int max_corners, float *pts_dev,
                                float *lam_dev, int *n_dev, int *ncand_dev, void *stream);

/* Pyramidal Lucas-Kanade (Sec. 3.2, Eq. 3-6) of n given points from frame
 * `prev` to frame `next` (gray, same size as the context), followed by the
 * backward pass of the forward-backward check (Sec. 4.1).  Outputs (n each):
 * fwd_dev (2n floats), back_dev (2n), fb_dev (round-trip error, -1 if the
 * forward pass failed), status_dev (1 = kept), status_fwd_dev (1 = forward
 * pass tracked; may be NULL).  n <= max_corners.  Test hook of the tracker. */
stab_status stab_lk(stab_ctx *ctx, const uint8_t *prev_dev, const uint8_t *next_dev, int pitch,
                    const float *pts_dev, int n, float *fwd_dev, float *back_dev, float *fb_dev,
                    uint8_t *status_dev, uint8_t *status_fwd_dev, void *stream);

#define STAB_TRACK_CONTINUE 1  /* prev is the frame given as next on the previous call */

/* Motion-estimation front end for one frame pair (Sec. 3.2 and Fig. of
 * Sec. 4.1): pyramids of prev (rebuilt unless STAB_TRACK_CONTINUE) and next;
 * corners re-detected on prev when due (no features yet, the frame index is
 * a multiple of redetect_period, or fewer than min_tracks live tracks); the
 * context's features tracked forward and backward; the kept pairs compacted
 * in their original order into pts_prev_dev / pts_next_dev (capacity
 * max_corners each) with their count in *n_dev (device int); status_dev
 * (max_corners bytes, may be NULL) holds the per-feature result.  The kept
 * next points become the context's features (Sec. 3.2: next points are
 * passed as previous points).  The frame index advances by one. */
stab_status stab_track(stab_ctx *ctx, const uint8_t *prev_dev, const uint8_t *next_dev, int pitch, int channels,
                       int flags, float *pts_prev_dev, float *pts_next_dev, uint8_t *status_dev, int *n_dev,
                       void *stream);

/* Robust fit of the frame motion (Sec. 4, Eq. 7 with 3 or 4 DOF): `hypotheses`
 * two-point samples (pair of hypothesis h drawn by SplitMix64 from seed, t, h)
 * scored by inlier count (residual < inlier_thresh, FP32), the first best
 * kept, then the closed-form least-squares similarity (or rotation for
 * rigid) on its inliers.  src/dst: device points, count from *n_dev (device).
 * Fewer than min_fit pairs => identity with STAB_FLAG_SKIPPED.  Writes one
 * stab_motion to out_dev (device).  model STAB_HYBRID (Sec. 4.1): when
 * (t - 1) % dwell == 0 both models are fitted and the rigid one is chosen iff
 * both fits succeed and its RMS over its own inliers is strictly lower (only
 * one fit succeeding chooses that one; none keeps the current choice, which
 * starts as similarity); the choice is kept in the context and used alone on
 * the other transitions. */
stab_status stab_fit(stab_ctx *ctx, const float *src_dev, const float *dst_dev, const int *n_dev, int model,
                     int t, stab_motion *out_dev, void *stream);

/* Robust 6-DOF affine fit (Eq. 7-8: [A|t] minimising the squared distances
 * of the inliers; three non-degenerate pairs determine it): `hypotheses`
 * three-point samples (hypothesis h: the pair sample of h plus a third index
 * k = r2 mod (n-2) stepped past the two, r2 the SplitMix64 value of
 * (seed ^ t << 32 ^ h << 8) ^ 2), each solved exactly in a fixed FP32 order
 * (degenerate when twice the triangle area is below 1 px^2) and scored by
 * inlier count (residual < inlier_thresh); the first best is refitted by the
 * closed-form least squares of Eq. 7 on its inliers.  src/dst: device points,
 * count from *n_dev (device); fewer than max(3, min_fit) pairs, no valid
 * sample or collinear inliers => identity with STAB_FLAG_SKIPPED.  Writes one
 * stab_affine to out_dev (device). */
stab_status stab_fit_affine(stab_ctx *ctx, const float *src_dev, const float *dst_dev, const int *n_dev, int t,
                            stab_affine *out_dev, void *stream);

/* Offline averaging-window smoothing (Sec. 5.1) of T motions (frame 0's
 * motion must be the identity): C_t = sum_{k<=t} m_k, S_t = mean of C over
 * [t - (W-1)/2, t + W/2] clipped to [0, T-1], m'_t = m_t + S_t - C_t.
 * Writes mprime_dev (T x 4 floats) and Minv_dev (T x 6: the inverse warp of
 * m'_t composed with the crop zoom z of the context's parameters, i.e. output
 * pixel p samples the compensated frame at c + (p - c) / z; frame t-1 is
 * composed with Minv_t). */
stab_status stab_smooth(stab_ctx *ctx, const stab_motion *motions_dev, int T, int window, float *mprime_dev,
                        float *Minv_dev, void *stream);

/* Streaming form of the same smoothing (the GPU analogue of the paper's
 * motion-compensation thread, Sec. 6): push the motion of frame t (t = number
 * of previous pushes + 1; the first push is frame 1).  When frame
 * u = t - 1 - W/2 >= 0 is ready, writes its inverse warp (6 floats) to
 * Minv_dev and sets *ready_dev = u, else *ready_dev = -1. */
stab_status stab_smooth_push(stab_ctx *ctx, const stab_motion *motion_dev, float *Minv_dev, int *ready_dev,
                             void *stream);

/* Compensating warp (Sec. 5.1): out(p) = bilinear(src, Minv p), taps outside
 * the image read 0, rounded half up; channels 1 or 3 interleaved; frame size
 * of the context.  Minv_dev: 6 floats in device memory. */
stab_status stab_warp(stab_ctx *ctx, const uint8_t *src_dev, int src_pitch, uint8_t *dst_dev, int dst_pitch,
                      int channels, const float *Minv_dev, void *stream);

/* ---------------------------------------------------------------------- */
/* Batched multi-stream pipeline (one CUDA-graph launch per frame step).
 * Stream i has its own size, channel count and parameters.  The step that
 * takes frame t of every stream from its input ring slot (t % ring) builds
 * frame t's pyramid and, as parallel branches of the same graph, tracks the
 * previous transition (frames t-2 -> t-1: detection when due, tracker, fit,
 * smoothing) and composes the frame whose smoothed map the previous step
 * produced, writing the stabilised frame u = t - 3 - W_i/2 of stream i to its
 * output buffer (when u >= 0).  The motions it reports are those of the
 * transition t-1; the results equal those of the single-stream calls. */
typedef struct {
    int w, h, channels;
    stab_params params;
} stab_stream_desc;

/* ring >= W/2 + 4 frames per stream (0 = that minimum); with ring >= W/2 + 5
 * the input copies of stab_batch_step_host run two steps ahead. */
stab_status stab_batch_create(int n, const stab_stream_desc *descs, int ring, stab_batch **out);
void stab_batch_destroy(stab_batch *b);
/* Device pointer of input slot `slot` of stream i (w * channels bytes per
 * row, pitch from stab_batch_pitch) and of its output frame buffer. */
uint8_t *stab_batch_input(stab_batch *b, int i, int slot);
uint8_t *stab_batch_output(stab_batch *b, int i);
int stab_batch_pitch(const stab_batch *b, int i);
int stab_batch_ring(const stab_batch *b);
/* Index t of the next step (frames already stepped). */
int64_t stab_batch_frame(const stab_batch *b);
/* Run one step on `stream` (frame t must already be in slot t % ring).
 * use_graph = 1: the step is captured once into a CUDA graph and replayed. */
stab_status stab_batch_step(stab_batch *b, int use_graph, void *stream);
/* End-to-end step with host buffers: copy frames_host[i] (pinned, pitch
 * w * channels) into the ring, step, and copy each stream's output into
 * out_host[i] (pinned; NULL to skip).  Returns after enqueuing; the caller
 * synchronises `stream` before reading out_host. */
stab_status stab_batch_step_host(stab_batch *b, const uint8_t *const *frames_host, uint8_t *const *out_host,
                                 void *stream);
/* Autotuner of the batched step: times each variant of the tracker kernel
 * (one or two warps per feature, register budgets) on the batch's current
 * state with CUDA events and keeps the fastest for later steps.  cache_path
 * (may be NULL) names a JSON file of earlier choices keyed by GPU name and
 * batch shape; a cached choice is applied without timing and new choices are
 * added to it.  Needs at least three steps run (the tracker has features from
 * the third); synchronous on `stream`.
 * *variant (may be NULL) receives the choice; ms_out (may be NULL, one float
 * per variant: stab_lk_variants() floats) the measured mean ms per launch (-1
 * when taken from the cache). */
stab_status stab_batch_autotune(stab_batch *b, const char *cache_path, int *variant, float *ms_out, void *stream);
/* Bound the candidate list of corner detection (the NMS survivors kept
 * before the top-K selection, Sec. 3.1) of every stream of a context or batch
 * to `cap` keys; cap = 0 restores the capacity sized at creation (every
 * possible survivor of the ROI), larger values are clipped to it.  A
 * detection with more survivors keeps `cap` of them (its corner list is then
 * not the exact top K) and latches STAB_ERR_CAPACITY in the device error word,
 * which the next stab_sync / stab_batch_sync returns and clears.  For callers
 * that bound the scratch a detection may fill, and the test hook of the
 * latched-error path.  Synchronous: waits for the context's last stream. */
stab_status stab_set_candidate_capacity(stab_ctx *ctx, int cap);
stab_status stab_batch_set_candidate_capacity(stab_batch *b, int cap);
/* Force a tracker variant (0..8) for a batch or a single-stream context:
 * 0 / 1: one warp per feature, template in registers, register budgets of
 * 128 / 168; 2 / 3: two warps per feature, budgets of 80 / 128; 4: one warp
 * per feature, template in shared memory, budget of 96 (more resident warps);
 * 5 / 6: two features per warp (a half-warp each), budgets of 255 / 168;
 * 7 / 8: as 0 / 1, with patches inside their pyramid level copied by tensor
 * (TMA) copies.  Variants 0, 1, 4, 7 and 8 give identical results; the others
 * sum the window in another order (FP32 rounding differences only).
 * Variants other than 0 serve the 21 x 21 window; other windows run
 * variant 0. */
stab_status stab_batch_set_lk_variant(stab_batch *b, int variant);
stab_status stab_set_lk_variant(stab_ctx *ctx, int variant);
/* Number of tracker variants (the size stab_batch_autotune's ms_out must have). */
int stab_lk_variants(void);
/* Copy the motions of the last step (n entries) to host memory (synchronous). */
stab_status stab_batch_motions(stab_batch *b, stab_motion *out_host);
/* Copy stream i's current feature set (2 * max_corners floats) and its count. */
stab_status stab_batch_features(stab_batch *b, int i, float *pts_host, int *n_host);
stab_status stab_batch_sync(stab_batch *b);
/* Measurement hooks (not used on the production path).  Run one step without
 * a graph, with a CUDA event pair around each kernel, synchronise, and write
 * each kernel's duration in ms to ms[0 .. min(n_ms, *n_kernels) - 1]; the
 * kernels' names are returned by stab_batch_kernel_name (valid until the next
 * profiled step). */
stab_status stab_batch_step_profiled(stab_batch *b, void *stream, float *ms, int n_ms, int *n_kernels);
const char *stab_batch_kernel_name(const stab_batch *b, int i);
/* Work done by the tracker in the last step, summed over streams: LK
 * iterations and template passes (one per feature, level and direction).
 * Synchronous. */
stab_status stab_batch_lk_work(stab_batch *b, int64_t *iterations, int64_t *templates);
const char *stab_batch_last_error(const stab_batch *b);

/* ---------------------------------------------------------------------- */
/* Photometric refinement (direct Gauss-Newton on the warp of Sec. 5.1 with the
 * model of Sec. 4): for P frame pairs (I_t, I_prev), FP32 w x h planes
 * (contiguous, pair p at offset p*w*h), parameters theta (P x 4 floats):
 *   L_p = sum_{x in Omega} sqrt(r^2 + eps^2), r = I_t(W(x; theta_p)) - I_prev(x),
 *   W(x) = c + s R(th) (x - c) + t, Omega = [margin, w-margin) x [margin, h-margin).
 * I_t is read bilinearly (zero outside).  Outputs (device; NULL to skip):
 *   loss_dev (P), dtheta_dev (P x 4) = dL/dtheta,
 *   gn_dev (P x 14) = IRLS Gauss-Newton system: 10 entries of the upper
 *   triangle of H = sum w J^T J (row-major a<=b) then g = sum w J^T r (4),
 *   w = 1 / sqrt(r^2 + eps^2).
 * Deterministic: fixed-order reductions. */
stab_status stab_charb_forward(const float *It_dev, const float *Ip_dev, int w, int h, int P, const float *theta_dev,
                               int margin, float eps, float *loss_dev, float *dtheta_dev, float *gn_dev,
                               void *stream);
/* dL/dI_t (P x w x h) and dL/dI_prev (may be NULL) of the same objective,
 * scaled by gout (P floats, device; NULL = ones).  dL/dI_t is computed as a
 * gather over the output pixels that sample each input pixel (deterministic). */
stab_status stab_charb_backward_image(const float *It_dev, const float *Ip_dev, int w, int h, int P,
                                      const float *theta_dev, int margin, float eps, const float *gout_dev,
                                      float *dIt_dev, float *dIp_dev, void *stream);
/* `steps` Gauss-Newton updates theta <- theta - H^-1 g in place (P x 4). */
stab_status stab_charb_gauss_newton(const float *It_dev, const float *Ip_dev, int w, int h, int P, float *theta_dev,
                                    int margin, float eps, int steps, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* STAB_H */
