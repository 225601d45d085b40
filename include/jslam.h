/*
 * jslam.h -- C ABI of libjslam, a GB300 (sm_103a) implementation of the
 * stereo frontend hot path of "High-Speed Stereo Visual SLAM for
 * Low-Powered Computing Devices" (Jetson-SLAM, arXiv 2410.04090).
 *
 * For both images of each rectified stereo pair the library builds the
 * image pyramid (Sec. III, streamlined multiscale detection), detects FAST
 * corners with Bounded Rectification (Sec. II-A, Eq. 1-3), culls them per
 * grid cell (Sec. II-C-1, Feature Culling) and aggregates the survivors
 * across levels (Sec. II-C-2, Pyramidal Feature Aggregation), computes the
 * intensity-centroid orientation and a 256-bit steered BRIEF descriptor of
 * every keypoint (Sec. III, ORB extraction for all scales at once), and
 * matches left keypoints to right keypoints along image rows by descriptor
 * distance (Sec. III, middle-end stereo matching).
 *
 * Conventions shared by every entry point:
 *  - Status codes only; nothing is thrown across the ABI.  A CUDA error is
 *    reported as JSLAM_ERR_CUDA and is sticky: the context refuses further
 *    work until it is destroyed.
 *  - All work is enqueued on the context's stream and is asynchronous.
 *    Counts and device-side error flags are valid after jslam_sync().
 *  - Images passed as device memory are owned by the caller and must stay
 *    valid until jslam_sync() returns.  Output views point into memory owned
 *    by the context; they stay valid until the next jslam_extract*,
 *    jslam_match or jslam_destroy on that context.
 *  - Device buffers only grow: a call that needs more than the context holds
 *    reallocates once; later calls of the same or smaller size reuse it (the
 *    paper's Synchronized Shared Memory, Sec. III).
 *  - One context per host thread.  A context drives one device.
 *  - Keypoints of one image are in canonical order: level ascending, then
 *    y ascending, then x ascending (level coordinates).
 */
#ifndef JSLAM_H
#define JSLAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JSLAM_OK = 0,
    JSLAM_ERR_ARG = -1,      /* invalid argument (null pointer, size, parameter range) */
    JSLAM_ERR_CUDA = -2,     /* a CUDA runtime call failed; the context is unusable */
    JSLAM_ERR_NOMEM = -3,    /* device or pinned host allocation failed */
    JSLAM_ERR_CAPACITY = -4, /* request exceeds a limit fixed at jslam_create */
    JSLAM_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up */
    JSLAM_ERR_STATE = -6     /* call out of order (e.g. match before extract) */
} jslam_status;

/* Opaque context: device buffers, tables, stream and sticky status. */
typedef struct jslam_ctx jslam_ctx;

/* Where the bytes of a jslam_image live. */
enum { JSLAM_MEM_DEVICE = 0, JSLAM_MEM_HOST = 1 };

/* One 8-bit grayscale image, row-major with `pitch` bytes between rows
 * (pitch >= width, and pitch x height below 4 GiB: the kernels address an
 * image with 32-bit offsets; larger spans are refused with JSLAM_ERR_ARG).
 * memory == JSLAM_MEM_DEVICE: `data` is device memory of the context's
 *   device and is read in place.
 * memory == JSLAM_MEM_HOST: `data` is host memory (pinned memory makes the
 *   copy asynchronous); the library copies it into its own device staging
 *   buffer on the context stream.  Host images of one call that lie back to
 *   back in host memory (image k + 1 starting at data_k + pitch_k x
 *   height_k, in the order left 0, right 0, left 1, ...) with pitch <= width
 *   rounded up to 128 are copied with a single transfer; keeping a step's
 *   frames in one pinned buffer therefore makes the upload one copy. */
typedef struct {
    int32_t width, height, pitch;
    int32_t memory;
    const uint8_t *data;
} jslam_image;

/* Context configuration.  Fields marked (paper) take the paper's values by
 * default; the others are readings of points the paper leaves open. */
typedef struct {
    int32_t device;          /* CUDA device ordinal */
    void *cuda_stream;       /* cudaStream_t to enqueue on; NULL: the context creates one */
    int32_t max_width;       /* largest image width accepted (<= 4096) */
    int32_t max_height;      /* largest image height accepted (<= 4096) */
    int32_t max_levels;      /* largest pyramid depth accepted (<= 8) */
    int32_t max_feats;       /* largest keypoint cap accepted per image */
    int32_t max_pairs;       /* largest batch accepted by jslam_extract_batch */
    int32_t fast_thresh_lo;  /* fallback FAST threshold for cells with no corner; <= 0: off */
    int32_t p_min, p_max;    /* (paper) bounds of Eq. 3: 9 and 13 */
    int32_t k_per_cell;      /* corners kept per culling cell: 1..8 (paper: 1) */
    int32_t nms_q;           /* (paper) PFA NMS window: odd, 1..7, default 3 */
    int32_t border;          /* pixels skipped at each level edge, >= 16 (default 19) */
    int32_t max_disp;        /* stereo search range in s0 pixels (default 128) */
    int32_t row_band_px;     /* stereo row band at s0, scaled by zeta^n (default 2) */
    int32_t match_max_dist;  /* Hamming distance accepted as a match (default 100) */
    int32_t pfa_rule;        /* 0: suppress when a neighbour has larger K_l AND K_r; 1: lexicographic */
    int32_t response_mode;   /* corner response: 0 the sum of |I_p - I_c| over all 16 ring pixels (default);
                              * 1 the arc reading: for each polarity whose longest run satisfies Eq. 3, the
                              * sum of (|I_p - I_c| - eps) over the pixels of its longest run, the larger of
                              * the two (with the fallback threshold for fallback corners) */
    int32_t pyramid_mode;    /* 0: every level resampled from level 0 by zeta^n (default); 1: cascaded, level
                              * n resampled from level n - 1 by zeta (one launch per level) */
} jslam_config;

/* One stereo pair of a batch; the per-pair parameters of jslam_extract. */
typedef struct {
    jslam_image left, right;
    int32_t levels;          /* pyramid depth, 1..max_levels */
    float scale;             /* scale factor zeta between levels, > 1 (paper: 1.2) */
    int32_t fast_thresh;     /* epsilon of Eq. 1, 1..254 (paper: 20) */
    int32_t cell;            /* culling cell size at s0, 1..128 (paper: 32) */
    int32_t max_feats;       /* keypoint cap per image, 1..config.max_feats */
} jslam_stereo_job;

/* Device views of one image's keypoints (arrays of `capacity` entries; the
 * first `count` are valid).  `count` is -1 until jslam_sync() has run. */
typedef struct {
    int32_t count;
    int32_t capacity;
    const uint16_t *x, *y;        /* level coordinates */
    const uint16_t *X, *Y;        /* projection to the native scale s0 */
    const uint8_t *level;         /* pyramid level */
    const uint8_t *angle_bin;     /* orientation sector 0..29 (12 degrees each) */
    const uint16_t *response;     /* FAST response: sum of |I_p - I_c| over the ring */
    const uint8_t *k_levels;      /* PFA K_l: levels detecting this s0 pixel */
    const uint32_t *k_resp;       /* PFA K_r: summed response at this s0 pixel */
    const float *angle;           /* intensity-centroid angle, radians, (-pi, pi] */
    const uint32_t *desc;         /* capacity x 8 words; bit i of pair i in word i/32 */
} jslam_keypoints;

/* Device views of one pair's stereo matches, one entry per left keypoint. */
typedef struct {
    int32_t count;                /* == left keypoint count; -1 until jslam_sync() */
    const int32_t *right_idx;     /* canonical index of the right keypoint, -1 if none */
    const int16_t *disparity;     /* X_left - X_right in s0 pixels (0 if none) */
    const uint16_t *dist;         /* Hamming distance of the best candidate (65535: no candidate) */
} jslam_matches;

/* Correlation minimisation (Sec. III, middle-end stereo matching; the
 * paper names the step and gives no detail, so this is the sub-pixel
 * refinement of the stereo SLAM system it builds on, restated).  For every
 * left keypoint of every pair of the last jslam_match with an accepted
 * match j, on the left keypoint's level n (s = zeta^n) of both raw pyramids:
 * xr0 = floor(X_j / s + 0.5); SAD(t) = sum over the (2w+1)^2 window of
 * |(left - its centre) - (right shifted by t - its centre)| for t = -L..L;
 * t* = the first minimum; rejected when a window leaves the level, t* is
 * -L or L, the minimum is flat, the parabola offset delta = (d1 - d3) /
 * (2 (d1 + d3 - 2 d2)) exceeds 1 in size, or the disparity s (x - xr0 - t*
 * - delta) leaves [0, max_disp]; depth = bf / max(disparity, 0.01) when bf
 * > 0.  Then matches whose SAD is above 2.1 times the pair's median SAD
 * (of the surviving matches) are rejected.  Enqueued on the context stream
 * after jslam_match; results in jslam_get_refined / the result block.
 * JSLAM_ERR_ARG unless 1 <= half_window <= 10, 1 <= search <= 7, bf >= 0;
 * JSLAM_ERR_STATE before jslam_match. */
jslam_status jslam_refine_matches(jslam_ctx *ctx, int32_t half_window, int32_t search, float bf);

/* Feature tracking by projection (Sec. III, middle-end feature tracking;
 * the paper gives no detail, so this is a restatement of the usual search
 * by projection).  The caller projects its map points (or the previous
 * frame's keypoints) into the frame with its own pose or motion model; for
 * each of the n queries (device arrays: predicted s0 position u, v, predicted
 * level, 8-word descriptor) the kernel searches the keypoints of `side` of
 * pair `pair` of the last extraction at levels level-1..level+1 inside the
 * square window |X - u| <= r, |Y - v| <= r with r = radius * zeta^level
 * (window test in IEEE float), and keeps the smallest (Hamming distance,
 * index).  It is accepted when its distance is <= max_dist and, when
 * another candidate exists, 10 best <= 9 second (ratio 0.9 against the
 * second-smallest distance).  Writes out_idx (canonical keypoint index, -1
 * none or rejected) and out_dist (best distance, 0xFFFF: no candidate),
 * caller-owned device arrays of n entries.  The band is clipped to the
 * frame's levels, so a query one level past the deepest meets that level and
 * deeper queries meet none.
 * Enqueued on the context stream.  JSLAM_ERR_ARG for bad sizes, pointers,
 * radius (< 0) or max_dist (outside 0..256); JSLAM_ERR_STATE before an
 * extraction; n == 0 returns JSLAM_OK. */
jslam_status jslam_track(jslam_ctx *ctx, int32_t pair, int32_t side, const float *u, const float *v,
                         const uint8_t *level, const uint32_t *desc, int32_t n, float radius, int32_t max_dist,
                         int32_t *out_idx, uint16_t *out_dist);

/* Feature Culling the paper's way, kept as an ablation baseline (Sec.
 * II-C-1; no counterpart in the exact path, which culls inside detection
 * without a CRF-matrix): for the last extraction, writes the CRF-matrix of
 * every level (response of primary-threshold corners, 0 elsewhere) to
 * device memory, then culls it per cell with Multi-Location-Per-Thread
 * passes under Thread-Efficient Warp Allocation (blocks 128 threads wide
 * holding whole cells, N_t = ceil(c / n_max) threads tall).  Each cell's
 * result is the key response << 16 | (0xFFFF - index in cell) of its
 * strongest corner (0: none) -- with the fallback threshold off, the same
 * keys the fused detection kernel produced.  Enqueued on the context
 * stream, timed by its own events.  JSLAM_ERR_ARG when k_per_cell != 1,
 * n_max < 1 or ceil(c / n_max) > 8 at some level; JSLAM_ERR_STATE before an
 * extraction. */
jslam_status jslam_fc_ablation(jslam_ctx *ctx, int32_t n_max);

/* Device views of one level's per-cell keys (cells_y x cells_x, row-major)
 * from the ablation and from the fused detection kernel: each cell's
 * Feature Culling result (Sec. II-C-1), computed both ways. */
jslam_status jslam_fc_ablation_view(jslam_ctx *ctx, int32_t pair, int32_t side, int32_t level,
                                    const uint32_t **ablation_keys, const uint32_t **fused_keys,
                                    int32_t *cells_x, int32_t *cells_y);

/* Failure-detection self-test (no counterpart in the paper): enqueues one
 * kernel whose bounded wait -- on an mbarrier that nothing arrives on, the
 * wait the detection kernels use for their tile loads -- runs out after
 * about a second and sets the context's timeout flag.  The next jslam_sync()
 * returns JSLAM_ERR_TIMEOUT, and the context keeps that status (create a new
 * one to continue); the device itself stays usable.  JSLAM_ERR_ARG for a
 * null context; the context's own status if it already failed. */
jslam_status jslam_selftest_wait(jslam_ctx *ctx);

/* Device view of one level's CRF-matrix from the last jslam_fc_ablation()
 * (Sec. II-C-1: the corner response of every pixel before culling): Eq. 1-3
 * at the image's primary threshold with the context's P_min, P_max, the
 * SAD response of every corner and 0 for every other pixel and inside the
 * border; height x width uint16, row-major, no padding, ctx-owned and valid
 * until the next extraction or ablation.  The repeatability study of
 * Bounded Rectification reads its corner sets here.  JSLAM_ERR_STATE before
 * an ablation; JSLAM_ERR_ARG for a pair, side or level outside the last
 * batch or a null output. */
jslam_status jslam_crf_view(jslam_ctx *ctx, int32_t pair, int32_t side, int32_t level, const uint16_t **crf,
                            int32_t *width, int32_t *height);

/* Milliseconds of the ablation's CRF-matrix kernel and of its culling
 * kernels (after jslam_sync); the per-stage kernel times the paper reports
 * for Feature Culling (Sec. IV-B) are measured this way. */
jslam_status jslam_fc_ablation_times(jslam_ctx *ctx, float *crf_ms, float *fc_ms);

/* Views of one pair's refinement, one entry per left keypoint. */
typedef struct {
    int32_t count;                /* == left keypoint count; -1 until jslam_sync() */
    const float *disparity;       /* sub-pixel disparity in s0 pixels, -1 when rejected or unmatched */
    const float *depth;           /* bf / disparity, 0 when rejected (or bf == 0) */
    const uint32_t *sad;          /* SAD at the best shift; 0xFFFFFFFF when none was computed */
} jslam_refined;

/* Device views of pair `pair`'s refinement (after jslam_refine_matches):
 * the correlation-minimisation outputs of the middle-end (Sec. III). */
jslam_status jslam_get_refined(jslam_ctx *ctx, int32_t pair, jslam_refined *out);

/* Host views of the refinement (Sec. III, middle-end correlation
 * minimisation) inside a downloaded result block of pair `pair`. */
jslam_status jslam_result_refined_view(jslam_ctx *ctx, int32_t pair, const void *block, jslam_refined *out);

/* Device views of one pyramid level of one image (for consumers that share
 * the frontend's images, as the paper's middle-end does). */
typedef struct {
    int32_t width, height;
    int32_t raw_pitch, blurred_pitch;
    const uint8_t *raw;           /* level n resampled from level 0 (level 0: the input) */
    const uint8_t *blurred;       /* 7-tap Gaussian of the raw level (descriptor input) */
} jslam_level_view;

/* Fill `cfg` with the defaults (device 0, NULL stream, 1920x1080, 8 levels,
 * 4000 features, 64 pairs, P_min 9, P_max 13, k 1, q 3, border 19,
 * max_disp 128, band 2, distance 100, fallback off, dominance rule, circle
 * response, direct pyramid).  The
 * paper fixes P_min, P_max (Sec. II-A, Eq. 3), one corner per cell
 * (Sec. II-C-1) and the 3x3 PFA window (Sec. II-C-2); the other values are
 * this library's readings of points the paper leaves open. */
void jslam_default_config(jslam_config *cfg);

/* Create a context on cfg->device.  Validates the configuration
 * (JSLAM_ERR_ARG), uploads the constant tables (ring, blur weights, angle
 * sectors, rotated BRIEF pattern) and creates the stream if none is given.
 * The context's grow-only device buffers play the part of the paper's
 * Synchronized Shared Memory (Sec. III): frames, levels and keypoints stay
 * on the GPU between stages.  The ring and the corner rule are those of
 * Sec. II-A (Eq. 1-3).
 * On success *out owns the context; release it with jslam_destroy. */
jslam_status jslam_create(jslam_ctx **out, const jslam_config *cfg);

/* Enqueue the frontend for one stereo pair: pyramid and Gaussian filter
 * (Sec. III, streamlined multiscale detection and extraction), FAST with
 * Bounded Rectification (Sec. II-A, Eq. 1-3; Sec. III, efficient FAST
 * detection: bit masks and the sum-of-absolute-differences response),
 * per-cell culling (Sec. II-C-1, Feature Culling), Pyramidal Feature
 * Aggregation (Sec. II-C-2), keypoint cap, orientation and descriptors
 * (Sec. III, ORB for all scales at once) for both images.  Arguments as in
 * jslam_stereo_job.  JSLAM_ERR_ARG: null context, bad image (null data,
 * pitch < width, size above the configured maximum), levels out of range,
 * scale <= 1, threshold or cell out of range, or a level smaller than
 * 2*border+1. */
jslam_status jslam_extract(jslam_ctx *ctx, jslam_image left, jslam_image right,
                           int32_t levels, float scale, int32_t fast_thresh,
                           int32_t cell, int32_t max_feats);

/* Enqueue the frontend for n stereo pairs (1 <= n <= config.max_pairs) of
 * possibly different sizes and depths in one set of launches: the steps of
 * jslam_extract (Sec. II-A, II-C-1, II-C-2, III) for every image at once.
 * Batching many streams is this library's own addition (no counterpart in
 * the paper, which runs one camera).  Results of pair i are read with pair
 * index i. */
jslam_status jslam_extract_batch(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n);

/* Enqueue stereo row matching for every pair of the last extraction: the
 * middle-end's descriptor-distance minimisation along rectified rows
 * (Sec. III, Middle-end; the paper names the step, the search band and
 * tie-break are readings).  Results are read with jslam_get_matches (one
 * call enqueues, a second reads, instead of one call filling a struct).
 * JSLAM_ERR_STATE before any extraction. */
jslam_status jslam_match(jslam_ctx *ctx);

/* Wait for the context stream, copy counts to the host and surface any
 * device-side error flag.  Returns the context's sticky status.  The
 * paper's Synchronized Shared Memory (Sec. III) synchronises host and
 * device views of the frontend's data; here this is the one point where the
 * host waits for the device. */
jslam_status jslam_sync(jslam_ctx *ctx);

/* Keypoint views of `side` (0 = left, 1 = right) of pair `pair` of the last
 * extraction: the keypoints kept by Pyramidal Feature Aggregation
 * (Sec. II-C-2) with their K_l, K_r scores, FAST response (Sec. II-A) and
 * ORB angle and descriptor (Sec. III).  The `pair` argument selects one
 * pair of a batch.  JSLAM_ERR_ARG for an out-of-range pair or side. */
jslam_status jslam_get_keypoints(jslam_ctx *ctx, int32_t pair, int32_t side, jslam_keypoints *out);

/* Match views of pair `pair` (valid after jslam_match): the stereo matches
 * of the middle-end (Sec. III). */
jslam_status jslam_get_matches(jslam_ctx *ctx, int32_t pair, jslam_matches *out);

/* Level views of `side` of pair `pair` (valid after extraction): the
 * pyramid of Sec. III, shared with the middle-end as the paper's
 * Synchronized Shared Memory shares frames. */
jslam_status jslam_get_level(jslam_ctx *ctx, int32_t pair, int32_t side, int32_t level,
                             jslam_level_view *out);

/* Size in bytes of pair `pair`'s result block: a 16-byte header of int32
 * counts (left keypoints, right keypoints, two reserved), both images'
 * keypoints at capacity and the matches.  Result blocks and
 * their download are this library's transport (no counterpart in the
 * paper). */
jslam_status jslam_result_bytes(jslam_ctx *ctx, int32_t pair, size_t *bytes);

/* Enqueue an asynchronous copy of pair `pair`'s result block into host
 * memory `dst` of at least jslam_result_bytes bytes (pinned memory keeps it
 * asynchronous).  After jslam_sync the block can be read with
 * jslam_result_view.  The keypoint download that the paper's throughput
 * figures include (Sec. IV-C). */
jslam_status jslam_download(jslam_ctx *ctx, int32_t pair, void *dst, size_t bytes);

/* The result blocks of pairs [first, first + count) lie back to back in
 * device memory: their total size in *bytes and, if `offsets` is not NULL,
 * pair first + i's block at offsets[i] (count entries) from the first
 * (transport; no counterpart in the paper).
 * JSLAM_ERR_ARG for an empty or out-of-range span, JSLAM_ERR_STATE before
 * the first extraction. */
jslam_status jslam_result_range(jslam_ctx *ctx, int32_t first, int32_t count, size_t *bytes, size_t *offsets);

/* Enqueue ONE asynchronous copy of the result blocks of pairs [first,
 * first + count) into host memory `dst` of at least the jslam_result_range
 * bytes; pair first + i's block is then at dst + offsets[i], readable with
 * jslam_result_view after jslam_sync (the keypoint download of Sec. IV-C,
 * for a whole batch). */
jslam_status jslam_download_range(jslam_ctx *ctx, int32_t first, int32_t count, void *dst, size_t bytes);

/* Interpret a downloaded result block: fill host views of `side` (0 or 1)
 * into *kp and, for side 0, the matches into *m (may be NULL).  The count
 * comes from the block's own header, so a block downloaded from an earlier
 * extraction of the same batch shape reads correctly.  Pure host function;
 * `block` must hold jslam_result_bytes bytes of pair `pair`
 * (transport; no counterpart in the paper). */
jslam_status jslam_result_view(jslam_ctx *ctx, int32_t pair, const void *block, int32_t side,
                               jslam_keypoints *kp, jslam_matches *m);

/* Stages of the launch sequence, in launch order. */
enum {
    JSLAM_STAGE_PYRAMID = 0,      /* pyramid + Gaussian filter */
    JSLAM_STAGE_SKIP = 1,         /* learned cell-skip proposal (0 ms in exact mode) */
    JSLAM_STAGE_DETECT = 2,       /* FAST + Bounded Rectification + cell culling + PFA scatter */
    JSLAM_STAGE_PFA_NMS = 3,      /* PFA sparse NMS and per-row ranking */
    JSLAM_STAGE_PFA_FINAL = 4,    /* PFA aggregation, cap, canonical compaction */
    JSLAM_STAGE_ORB = 5,          /* orientation + descriptors */
    JSLAM_STAGE_MATCH = 6,        /* stereo row matching */
    JSLAM_STAGE_REFINE = 7,       /* correlation minimisation (jslam_refine_matches) */
    JSLAM_NUM_STAGES = 8
};

/* Turn per-stage timing on or off.  When on, every extraction and match
 * records a CUDA event on the context stream after each stage (a small
 * overhead per stage).  Per-stage times as the paper reports them for CRF,
 * FC and PFA (Sec. IV-B, IV-C). */
jslam_status jslam_enable_stage_timing(jslam_ctx *ctx, int32_t enable);

/* Device durations in milliseconds of each stage of the last extraction
 * (and match, if one followed it), measured between the recorded events
 * (the stage timings of Sec. IV-B, IV-C).  Valid after jslam_sync();
 * JSLAM_ERR_STATE if timing was off. */
jslam_status jslam_stage_times(jslam_ctx *ctx, float *ms /* JSLAM_NUM_STAGES entries */);

/* Launch-shape tuning.  None of these changes a result: detection tiles hold
 * whole culling cells, and every kernel variant computes the same outputs. */
typedef struct {
    int32_t tile_w_px;           /* detection tile width: 32..128, multiple of 4 (default 128) */
    int32_t tile_h_px;           /* detection tile height: 8..128 (default 64) */
    int32_t nms_kernel;          /* PFA NMS: 0 one warp per segment when every segment of the batch has at most
                                  * 96 candidate slots, else one CTA per segment (default); 1 one CTA per
                                  * segment always */
    int32_t detect_ctas_per_sm;  /* persistent detection CTAs per SM: 0 as many as fit (default), 1..8 at most
                                  * that many (never more than fit) */
    int32_t tile_order;          /* order in which the persistent detection CTAs take the tiles: 0 by image,
                                  * level and tile row (default); 1 by decreasing work (evaluated rows x
                                  * 32-pixel chunks), so the last rounds hold the smallest tiles */
} jslam_tuning;

/* Use `t` for the following extractions (plans are rebuilt when the tile
 * or the tile order changes).  Launch-shape tuning has no counterpart in the paper (its MLPT /
 * TEWA thread allocation, Sec. II-C-1, is fixed per cell size).
 * JSLAM_ERR_ARG for values outside the ranges above. */
jslam_status jslam_set_tuning(jslam_ctx *ctx, const jslam_tuning *t);

/* Tune the launch shapes on the batch `jobs` (n pairs, as for
 * jslam_extract_batch), timing the stages with the stage events: the
 * detection tile among five shapes, then the number of persistent detection
 * CTAs per SM, then (when every segment fits a warp) the NMS kernel, then the
 * tile order.  Keeps
 * the fastest for the context and returns it in *out (may be NULL).  Runs the
 * batch several times; results are unaffected.  No counterpart in the paper
 * (an autotuner in place of the fixed thread allocation of Sec. II-C-1). */
jslam_status jslam_autotune(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n, jslam_tuning *out);

/* jslam_autotune with a persistent cache: looks the batch up in the JSON
 * file `cache_path` under the key of jslam_tune_key (GPU name and SM count of
 * the context's device, its configuration, the batch's shapes and
 * parameters).  On a hit the stored pick is applied without any device work
 * and *hit = 1; on a miss the batch is tuned, the pick is added to the file
 * (created if missing) and *hit = 0.  `hit` may be NULL.  A file that does
 * not parse counts as empty and is rewritten.  JSLAM_ERR_ARG for a null
 * path or an unwritable file.  No counterpart in the paper. */
jslam_status jslam_autotune_cached(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n, const char *cache_path,
                                   jslam_tuning *out, int32_t *hit);

/* Key of a batch in the tuning cache (host only, no device work): GPU name
 * and SM count, the configuration fields that shape the kernels' work
 * (P_min, P_max, k, q, border, rule, fallback threshold) and every pair's
 * size, depth, scale bits, threshold, cell, cap and memory kinds, written to
 * buf (len bytes) as a NUL-terminated string.  JSLAM_ERR_CAPACITY when it
 * does not fit, JSLAM_ERR_ARG for null arguments.  No counterpart in the
 * paper. */
jslam_status jslam_tune_key(const char *gpu_name, int32_t sm_count, const jslam_config *cfg,
                            const jslam_stereo_job *jobs, int32_t n, char *buf, size_t len);

/* Look `key` up in the tuning cache file (host only): *found = 1 and *out
 * set on a hit, *found = 0 when the file is missing, does not parse or has
 * no valid entry for the key.  No counterpart in the paper. */
jslam_status jslam_tune_cache_get(const char *path, const char *key, jslam_tuning *out, int32_t *found);

/* Add or replace the entry of `key` in the tuning cache file (host only),
 * with the tuned stage time for reference; the file is rewritten through a
 * temporary file and a rename.  JSLAM_ERR_ARG for an invalid tuning, a key
 * holding a quote or backslash, or a file that cannot be written.  No
 * counterpart in the paper. */
jslam_status jslam_tune_cache_put(const char *path, const char *key, const jslam_tuning *t, float stage_ms);

/* Capture extraction + matching of the batch `jobs` into a CUDA graph owned
 * by the context (the batch runs once uncaptured first, so that the plan
 * and buffers exist); no counterpart in the paper, which launches per
 * scale on streams (Sec. III).  Replays read the same input buffers: device images
 * in place, host images (which must then be pinned) copied again.  The
 * context stream must not be the legacy default stream.  Replaces any
 * earlier graph. */
jslam_status jslam_graph_capture(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n);

/* Enqueue one replay of the captured graph on the context stream; results
 * are read as after jslam_extract_batch + jslam_match.  JSLAM_ERR_STATE if
 * nothing was captured, or if an extraction since the capture rebuilt the
 * context's plan (another batch shape, tuning or skip model: the graph's
 * tables and buffers are gone).  No counterpart in the paper. */
jslam_status jslam_graph_launch(jslam_ctx *ctx);

/* Replay the captured graph on new frames: `jobs` (n pairs) must match the
 * capture pair for pair in sizes, depths and parameters, with every image in
 * device memory; their pointers and pitches replace the captured ones (the
 * pyramid launch, the one kernel that reads the frames, is updated in the
 * instantiated graph).  For a camera stream processed one stereo pair per
 * call this makes every call one graph launch.  The images must stay valid
 * until jslam_sync().  JSLAM_ERR_ARG when the batch differs from the capture
 * or an image is in host memory; JSLAM_ERR_STATE as for jslam_graph_launch.
 * No counterpart in the paper (it launches per scale on streams, Sec. III). */
jslam_status jslam_graph_launch_jobs(jslam_ctx *ctx, const jslam_stereo_job *jobs, int32_t n);

/* PFA scores of one image's culled corners, computed without allocating
 * device memory.  The allocation-free variant itself has no counterpart in
 * the paper (the scores are those of Sec. II-C-2): it exists for callers that
 * cannot call cudaMalloc -- a real-time loop that forbids allocation after
 * start-up, a plug-in running inside another framework's enqueue hook, a
 * process whose device memory comes from a fixed pool.
 *
 * For the n corners (level[i], x[i], y[i], response[i]) (device arrays, level
 * coordinates) it writes, per corner, its s0 projection X[i], Y[i], the
 * number of levels k_levels[i] and summed response k_resp[i] at that s0
 * pixel, and alive[i] = 1 when no occupied pixel of the nms_q x nms_q window
 * dominates it, 0 when one does (pfa_rule as in jslam_config) -- the
 * k_levels / k_resp that jslam_extract reports for the corners it keeps.
 * A corner outside the domain -- level[i] >= levels, response[i] > 4080 (the
 * largest sum of 16 differences of 8-bit pixels), or a repeat of an earlier
 * (level, x, y) of the list -- takes no part in the scores and gets alive[i]
 * = 2, X = Y = 0xFFFF, k_levels = k_resp = 0 (of repeated corners, one is
 * scored and the others are marked, whichever the GPU reaches first).
 * Outputs are device arrays of n entries, owned by the caller.  Runs
 * asynchronously on `cuda_stream` (NULL: legacy default stream) of
 * `device`; the calling thread's current device is restored on return.
 *
 * Scratch: a 256 KB table in a statically allocated device array that every
 * GPU loading the library holds until the process exits.  Every call clears
 * and reuses it, so calls whose work overlaps on a GPU race and give wrong
 * results: serialise them (one stream, or events).  The first call on a
 * device looks up the table's device address; make that first call before
 * any stream capture.  The address is kept for the life of the process, so
 * after cudaDeviceReset the entry point must not be called on that device
 * again.  Nothing is allocated, ever.
 *
 * JSLAM_ERR_CAPACITY when n > 16384; JSLAM_ERR_ARG for n < 0, a null array
 * with n > 0, a size outside 1..4096, levels outside 1..8, scale outside the open
 * interval (1, 16), nms_q not odd in 1..7, a bad rule or device; JSLAM_ERR_CUDA if the table's address
 * or the launch fails.  n == 0 returns JSLAM_OK without work. */
jslam_status jslam_pfa_scores_static(const uint8_t *level, const uint16_t *x, const uint16_t *y,
                                     const uint16_t *response, int32_t n, int32_t width0, int32_t height0,
                                     int32_t levels, float scale, int32_t nms_q, int32_t pfa_rule,
                                     uint16_t *X, uint16_t *Y, uint8_t *k_levels, uint32_t *k_resp,
                                     uint8_t *alive, int32_t device, void *cuda_stream);

/* Learned cell-skip proposal (opt-in, approximate; no counterpart in the
 * paper: it proposes which Feature Culling cells of Sec. II-C-1 to skip).  `blob` holds a versioned model: the 16-byte header
 * {"JSKP", version 1, channels 16, downsample 8} (little-endian uint32
 * fields after the 4 magic bytes), then FP32 biases b1[16], b2[16], b3[1],
 * then BF16 weights w1[16][1][3][3], w2[16][16][3][3], w3[1][16][3][3] of
 * three 3x3 convolutions (zero padding, ReLU after the first two) applied to
 * the 8x8 box mean of level 0 scaled to [-0.5, 0.5].  An s0 culling cell
 * whose largest logit is below `thresh` is skipped: detection ignores every
 * cell of every level whose centre projects into it.  blob == NULL returns
 * to the exact path.  JSLAM_ERR_ARG for a malformed blob. */
jslam_status jslam_set_skip_model(jslam_ctx *ctx, const void *blob, size_t bytes, float thresh);

/* Device views of the skip proposal of `side` of pair `pair` (after an
 * extraction in skip mode): the 1/8-scale logits (h8 x w8 floats) and the
 * per-cell skip flags (cells_y x cells_x bytes, 1 = skipped).  No
 * counterpart in the paper. */
typedef struct {
    int32_t w8, h8, cells_x, cells_y;
    const float *logits;
    const uint8_t *skip;
} jslam_skip_view;
jslam_status jslam_get_skip_view(jslam_ctx *ctx, int32_t pair, int32_t side, jslam_skip_view *out);

/* Release the context and everything it owns (the device buffers that
 * stand for the Synchronized Shared Memory of Sec. III).  NULL is ignored. */
void jslam_destroy(jslam_ctx *ctx);

/* Static description of a status code (error reporting; no counterpart in
 * the paper). */
const char *jslam_status_str(jslam_status s);

/* ---- host-side tables (no device work; usable without a GPU) ---- */

/* The 256-pair steered BRIEF pattern rotated to each of the 30 angle
 * sectors: out[(b * 256 + i) * 4 + {0,1,2,3}] = (px, py, qx, qy) of pair i
 * in sector b.  `out` holds 30 * 256 * 4 bytes.  The descriptor of the
 * ORB extraction of Sec. III; the pattern is this library's own seeded
 * draw, not ORB's learned one. */
void jslam_pattern_table(int8_t *out);

/* Level geometry of an image: width, height and culling cell size of each
 * of `levels` levels for scale factor `scale` and s0 cell `cell` (the
 * pyramid of Sec. III; the cell shrinks with the level as Sec. IV-F states,
 * 32 x 32 at s0 to 8 x 8 at the eighth scale). */
jslam_status jslam_level_geometry(int32_t width, int32_t height, int32_t levels, float scale,
                                  int32_t cell, int32_t *w, int32_t *h, int32_t *c);

/* Projection of level-n coordinate v to s0 (clamped to extent-1): step 1
 * of Pyramidal Feature Aggregation (Sec. II-C-2), rounded to nearest. */
int32_t jslam_project(int32_t v, int32_t level, float scale, int32_t extent);

/* Corner look-up table of Sec. III for Eq. 3: bit m of out[m / 32] (bit
 * m % 32) is set when the 16-bit ring mask m has its longest circular run of
 * set bits in [p_min, p_max].  `out` holds 2048 words. */
jslam_status jslam_corner_table(int32_t p_min, int32_t p_max, uint32_t *out);

/* Stereo row band at level n: ceil(row_band_px * zeta^n), the search band
 * of the middle-end's stereo matching (Sec. III). */
int32_t jslam_match_band(int32_t level, float scale, int32_t row_band_px);

#ifdef __cplusplus
}
#endif

#endif /* JSLAM_H */
