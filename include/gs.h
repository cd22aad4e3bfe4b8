/*
 * gs.h - C ABI of the GB300 (sm_103a) mapping hot path of MonoGS++
 * (arXiv 2504.02437): differentiable 3D Gaussian splatting forward and
 * backward passes, the photometric + planar loss, Adam, dynamic insertion
 * and densification, over a window of keyframes.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Gaussian parameters are float32, planar SoA of shape [14][n]:
 *   rows 0-2 mean xyz (mu, Eq. 1), 3-5 log-scale (s = exp(.), Eq. 1),
 *   6-9 quaternion w,x,y,z (r of Eq. 1; normalised inside the forward pass),
 *   10 opacity logit (alpha = sigmoid(.)), 11-13 RGB colour (c of Eq. 1, k = 3).
 * - Images are float32, contiguous, channel-planar [n_views][3][H][W];
 *   per-pixel maps are [n_views][H][W].
 * - Pointers named *_dev are device pointers on the context's device; the
 *   library never frees caller memory. Pointers named *_host are host memory.
 * - `stream` is a cudaStream_t (NULL = legacy default stream). Every call
 *   enqueues its work on that stream and returns without waiting, unless its
 *   comment says it synchronises.
 * - Return value: GS_OK (0) or a negative GS_ERR_* code; gs_last_error()
 *   then holds a message. A call that fails with GS_ERR_ARG or
 *   GS_ERR_CAPACITY leaves the map state (parameters, Adam moments,
 *   densification statistics) unchanged.
 * - A context is bound to one device and is not thread-safe; use one context
 *   per host thread and keep its calls on one stream.
 */
#ifndef GS_GB300_H
#define GS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#define GS_OK 0
#define GS_ERR_ARG (-1)        /* invalid argument (null pointer, size, camera)          */
#define GS_ERR_OOM (-2)        /* device or pinned-host allocation failed               */
#define GS_ERR_CAPACITY (-3)   /* more Gaussians or pairs than the context can hold     */
#define GS_ERR_CUDA (-4)       /* a CUDA runtime call or kernel launch failed           */
#define GS_ERR_TIMEOUT (-5)    /* a bounded device-side wait gave up                    */
#define GS_ERR_NONFINITE (-6)  /* a non-finite loss or parameter was detected          */
#define GS_ERR_STATE (-7)      /* call out of order (e.g. backward before render)       */
#define GS_ERR_IO (-8)         /* a file could not be read or written, or is not a
                                  valid checkpoint of this format and version          */

#define GS_MAX_VIEWS 16

typedef struct gs_ctx gs_ctx;

/* Pinhole camera with world-to-camera pose (the viewing transform W of Eq. 2):
 * x_cam = R x_world + t; camera x right, y down, z forward. Pixel (px, py)
 * samples the image plane at (px, py) in the frame where u = fx x/z + cx. */
typedef struct gs_camera {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];   /* row-major */
    float t[3];
} gs_camera;

/* Every constant of the method. The paper fixes only reg_floor (Eq. 10) and
 * gives no value for the others; gs_default_config() sets the readings
 * documented with each field. */
typedef struct gs_config {
    float near_z;        /* cull t_z <= near_z (0.2)                                  */
    float fov_clamp;     /* J uses x/z, y/z clamped to fov_clamp x half-FOV tan (1.3)  */
    float dilation;      /* Sigma2D += dilation I (0.3)                               */
    float lambda_floor;  /* discriminant floor of the largest eigenvalue (0.1)        */
    float radius_sigma;  /* r = ceil(radius_sigma sqrt(lambda_max)) (3)               */
    float alpha_min;     /* skip alpha < alpha_min (1/255)                            */
    float alpha_max;     /* alpha = min(alpha_max, o G) (0.99)                        */
    float T_min;         /* stop before T (1 - alpha) < T_min (1e-4)                  */
    float lambda_color;  /* Eq. 11 weight of the photometric term (1)                 */
    float lambda_reg;    /* Eq. 11 weight of the planar term (1)                      */
    float reg_floor;     /* Eq. 10 floor of min(s) (0.01)                             */
    float lambda_photo;  /* Eq. 10 weight of L_SSIM = 1 - SSIM in L_color (0 = pure L1,
                            the paper's value is 0.2); in [0, 1]                      */
    float beta1, beta2, eps;     /* Adam (0.9, 0.999, 1e-15)                          */
    float lr[5];         /* Adam learning rates: means, log-scales, quaternions,
                            opacity logits, colours (1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3) */
    float split_thresh;  /* split if mean NDC position-grad norm > this (2e-4)        */
    float split_factor;  /* children log-scale -= ln(split_factor) (1.6)              */
    float insert_opacity;/* skip a new point if rendered opacity > this (0.99)        */
    float insert_tau;    /* > 0: Eq. 7 distance rule instead of the opacity gate: insert
                            iff the nearest existing mean is farther than this (0)    */
    float clarity_sigma; /* > 0: Eq. 9 split mask, split a Gaussian that dominates more
                            than this many pixels (gs_count_dominant) (0 = off)       */
    int32_t tile_size;   /* 8 or 16 pixels; 0 = pick by the built-in autotuner        */
    int32_t pixels_per_thread; /* compositing kernels: 1, 2 or 4 (16-px tiles), 1 or 2
                                  (8-px tiles); 0 = the autotuner's or the default      */
    int32_t capacity;    /* maximum number of Gaussians                               */
    int32_t max_views;   /* maximum views per render call (<= GS_MAX_VIEWS)           */
    int32_t max_width, max_height; /* largest image of any view                       */
    int64_t pair_capacity; /* (view, tile, Gaussian) pairs per render; 0 = 8 x capacity x max_views */
    uint64_t seed;       /* counter-based generator seed (split samples)              */
    int32_t deterministic; /* != 0: bitwise-repeatable results (0). No floating-point
                            atomics: the compositing adjoint writes each (view, tile,
                            Gaussian) pair's screen gradient into its own slot and a
                            per-Gaussian pass adds the slots in a fixed order; the
                            photometric loss is summed per tile. Uses 8-px tiles with 2
                            pixels per thread (one warp per tile) whatever tile_size and
                            pixels_per_thread say; slower than the default mode      */
} gs_config;

/* Fill *cfg with the defaults listed above (capacity 1<<20, 8 views, 1280x720). */
GS_API void gs_default_config(gs_config* cfg);

/* Create a context on CUDA device `device`; allocates every buffer for the
 * configured capacities (device memory, owned by the context).
 * Errors: GS_ERR_ARG (bad config), GS_ERR_OOM, GS_ERR_CUDA. */
GS_API int gs_create(const gs_config* cfg, int device, gs_ctx** out);

/* Free the context and all its device memory. Accepts NULL. */
GS_API void gs_destroy(gs_ctx* ctx);

/* Last error message of this context ("" if none); valid until the next call. */
GS_API const char* gs_last_error(const gs_ctx* ctx);

/* Number of Gaussians currently in the map. */
GS_API int gs_num_gaussians(const gs_ctx* ctx);

/* Replace the map by n Gaussians copied from params_dev ([14][n] float32,
 * row stride n). Resets Adam moments, the Adam step count and the
 * densification statistics. Errors: GS_ERR_ARG, GS_ERR_CAPACITY (n > capacity). */
GS_API int gs_set_params(gs_ctx* ctx, const float* params_dev, int n, void* stream);

/* Copy the current parameters to params_dev ([14][n], row stride n = gs_num_gaussians). */
GS_API int gs_get_params(gs_ctx* ctx, float* params_dev, void* stream);

/* Copy the gradient of the last gs_backward ([14][n] float32, row stride n). */
GS_API int gs_get_grads(gs_ctx* ctx, float* grads_dev, void* stream);

/* Overwrite the gradient that the next gs_step applies with grads_dev
 * ([14][n] float32, row stride n = gs_num_gaussians; caller-owned, read
 * before the call's work on `stream` completes), for a loss computed outside
 * the library. Errors: GS_ERR_ARG (NULL with n > 0). */
GS_API int gs_set_grads(gs_ctx* ctx, const float* grads_dev, void* stream);

/* Map initialisation from back-projected patch centres (Eq. 6, Section 3.2
 * "Map Initialization"): appends one Gaussian per point of points_dev
 * ([n][3] world xyz) with colour rgb_dev ([n][3]) and the plain
 * initialisation: log-scale = ln of the RMS distance to the 3 nearest other
 * points (clamped to [-7, -1], isotropic), quaternion (1,0,0,0), opacity
 * logit 0. Errors: GS_ERR_ARG, GS_ERR_CAPACITY. */
GS_API int gs_init_map(gs_ctx* ctx, const float* points_dev, const float* rgb_dev, int n, void* stream);

/* Render n_views views (Eq. 2 projection, tile binning, (tile, depth) sort,
 * Eq. 3 front-to-back compositing; Section 3.1). cams_host: n_views cameras.
 * rgb_dev: [n_views][3][H][W] output (H, W of each view; all views must
 * share one size). T_dev: optional [n_views][H][W] final transmittance.
 * argmax_dev: optional [n_views][H][W] int32 id of the Gaussian with the
 * largest blend weight (Eq. 8), -1 where nothing blends.
 * Keeps the per-pixel state that gs_backward needs. Synchronises the stream
 * once to size the pair buffers. Errors: GS_ERR_ARG, GS_ERR_CAPACITY (pair
 * buffer too small; the context grows it when possible), GS_ERR_CUDA,
 * GS_ERR_NONFINITE (an earlier loss or gradient was not finite; reported once,
 * the render is not made). */
GS_API int gs_render(gs_ctx* ctx, const gs_camera* cams_host, int n_views, float* rgb_dev, float* T_dev,
              int32_t* argmax_dev, void* stream);

/* Loss of the last render (Eq. 10-11, Section 3.2 "Map Optimization"):
 * L = sum_views lambda_color mean_{3HW}|C - I| + lambda_reg mean_i max(reg_floor, min_k s_ik).
 * target_dev: [n_views][3][H][W]. loss_dev: optional float[3] = {L, photometric, planar}.
 * Stores dL/dC for gs_backward(ctx, NULL, ...). */
GS_API int gs_loss(gs_ctx* ctx, const float* target_dev, float* loss_dev, void* stream);

/* Adjoint of the last render: gradients of the loss with respect to all
 * parameters (means, log-scales, quaternions, opacity logits, colours),
 * overwriting the context's gradient buffer. dL_drgb_dev: [n_views][3][H][W]
 * upstream gradient of the rendered image, or NULL to use the L1 gradient
 * stored by gs_loss, in which case the planar-term gradient is added too.
 * Recomputes per-pixel transmittance back to front from the stored final T
 * (no per-Gaussian blend state is stored). Errors: GS_ERR_STATE if no render. */
GS_API int gs_backward(gs_ctx* ctx, const float* dL_drgb_dev, void* stream);

/* One Adam step on every parameter with the gradient of the last gs_backward.
 * A parameter whose gradient is not finite keeps its value and moments; the
 * next gs_render or gs_iterate then returns GS_ERR_NONFINITE (once). */
GS_API int gs_step(gs_ctx* ctx, void* stream);

/* One full mapping iteration (Section 3.2 "Map Optimization") over a window
 * of n_views keyframes: projection, binning and sort for all views, then one
 * persistent kernel that composites, takes the L1 gradient and runs the
 * adjoint for every (view, tile), then the projection adjoint and Adam. The
 * first call for a shape runs these kernels directly, synchronising the stream
 * once after the projection to size the pair buffers; the iteration is then
 * recorded into a CUDA graph that later calls replay with their cameras.
 * target_dev [n_views][3][H][W]; loss_dev optional float[3]; rgb_dev optional
 * output image. With tile_size 0 in the config, the first call for a new
 * (image size, views, map-size bucket) first times the (tile size, pixels per
 * thread) candidates without updating the map and keeps the fastest (not in
 * the deterministic mode, which has one layout and adds a fixed-order
 * per-Gaussian sum of the adjoint's per-pair gradients). An
 * overflow of the pair buffer during a replay skips that iteration's Adam
 * step; a later call then grows the buffer and returns GS_ERR_CAPACITY. A
 * non-finite loss, or a non-finite gradient (its parameter and moments are
 * left unchanged by the Adam step), makes a later call return
 * GS_ERR_NONFINITE once, before it does any work. */
GS_API int gs_iterate(gs_ctx* ctx, const gs_camera* cams_host, int n_views, const float* target_dev,
               float* loss_dev, float* rgb_dev, void* stream);

/* gs_iterate with the target image and the loss in host memory (the same
 * mapping iteration, Section 3.2 "Map Optimization", Eq. 3, 10-11).
 * target_host [n_views][3][H][W] float32 is copied into one of two device
 * buffers the context owns, on a copy stream of its own: the copy starts once
 * the previous gs_iterate_host call's iteration has started on its stream (so
 * with the host ahead of the device it runs beside that iteration) and the
 * call before that, the last reader of the buffer, is done; this call's
 * iteration waits for it on `stream`. loss_host (optional, float[3]: total,
 * photometric, planar) receives the loss by a copy on `stream` after the
 * iteration: it holds the values once the stream has reached that point
 * (synchronise the stream or an event recorded after the call). Pinned host
 * memory (cudaMallocHost or equivalent) keeps both copies asynchronous;
 * pageable memory works, with the host then waiting for the copies. The
 * caller must not change target_host before the stream has passed the call.
 * rgb_dev as in gs_iterate. Errors as gs_iterate, plus GS_ERR_ARG for a NULL
 * target_host or an invalid camera and GS_ERR_OOM when the target buffers
 * cannot grow. gs_iterate with loss_dev NULL and gs_iterate_host write the
 * loss to one internal slot, so alternating the two keeps one recorded graph. */
GS_API int gs_iterate_host(gs_ctx* ctx, const gs_camera* cams_host, int n_views, const float* target_host,
                           float* loss_host, float* rgb_dev, void* stream);

/* Dynamic insertion for keyframe `cam` (Eq. 7 reading, Section 3.2 "Dynamic
 * 3D Gaussian Insertion"): renders the accumulated opacity of the current map
 * in that view; a point of points_dev ([n][3] world xyz) that projects in
 * front of the camera to a pixel whose opacity 1 - T exceeds insert_opacity
 * is skipped; every other point is appended with the plain initialisation
 * (log-scale from the 3 nearest existing means, colour of image_dev
 * [3][H][W] at the point's pixel), or the learned initialiser when one is
 * set (gs_set_initializer). With insert_tau > 0 the distance rule of Eq. 7's
 * text replaces the opacity gate (nothing is rendered): a point is appended
 * iff its nearest existing Gaussian mean is farther than insert_tau. Writes
 * the number appended to *n_inserted_host and, when inserted_dev is not
 * NULL, 1 or 0 per point to inserted_dev [n]. Synchronises the stream. */
GS_API int gs_insert(gs_ctx* ctx, const gs_camera* cam_host, const float* image_dev, const float* points_dev,
                     int n, int* n_inserted_host, uint8_t* inserted_dev, void* stream);

/* ---- learned initialiser (the BF16 MLP of the learned-initialisation reading) ----
 * A 3-layer MLP 80 -> 128 -> 128 -> 16 (GELU; the first 11 outputs are used)
 * run on the tensor cores in BF16 with FP32 accumulation. Input per VO point:
 * the keyframe's 5x5 RGB patch around the point's nearest pixel (borders
 * clamped, row-major, RGB interleaved), its depth, its camera-frame position
 * and a zero (80 floats). Output: log-scale (3), quaternion (4), opacity
 * logit (1), colour (3). Parameters are float32, one flat array of
 * gs_mlp_num_params() values: W1 [128][80], b1 [128], W2 [128][128], b2 [128],
 * W3 [16][128], b3 [16] (rows 11..15 of W3 and b3 stay zero). */
typedef struct gs_mlp gs_mlp;
/* Create an MLP on `device` with uniform(+-1/sqrt(fan_in)) weights drawn from
 * SplitMix64(seed) and zero biases. */
GS_API int gs_mlp_create(int device, uint64_t seed, gs_mlp** out);
GS_API void gs_mlp_destroy(gs_mlp* mlp);
GS_API int gs_mlp_num_params(void);
/* Copy parameters in (resets the Adam state) / out; flat_dev device float[gs_mlp_num_params()]. */
GS_API int gs_mlp_set_params(gs_mlp* mlp, const float* flat_dev, void* stream);
GS_API int gs_mlp_get_params(gs_mlp* mlp, float* flat_dev, void* stream);
/* Gradient of the last gs_mlp_backward (same layout). */
GS_API int gs_mlp_get_grads(gs_mlp* mlp, float* flat_dev, void* stream);
/* Input features of n points (points_dev [n][3] world xyz) seen by cam in image_dev
 * [3][H][W]: feat_dev [n][80]. */
GS_API int gs_mlp_features(const gs_camera* cam_host, const float* image_dev, const float* points_dev, int n,
                           float* feat_dev, void* stream);
/* Predictions out_dev [n][16] of feat_dev [n][80]. */
GS_API int gs_mlp_forward(gs_mlp* mlp, const float* feat_dev, int n, float* out_dev, void* stream);
/* Mean-squared error over the 11 outputs against target_dev [n][16] (loss_dev optional
 * float[1]) and its gradient w.r.t. all parameters (kept for gs_mlp_step). */
GS_API int gs_mlp_backward(gs_mlp* mlp, const float* feat_dev, const float* target_dev, int n, float* loss_dev,
                           void* stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) with learning rate lr. */
GS_API int gs_mlp_step(gs_mlp* mlp, float lr, void* stream);
/* Training targets of the learned initialiser for the map's Gaussians first ..
 * first + count - 1: out_dev [count][16] = log-scale (3), the quaternion
 * normalised with w >= 0 (q and -q are one rotation; a zero quaternion stays
 * zero), opacity logit (1), colour (3), then five zeros: the output layout of
 * gs_mlp_forward, for gs_mlp_backward. Errors: GS_ERR_ARG (range outside the
 * map, NULL out_dev), GS_ERR_CUDA. */
GS_API int gs_mlp_targets(gs_ctx* ctx, int first, int count, float* out_dev, void* stream);
/* Make gs_insert initialise new Gaussians with `mlp` (NULL restores the plain
 * initialisation). A point whose prediction is non-finite, has a log-scale
 * outside [-9, 1] or a zero quaternion keeps the plain initialisation. The
 * context does not own the MLP. */
GS_API int gs_set_initializer(gs_ctx* ctx, gs_mlp* mlp);

/* Densification by splitting (reading of Section 3.2 "Clarity-Enhancing
 * Gaussian Densification" with the 3DGS gradient criterion the paper builds
 * on): every Gaussian whose mean position-gradient norm in normalised device
 * coordinates, |(dL/du W/2, dL/dv H/2)| with u, v in pixels, over the backward
 * passes in which it was visible exceeds split_thresh is replaced by
 * two children with means mu + R S z (z standard normal), log-scales reduced
 * by ln(split_factor), other parameters copied and Adam moments zeroed. The
 * survivors keep their order; children follow in parent order.
 * normals_dev: optional [n][2][3] standard normal samples (NULL = draw them
 * with the context's counter-based generator). Resets the statistics.
 * Writes the number of split parents to *n_split_host. Synchronises. */
GS_API int gs_densify(gs_ctx* ctx, const float* normals_dev, int* n_split_host, void* stream);

/* Eq. 8-9 (Section 3.2 "Clarity-Enhancing Gaussian Densification"): renders
 * the views (cams_host: n_views cameras of one image size) with the per-pixel
 * argmax of the blend weight w_m (Eq. 8) and adds, per Gaussian, the number of
 * pixels it dominates to its count. gs_densify then also splits every
 * Gaussian whose count exceeds clarity_sigma (when > 0) and resets the counts.
 * Synchronises. Errors: GS_ERR_ARG, GS_ERR_OOM, GS_ERR_CUDA. */
GS_API int gs_count_dominant(gs_ctx* ctx, const gs_camera* cams_host, int n_views, void* stream);

/* Peak signal-to-noise ratio of n floats of img_dev against ref_dev (images in
 * [0, 1]): out_dev[0] = 10 log10(1 / max(MSE, 1e-12)), the evaluation measure
 * of the time-to-PSNR comparison. Sums in float64 in a fixed order (repeatable
 * bit for bit); uses the context's scratch, so calls of one context stay on
 * one stream. Errors: GS_ERR_ARG, GS_ERR_CUDA. */
GS_API int gs_psnr(gs_ctx* ctx, const float* img_dev, const float* ref_dev, int64_t n, float* out_dev, void* stream);

/* Device-side timing of the path's phases with CUDA events recorded on the
 * launching stream around each phase's kernels (a profiling aid; off by
 * default). Phases: */
#define GS_PHASE_PROJECT 0      /* Eq. 2 projection, depth sort, scan of tile counts    */
#define GS_PHASE_BIN 1          /* pair emission, (tile, depth) sort, tile ranges        */
#define GS_PHASE_RASTER_FWD 2   /* Eq. 3 compositing kernel                              */
#define GS_PHASE_LOSS 3         /* Eq. 10-11 loss and dL/dC                              */
#define GS_PHASE_RASTER_BWD 4   /* adjoint compositing kernel                            */
#define GS_PHASE_PROJECT_BWD 5  /* adjoint of the projection + planar gradient           */
#define GS_PHASE_ADAM 6         /* Adam update                                           */
#define GS_PHASE_RASTER_FUSED 7 /* gs_iterate: compositing + L1 + adjoint in one kernel  */
#define GS_N_PHASES 8
/* enable != 0 starts recording (discarding earlier records); 0 stops. */
GS_API int gs_timing_enable(gs_ctx* ctx, int enable);
/* Time only the phases whose bit is set in mask (bit p = phase p); fewer event
 * records in a replayed iteration disturb it less. Clears earlier records. */
GS_API int gs_timing_phases(gs_ctx* ctx, uint32_t mask);
/* Synchronise on the recorded events and write, per phase, the summed
 * milliseconds (ms_host[GS_N_PHASES]) and the number of recorded intervals
 * (counts_host[GS_N_PHASES], may be NULL); clears the records. */
GS_API int gs_timing_read(gs_ctx* ctx, float* ms_host, int32_t* counts_host);

/* Checkpoint and resume of the map being optimised (Section 3.2); the paper
 * has no counterpart, the format is this library's own. A checkpoint holds
 * everything a later mapping iteration reads besides the cameras and
 * images: the n Gaussians' parameters, their Adam first and second moments,
 * the Adam step counters and running powers of beta1, beta2 (so the bias
 * correction continues where it stopped), and the densification statistics
 * (summed screen-gradient norms, their counts, the dominance counts of
 * gs_count_dominant). The splitting noise is a counter-based function of the
 * seed in gs_config and needs no state.
 *
 * File format, little-endian, version 1: a 64-byte header
 *   char magic[8] = "GSMAPCK1"; uint32 version = 1; uint32 rows = 14;
 *   uint32 n; uint32 adam_steps_device; int32 adam_steps_host; uint32 0;
 *   float64 beta_powers[2]; uint64 payload_bytes; uint64 fnv1a64(payload)
 * followed by the payload (payload_bytes = 180 n): float32 params[14][n],
 * float32 m[14][n], float32 v[14][n], float32 grad_norm_sum[n],
 * float32 grad_norm_count[n], uint32 dominance[n]. */
/* Synchronises `stream`, then writes the context's map state to `path`
 * (created or replaced). Errors: GS_ERR_ARG (NULL argument), GS_ERR_IO (the
 * file cannot be written), GS_ERR_CUDA. The context is not changed. */
GS_API int gs_save(gs_ctx* ctx, const char* path, void* stream);
/* Reads and checks the whole file at `path` (magic, version, sizes, checksum)
 * before it touches the context, then replaces the context's map state with
 * it, synchronising `stream`. Per-render state is dropped: a gs_render or
 * gs_iterate comes next. Errors: GS_ERR_ARG (NULL argument), GS_ERR_IO
 * (missing, truncated, corrupt or other-format file), GS_ERR_CAPACITY (more
 * Gaussians than the context holds); on any of these the context is
 * unchanged. GS_ERR_CUDA. */
GS_API int gs_load(gs_ctx* ctx, const char* path, void* stream);
/* Checks the checkpoint at `path` as gs_load does, without a context or a
 * GPU, and writes its number of Gaussians and format version (either pointer
 * may be NULL). Returns GS_OK or GS_ERR_ARG (NULL path) or GS_ERR_IO. */
GS_API int gs_checkpoint_info(const char* path, int* n_host, int* version_host);

/* Stable LSD radix sort of n (key, value) pairs by the low `bits` bits of the
 * key, for callers that cannot allocate device memory: those that run while
 * another component owns the device allocator, or inside a loop that must
 * not call cudaMalloc. The paper has no counterpart; it is the pair sort of
 * gs_render offered on its own. It allocates nothing: its scratch (about
 * 8.7 MB) is a static device array that every GPU loading this library
 * holds until the process exits, so n is limited to 1048576 pairs
 * (GS_ERR_CAPACITY above that). keys_in/vals_in ([n] device) are read,
 * keys_out/vals_out ([n] device) receive the pairs sorted by the low `bits`
 * bits of the key (the other bits are kept), equal sort keys keeping their
 * input order; ceil(bits / 8) radix passes. Neither output range may overlap
 * an input range or the other output (GS_ERR_ARG); the inputs may overlap.
 * Enqueued on `stream` without waiting. Each call looks up the array's
 * address on the current device; the first call on a device loads the
 * library's device code, so make it before any stream capture. Every call
 * shares the one scratch array, so calls that overlap on the GPU (different
 * streams or host threads) race; the array keeps the last call's contents,
 * and each call writes every word it reads. If the CUDA runtime already holds
 * an unchecked error from earlier work, the call launches nothing, leaves
 * that error in place and returns GS_ERR_CUDA. Errors: GS_ERR_ARG (bits
 * outside 1..32, NULL or overlapping buffers), GS_ERR_CAPACITY, GS_ERR_CUDA
 * (a failed lookup, memset or launch of this call). */
GS_API int gs_sort_pairs_static(const uint32_t* keys_in_dev, const uint32_t* vals_in_dev, uint32_t* keys_out_dev,
                                uint32_t* vals_out_dev, int64_t n, int bits, void* stream);

/* Introspection for tests (synchronising, host outputs). */
/* Per-view screen quantities of the last render, float64 host arrays of n each:
 * out_host[k*n + i] for k = 0 u, 1 v, 2 conic a, 3 conic b, 4 conic c, 5 depth
 * (the float32 value the sort uses), 6 radius, 7 tiles touched; row 8 is 1.0
 * for a valid Gaussian else 0. */
GS_API int gs_debug_projection(gs_ctx* ctx, int view, double* out_host);
/* Sorted pairs of the last render: bins (view * tiles_per_view + tile) and
 * values (view * n + id). Writes *count_host = P; copies min(P, max) pairs. */
GS_API int gs_debug_pairs(gs_ctx* ctx, uint32_t* bins_host, uint32_t* vals_host, int64_t max, int64_t* count_host);
/* Gradients of the last backward with respect to each view's screen
 * quantities, host [n_views][9][n]: u, v, conic a, b, c, opacity, r, g, b. */
GS_API int gs_debug_grad2d(gs_ctx* ctx, float* out_host);
/* Algorithmic work of the last render, out_host[4]: pairs P, (pixel, Gaussian)
 * tests of the forward pass up to each pixel's stop, blended pairs, and the
 * pairs the backward pass walks (entries up to each pixel's last blend). */
GS_API int gs_debug_work(gs_ctx* ctx, int64_t* out_host);
/* Number of kernels this context has launched since it was created. */
GS_API int64_t gs_launch_count(const gs_ctx* ctx);
/* Tile size the last render used. */
GS_API int gs_tile_size(const gs_ctx* ctx);
/* Pixels per thread of the compositing kernels of the last render. */
GS_API int gs_pixels_per_thread(const gs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GS_GB300_H */
