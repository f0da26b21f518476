/*
 * rara.h -- C ABI of the GB300 (sm_103a) RaRa clipped Gaussian-splat renderer.
 *
 * The render has four steps (arXiv 2506.20202, "RaRa Clipper"):
 *   rara_preprocess  per-Gaussian three-way classification against the clip plane
 *                    (Section 3.2, Eq. 3; Algorithm 1 step 1), EWA projection to a 2D
 *                    conic (Section 3.4, Eq. 9-10), SH colour, tile rectangle
 *   rara_bin         one (tile id | depth) key per listing tile, radix-sorted so every tile
 *                    holds its Gaussians front to back (Section 3.1, "sorted by depth"); a
 *                    tile of the 3-sigma rectangle lists a Gaussian where some pixel centre
 *                    of the tile can blend it (alpha0 >= 1/255, Algorithm 1 step 3)
 *   rara_render      per pixel, front-to-back compositing (Eq. 2) of alpha from Eq. 10,
 *                    with the ray-ellipsoid decay weight (Eq. 4-8, Eq. 11, Eq. 12;
 *                    Algorithm 1 steps 2-3) for cutoff Gaussians and early termination
 *   rara_render_frame   the three calls in sequence
 *   rara_render_batch   many views (cameras, planes, resolutions) of one or more scenes in
 *                    one launch per stage; rara_render_batch_graph replays the batch's stage
 *                    sequence as a captured CUDA graph
 *   rara_render_backward   gradients of a loss on the rendered images with respect to the
 *                    Gaussians' parameters and the clip planes (an extension: the paper
 *                    renders only)
 *
 * Conventions
 *   - All device pointers are CUDA device memory on the current device; sizes are
 *     elements. Arrays are planar (structure of arrays): means[3][n] holds all x, then all
 *     y, then all z. quats[4][n] is (w, x, y, z), normalised inside. sh[(L+1)^2 * 3][n]:
 *     plane k*3 + c is real-SH coefficient k = l*l + l + m of colour channel c.
 *   - Camera: world_to_cam = [R | t] row-major 3x4, OpenCV axes (x right, y down,
 *     z forward); pixel (i, j) has its centre at (i + 0.5, j + 0.5); fx, fy, cx, cy in
 *     pixels.
 *   - Plane: n . x + d = 0, the visible side is where n points (Section 3.2). (n, d) are
 *     used as given, so pass a unit n for d to be a distance. k_sigma scales the
 *     ray-traced ellipsoid M = k_sigma R S (3 = the 3-sigma support; Section 3).
 *   - Every call is asynchronous on the given stream (a cudaStream_t, or NULL for the
 *     legacy default stream), except that rara_bin waits for the stream once to read the
 *     number of rendered Gaussians and pairs. The caller keeps inputs alive and unchanged
 *     until the work queued on the stream has finished.
 *   - Errors: every call returns a rara_status. RARA_OK is 0. On error nothing further is
 *     queued and rara_last_error() holds a message. Device-side faults of the bounded
 *     waits inside the kernels (RARA_ERR_TIMEOUT) are reported by the next rara_bin or
 *     rara_ctx_sync call. Nothing traps or exits.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef RARA_H
#define RARA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rara_status {
    RARA_OK = 0,
    RARA_ERR_INVALID_ARG = 1, /* null pointer, n < 0, sh_degree outside [0,3], W or H <= 0,
                                 non-finite camera/plane, unknown mode, call out of order;
                                 and, detected on the device and reported at the next host
                                 wait, a Gaussian with a non-finite mean, log-scale (a zero
                                 scale is log-scale -inf), quaternion, opacity logit or SH
                                 colour, or a zero quaternion (such Gaussians are not
                                 rendered and the frame is invalid) */
    RARA_ERR_BUDGET = 2,      /* the context's device-memory budget cannot hold this frame */
    RARA_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    RARA_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up (results invalid) */
    RARA_ERR_OVERFLOW = 5     /* a graph replay produced more pairs than its capacity: the
                                 batch's images are invalid; render it again (the context has
                                 grown the capacity and recaptures on the next call) */
} rara_status;

typedef enum rara_mode {
    RARA_MODE_NONE = 0,     /* no clipping: every Gaussian visible */
    RARA_MODE_HARD = 1,     /* centre test only: invisible iff n.mu + d < 0 (Section 1) */
    RARA_MODE_RARA = 2,     /* the paper's method (Algorithm 1) */
    RARA_MODE_RARA_ALL = 3  /* ablation "wo RaRa" (Section 4.3): weight on every
                               non-invisible Gaussian */
} rara_mode;

typedef enum rara_label { RARA_INVISIBLE = 0, RARA_VISIBLE = 1, RARA_CUTOFF = 2 } rara_label;

typedef struct rara_gaussians {
    const float *means;          /* device [3][n] */
    const float *log_scales;     /* device [3][n], log of the per-axis standard deviation */
    const float *quats;          /* device [4][n], (w, x, y, z) */
    const float *opacity_logits; /* device [n], opacity delta = sigmoid(logit) */
    const float *sh;             /* device [(sh_degree+1)^2 * 3][n] */
    int64_t n;                   /* number of Gaussians, 0 <= n < 2^31 */
    int32_t sh_degree;           /* 0..3 */
} rara_gaussians;

typedef struct rara_camera {
    float world_to_cam[12]; /* row-major [R | t] */
    float fx, fy, cx, cy;
    int32_t width, height;
} rara_camera;

#define RARA_MAX_EXTRA_PLANES 3

/* The clip plane n.x + d = 0 (visible side n.x + d >= 0), or a convex clip volume: with
 * n_extra > 0, the planes extra[k] = (n.x, n.y, n.z, d) for k < n_extra are added and the
 * visible region is the intersection of the visible sides of all 1 + n_extra planes. The
 * paper clips by one plane and names other clipping primitives, wherever the ray meets
 * them cheaply, as its extension (Discussion, Limitations); for a convex volume its rules
 * read: a Gaussian is invisible if its sphere of radius 3 max(sigma) lies wholly behind
 * some plane, visible if it lies wholly in front of every plane, cutoff otherwise
 * (Section 3.2, Algorithm 1 step 1 per plane); the decay weight is the share of the pixel
 * ray's chord through the ellipsoid that lies inside the volume (Eq. 11 with the chord
 * clipped by every plane, Eq. 8 per plane); hard clipping removes a Gaussian whose centre
 * is behind some plane. Zero-initialise the struct: n_extra = 0 is the single plane.
 * rara_render_backward and rara_render_frame_noalloc accept single planes only
 * (RARA_ERR_INVALID_ARG for n_extra > 0). */
typedef struct rara_plane {
    float n[3];
    float d;
    float k_sigma;   /* > 0 */
    int32_t mode;    /* rara_mode */
    int32_t n_extra; /* 0..RARA_MAX_EXTRA_PLANES further planes of a convex clip volume */
    float extra[RARA_MAX_EXTRA_PLANES][4];
} rara_plane;

/* One view of a batch: a camera, a clip plane and output buffers over one of the batch's
 * scenes. image is device float [3][H][W]; final_T float [H][W] and n_contrib uint32 [H][W]
 * may be NULL. */
typedef struct rara_view {
    int32_t scene;       /* index into the batch's scene array */
    rara_camera camera;
    rara_plane plane;
    float bg[3];
    float *image;
    float *final_T;
    uint32_t *n_contrib;
} rara_view;

typedef struct rara_ctx rara_ctx;

/* Create a context on the current CUDA device. budget_bytes caps the device scratch the
 * context may hold (0 = no cap). tile_w x tile_h is the screen tile the binning and the
 * render use: 16 x 16, 32 x 8, 8 x 32 (256 pixels), 8 x 8 (64) or 32 x 16, 16 x 32 (512);
 * RARA_ERR_INVALID_ARG for other shapes. Images do not depend on the tile (a tile lists a
 * Gaussian wherever one of its pixels can blend it); n_contrib, a position in the pixel's
 * tile list, does. The blend batch depth starts at 256 (rara_ctx_set_tiling). */
int rara_ctx_create(size_t budget_bytes, int32_t tile_w, int32_t tile_h, rara_ctx **out);

/* Tile shape (as for rara_ctx_create) and blend batch depth of the context's next frames and
 * batches: 128, 256 or 512 list entries staged in shared memory by the whole block per render
 * batch, or 32 for each warp staging and walking its own 32-entry chunks (no block barrier
 * inside a work item); the
 * autotuner's knobs (the paper renders 16 x 16 tiles and names no batch depth). The
 * current frame's state is dropped when the tile changes, and a captured graph is
 * recaptured on the next rara_render_batch_graph. RARA_ERR_INVALID_ARG for unsupported
 * values. */
int rara_ctx_set_tiling(rara_ctx *ctx, int32_t tile_w, int32_t tile_h, int32_t blend_depth);

/* Free every device and pinned buffer the context owns. Waits for the device first.
 * NULL is accepted. */
int rara_ctx_destroy(rara_ctx *ctx);

/* Last error message of the context ("" if none). Valid until the next call. */
const char *rara_last_error(const rara_ctx *ctx);

/* Bytes of device scratch currently held by the context. */
size_t rara_ctx_bytes(const rara_ctx *ctx);

/* Allocate the context's scratch up front (serving: no allocation, and so no device-wide
 * synchronisation of cudaFree / cudaMalloc, inside the request loop; the paper has no
 * counterpart). Later frames and batches of up to `slots` (view, Gaussian) slots (the sum
 * over the views of their scenes' sizes), `pairs` listed (Gaussian, tile) pairs, `views`
 * views and `max_view_tiles` tiles in the largest view use these buffers without
 * allocating; larger ones grow them as usual. Counts within the budget of
 * rara_ctx_create, else RARA_ERR_BUDGET (what was reserved before the refusal stays
 * held). Convex clip volumes and the backward allocate their own extra buffers on first
 * use. Synchronous (it allocates). */
int rara_ctx_reserve(rara_ctx *ctx, int64_t slots, int64_t pairs, int32_t views, int32_t max_view_tiles);

/* Wait for `stream` and report a device-side wait failure of earlier work. */
int rara_ctx_sync(rara_ctx *ctx, void *stream);

/* Render scheduling knobs of the context. The render gives a tile whose list holds at
 * least 2^(split2_bits - 1) entries 2 lanes per pixel (a 16x16 tile becomes 2 work items of
 * 16x8 pixels), and one with at least 2^(split4_bits - 1) entries 4 lanes per pixel (4 items
 * of 16x4; split4 wins when both apply); the lanes of a pixel combine consecutive entries,
 * which shortens the pixel's dependent chain. 8x8 tiles always take 4 lanes per pixel and
 * 512-pixel tiles at most 2. Values are clamped to [0, 33] (0: always split, 33: never).
 * Images do not depend on them beyond the float rounding order of the compositing sums.
 * Defaults: 11 and 12. */
int rara_ctx_set_tuning(rara_ctx *ctx, int32_t split2_bits, int32_t split4_bits);

/* Test hook of the bounded device-side waits (the paper has no counterpart: its renderer
 * has no multi-block scans). It applies to the next rara_preprocess / rara_render_batch on
 * this context only, and only outside a graph capture: the compaction's look-back waits
 * give up after spin_limit polls (0 = the default bound of about a second), and with
 * orphan_first_partition != 0 its partition tickets start at 1, so partition 0 is never
 * processed and every later partition's wait on its look-back word runs out. The kernel
 * then records the time-out in the context's status word and returns; the next host wait
 * (rara_bin, rara_render_batch, rara_ctx_sync) reports RARA_ERR_TIMEOUT and the frame is
 * invalid. The context stays usable: the next call clears the status. */
int rara_ctx_debug_waits(rara_ctx *ctx, int32_t spin_limit, int32_t orphan_first_partition);

/* GPU time (ms) of the stages of the last frame or batch (a graph replay included):
 * out[0] preprocess + compaction, out[1] sorts, emission, ranges and render order, out[2]
 * render. Waits for that render to finish. */
int rara_ctx_stage_ms(rara_ctx *ctx, float out[3]);

/* The same, finer: out[0] k_preprocess (with the counter memsets before it), out[1] the
 * compaction, out[2] the depth sort, out[3] the pair emission, out[4] the tile sort,
 * out[5] the ranges and the render work order. Measurement only (the paper times whole
 * frames). Waits for the last render to finish. */
int rara_ctx_kernel_ms(rara_ctx *ctx, float out[6]);

/* Number of kernel launches this context has queued since creation (all entry points). */
int64_t rara_ctx_launches(const rara_ctx *ctx);

/* Step (a): classify, project and shade the Gaussians for one camera and plane.
 * Section 3.2 (Eq. 3), Algorithm 1 step 1, Section 3.4 (Eq. 9-10). Inputs are read on
 * the stream; the frame state lives in ctx until the next rara_preprocess. */
int rara_preprocess(rara_ctx *ctx, const rara_gaussians *g, const rara_camera *cam,
                    const rara_plane *plane, void *stream);

/* Step (b): emit one pair per (Gaussian, listing tile): a tile of the Gaussian's rectangle
 * whose box of pixel centres reaches q <= q_cut = min(9, 2 ln(255 opacity)), the pixels
 * where alpha0 = opacity exp(-q/2) can reach 1/255 (no other pixel can blend the Gaussian);
 * radix-sort by (tile id, depth), and build per-tile ranges. Must follow rara_preprocess on the same context. Blocks the
 * host once (stream synchronisation) to size the pair buffers. */
int rara_bin(rara_ctx *ctx, void *stream);

/* Steps (c)+(d): composite every pixel. image is device float [3][H][W] (planar RGB),
 * final_T device float [H][W] (transmittance left after the last blended Gaussian),
 * n_contrib device uint32 [H][W] (1 + position, within the pixel's tile list, of the last
 * blended Gaussian; 0 if none). final_T and n_contrib may be NULL. bg is a host float[3].
 * Eq. 2, Eq. 10-12, Algorithm 1 steps 2-3. Must follow rara_bin. */
int rara_render(rara_ctx *ctx, const float bg[3], float *image, float *final_T,
                uint32_t *n_contrib, void *stream);

/* rara_preprocess + rara_bin + rara_render. */
int rara_render_frame(rara_ctx *ctx, const rara_gaussians *g, const rara_camera *cam,
                      const rara_plane *plane, const float bg[3], float *image,
                      float *final_T, uint32_t *n_contrib, void *stream);

/* Batched render: every view of `views` (any order, any resolutions, any of the scenes)
 * goes through the same steps as rara_render_frame, each step one launch for the whole
 * batch (Section 3.2-3.4 and Algorithm 1 per view). At most 4096 views and 64 scenes; the
 * sum over views of the scene sizes must stay below 2^32. Waits for the stream once (after
 * the preprocess) to size the pair buffers. The per-view results and counts stay available
 * through the rara_frame_* calls with the view's index until the next batch or frame. */
int rara_render_batch(rara_ctx *ctx, const rara_gaussians *scenes, int32_t num_scenes, const rara_view *views,
                      int32_t num_views, void *stream);

/* Same as rara_render_batch, without any host synchronisation: the first call for a batch
 * shape (scene sizes and SH degrees, view count, per-view resolution and scene, whether a view
 * clips by a convex volume, whether the batch is one scene seen from one camera) renders it
 * with rara_render_batch, sizes the pair capacity from it (+25%), and captures the whole
 * stage sequence on a private stream into a CUDA graph; later calls with the same shape
 * copy the new cameras, planes, scene and output pointers into the graph's tables and
 * launch the graph on `stream`. A replay that would exceed the pair capacity writes no pair
 * past it and is reported as RARA_ERR_OVERFLOW by the next rara_ctx_sync, which also grows
 * the capacity so the next call recaptures. */
int rara_render_batch_graph(rara_ctx *ctx, const rara_gaussians *scenes, int32_t num_scenes,
                            const rara_view *views, int32_t num_views, void *stream);

/* Gradients of one scene, device arrays in the layouts of rara_gaussians (means[3][n],
 * log_scales[3][n], quats[4][n] with respect to the unnormalised input quaternion,
 * opacity_logits[n], sh[(L+1)^2 * 3][n]). */
typedef struct rara_gaussian_grads {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
} rara_gaussian_grads;

/* Backward of the last render on this context (rara_render / rara_render_frame,
 * rara_render_batch, or rara_render_batch_graph): given dL/dimage for every view, writes
 * the gradients of the Gaussians' parameters and of every view's clip plane. The paper
 * renders only (the Discussion's limitations leave re-optimising Gaussians after clipping
 * to future work); this differentiates the forward of Eq. 2, Eq. 9-12 and Algorithm 1 as
 * the kernels compute it: where the weight w is 0 or 1 (the chord on one side of the
 * plane, a ray that misses the ellipsoid), where alpha is clamped at 0.99 or the colour
 * at 0, the gradient through that factor is 0; the class thresholds, the q <= 9 support, the 1/255 alpha
 * cut-off and the 1e-4 transmittance stop are discontinuities and pass none.
 *   dL_dimages   [num_views] device pointers, view v's dL/dimage [3][H][W] (the caller's
 *                view order, as given to the forward)
 *   grads        [num_scenes] gradient arrays, written (not accumulated): every Gaussian of
 *                every scene gets its sum over the views that render it, 0 if none
 *   plane_grads  device float[num_views][4] = dL/d(n.x, n.y, n.z, d) per view, written; or
 *                NULL. k_sigma and the mode are not differentiated.
 * The forward must have been given final_T and n_contrib buffers for every view, and its
 * inputs and outputs must be unchanged. Returns RARA_ERR_INVALID_ARG if there is no
 * rendered frame or batch on the context, a view lacks final_T / n_contrib, or a pointer is
 * NULL. Asynchronous on `stream`; gradient sums use float atomics, so they are not
 * bit-reproducible. */
int rara_render_backward(rara_ctx *ctx, const float *const *dL_dimages, const rara_gaussian_grads *grads,
                         float *plane_grads, void *stream);

/* The L2 objective of a differentiation step on the last render's images, with its gradient,
 * in one launch (the input rara_render_backward takes). The paper renders only; re-fitting
 * Gaussians after clipping, which its Discussion leaves to future work, needs an objective,
 * and the differentiation workload and the baking loop use this one. For every view v of the
 * last render (the caller's view order) with d = image_v - target_v over its [3][H][W] image:
 *   loss[v] = scale[v] * sum(d^2)   and   dL_dimages[v] = 2 scale[v] d
 * (scale[v] = 1 / (3 H W) makes loss[v] the view's mean squared error).
 *   targets     [num_views] device pointers, view v's target [3][H][W], read
 *   dL_dimages  [num_views] device pointers, view v's gradient [3][H][W], written; it may be
 *               the target itself, not the rendered image
 *   scale       host float[num_views]
 *   loss        device double[num_views], written
 * Returns RARA_ERR_INVALID_ARG if there is no rendered frame or batch on the context, a
 * pointer is NULL, a gradient output is the rendered image or a scale is not finite.
 * Asynchronous on `stream`; the loss sums use double atomics, so their last bits are not
 * reproducible. */
int rara_loss_l2(rara_ctx *ctx, const float *const *targets, float *const *dL_dimages, const float *scale,
                 double *loss, void *stream);

/* GPU milliseconds of the last rara_render_backward: [0] the per-tile render backward,
 * [1] the per-Gaussian preprocess backward. Waits for them to finish. */
int rara_ctx_backward_ms(rara_ctx *ctx, float out[2]);

/* Measurement: with on != 0 the renders of this context launched outside a CUDA graph
 * (rara_render, rara_render_batch) count their work in the device counters that
 * rara_frame_info_get reports (n_evaluated, n_walked, n_cut_evaluated, n_tested); the
 * counting costs the render a few percent, so it is off by default. */
int rara_ctx_count_work(rara_ctx *ctx, int32_t on);

/* Counts of one view of the current frame or batch (view 0 for a single frame), valid after
 * rara_bin; the render counts are totals over all views of the last render launched outside
 * a CUDA graph with counting on (rara_ctx_count_work): graph replays render without the work
 * counters and leave them 0. Waits for the context's last stream to read them. */
typedef struct rara_frame_info {
    int64_t n;            /* Gaussians in the frame */
    int64_t n_rendered;   /* not invisible, not culled, at least one tile */
    int64_t n_cutoff;     /* rendered and labelled cutoff */
    int64_t n_pairs;      /* (Gaussian, tile) pairs listed: a tile of the Gaussian's 3-sigma
                             rectangle lists it where some pixel centre of the tile can have
                             alpha0 = opacity exp(-q/2) >= 1/255 with q <= 9 */
    int32_t tiles_x, tiles_y;
    int64_t n_evaluated;  /* (pixel, Gaussian) pairs of the last rara_render with
                             alpha0 >= 1/255 inside the q <= 9 support (this and the next
                             three: only with rara_ctx_count_work on, else 0) */
    int64_t n_walked;     /* (pixel, Gaussian) pairs whose q was computed, i.e. tile-list
                             entries visited by pixels still compositing */
    int64_t n_cut_evaluated; /* evaluated pairs that needed the ray-traced weight */
    int64_t n_tested;     /* (warp rectangle, Gaussian) culling tests of the last render */
    int64_t n_pair_candidates; /* tiles of the view's rendered rectangles: the upper bound of
                                  n_pairs the preprocess sizes the pair buffers by */
    int64_t n_depth_keys; /* keys the depth sort of the frame or batch sorted: the rendered
                             (view, Gaussian) slots of all views, or, when the batch is one scene
                             whose views all share one camera, the Gaussians some view renders
                             (sorted once) */
    int64_t n_shared_pairs; /* a one-camera batch of at most 32 views lists and tile-sorts the
                               Gaussians some view renders once (every view's tile lists are
                               that list without the Gaussians the view does not render): the
                               pairs of that shared list; 0 for any other frame or batch (a
                               one-camera batch of more views expands the depth order into
                               every view's slots and lists each view) */
} rara_frame_info;

int rara_frame_info_get(rara_ctx *ctx, int32_t view, rara_frame_info *out);

/* Copy per-Gaussian preprocess results of one view into caller device buffers (any may be
 * NULL; n is the view's scene size):
 * labels uint8[n]; depth float[n] (camera z); mean2d float[2][n]; conic float[3][n]
 * (a, b, c of [[a,b],[b,c]], the inverse 2D covariance); rgb float[3][n]; opacity float[n];
 * rect int32[4][n] (inclusive tx0, ty0, tx1, ty1); tiles uint32[n] (tiles of the rectangle,
 * 0 when culled).
 * Fields other than labels are defined only where tiles > 0. */
int rara_frame_gaussians(rara_ctx *ctx, int32_t view, uint8_t *labels, float *depth, float *mean2d,
                         float *conic, float *rgb, float *opacity, int32_t *rect,
                         uint32_t *tiles, void *stream);

/* Copy one view's sorted pair list into caller device buffers: keys uint64[n_pairs]
 * (tile id << 32 | float bits of the depth), values uint32[n_pairs] (Gaussian index), and
 * ranges int64[num_tiles][2] ([start, end) of each tile, tile id = ty * tiles_x + tx),
 * where n_pairs and the tile counts are the view's (rara_frame_info_get). Waits for the
 * context's last stream. */
int rara_frame_pairs(rara_ctx *ctx, int32_t view, uint64_t *keys, uint32_t *values, int64_t *ranges,
                     void *stream);

/* Allocation-free variant of rara_render_frame (the paper has no counterpart).
 *
 * For callers that cannot call cudaMalloc: a plug-in running inside another engine's
 * frame loop or a host callback, where an allocation would block or is not allowed, or a
 * process whose device memory belongs to another allocator. The call allocates nothing
 * (no cudaMalloc, cudaFree, pinned or heap memory): every scratch buffer is carved from one
 * file-scope static __device__ array of about 22.0 MB (21.0 MiB), which each GPU that loads
 * the library holds until the process exits. The caller passes inputs and outputs as for
 * rara_render_frame, with the same layouts and results.
 *
 * Limits: n <= 65536 Gaussians, at most 2^19 (Gaussian, tile) pairs and 16384 tiles (for
 * example 2048 x 2048 pixels). Larger inputs return RARA_ERR_BUDGET before any work is
 * queued (the pair limit is checked after the preprocess, which waits for the stream).
 * Other errors: RARA_ERR_INVALID_ARG, RARA_ERR_CUDA, RARA_ERR_TIMEOUT as above; there is no
 * context, so no message is kept.
 *
 * The first call on a device resolves the static array's device address (set-up, once per
 * device, with that device current); make that first call before any stream capture.
 * Every call on a device shares the one array and leaves the last call's contents in it:
 * calls that overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. The call waits for the stream three times (once to read the pair
 * count, then twice more inside the binning, where the stream is already idle). It is not
 * thread-safe. */
int rara_render_frame_noalloc(const rara_gaussians *g, const rara_camera *cam, const rara_plane *plane,
                              const float bg[3], float *image, float *final_T, uint32_t *n_contrib,
                              void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RARA_H */
