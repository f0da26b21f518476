// C ABI of librara.so: context, buffer management, argument checks, batch set-up, stage
// order, CUDA-graph capture of a batch, and the allocation-free frame render.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "rara_internal.cuh"

using namespace rara;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    unsigned gen = 0;  // bumped whenever the allocation is replaced or released
};

constexpr int kMaxViews = 4096;
constexpr int kMaxScenes = 64;

// Host staging of the batch tables (pinned, so uploads are asynchronous). Two copies are
// used in turn; a copy is refilled only after the upload that last read it has completed.
struct Staging {
    ViewDev *views = nullptr;
    SceneDev *scenes = nullptr;
    cudaEvent_t uploaded = nullptr;
};

}  // namespace

struct rara_ctx {
    size_t budget = 0;
    size_t held = 0;
    int device = 0;
    char err[512] = {0};
    int64_t launches = 0;
    int sm_count = 0, bpsm_sort = 0, bpsm_emit = 0, bpsm_compact = 0;
    int bpsm_render[4] = {0, 0, 0, 0};  // render blocks per SM for batch depths 32, 128, 256, 512
    int split2_bits = 11, split4_bits = 12;  // heavy-tile split thresholds (list length bit counts)
    int tile_w = kTile, tile_h = kTile;      // screen tile of the next batch
    int blend_depth = kBlock;                // list entries staged per render batch
    bool count_work = false;                 // renders outside graphs fill the work counters

    // current batch
    int stage = 0;  // 0 empty, 1 preprocessed, 2 binned
    int num_views = 0, num_scenes = 0;
    uint32_t num_slots = 0, num_tiles = 0, num_units = 0;
    int tile_bits = 0;                  // global tile id = internal view << tile_bits | local tile
    int tile_passes = 1;                // digit passes of the tile sort
    int tile_digit_bits = 8;            // bits per tile-sort pass (the tile bits split evenly)
    int view_passes = 0;                // view digit passes of the depth sort (several views)
    uint32_t cap_pairs = 0;             // pair capacity the binning kernels were launched with
    cudaStream_t last_stream = nullptr;
    int max_views = 0, max_scenes = 0;
    Staging staging[2];
    int staging_next = 0;
    ViewDev *h_views = nullptr;         // the staging copy holding the current batch
    SceneDev *h_scenes = nullptr;
    int *h_view_map = nullptr;          // caller's view index -> internal (scene-grouped) index
    int *h_view_n = nullptr;            // scene size of each internal view
    Counters *h_counters = nullptr;     // pinned
    ViewCounters *h_view_counters = nullptr;  // pinned [max_views]

    // device
    DevBuf views_d, scenes_d, view_counters_d, counters;
    DevBuf labels, tiles, erec, rec, cut, depth;
    DevBuf cut_x;                       // further planes of clip-volume cutoff slots
    DevBuf gkey;                        // one-camera batches: per-Gaussian depth keys
    DevBuf vmask, list_counts;          // shared listing: per-Gaussian view masks, partition counts
    bool one_camera = false;            // the batch is one scene whose views share one camera
    bool shared_list = false;           // ... of at most kListViews views: its tile lists are built once
    bool multi = false;                 // the batch has a view with a convex clip volume
    bool extra_planes = false;          // the batch has a view with further planes
    DevBuf ckeys, cvals, ckeys_b, cvals_b, lookback_c;
    DevBuf pkeys, pvals, pkeys_b, pvals_b, lookback_e;
    DevBuf hist, ranges, items, sort_scratch, seg_base, export_off;

    // captured batch
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int *shape = nullptr;               // host copy of the captured batch shape
    size_t shape_len = 0;
    uint32_t graph_cap_pairs = 0;
    uint32_t min_cap_pairs = 0;         // raised after an overflow
    int64_t graph_kernels = 0;          // kernel launches one replay makes

    bool owns_host = true;              // false for the static context
    bool rendered = false;              // the current batch has been rendered (backward may follow)

    // backward: gradient records, tables of the dL/dimage and gradient pointers
    DevBuf grec, bviews_d, bscenes_d;
    // grec is known to be all zero (allocation generation grec_zero_gen): the preprocess
    // backward zeroes every record it reads, and the render backward adds only to those
    bool grec_zero = false;
    unsigned grec_zero_gen = 0;
    BwdView *h_bviews = nullptr;        // pinned [max_views]
    BwdScene *h_bscenes = nullptr;      // pinned [max_scenes]
    cudaEvent_t bwd_uploaded = nullptr;
    // the L2 objective (rara_loss_l2): its view table
    DevBuf lviews_d;
    LossView *h_lviews = nullptr;       // pinned [max_views]
    cudaEvent_t loss_uploaded = nullptr;
    cudaEvent_t bev[3] = {nullptr, nullptr, nullptr};
    int bpsm_render_bwd = 0;

    // test hook of the bounded waits (rara_ctx_debug_waits), applied to the next batch's
    // compaction only: its look-back poll limit, and whether its first partition is left
    // unprocessed (its look-back word is then never written)
    int debug_spin_limit = 0;
    bool debug_orphan = false;

    // stage timing of the last batch rendered outside a graph: preprocess start, bin start,
    // render start, render end, then inside the stages: after the depth sort, after the
    // emission, after the tile sort, after k_preprocess (before the compaction)
    cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool capturing = false;
};

namespace {

int fail(rara_ctx *c, int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
    return code;
}

int check_cuda(rara_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return RARA_OK;
    return fail(c, RARA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Errors the kernels record in the device status word (read after a host wait).
int device_status(rara_ctx *c, uint32_t status)
{
    if (status & kStatusLookbackTimeout)
        return fail(c, RARA_ERR_TIMEOUT, "a bounded device-side wait gave up; the frame is invalid");
    if (status & kStatusBadInput)
        return fail(c, RARA_ERR_INVALID_ARG,
                    "a Gaussian has a non-finite mean, log-scale, quaternion, opacity logit or colour, or a zero "
                    "quaternion; the frame is invalid");
    return RARA_OK;
}

// Grow-only device buffer within the context budget.
int ensure(rara_ctx *c, DevBuf &b, size_t bytes, const char *name)
{
    if (bytes <= b.cap) return RARA_OK;
    // the static context's buffers are carved from a fixed array: never freed or replaced
    if (!c->owns_host)
        return fail(c, RARA_ERR_BUDGET, "buffer %s needs %zu bytes; the static scratch holds %zu", name, bytes, b.cap);
    size_t want = bytes + bytes / 4;  // headroom so small growth does not reallocate
    want = (want + 255) & ~(size_t)255;
    if (c->budget && c->held - b.cap + want > c->budget) {
        want = bytes;
        if (c->held - b.cap + want > c->budget)
            return fail(c, RARA_ERR_BUDGET, "buffer %s needs %zu bytes; context holds %zu of a %zu budget", name,
                        bytes, c->held - b.cap, c->budget);
    }
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        if (e != cudaSuccess) return check_cuda(c, e, "cudaFree");
        c->held -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    ++b.gen;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, e == cudaErrorMemoryAllocation ? RARA_ERR_BUDGET : RARA_ERR_CUDA,
                    "cudaMalloc(%zu) for %s: %s", want, name, cudaGetErrorString(e));
    }
    b.cap = want;
    c->held += want;
    return RARA_OK;
}

void release(rara_ctx *c, DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    c->held -= b.cap;
    b.p = nullptr;
    b.cap = 0;
    ++b.gen;
}

bool finite(float v) { return isfinite(v) != 0; }

// Stage events. Inside a graph capture they become event-record nodes of the graph, so a
// replay records them too and the stage times of the last replay can be read.
void mark(rara_ctx *c, int k, cudaStream_t s)
{
    if (!c->ev[k]) return;
    if (c->capturing) cudaEventRecordWithFlags(c->ev[k], s, cudaEventRecordExternal);
    else cudaEventRecord(c->ev[k], s);
}

int launched(rara_ctx *c, const char *what, int count = 1)
{
    c->launches += count;
    return check_cuda(c, cudaGetLastError(), what);
}

int ceil_bits(uint32_t v)
{
    int b = 0;
    while ((1ull << b) < (unsigned long long)v) ++b;
    return b;
}

void occupancy_setup(rara_ctx *c)
{
    if (c->sm_count) return;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        c->sm_count < 1) {
        cudaGetLastError();
        c->sm_count = 1;
    }
    const int depths[4] = {32, 128, 256, 512};
    for (int k = 0; k < 4; ++k) c->bpsm_render[k] = render_blocks_per_sm(depths[k]);
    c->bpsm_sort = sort_blocks_per_sm();
    c->bpsm_emit = emit_blocks_per_sm();
    c->bpsm_compact = compact_blocks_per_sm();
    c->bpsm_render_bwd = render_bwd_blocks_per_sm();
    if (preprocess_configure()) cudaGetLastError();  // a launch that needs it then reports the error
}

int check_gaussians(rara_ctx *c, const rara_gaussians *g)
{
    if (!g) return fail(c, RARA_ERR_INVALID_ARG, "null scene");
    if (g->n < 0 || g->n >= (int64_t)1 << 31) return fail(c, RARA_ERR_INVALID_ARG, "n = %lld out of range", (long long)g->n);
    if (g->sh_degree < 0 || g->sh_degree > 3) return fail(c, RARA_ERR_INVALID_ARG, "sh_degree %d not in [0,3]", g->sh_degree);
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail(c, RARA_ERR_INVALID_ARG, "null Gaussian array");
    return RARA_OK;
}

int check_view(rara_ctx *c, const rara_camera *cam, const rara_plane *pl)
{
    if (!cam || !pl) return fail(c, RARA_ERR_INVALID_ARG, "null camera or plane");
    if (cam->width <= 0 || cam->height <= 0 || cam->width / c->tile_w >= 65535 || cam->height / c->tile_h >= 65535)
        return fail(c, RARA_ERR_INVALID_ARG, "image size %dx%d", cam->width, cam->height);
    for (int k = 0; k < 12; ++k)
        if (!finite(cam->world_to_cam[k])) return fail(c, RARA_ERR_INVALID_ARG, "non-finite camera pose");
    if (!(finite(cam->fx) && finite(cam->fy) && finite(cam->cx) && finite(cam->cy) && cam->fx > 0 && cam->fy > 0))
        return fail(c, RARA_ERR_INVALID_ARG, "bad intrinsics");
    if (!(finite(pl->n[0]) && finite(pl->n[1]) && finite(pl->n[2]) && finite(pl->d)))
        return fail(c, RARA_ERR_INVALID_ARG, "non-finite plane");
    if (!(finite(pl->k_sigma) && pl->k_sigma > 0)) return fail(c, RARA_ERR_INVALID_ARG, "k_sigma must be > 0");
    if (pl->mode < RARA_MODE_NONE || pl->mode > RARA_MODE_RARA_ALL)
        return fail(c, RARA_ERR_INVALID_ARG, "unknown mode %d", pl->mode);
    if (pl->n_extra < 0 || pl->n_extra > RARA_MAX_EXTRA_PLANES)
        return fail(c, RARA_ERR_INVALID_ARG, "n_extra %d outside [0, %d]", pl->n_extra, RARA_MAX_EXTRA_PLANES);
    for (int e = 0; e < pl->n_extra; ++e)
        for (int k = 0; k < 4; ++k)
            if (!finite(pl->extra[e][k])) return fail(c, RARA_ERR_INVALID_ARG, "non-finite clip-volume plane");
    return RARA_OK;
}

// Bitwise-equal cameras (the preprocess reuses a Gaussian's projection across such views).
bool same_camera(const rara_camera &a, const rara_camera &b)
{
    return memcmp(a.world_to_cam, b.world_to_cam, sizeof(a.world_to_cam)) == 0 && a.fx == b.fx && a.fy == b.fy &&
           a.cx == b.cx && a.cy == b.cy && a.width == b.width && a.height == b.height;
}

// One scene whose views all share one camera: its depth order is the same in every view.
bool one_camera_batch(int ns, const rara_view *views, int nv)
{
    if (ns != 1 || nv < 2) return false;
    for (int v = 1; v < nv; ++v)
        if (!same_camera(views[v].camera, views[0].camera)) return false;
    return true;
}

void fill_view(ViewDev &v, const rara_camera *cam, const rara_plane *pl, int tile_w, int tile_h)
{
    for (int k = 0; k < 9; ++k) v.cam.R[k] = cam->world_to_cam[(k / 3) * 4 + (k % 3)];
    for (int k = 0; k < 3; ++k) v.cam.t[k] = cam->world_to_cam[k * 4 + 3];
    v.cam.fx = cam->fx; v.cam.fy = cam->fy; v.cam.cx = cam->cx; v.cam.cy = cam->cy;
    v.cam.W = cam->width; v.cam.H = cam->height;
    for (int j = 0; j < 3; ++j)  // e = -R^T t
        v.cam.eye[j] = -(v.cam.R[j] * v.cam.t[0] + v.cam.R[3 + j] * v.cam.t[1] + v.cam.R[6 + j] * v.cam.t[2]);
    for (int k = 0; k < 3; ++k) v.plane.n[k] = pl->n[k];
    v.plane.d = pl->d;
    v.plane.k = pl->k_sigma;
    v.plane.mode = pl->mode;
    v.plane.n_extra = pl->n_extra;
    for (int e = 0; e < RARA_MAX_EXTRA_PLANES; ++e)
        for (int k = 0; k < 4; ++k) v.plane.ex[e][k] = e < pl->n_extra ? pl->extra[e][k] : 0.0f;
    v.tile_w = tile_w;
    v.tile_h = tile_h;
    v.tiles_x = (cam->width + tile_w - 1) / tile_w;
    v.tiles_y = (cam->height + tile_h - 1) / tile_h;
}

// Take the next staging copy, waiting for the upload that last read it.
int next_staging(rara_ctx *c)
{
    Staging &st = c->staging[c->staging_next];
    if (st.uploaded) {
        int rc = check_cuda(c, cudaEventSynchronize(st.uploaded), "staging wait");
        if (rc) return rc;
    }
    c->h_views = st.views;
    c->h_scenes = st.scenes;
    return RARA_OK;
}

int upload_tables(rara_ctx *c, cudaStream_t s)
{
    int rc;
    if ((rc = check_cuda(c, cudaMemcpyAsync(c->views_d.p, c->h_views, sizeof(ViewDev) * (size_t)c->num_views,
                                            cudaMemcpyHostToDevice, s), "view table upload")))
        return rc;
    if ((rc = check_cuda(c, cudaMemcpyAsync(c->scenes_d.p, c->h_scenes, sizeof(SceneDev) * (size_t)c->num_scenes,
                                            cudaMemcpyHostToDevice, s), "scene table upload")))
        return rc;
    Staging &st = c->staging[c->staging_next];
    if (st.uploaded && (rc = check_cuda(c, cudaEventRecord(st.uploaded, s), "staging event"))) return rc;
    c->staging_next ^= 1;
    return RARA_OK;
}

// Build the batch tables (views grouped by scene, in the caller's order within a scene),
// size the per-slot buffers and upload the tables.
int batch_setup(rara_ctx *c, const rara_gaussians *scenes, int ns, const rara_view *views, int nv, cudaStream_t s)
{
    c->stage = 0;
    c->rendered = false;
    if (ns < 1 || ns > c->max_scenes) return fail(c, RARA_ERR_INVALID_ARG, "%d scenes (1..%d)", ns, c->max_scenes);
    if (nv < 1 || nv > c->max_views) return fail(c, RARA_ERR_INVALID_ARG, "%d views (1..%d)", nv, c->max_views);
    int rc;
    for (int i = 0; i < ns; ++i)
        if ((rc = check_gaussians(c, &scenes[i]))) return rc;
    for (int v = 0; v < nv; ++v) {
        if (views[v].scene < 0 || views[v].scene >= ns)
            return fail(c, RARA_ERR_INVALID_ARG, "view %d refers to scene %d of %d", v, views[v].scene, ns);
        if ((rc = check_view(c, &views[v].camera, &views[v].plane))) return rc;
        if (!views[v].image) return fail(c, RARA_ERR_INVALID_ARG, "view %d has no image buffer", v);
    }
    if ((rc = next_staging(c))) return rc;
    c->multi = false;
    c->extra_planes = false;
    for (int v = 0; v < nv; ++v) {
        const rara_plane &pl = views[v].plane;
        c->extra_planes = c->extra_planes || pl.n_extra > 0;
        c->multi = c->multi || (pl.n_extra > 0 && (pl.mode == RARA_MODE_RARA || pl.mode == RARA_MODE_RARA_ALL));
    }
    uint64_t max_tiles = 1;
    for (int v = 0; v < nv; ++v) {
        const uint64_t t = (uint64_t)((views[v].camera.width + c->tile_w - 1) / c->tile_w) *
                           (uint64_t)((views[v].camera.height + c->tile_h - 1) / c->tile_h);
        if (t > max_tiles) max_tiles = t;
    }
    const int tile_bits = ceil_bits((uint32_t)(max_tiles < 0xffffffffull ? max_tiles : 0xffffffffull));
    uint64_t slots = 0, tiles = 0;
    uint32_t units = 0;
    int k = 0;
    for (int si = 0; si < ns; ++si) {
        SceneDev &sd = c->h_scenes[si];
        const rara_gaussians &g = scenes[si];
        sd.means = g.means; sd.log_scales = g.log_scales; sd.quats = g.quats; sd.logits = g.opacity_logits;
        sd.sh = g.sh;
        sd.n = (int)g.n;
        sd.sh_degree = g.sh_degree;
        sd.view_begin = k;
        sd.unit_begin = units;
        int prev_v = -1;    // the caller's index of the scene's previous view
        for (int v = 0; v < nv; ++v) {
            if (views[v].scene != si) continue;
            ViewDev &vd = c->h_views[k];
            fill_view(vd, &views[v].camera, &views[v].plane, c->tile_w, c->tile_h);
            vd.scene = si;
            vd.tile_base = (uint32_t)((uint64_t)k << tile_bits);
            vd.slot_base = (uint32_t)slots;
            for (int j = 0; j < 3; ++j) vd.bg[j] = views[v].bg[j];
            vd.image = views[v].image;
            vd.final_T = views[v].final_T;
            vd.n_contrib = views[v].n_contrib;
            // views of one scene with the same camera share the preprocess's projection
            vd.same_cam = prev_v >= 0 && same_camera(views[prev_v].camera, views[v].camera) ? 1 : 0;
            prev_v = v;
            c->h_view_map[v] = k;
            c->h_view_n[k] = (int)g.n;
            slots += (uint64_t)g.n;
            ++k;
        }
        sd.view_count = k - sd.view_begin;
        if (sd.view_count > 0) units += (uint32_t)((g.n + kBlock - 1) / kBlock);
    }
    tiles = (uint64_t)nv << tile_bits;
    if (slots >= ((uint64_t)1 << 32) - 1)
        return fail(c, RARA_ERR_INVALID_ARG, "%llu slots exceed 2^32", (unsigned long long)slots);
    if (tiles >= ((uint64_t)1 << 28))
        return fail(c, RARA_ERR_INVALID_ARG, "%llu tiles exceed 2^28", (unsigned long long)tiles);
    c->num_views = nv;
    c->num_scenes = ns;
    c->num_slots = (uint32_t)slots;
    c->num_tiles = (uint32_t)tiles;
    c->num_units = units;
    c->tile_bits = tile_bits;
    c->tile_passes = (tile_bits + 7) / 8;
    if (c->tile_passes < 1) c->tile_passes = 1;
    c->tile_digit_bits = tile_bits > 0 ? (tile_bits + c->tile_passes - 1) / c->tile_passes : 1;
    c->view_passes = nv > 256 ? 2 : (nv > 1 ? 1 : 0);
    // One scene whose views all share one camera (a plane sweep from one viewpoint): the depth
    // order is the same in every view, so the Gaussians are depth-sorted once and expanded
    // per view (no view passes)
    c->one_camera = one_camera_batch(ns, views, nv);
    if (c->one_camera) c->view_passes = 0;
    // ... and with at most kListViews views, its tile lists too: every view's list is the
    // union's (listed and tile-sorted once) without the Gaussians the view does not render
    c->shared_list = c->one_camera && nv <= kListViews;
    const size_t nn = slots > 0 ? (size_t)slots : 1;
    const size_t nt = tiles > 0 ? (size_t)tiles : 1;
    if ((rc = ensure(c, c->views_d, sizeof(ViewDev) * (size_t)nv, "view table")) ||
        (rc = ensure(c, c->scenes_d, sizeof(SceneDev) * (size_t)ns, "scene table")) ||
        (rc = ensure(c, c->view_counters_d, sizeof(ViewCounters) * (size_t)nv, "view counters")) ||
        (rc = ensure(c, c->labels, nn, "labels")) || (rc = ensure(c, c->tiles, nn * 4, "tiles")) ||
        (rc = ensure(c, c->erec, nn * sizeof(EmitRec), "emission records")) || (rc = ensure(c, c->rec, nn * sizeof(SplatRec), "records")) ||
        (rc = ensure(c, c->cut, nn * sizeof(CutRec), "cutoff records")) ||
        (rc = ensure(c, c->depth, nn * 4, "depth")) || (rc = ensure(c, c->ckeys, nn * 4, "depth keys")) ||
        (rc = ensure(c, c->cvals, nn * 4, "depth values")) || (rc = ensure(c, c->ckeys_b, nn * 4, "depth keys B")) ||
        (rc = ensure(c, c->cvals_b, nn * 4, "depth values B")) ||
        (rc = ensure(c, c->lookback_c, (nn / 1024 + 2) * 8, "compaction scan words")) ||
        (rc = ensure(c, c->lookback_e, (nn / kBlock + 2) * 8, "emission scan words")) ||
        (rc = ensure(c, c->hist, kHistPasses * 256 * 4, "digit histograms")) ||
        (rc = ensure(c, c->seg_base, sizeof(uint32_t) * (size_t)nv, "view slot bases")) ||
        (rc = ensure(c, c->ranges, nt * sizeof(int2), "ranges")) ||
        (rc = ensure(c, c->items, nt * 16, "render items")) ||
        (c->multi && (rc = ensure(c, c->cut_x, nn * sizeof(CutExtra), "clip-volume records"))) ||
        (c->one_camera && (rc = ensure(c, c->gkey, (size_t)(scenes[0].n > 0 ? scenes[0].n : 1) * 4, "depth keys"))) ||
        (c->shared_list && (rc = ensure(c, c->vmask, (size_t)(scenes[0].n > 0 ? scenes[0].n : 1) * 4, "view masks"))))
        return rc;
    return upload_tables(c, s);
}

// Stage (a): preprocess + compaction.
int batch_preprocess(rara_ctx *c, cudaStream_t s)
{
    int rc;
    occupancy_setup(c);
    Counters *dc = (Counters *)c->counters.p;
    const size_t nn = c->num_slots > 0 ? (size_t)c->num_slots : 1;
    mark(c, 0, s);
    if ((rc = check_cuda(c, cudaMemsetAsync(dc, 0, sizeof(Counters), s), "memset counters")) ||
        (rc = check_cuda(c, cudaMemsetAsync(c->view_counters_d.p, 0, sizeof(ViewCounters) * (size_t)c->num_views, s),
                         "memset view counters")) ||
        (rc = check_cuda(c, cudaMemsetAsync(c->hist.p, 0, kHistPasses * 256 * 4, s), "memset histograms")) ||
        (rc = check_cuda(c, cudaMemsetAsync(c->lookback_c.p, 0, (nn / 1024 + 2) * 8, s), "memset scan")))
        return rc;
    PreprocessArgs a;
    a.scenes = (const SceneDev *)c->scenes_d.p;
    a.num_scenes = c->num_scenes;
    a.views = (const ViewDev *)c->views_d.p;
    a.num_units = (int)c->num_units;
    a.labels = (uint8_t *)c->labels.p;
    a.tiles = (uint32_t *)c->tiles.p;
    a.erec = (EmitRec *)c->erec.p;
    a.rec = (SplatRec *)c->rec.p;
    a.cut = (CutRec *)c->cut.p;
    a.cut_x = c->multi ? (CutExtra *)c->cut_x.p : nullptr;
    a.depth = (float *)c->depth.p;
    a.gkey = c->one_camera ? (uint32_t *)c->gkey.p : nullptr;
    a.vmask = c->shared_list ? (uint32_t *)c->vmask.p : nullptr;
    a.view_counters = (ViewCounters *)c->view_counters_d.p;
    a.counters = dc;
    int max_degree = 0, max_views = 0;
    for (int si = 0; si < c->num_scenes; ++si) {
        if (c->h_scenes[si].view_count > 0 && c->h_scenes[si].sh_degree > max_degree)
            max_degree = c->h_scenes[si].sh_degree;
        if (c->h_scenes[si].view_count > max_views) max_views = c->h_scenes[si].view_count;
    }
    launch_preprocess(a, (int)c->num_units, max_degree, max_views, s);
    if ((rc = launched(c, "preprocess launch", c->num_units > 0))) return rc;
    mark(c, 7, s);

    CompactArgs ca;
    ca.tiles = (const uint32_t *)c->tiles.p;
    ca.depth = (const float *)c->depth.p;
    ca.gkey = c->one_camera ? (const uint32_t *)c->gkey.p : nullptr;
    ca.num_slots = c->one_camera ? (uint32_t)c->h_scenes[0].n : c->num_slots;
    ca.keys = (uint32_t *)c->ckeys.p;
    ca.vals = (uint32_t *)c->cvals.p;
    ca.hist = (uint32_t *)c->hist.p;
    ca.views = (const ViewDev *)c->views_d.p;
    ca.view_counters = (const ViewCounters *)c->view_counters_d.p;
    ca.num_views = c->num_views;
    ca.seg_base = (uint32_t *)c->seg_base.p;
    ca.lookback = (unsigned long long *)c->lookback_c.p;
    ca.counters = dc;
    ca.spin_limit = c->debug_spin_limit > 0 ? c->debug_spin_limit : kSpinLimit;
    if (c->debug_orphan && !c->capturing &&
        (rc = check_cuda(c, cudaMemsetAsync(&dc->ticket[kTicketCompact], 1, 1, s), "debug ticket")))
        return rc;  // tickets then start at 1: partition 0 is never taken
    c->debug_spin_limit = 0;
    c->debug_orphan = false;
    const uint32_t parts = (ca.num_slots + 1023) / 1024;
    const uint32_t slots = (uint32_t)(c->sm_count * c->bpsm_compact);
    const int cgrid = (int)(parts < slots ? parts : slots);
    launch_compact(ca, cgrid, s);
    return launched(c, "compaction launch", cgrid > 0);
}

int copy_counters(rara_ctx *c, cudaStream_t s)
{
    int rc;
    if ((rc = check_cuda(c, cudaMemcpyAsync(c->h_counters, c->counters.p, sizeof(Counters), cudaMemcpyDeviceToHost, s),
                         "counter copy")))
        return rc;
    return check_cuda(c, cudaMemcpyAsync(c->h_view_counters, c->view_counters_d.p,
                                         sizeof(ViewCounters) * (size_t)c->num_views, cudaMemcpyDeviceToHost, s),
                      "view counter copy");
}

// Buffers that depend on the pair capacity.
int ensure_pairs(rara_ctx *c, uint32_t cap)
{
    const size_t pp = cap > 0 ? (size_t)cap : 1;
    const size_t nn = c->num_slots > 0 ? (size_t)c->num_slots : 1;
    const size_t sb1 = sort_scratch_bytes((int64_t)nn, 4 + c->view_passes);
    const size_t sb2 = sort_scratch_bytes((int64_t)pp, c->tile_passes);
    int rc;
    if ((rc = ensure(c, c->pkeys, pp * 4, "pair keys")) || (rc = ensure(c, c->pvals, pp * 4, "pair values")) ||
        (rc = ensure(c, c->pkeys_b, pp * 4, "pair keys B")) || (rc = ensure(c, c->pvals_b, pp * 4, "pair values B")) ||
        (rc = ensure(c, c->sort_scratch, sb1 > sb2 ? sb1 : sb2, "sort scratch")) ||
        (c->shared_list && (rc = ensure(c, c->list_counts, list_count_words(cap) * 4, "list partition counts"))))
        return rc;
    return RARA_OK;
}

// Stage (b): depth sort, emission, tile sort, ranges, render order. The pair buffers must
// hold cap pairs (ensure_pairs); counts come from the device.
int batch_bin(rara_ctx *c, uint32_t cap, cudaStream_t s)
{
    int rc;
    occupancy_setup(c);
    Counters *dc = (Counters *)c->counters.p;
    uint32_t *hist = (uint32_t *)c->hist.p;
    const size_t nn = c->num_slots > 0 ? (size_t)c->num_slots : 1;
    c->cap_pairs = cap;
    mark(c, 1, s);
    const int sgrid = c->sm_count * c->bpsm_sort;
    const uint32_t ng = c->one_camera ? (uint32_t)(c->h_scenes[0].n > 0 ? c->h_scenes[0].n : 1) : (uint32_t)nn;
    int nl = sort_launch((uint32_t *)c->ckeys.p, (uint32_t *)c->cvals.p, (uint32_t *)c->ckeys_b.p,
                         (uint32_t *)c->cvals_b.p, c->one_camera ? &dc->n_union : &dc->n_rendered, ng,
                         4 + c->view_passes, hist + kHistDepth * 256, c->sort_scratch.p,
                         &dc->ticket[kTicketSortDepth], &dc->status, &dc->depth_in_b, sgrid, s,
                         (const uint32_t *)c->seg_base.p, c->view_passes ? c->num_views : 0, 4);
    if ((rc = launched(c, "depth sort", nl))) return rc;
    if (c->one_camera && !c->shared_list) {
        // every view's rendered slots in (view, depth) order from the one depth order
        if ((rc = check_cuda(c, cudaMemsetAsync(c->lookback_c.p, 0, (nn / 1024 + 2) * 8, s), "memset scan")))
            return rc;
        ExpandArgs xa;
        xa.sorted_a = (const uint32_t *)c->cvals.p;
        xa.sorted_b = (const uint32_t *)c->cvals_b.p;
        xa.out_a = (uint32_t *)c->cvals.p;
        xa.out_b = (uint32_t *)c->cvals_b.p;
        xa.tiles = (const uint32_t *)c->tiles.p;
        xa.views = (const ViewDev *)c->views_d.p;
        xa.num_views = c->num_views;
        xa.lookback = (unsigned long long *)c->lookback_c.p;
        xa.counters = dc;
        const uint32_t xparts = (uint32_t)((nn + 1023) / 1024);
        const uint32_t xslots = (uint32_t)(c->sm_count * c->bpsm_compact);
        launch_expand(xa, (int)(xparts < xslots ? xparts : xslots), s);
        if ((rc = launched(c, "expansion"))) return rc;
    }
    mark(c, 4, s);

    if ((rc = check_cuda(c, cudaMemsetAsync(c->lookback_e.p, 0, (nn / kBlock + 2) * 8, s), "memset emit")))
        return rc;
    EmitArgs e;
    e.keys_a = (const uint32_t *)c->ckeys.p;
    e.vals_a = (const uint32_t *)c->cvals.p;
    e.keys_b = (const uint32_t *)c->ckeys_b.p;
    e.vals_b = (const uint32_t *)c->cvals_b.p;
    e.tiles = (const uint32_t *)c->tiles.p;
    e.erec = (const EmitRec *)c->erec.p;
    e.views = (const ViewDev *)c->views_d.p;
    e.num_views = c->num_views;
    e.cap_pairs = cap;
    e.expanded = c->one_camera && !c->shared_list ? 1 : 0;
    e.shared_list = c->shared_list ? 1 : 0;
    e.vmask = (const uint32_t *)c->vmask.p;
    e.tile_passes = c->tile_passes;
    e.tile_digit_bits = c->tile_digit_bits;
    e.pair_keys = (uint32_t *)c->pkeys.p;
    e.pair_vals = (uint32_t *)c->pvals.p;
    e.tile_hist = hist + kHistTile * 256;
    e.lookback = (unsigned long long *)c->lookback_e.p;
    e.counters = dc;
    launch_emit(e, c->sm_count * c->bpsm_emit, s);
    if ((rc = launched(c, "emit"))) return rc;
    mark(c, 5, s);

    nl = sort_launch((uint32_t *)c->pkeys.p, (uint32_t *)c->pvals.p, (uint32_t *)c->pkeys_b.p,
                     (uint32_t *)c->pvals_b.p, &dc->n_pairs, cap, c->tile_passes, hist + kHistTile * 256, c->sort_scratch.p,
                     &dc->ticket[kTicketSortTile], &dc->status, &dc->tile_in_b, sgrid, s, nullptr, 0, 0,
                     c->tile_digit_bits);
    if ((rc = launched(c, "tile sort", nl))) return rc;
    mark(c, 6, s);

    const size_t nt = c->num_tiles > 0 ? (size_t)c->num_tiles : 1;
    if ((rc = check_cuda(c, cudaMemsetAsync(c->ranges.p, 0, nt * sizeof(int2), s), "memset ranges"))) return rc;
    const uint32_t rblocks = (cap + 255) / 256;
    const uint32_t rmax = (uint32_t)(c->sm_count * 8);
    const int rgrid = (int)(rblocks < rmax ? (rblocks > 0 ? rblocks : 1) : rmax);
    if (c->shared_list) {
        ListArgs la;
        la.keys_a = (const uint32_t *)c->pkeys.p;
        la.keys_b = (const uint32_t *)c->pkeys_b.p;
        la.vals_a = (uint32_t *)c->pvals.p;
        la.vals_b = (uint32_t *)c->pvals_b.p;
        la.vmask = (const uint32_t *)c->vmask.p;
        la.views = (const ViewDev *)c->views_d.p;
        la.num_views = c->num_views;
        la.tile_bits = c->tile_bits;
        la.slot_stride = (uint32_t)c->h_scenes[0].n;
        la.part_counts = (uint32_t *)c->list_counts.p;
        la.max_parts = (cap + kListPart - 1) / kListPart + 1;
        la.ranges = (int2 *)c->ranges.p;
        la.cap_pairs = cap;
        la.counters = dc;
        launch_lists(la, c->sm_count * 8, s);   // a warp per partition of the 40M-pair benchmark list
        if ((rc = launched(c, "shared listing", 3))) return rc;
    } else {
        launch_ranges((const uint32_t *)c->pkeys.p, (const uint32_t *)c->pkeys_b.p, dc, cap, c->num_tiles,
                      (int2 *)c->ranges.p, rgrid, s);
        if ((rc = launched(c, "ranges"))) return rc;
    }
    const int area = c->tile_w * c->tile_h;
    const int area_log2 = area == 64 ? 0 : (area == 256 ? 2 : 3);
    launch_tile_order((const int2 *)c->ranges.p, (int)c->num_tiles, c->split2_bits, c->split4_bits, area_log2,
                      (uint32_t *)c->items.p, dc, (const ViewDev *)c->views_d.p, c->tile_bits, c->sm_count * 2, s);
    return launched(c, "tile order", c->num_tiles > 0 ? 2 : 0);
}

// Stages (c)+(d): the render of every view.
int batch_render(rara_ctx *c, cudaStream_t s)
{
    int rc;
    occupancy_setup(c);
    Counters *dc = (Counters *)c->counters.p;
    mark(c, 2, s);
    if ((rc = check_cuda(c, cudaMemsetAsync(&dc->n_evaluated, 0, kRenderCounterBytes, s), "memset render counters")))
        return rc;
    RenderArgs a;
    a.ranges = (const int2 *)c->ranges.p;
    a.tile_order = (const uint32_t *)c->items.p;
    a.vals_a = (const uint32_t *)c->pvals.p;
    a.vals_b = (const uint32_t *)c->pvals_b.p;
    a.rec = (const SplatRec *)c->rec.p;
    a.cut = (const CutRec *)c->cut.p;
    a.cut_x = c->multi ? (const CutExtra *)c->cut_x.p : nullptr;
    a.views = (const ViewDev *)c->views_d.p;
    a.num_views = c->num_views;
    a.counters = dc;
    const int di = c->blend_depth == 32 ? 0 : (c->blend_depth == 128 ? 1 : (c->blend_depth == 512 ? 3 : 2));
    const long long slots = (long long)c->sm_count * c->bpsm_render[di];
    const long long items = 4ll * c->num_tiles;
    // graph captures run without the work counters (their replays are not read for them)
    if (launch_render(a, (int)(items < slots ? items : slots), s, c->count_work && !c->capturing, c->multi,
                      c->blend_depth))
        return fail(c, RARA_ERR_CUDA, "render: shared-memory size not accepted");
    rc = launched(c, "render launch", c->num_tiles > 0);
    mark(c, 3, s);
    return rc;
}

// Exact binning: wait for the preprocess to know the pair count, size the buffers, launch.
int bin_exact(rara_ctx *c, cudaStream_t s)
{
    int rc;
    if ((rc = check_cuda(c, cudaStreamSynchronize(s), "cudaStreamSynchronize"))) return rc;
    if ((rc = device_status(c, c->h_counters->status))) {
        c->stage = 0;
        return rc;
    }
    const unsigned long long np = c->h_counters->n_pairs;
    if (np >= (1ull << 30)) return fail(c, RARA_ERR_BUDGET, "%llu pairs exceed 2^30", np);
    const uint32_t cap = (uint32_t)(np > 0 ? np : 1);
    if ((rc = ensure_pairs(c, cap))) return rc;
    return batch_bin(c, cap, s);
}

void free_host(rara_ctx *c)
{
    if (!c->owns_host) return;
    for (Staging &st : c->staging) {
        if (st.views) cudaFreeHost(st.views);
        if (st.scenes) cudaFreeHost(st.scenes);
        if (st.uploaded) cudaEventDestroy(st.uploaded);
    }
    if (c->h_bviews) cudaFreeHost(c->h_bviews);
    if (c->h_bscenes) cudaFreeHost(c->h_bscenes);
    if (c->bwd_uploaded) cudaEventDestroy(c->bwd_uploaded);
    if (c->h_lviews) cudaFreeHost(c->h_lviews);
    if (c->loss_uploaded) cudaEventDestroy(c->loss_uploaded);
    for (cudaEvent_t &e : c->bev)
        if (e) cudaEventDestroy(e);
    if (c->h_counters) cudaFreeHost(c->h_counters);
    if (c->h_view_counters) cudaFreeHost(c->h_view_counters);
    free(c->h_view_map);
    free(c->h_view_n);
    free(c->shape);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t &e : c->ev)
        if (e) cudaEventDestroy(e);
}

}  // namespace

extern "C" {

int rara_ctx_create(size_t budget_bytes, int32_t tile_w, int32_t tile_h, rara_ctx **out)
{
    if (!out) return RARA_ERR_INVALID_ARG;
    *out = nullptr;
    if (!tile_shape_ok(tile_w, tile_h)) return RARA_ERR_INVALID_ARG;
    rara_ctx *c = new (std::nothrow) rara_ctx();
    if (!c) return RARA_ERR_BUDGET;
    c->budget = budget_bytes;
    c->tile_w = tile_w;
    c->tile_h = tile_h;
    cudaGetDevice(&c->device);
    c->max_views = kMaxViews;
    c->max_scenes = kMaxScenes;
    bool ok = ensure(c, c->counters, sizeof(Counters), "counters") == RARA_OK;
    for (Staging &st : c->staging) {
        ok = ok && cudaHostAlloc((void **)&st.views, sizeof(ViewDev) * kMaxViews, cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaHostAlloc((void **)&st.scenes, sizeof(SceneDev) * kMaxScenes, cudaHostAllocDefault) ==
                       cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&st.uploaded, cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaHostAlloc((void **)&c->h_counters, sizeof(Counters), cudaHostAllocDefault) == cudaSuccess;
    ok = ok && cudaHostAlloc((void **)&c->h_view_counters, sizeof(ViewCounters) * kMaxViews, cudaHostAllocDefault) ==
                   cudaSuccess;
    c->h_view_map = (int *)malloc(sizeof(int) * kMaxViews);
    c->h_view_n = (int *)malloc(sizeof(int) * kMaxViews);
    ok = ok && c->h_view_map && c->h_view_n;
    for (cudaEvent_t &e : c->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    ok = ok && cudaHostAlloc((void **)&c->h_bviews, sizeof(BwdView) * kMaxViews, cudaHostAllocDefault) == cudaSuccess;
    ok = ok && cudaHostAlloc((void **)&c->h_bscenes, sizeof(BwdScene) * kMaxScenes, cudaHostAllocDefault) ==
                   cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->bwd_uploaded, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaHostAlloc((void **)&c->h_lviews, sizeof(LossView) * kMaxViews, cudaHostAllocDefault) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->loss_uploaded, cudaEventDisableTiming) == cudaSuccess;
    for (cudaEvent_t &e : c->bev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(c, c->counters);
        free_host(c);
        delete c;
        return RARA_ERR_CUDA;
    }
    memset(c->h_counters, 0, sizeof(Counters));
    *out = c;
    return RARA_OK;
}

int rara_ctx_destroy(rara_ctx *c)
{
    if (!c) return RARA_OK;
    cudaDeviceSynchronize();
    DevBuf *all[] = {&c->views_d, &c->scenes_d, &c->view_counters_d, &c->counters, &c->labels, &c->tiles,
                     &c->erec, &c->rec, &c->cut, &c->cut_x, &c->depth, &c->ckeys, &c->cvals, &c->ckeys_b, &c->cvals_b,
                     &c->lookback_c, &c->pkeys, &c->pvals, &c->pkeys_b, &c->pvals_b, &c->lookback_e, &c->hist,
                     &c->ranges, &c->items, &c->sort_scratch, &c->grec, &c->bviews_d, &c->bscenes_d,
                     &c->seg_base, &c->export_off, &c->gkey, &c->vmask, &c->list_counts, &c->lviews_d};
    for (DevBuf *b : all) release(c, *b);
    free_host(c);
    delete c;
    return RARA_OK;
}

const char *rara_last_error(const rara_ctx *c) { return c ? c->err : "null context"; }

size_t rara_ctx_bytes(const rara_ctx *c) { return c ? c->held : 0; }

int64_t rara_ctx_launches(const rara_ctx *c) { return c ? c->launches : 0; }

int rara_ctx_stage_ms(rara_ctx *c, float out[3])
{
    if (!c || !out) return RARA_ERR_INVALID_ARG;
    if (!c->ev[0]) return fail(c, RARA_ERR_INVALID_ARG, "no stage timing on this context");
    int rc = check_cuda(c, cudaEventSynchronize(c->ev[3]), "event wait");
    if (rc) return rc;
    for (int k = 0; k < 3; ++k)
        if ((rc = check_cuda(c, cudaEventElapsedTime(&out[k], c->ev[k], c->ev[k + 1]), "event elapsed time")))
            return rc;
    return RARA_OK;
}

int rara_ctx_reserve(rara_ctx *c, int64_t slots, int64_t pairs, int32_t views, int32_t max_view_tiles)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (!c->owns_host) return fail(c, RARA_ERR_INVALID_ARG, "the static context cannot reserve");
    if (slots < 0 || slots >= ((int64_t)1 << 32) - 1 || pairs < 0 || pairs >= ((int64_t)1 << 30) || views < 1 ||
        views > c->max_views || max_view_tiles < 1)
        return fail(c, RARA_ERR_INVALID_ARG, "reserve(%lld slots, %lld pairs, %d views, %d tiles) out of range",
                    (long long)slots, (long long)pairs, views, max_view_tiles);
    const uint64_t tiles = (uint64_t)views << ceil_bits((uint32_t)max_view_tiles);
    if (tiles >= ((uint64_t)1 << 28)) return fail(c, RARA_ERR_INVALID_ARG, "%llu tiles exceed 2^28",
                                                   (unsigned long long)tiles);
    const size_t nn = slots > 0 ? (size_t)slots : 1, pp = pairs > 0 ? (size_t)pairs : 1, nt = (size_t)tiles;
    const size_t sb1 = sort_scratch_bytes((int64_t)nn, 6), sb2 = sort_scratch_bytes((int64_t)pp, 4);
    int rc;
    if ((rc = ensure(c, c->views_d, sizeof(ViewDev) * (size_t)views, "view table")) ||
        (rc = ensure(c, c->scenes_d, sizeof(SceneDev) * (size_t)c->max_scenes, "scene table")) ||
        (rc = ensure(c, c->view_counters_d, sizeof(ViewCounters) * (size_t)views, "view counters")) ||
        (rc = ensure(c, c->labels, nn, "labels")) || (rc = ensure(c, c->tiles, nn * 4, "tiles")) ||
        (rc = ensure(c, c->erec, nn * sizeof(EmitRec), "emission records")) || (rc = ensure(c, c->rec, nn * sizeof(SplatRec), "records")) ||
        (rc = ensure(c, c->cut, nn * sizeof(CutRec), "cutoff records")) ||
        (rc = ensure(c, c->depth, nn * 4, "depth")) || (rc = ensure(c, c->ckeys, nn * 4, "depth keys")) ||
        (rc = ensure(c, c->cvals, nn * 4, "depth values")) || (rc = ensure(c, c->ckeys_b, nn * 4, "depth keys B")) ||
        (rc = ensure(c, c->cvals_b, nn * 4, "depth values B")) ||
        (rc = ensure(c, c->lookback_c, (nn / 1024 + 2) * 8, "compaction scan words")) ||
        (rc = ensure(c, c->lookback_e, (nn / kBlock + 2) * 8, "emission scan words")) ||
        (rc = ensure(c, c->hist, kHistPasses * 256 * 4, "digit histograms")) ||
        (rc = ensure(c, c->seg_base, sizeof(uint32_t) * (size_t)views, "view slot bases")) ||
        (rc = ensure(c, c->ranges, nt * sizeof(int2), "ranges")) || (rc = ensure(c, c->items, nt * 16, "render items")) ||
        (rc = ensure(c, c->pkeys, pp * 4, "pair keys")) || (rc = ensure(c, c->pvals, pp * 4, "pair values")) ||
        (rc = ensure(c, c->pkeys_b, pp * 4, "pair keys B")) || (rc = ensure(c, c->pvals_b, pp * 4, "pair values B")) ||
        (rc = ensure(c, c->sort_scratch, sb1 > sb2 ? sb1 : sb2, "sort scratch")))
        return rc;
    return RARA_OK;
}

int rara_ctx_debug_waits(rara_ctx *c, int32_t spin_limit, int32_t orphan_first_partition)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (spin_limit < 0) return fail(c, RARA_ERR_INVALID_ARG, "spin_limit %d < 0", spin_limit);
    c->debug_spin_limit = spin_limit;
    c->debug_orphan = orphan_first_partition != 0;
    return RARA_OK;
}

int rara_ctx_count_work(rara_ctx *c, int32_t on)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->count_work = on != 0;
    return RARA_OK;
}

int rara_ctx_set_tiling(rara_ctx *c, int32_t tile_w, int32_t tile_h, int32_t blend_depth)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (!tile_shape_ok(tile_w, tile_h))
        return fail(c, RARA_ERR_INVALID_ARG, "tile %dx%d is not one of 8x8, 16x16, 32x8, 8x32, 32x16, 16x32", tile_w,
                    tile_h);
    if (!batch_depth_ok(blend_depth))
        return fail(c, RARA_ERR_INVALID_ARG, "blend batch depth %d is not 32, 128, 256 or 512", blend_depth);
    if (!c->owns_host && (tile_w != kTile || tile_h != kTile || blend_depth != kBlock))
        return fail(c, RARA_ERR_INVALID_ARG, "the static context keeps 16x16 tiles and 256-entry batches");
    if (tile_w != c->tile_w || tile_h != c->tile_h) {
        c->stage = 0;          // the current frame's tiles no longer apply
        c->rendered = false;
    }
    c->tile_w = tile_w;
    c->tile_h = tile_h;
    c->blend_depth = blend_depth;
    c->shape_len = 0;          // a captured graph holds the old tiling: recapture
    return RARA_OK;
}

int rara_ctx_set_tuning(rara_ctx *c, int32_t split2_bits, int32_t split4_bits)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->split2_bits = split2_bits < 0 ? 0 : (split2_bits > 33 ? 33 : split2_bits);
    c->split4_bits = split4_bits < 0 ? 0 : (split4_bits > 33 ? 33 : split4_bits);
    c->shape_len = 0;  // a captured graph holds the old values: recapture
    return RARA_OK;
}

int rara_ctx_sync(rara_ctx *c, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = check_cuda(c, cudaMemcpyAsync(c->h_counters, c->counters.p, sizeof(Counters),
                                           cudaMemcpyDeviceToHost, s), "counter copy");
    if (rc) return rc;
    rc = check_cuda(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (rc) return rc;
    if ((rc = device_status(c, c->h_counters->status))) return rc;
    if (c->h_counters->status & kStatusOverflow) {
        const unsigned long long np = c->h_counters->n_pairs;
        const unsigned long long want = np + np / 4 + 4096;
        c->min_cap_pairs = (uint32_t)(want < (1ull << 30) ? want : (1ull << 30) - 1);
        c->shape_len = 0;  // recapture with the larger capacity
        return fail(c, RARA_ERR_OVERFLOW, "%llu pairs exceeded the captured capacity %u; render the batch again", np,
                    c->cap_pairs);
    }
    return RARA_OK;
}

int rara_preprocess(rara_ctx *c, const rara_gaussians *g, const rara_camera *cam, const rara_plane *pl,
                    void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->err[0] = 0;
    c->stage = 0;
    if (!g || !cam || !pl) return fail(c, RARA_ERR_INVALID_ARG, "null argument");
    rara_view v;
    memset(&v, 0, sizeof(v));
    v.scene = 0;
    v.camera = *cam;
    v.plane = *pl;
    v.image = (float *)1;  // placeholder checked by batch_setup; rara_render supplies the outputs
    cudaStream_t s = (cudaStream_t)stream;
    int rc = batch_setup(c, g, 1, &v, 1, s);
    if (rc) return rc;
    if ((rc = batch_preprocess(c, s))) return rc;
    if ((rc = copy_counters(c, s))) return rc;
    c->last_stream = s;
    c->stage = 1;
    return RARA_OK;
}

int rara_bin(rara_ctx *c, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (c->stage < 1) return fail(c, RARA_ERR_INVALID_ARG, "rara_bin called before rara_preprocess");
    // The counter copy was queued by rara_preprocess on its stream; wait for that stream.
    int rc = check_cuda(c, cudaStreamSynchronize(c->last_stream), "cudaStreamSynchronize");
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = bin_exact(c, s))) return rc;
    c->last_stream = s;
    c->stage = 2;
    return RARA_OK;
}

int rara_render(rara_ctx *c, const float bg[3], float *image, float *final_T, uint32_t *n_contrib, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (c->stage < 2) return fail(c, RARA_ERR_INVALID_ARG, "rara_render called before rara_bin");
    if (!bg || !image) return fail(c, RARA_ERR_INVALID_ARG, "null bg or image");
    if (c->num_views != 1) return fail(c, RARA_ERR_INVALID_ARG, "rara_render follows a single-view rara_preprocess");
    cudaStream_t s = (cudaStream_t)stream;
    // The staging copy holding this view was uploaded by rara_preprocess, which rara_bin
    // waited for; refill its output fields and upload the view again.
    ViewDev &v = c->h_views[0];
    for (int j = 0; j < 3; ++j) v.bg[j] = bg[j];
    v.image = image;
    v.final_T = final_T;
    v.n_contrib = n_contrib;
    int rc = check_cuda(c, cudaMemcpyAsync(c->views_d.p, c->h_views, sizeof(ViewDev), cudaMemcpyHostToDevice, s),
                        "view table upload");
    if (rc) return rc;
    Staging &st = c->staging[c->staging_next ^ 1];  // the copy that holds h_views
    if (st.uploaded && (rc = check_cuda(c, cudaEventRecord(st.uploaded, s), "staging event"))) return rc;
    if ((rc = batch_render(c, s))) return rc;
    c->last_stream = s;
    c->rendered = true;
    return RARA_OK;
}

int rara_render_frame(rara_ctx *c, const rara_gaussians *g, const rara_camera *cam, const rara_plane *plane,
                      const float bg[3], float *image, float *final_T, uint32_t *n_contrib, void *stream)
{
    int rc = rara_preprocess(c, g, cam, plane, stream);
    if (rc) return rc;
    rc = rara_bin(c, stream);
    if (rc) return rc;
    return rara_render(c, bg, image, final_T, n_contrib, stream);
}

int rara_render_batch(rara_ctx *c, const rara_gaussians *scenes, int32_t num_scenes, const rara_view *views,
                      int32_t num_views, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (!scenes || !views) return fail(c, RARA_ERR_INVALID_ARG, "null scenes or views");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = batch_setup(c, scenes, num_scenes, views, num_views, s))) return rc;
    if ((rc = batch_preprocess(c, s))) return rc;
    if ((rc = copy_counters(c, s))) return rc;
    if ((rc = bin_exact(c, s))) return rc;
    if ((rc = batch_render(c, s))) return rc;
    c->last_stream = s;
    c->stage = 2;
    c->rendered = true;
    return RARA_OK;
}

int rara_render_batch_graph(rara_ctx *c, const rara_gaussians *scenes, int32_t num_scenes, const rara_view *views,
                            int32_t num_views, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (!scenes || !views || num_scenes < 1 || num_views < 1 || num_scenes > c->max_scenes ||
        num_views > c->max_views)
        return fail(c, RARA_ERR_INVALID_ARG, "bad batch (%d scenes, %d views)", num_scenes, num_views);
    if (!c->owns_host) return fail(c, RARA_ERR_INVALID_ARG, "graph batches need a regular context");
    // batch shape: scene sizes and degrees, views' scene and resolution, and whether a view
    // clips by a convex volume (the render kernel's variant and buffers depend on it)
    const size_t len = 4 + 2 * (size_t)num_scenes + 3 * (size_t)num_views;
    int *shape = (int *)malloc(sizeof(int) * len);
    if (!shape) return fail(c, RARA_ERR_BUDGET, "host allocation failed");
    size_t k = 0;
    shape[k++] = num_scenes;
    shape[k++] = num_views;
    int multi = 0;
    for (int v = 0; v < num_views; ++v)
        multi |= views[v].plane.n_extra > 0 &&
                 (views[v].plane.mode == RARA_MODE_RARA || views[v].plane.mode == RARA_MODE_RARA_ALL);
    shape[k++] = multi;
    shape[k++] = one_camera_batch(num_scenes, views, num_views) ? 1 : 0;  // the depth order's kernels differ
    for (int i = 0; i < num_scenes; ++i) {
        shape[k++] = (int)scenes[i].n;
        shape[k++] = scenes[i].sh_degree;
    }
    for (int v = 0; v < num_views; ++v) {
        shape[k++] = views[v].scene;
        shape[k++] = views[v].camera.width;
        shape[k++] = views[v].camera.height;
    }
    const bool same = c->graph && c->shape && c->shape_len == len && memcmp(c->shape, shape, sizeof(int) * len) == 0;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if (same) {
        free(shape);
        if ((rc = batch_setup(c, scenes, num_scenes, views, num_views, s))) return rc;
        c->cap_pairs = c->graph_cap_pairs;
        if ((rc = check_cuda(c, cudaGraphLaunch(c->graph, s), "cudaGraphLaunch"))) return rc;
        c->launches += c->graph_kernels;
        c->last_stream = s;
        c->stage = 2;
        c->rendered = true;
        return RARA_OK;
    }
    // First batch of this shape: render it exactly, then capture the stage sequence.
    if ((rc = rara_render_batch(c, scenes, num_scenes, views, num_views, stream))) {
        free(shape);
        return rc;
    }
    // the batch rendered above must finish before its buffers grow
    rc = check_cuda(c, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const unsigned long long np = c->h_counters->n_pairs;
    unsigned long long cap = np + np / 4 + 4096;
    if (cap < c->min_cap_pairs) cap = c->min_cap_pairs;
    if (cap >= (1ull << 30)) cap = (1ull << 30) - 1;
    if (!rc) rc = ensure_pairs(c, (uint32_t)cap);
    if (!rc && !c->cap_stream)
        rc = check_cuda(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
    if (rc) {
        free(shape);
        return rc;
    }
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    const int64_t launches0 = c->launches;
    cudaGraph_t g = nullptr;
    c->capturing = true;
    rc = check_cuda(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (!rc) {
        int rc2 = batch_preprocess(c, c->cap_stream);
        if (!rc2) rc2 = batch_bin(c, (uint32_t)cap, c->cap_stream);
        if (!rc2) rc2 = batch_render(c, c->cap_stream);
        if (!rc2)
            rc2 = check_cuda(c, cudaMemcpyAsync(c->h_counters, c->counters.p, sizeof(Counters), cudaMemcpyDeviceToHost,
                                                c->cap_stream), "counter copy");
        rc = check_cuda(c, cudaStreamEndCapture(c->cap_stream, &g), "end capture");
        if (rc2) rc = rc2;
    }
    c->capturing = false;
    c->graph_kernels = c->launches - launches0;
    c->launches = launches0;  // capturing launches nothing
    if (!rc) rc = check_cuda(c, cudaGraphInstantiate(&c->graph, g, 0), "graph instantiate");
    if (g) cudaGraphDestroy(g);
    if (rc) {
        free(shape);
        c->graph = nullptr;
        return rc;
    }
    free(c->shape);
    c->shape = shape;
    c->shape_len = len;
    c->graph_cap_pairs = (uint32_t)cap;
    // The pair buffers may have grown for the capture, which drops the exact render's pairs:
    // replay once so the batch's intermediate state matches its outputs again (a backward
    // may follow).
    c->rendered = false;
    if ((rc = check_cuda(c, cudaGraphLaunch(c->graph, s), "cudaGraphLaunch"))) return rc;
    c->launches += c->graph_kernels;
    c->cap_pairs = c->graph_cap_pairs;
    c->rendered = true;
    return RARA_OK;
}

int rara_render_backward(rara_ctx *c, const float *const *dL_dimages, const rara_gaussian_grads *grads,
                         float *plane_grads, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (!c->owns_host) return fail(c, RARA_ERR_INVALID_ARG, "the static context has no backward");
    if (!c->rendered || c->stage < 2)
        return fail(c, RARA_ERR_INVALID_ARG, "rara_render_backward needs a rendered frame or batch on this context");
    if (!dL_dimages || !grads) return fail(c, RARA_ERR_INVALID_ARG, "null dL_dimages or grads");
    if (c->extra_planes)
        return fail(c, RARA_ERR_INVALID_ARG, "the backward supports single clip planes (a view has n_extra > 0)");
    for (int v = 0; v < c->num_views; ++v) {
        if (!dL_dimages[v]) return fail(c, RARA_ERR_INVALID_ARG, "view %d has no dL/dimage", v);
        const ViewDev &vd = c->h_views[c->h_view_map[v]];
        if (!vd.final_T || !vd.n_contrib)
            return fail(c, RARA_ERR_INVALID_ARG, "view %d was rendered without final_T and n_contrib", v);
    }
    for (int si = 0; si < c->num_scenes; ++si) {
        const rara_gaussian_grads &g = grads[si];
        if (c->h_scenes[si].n > 0 && (!g.means || !g.log_scales || !g.quats || !g.opacity_logits || !g.sh))
            return fail(c, RARA_ERR_INVALID_ARG, "scene %d has a null gradient array", si);
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    occupancy_setup(c);
    // the pinned tables are refilled only after their last upload has been read
    if ((rc = check_cuda(c, cudaEventSynchronize(c->bwd_uploaded), "backward table wait"))) return rc;
    int max_degree = 0;
    for (int v = 0; v < c->num_views; ++v) {
        BwdView &b = c->h_bviews[c->h_view_map[v]];
        b.dimage = dL_dimages[v];
        b.plane_grad = plane_grads ? plane_grads + 4 * (size_t)v : nullptr;
    }
    for (int si = 0; si < c->num_scenes; ++si) {
        const rara_gaussian_grads &g = grads[si];
        BwdScene &b = c->h_bscenes[si];
        b.means = g.means; b.log_scales = g.log_scales; b.quats = g.quats; b.logits = g.opacity_logits; b.sh = g.sh;
        if (c->h_scenes[si].view_count > 0 && c->h_scenes[si].sh_degree > max_degree)
            max_degree = c->h_scenes[si].sh_degree;
    }
    const size_t nn = c->num_slots > 0 ? (size_t)c->num_slots : 1;
    rc = ensure(c, c->grec, nn * sizeof(GradRec), "gradient records");
    if (rc ||
        (rc = ensure(c, c->bviews_d, sizeof(BwdView) * (size_t)c->num_views, "backward view table")) ||
        (rc = ensure(c, c->bscenes_d, sizeof(BwdScene) * (size_t)c->num_scenes, "backward scene table")))
        return rc;
    if ((rc = check_cuda(c, cudaMemcpyAsync(c->bviews_d.p, c->h_bviews, sizeof(BwdView) * (size_t)c->num_views,
                                            cudaMemcpyHostToDevice, s), "backward view table upload")) ||
        (rc = check_cuda(c, cudaMemcpyAsync(c->bscenes_d.p, c->h_bscenes, sizeof(BwdScene) * (size_t)c->num_scenes,
                                            cudaMemcpyHostToDevice, s), "backward scene table upload")) ||
        (rc = check_cuda(c, cudaEventRecord(c->bwd_uploaded, s), "backward table event")))
        return rc;
    Counters *dc = (Counters *)c->counters.p;
    // The records are cleared in full only when the buffer is new or the last backward did not
    // complete both launches; otherwise the last preprocess backward left them zero.
    if (!(c->grec_zero && c->grec_zero_gen == c->grec.gen) &&
        (rc = check_cuda(c, cudaMemsetAsync(c->grec.p, 0, c->grec.cap, s), "memset gradient records")))
        return rc;
    c->grec_zero = false;
    if ((rc = check_cuda(c, cudaMemsetAsync(&dc->bwd_queue, 0, sizeof(unsigned int), s), "memset queue")))
        return rc;
    if (plane_grads &&
        (rc = check_cuda(c, cudaMemsetAsync(plane_grads, 0, sizeof(float) * 4 * (size_t)c->num_views, s),
                         "memset plane gradients")))
        return rc;
    cudaEventRecord(c->bev[0], s);
    RenderBwdArgs ra;
    ra.ranges = (const int2 *)c->ranges.p;
    ra.tile_order = (const uint32_t *)c->items.p;
    ra.vals_a = (const uint32_t *)c->pvals.p;
    ra.vals_b = (const uint32_t *)c->pvals_b.p;
    ra.rec = (const SplatRec *)c->rec.p;
    ra.cut = (const CutRec *)c->cut.p;
    ra.views = (const ViewDev *)c->views_d.p;
    ra.bviews = (const BwdView *)c->bviews_d.p;
    ra.num_views = c->num_views;
    ra.grec = (GradRec *)c->grec.p;
    ra.counters = dc;
    const long long slots = (long long)c->sm_count * c->bpsm_render_bwd;
    const long long items = 4ll * c->num_tiles;
    launch_render_bwd(ra, (int)(items < slots ? items : slots), s);
    if ((rc = launched(c, "render backward launch", c->num_tiles > 0))) return rc;
    cudaEventRecord(c->bev[1], s);
    PreprocessBwdArgs pa;
    pa.scenes = (const SceneDev *)c->scenes_d.p;
    pa.num_scenes = c->num_scenes;
    pa.views = (const ViewDev *)c->views_d.p;
    pa.bviews = (const BwdView *)c->bviews_d.p;
    pa.bscenes = (const BwdScene *)c->bscenes_d.p;
    pa.labels = (const uint8_t *)c->labels.p;
    pa.tiles = (const uint32_t *)c->tiles.p;
    pa.grec = (GradRec *)c->grec.p;
    if (launch_preprocess_bwd(pa, (int)c->num_units, max_degree, s))
        return fail(c, RARA_ERR_CUDA, "preprocess backward: shared-memory size not accepted");
    if ((rc = launched(c, "preprocess backward launch", c->num_units > 0))) return rc;
    c->grec_zero = true;
    c->grec_zero_gen = c->grec.gen;
    // Gaussians of scenes without views get zero gradients
    for (int si = 0; si < c->num_scenes; ++si) {
        const SceneDev &sd = c->h_scenes[si];
        if (sd.view_count > 0 || sd.n == 0) continue;
        const rara_gaussian_grads &g = grads[si];
        const size_t n = (size_t)sd.n, K = (size_t)(sd.sh_degree + 1) * (sd.sh_degree + 1);
        if ((rc = check_cuda(c, cudaMemsetAsync(g.means, 0, 12 * n, s), "memset gradients")) ||
            (rc = check_cuda(c, cudaMemsetAsync(g.log_scales, 0, 12 * n, s), "memset gradients")) ||
            (rc = check_cuda(c, cudaMemsetAsync(g.quats, 0, 16 * n, s), "memset gradients")) ||
            (rc = check_cuda(c, cudaMemsetAsync(g.opacity_logits, 0, 4 * n, s), "memset gradients")) ||
            (rc = check_cuda(c, cudaMemsetAsync(g.sh, 0, 12 * K * n, s), "memset gradients")))
            return rc;
    }
    cudaEventRecord(c->bev[2], s);
    c->last_stream = s;
    return RARA_OK;
}

int rara_loss_l2(rara_ctx *c, const float *const *targets, float *const *dL_dimages, const float *scale,
                 double *loss, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (!c->owns_host) return fail(c, RARA_ERR_INVALID_ARG, "the static context has no loss");
    if (!c->rendered || c->stage < 2)
        return fail(c, RARA_ERR_INVALID_ARG, "rara_loss_l2 needs a rendered frame or batch on this context");
    if (!targets || !dL_dimages || !scale || !loss) return fail(c, RARA_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    // the pinned table is refilled only after its last upload has been read
    if ((rc = check_cuda(c, cudaEventSynchronize(c->loss_uploaded), "loss table wait"))) return rc;
    uint64_t chunks = 0;
    for (int v = 0; v < c->num_views; ++v) {
        if (!targets[v] || !dL_dimages[v]) return fail(c, RARA_ERR_INVALID_ARG, "view %d has a null target or gradient", v);
        if (!finite(scale[v])) return fail(c, RARA_ERR_INVALID_ARG, "view %d has a non-finite scale", v);
        const ViewDev &vd = c->h_views[c->h_view_map[v]];
        if (dL_dimages[v] == vd.image)
            return fail(c, RARA_ERR_INVALID_ARG, "view %d: the gradient output is the rendered image", v);
        const uint64_t n = 3ull * (uint64_t)vd.cam.W * (uint64_t)vd.cam.H;
        if (n > 0xffffffffull) return fail(c, RARA_ERR_INVALID_ARG, "view %d has more than 2^32 image elements", v);
        LossView &l = c->h_lviews[v];
        l.image = vd.image;
        l.target = targets[v];
        l.dimage = dL_dimages[v];
        l.loss = loss + v;
        l.scale = scale[v];
        l.n = (uint32_t)n;
        l.chunk_begin = (uint32_t)chunks;
        l.pad = 0;
        chunks += (n + kLossChunk - 1) / kLossChunk;
    }
    if (chunks > 0x7fffffffull) return fail(c, RARA_ERR_INVALID_ARG, "the batch's images need too many blocks");
    if ((rc = ensure(c, c->lviews_d, sizeof(LossView) * (size_t)(c->num_views > 0 ? c->num_views : 1), "loss view table")) ||
        (rc = check_cuda(c, cudaMemcpyAsync(c->lviews_d.p, c->h_lviews, sizeof(LossView) * (size_t)c->num_views,
                                            cudaMemcpyHostToDevice, s), "loss view table upload")) ||
        (rc = check_cuda(c, cudaEventRecord(c->loss_uploaded, s), "loss table event")) ||
        (rc = check_cuda(c, cudaMemsetAsync(loss, 0, sizeof(double) * (size_t)c->num_views, s), "memset loss")))
        return rc;
    launch_loss_l2((const LossView *)c->lviews_d.p, c->num_views, (uint32_t)chunks, s);
    return launched(c, "loss launch", chunks > 0 && c->num_views > 0);
}

int rara_ctx_backward_ms(rara_ctx *c, float out[2])
{
    if (!c || !out) return RARA_ERR_INVALID_ARG;
    if (!c->bev[0]) return fail(c, RARA_ERR_INVALID_ARG, "no backward timing on this context");
    int rc = check_cuda(c, cudaEventSynchronize(c->bev[2]), "event wait");
    if (rc) return rc;
    for (int k = 0; k < 2; ++k)
        if ((rc = check_cuda(c, cudaEventElapsedTime(&out[k], c->bev[k], c->bev[k + 1]), "event elapsed time")))
            return rc;
    return RARA_OK;
}

int rara_ctx_kernel_ms(rara_ctx *c, float out[6])
{
    if (!c || !out) return RARA_ERR_INVALID_ARG;
    if (!c->ev[0]) return fail(c, RARA_ERR_INVALID_ARG, "no stage timing on this context");
    int rc = check_cuda(c, cudaEventSynchronize(c->ev[3]), "event wait");
    if (rc) return rc;
    // preprocess, compaction, depth sort, emission, tile sort, ranges and render order
    const int from[6] = {0, 7, 1, 4, 5, 6}, to[6] = {7, 1, 4, 5, 6, 2};
    for (int k = 0; k < 6; ++k)
        if ((rc = check_cuda(c, cudaEventElapsedTime(&out[k], c->ev[from[k]], c->ev[to[k]]), "event elapsed time")))
            return rc;
    return RARA_OK;
}

int rara_frame_info_get(rara_ctx *c, int32_t view, rara_frame_info *out)
{
    if (!c || !out) return RARA_ERR_INVALID_ARG;
    if (c->stage < 2) return fail(c, RARA_ERR_INVALID_ARG, "no binned frame");
    if (view < 0 || view >= c->num_views) return fail(c, RARA_ERR_INVALID_ARG, "view %d of %d", view, c->num_views);
    int rc = rara_ctx_sync(c, c->last_stream);
    if (rc) return rc;
    if ((rc = check_cuda(c, cudaMemcpy(c->h_view_counters, c->view_counters_d.p,
                                       sizeof(ViewCounters) * (size_t)c->num_views, cudaMemcpyDeviceToHost),
                         "view counter copy")))
        return rc;
    const int k = c->h_view_map[view];
    const ViewDev &v = c->h_views[k];
    out->n = c->h_view_n[k];
    out->n_rendered = (int64_t)c->h_view_counters[k].n_rendered;
    out->n_cutoff = (int64_t)c->h_view_counters[k].n_cutoff;
    // pairs the binning listed: the sum of the view's tile-list lengths
    const int nt = v.tiles_x * v.tiles_y;
    int2 *hr = (int2 *)malloc(sizeof(int2) * (size_t)(nt > 0 ? nt : 1));
    if (!hr) return fail(c, RARA_ERR_BUDGET, "host allocation failed");
    rc = check_cuda(c, cudaMemcpy(hr, (const int2 *)c->ranges.p + v.tile_base, sizeof(int2) * (size_t)nt,
                                  cudaMemcpyDeviceToHost), "ranges copy");
    int64_t np = 0;
    for (int t = 0; t < nt && !rc; ++t)
        if (hr[t].y > hr[t].x) np += hr[t].y - hr[t].x;
    free(hr);
    if (rc) return rc;
    out->n_pairs = np;
    out->tiles_x = v.tiles_x;
    out->tiles_y = v.tiles_y;
    out->n_evaluated = (int64_t)c->h_counters->n_evaluated;
    out->n_walked = (int64_t)c->h_counters->n_walked;
    out->n_cut_evaluated = (int64_t)c->h_counters->n_cut_evaluated;
    out->n_tested = (int64_t)c->h_counters->n_tested;
    out->n_pair_candidates = (int64_t)c->h_view_counters[k].n_pairs;
    out->n_depth_keys = (int64_t)(c->one_camera ? c->h_counters->n_union : c->h_counters->n_rendered);
    out->n_shared_pairs = c->shared_list ? (int64_t)c->h_counters->n_list : 0;
    return RARA_OK;
}

int rara_frame_gaussians(rara_ctx *c, int32_t view, uint8_t *labels, float *depth, float *mean2d, float *conic,
                         float *rgb, float *opacity, int32_t *rect, uint32_t *tiles, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (c->stage < 1) return fail(c, RARA_ERR_INVALID_ARG, "no preprocessed frame");
    if (view < 0 || view >= c->num_views) return fail(c, RARA_ERR_INVALID_ARG, "view %d of %d", view, c->num_views);
    const int k = c->h_view_map[view];
    launch_export_gaussians(c->h_view_n[k], c->h_views[k].slot_base, (const uint8_t *)c->labels.p,
                            (const uint32_t *)c->tiles.p, (const EmitRec *)c->erec.p,
                            c->shared_list ? (const uint32_t *)c->vmask.p : nullptr, (const ViewDev *)c->views_d.p,
                            (const SplatRec *)c->rec.p,
                            (const float *)c->depth.p, labels, depth, mean2d, conic, rgb, opacity, rect, tiles,
                            (cudaStream_t)stream);
    return launched(c, "export gaussians", c->h_view_n[k] > 0);
}

int rara_frame_pairs(rara_ctx *c, int32_t view, uint64_t *keys, uint32_t *values, int64_t *ranges, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (c->stage < 2) return fail(c, RARA_ERR_INVALID_ARG, "no binned frame");
    if (view < 0 || view >= c->num_views) return fail(c, RARA_ERR_INVALID_ARG, "view %d of %d", view, c->num_views);
    const int k = c->h_view_map[view];
    const ViewDev &v = c->h_views[k];
    const int nt = v.tiles_x * v.tiles_y;
    int rc = rara_ctx_sync(c, c->last_stream);
    if (rc) return rc;
    // the view's lists, in local tile order: output offsets from the list lengths
    int2 *hr = (int2 *)malloc(sizeof(int2) * (size_t)(nt > 0 ? nt : 1));
    uint32_t *ho = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nt > 0 ? nt : 1));
    if (!hr || !ho) {
        free(hr);
        free(ho);
        return fail(c, RARA_ERR_BUDGET, "host allocation failed");
    }
    rc = check_cuda(c, cudaMemcpy(hr, (const int2 *)c->ranges.p + v.tile_base, sizeof(int2) * (size_t)nt,
                                  cudaMemcpyDeviceToHost), "ranges copy");
    uint32_t acc = 0;
    for (int t = 0; t < nt && !rc; ++t) {
        ho[t] = acc;
        if (hr[t].y > hr[t].x) acc += (uint32_t)(hr[t].y - hr[t].x);
    }
    if (!rc) rc = ensure(c, c->export_off, sizeof(uint32_t) * (size_t)(nt > 0 ? nt : 1), "export offsets");
    if (!rc)
        rc = check_cuda(c, cudaMemcpy(c->export_off.p, ho, sizeof(uint32_t) * (size_t)nt, cudaMemcpyHostToDevice),
                        "offsets upload");
    free(hr);
    free(ho);
    if (rc) return rc;
    launch_export_pairs((const uint32_t *)c->pvals.p, (const uint32_t *)c->pvals_b.p, (const Counters *)c->counters.p,
                        (const float *)c->depth.p, (const int2 *)c->ranges.p, v.tile_base, v.slot_base, nt,
                        (const uint32_t *)c->export_off.p, keys, values, ranges, (cudaStream_t)stream);
    return launched(c, "export pairs", 1);
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Allocation-free frame render (no counterpart in the paper).
//
// For callers that cannot allocate device memory: code running inside another engine's
// render loop or a host callback where cudaMalloc would block or is not permitted, or
// a process whose device memory is owned entirely by someone else's allocator. All scratch
// lives in one file-scope static __device__ array, which every GPU that loads this library
// holds until the process exits.
// ------------------------------------------------------------------------------------

namespace {

constexpr int kStaticMaxGaussians = 1 << 16;
constexpr int kStaticMaxPairs = 1 << 19;
constexpr int kStaticMaxTiles = 1 << 14;
constexpr int kStaticMaxDevices = 64;

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Carve-out of the static array, in bytes.
constexpr size_t kSzCounters = align256(sizeof(Counters));
constexpr size_t kSzViews = align256(sizeof(ViewDev));
constexpr size_t kSzScenes = align256(sizeof(SceneDev));
constexpr size_t kSzViewCounters = align256(sizeof(ViewCounters));
constexpr size_t kSzLabels = align256(kStaticMaxGaussians);
constexpr size_t kSzU32G = align256((size_t)kStaticMaxGaussians * 4);
constexpr size_t kSzErec = align256((size_t)kStaticMaxGaussians * sizeof(EmitRec));
constexpr size_t kSzRec = align256((size_t)kStaticMaxGaussians * sizeof(SplatRec));
constexpr size_t kSzCut = align256((size_t)kStaticMaxGaussians * sizeof(CutRec));
constexpr size_t kSzLookC = align256((size_t)(kStaticMaxGaussians / 1024 + 2) * 8);
constexpr size_t kSzLookE = align256((size_t)(kStaticMaxGaussians / kBlock + 2) * 8);
constexpr size_t kSzU32P = align256((size_t)kStaticMaxPairs * 4);
constexpr size_t kSzHist = align256(kHistPasses * 256 * 4);
constexpr size_t kSzSeg = align256(sizeof(uint32_t));
constexpr size_t kSzRanges = align256((size_t)kStaticMaxTiles * sizeof(int2));
constexpr size_t kSzOrder = align256((size_t)kStaticMaxTiles * 16);
// sort scratch for 4 digit passes over kStaticMaxPairs keys, sized for partitions as small as
// 1024 keys; static_setup checks it against the sort's own requirement
constexpr size_t kSzSort = align256(4 * (4 * (size_t)((kStaticMaxPairs + 1023) / 1024) * 256));
constexpr size_t kStaticBytes = kSzCounters + kSzViews + kSzScenes + kSzViewCounters + kSzLabels + 2 * kSzU32G +
                                kSzErec + kSzRec + kSzCut + 4 * kSzU32G + kSzLookC + kSzLookE + 4 * kSzU32P +
                                kSzHist + kSzSeg + kSzRanges + kSzOrder + kSzSort;

// 21,969,408 bytes with the current record sizes; the header states "about 22.0 MB"
static_assert(kStaticBytes <= 22000000, "the static scratch outgrew the size the header states");

static __device__ __align__(256) unsigned char g_rara_static_scratch[kStaticBytes];

rara_ctx g_static_ctx[kStaticMaxDevices];
Counters g_static_host_counters[kStaticMaxDevices];
ViewCounters g_static_host_view_counters[kStaticMaxDevices];
ViewDev g_static_host_views[kStaticMaxDevices][2];
SceneDev g_static_host_scenes[kStaticMaxDevices][2];
int g_static_view_map[kStaticMaxDevices];
int g_static_view_n[kStaticMaxDevices];
bool g_static_ready[kStaticMaxDevices];

// Once per device, with that device current: resolve the device address of the static
// array (its host-side name is only a stand-in) and carve the context's buffers from it.
int static_setup(int dev)
{
    if (g_static_ready[dev]) return RARA_OK;
    if (sort_scratch_bytes(kStaticMaxPairs, 4) > kSzSort) return RARA_ERR_BUDGET;
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_rara_static_scratch) != cudaSuccess || !base) {
        cudaGetLastError();
        return RARA_ERR_CUDA;
    }
    rara_ctx *c = &g_static_ctx[dev];
    unsigned char *p = (unsigned char *)base;
    auto take = [&](DevBuf &b, size_t bytes) { b.p = p; b.cap = bytes; p += bytes; };
    take(c->counters, kSzCounters);
    take(c->views_d, kSzViews);
    take(c->scenes_d, kSzScenes);
    take(c->view_counters_d, kSzViewCounters);
    take(c->labels, kSzLabels);
    take(c->tiles, kSzU32G);
    take(c->erec, kSzErec);
    take(c->rec, kSzRec);
    take(c->cut, kSzCut);
    take(c->depth, kSzU32G);
    take(c->ckeys, kSzU32G);
    take(c->cvals, kSzU32G);
    take(c->ckeys_b, kSzU32G);
    take(c->cvals_b, kSzU32G);
    take(c->lookback_c, kSzLookC);
    take(c->lookback_e, kSzLookE);
    take(c->pkeys, kSzU32P);
    take(c->pvals, kSzU32P);
    take(c->pkeys_b, kSzU32P);
    take(c->pvals_b, kSzU32P);
    take(c->hist, kSzHist);
    take(c->seg_base, kSzSeg);
    take(c->ranges, kSzRanges);
    take(c->items, kSzOrder);
    take(c->sort_scratch, kSzSort);
    c->budget = 0;
    c->device = dev;
    c->max_views = 1;
    c->max_scenes = 1;
    c->owns_host = false;
    for (int k = 0; k < 2; ++k) {
        c->staging[k].views = &g_static_host_views[dev][k];
        c->staging[k].scenes = &g_static_host_scenes[dev][k];
        c->staging[k].uploaded = nullptr;
    }
    c->h_view_map = &g_static_view_map[dev];
    c->h_view_n = &g_static_view_n[dev];
    c->h_counters = &g_static_host_counters[dev];
    c->h_view_counters = &g_static_host_view_counters[dev];
    g_static_ready[dev] = true;
    return RARA_OK;
}

}  // namespace

extern "C" int rara_render_frame_noalloc(const rara_gaussians *g, const rara_camera *cam, const rara_plane *plane,
                                         const float bg[3], float *image, float *final_T, uint32_t *n_contrib,
                                         void *stream)
{
    if (!g || !cam || !plane || !bg || !image) return RARA_ERR_INVALID_ARG;
    if (plane->n_extra != 0) return RARA_ERR_INVALID_ARG;  // single planes only: no clip-volume scratch
    if (g->n < 0 || g->n > kStaticMaxGaussians) return RARA_ERR_BUDGET;
    if (cam->width <= 0 || cam->height <= 0) return RARA_ERR_INVALID_ARG;
    const int64_t tiles = (int64_t)((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
    if (tiles > kStaticMaxTiles) return RARA_ERR_BUDGET;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return RARA_ERR_CUDA;
    int rc = static_setup(dev);
    if (rc) return rc;
    rara_ctx *c = &g_static_ctx[dev];
    rc = rara_preprocess(c, g, cam, plane, stream);
    if (rc) return rc;
    // The pair count is known only after the preprocess: wait for it and refuse frames whose
    // pairs exceed the static buffers, before rara_bin would need more.
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return RARA_ERR_CUDA;
    if (c->h_counters->n_pairs > (unsigned long long)kStaticMaxPairs) {
        c->stage = 0;
        return RARA_ERR_BUDGET;
    }
    rc = rara_bin(c, stream);
    if (rc) return rc;
    return rara_render(c, bg, image, final_T, n_contrib, stream);
}
