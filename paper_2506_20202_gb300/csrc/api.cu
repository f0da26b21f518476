// C ABI of librara.so: context, buffer management, argument checks and stage order.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "rara_internal.cuh"

using namespace rara;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct rara_ctx {
    size_t budget = 0;
    size_t held = 0;
    int device = 0;
    char err[512] = {0};
    int64_t launches = 0;

    // frame state
    int stage = 0;  // 0 empty, 1 preprocessed, 2 binned
    int n = 0;
    int W = 0, H = 0;
    int tiles_x = 0, tiles_y = 0, num_tiles = 0;
    int64_t n_rendered = 0, n_pairs = 0, n_cutoff = 0;
    cudaStream_t last_stream = nullptr;

    int sm_count = 0, render_bpsm = 0;
    int split2_bits = 11, split4_bits = 12;  // heavy-tile split thresholds (list length bit counts)

    // per-Gaussian
    DevBuf labels, tiles, rect, rec, cut, depth, ckeys, cvals, ckeys_alt, cvals_alt, lookback_g;
    // per-pair
    DevBuf pkeys, pvals, pkeys_alt, pvals_alt, lookback_p;
    DevBuf ranges, tile_order, sort_scratch, counters;
    Counters *h_counters = nullptr;  // pinned
    const uint32_t *sorted_gauss = nullptr;  // depth-ordered indices (ckeys/cvals or alt)
    const uint32_t *sorted_tile_keys = nullptr;
    const uint32_t *sorted_pair_vals = nullptr;
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

// Grow-only device buffer within the context budget.
int ensure(rara_ctx *c, DevBuf &b, size_t bytes, const char *name)
{
    if (bytes <= b.cap) return RARA_OK;
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
}

bool finite(float v) { return isfinite(v) != 0; }

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

}  // namespace

extern "C" {

int rara_ctx_create(size_t budget_bytes, int32_t tile_w, int32_t tile_h, rara_ctx **out)
{
    if (!out) return RARA_ERR_INVALID_ARG;
    *out = nullptr;
    if (tile_w != kTile || tile_h != kTile) return RARA_ERR_INVALID_ARG;
    rara_ctx *c = new (std::nothrow) rara_ctx();
    if (!c) return RARA_ERR_BUDGET;
    c->budget = budget_bytes;
    cudaGetDevice(&c->device);
    int rc = ensure(c, c->counters, sizeof(Counters), "counters");
    if (rc == RARA_OK && cudaHostAlloc((void **)&c->h_counters, sizeof(Counters), cudaHostAllocDefault) != cudaSuccess)
        rc = fail(c, RARA_ERR_CUDA, "cudaHostAlloc failed");
    if (rc != RARA_OK) {
        release(c, c->counters);
        delete c;
        return rc;
    }
    memset(c->h_counters, 0, sizeof(Counters));
    *out = c;
    return RARA_OK;
}

int rara_ctx_destroy(rara_ctx *c)
{
    if (!c) return RARA_OK;
    cudaDeviceSynchronize();
    DevBuf *all[] = {&c->labels, &c->tiles, &c->rect, &c->rec, &c->cut, &c->depth, &c->ckeys, &c->cvals,
                     &c->ckeys_alt, &c->cvals_alt, &c->lookback_g, &c->pkeys, &c->pvals, &c->pkeys_alt,
                     &c->pvals_alt, &c->lookback_p, &c->ranges, &c->tile_order, &c->sort_scratch, &c->counters};
    for (DevBuf *b : all) release(c, *b);
    if (c->h_counters) cudaFreeHost(c->h_counters);
    delete c;
    return RARA_OK;
}

const char *rara_last_error(const rara_ctx *c) { return c ? c->err : "null context"; }

size_t rara_ctx_bytes(const rara_ctx *c) { return c ? c->held : 0; }

int64_t rara_ctx_launches(const rara_ctx *c) { return c ? c->launches : 0; }

int rara_ctx_set_tuning(rara_ctx *c, int32_t split2_bits, int32_t split4_bits)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->split2_bits = split2_bits < 0 ? 0 : (split2_bits > 33 ? 33 : split2_bits);
    c->split4_bits = split4_bits < 0 ? 0 : (split4_bits > 33 ? 33 : split4_bits);
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
    if (c->h_counters->status & kStatusLookbackTimeout)
        return fail(c, RARA_ERR_TIMEOUT, "a chained-scan wait exceeded its bound; the frame is invalid");
    return RARA_OK;
}

int rara_preprocess(rara_ctx *c, const rara_gaussians *g, const rara_camera *cam, const rara_plane *pl,
                    void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    c->err[0] = 0;
    c->stage = 0;
    if (!g || !cam || !pl) return fail(c, RARA_ERR_INVALID_ARG, "null argument");
    if (g->n < 0 || g->n >= (int64_t)1 << 31) return fail(c, RARA_ERR_INVALID_ARG, "n = %lld out of range", (long long)g->n);
    if (g->sh_degree < 0 || g->sh_degree > 3) return fail(c, RARA_ERR_INVALID_ARG, "sh_degree %d not in [0,3]", g->sh_degree);
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail(c, RARA_ERR_INVALID_ARG, "null Gaussian array");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 65535 * kTile || cam->height > 65535 * kTile)
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

    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)g->n;
    c->n = n;
    c->W = cam->width;
    c->H = cam->height;
    c->tiles_x = (cam->width + kTile - 1) / kTile;
    c->tiles_y = (cam->height + kTile - 1) / kTile;
    c->num_tiles = c->tiles_x * c->tiles_y;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const int blocks = (n + kBlock - 1) / kBlock;
    int rc;
    if ((rc = ensure(c, c->labels, nn, "labels")) || (rc = ensure(c, c->tiles, nn * 4, "tiles")) ||
        (rc = ensure(c, c->rect, nn * 8, "rect")) || (rc = ensure(c, c->rec, nn * sizeof(SplatRec), "records")) ||
        (rc = ensure(c, c->cut, nn * sizeof(CutRec), "cutoff records")) ||
        (rc = ensure(c, c->depth, nn * 4, "depth")) ||
        (rc = ensure(c, c->ckeys, nn * 4, "depth keys")) || (rc = ensure(c, c->cvals, nn * 4, "depth values")) ||
        (rc = ensure(c, c->ckeys_alt, nn * 4, "depth keys alt")) ||
        (rc = ensure(c, c->cvals_alt, nn * 4, "depth values alt")) ||
        (rc = ensure(c, c->lookback_g, (size_t)(blocks + 1) * 8, "scan words")))
        return rc;

    PreprocessArgs a;
    a.means = g->means; a.log_scales = g->log_scales; a.quats = g->quats; a.logits = g->opacity_logits; a.sh = g->sh;
    a.n = n;
    a.sh_degree = g->sh_degree;
    for (int k = 0; k < 9; ++k) a.cam.R[k] = cam->world_to_cam[(k / 3) * 4 + (k % 3)];
    for (int k = 0; k < 3; ++k) a.cam.t[k] = cam->world_to_cam[k * 4 + 3];
    a.cam.fx = cam->fx; a.cam.fy = cam->fy; a.cam.cx = cam->cx; a.cam.cy = cam->cy;
    a.cam.W = cam->width; a.cam.H = cam->height;
    for (int j = 0; j < 3; ++j)  // e = -R^T t
        a.cam.eye[j] = -(a.cam.R[j] * a.cam.t[0] + a.cam.R[3 + j] * a.cam.t[1] + a.cam.R[6 + j] * a.cam.t[2]);
    for (int k = 0; k < 3; ++k) a.plane.n[k] = pl->n[k];
    a.plane.d = pl->d;
    a.plane.k = pl->k_sigma;
    a.plane.mode = pl->mode;
    a.tiles_x = c->tiles_x;
    a.tiles_y = c->tiles_y;
    a.labels = (uint8_t *)c->labels.p;
    a.tiles = (uint32_t *)c->tiles.p;
    a.rect = (uint2 *)c->rect.p;
    a.rec = (SplatRec *)c->rec.p;
    a.cut = (CutRec *)c->cut.p;
    a.depth = (float *)c->depth.p;
    a.ckeys = (uint32_t *)c->ckeys.p;
    a.cvals = (uint32_t *)c->cvals.p;
    a.lookback = (unsigned long long *)c->lookback_g.p;
    a.counters = (Counters *)c->counters.p;

    if ((rc = check_cuda(c, cudaMemsetAsync(c->counters.p, 0, sizeof(Counters), s), "memset counters"))) return rc;
    if ((rc = check_cuda(c, cudaMemsetAsync(c->lookback_g.p, 0, (size_t)(blocks + 1) * 8, s), "memset scan")))
        return rc;
    launch_preprocess(a, blocks, s);
    if ((rc = launched(c, "preprocess launch", blocks > 0))) return rc;
    if ((rc = check_cuda(c, cudaMemcpyAsync(c->h_counters, c->counters.p, sizeof(Counters), cudaMemcpyDeviceToHost, s),
                         "counter copy")))
        return rc;
    c->last_stream = s;
    c->stage = 1;
    return RARA_OK;
}

int rara_bin(rara_ctx *c, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (c->stage < 1) return fail(c, RARA_ERR_INVALID_ARG, "rara_bin called before rara_preprocess");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    // The counter copy was queued by rara_preprocess on its stream; wait for that stream.
    if ((rc = check_cuda(c, cudaStreamSynchronize(c->last_stream), "cudaStreamSynchronize"))) return rc;
    if (c->h_counters->status & kStatusLookbackTimeout) {
        c->stage = 0;
        return fail(c, RARA_ERR_TIMEOUT, "a chained-scan wait exceeded its bound; the frame is invalid");
    }
    c->n_rendered = (int64_t)c->h_counters->n_rendered;
    c->n_pairs = (int64_t)c->h_counters->n_pairs;
    c->n_cutoff = (int64_t)c->h_counters->n_cutoff;
    if (c->n_pairs >= (int64_t)1 << 30) return fail(c, RARA_ERR_BUDGET, "%lld pairs exceed 2^30", (long long)c->n_pairs);
    const int nr = (int)c->n_rendered;
    const int np = (int)c->n_pairs;
    const size_t pp = (size_t)(np > 0 ? np : 1);
    const int tile_bits = ceil_bits((uint32_t)c->num_tiles);
    const size_t sbytes = sort_scratch_bytes(np > nr ? np : nr, 32);  // both sorts, worst case
    const int eblocks = (nr + kBlock - 1) / kBlock;
    if ((rc = ensure(c, c->pkeys, pp * 4, "pair keys")) || (rc = ensure(c, c->pvals, pp * 4, "pair values")) ||
        (rc = ensure(c, c->pkeys_alt, pp * 4, "pair keys alt")) ||
        (rc = ensure(c, c->pvals_alt, pp * 4, "pair values alt")) ||
        (rc = ensure(c, c->lookback_p, (size_t)(eblocks + 1) * 8, "emit scan words")) ||
        (rc = ensure(c, c->ranges, (size_t)c->num_tiles * sizeof(int2), "ranges")) ||
        (rc = ensure(c, c->tile_order, (size_t)c->num_tiles * 16, "render items")) ||
        (rc = ensure(c, c->sort_scratch, sbytes, "sort scratch")))
        return rc;
    uint32_t *status = &((Counters *)c->counters.p)->status;

    // 1. depth sort of the rendered Gaussians (ascending float bits = ascending depth > 0)
    bool in_alt = false;
    int nl = sort_pairs((uint32_t *)c->ckeys.p, (uint32_t *)c->cvals.p, (uint32_t *)c->ckeys_alt.p,
                        (uint32_t *)c->cvals_alt.p, nr, 32, c->sort_scratch.p, status, s, &in_alt);
    if ((rc = launched(c, "depth sort", nl))) return rc;
    c->sorted_gauss = (const uint32_t *)(in_alt ? c->cvals_alt.p : c->cvals.p);

    // 2. emit (tile id, index) pairs in depth order
    if ((rc = check_cuda(c, cudaMemsetAsync(c->lookback_p.p, 0, (size_t)(eblocks + 1) * 8, s), "memset emit")))
        return rc;
    EmitArgs e;
    e.sorted_vals = c->sorted_gauss;
    e.tiles = (const uint32_t *)c->tiles.p;
    e.rect = (const uint2 *)c->rect.p;
    e.n_rendered = nr;
    e.tiles_x = c->tiles_x;
    e.n_pairs = (unsigned long long)np;
    e.pair_keys = (uint32_t *)c->pkeys.p;
    e.pair_vals = (uint32_t *)c->pvals.p;
    e.lookback = (unsigned long long *)c->lookback_p.p;
    e.counters = (Counters *)c->counters.p;
    launch_emit(e, eblocks, s);
    if ((rc = launched(c, "emit", eblocks > 0))) return rc;

    // 3. stable sort of the pairs by tile id (the depth order is kept within a tile)
    nl = sort_pairs((uint32_t *)c->pkeys.p, (uint32_t *)c->pvals.p, (uint32_t *)c->pkeys_alt.p,
                    (uint32_t *)c->pvals_alt.p, np, tile_bits, c->sort_scratch.p, status, s, &in_alt);
    if ((rc = launched(c, "tile sort", nl))) return rc;
    c->sorted_tile_keys = (const uint32_t *)(in_alt ? c->pkeys_alt.p : c->pkeys.p);
    c->sorted_pair_vals = (const uint32_t *)(in_alt ? c->pvals_alt.p : c->pvals.p);

    // 4. tile ranges
    if ((rc = check_cuda(c, cudaMemsetAsync(c->ranges.p, 0, (size_t)c->num_tiles * sizeof(int2), s), "memset ranges")))
        return rc;
    launch_ranges(c->sorted_tile_keys, np, c->num_tiles, (int2 *)c->ranges.p, s);
    if ((rc = launched(c, "ranges", np > 0))) return rc;

    // 5. heaviest-first order of the tiles for the render's persistent blocks
    launch_tile_order((const int2 *)c->ranges.p, c->num_tiles, c->split2_bits, c->split4_bits,
                      (uint32_t *)c->tile_order.p, (Counters *)c->counters.p, s);
    if ((rc = launched(c, "tile order", c->num_tiles > 0))) return rc;
    c->last_stream = s;
    c->stage = 2;
    return RARA_OK;
}

int rara_render(rara_ctx *c, const float bg[3], float *image, float *final_T, uint32_t *n_contrib, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (c->stage < 2) return fail(c, RARA_ERR_INVALID_ARG, "rara_render called before rara_bin");
    if (!bg || !image) return fail(c, RARA_ERR_INVALID_ARG, "null bg or image");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->sm_count == 0) {
        if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
            c->sm_count < 1) {
            cudaGetLastError();
            c->sm_count = 1;
        }
        c->render_bpsm = render_blocks_per_sm();
    }
    RenderArgs a;
    a.ranges = (const int2 *)c->ranges.p;
    a.tile_order = (const uint32_t *)c->tile_order.p;
    a.num_tiles = c->num_tiles;
    a.pair_vals = c->sorted_pair_vals;
    a.rec = (const SplatRec *)c->rec.p;
    a.cut = (const CutRec *)c->cut.p;
    a.W = c->W;
    a.H = c->H;
    a.tiles_x = c->tiles_x;
    a.bg[0] = bg[0]; a.bg[1] = bg[1]; a.bg[2] = bg[2];
    a.image = image;
    a.final_T = final_T;
    a.n_contrib = n_contrib;
    a.counters = (Counters *)c->counters.p;
    int rc;
    if ((rc = check_cuda(c, cudaMemsetAsync(&a.counters->n_evaluated, 0, kRenderCounterBytes, s),
                         "memset render counters")))
        return rc;
    const int slots = c->sm_count * c->render_bpsm;
    const int grid = 4 * c->num_tiles < slots ? 4 * c->num_tiles : slots;
    launch_render(a, grid, s);
    if ((rc = launched(c, "render launch", c->num_tiles > 0))) return rc;
    c->last_stream = s;
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

int rara_frame_info_get(rara_ctx *c, rara_frame_info *out)
{
    if (!c || !out) return RARA_ERR_INVALID_ARG;
    if (c->stage < 2) return fail(c, RARA_ERR_INVALID_ARG, "no binned frame");
    int rc = rara_ctx_sync(c, c->last_stream);
    if (rc) return rc;
    out->n = c->n;
    out->n_rendered = c->n_rendered;
    out->n_cutoff = c->n_cutoff;
    out->n_pairs = c->n_pairs;
    out->tiles_x = c->tiles_x;
    out->tiles_y = c->tiles_y;
    out->n_evaluated = (int64_t)c->h_counters->n_evaluated;
    out->n_walked = (int64_t)c->h_counters->n_walked;
    out->n_cut_evaluated = (int64_t)c->h_counters->n_cut_evaluated;
    out->n_tested = (int64_t)c->h_counters->n_tested;
    return RARA_OK;
}

int rara_frame_gaussians(rara_ctx *c, uint8_t *labels, float *depth, float *mean2d, float *conic, float *rgb,
                         float *opacity, int32_t *rect, uint32_t *tiles, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (c->stage < 1) return fail(c, RARA_ERR_INVALID_ARG, "no preprocessed frame");
    launch_export_gaussians(c->n, (const uint8_t *)c->labels.p, (const uint32_t *)c->tiles.p,
                            (const uint2 *)c->rect.p, (const SplatRec *)c->rec.p, (const float *)c->depth.p, labels,
                            depth, mean2d, conic,
                            rgb, opacity, rect, tiles, (cudaStream_t)stream);
    return launched(c, "export gaussians", c->n > 0);
}

int rara_frame_pairs(rara_ctx *c, uint64_t *keys, uint32_t *values, int64_t *ranges, void *stream)
{
    if (!c) return RARA_ERR_INVALID_ARG;
    if (c->stage < 2) return fail(c, RARA_ERR_INVALID_ARG, "no binned frame");
    launch_export_pairs((int)c->n_pairs, c->sorted_tile_keys, c->sorted_pair_vals, (const float *)c->depth.p,
                        (const int2 *)c->ranges.p, c->num_tiles, keys, values, ranges, (cudaStream_t)stream);
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
constexpr size_t kSzLabels = align256(kStaticMaxGaussians);
constexpr size_t kSzU32G = align256((size_t)kStaticMaxGaussians * 4);
constexpr size_t kSzRect = align256((size_t)kStaticMaxGaussians * 8);
constexpr size_t kSzRec = align256((size_t)kStaticMaxGaussians * sizeof(SplatRec));
constexpr size_t kSzCut = align256((size_t)kStaticMaxGaussians * sizeof(CutRec));
constexpr size_t kSzLookG = align256((size_t)(kStaticMaxGaussians / kBlock + 1) * 8);
constexpr size_t kSzU32P = align256((size_t)kStaticMaxPairs * 4);
constexpr size_t kSzRanges = align256((size_t)kStaticMaxTiles * sizeof(int2));
// sort scratch for 4 digit passes over kStaticMaxPairs keys, sized for partitions as small as
// 1024 keys; static_setup checks it against the sort's own requirement
constexpr size_t kSzSort = align256(4 * (4 * 256 + 64 + 4 * (size_t)((kStaticMaxPairs + 1023) / 1024) * 256));
constexpr size_t kSzOrder = align256((size_t)kStaticMaxTiles * 16);
constexpr size_t kStaticBytes = kSzCounters + kSzLabels + kSzU32G + kSzRect + kSzRec + kSzCut + kSzU32G +
                                4 * kSzU32G + kSzLookG + 4 * kSzU32P + kSzLookG + kSzRanges + kSzOrder + kSzSort;

static __device__ __align__(256) unsigned char g_rara_static_scratch[kStaticBytes];

rara_ctx g_static_ctx[kStaticMaxDevices];
Counters g_static_host_counters[kStaticMaxDevices];
bool g_static_ready[kStaticMaxDevices];

// Once per device, with that device current: resolve the device address of the static
// array (its host-side name is only a stand-in) and carve the context's buffers from it.
int static_setup(int dev)
{
    if (g_static_ready[dev]) return RARA_OK;
    if (sort_scratch_bytes(kStaticMaxPairs, 32) > kSzSort) return RARA_ERR_BUDGET;
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_rara_static_scratch) != cudaSuccess || !base) {
        cudaGetLastError();
        return RARA_ERR_CUDA;
    }
    rara_ctx *c = &g_static_ctx[dev];
    unsigned char *p = (unsigned char *)base;
    auto take = [&](DevBuf &b, size_t bytes) { b.p = p; b.cap = bytes; p += bytes; };
    take(c->counters, kSzCounters);
    take(c->labels, kSzLabels);
    take(c->tiles, kSzU32G);
    take(c->rect, kSzRect);
    take(c->rec, kSzRec);
    take(c->cut, kSzCut);
    take(c->depth, kSzU32G);
    take(c->ckeys, kSzU32G);
    take(c->cvals, kSzU32G);
    take(c->ckeys_alt, kSzU32G);
    take(c->cvals_alt, kSzU32G);
    take(c->lookback_g, kSzLookG);
    take(c->pkeys, kSzU32P);
    take(c->pvals, kSzU32P);
    take(c->pkeys_alt, kSzU32P);
    take(c->pvals_alt, kSzU32P);
    take(c->lookback_p, kSzLookG);
    take(c->ranges, kSzRanges);
    take(c->tile_order, kSzOrder);
    take(c->sort_scratch, kSzSort);
    c->budget = 0;
    c->device = dev;
    c->h_counters = &g_static_host_counters[dev];
    g_static_ready[dev] = true;
    return RARA_OK;
}

}  // namespace

extern "C" int rara_render_frame_noalloc(const rara_gaussians *g, const rara_camera *cam, const rara_plane *plane,
                                         const float bg[3], float *image, float *final_T, uint32_t *n_contrib,
                                         void *stream)
{
    if (!g || !cam || !plane || !bg || !image) return RARA_ERR_INVALID_ARG;
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
