// Internal declarations shared by the CUDA translation units of librara.so.
//
// The render works on a batch: one or more scenes (Gaussian sets) and one or more views,
// each view a camera, a clip plane, a background and output buffers over one scene. A
// single frame is a batch of one view. Every stage is one launch for the whole batch:
//   preprocess   (scene, 256-Gaussian block) units; each loops over the scene's views and
//                fills dense per-(view, Gaussian) slots: label, tiles touched, rectangle,
//                splat record, depth, ray-tracing record
//   compact      rendered slots in slot order -> (depth bits, slot), depth-digit histogram
//   depth sort   one-sweep radix sort of those pairs by depth, then (batches of several
//                views) by view: slots in (view, depth) order
//   emit         one (global tile id, slot) pair per touched tile in that order (so each
//                view's pairs are contiguous and in depth order), plus the tile-digit
//                histogram
//   tile sort    one-sweep radix sort of the pairs on the local tile bits only
//   ranges       [start, end) of every global tile
// Global tile ids are view << tile_bits | local tile, tile_bits the bit length of the
// largest view's tile count: sorting the view-grouped pairs stably by the local bits leaves
// every (view, tile) list contiguous and in depth order with ceil(tile_bits / 8) digit
// passes, however many views the batch has. Ids past a view's last tile are holes (no
// pairs, no work items).
//   item order   render work items, heaviest first
//   render       compositing of every view's pixels
// Element counts after the preprocess live in device memory (Counters), so the sequence
// needs no host synchronisation and can be captured in a CUDA graph; a buffer sized from a
// capacity that a count exceeds sets kStatusOverflow instead of being written past its end.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rara.h"

namespace rara {

constexpr int kTile = 16;              // default screen tile edge (pixels), 16 x 16
constexpr int kBlock = 256;            // threads per block for per-Gaussian and per-pixel kernels
constexpr float kNearZ = 0.2f;         // near-plane cull (camera z)
constexpr float kDilation = 0.3f;      // low-pass dilation added to the 2D covariance (px^2)
constexpr float kSupportQ = 9.0f;      // per-pixel support: (3 sigma)^2 in Mahalanobis units
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// Polls of a bounded device-side wait (chained-scan look-back, bulk-copy barrier) before it
// gives up and records kStatusLookbackTimeout.
constexpr int kSpinLimit = 1 << 22;

// Device status word bits.
constexpr uint32_t kStatusLookbackTimeout = 1u;  // a bounded wait (chained scan, bulk copy) gave up
constexpr uint32_t kStatusOverflow = 2u;         // a count exceeded its buffer's capacity
constexpr uint32_t kStatusBadInput = 4u;         // a Gaussian had a non-finite parameter or colour

// Per-slot splat record, written by preprocess for rendered slots and gathered by the
// render kernel: 3 x float4 = 48 bytes.
//   r0 = (mean2d.x, mean2d.y, conic.a, conic.b)
//   r1 = (conic.c, opacity, rgb.r, rgb.g)
//   r2 = (rgb.b, decay-weight mode as float (kWeight*), -b/a, -b/c)
// The last two are the minimisers of q along a horizontal / vertical line (dx* = -b/a dy,
// dy* = -b/c dx), used by the render's exact rectangle test.
struct __align__(16) SplatRec {
    float4 r0, r1, r2;
};

// Per-slot emission record, written by the preprocess for rendered slots and gathered in
// depth order by the emission (so in no particular slot order): what the exact row spans of
// the slot's q <= q_cut ellipse need, in one 32-byte sector. In a shared listing (one-camera
// batch) only the first view that renders a Gaussian writes its record.
//   rect = (tx0 | ty0 << 16, tx1 | ty1 << 16), the tile rectangle in the view
//   (mx, my) the projected centre, (ca, cb, cc) the conic a, b, c
//   qcut = splat_qcut(log2 opacity), the support the render culls with
struct __align__(32) EmitRec {
    uint2 rect;
    float mx, my, ca, cb, cc, qcut;
};

// Decay-weight mode of a rendered slot (SplatRec r2.y). Only cutoff Gaussians whose
// ellipsoid the plane actually meets need the per-pixel weight; a cutoff Gaussian wholly on
// the visible side has w = 1 for every ray, one wholly on the invisible side has w = 0 for
// the rays that hit it in front and 1 for the others.
constexpr float kWeightNone = 0.0f, kWeightSplit = 1.0f, kWeightHidden = 2.0f;
// A cutoff Gaussian that two or more planes of a convex clip volume split (and none hides):
// its CutRec holds the first splitting plane, CutExtra the others.
constexpr float kWeightMulti = 3.0f;

// Per-cutoff-slot ray-tracing record, 4 x float4 = 64 bytes, relative to the Gaussian's own
// frame (see preprocess.cu for the derivation). With G = M^-1 (mu - e), the columns Px, Py
// of the 3x2 map P from a pixel offset to the local ray offset (scaled by the centre
// depth), m = M^T n and d_ep = n.mu + d, the record holds their products:
//   c0 = (G.G, G.Px, G.Py, d_ep)
//   c1 = (Px.Px, Px.Py, Py.Py, m.G)
//   c2 = (m.Px, m.Py, A.x, A.y)        A = Px x G
//   c3 = (A.z, B.x, B.y, B.z)          B = Py x G
struct __align__(16) CutRec {
    float4 c0, c1, c2, c3;
};

// The further splitting planes of a kWeightMulti slot, in the CutRec's terms:
// p[k] = (d_ep, m.G, m.Px, m.Py) of the plane; unused entries are (1, 0, 0, 0), a plane with
// s = 1 everywhere, which constrains nothing.
struct __align__(16) CutExtra {
    float4 p[3];
};

struct CamDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int W, H;
    float eye[3];
};

struct PlaneDev {
    float n[3];
    float d;
    float k;
    int mode;
    int n_extra;      // further planes of a convex clip volume (0..3)
    float ex[3][4];   // their (n, d)
};

struct ViewDev {
    CamDev cam;
    PlaneDev plane;
    int scene;
    int tile_w, tile_h;   // screen tile (the batch's tile shape: 64, 256 or 512 pixels)
    int same_cam;         // 1 if the previous view of the same scene has the same camera
    int tiles_x, tiles_y;
    uint32_t tile_base;   // first global tile id of the view (view << tile_bits)
    uint32_t slot_base;   // first dense (view, Gaussian) slot of the view
    float bg[3];
    float *image;         // [3][H][W]
    float *final_T;       // [H][W] or null
    uint32_t *n_contrib;  // [H][W] or null
};

struct SceneDev {
    const float *means, *log_scales, *quats, *logits, *sh;
    int n;
    int sh_degree;
    int view_begin, view_count;  // the scene's views are contiguous in the view table
    uint32_t unit_begin;         // first preprocess unit (256-Gaussian block) of the scene
};

// n_pairs counts candidate pairs (the tiles of the rendered slots' rectangles), an upper
// bound of the pairs the emission lists; it sizes the pair buffers.
struct ViewCounters {
    unsigned long long n_rendered, n_pairs, n_cutoff;
};

// Counters written by the kernels (device), copied to pinned host memory in one block.
struct Counters {
    unsigned long long n_rendered;       // rendered slots (all views)
    unsigned long long n_pairs;          // candidate pairs after the preprocess; the emission
                                         // replaces them with the pairs it lists (all views)
    unsigned long long n_cutoff;
    unsigned int num_items;              // render work items (written by the item-order kernel)
    unsigned int depth_in_b;             // 1 if the depth sort's result is in its B buffers
    // render counters, zeroed together before each render (n_evaluated .. tile_queue)
    unsigned long long n_evaluated;      // (pixel, Gaussian) pairs inside the q <= 9 support
    unsigned long long n_walked;         // (pixel, Gaussian) pairs whose q was computed
    unsigned long long n_cut_evaluated;  // evaluated pairs that needed the ray-traced weight
    unsigned long long n_tested;         // (warp, Gaussian) rectangle tests
    unsigned int tile_queue;             // next entry of the heaviest-first item order
    unsigned int status;
    unsigned int tile_in_b;              // 1 if the tile sort's result is in its B buffers
    unsigned int ticket[14];             // partition tickets of the persistent kernels
    unsigned long long n_union;          // one-camera batches: Gaussians rendered in some view
    unsigned int bwd_queue;              // next entry of the item order (render backward)
    unsigned int list_src;               // shared listing: 1 if the union's tile-sorted pairs are in B
    unsigned long long n_list;           // shared listing: the union's pairs
    unsigned int order_hist[33];         // tiles per list-length bucket (item order)
    unsigned int order_cursor[33];       // items placed per bucket (item order)
};
constexpr size_t kRenderCounterBytes = 4 * sizeof(unsigned long long) + sizeof(unsigned int);
// ticket slots
// (the depth sort has up to 4 depth + 2 view passes, the tile sort up to 4 passes)
constexpr int kTicketPre = 0, kTicketCompact = 1, kTicketEmit = 2, kTicketSortDepth = 3, kTicketSortTile = 9,
              kTicketExpand = 13;
// digit histograms: [0, 4) depth passes, [4, 6) view passes, [6, 10) tile passes (256 each)
constexpr int kHistDepth = 0, kHistView = 4, kHistTile = 6, kHistPasses = 10;

// Stage 1: preprocess
struct PreprocessArgs {
    const SceneDev *scenes;
    int num_scenes;
    const ViewDev *views;
    int num_units;         // sum over scenes of ceil(n / 256)
    // dense per-slot outputs
    uint8_t *labels;
    uint32_t *tiles;       // tiles touched (0 = not rendered)
    EmitRec *erec;         // emission record (tile rectangle, centre, conic, q_cut)
    SplatRec *rec;
    CutRec *cut;
    CutExtra *cut_x;  // per slot, only for batches with clip volumes (else null)
    float *depth;          // camera-space depth (the float32 sort key) of rendered slots
    uint32_t *gkey;        // one-camera batches (one scene, every view the same camera): per
                           // Gaussian, its depth bits if some view renders it, else kNoKey; null otherwise
    uint32_t *vmask;       // shared listing (a one-camera batch of at most kListViews views): per
                           // Gaussian, bit v set when view v renders it; null otherwise
    ViewCounters *view_counters;
    Counters *counters;
};
// max_sh_degree sizes the shared-memory staging of the SH coefficients (the largest degree
// of a scene with views); preprocess_configure() must have succeeded once per device.
// max_views: the most views of one scene in the batch (unused: one kernel instance serves all).
void launch_preprocess(const PreprocessArgs &a, int grid, int max_sh_degree, int max_views, cudaStream_t s);
int preprocess_configure();

// Stage 2: compaction of rendered slots (slot order) + histogram of the depth-key digits
struct CompactArgs {
    const uint32_t *tiles;
    const float *depth;
    uint32_t num_slots;
    uint32_t *keys;        // depth bits
    uint32_t *vals;        // slot
    uint32_t *hist;        // [kHistPasses][256] digit histograms, zeroed before
    unsigned long long *lookback;
    Counters *counters;
    // view passes of the depth sort: the views' first slots and rendered counts
    const ViewDev *views;
    const ViewCounters *view_counters;
    int num_views;
    uint32_t *seg_base;    // [num_views] first slot of each view (written)
    int spin_limit;        // polls of a look-back wait before it gives up
    // one-camera batches: compact the Gaussians with gkey[i] != kNoKey (num_slots = the scene
    // size; keys = their depth bits, values = Gaussian indices) and store the count in
    // counters->n_union; null otherwise
    const uint32_t *gkey;
};
constexpr uint32_t kNoKey = 0xffffffffu;  // gkey of a Gaussian no view renders
void launch_compact(const CompactArgs &a, int grid, cudaStream_t s);
int compact_blocks_per_sm();

// One-sweep LSD radix sort of (uint32 key, uint32 value) over bits [0, digit_bits * passes),
// digit_bits <= 8 bits per pass.
// The element count is read from device memory (*n, clamped to cap). hist holds the
// 8-bit digit histograms of all passes (built by the producer of the keys). A pass whose
// digit is the same for every key is skipped; *result_in_b is set on the device to 1 when
// the result ends in the B buffers. scratch: sort_scratch_bytes(cap, passes) bytes.
size_t sort_scratch_bytes(int64_t cap, int passes);
// Passes from first_seg_pass on (if num_segs > 0) sort by the segment of the value instead
// of the key: the index of the last seg_base entry <= value (seg_base ascending), 8 bits
// per pass; the keys those passes write out are the segment indices.
int sort_launch(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, const unsigned long long *n,
                uint32_t cap, int passes, const uint32_t *hist, void *scratch, unsigned int *tickets,
                unsigned int *status, unsigned int *result_in_b, int grid, cudaStream_t s,
                const uint32_t *seg_base = nullptr, int num_segs = 0, int first_seg_pass = 0, int digit_bits = 8);
int sort_blocks_per_sm();

// One-camera batches: the depth-sorted Gaussians (sorted_a / sorted_b by the sort's result
// flag, counters->n_union of them) expanded into every view's rendered slots in (view, depth)
// order: element e of the virtual sequence over views x sorted Gaussians is slot
// slot_base[v] + g, kept where that slot is rendered (tiles[slot] != 0); written to the
// depth-sort buffer the sort's result is not in (out_a / out_b), which the emission then reads.
struct ExpandArgs {
    const uint32_t *sorted_a, *sorted_b;
    uint32_t *out_a, *out_b;
    const uint32_t *tiles;
    const ViewDev *views;
    int num_views;
    unsigned long long *lookback;
    Counters *counters;
};
void launch_expand(const ExpandArgs &a, int grid, cudaStream_t s);

// Stage 4: emission of (global tile, slot) pairs in depth order + tile-digit histogram
struct EmitArgs {
    const uint32_t *keys_a, *vals_a, *keys_b, *vals_b;  // the depth sort's two buffers
    const uint32_t *tiles;
    const EmitRec *erec;     // the slots' rectangles and ellipses (the exact row spans)
    const ViewDev *views;
    int num_views;
    uint32_t cap_pairs;
    int tile_passes;
    int tile_digit_bits;     // bits per tile-sort pass
    int expanded;            // the slots are in the buffer the depth sort's result is not in (launch_expand)
    // shared listing: the depth-sorted values are the Gaussians of a one-camera batch that
    // some view renders (counters->n_union of them); each is listed once with the local tile
    // ids of the common tile grid and the Gaussian index as value, its rectangle and splat
    // read from the first view that renders it (vmask)
    int shared_list;
    const uint32_t *vmask;
    uint32_t *pair_keys;     // global tile id (local with shared_list)
    uint32_t *pair_vals;     // slot (Gaussian index with shared_list)
    uint32_t *tile_hist;     // [tile_passes][256], zeroed before
    unsigned long long *lookback;
    Counters *counters;
};
void launch_emit(const EmitArgs &a, int grid, cudaStream_t s);
int emit_blocks_per_sm();

// Shared listing of a one-camera batch. All views share the camera, so a Gaussian covers the
// same tiles in each view that renders it, and the depth order is common: view v's list of
// tile t is the union's list of t (tile-sorted once) without the Gaussians v does not render.
// With C_v(j) = the union pairs before position j whose Gaussian view v renders and B_v = the
// pairs of the views before v, union pair j goes to position B_v + C_v(j) of the views' pair
// list, and view v's range of tile t is [B_v + C_v(start of t), B_v + C_v(end of t)). Three
// launches over partitions of kListPart union pairs (one warp each): every view's count per
// partition, their exclusive scan per view (one block per view) with the view totals, and the
// scatter of values (slot_base[v] + Gaussian) and ranges. The lists land in the value buffer
// the union's are not in, and counters->tile_in_b is switched to it.
constexpr int kListViews = 32;          // views of a shared listing (bits of vmask)
constexpr uint32_t kListPart = 512;     // union pairs per partition (16 rounds of a warp)
struct ListArgs {
    const uint32_t *keys_a, *keys_b;    // the union's tile-sorted pairs (local tile ids)
    uint32_t *vals_a, *vals_b;          // ... their Gaussians; the views' slots go to the other buffer
    const uint32_t *vmask;
    const ViewDev *views;
    int num_views;
    int tile_bits;
    uint32_t slot_stride;               // the scene's size: view v's slot of Gaussian g is v * slot_stride + g
    uint32_t *part_counts;              // [kListViews][max_parts] counts, then exclusive prefixes,
                                        // followed by the kListViews view totals
    uint32_t max_parts;                 // >= cap_pairs / kListPart rounded up
    int2 *ranges;                       // global tile ranges, zeroed before
    uint32_t cap_pairs;
    Counters *counters;
};
// 4-byte words of part_counts for a pair capacity
inline size_t list_count_words(uint32_t cap_pairs)
{
    return (size_t)kListViews * ((cap_pairs + kListPart - 1) / kListPart + 1) + kListViews;
}
// grid: blocks of kBlock threads for the count and scatter launches (persistent over partitions)
void launch_lists(const ListArgs &a, int grid, cudaStream_t s);

// Stage 6: ranges of the sorted pairs (ranges zeroed before)
void launch_ranges(const uint32_t *keys_a, const uint32_t *keys_b, const Counters *counters, uint32_t cap_pairs,
                   uint32_t num_tiles, int2 *ranges, int grid, cudaStream_t s);

// Stage 7: render work items ordered by descending list length (log2 buckets), heaviest
// first. A work item is 256 lanes over a band of a tile's rows with L = 1, 2 or 4 lanes per
// pixel (256 / L pixels). A tile whose list has at least 2^(split4_bits-1) entries gets
// L = 4, at least 2^(split2_bits-1) entries L = 2, otherwise L = 1, clamped so that an item
// holds at most the tile's pixels and a tile is at most 4 items: 64-pixel tiles always take
// L = 4, 512-pixel tiles at most L = 2. The tile then becomes L * pixels / 256 items.
// Item = tile << 4 | log2(L) << 2 | part. area_log2 = log2(tile pixels / 64) (0, 2 or 3).
// order holds 4 * num_tiles entries; the item count goes to counters->num_items.
void launch_tile_order(const int2 *ranges, int num_tiles, int split2_bits, int split4_bits, int area_log2,
                       uint32_t *order, Counters *counters, const ViewDev *views, int tile_bits, int grid,
                       cudaStream_t s);

// Stage 8: render
struct RenderArgs {
    const int2 *ranges;
    const uint32_t *tile_order;
    const uint32_t *vals_a, *vals_b;  // the tile sort's value buffers (slots)
    const SplatRec *rec;
    const CutRec *cut;
    const CutExtra *cut_x;  // per slot, only for batches with clip volumes (else null)
    const ViewDev *views;
    int num_views;
    Counters *counters;
};
// count: accumulate the work counters (n_evaluated .. n_tested) of the launch. depth: the
// blend batch depth (entries staged in shared memory per batch: 128, 256 or 512).
int launch_render(const RenderArgs &a, int grid, cudaStream_t s, bool count, bool multi, int depth);
int render_blocks_per_sm(int depth);
// Tile shapes and blend batch depths the kernels support.
bool tile_shape_ok(int tile_w, int tile_h);
bool batch_depth_ok(int depth);

// Backward. Per-slot gradient record, 7 x float4 = 112 bytes, accumulated (atomics) by the
// render backward and read by the preprocess backward:
//   v[0..8]   dL/d(mean2d.x, mean2d.y, conic.a, conic.b, conic.c, opacity, rgb.r, rgb.g, rgb.b)
//   v[9..24]  dL/d(the 16 products of the CutRec, in its order), split-weight slots only
//   v[25..27] unused
// conic.b is the off-diagonal entry, which q uses twice.
constexpr int kGradCut = 9;
struct __align__(16) GradRec {
    float v[28];
};

struct BwdView {
    const float *dimage;  // dL/dimage [3][H][W]
    float *plane_grad;    // 4 floats (dL/dn, dL/dd) or null
};

struct BwdScene {
    float *means, *log_scales, *quats, *logits, *sh;  // gradients, the scene's layouts
};

struct RenderBwdArgs {
    const int2 *ranges;
    const uint32_t *tile_order;
    const uint32_t *vals_a, *vals_b;
    const SplatRec *rec;
    const CutRec *cut;
    const ViewDev *views;
    const BwdView *bviews;
    int num_views;
    GradRec *grec;        // [slots], all zero on entry
    Counters *counters;
};
void launch_render_bwd(const RenderBwdArgs &a, int grid, cudaStream_t s);
int render_bwd_blocks_per_sm();

struct PreprocessBwdArgs {
    const SceneDev *scenes;
    int num_scenes;
    const ViewDev *views;
    const BwdView *bviews;
    const BwdScene *bscenes;
    const uint8_t *labels;
    const uint32_t *tiles;
    GradRec *grec;         // read, then zeroed, for every rendered slot
    int sh_stride;         // set by the launcher
};
// grid = preprocess units; max_sh_degree sizes the per-block SH gradient accumulators.
int launch_preprocess_bwd(const PreprocessBwdArgs &a, int grid, int max_sh_degree, cudaStream_t s);

// The L2 objective on a render's images (rara_loss_l2): per view its image, target, gradient
// output and loss accumulator, and the first of its blocks (kLossChunk elements per block).
struct LossView {
    const float *image;
    const float *target;
    float *dimage;
    double *loss;
    float scale;
    uint32_t n;            // elements, 3 H W
    uint32_t chunk_begin;  // first block of this view
    uint32_t pad;
};
constexpr int kLossChunk = 16 * kBlock;
void launch_loss_l2(const LossView *views, int num_views, uint32_t grid, cudaStream_t s);

// Debug exports of one view
void launch_export_gaussians(int n, uint32_t slot_base, const uint8_t *labels_src, const uint32_t *tiles_src,
                             const EmitRec *erec_src, const uint32_t *vmask, const ViewDev *views,
                             const SplatRec *rec, const float *depth_src, uint8_t *labels,
                             float *depth, float *mean2d, float *conic, float *rgb, float *opacity, int32_t *rect,
                             uint32_t *tiles, cudaStream_t s);
// Pairs of one view in (local tile, depth) order: tile t's list goes to out_offset[t]
// (exclusive prefix of the view's list lengths, computed by the caller).
void launch_export_pairs(const uint32_t *vals_a, const uint32_t *vals_b, const Counters *counters, const float *depth,
                         const int2 *ranges, uint32_t tile_base, uint32_t slot_base, int num_tiles,
                         const uint32_t *out_offset, uint64_t *keys, uint32_t *values, int64_t *ranges_out,
                         cudaStream_t s);

}  // namespace rara
