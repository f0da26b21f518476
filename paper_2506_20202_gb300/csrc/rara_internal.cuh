// Internal declarations shared by the CUDA translation units of librara.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rara.h"

namespace rara {

constexpr int kTile = 16;              // screen tile edge (pixels); one 256-thread block per tile
constexpr int kBlock = 256;            // threads per block for per-Gaussian and per-pixel kernels
constexpr float kNearZ = 0.2f;         // near-plane cull (camera z)
constexpr float kDilation = 0.3f;      // low-pass dilation added to the 2D covariance (px^2)
constexpr float kSupportQ = 9.0f;      // per-pixel support: (3 sigma)^2 in Mahalanobis units
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// Device status word bits (bounded waits that gave up).
constexpr uint32_t kStatusLookbackTimeout = 1u;

// Per-Gaussian splat record, written by preprocess for rendered Gaussians and gathered
// by the render kernel: 3 x float4 = 48 bytes.
//   r0 = (mean2d.x, mean2d.y, conic.a, conic.b)
//   r1 = (conic.c, opacity, rgb.r, rgb.g)
//   r2 = (rgb.b, cutoff flag as float (1 or 0), -b/a, -b/c)
// The last two are the minimisers of q along a horizontal / vertical line (dx* = -b/a dy,
// dy* = -b/c dx), used by the render's exact rectangle test.
struct __align__(16) SplatRec {
    float4 r0, r1, r2;
};

// Per-cutoff-Gaussian ray-tracing record, 4 x float4 = 64 bytes, relative to the
// Gaussian's own frame (see preprocess.cu for the derivation):
//   c0 = (G.x, G.y, G.z, d_ep)         G = M^-1 (mu - e), d_ep = n.mu + d
//   c1 = (P00, P10, P20, m.x)          P: 3x2 map from a pixel offset to the local ray
//   c2 = (P01, P11, P21, m.y)              offset, scaled by the centre depth
//   c3 = (m.z, 0, 0, 0)                m = M^T n
struct __align__(16) CutRec {
    float4 c0, c1, c2, c3;
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
};

// Counters written by the kernels (device), copied to pinned host memory in one block.
struct Counters {
    unsigned long long n_rendered;
    unsigned long long n_pairs;
    unsigned long long n_cutoff;
    unsigned int num_items;              // render work items (written by the item-order kernel)
    unsigned int pad0;
    // render counters, zeroed together before each render (n_evaluated .. tile_queue)
    unsigned long long n_evaluated;      // (pixel, Gaussian) pairs inside the q <= 9 support
    unsigned long long n_walked;         // (pixel, Gaussian) pairs whose q was computed
    unsigned long long n_cut_evaluated;  // evaluated pairs that needed the ray-traced weight
    unsigned long long n_tested;         // (warp, Gaussian) rectangle tests
    unsigned int tile_queue;             // next entry of the heaviest-first item order
    unsigned int status;
    unsigned int part_counter[8];  // partition tickets for chained scans
};
constexpr size_t kRenderCounterBytes = 4 * sizeof(unsigned long long) + sizeof(unsigned int);

struct PreprocessArgs {
    const float *means, *log_scales, *quats, *logits, *sh;
    int n;
    int sh_degree;
    CamDev cam;
    PlaneDev plane;
    int tiles_x, tiles_y;
    // outputs
    uint8_t *labels;
    uint32_t *tiles;       // tiles touched (0 = not rendered)
    uint2 *rect;           // (tx0 | ty0 << 16, tx1 | ty1 << 16)
    SplatRec *rec;
    CutRec *cut;
    float *depth;          // camera-space depth (float32 key value) of rendered Gaussians
    uint32_t *ckeys;       // compacted depth keys (float bits) of rendered Gaussians
    uint32_t *cvals;       // their indices, ascending
    unsigned long long *lookback;  // per-block chained-scan words, zeroed before launch
    Counters *counters;
};

void launch_preprocess(const PreprocessArgs &a, int num_blocks, cudaStream_t s);

// Stable LSD radix sort of (uint32 key, uint32 value) pairs on bits [0, key_bits).
// Buffers: keys/vals hold the input and receive the output (ping-pong through alt_*).
// Returns the number of launches queued; *result_in_alt tells which buffer pair holds the
// sorted result. scratch must hold sort_scratch_bytes(n, key_bits) bytes.
size_t sort_scratch_bytes(int64_t n, int key_bits);
int sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *alt_keys, uint32_t *alt_vals,
               int n, int key_bits, void *scratch, uint32_t *status, cudaStream_t s,
               bool *result_in_alt);

struct EmitArgs {
    const uint32_t *sorted_vals;   // Gaussian indices in depth order, n_rendered of them
    const uint32_t *tiles;
    const uint2 *rect;
    int n_rendered;
    int tiles_x;
    unsigned long long n_pairs;    // capacity of pair_keys / pair_vals
    uint32_t *pair_keys;           // tile id
    uint32_t *pair_vals;           // Gaussian index
    unsigned long long *lookback;
    Counters *counters;
};
void launch_emit(const EmitArgs &a, int num_blocks, cudaStream_t s);

void launch_ranges(const uint32_t *sorted_tile_keys, int n_pairs, int num_tiles, int2 *ranges, cudaStream_t s);

// Render work items ordered by descending list length (log2 buckets): heaviest first.
// A tile whose list has at least 2^(split4_bits-1) entries becomes 4 items (16x4 pixels,
// 4 lanes per pixel), at least 2^(split2_bits-1) entries 2 items (16x8, 2 lanes per pixel),
// otherwise 1 item. Item = tile << 4 | log2(lanes per pixel) << 2 | part. order must hold
// 4 * num_tiles entries; the item count goes to counters->num_items.
void launch_tile_order(const int2 *ranges, int num_tiles, int split2_bits, int split4_bits, uint32_t *order,
                       Counters *counters, cudaStream_t s);

struct RenderArgs {
    const int2 *ranges;
    const uint32_t *tile_order;
    int num_tiles;
    const uint32_t *pair_vals;
    const SplatRec *rec;
    const CutRec *cut;
    int W, H, tiles_x;
    float bg[3];
    float *image;
    float *final_T;
    uint32_t *n_contrib;
    Counters *counters;
};
void launch_render(const RenderArgs &a, int grid, cudaStream_t s);
int render_blocks_per_sm();

// Debug exports
void launch_export_gaussians(int n, const uint8_t *labels_src, const uint32_t *tiles_src,
                             const uint2 *rect_src, const SplatRec *rec, const float *depth_src, uint8_t *labels,
                             float *depth, float *mean2d, float *conic, float *rgb,
                             float *opacity, int32_t *rect, uint32_t *tiles, cudaStream_t s);
void launch_export_pairs(int n_pairs, const uint32_t *tile_keys, const uint32_t *vals,
                         const float *depth, const int2 *ranges, int num_tiles,
                         uint64_t *keys, uint32_t *values, int64_t *ranges_out, cudaStream_t s);

}  // namespace rara
