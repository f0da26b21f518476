// Step (b) around the sort: pair emission in depth order, per-tile ranges, and the
// debug exports that rebuild full 64-bit (tile | depth) keys.
//
// Sorting the 64-bit keys (tile id << 32 | depth bits) with an LSD radix sort processes
// the 32 depth bits first. Those bits are the same for every pair of one Gaussian, so the
// build sorts the rendered Gaussians by depth once (n_rendered elements instead of
// n_pairs), emits each Gaussian's pairs in that order, and finishes with the tile-id digit
// passes over the pairs. The result is the same list as the full stable key sort.
#include "chained_scan.cuh"
#include "rara_internal.cuh"

namespace rara {

namespace {

__global__ void __launch_bounds__(kBlock) k_emit(EmitArgs a)
{
    __shared__ unsigned s_part;
    __shared__ unsigned long long s_warp[kBlock / 32];
    __shared__ unsigned long long s_prefix;
    if (threadIdx.x == 0) s_part = atomicAdd(&a.counters->part_counter[1], 1u);
    __syncthreads();
    const int part = (int)s_part;
    const int j = part * kBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t g = 0, nt = 0;
    if (j < a.n_rendered) {
        g = a.sorted_vals[j];
        nt = a.tiles[g];
    }
    // block exclusive scan of nt
    unsigned long long incl = nt;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < kBlock / 32 ? s_warp[lane] : 0ull;
        unsigned long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        const unsigned long long total = __shfl_sync(0xffffffffu, wi, 31);
        if (lane < kBlock / 32) s_warp[lane] = wi - w;
        const unsigned long long prefix = warp_chained_prefix(a.lookback, part, total, &a.counters->status);
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    if (nt) {
        unsigned long long off = s_prefix + s_warp[warp] + incl - nt;
        const uint2 rc = a.rect[g];
        const int x0 = rc.x & 0xffff, y0 = rc.x >> 16, x1 = rc.y & 0xffff, y1 = rc.y >> 16;
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                if (off < a.n_pairs) {  // always true unless a bounded wait gave up
                    a.pair_keys[off] = (uint32_t)(y * a.tiles_x + x);
                    a.pair_vals[off] = g;
                }
                ++off;
            }
    }
}

__global__ void k_ranges(const uint32_t *__restrict__ keys, int n, int num_tiles, int2 *__restrict__ ranges)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = keys[i];
    if (t >= (uint32_t)num_tiles) return;
    if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
    if (i == n - 1 || keys[i + 1] != t) ranges[t].y = i + 1;
}

__global__ void k_export_gaussians(int n, const uint8_t *labels_src, const uint32_t *tiles_src,
                                   const uint2 *rect_src, const SplatRec *rec, const float *depth_src,
                                   uint8_t *labels, float *depth,
                                   float *mean2d, float *conic, float *rgb, float *opacity, int32_t *rect,
                                   uint32_t *tiles)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (labels) labels[i] = labels_src[i];
    const uint32_t nt = tiles_src[i];
    if (tiles) tiles[i] = nt;
    if (!nt) return;
    const SplatRec r = rec[i];
    if (depth) depth[i] = depth_src[i];
    if (mean2d) { mean2d[i] = r.r0.x; mean2d[n + i] = r.r0.y; }
    if (conic) { conic[i] = r.r0.z; conic[n + i] = r.r0.w; conic[2 * n + i] = r.r1.x; }
    if (rgb) { rgb[i] = r.r1.z; rgb[n + i] = r.r1.w; rgb[2 * n + i] = r.r2.x; }
    if (opacity) opacity[i] = r.r1.y;
    if (rect) {
        const uint2 rc = rect_src[i];
        rect[i] = rc.x & 0xffff; rect[n + i] = rc.x >> 16;
        rect[2 * n + i] = rc.y & 0xffff; rect[3 * n + i] = rc.y >> 16;
    }
}

__global__ void k_export_pairs(int np, const uint32_t *tile_keys, const uint32_t *vals, const float *depth,
                               const int2 *ranges, int num_tiles, uint64_t *keys, uint32_t *values,
                               int64_t *ranges_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) {
        const uint32_t g = vals[i];
        if (keys) keys[i] = ((uint64_t)tile_keys[i] << 32) | __float_as_uint(depth[g]);
        if (values) values[i] = g;
    }
    if (ranges_out && i < num_tiles) {
        const int2 r = ranges[i];
        ranges_out[2 * i] = r.x;
        ranges_out[2 * i + 1] = r.y;
    }
}

// One block: bucket the tiles by the bit length of their list length, longest first, and
// expand heavy tiles into 2 or 4 work items. The order inside a bucket is whatever the
// atomics give; it only affects scheduling, never the image.
__global__ void __launch_bounds__(1024) k_tile_order(const int2 *__restrict__ ranges, int num_tiles, int split2_bits,
                                                     int split4_bits, uint32_t *__restrict__ order,
                                                     Counters *__restrict__ counters)
{
    __shared__ unsigned s_cnt[33];
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < num_tiles; t += blockDim.x) {
        const int2 r = ranges[t];
        atomicAdd(&s_cnt[__clz((unsigned)(r.y - r.x))], 1u);  // bucket = 32 - bit length
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = 0; b < 33; ++b) {
            const int bits = 32 - b;
            const unsigned per = bits >= split4_bits ? 4u : (bits >= split2_bits ? 2u : 1u);
            const unsigned c = s_cnt[b];
            s_cnt[b] = acc;
            acc += c * per;
        }
        counters->num_items = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < num_tiles; t += blockDim.x) {
        const int2 r = ranges[t];
        const int b = __clz((unsigned)(r.y - r.x));
        const int bits = 32 - b;
        const unsigned lg = bits >= split4_bits ? 2u : (bits >= split2_bits ? 1u : 0u);
        const unsigned per = 1u << lg;
        const unsigned pos = atomicAdd(&s_cnt[b], per);
        for (unsigned p = 0; p < per; ++p) order[pos + p] = ((uint32_t)t << 4) | (lg << 2) | p;
    }
}

}  // namespace

void launch_tile_order(const int2 *ranges, int num_tiles, int split2_bits, int split4_bits, uint32_t *order,
                       Counters *counters, cudaStream_t s)
{
    if (num_tiles > 0)
        k_tile_order<<<1, 1024, 0, s>>>(ranges, num_tiles, split2_bits, split4_bits, order, counters);
}

void launch_emit(const EmitArgs &a, int num_blocks, cudaStream_t s)
{
    if (num_blocks > 0) k_emit<<<num_blocks, kBlock, 0, s>>>(a);
}

void launch_ranges(const uint32_t *keys, int n, int num_tiles, int2 *ranges, cudaStream_t s)
{
    if (n > 0) k_ranges<<<(n + 255) / 256, 256, 0, s>>>(keys, n, num_tiles, ranges);
}

void launch_export_gaussians(int n, const uint8_t *labels_src, const uint32_t *tiles_src, const uint2 *rect_src,
                             const SplatRec *rec, const float *depth_src, uint8_t *labels, float *depth,
                             float *mean2d, float *conic, float *rgb, float *opacity, int32_t *rect, uint32_t *tiles,
                             cudaStream_t s)
{
    if (n > 0)
        k_export_gaussians<<<(n + 255) / 256, 256, 0, s>>>(n, labels_src, tiles_src, rect_src, rec, depth_src,
                                                           labels, depth, mean2d, conic, rgb, opacity, rect, tiles);
}

void launch_export_pairs(int np, const uint32_t *tile_keys, const uint32_t *vals, const float *depth,
                         const int2 *ranges, int num_tiles, uint64_t *keys, uint32_t *values, int64_t *ranges_out,
                         cudaStream_t s)
{
    const int m = np > num_tiles ? np : num_tiles;
    if (m > 0)
        k_export_pairs<<<(m + 255) / 256, 256, 0, s>>>(np, tile_keys, vals, depth, ranges, num_tiles, keys, values,
                                                       ranges_out);
}

}  // namespace rara
