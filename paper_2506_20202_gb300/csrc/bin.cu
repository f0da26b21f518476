// Step (b) around the sorts: pair emission in depth order, per-tile ranges, the render's
// heaviest-first work order, and the debug exports that rebuild full 64-bit keys.
//
// Sorting the 64-bit keys (tile id << 32 | depth bits) with an LSD radix sort processes
// the 32 depth bits first. Those bits are the same for every pair of one Gaussian, so the
// build sorts the rendered slots by depth once (one entry per slot instead of one per
// pair), emits each slot's pairs in that order, and finishes with the tile-id digit passes
// over the pairs. The result is the same list as the full stable key sort. Tile ids are
// global over the batch (view << tile_bits | ty * tiles_x + tx); with several views the
// slots are ordered by (view, depth) before the emission, so each view's pairs are
// contiguous and the tile sort only needs the local tile bits.
#include "chained_scan.cuh"
#include "rara_internal.cuh"

namespace rara {

namespace {

// View owning a slot: the last view whose slot base is <= the slot.
__device__ __forceinline__ int view_of_slot(const ViewDev *views, int num_views, uint32_t slot)
{
    int lo = 0, hi = num_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].slot_base <= slot) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Emission, persistent over partitions of kEmitPart consecutive depth-ordered slots. A
// partition loads its slots (thread t takes slot r * kBlock + t of row r, coalesced), scans
// their tile counts into per-slot offsets, gets its first pair position from a chained scan,
// and then writes its pairs striped over the block: output k of the partition goes to
// thread k mod kBlock, which finds the slot owning k by binary search over the offsets and
// the tile from k's position inside the slot's rectangle (row-major). Consecutive threads
// thus store consecutive pairs (full 128-byte lines per warp), however uneven the
// rectangles, and a slot with many tiles is spread over the whole block.
constexpr int kEmitItems = 4;
constexpr uint32_t kEmitPart = kBlock * kEmitItems;

__global__ void __launch_bounds__(kBlock) k_emit(EmitArgs a)
{
    __shared__ uint32_t s_hist[4][256];
    __shared__ uint32_t s_off[kEmitPart + 1];      // tile counts, then exclusive offsets
    __shared__ uint32_t s_slot[kEmitPart];
    __shared__ uint32_t s_t0[kEmitPart];           // global tile id of the rectangle's first tile
    __shared__ uint32_t s_geo[kEmitPart];          // rectangle width | view's tiles_x << 16
    __shared__ unsigned s_part;
    __shared__ unsigned long long s_warp[kBlock / 32];
    __shared__ unsigned long long s_prefix;
    for (int t = threadIdx.x; t < 4 * 256; t += kBlock) (&s_hist[0][0])[t] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n = (uint32_t)a.counters->n_rendered;
    const uint32_t *vals = a.counters->depth_in_b ? a.vals_b : a.vals_a;
    const uint32_t parts = (n + kEmitPart - 1) / kEmitPart;
    const int passes = a.tile_passes, dbits = a.tile_digit_bits;
    const uint32_t dmask = (1u << dbits) - 1u;
    bool overflow = false;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_part = atomicAdd(&a.counters->ticket[kTicketEmit], 1u);
        __syncthreads();
        const uint32_t part = s_part;
        if (part >= parts) break;
        const uint32_t first = part * kEmitPart;
        uint32_t slot[kEmitItems];
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            const uint32_t i = first + r * kBlock + threadIdx.x;
            slot[r] = i < n ? __ldg(&vals[i]) : 0u;
        }
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            const int j = r * kBlock + threadIdx.x;
            uint32_t cnt = 0, t0 = 0, geo = 0;
            if (first + j < n) {
                const uint2 rc = __ldg(&a.rect[slot[r]]);
                const int x0 = rc.x & 0xffff, y0 = rc.x >> 16, x1 = rc.y & 0xffff, y1 = rc.y >> 16;
                if (x0 <= x1 && y0 <= y1) {
                    const ViewDev &vw = a.views[view_of_slot(a.views, a.num_views, slot[r])];
                    cnt = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
                    t0 = vw.tile_base + (uint32_t)(y0 * vw.tiles_x + x0);
                    geo = (uint32_t)(x1 - x0 + 1) | ((uint32_t)vw.tiles_x << 16);
                }
            }
            s_off[j] = cnt;
            s_slot[j] = slot[r];
            s_t0[j] = t0;
            s_geo[j] = geo;
        }
        __syncthreads();
        // thread t scans the kEmitItems consecutive counts [t * kEmitItems, ...)
        uint32_t c[kEmitItems];
        uint32_t sum = 0;
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            c[r] = s_off[threadIdx.x * kEmitItems + r];
            sum += c[r];
        }
        unsigned long long incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long w = lane < kBlock / 32 ? s_warp[lane] : 0ull;
            unsigned long long wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += v;
            }
            const unsigned long long total = __shfl_sync(0xffffffffu, wi, 31);
            if (lane < kBlock / 32) s_warp[lane] = wi - w;
            const unsigned long long prefix = warp_chained_prefix(a.lookback, (int)part, total, &a.counters->status);
            if (lane == 0) {
                s_prefix = prefix;
                s_off[kEmitPart] = (uint32_t)total;  // a partition's pairs are < 2^32
            }
        }
        __syncthreads();
        uint32_t run = (uint32_t)(s_warp[warp] + incl - sum);
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            s_off[threadIdx.x * kEmitItems + r] = run;
            run += c[r];
        }
        __syncthreads();
        const unsigned long long pbase = s_prefix;
        const uint32_t total = s_off[kEmitPart];
        int j = 0;  // owner of the previous output of this thread (owners never decrease)
        for (uint32_t k = threadIdx.x; k < total; k += kBlock) {
            // last j with s_off[j] <= k (empty slots share their successor's offset)
            int lo = j, hi = (int)kEmitPart - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= k) lo = mid;
                else hi = mid - 1;
            }
            j = lo;
            const uint32_t r = k - s_off[j];
            const uint32_t geo = s_geo[j];
            const uint32_t w = geo & 0xffffu;
            const uint32_t y = r / w, x = r - y * w;
            const uint32_t t = s_t0[j] + y * (geo >> 16) + x;
            const unsigned long long off = pbase + k;
            if (off < a.cap_pairs) {
                a.pair_keys[off] = t;
                a.pair_vals[off] = s_slot[j];
                for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(t >> (dbits * p)) & dmask], 1u);
            } else {
                overflow = true;
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < a.tile_passes * 256; t += kBlock) {
        const uint32_t v = (&s_hist[0][0])[t];
        if (v) atomicAdd(&a.tile_hist[t], v);
    }
    if (overflow) atomicOr(&a.counters->status, kStatusOverflow);
}

// Ranges: each thread takes 4 consecutive keys (one 16-byte load) and compares them with
// their neighbours; a tile's range starts and ends where its id changes.
__global__ void k_ranges(const uint32_t *keys_a, const uint32_t *keys_b, const Counters *counters,
                         uint32_t cap_pairs, uint32_t num_tiles, int2 *__restrict__ ranges)
{
    const unsigned long long np = counters->n_pairs;
    const uint32_t n = (uint32_t)(np < cap_pairs ? np : cap_pairs);
    const uint32_t *keys = counters->tile_in_b ? keys_b : keys_a;
    const uint32_t nq = (n + 3) / 4;
    constexpr uint32_t kNone = 0xffffffffu;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4 * q;
        uint32_t k[4];
        if (i0 + 4 <= n) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(keys + i0));
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) k[r] = i0 + r < n ? __ldg(&keys[i0 + r]) : kNone;
        }
        const uint32_t prev = i0 > 0 ? __ldg(&keys[i0 - 1]) : kNone;
        const uint32_t next = i0 + 4 < n ? __ldg(&keys[i0 + 4]) : kNone;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t t = k[r];
            if (t >= num_tiles) continue;  // also the padding past n
            const uint32_t before = r > 0 ? k[r - 1] : prev;
            const uint32_t after = r < 3 ? k[r + 1] : next;
            if (before != t) ranges[t].x = (int)(i0 + r);
            if (after != t) ranges[t].y = (int)(i0 + r + 1);
        }
    }
}

// Render work order, heaviest first: tiles are bucketed by the bit length of their list
// length (bucket 32 - bits), and a heavy tile becomes 2 or 4 items. Two launches over all
// tiles: bucket counts, then each block reserves its run in every bucket and writes its
// items there. The order inside a bucket follows the atomics; it only affects scheduling,
// never the image.
__device__ __forceinline__ unsigned items_of(int bits, int split2_bits, int split4_bits)
{
    return bits >= split4_bits ? 2u : (bits >= split2_bits ? 1u : 0u);  // log2 of the items
}

// A global tile id is a real tile unless it is a hole past its view's last tile.
__device__ __forceinline__ bool real_tile(const ViewDev *views, int tile_bits, int t)
{
    const ViewDev &v = views[t >> tile_bits];
    return (t & ((1 << tile_bits) - 1)) < v.tiles_x * v.tiles_y;
}

__global__ void __launch_bounds__(kBlock) k_order_hist(const int2 *__restrict__ ranges, int num_tiles,
                                                       Counters *__restrict__ counters, const ViewDev *views,
                                                       int tile_bits)
{
    __shared__ unsigned s_cnt[33];
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < num_tiles; t += gridDim.x * blockDim.x) {
        if (!real_tile(views, tile_bits, t)) continue;
        const int2 r = ranges[t];
        atomicAdd(&s_cnt[__clz((unsigned)(r.y - r.x))], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 33 && s_cnt[threadIdx.x]) atomicAdd(&counters->order_hist[threadIdx.x], s_cnt[threadIdx.x]);
}

__global__ void __launch_bounds__(kBlock) k_order_scatter(const int2 *__restrict__ ranges, int num_tiles,
                                                          int split2_bits, int split4_bits,
                                                          uint32_t *__restrict__ order, Counters *__restrict__ counters,
                                                          const ViewDev *views, int tile_bits)
{
    __shared__ unsigned s_base[33], s_cnt[33];
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = 0; b < 33; ++b) {
            s_base[b] = acc;
            acc += counters->order_hist[b] << items_of(32 - b, split2_bits, split4_bits);
        }
        if (blockIdx.x == 0) counters->num_items = acc;
    }
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int chunk = (num_tiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * chunk, t1 = min(num_tiles, t0 + chunk);
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        if (!real_tile(views, tile_bits, t)) continue;
        const int2 r = ranges[t];
        const int b = __clz((unsigned)(r.y - r.x));
        atomicAdd(&s_cnt[b], 1u << items_of(32 - b, split2_bits, split4_bits));
    }
    __syncthreads();
    if (threadIdx.x < 33) {
        const unsigned c = s_cnt[threadIdx.x];
        s_base[threadIdx.x] += c ? atomicAdd(&counters->order_cursor[threadIdx.x], c) : 0u;
        s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        if (!real_tile(views, tile_bits, t)) continue;
        const int2 r = ranges[t];
        const int b = __clz((unsigned)(r.y - r.x));
        const unsigned lg = items_of(32 - b, split2_bits, split4_bits);
        const unsigned per = 1u << lg;
        const unsigned pos = s_base[b] + atomicAdd(&s_cnt[b], per);
        for (unsigned p = 0; p < per; ++p) order[pos + p] = ((uint32_t)t << 4) | (lg << 2) | p;
    }
}

__global__ void k_export_gaussians(int n, uint32_t slot_base, const uint8_t *labels_src, const uint32_t *tiles_src,
                                   const uint2 *rect_src, const SplatRec *rec, const float *depth_src,
                                   uint8_t *labels, float *depth, float *mean2d, float *conic, float *rgb,
                                   float *opacity, int32_t *rect, uint32_t *tiles)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t s = slot_base + (uint32_t)i;
    if (labels) labels[i] = labels_src[s];
    const uint32_t nt = tiles_src[s];
    if (tiles) tiles[i] = nt;
    if (!nt) return;
    const SplatRec r = rec[s];
    if (depth) depth[i] = depth_src[s];
    if (mean2d) { mean2d[i] = r.r0.x; mean2d[n + i] = r.r0.y; }
    if (conic) { conic[i] = r.r0.z; conic[n + i] = r.r0.w; conic[2 * n + i] = r.r1.x; }
    if (rgb) { rgb[i] = r.r1.z; rgb[n + i] = r.r1.w; rgb[2 * n + i] = r.r2.x; }
    if (opacity) opacity[i] = r.r1.y;
    if (rect) {
        const uint2 rc = rect_src[s];
        rect[i] = rc.x & 0xffff; rect[n + i] = rc.x >> 16;
        rect[2 * n + i] = rc.y & 0xffff; rect[3 * n + i] = rc.y >> 16;
    }
}

// One block per local tile of the view: its list, in order, at out_offset[t].
__global__ void k_export_pairs(const uint32_t *vals_a, const uint32_t *vals_b, const Counters *counters,
                               const float *depth, const int2 *ranges, uint32_t tile_base, uint32_t slot_base,
                               const uint32_t *out_offset, uint64_t *keys, uint32_t *values, int64_t *ranges_out)
{
    const uint32_t *tv = counters->tile_in_b ? vals_b : vals_a;
    const int t = blockIdx.x;
    const int2 r = ranges[tile_base + t];
    const int len = r.y > r.x ? r.y - r.x : 0;
    const uint32_t off = out_offset[t];
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        const uint32_t slot = tv[r.x + k];
        if (keys) keys[off + k] = ((uint64_t)t << 32) | __float_as_uint(depth[slot]);
        if (values) values[off + k] = slot - slot_base;
    }
    if (ranges_out && threadIdx.x == 0) {
        ranges_out[2 * t] = len ? (int64_t)off : 0;
        ranges_out[2 * t + 1] = len ? (int64_t)off + len : 0;
    }
}

}  // namespace

int emit_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_emit, kBlock, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

void launch_emit(const EmitArgs &a, int grid, cudaStream_t s)
{
    if (grid > 0) k_emit<<<grid, kBlock, 0, s>>>(a);
}

void launch_ranges(const uint32_t *keys_a, const uint32_t *keys_b, const Counters *counters, uint32_t cap_pairs,
                   uint32_t num_tiles, int2 *ranges, int grid, cudaStream_t s)
{
    if (grid > 0) k_ranges<<<grid, 256, 0, s>>>(keys_a, keys_b, counters, cap_pairs, num_tiles, ranges);
}

void launch_tile_order(const int2 *ranges, int num_tiles, int split2_bits, int split4_bits, uint32_t *order,
                       Counters *counters, const ViewDev *views, int tile_bits, int grid, cudaStream_t s)
{
    if (num_tiles <= 0) return;
    const int want = (num_tiles + kBlock * 4 - 1) / (kBlock * 4);
    const int g = want < grid ? want : grid;
    k_order_hist<<<g, kBlock, 0, s>>>(ranges, num_tiles, counters, views, tile_bits);
    k_order_scatter<<<g, kBlock, 0, s>>>(ranges, num_tiles, split2_bits, split4_bits, order, counters, views,
                                         tile_bits);
}

void launch_export_gaussians(int n, uint32_t slot_base, const uint8_t *labels_src, const uint32_t *tiles_src,
                             const uint2 *rect_src, const SplatRec *rec, const float *depth_src, uint8_t *labels,
                             float *depth, float *mean2d, float *conic, float *rgb, float *opacity, int32_t *rect,
                             uint32_t *tiles, cudaStream_t s)
{
    if (n > 0)
        k_export_gaussians<<<(n + 255) / 256, 256, 0, s>>>(n, slot_base, labels_src, tiles_src, rect_src, rec,
                                                           depth_src, labels, depth, mean2d, conic, rgb, opacity,
                                                           rect, tiles);
}

void launch_export_pairs(const uint32_t *vals_a, const uint32_t *vals_b, const Counters *counters, const float *depth,
                         const int2 *ranges, uint32_t tile_base, uint32_t slot_base, int num_tiles,
                         const uint32_t *out_offset, uint64_t *keys, uint32_t *values, int64_t *ranges_out,
                         cudaStream_t s)
{
    if (num_tiles > 0)
        k_export_pairs<<<num_tiles, 128, 0, s>>>(vals_a, vals_b, counters, depth, ranges, tile_base, slot_base,
                                                 out_offset, keys, values, ranges_out);
}

}  // namespace rara
