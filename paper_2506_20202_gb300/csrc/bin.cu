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
#include "render_common.cuh"

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

// Emission, persistent over partitions of kEmitPart consecutive depth-ordered slots.
//
// A tile of a slot's rectangle lists the slot when some pixel centre of the tile can have
// q <= q_cut (elsewhere alpha0 = opacity exp(-q/2) < 1/255 or q > 9, and the pixel would skip
// the Gaussian). In tile row ty the pixel centres span the band y in [py0, py1]; the part of
// the ellipse q <= q_cut inside the band is convex, so its x-extent is one interval [XL, XR]
// and the listing tiles of the row are the contiguous columns whose pixel centres reach it.
// With the conic (a, b, c) and D = ac - b^2, the ellipse's left boundary
// x_l(y) = (-b y - sqrt(a q_cut - D y^2)) / a is convex with its minimum at the leftmost point
// y_L = b sqrt(q_cut / (c D)), so XL = x_l(y_L clamped to the band); XR mirrors it
// (row_span below; offsets relative to the projected centre).
//
// A partition loads its slots and reserves room for their rectangles' rows in a
// shared-memory row pool (block scan of the rectangle heights); thread t owns slots 2t and
// 2t + 1. Each thread computes its slots' row spans into the pool (first column and the
// slot's pairs before the row) and their listed-pair counts; the block scans the counts into
// per-slot offsets and a chained scan places the partition. Each warp then writes the pairs
// of its own 64 slots, 32 consecutive pairs at a time (coalesced stores): the slots starting
// in the window mark their first position in a warp-private array, a shuffle prefix maximum
// gives every lane the slot owning its pair, and a binary search over the slot's pooled rows
// gives the tile. A slot whose rows do not fit the pool recomputes its spans when it writes.
constexpr int kEmitItems = 2;
constexpr uint32_t kEmitPart = kBlock * kEmitItems;
constexpr uint32_t kRowPool = 4096;
constexpr uint32_t kNoPool = 0xffffffffu;

// Per-splat constants of the listing spans: conic (a, b, c), q_cut and their derived terms.
struct SpanGeo {
    float mx, my, aq, D, ia, b, ymax, yl;
    int x0, x1, y0, W, H, tw, th;
    bool ok;
};

// From the slot's emission record (rectangle, centre, conic, q_cut).
// sqrt(x) for x >= 0 from the special function unit's reciprocal square root (0 at 0);
// the listing needs the spans only to within the float32 tolerance of its threshold.
__device__ __forceinline__ float fast_sqrt(float x)
{
    return x > 0.0f ? __fmul_rn(x, rsqrtf(x)) : 0.0f;
}

__device__ __forceinline__ SpanGeo span_geo(const EmitRec &e, const ViewDev &vw)
{
    SpanGeo g;
    const float a = e.ca, b = e.cb, c = e.cc;
    const float qc = e.qcut;
    const uint2 rc = e.rect;
    g.mx = e.mx; g.my = e.my; g.b = b;
    g.D = fmaf(a, c, -__fmul_rn(b, b));
    g.aq = __fmul_rn(a, qc);
    g.ia = __fdividef(1.0f, a);
    g.ok = qc >= 0.0f && g.D > 0.0f;
    g.ymax = g.ok ? fast_sqrt(__fdividef(g.aq, g.D)) : 0.0f;
    g.yl = g.ok ? __fmul_rn(b, fast_sqrt(__fdividef(qc, __fmul_rn(c, g.D)))) : 0.0f;
    g.x0 = rc.x & 0xffff; g.y0 = rc.x >> 16; g.x1 = rc.y & 0xffff;
    g.W = vw.cam.W; g.H = vw.cam.H;
    g.tw = vw.tile_w; g.th = vw.tile_h;
    return g;
}

// Listing columns [lo, lo + count) of tile row ty (count 0 when none). Every product that
// feeds a sum is rounded on its own (__fmul_rn), so each call site computes the same spans.
__device__ __forceinline__ void row_span(const SpanGeo &g, int ty, int &lo, int &count)
{
    const float by0 = __fsub_rn((float)(ty * g.th) + 0.5f, g.my);
    const float by1 = __fsub_rn((float)min((ty + 1) * g.th, g.H) - 0.5f, g.my);
    const float y0 = fmaxf(by0, -g.ymax), y1 = fminf(by1, g.ymax);
    count = 0;
    lo = g.x0;
    if (!(g.ok && y0 <= y1)) return;
    const float ya = fminf(y1, fmaxf(y0, g.yl)), yb = fminf(y1, fmaxf(y0, -g.yl));
    const float ra = fast_sqrt(fmaxf(0.0f, fmaf(-__fmul_rn(g.D, ya), ya, g.aq)));
    const float rb = fast_sqrt(fmaxf(0.0f, fmaf(-__fmul_rn(g.D, yb), yb, g.aq)));
    const float XL = __fmul_rn(__fsub_rn(-__fmul_rn(g.b, ya), ra), g.ia);
    const float XR = __fmul_rn(__fadd_rn(-__fmul_rn(g.b, yb), rb), g.ia);
    if (XL > __fsub_rn((float)g.W - 0.5f, g.mx)) return;  // right of the image's last pixel centres
    // column tx reaches the interval iff tx tw + (tw - 0.5) - mx >= XL and tx tw + 0.5 - mx <= XR
    // (tile widths are powers of two, so 1 / tw is exact and the products are the quotients)
    const float itw = 1.0f / (float)g.tw;
    const int c0 = max(g.x0, (int)ceilf(__fmul_rn(__fsub_rn(__fadd_rn(XL, g.mx), (float)g.tw - 0.5f), itw)));
    const int c1 = min(g.x1, (int)floorf(__fmul_rn(__fsub_rn(__fadd_rn(XR, g.mx), 0.5f), itw)));
    lo = c0;
    count = max(0, c1 - c0 + 1);
}

// Exclusive block scan (256 threads) of per-thread sums; returns this thread's prefix and
// the block total in *total. Uses s_w[8].
__device__ __forceinline__ uint32_t block_scan_u32(uint32_t v, uint32_t *s_w, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int w = 0; w < kBlock / 32; ++w) {
        const uint32_t u = s_w[w];
        if (w < warp) before += u;
        all += u;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(kBlock) k_emit(EmitArgs a)
{
    __shared__ uint32_t s_hist[4][256];
    __shared__ uint32_t s_off[kEmitPart + 1];       // pair offsets of the slots, then the total
    __shared__ uint32_t s_roff[kEmitPart];          // first pooled row of the slot, or kNoPool
    __shared__ uint32_t s_nrows[kEmitPart];         // rows of the rectangle
    __shared__ uint32_t s_slot[kEmitPart];
    __shared__ uint32_t s_view[kEmitPart];
    __shared__ uint32_t s_t0[kEmitPart];            // global tile id of the rectangle's origin
    __shared__ uint32_t s_tx[kEmitPart];            // the view's tiles per row
    __shared__ uint16_t s_rcol[kRowPool];           // first listing column of a pooled row (from x0)
    __shared__ uint32_t s_rcum[kRowPool];           // the slot's pairs before the row
    __shared__ int s_mark[kBlock / 32][32];
    __shared__ uint32_t s_w[kBlock / 32];
    __shared__ unsigned s_part;
    __shared__ unsigned long long s_warp[kBlock / 32];
    __shared__ unsigned long long s_prefix;
    for (int t = threadIdx.x; t < 4 * 256; t += kBlock) (&s_hist[0][0])[t] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool shared = a.shared_list != 0;
    const uint32_t n = (uint32_t)(shared ? a.counters->n_union : a.counters->n_rendered);
    // the slots in (view, depth) order: the depth sort's result, or (one-camera batches) the
    // expansion's, which is in the other buffer; with a shared listing, the union's Gaussians
    // in depth order (the depth sort's result)
    const uint32_t *vals = (a.counters->depth_in_b != 0u) != (a.expanded != 0) ? a.vals_b : a.vals_a;
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
        uint32_t slot[kEmitItems], rows[kEmitItems], lslot[kEmitItems];
        int sview[kEmitItems];
        uint2 rc[kEmitItems];
        uint32_t nrows = 0;
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            const uint32_t i = first + threadIdx.x * kEmitItems + r;
            slot[r] = i < n ? __ldg(&vals[i]) : 0u;  // the value the pairs carry
            lslot[r] = slot[r];                      // the slot whose rectangle and splat are read
            sview[r] = 0;
            if (shared && i < n) {
                const uint32_t vm = __ldg(&a.vmask[slot[r]]);   // non-zero: some view renders it
                sview[r] = vm ? __ffs(vm) - 1 : 0;
                lslot[r] = a.views[sview[r]].slot_base + slot[r];
            }
            rc[r] = i < n ? __ldg(&a.erec[lslot[r]].rect) : make_uint2(0u, 0u);
            const int y0 = rc[r].x >> 16, y1 = rc[r].y >> 16;
            const int x0 = rc[r].x & 0xffff, x1 = rc[r].y & 0xffff;
            rows[r] = (i < n && x0 <= x1 && y0 <= y1) ? (uint32_t)(y1 - y0 + 1) : 0u;
            nrows += rows[r];
        }
        uint32_t allrows;
        uint32_t rbase = block_scan_u32(nrows, s_w, &allrows);
        uint32_t cnt[kEmitItems];
        uint32_t sum = 0;
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            const int j = threadIdx.x * kEmitItems + r;
            cnt[r] = 0;
            uint32_t v = 0, roff = kNoPool, t0 = 0, txs = 0;
            if (rows[r]) {
                v = shared ? (uint32_t)sview[r] : (uint32_t)view_of_slot(a.views, a.num_views, slot[r]);
                const ViewDev &vw = a.views[v];
                const SpanGeo g = span_geo(a.erec[lslot[r]], vw);
                t0 = (shared ? 0u : vw.tile_base) + (uint32_t)(g.y0 * vw.tiles_x + g.x0);
                txs = (uint32_t)vw.tiles_x;
                const bool pooled = rbase + rows[r] <= kRowPool;
                if (pooled) roff = rbase;
                for (uint32_t k = 0; k < rows[r]; ++k) {
                    int lo, c;
                    row_span(g, g.y0 + (int)k, lo, c);
                    if (pooled) {
                        s_rcol[rbase + k] = (uint16_t)(lo - g.x0);
                        s_rcum[rbase + k] = cnt[r];
                    }
                    cnt[r] += (uint32_t)c;
                }
            }
            rbase += rows[r];
            s_roff[j] = roff;
            s_nrows[j] = rows[r];
            s_slot[j] = slot[r];
            s_view[j] = v;
            s_t0[j] = t0;
            s_tx[j] = txs;
            sum += cnt[r];
        }
        // pair offsets of the slots, and the partition's place among all pairs
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
                if (part == parts - 1) a.counters->n_pairs = prefix + total;  // all listed pairs
            }
        }
        __syncthreads();
        uint32_t run = (uint32_t)(s_warp[warp] + incl - sum);
#pragma unroll
        for (int r = 0; r < kEmitItems; ++r) {
            s_off[threadIdx.x * kEmitItems + r] = run;
            run += cnt[r];
        }
        __syncthreads();
        // this warp's slots [jw, jw + 64) and pairs [ws, we)
        const unsigned long long pbase = s_prefix;
        const int jw = warp * 32 * kEmitItems;
        const uint32_t ws = s_off[jw], we = s_off[jw + 32 * kEmitItems];
        int carry = -1;
        for (uint32_t c0 = ws; c0 < we; c0 += 32) {
            s_mark[warp][lane] = -1;
            __syncwarp();
#pragma unroll
            for (int r = 0; r < kEmitItems; ++r) {
                const int j = jw + lane * kEmitItems + r;
                const uint32_t st = s_off[j];
                if (s_off[j + 1] > st && st >= c0 && st < c0 + 32u) s_mark[warp][st - c0] = j;
            }
            __syncwarp();
            int owner = s_mark[warp][lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, owner, o);
                if (lane >= o) owner = max(owner, u);
            }
            owner = max(owner, carry);
            carry = __shfl_sync(0xffffffffu, owner, 31);
            __syncwarp();
            const uint32_t k = c0 + (uint32_t)lane;
            if (k >= we || owner < 0) continue;
            const int j = owner;
            const uint32_t r = k - s_off[j];
            int dy = 0, dx = 0;
            const uint32_t roff = s_roff[j];
            if (roff != kNoPool) {
                // last pooled row of the slot with s_rcum <= r (rows without pairs share the
                // next row's value, so the row found has pairs)
                int rl = (int)roff, rh = (int)roff + (int)s_nrows[j] - 1;
                while (rl < rh) {
                    const int mid = (rl + rh + 1) >> 1;
                    if (s_rcum[mid] <= r) rl = mid;
                    else rh = mid - 1;
                }
                dy = rl - (int)roff;
                dx = (int)s_rcol[rl] + (int)(r - s_rcum[rl]);
            } else {
                const uint32_t sl = shared ? a.views[s_view[j]].slot_base + s_slot[j] : s_slot[j];
                const SpanGeo g = span_geo(a.erec[sl], a.views[s_view[j]]);
                uint32_t rr = r;
                for (int k2 = 0; k2 < (int)s_nrows[j]; ++k2) {  // the spans of the count phase
                    int lo2, c2;
                    row_span(g, g.y0 + k2, lo2, c2);
                    if (rr < (uint32_t)c2) {
                        dy = k2;
                        dx = lo2 - g.x0 + (int)rr;
                        break;
                    }
                    rr -= (uint32_t)c2;
                }
            }
            const uint32_t t = s_t0[j] + (uint32_t)dy * s_tx[j] + (uint32_t)dx;
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

// Shared listing, launch 1: view v's count of partition p (the union pairs [p kListPart,
// (p + 1) kListPart) whose Gaussian view v renders), one warp per partition. Lane v adds up
// the ballots of bit v of the pairs' view masks, four rounds of 32 pairs at a time (their
// values, then their masks, loaded together).
__global__ void __launch_bounds__(kBlock) k_list_count(ListArgs a)
{
    const int lane = threadIdx.x & 31;
    const bool in_b = a.counters->tile_in_b != 0u;
    const uint32_t *vals = in_b ? a.vals_b : a.vals_a;
    const unsigned long long np = a.counters->n_pairs;
    const uint32_t n = (uint32_t)(np < a.cap_pairs ? np : a.cap_pairs);
    const uint32_t parts = (n + kListPart - 1) / kListPart;
    const int nv = a.num_views;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.counters->list_src = in_b ? 1u : 0u;
        a.counters->n_list = n;
    }
    const uint32_t warps = gridDim.x * (kBlock / 32);
    for (uint32_t part = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); part < parts; part += warps) {
        const uint32_t first = part * kListPart, last = min(first + kListPart, n);
        uint32_t c = 0;
        for (uint32_t j0 = first; j0 < last; j0 += 128) {
            uint32_t m[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t j = j0 + 32u * k + (uint32_t)lane;
                m[k] = j < last ? __ldg(&vals[j]) : 0xffffffffu;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) m[k] = m[k] != 0xffffffffu ? __ldg(&a.vmask[m[k]]) : 0u;
            for (int v = 0; v < nv; ++v) {
                uint32_t s = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) s += (uint32_t)__popc(__ballot_sync(0xffffffffu, (m[k] >> v) & 1u));
                if (lane == v) c += s;
            }
        }
        if (lane < nv) a.part_counts[(size_t)lane * a.max_parts + part] = c;
    }
}

// Launch 2: one block per view scans its partition counts in place (exclusive) and stores the
// view's total after the columns.
__global__ void __launch_bounds__(1024) k_list_scan(ListArgs a)
{
    __shared__ uint32_t s_w[32];
    const int v = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n = (uint32_t)a.counters->n_list;
    const uint32_t parts = (n + kListPart - 1) / kListPart;
    uint32_t *col = a.part_counts + (size_t)v * a.max_parts;
    const uint32_t per = (parts + 1023) / 1024;
    const uint32_t p0 = threadIdx.x * per, p1 = min(p0 + per, parts);
    uint32_t sum = 0;
    for (uint32_t p = p0; p < p1; ++p) sum += col[p];
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < 32; ++w) {
        const uint32_t u = s_w[w];
        if (w < warp) before += u;
        total += u;
    }
    uint32_t run = before + incl - sum;
    for (uint32_t p = p0; p < p1; ++p) {
        const uint32_t c = col[p];
        col[p] = run;
        run += c;
    }
    if (threadIdx.x == 0) a.part_counts[(size_t)kListViews * a.max_parts + v] = total;
}

// Launch 3: one warp per partition writes every view's slots of its pairs at B_v + C_v(j) and,
// where a tile's run starts or ends, that tile's range bound in every view.
__global__ void __launch_bounds__(kBlock) k_list_scatter(ListArgs a)
{
    const int lane = threadIdx.x & 31;
    const bool in_b = a.counters->list_src != 0u;
    const uint32_t *keys = in_b ? a.keys_b : a.keys_a;
    const uint32_t *vals = in_b ? a.vals_b : a.vals_a;
    uint32_t *out = in_b ? a.vals_a : a.vals_b;
    const uint32_t n = (uint32_t)a.counters->n_list;
    const uint32_t parts = (n + kListPart - 1) / kListPart;
    const int nv = a.num_views;
    const uint32_t cap = a.cap_pairs;
    // lane v: B_v (the pairs of the views before v) and the view's first slot
    const uint32_t tot = lane < nv ? a.part_counts[(size_t)kListViews * a.max_parts + lane] : 0u;
    unsigned long long base = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, base, o);
        if (lane >= o) base += u;
    }
    const unsigned long long all = __shfl_sync(0xffffffffu, base, 31);
    base -= tot;
    const uint32_t stride = a.slot_stride;  // view v's slot of Gaussian g is v * stride + g
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.counters->n_pairs = all;
        if (all > cap) atomicOr(&a.counters->status, kStatusOverflow);
        a.counters->tile_in_b = in_b ? 0u : 1u;   // the views' lists are in the other buffer
    }
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t warps = gridDim.x * (kBlock / 32);
    constexpr uint32_t kNone = 0xffffffffu;
    for (uint32_t part = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); part < parts; part += warps) {
        const uint32_t first = part * kListPart, last = min(first + kListPart, n);
        // lane v: view v's next position, clamped at the capacity (positions past it are not
        // written; the overflow is flagged above)
        unsigned long long r64 = lane < nv ? base + a.part_counts[(size_t)lane * a.max_parts + part] : 0ull;
        uint32_t run = (uint32_t)(r64 < cap ? r64 : cap);
        const uint32_t key_before = first > 0 ? __ldg(&keys[first - 1]) : kNone;
        const uint32_t key_after = last < n ? __ldg(&keys[last]) : kNone;
        // loads run ahead: this round's value, key and mask, the next round's value and key
        uint32_t j = first + (uint32_t)lane;
        uint32_t g = j < last ? __ldg(&vals[j]) : 0u, t = j < last ? __ldg(&keys[j]) : kNone;
        uint32_t g1 = j + 32 < last ? __ldg(&vals[j + 32]) : 0u, t1 = j + 32 < last ? __ldg(&keys[j + 32]) : kNone;
        uint32_t m = j < last ? __ldg(&a.vmask[g]) : 0u;
        uint32_t t_prev = key_before;  // the previous round's keys (every lane: the key before)
        for (uint32_t j0 = first; j0 < last; j0 += 32) {
            j = j0 + (uint32_t)lane;
            const bool ok = j < last;
            const uint32_t m1 = j + 32 < last ? __ldg(&a.vmask[g1]) : 0u;
            const uint32_t g2 = j + 64 < last ? __ldg(&vals[j + 64]) : 0u;
            const uint32_t t2 = j + 64 < last ? __ldg(&keys[j + 64]) : kNone;
            uint32_t tp = __shfl_up_sync(0xffffffffu, t, 1);
            uint32_t tn = __shfl_down_sync(0xffffffffu, t, 1);
            const uint32_t round_before = __shfl_sync(0xffffffffu, t_prev, 31);
            const uint32_t round_after = __shfl_sync(0xffffffffu, t1, 0);
            if (lane == 0) tp = round_before;
            if (j + 1 == last) tn = key_after;
            else if (lane == 31) tn = round_after;
            const bool start = ok && tp != t, end = ok && tn != t;
            uint32_t gv = g;  // the pair's slot in view v
            for (int v = 0; v < nv; ++v, gv += stride) {
                const bool bit = ((m >> v) & 1u) != 0u;
                const uint32_t b = __ballot_sync(0xffffffffu, bit);
                const uint32_t pos = __shfl_sync(0xffffffffu, run, v) + (uint32_t)__popc(b & lt);
                if (bit && pos < cap) out[pos] = gv;
                if (start || end) {
                    int2 *rg = &a.ranges[((uint32_t)v << a.tile_bits) | t];
                    if (start) rg->x = (int)(pos < cap ? pos : cap);
                    const uint32_t e = pos + (bit ? 1u : 0u);
                    if (end) rg->y = (int)(e < cap ? e : cap);
                }
                if (lane == v) {
                    const uint32_t nr = run + (uint32_t)__popc(b);
                    run = nr < cap ? nr : cap;
                }
            }
            t_prev = t;
            g = g1; t = t1; m = m1;
            g1 = g2; t1 = t2;
        }
    }
}

// Render work order, heaviest first: tiles are bucketed by the bit length of their list
// length (bucket 32 - bits), and a heavy tile becomes 2 or 4 items. Two launches over all
// tiles: bucket counts, then each block reserves its run in every bucket and writes its
// items there. The order inside a bucket follows the atomics; it only affects scheduling,
// never the image.
// log2 of the lanes per pixel of a tile whose list length has `bits` bits, clamped to what
// the tile's area allows (at least 1 and at most 4 items of 256 lanes: area_log2 =
// log2(pixels / 64) gives log2(L) in [2 - area_log2, 4 - area_log2]).
__device__ __forceinline__ unsigned lpp_of(int bits, int split2_bits, int split4_bits, int area_log2)
{
    const int l = bits >= split4_bits ? 2 : (bits >= split2_bits ? 1 : 0);
    return (unsigned)min(min(2, 4 - area_log2), max(2 - area_log2, l));
}

// log2 of the items of such a tile: L pixels-worth of lanes / 256 = L * 2^area_log2 / 4.
__device__ __forceinline__ unsigned items_of(int bits, int split2_bits, int split4_bits, int area_log2)
{
    return lpp_of(bits, split2_bits, split4_bits, area_log2) + (unsigned)area_log2 - 2u;
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
                                                          int split2_bits, int split4_bits, int area_log2,
                                                          uint32_t *__restrict__ order, Counters *__restrict__ counters,
                                                          const ViewDev *views, int tile_bits)
{
    __shared__ unsigned s_base[33], s_cnt[33];
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int b = 0; b < 33; ++b) {
            s_base[b] = acc;
            acc += counters->order_hist[b] << items_of(32 - b, split2_bits, split4_bits, area_log2);
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
        atomicAdd(&s_cnt[b], 1u << items_of(32 - b, split2_bits, split4_bits, area_log2));
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
        const unsigned lg = lpp_of(32 - b, split2_bits, split4_bits, area_log2);
        const unsigned per = 1u << items_of(32 - b, split2_bits, split4_bits, area_log2);
        const unsigned pos = s_base[b] + atomicAdd(&s_cnt[b], per);
        for (unsigned p = 0; p < per; ++p) order[pos + p] = ((uint32_t)t << 4) | (lg << 2) | p;
    }
}

__global__ void k_export_gaussians(int n, uint32_t slot_base, const uint8_t *labels_src, const uint32_t *tiles_src,
                                   const EmitRec *erec_src, const uint32_t *vmask, const ViewDev *views,
                                   const SplatRec *rec, const float *depth_src,
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
        // a shared listing keeps the emission record in the first view that renders the
        // Gaussian (the lowest bit of its view mask, set since this view renders it)
        const uint32_t vm = vmask ? vmask[i] : 0u;
        const uint32_t es = vm ? views[__ffs(vm) - 1].slot_base + (uint32_t)i : s;
        const uint2 rc = erec_src[es].rect;
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

void launch_lists(const ListArgs &a, int grid, cudaStream_t s)
{
    if (grid <= 0 || a.num_views <= 0 || a.num_views > kListViews) return;
    k_list_count<<<grid, kBlock, 0, s>>>(a);
    k_list_scan<<<a.num_views, 1024, 0, s>>>(a);
    k_list_scatter<<<grid, kBlock, 0, s>>>(a);
}

void launch_tile_order(const int2 *ranges, int num_tiles, int split2_bits, int split4_bits, int area_log2,
                       uint32_t *order, Counters *counters, const ViewDev *views, int tile_bits, int grid,
                       cudaStream_t s)
{
    if (num_tiles <= 0) return;
    const int want = (num_tiles + kBlock * 4 - 1) / (kBlock * 4);
    const int g = want < grid ? want : grid;
    k_order_hist<<<g, kBlock, 0, s>>>(ranges, num_tiles, counters, views, tile_bits);
    k_order_scatter<<<g, kBlock, 0, s>>>(ranges, num_tiles, split2_bits, split4_bits, area_log2, order, counters,
                                         views, tile_bits);
}

void launch_export_gaussians(int n, uint32_t slot_base, const uint8_t *labels_src, const uint32_t *tiles_src,
                             const EmitRec *erec_src, const uint32_t *vmask, const ViewDev *views,
                             const SplatRec *rec, const float *depth_src, uint8_t *labels,
                             float *depth, float *mean2d, float *conic, float *rgb, float *opacity, int32_t *rect,
                             uint32_t *tiles, cudaStream_t s)
{
    if (n > 0)
        k_export_gaussians<<<(n + 255) / 256, 256, 0, s>>>(n, slot_base, labels_src, tiles_src, erec_src, vmask, views, rec,
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
