// Steps (c)+(d): per-tile front-to-back compositing with the RaRa decay weight.
//
// Work items come from a queue ordered heaviest first (by tile-list length). An item is a
// 256-thread block over a band of a tile's rows with L = 1, 2 or 4 lanes per pixel (256 / L
// pixels): a light 16x16 tile is one item of one lane per pixel, a heavy one 2 or 4 items of
// 16x8 or 16x4 pixels with 2 or 4 lanes per pixel (an 8x8 tile is always one item of 4 lanes
// per pixel, a 32x16 tile 2 or 4 items). The lanes of a pixel take consecutive list entries
// and combine them with a prefix product of (1 - alpha), so the pixel's chain of dependent
// steps is 2 or 4 times shorter. That
// matters because a pixel that never saturates (for example one that looks through the
// clipped region, where cutoff Gaussians get w ~ 0) walks its whole list, and the longest
// such walk bounds the launch.
//
// The tile's depth-sorted list is walked in batches of D entries (the blend batch depth, 128,
// 256 or 512, chosen by the autotuner): the threads gather the batch's splat records (and,
// for cutoff Gaussians, their ray-tracing records) into shared memory.
// Each warp owns a rectangle of the item's pixels; before walking a 32-entry chunk of the
// batch, its lanes test one entry each against the rectangle (exact minimum of q over the
// rectangle of pixel centres) and the warp walks only the entries whose q <= 9 support
// reaches the rectangle, in list order. An entry it skips has q > 9 at all its pixels and
// would have been skipped pixel by pixel.
//
// Decay weight (Eq. 4-8, Eq. 11, Algorithm 1 step 2), evaluated in the unit-sphere frame
// of the ellipsoid M = k R S without forming t1, t2 or t_p explicitly (render_common.cuh):
//   local ray   u(tau) = -G + tau V,  V = G + p,  p = P (dx, dy)   (tau = 1 at the centre
//               depth for the central ray; dx, dy = pixel offset from the projected centre)
//   chord       the ray meets the sphere iff its squared distance from the centre,
//               cc = |p x G|^2 / V.V, is below 1; the chord's midpoint is c = p - (p.V/V.V) V
//   in front    t1 > 0  <=>  G.V > 0 and (G.V)^2 > (1 - cc) V.V
//   plane       s(u) = d_ep + m . u with m = M^T n, linear along the ray:
//               s1,2 = d_ep + m.c -/+ sqrt(1 - cc) (m.V) / |V|
//   weight      both >= 0: 1; both < 0: 0; otherwise the visible share of the chord,
//               max(s1, s2) / |s2 - s1|  (= (t2 - t_p)/(t2 - t1) or (t_p - t1)/(t2 - t1));
//               all three cases are clamp(1/2 + (d_ep + m.c) / (2 |h|), 0, 1), h = s2 - s_mid.
// Everything is a polynomial in (dx, dy) with coefficients the products of G, P and m that
// the preprocess stores, so a pixel needs about 50 instructions for the full weight.
// Because w <= 1, an entry whose unweighted alpha is already below 1/255 is skipped before
// the weight is computed (the weighted alpha could only be smaller). The preprocess marks
// which cutoff Gaussians the plane actually meets (|d_ep| <= |m|); only those evaluate the
// full weight, the others are w = 1 (visible side) or a hit test (invisible side).
#include "rara_internal.cuh"
#include "render_common.cuh"

namespace rara {

namespace {

// Work counters of a render launch (the units of its roofline). COUNT = false drops them:
// the graph replays of a batch, which nothing reads them from, run without them.
template <bool COUNT>
struct Tally {
    uint32_t evaluated = 0, walked = 0, cut = 0, tested = 0;
    __device__ __forceinline__ void add(uint32_t &c, bool v)
    {
        if (COUNT) c += v ? 1u : 0u;
    }
};

// Shared-memory entries of a block for batch depth D: D, or with D = 32 (each warp staging its
// own 32-entry chunks) 32 per warp.
template <int D>
__host__ __device__ constexpr int stage_entries() { return D == 32 ? kBlock : D; }

// One work item: LPP lanes per pixel over rows [part * rows, (part + 1) * rows) of a
// tile_w x tile_h tile, rows = 256 / (LPP tile_w). Warp rectangles of RW x RH pixels:
//   LPP 1: 8x4, LPP 2: 8x2, LPP 4: 4x2 (32 lanes each), tile_w / RW of them per row.
// The batch depth D is the number of list entries staged in shared memory at a time: with
// D = 128, 256 or 512 the block stages them together and every warp walks the batch between
// two block barriers; with D = 32 each warp stages and walks its own 32-entry chunks of the
// list with no block barrier inside the item, so a warp with little to do in a stretch of
// the list runs ahead instead of waiting for the block's slowest warp (each warp then reads
// every record of the list, mostly from L1).
// A clip-volume batch (MULTI) also stages each kWeightMulti entry's further planes (CutExtra)
// in sx, next to its ray-tracing record.
template <int LPP, int D, bool COUNT, bool MULTI>
__device__ __forceinline__ void render_item(const RenderArgs &a, const ViewDev &vw, const uint32_t *pair_vals,
                                            StageT<stage_entries<D>()> &st, CutExtra *sx, int gtile, int tile,
                                            int part, Tally<COUNT> &ty)
{
    constexpr bool WARP = D == 32;
    constexpr int RW = LPP == 4 ? 4 : 8;     // warp rectangle width
    constexpr int RH = LPP == 1 ? 4 : 2;     // warp rectangle height
    constexpr int NB = WARP ? 1 : (D + kBlock - 1) / kBlock;  // entries a thread stages per batch
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane % LPP, pix = lane / LPP;
    const int W = vw.cam.W, H = vw.cam.H;
    const int TW = vw.tile_w, TH = vw.tile_h;
    const int wpr = TW / RW;                 // warp rectangles per row
    const int rows = (kBlock / LPP) / TW;    // rows of the item
    const int tx = tile % vw.tiles_x, ty0 = tile / vw.tiles_x;
    const int wx0 = (warp % wpr) * RW;
    const int wy0 = part * rows + (warp / wpr) * RH;
    const int px = tx * TW + wx0 + pix % RW, py = ty0 * TH + wy0 + pix / RW;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    // the warp's rectangle of pixel centres is [rx0, rx0 + RW - 1] x [ry0, ry0 + RH - 1]
    const float rx0 = (float)(tx * TW + wx0) + 0.5f;
    const float ry0 = (float)(ty0 * TH + wy0) + 0.5f;
    const int2 range = a.ranges[gtile];

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    bool done = !(px < W && py < H);
    uint32_t last = 0;
    // Walk the staged entries [jbase, jbase + cnt_here) (list positions pbase, pbase + 1, ...):
    // each lane tests one entry against the warp's rectangle, then the warp walks the kept
    // entries in list order.
    auto walk_chunk = [&](const int jbase, const int pbase, const int cnt_here) {
        bool keep = false, weighted = false;
        const int jt = jbase + lane;
        if (lane < cnt_here) {
            keep = entry_reaches(st, jt, rx0, rx0 + (float)(RW - 1), ry0, ry0 + (float)(RH - 1));
            weighted = st.s1[jt].w != kWeightNone;
            ty.add(ty.tested, true);
        }
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (LPP == 1) {
            const unsigned mw = __ballot_sync(0xffffffffu, keep && weighted);
            // Entries in list order; every lane runs the same straight-line step (the
            // only branch, on the entry's weight mode, is uniform across the warp), with
            // lanes that are done or outside the support contributing alpha = 0.
            auto step = [&](const int bit, const bool wt) {
                const int j = jbase + bit;
                const float4 s0 = st.s0[j];
                const float4 s1 = st.s1[j];
                const float dx = pxf - s0.x, dy = pyf - s0.y;
                const float q = splat_q(s0.z, s0.w, s1.x, dx, dy);
                ty.add(ty.walked, !done);
                const float a0 = splat_alpha0(q, s1.y);
                // alpha <= alpha0, so alpha >= 1/255 below also stands for alpha0 >= 1/255
                const bool inq = !done && q <= s1.z;
                ty.add(ty.evaluated, inq && a0 >= kAlphaMin);
                float alpha = a0;
                if (wt) {
                    const float mode = s1.w;
                    ty.add(ty.cut, inq && a0 >= kAlphaMin && (mode == kWeightSplit || (MULTI && mode == kWeightMulti)));
                    if (MULTI && mode == kWeightMulti) {
                        const float4 c3 = st.c3[j];
                        alpha = __fmul_rn(a0, rara_weight_multi(st.c0[j], st.c1[j], st.c2[j], c3, sx[j], dx, dy));
                    } else {
                        alpha = __fmul_rn(a0, decay_weight(mode, st.c0[j], st.c1[j], st.c2[j], st.c3[j], dx, dy));
                    }
                }
                alpha = fminf(kAlphaMax, alpha);
                const bool valid = inq && alpha >= kAlphaMin;
                const float aT = alpha * T;
                const float Tn = T - aT;  // T (1 - alpha)
                const bool stop = valid && Tn < kTMin;
                const bool blend = valid && !stop;
                const float wgt = blend ? aT : 0.0f;
                const float4 s2 = st.s2[j];
                C0 = fmaf(s2.x, wgt, C0);
                C1 = fmaf(s2.y, wgt, C1);
                C2 = fmaf(s2.z, wgt, C2);
                T = blend ? Tn : T;
                last = blend ? (uint32_t)(pbase + bit) : last;
                done = done || stop;
            };
            if (mw == 0u) {
                // no entry of the chunk needs the decay weight (most chunks): no per-entry
                // test, two entries per loop trip
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    step(bit, false);
                    if (!m) break;
                    const int bit2 = __ffs(m) - 1;
                    m &= m - 1;
                    step(bit2, false);
                }
            } else {
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    step(bit, ((mw >> bit) & 1u) != 0u);
                    if (!m) break;
                    const int bit2 = __ffs(m) - 1;
                    m &= m - 1;
                    step(bit2, ((mw >> bit2) & 1u) != 0u);
                }
            }
        } else {
            // LPP lanes per pixel: in each step the lanes of a pixel take the next LPP
            // kept entries (sub-lane s the (s+1)-th), evaluate their alphas, exchange
            // (1 - alpha) with shuffles, and every lane of the pixel applies the same
            // steps of the front-to-back recursion in list order, so all of them agree on
            // T, on which entries blend and on where the pixel stops. Each lane adds only
            // its own entry's colour to its partial sums, which are added up at the end.
            const int group = pix * LPP;          // first lane of this pixel's group
            while (m) {
                const unsigned m1 = m & (m - 1u), m2 = m1 & (m1 - 1u), m3 = m2 & (m2 - 1u);
                const unsigned mine = sub == 0 ? m : (sub == 1 ? m1 : (sub == 2 ? m2 : m3));
                m = LPP == 2 ? m2 : (m3 & (m3 - 1u));
                const bool has = mine != 0u && !done;
                const int bit = mine ? __ffs(mine) - 1 : 0;
                const int j = jbase + bit;
                const float4 s0 = st.s0[j];
                const float4 s1 = st.s1[j];
                const float dx = pxf - s0.x, dy = pyf - s0.y;
                const float q = splat_q(s0.z, s0.w, s1.x, dx, dy);
                ty.add(ty.walked, has);
                const float a0 = splat_alpha0(q, s1.y);
                const bool live = has && q <= s1.z && a0 >= kAlphaMin;
                ty.add(ty.evaluated, live);
                float alpha = a0;
                const bool wt = live && s1.w != kWeightNone;
                if (__any_sync(0xffffffffu, wt)) {
                    ty.add(ty.cut, live && (s1.w == kWeightSplit || (MULTI && s1.w == kWeightMulti)));
                    float w = decay_weight_any(wt ? s1.w : kWeightNone, st.c0[j], st.c1[j], st.c2[j],
                                               st.c3[j], dx, dy);
                    if (MULTI) {
                        const bool wm = wt && s1.w == kWeightMulti;
                        if (__any_sync(0xffffffffu, wm)) {
                            const float4 c3 = st.c3[j];
                            // (a lane without such an entry reads another entry's planes; unused)
                            const float w2 = rara_weight_multi(st.c0[j], st.c1[j], st.c2[j], c3, sx[j], dx, dy);
                            if (wm) w = w2;
                        }
                    }
                    alpha = __fmul_rn(a0, w);
                }
                alpha = fminf(kAlphaMax, alpha);
                const bool valid = live && alpha >= kAlphaMin;
                const float om = valid ? 1.0f - alpha : 1.0f;
                // the recursion over the group's entries, identical in its lanes: an entry
                // with alpha > 0 (1 - alpha < 1) that would take T below 1e-4 stops the pixel
                float t = T, tb = T;
                int first = LPP;
#pragma unroll
                for (int k = 0; k < LPP; ++k) {
                    const float ok = __shfl_sync(0xffffffffu, om, group + k);
                    if (sub == k) tb = t;
                    const float tn = t * ok;
                    if (first == LPP && ok < 1.0f && tn < kTMin) first = k;
                    if (first == LPP) t = tn;
                }
                const bool blend = valid && sub < first;
                const float wgt = blend ? alpha * tb : 0.0f;
                const float4 s2 = st.s2[j];
                C0 = fmaf(s2.x, wgt, C0);
                C1 = fmaf(s2.y, wgt, C1);
                C2 = fmaf(s2.z, wgt, C2);
                last = blend ? (uint32_t)(pbase + bit) : last;
                if (!done) T = t;
                done = done || first < LPP;
            }
        }
    };

    if (WARP) {
        const int wbase = warp * 32;          // this warp's staging entries
        for (int base = range.x; base < range.y; base += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const int k = base + lane;
            __syncwarp();                     // the previous chunk has been read
            if (k < range.y) {
                const uint32_t g = __ldg(&pair_vals[k]);
                const SplatRec rec = a.rec[g];
                stage_splat(st, wbase + lane, rec);
                if (rec.r2.y != kWeightNone) {
                    stage_cut(st, wbase + lane, a.cut[g]);
                    if (MULTI && rec.r2.y == kWeightMulti) sx[wbase + lane] = a.cut_x[g];
                }
            }
            __syncwarp();
            walk_chunk(wbase, base - range.x + 1, min(32, range.y - base));
        }
    } else {
        // slots of this thread's entries in the next batch, loaded one batch ahead
        uint32_t g_next[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            const int e = (int)threadIdx.x + r * kBlock;
            g_next[r] = e < D && range.x + e < range.y ? __ldg(&pair_vals[range.x + e]) : 0u;
        }
        for (int base = range.x; base < range.y; base += D) {
            if (__syncthreads_count(done) == kBlock) break;
#pragma unroll
            for (int r = 0; r < NB; ++r) {
                const int e = (int)threadIdx.x + r * kBlock;  // entry of the batch this thread stages
                const int k = base + e;
                const uint32_t g = g_next[r];
                if (e < D && k + D < range.y) g_next[r] = __ldg(&pair_vals[k + D]);
                if (e < D && k < range.y) {
                    const SplatRec rec = a.rec[g];
                    stage_splat(st, e, rec);
                    if (rec.r2.y != kWeightNone) {
                        stage_cut(st, e, a.cut[g]);
                        // a Gaussian split by several planes of a clip volume: its further planes
                        if (MULTI && rec.r2.y == kWeightMulti) sx[e] = a.cut_x[g];
                    }
                }
            }
            __syncthreads();
            const int cnt = min(D, range.y - base);
            const int pos0 = base - range.x + 1;  // list position (1-based) of batch entry 0
            for (int chunk = 0; chunk < cnt; chunk += 32) {
                if (__all_sync(0xffffffffu, done)) break;
                walk_chunk(chunk, pos0 + chunk, min(32, cnt - chunk));
            }
        }
    }

    if (LPP > 1) {  // partial colour sums and last blended position over the pixel's lanes
#pragma unroll
        for (int o = 1; o < LPP; o <<= 1) {
            C0 += __shfl_xor_sync(0xffffffffu, C0, o, LPP);
            C1 += __shfl_xor_sync(0xffffffffu, C1, o, LPP);
            C2 += __shfl_xor_sync(0xffffffffu, C2, o, LPP);
            last = max(last, __shfl_xor_sync(0xffffffffu, last, o, LPP));
        }
    }

    // the pixel again from its centre (fewer values live across the loop)
    const int W2 = vw.cam.W, H2 = vw.cam.H, px2 = (int)pxf, py2 = (int)pyf;
    if (px2 < W2 && py2 < H2 && sub == 0) {
        const size_t p = (size_t)py2 * W2 + px2;
        const size_t plane = (size_t)W2 * H2;
        vw.image[p] = fmaf(T, vw.bg[0], C0);
        vw.image[plane + p] = fmaf(T, vw.bg[1], C1);
        vw.image[2 * plane + p] = fmaf(T, vw.bg[2], C2);
        if (vw.final_T) vw.final_T[p] = T;
        if (vw.n_contrib) vw.n_contrib[p] = last;
    }
}

// Blocks per SM the register budget is sized for: the shared memory of a 512-entry batch
// (61 KB) allows 3 blocks per SM, the others 5.
template <int D>
__host__ __device__ constexpr int render_minb() { return D >= 512 ? 3 : 5; }

template <int D, bool MULTI>
constexpr size_t render_smem()
{
    return sizeof(StageT<stage_entries<D>()>) + (MULTI ? stage_entries<D>() * sizeof(CutExtra) : 0);
}

template <int D, bool COUNT, bool MULTI>
__global__ void __launch_bounds__(kBlock, render_minb<D>()) k_render(RenderArgs a)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    StageT<stage_entries<D>()> &st = *reinterpret_cast<StageT<stage_entries<D>()> *>(s_dyn);
    CutExtra *sx = MULTI ? reinterpret_cast<CutExtra *>(s_dyn + sizeof(StageT<stage_entries<D>()>)) : nullptr;
    __shared__ unsigned s_item;
    Tally<COUNT> ty;
    const unsigned num_items = *(volatile unsigned *)&a.counters->num_items;
    const uint32_t *pair_vals = a.counters->tile_in_b ? a.vals_b : a.vals_a;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned q = atomicAdd(&a.counters->tile_queue, 1u);
            s_item = q < num_items ? a.tile_order[q] : 0xffffffffu;
        }
        __syncthreads();
        const unsigned item = s_item;
        if (item == 0xffffffffu) break;
        const int gtile = (int)(item >> 4), lpp_log2 = (int)((item >> 2) & 3u), part = (int)(item & 3u);
        // view owning the global tile: the last view whose tile base is <= gtile
        int lo = 0, hi = a.num_views - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.views[mid].tile_base <= (uint32_t)gtile) lo = mid;
            else hi = mid - 1;
        }
        const ViewDev &vw = a.views[lo];
        const int tile = gtile - (int)vw.tile_base;
        if (lpp_log2 == 0) render_item<1, D, COUNT, MULTI>(a, vw, pair_vals, st, sx, gtile, tile, part, ty);
        else if (lpp_log2 == 1) render_item<2, D, COUNT, MULTI>(a, vw, pair_vals, st, sx, gtile, tile, part, ty);
        else render_item<4, D, COUNT, MULTI>(a, vw, pair_vals, st, sx, gtile, tile, part, ty);
        __syncthreads();  // everyone has read s_item and the staged batch
    }

    if (!COUNT) return;
    unsigned long long ev = ty.evaluated, wk = ty.walked, ce = ty.cut, ts = ty.tested;
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
        wk += __shfl_xor_sync(0xffffffffu, wk, o);
        ce += __shfl_xor_sync(0xffffffffu, ce, o);
        ts += __shfl_xor_sync(0xffffffffu, ts, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ev) atomicAdd(&a.counters->n_evaluated, ev);
        if (wk) atomicAdd(&a.counters->n_walked, wk);
        if (ce) atomicAdd(&a.counters->n_cut_evaluated, ce);
        if (ts) atomicAdd(&a.counters->n_tested, ts);
    }
}

template <int D, bool COUNT, bool MULTI>
int configure_render()
{
    return cudaFuncSetAttribute(k_render<D, COUNT, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)render_smem<D, MULTI>()) == cudaSuccess ? 0 : -1;
}

template <int D>
int launch_render_d(const RenderArgs &a, int grid, cudaStream_t s, bool count, bool multi)
{
    // the shared-memory opt-in is set once per device and instance (512 entries exceed the
    // 48 KB default); a failure is reported like a launch failure
    static bool configured[64][4] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int k = (count ? 1 : 0) + (multi ? 2 : 0);
    if (dev >= 0 && dev < 64 && !configured[dev][k]) {
        const int rc = count ? (multi ? configure_render<D, true, true>() : configure_render<D, true, false>())
                             : (multi ? configure_render<D, false, true>() : configure_render<D, false, false>());
        if (rc) return -1;
        configured[dev][k] = true;
    }
    if (multi) {  // batches with a convex clip volume
        const size_t smem = render_smem<D, true>();
        if (count) k_render<D, true, true><<<grid, kBlock, smem, s>>>(a);
        else k_render<D, false, true><<<grid, kBlock, smem, s>>>(a);
    } else {
        const size_t smem = render_smem<D, false>();
        if (count) k_render<D, true, false><<<grid, kBlock, smem, s>>>(a);
        else k_render<D, false, false><<<grid, kBlock, smem, s>>>(a);
    }
    return 0;
}

template <int D>
int render_bpsm_d()
{
    int b = 0;
    if (configure_render<D, true, false>() ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_render<D, true, false>, kBlock, render_smem<D, false>()) !=
            cudaSuccess ||
        b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

}  // namespace

bool tile_shape_ok(int tile_w, int tile_h)
{
    // 64, 256 or 512 pixels whose rows split evenly into the warp rectangles of every
    // lane count an item of that tile may use
    const int a = tile_w * tile_h;
    return (a == 64 && tile_w == 8 && tile_h == 8) ||
           (a == 256 && (tile_w == 16 || tile_w == 32 || tile_w == 8)) ||
           (a == 512 && (tile_w == 32 || tile_w == 16));
}

bool batch_depth_ok(int depth) { return depth == 32 || depth == 128 || depth == 256 || depth == 512; }

int render_blocks_per_sm(int depth)
{
    switch (depth) {
    case 32: return render_bpsm_d<32>();
    case 128: return render_bpsm_d<128>();
    case 512: return render_bpsm_d<512>();
    default: return render_bpsm_d<256>();
    }
}

int launch_render(const RenderArgs &a, int grid, cudaStream_t s, bool count, bool multi, int depth)
{
    if (grid <= 0) return 0;
    if (depth == 32) return launch_render_d<32>(a, grid, s, count, multi);
    if (depth == 128) return launch_render_d<128>(a, grid, s, count, multi);
    if (depth == 512) return launch_render_d<512>(a, grid, s, count, multi);
    return launch_render_d<256>(a, grid, s, count, multi);
}

}  // namespace rara
