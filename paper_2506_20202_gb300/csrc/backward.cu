// Backward of the clipped render: dL/dimage -> gradients of the Gaussians' parameters
// (means, log-scales, quaternions, opacity logits, SH coefficients) and of every view's
// clip plane (n, d). The paper renders only; this differentiates the forward exactly as
// the forward kernels compute it, in two launches:
//
// Render backward (per tile, the reverse of Eq. 2): every pixel starts from its final
// transmittance and the list position of its last blended entry (both written by the
// forward) and walks its tile's list back to front. Entry alphas are re-evaluated with the
// forward's own functions, so the set of blended entries is the forward's; the
// transmittance before an entry is recovered as T / (1 - alpha), and the colour composited
// behind it as a running sum, giving
//   dC/dalpha_j = T_j (c_j - B_j) - T_final bg / (1 - alpha_j)
//   B_{j-1}     = alpha_j c_j + (1 - alpha_j) B_j
// Through alpha = min(0.99, o exp(-q/2) w) the pixel's contribution flows to the entry's
// 2D mean, conic, opacity, colour and, for a cutoff Gaussian whose chord the plane splits,
// to its ray-tracing record (G, P, m, d_ep) via the weight's closed form
//   w = 1/2 + s_mid / (2 |h|)   (s_mid = d_ep + m.c, h = sqrt(1 - |c|^2) m.V / |V|).
// Where w is 0 or 1 (chord on one side of the plane, ray missing or behind) it is constant
// and passes no gradient; where 0.99 clamps alpha, alpha passes none either. Per entry, when
// more than kDirectAdds of the warp's pixels contribute, they are summed with a shuffle
// reduce-scatter (9 or 25 components) and one lane per component adds its total to the
// slot's gradient record; fewer contributing pixels add their own values with vector
// atomics. Warps skip entries whose q <= 9 support misses their 8x4 rectangle, as in the
// forward.
//
// Preprocess backward (per Gaussian, over the views of its scene that render it):
// the slot's gradient record is carried back through the projection (Eq. 9-10: conic ->
// Sigma2 -> J W R S -> camera-space mean), the SH colour, the sigmoid opacity and the
// ray-tracing record (G = M^-1 (mu - e), P, m = M^T n, d_ep = n.mu + d) to mu, sigma, R,
// the opacity logit, the SH coefficients and the plane; the rotation's gradient goes
// through the quaternion's normalisation once, after the views. Each Gaussian's gradients
// have one writer (no atomics); each view's plane gradient is a sum over Gaussians (block
// sums in shared memory, then one atomic per view, component and block).
#include "rara_internal.cuh"
#include "render_common.cuh"
#include "sh.cuh"

namespace rara {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Gradient of the decay weight where the plane splits the chord (0 < w < 1; ok is false where
// w is constant or the pixel does not contribute). It starts from the terms that
// rara_weight_terms computed for the weight itself (sp); with w = 1/2 + s_mid / (2 H),
// H = sqrt(h2) |m.V| / |V|, it goes back through
// s_mid = d_ep + m.p - f (m.V), f = (G.p + p.p) / V.V, h2 = 1 - |u|^2 / V.V,
// V.V = G.G + 2 G.p + p.p, m.V = m.G + m.p and the per-pixel polynomials G.p, p.p, m.p,
// u = dx A + dy B. c0..c2 is the record's staged form (stage_cut), r2, r3 its own c2, c3
// (which hold A and B). Outputs: dL/d(record products) in CutRec order (c0.x .. c3.w) in
// gc[16], and dL/d(dx, dy) added to gdx, gdy.
__device__ __forceinline__ void rara_weight_grad(const SplitTerms &sp, const float4 c0, const float4 c1,
                                                 const float4 c2, const float4 r2, const float4 r3, float dx, float dy,
                                                 float gw, bool ok, float gc[16], float &gdx, float &gdy)
{
    // Every lane evaluates the expressions; where ok is false (no contribution, or w constant)
    // the results, which may then be infinite or NaN, are replaced by zeros.
    const RayTerms &t = sp.t;
    const float mp = sp.mp, mV = sp.mV;
    const float cc = __fmul_rn(t.uu, t.rVV);
    const float h2 = 1.0f - cc;
    const float f = __fmul_rn(t.Gp + t.pp, t.rVV);
    const float smid = c0.w + fmaf(-f, mV, mp);
    // H > 0 and mV != 0 here (the share is finite and strictly inside (0, 1)), h2 > 0 (cc < 1)
    const float H = fabsf(__fmul_rn(__fmul_rn(__fmul_rn(h2, rsqrtf(h2)), mV), rsqrtf(t.VV)));
    const float g_smid = __fdividef(0.5f * gw, H);
    const float gHH = -g_smid * smid;   // dL/dH * H
    const float iVV = t.rVV;
    float g_VV = -0.5f * gHH * iVV;
    const float g_h2 = __fdividef(0.5f * gHH, h2);
    float g_mV = __fdividef(gHH, mV) - g_smid * f;
    const float g_f = -g_smid * mV;
    float g_mp = g_smid + g_mV;
    const float g_pV = g_f * iVV;
    g_VV -= g_f * f * iVV;
    const float g_cc = -g_h2;
    const float g_uu = g_cc * iVV;
    g_VV -= g_cc * cc * iVV;
    const float g_Gp = 2.0f * g_VV + g_pV;
    const float g_pp = g_VV + g_pV;
    gc[0] = g_VV;                       // G.G
    gc[1] = g_Gp * dx;                  // G.Px
    gc[2] = g_Gp * dy;                  // G.Py
    gc[3] = g_smid;                     // d_ep
    gc[4] = g_pp * dx * dx;             // Px.Px
    gc[5] = 2.0f * g_pp * dx * dy;      // Px.Py
    gc[6] = g_pp * dy * dy;             // Py.Py
    gc[7] = g_mV;                       // m.G
    gc[8] = g_mp * dx;                  // m.Px
    gc[9] = g_mp * dy;                  // m.Py
    // u = dx A + dy B from the stored A = (r2.z, r2.w, r3.x), B = (r3.y, r3.z, r3.w)
    const float u0 = fmaf(r2.z, dx, r3.y * dy), u1 = fmaf(r2.w, dx, r3.z * dy), u2 = fmaf(r3.x, dx, r3.w * dy);
    const float gu0 = 2.0f * g_uu * u0, gu1 = 2.0f * g_uu * u1, gu2 = 2.0f * g_uu * u2;
    gc[10] = gu0 * dx; gc[11] = gu1 * dx; gc[12] = gu2 * dx;   // A
    gc[13] = gu0 * dy; gc[14] = gu1 * dy; gc[15] = gu2 * dy;   // B
#pragma unroll
    for (int k = 0; k < 16; ++k) gc[k] = ok ? gc[k] : 0.0f;
    const float ddx = g_Gp * c0.y + g_pp * fmaf(2.0f * dx, c1.x, dy * c1.y) + g_mp * c2.x +
                      (gu0 * r2.z + gu1 * r2.w + gu2 * r3.x);
    const float ddy = g_Gp * c0.z + g_pp * fmaf(dx, c1.y, 2.0f * dy * c1.z) + g_mp * c2.y +
                      (gu0 * r3.y + gu1 * r3.z + gu2 * r3.w);
    gdx += ok ? ddx : 0.0f;
    gdy += ok ? ddy : 0.0f;
}

// Contributing pixels of an entry up to which each adds its own gradient values (2 or 7 vector
// atomics) rather than the warp summing them first: the reduce-scatter costs 16 or 32 shuffle
// steps per entry and pays only when most lanes contribute. On the 64-view differentiation
// workload the render backward took 40.2 ms with the sum for 2 or more pixels, 36.0 ms at 10,
// 34.9 at 16, 34.5 at 24 and 36.6 when every entry was added per pixel.
constexpr int kDirectAdds = 24;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sums N = 16 or 32 values per lane over the warp and scatters the totals (reduce-scatter:
// at each step a lane keeps half of its values and trades the other half with its partner,
// N/2 + N/4 + ... shuffles instead of 5 N). Afterwards v[0] holds the total of component
// `lane` (N = 32) or `lane >> 1` (N = 16, the pair of lanes 2c, 2c+1 both hold it).
template <int N>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[N])
{
    const int lane = threadIdx.x & 31;
    int o = 16;
#pragma unroll
    for (int h = N / 2; h >= 1; h >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = upper ? v[i] : v[i + h];
            const float keep = upper ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    if (N == 16) v[0] += __shfl_xor_sync(kFull, v[0], 1);
}

// One band of up to 256 pixels of a tile (rows [band * rows, (band + 1) * rows), rows =
// min(tile_h, 256 / tile_w)), one thread per pixel, warp rectangles of 8x4 pixels; the warps
// past a 64-pixel tile's rows have no pixels.
__device__ __forceinline__ void tile_bwd(const RenderBwdArgs &a, const ViewDev &vw, const BwdView &bv,
                                         const uint32_t *pair_vals, Stage &st, float4 (*s_ab)[kBlock],
                                         uint32_t *s_slot, int *s_max,
                                         int gtile, int tile, int band)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = vw.cam.W, H = vw.cam.H;
    const int TW = vw.tile_w, TH = vw.tile_h;
    const int rows = min(TH, kBlock / TW), wpr = TW / 8;
    const int tx = tile % vw.tiles_x, ty0 = tile / vw.tiles_x;
    const int wx0 = (warp % wpr) * 8, wy0 = (warp / wpr) * 4;   // within the band
    const int px = tx * TW + wx0 + (lane & 7);
    const int py = ty0 * TH + band * rows + wy0 + (lane >> 3);
    const bool inside = px < W && py < H && wy0 + (lane >> 3) < rows;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    // the warp's rectangle of pixel centres: [rx0, rx0 + 7] x [ry0, ry0 + 3]
    const float rx0 = (float)(tx * TW + wx0) + 0.5f;
    const float ry0 = (float)(ty0 * TH + band * rows + wy0) + 0.5f;
    const int2 range = a.ranges[gtile];

    float T = 1.0f, dC0 = 0.0f, dC1 = 0.0f, dC2 = 0.0f;
    uint32_t last = 0;
    if (inside) {
        const size_t p = (size_t)py * W + px, plane = (size_t)W * H;
        T = vw.final_T[p];
        last = vw.n_contrib[p];
        dC0 = bv.dimage[p];
        dC1 = bv.dimage[plane + p];
        dC2 = bv.dimage[2 * plane + p];
    }
    const float Tfin = T;
    const float bgdot = vw.bg[0] * dC0 + vw.bg[1] * dC1 + vw.bg[2] * dC2;
    float B0 = 0.0f, B1 = 0.0f, B2 = 0.0f;  // colour composited behind the current entry
    const uint32_t wlast = __reduce_max_sync(kFull, last);
    if (threadIdx.x == 0) *s_max = 0;
    __syncthreads();
    if (lane == 0 && wlast) atomicMax(s_max, (int)wlast);
    __syncthreads();
    const int end = range.x + *s_max;

    for (int bend = end; bend > range.x; bend -= kBlock) {
        const int bbeg = max(range.x, bend - kBlock);
        const int cnt = bend - bbeg;
        __syncthreads();  // the previous batch has been consumed
        if ((int)threadIdx.x < cnt) {
            const uint32_t g = __ldg(&pair_vals[bbeg + threadIdx.x]);
            const SplatRec rec = a.rec[g];
            stage_splat(st, threadIdx.x, rec);
            if (rec.r2.y != kWeightNone) {
                const CutRec c = a.cut[g];
                stage_cut(st, threadIdx.x, c);
                s_ab[0][threadIdx.x] = c.c2;  // A, B as stored, for the gradient
                s_ab[1][threadIdx.x] = c.c3;
            }
            s_slot[threadIdx.x] = g;
        }
        __syncthreads();
        for (int hi = cnt; hi > 0; hi -= 32) {
            const int lo = max(0, hi - 32);
            const int jt = lo + lane;
            bool keep = false;
            if (jt < hi && (uint32_t)(bbeg - range.x + jt) < wlast) keep = entry_reaches(st, jt, rx0, rx0 + 7.0f, ry0, ry0 + 3.0f);
            unsigned m = __ballot_sync(kFull, keep);
            while (m) {
                const int b = 31 - __clz(m);
                m &= ~(1u << b);
                const int j = lo + b;
                const uint32_t pos = (uint32_t)(bbeg - range.x + j);
                const float4 s0 = st.s0[j], s1 = st.s1[j], s2 = st.s2[j];
                const float ca = s0.z, cb = 0.5f * s0.w, cc = s1.x;  // conic (a, b, c)
                const float mode = s1.w;
                const bool cut = mode == kWeightSplit;  // the weight varies with the inputs
                // Every lane evaluates the entry (the branches below are uniform over the warp);
                // lanes that do not contribute select zero gradients and keep their state.
                const float dx = pxf - s0.x, dy = pyf - s0.y;
                const float q = splat_q(s0.z, s0.w, s1.x, dx, dy);
                const float a0 = splat_alpha0(q, s1.y);
                float w = 1.0f;
                SplitTerms sp;  // a split weight's terms, reused by its gradient
                if (cut) w = rara_weight_terms(st.c0[j], st.c1[j], st.c2[j], st.c3[j], dx, dy, sp);
                else if (mode != kWeightNone) w = rara_weight_hidden(st.c0[j], st.c1[j], st.c2[j], st.c3[j], dx, dy);
                const float au = __fmul_rn(a0, w);
                const float alpha = fminf(kAlphaMax, au);
                // (last = 0 outside the image)
                const bool contrib = pos < last && q <= s1.z && a0 >= kAlphaMin && alpha >= kAlphaMin;
                const unsigned who = __ballot_sync(kFull, contrib);
                if (!who) continue;
                const float oma = 1.0f - alpha;   // in [0.01, 1]
                const float roma = __fdividef(1.0f, oma);
                const float Tj = T * roma;
                const float wgt = contrib ? alpha * Tj : 0.0f;
                const float gr = dC0 * wgt, gg = dC1 * wgt, gb = dC2 * wgt;
                float ga = Tj * (dC0 * (s2.x - B0) + dC1 * (s2.y - B1) + dC2 * (s2.z - B2)) - Tfin * bgdot * roma;
                if (contrib) {
                    B0 = fmaf(alpha, s2.x, oma * B0);
                    B1 = fmaf(alpha, s2.y, oma * B1);
                    B2 = fmaf(alpha, s2.z, oma * B2);
                    T = Tj;
                }
                if (!contrib || au > kAlphaMax) ga = 0.0f;  // no contribution, or clamped at 0.99
                const float ga0 = ga * w;
                const float gop = contrib ? ga0 * __fdividef(a0, s2.w) : 0.0f;  // d alpha0 / d opacity = exp(-q/2)
                const float gq = -0.5f * ga0 * a0;
                const float gCa = gq * dx * dx;
                const float gCb = 2.0f * gq * dx * dy;
                const float gCc = gq * dy * dy;
                float gdx = 2.0f * gq * fmaf(ca, dx, cb * dy);
                float gdy = 2.0f * gq * fmaf(cb, dx, cc * dy);
                float gc[16];  // cutoff record products (split weights only)
#pragma unroll
                for (int k = 0; k < 16; ++k) gc[k] = 0.f;
                if (cut) {
                    // w is constant (0 or 1) unless the ray hits and the unclamped share lies
                    // strictly inside (0, 1)
                    const bool wok = contrib && sp.hit && sp.v > 0.0f && sp.v < 1.0f;
                    if (__any_sync(kFull, wok))
                        rara_weight_grad(sp, st.c0[j], st.c1[j], st.c2[j], s_ab[0][j], s_ab[1][j], dx, dy, ga * a0, wok,
                                         gc, gdx, gdy);
                }
                const float gmx = -gdx, gmy = -gdy;
                float *dst = a.grec[s_slot[j]].v;
                if (__popc(who) <= kDirectAdds) {  // few pixels: each adds its own values
                    if (contrib) {
                        float4 *d4 = reinterpret_cast<float4 *>(dst);
                        atomicAdd(&d4[0], make_float4(gmx, gmy, gCa, gCb));
                        atomicAdd(&d4[1], make_float4(gCc, gop, gr, gg));
                        if (cut) {
                            atomicAdd(&d4[2], make_float4(gb, gc[0], gc[1], gc[2]));
                            atomicAdd(&d4[3], make_float4(gc[3], gc[4], gc[5], gc[6]));
                            atomicAdd(&d4[4], make_float4(gc[7], gc[8], gc[9], gc[10]));
                            atomicAdd(&d4[5], make_float4(gc[11], gc[12], gc[13], gc[14]));
                            atomicAdd(&dst[24], gc[15]);
                        } else {
                            atomicAdd(&dst[8], gb);
                        }
                    }
                } else if (!cut) {  // components 0..8 of the record
                    float v[16] = {gmx, gmy, gCa, gCb, gCc, gop, gr, gg, gb, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    warp_reduce_scatter<16>(v);
                    if (!(lane & 1) && (lane >> 1) < 9) atomicAdd(&dst[lane >> 1], v[0]);
                } else {  // components 0..24 of the record
                    float v[32] = {gmx,    gmy,    gCa,    gCb,    gCc,    gop,    gr,     gg,
                                   gb,     gc[0],  gc[1],  gc[2],  gc[3],  gc[4],  gc[5],  gc[6],
                                   gc[7],  gc[8],  gc[9],  gc[10], gc[11], gc[12], gc[13], gc[14],
                                   gc[15], 0.f,    0.f,    0.f,    0.f,    0.f,    0.f,    0.f};
                    warp_reduce_scatter<32>(v);
                    if (lane < kGradCut + 16) atomicAdd(&dst[lane], v[0]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kBlock, 4) k_render_bwd(RenderBwdArgs a)
{
    __shared__ Stage st;
    __shared__ float4 s_ab[2][kBlock];  // stored c2, c3 (A, B) of the staged cutoff entries
    __shared__ uint32_t s_slot[kBlock];
    __shared__ unsigned s_item;
    __shared__ int s_max;
    const unsigned num_items = *(volatile unsigned *)&a.counters->num_items;
    const uint32_t *pair_vals = a.counters->tile_in_b ? a.vals_b : a.vals_a;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned q = atomicAdd(&a.counters->bwd_queue, 1u);
            s_item = q < num_items ? a.tile_order[q] : 0xffffffffu;
        }
        __syncthreads();
        const unsigned item = s_item;
        if (item == 0xffffffffu) break;
        const int gtile = (int)(item >> 4), part = (int)(item & 3u);
        int lo = 0, hi = a.num_views - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.views[mid].tile_base <= (uint32_t)gtile) lo = mid;
            else hi = mid - 1;
        }
        const ViewDev &vw = a.views[lo];
        // the forward's items of a tile are bands of its rows with 1, 2 or 4 lanes per pixel;
        // the backward walks bands of 256 pixels with one lane each: the first bands' items
        // take them, the others have nothing to do
        const int bands = max(1, vw.tile_w * vw.tile_h / kBlock);
        if (part < bands)
            tile_bwd(a, vw, a.bviews[lo], pair_vals, st, s_ab, s_slot, &s_max, gtile, gtile - (int)vw.tile_base,
                     part);
        __syncthreads();  // everyone has read s_item and the staged batch
    }
}

// Per-Gaussian backward over the scene's views. Dynamic shared memory: the block's SH
// coefficient gradients, [3 (degree+1)^2][kBlock].
constexpr int kViewChunkBwd = 32;  // views staged in shared memory at a time

__global__ void __launch_bounds__(kBlock, 2) k_preprocess_bwd(PreprocessBwdArgs a)
{
    // dynamic shared memory: SH coefficient gradients, then the SH coefficients themselves,
    // each [3 (max degree+1)^2][kBlock]
    extern __shared__ float s_gsh[];
    float *s_shc = s_gsh + a.sh_stride;
    __shared__ ViewDev s_views[kViewChunkBwd];
    const int unit = blockIdx.x;
    int si = 0;
    while (si + 1 < a.num_scenes && (int)a.scenes[si + 1].unit_begin <= unit) ++si;
    const SceneDev &sc = a.scenes[si];
    const BwdScene &bs = a.bscenes[si];
    const int n = sc.n;
    const int i = (unit - (int)sc.unit_begin) * kBlock + threadIdx.x;
    const bool valid = i < n;
    const int K = sh_count(sc.sh_degree);
    for (int k = 0; k < 3 * K; ++k) {
        s_gsh[k * kBlock + threadIdx.x] = 0.0f;
        s_shc[k * kBlock + threadIdx.x] = valid ? __ldg(&sc.sh[(size_t)k * n + i]) : 0.0f;
    }

    float mu[3] = {0.f, 0.f, 0.f}, sg[3] = {1.f, 1.f, 1.f}, logit = 0.f;
    float qv[4] = {1.f, 0.f, 0.f, 0.f}, qinv = 1.0f;
    float Rg[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    if (valid) {
        mu[0] = __ldg(&sc.means[i]); mu[1] = __ldg(&sc.means[n + i]); mu[2] = __ldg(&sc.means[2 * n + i]);
        sg[0] = expf(__ldg(&sc.log_scales[i]));
        sg[1] = expf(__ldg(&sc.log_scales[n + i]));
        sg[2] = expf(__ldg(&sc.log_scales[2 * n + i]));
        logit = __ldg(&sc.logits[i]);
        float qw = __ldg(&sc.quats[i]), qx = __ldg(&sc.quats[n + i]);
        float qy = __ldg(&sc.quats[2 * n + i]), qz = __ldg(&sc.quats[3 * n + i]);
        qinv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw *= qinv; qx *= qinv; qy *= qinv; qz *= qinv;
        qv[0] = qw; qv[1] = qx; qv[2] = qy; qv[3] = qz;
        Rg[0] = 1.f - 2.f * (qy * qy + qz * qz); Rg[1] = 2.f * (qx * qy - qw * qz); Rg[2] = 2.f * (qx * qz + qw * qy);
        Rg[3] = 2.f * (qx * qy + qw * qz); Rg[4] = 1.f - 2.f * (qx * qx + qz * qz); Rg[5] = 2.f * (qy * qz - qw * qx);
        Rg[6] = 2.f * (qx * qz - qw * qy); Rg[7] = 2.f * (qy * qz + qw * qx); Rg[8] = 1.f - 2.f * (qx * qx + qy * qy);
    }
    float gmu[3] = {0.f, 0.f, 0.f}, gsg[3] = {0.f, 0.f, 0.f}, gR[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float gopacity = 0.f;

    const int view_end = sc.view_begin + sc.view_count;
    // Per chunk of views, each thread first finds the views that render its Gaussian (one
    // tile-count load per view, issued together). The views are then taken in rounds: in each
    // round every lane takes its own next such view, so a lane does not sit through the views
    // that render only its neighbours' Gaussians. Each view's plane gradient is summed in shared
    // memory over the block and added once per chunk. The next round's gradient record is
    // prefetched into L2.
    __shared__ float s_gpl[kViewChunkBwd][4];
    for (int vbase = sc.view_begin; vbase < view_end; vbase += kViewChunkBwd) {
        const int nv = min(kViewChunkBwd, view_end - vbase);
        __syncthreads();  // the previous chunk's tables and plane sums are no longer read
        {
            constexpr int kWords = (int)(sizeof(ViewDev) / sizeof(uint32_t));
            const uint32_t *src = reinterpret_cast<const uint32_t *>(a.views + vbase);
            uint32_t *dst = reinterpret_cast<uint32_t *>(s_views);
            for (int t = threadIdx.x; t < nv * kWords; t += kBlock) dst[t] = __ldg(&src[t]);
            if (threadIdx.x < 4 * kViewChunkBwd) (&s_gpl[0][0])[threadIdx.x] = 0.0f;
        }
        __syncthreads();
        uint32_t vm = 0;  // the chunk's views that render this Gaussian
        if (valid) {
            for (int vv = 0; vv < nv; ++vv)
                if (__ldg(&a.tiles[s_views[vv].slot_base + (uint32_t)i]) != 0u) vm |= 1u << vv;
        }
        while (__any_sync(kFull, vm != 0u)) {
            const bool has = vm != 0u;
            const int vv = has ? __ffs(vm) - 1 : 0;
            vm &= vm - 1u;
            if (vm) {
                const char *nr = reinterpret_cast<const char *>(a.grec + (s_views[__ffs(vm) - 1].slot_base + (uint32_t)i));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nr));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nr + 96));
            }
            const ViewDev &vw = s_views[vv];
            const CamDev &cam = vw.cam;
            const PlaneDev &pl = vw.plane;
            float gpn[4] = {0.f, 0.f, 0.f, 0.f};
            bool has_plane = false;
            const uint32_t slot = vw.slot_base + (uint32_t)i;
            if (has) {
                const float *grc = a.grec[slot].v;
                const float4 g0 = reinterpret_cast<const float4 *>(grc)[0];
                const float4 g1 = reinterpret_cast<const float4 *>(grc)[1];
                const float gblue = grc[8];
                const bool cutoff = a.labels[slot] == RARA_CUTOFF;
                // ---- projection, as in the forward
                const float tx = fmaf(cam.R[0], mu[0], fmaf(cam.R[1], mu[1], fmaf(cam.R[2], mu[2], cam.t[0])));
                const float ty = fmaf(cam.R[3], mu[0], fmaf(cam.R[4], mu[1], fmaf(cam.R[5], mu[2], cam.t[1])));
                const float tz = fmaf(cam.R[6], mu[0], fmaf(cam.R[7], mu[1], fmaf(cam.R[8], mu[2], cam.t[2])));
                const float itz = 1.0f / tz;
                const float limx = 1.3f * (0.5f * cam.W / cam.fx), limy = 1.3f * (0.5f * cam.H / cam.fy);
                const float vx = tx * itz, vy = ty * itz;
                const float txz = fminf(limx, fmaxf(-limx, vx));
                const float tyz = fminf(limy, fmaxf(-limy, vy));
                const float J00 = cam.fx * itz, J02 = -cam.fx * txz * itz;
                const float J11 = cam.fy * itz, J12 = -cam.fy * tyz * itz;
                float T0[3], T1[3], u0[3], u1[3], A0[3], A1[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    T0[k] = fmaf(J00, cam.R[k], J02 * cam.R[6 + k]);
                    T1[k] = fmaf(J11, cam.R[3 + k], J12 * cam.R[6 + k]);
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    u0[k] = T0[0] * Rg[k] + T0[1] * Rg[3 + k] + T0[2] * Rg[6 + k];
                    u1[k] = T1[0] * Rg[k] + T1[1] * Rg[3 + k] + T1[2] * Rg[6 + k];
                    A0[k] = u0[k] * sg[k];
                    A1[k] = u1[k] * sg[k];
                }
                const float a0 = A0[0] * A0[0] + A0[1] * A0[1] + A0[2] * A0[2];
                const float b0 = A0[0] * A1[0] + A0[1] * A1[1] + A0[2] * A1[2];
                const float c0 = A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2];
                const float x0 = A0[1] * A1[2] - A0[2] * A1[1];
                const float x1 = A0[2] * A1[0] - A0[0] * A1[2];
                const float x2 = A0[0] * A1[1] - A0[1] * A1[0];
                const float ca = a0 + kDilation, cb = b0, cc = c0 + kDilation;
                const float det = (x0 * x0 + x1 * x1 + x2 * x2) + kDilation * (a0 + c0) + kDilation * kDilation;
                const float idet = 1.0f / det;
                // ---- conic (Ka, Kb, Kc) = (cc, -cb, ca) / det is the inverse of Sigma2:
                // dL/dSigma2 = -K G K with G = [[gKa, gKb / 2], [gKb / 2, gKc]]
                const float Ka = cc * idet, Kb = -cb * idet, Kc = ca * idet;
                const float gKa = g0.z, gKb = 0.5f * g0.w, gKc = g1.x;
                const float P00 = Ka * gKa + Kb * gKb, P01 = Ka * gKb + Kb * gKc;
                const float P10 = Kb * gKa + Kc * gKb, P11 = Kb * gKb + Kc * gKc;
                const float g_ca = -(P00 * Ka + P01 * Kb);
                const float g_cb = -2.0f * (P00 * Kb + P01 * Kc);
                const float g_cc = -(P10 * Kb + P11 * Kc);
                // ---- Sigma2 = A A^T + 0.3 I, A = (J W) R S
                float gT0[3] = {0.f, 0.f, 0.f}, gT1[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float gA0 = 2.0f * g_ca * A0[k] + g_cb * A1[k];
                    const float gA1 = 2.0f * g_cc * A1[k] + g_cb * A0[k];
                    gsg[k] += gA0 * u0[k] + gA1 * u1[k];
                    const float s0 = gA0 * sg[k], s1 = gA1 * sg[k];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        gR[3 * j + k] += s0 * T0[j] + s1 * T1[j];
                        gT0[j] += s0 * Rg[3 * j + k];
                        gT1[j] += s1 * Rg[3 * j + k];
                    }
                }
                const float gJ00 = gT0[0] * cam.R[0] + gT0[1] * cam.R[1] + gT0[2] * cam.R[2];
                const float gJ02 = gT0[0] * cam.R[6] + gT0[1] * cam.R[7] + gT0[2] * cam.R[8];
                const float gJ11 = gT1[0] * cam.R[3] + gT1[1] * cam.R[4] + gT1[2] * cam.R[5];
                const float gJ12 = gT1[0] * cam.R[6] + gT1[1] * cam.R[7] + gT1[2] * cam.R[8];
                // ---- J(t) with clamped x/z, y/z, and the 2D mean fx x/z + cx, fy y/z + cy
                const float gmx2 = g0.x, gmy2 = g0.y;
                float g_itz = cam.fx * (gJ00 - gJ02 * txz + gmx2 * tx) + cam.fy * (gJ11 - gJ12 * tyz + gmy2 * ty);
                float gt[3] = {gmx2 * cam.fx * itz, gmy2 * cam.fy * itz, 0.0f};
                if (vx > -limx && vx < limx) {
                    const float gv = -gJ02 * cam.fx * itz;
                    gt[0] += gv * itz;
                    g_itz += gv * tx;
                }
                if (vy > -limy && vy < limy) {
                    const float gv = -gJ12 * cam.fy * itz;
                    gt[1] += gv * itz;
                    g_itz += gv * ty;
                }
                gt[2] = -g_itz * itz * itz;
                // ---- opacity
                gopacity += g1.y;
                // ---- colour at normalize(mu - e)
                const float e[3] = {mu[0] - cam.eye[0], mu[1] - cam.eye[1], mu[2] - cam.eye[2]};
                const float il = rsqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
                const float dir[3] = {e[0] * il, e[1] * il, e[2] * il};
                {
                    float basis[16];
                    sh_basis(sc.sh_degree, dir[0], dir[1], dir[2], basis);
                    float grgb[3] = {g1.z, g1.w, gblue};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float acc = 0.0f;
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (k < K) acc = fmaf(s_shc[(k * 3 + c) * kBlock + threadIdx.x], basis[k], acc);
                        if (!(acc + 0.5f > 0.0f)) grgb[c] = 0.0f;  // clamped at 0
                    }
                    float s[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        s[k] = 0.0f;
                        if (k < K) {
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                s[k] = fmaf(grgb[c], s_shc[(k * 3 + c) * kBlock + threadIdx.x], s[k]);
                                s_gsh[(k * 3 + c) * kBlock + threadIdx.x] += grgb[c] * basis[k];
                            }
                        }
                    }
                    float gdir[3];
                    sh_basis_vjp(sc.sh_degree, dir[0], dir[1], dir[2], s, gdir);
                    const float dd = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
#pragma unroll
                    for (int j = 0; j < 3; ++j) gmu[j] += (gdir[j] - dd * dir[j]) * il;
                }
                // ---- ray-tracing record of a cutoff Gaussian
                if (cutoff) {
                    // gradients of the record products -> G, Px, Py, m (A = Px x G, B = Py x G)
                    const float *gq = grc + kGradCut;
                    const float kk = pl.k;
                    const float sx = tz / cam.fx, sy = tz / cam.fy;
                    float G[3], Px[3], Py[3], m[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float rk0 = Rg[k], rk1 = Rg[3 + k], rk2 = Rg[6 + k];
                        const float iks = 1.0f / (kk * sg[k]);
                        G[k] = iks * (rk0 * e[0] + rk1 * e[1] + rk2 * e[2]);
                        Px[k] = iks * sx * (rk0 * cam.R[0] + rk1 * cam.R[1] + rk2 * cam.R[2]);
                        Py[k] = iks * sy * (rk0 * cam.R[3] + rk1 * cam.R[4] + rk2 * cam.R[5]);
                        m[k] = kk * sg[k] * (rk0 * pl.n[0] + rk1 * pl.n[1] + rk2 * pl.n[2]);
                    }
                    const float gA[3] = {gq[10], gq[11], gq[12]}, gB[3] = {gq[13], gq[14], gq[15]};
                    float gG[3], gPx[3], gPy[3], gm[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                        // d(Px x G): G gets gA x Px, Px gets G x gA (likewise for B = Py x G)
                        gG[k] = 2.0f * gq[0] * G[k] + gq[1] * Px[k] + gq[2] * Py[k] + gq[7] * m[k] +
                                (gA[k1] * Px[k2] - gA[k2] * Px[k1]) + (gB[k1] * Py[k2] - gB[k2] * Py[k1]);
                        gPx[k] = gq[1] * G[k] + 2.0f * gq[4] * Px[k] + gq[5] * Py[k] + gq[8] * m[k] +
                                 (G[k1] * gA[k2] - G[k2] * gA[k1]);
                        gPy[k] = gq[2] * G[k] + gq[5] * Px[k] + 2.0f * gq[6] * Py[k] + gq[9] * m[k] +
                                 (G[k1] * gB[k2] - G[k2] * gB[k1]);
                        gm[k] = gq[7] * G[k] + gq[8] * Px[k] + gq[9] * Py[k];
                    }
                    const float gdep = gq[3];
                    float gtz_p = 0.0f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float iks = 1.0f / (kk * sg[k]);
                        gsg[k] += (-gG[k] * G[k] - gPx[k] * Px[k] - gPy[k] * Py[k] + gm[k] * m[k]) / sg[k];
                        gtz_p += gPx[k] * Px[k] + gPy[k] * Py[k];
                        const float aG = iks * gG[k], aPx = iks * sx * gPx[k], aPy = iks * sy * gPy[k];
                        const float am = kk * sg[k] * gm[k];
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            gR[3 * j + k] += aG * e[j] + aPx * cam.R[j] + aPy * cam.R[3 + j] + am * pl.n[j];
                            gmu[j] += aG * Rg[3 * j + k];
                            gpn[j] += am * Rg[3 * j + k];
                        }
                    }
                    gt[2] += gtz_p * itz;
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        gmu[j] += gdep * pl.n[j];
                        gpn[j] += gdep * mu[j];
                    }
                    gpn[3] = gdep;
                    has_plane = true;
                }
                // ---- camera-space mean t = W mu + t0
#pragma unroll
                for (int j = 0; j < 3; ++j) gmu[j] += cam.R[j] * gt[0] + cam.R[3 + j] * gt[1] + cam.R[6 + j] * gt[2];
                // leave the record zeroed for the next backward: the render backward adds to
                // v[0..8] of every listed slot and v[9..24] of split-weight (cutoff) slots only
                float4 *gw = reinterpret_cast<float4 *>(a.grec[slot].v);
                const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                gw[0] = z4; gw[1] = z4; gw[2] = z4;
                if (cutoff) { gw[3] = z4; gw[4] = z4; gw[5] = z4; gw[6] = z4; }
            }
            if (has_plane) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (gpn[j] != 0.0f) atomicAdd(&s_gpl[vv][j], gpn[j]);
            }
        }
        __syncthreads();
        if (threadIdx.x < 4 * nv) {
            const int vv = threadIdx.x >> 2, j = threadIdx.x & 3;
            float *pg = a.bviews[vbase + vv].plane_grad;
            const float g = s_gpl[vv][j];
            if (pg && g != 0.0f) atomicAdd(&pg[j], g);
        }
    }
    if (!valid) return;
    // rotation of the normalised quaternion (w, x, y, z), then the normalisation
    const float w = qv[0], x = qv[1], y = qv[2], z = qv[3];
    float gq[4];
    gq[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gq[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] -
                   2.f * x * gR[8]);
    gq[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] -
                   2.f * y * gR[8]);
    gq[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] + x * gR[6] +
                   y * gR[7]);
    const float qd = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
#pragma unroll
    for (int k = 0; k < 4; ++k) bs.quats[(size_t)k * n + i] = (gq[k] - qd * qv[k]) * qinv;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        bs.means[(size_t)k * n + i] = gmu[k];
        bs.log_scales[(size_t)k * n + i] = gsg[k] * sg[k];
    }
    const float op = 1.0f / (1.0f + expf(-logit));
    bs.logits[i] = gopacity * op * (1.0f - op);
    for (int k = 0; k < 3 * K; ++k) bs.sh[(size_t)k * n + i] = s_gsh[k * kBlock + threadIdx.x];
}

// The L2 objective of the differentiation step on the rendered images: d = image - target,
// loss += scale sum(d^2), dimage = 2 scale d. A block takes kLossChunk consecutive elements
// of one view (16 per thread: four float4 loads of each input, issued together, when the
// chunk is whole and the pointers are 16-byte aligned) and adds its partial sum to the view's
// loss once. The target is read with plain loads: it may be the gradient output itself.
__global__ void __launch_bounds__(kBlock) k_loss_l2(const LossView *views, int num_views)
{
    const uint32_t b = blockIdx.x;
    int lo = 0, hi = num_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].chunk_begin <= b) lo = mid;
        else hi = mid - 1;
    }
    const LossView lv = views[lo];
    const size_t e0 = (size_t)(b - lv.chunk_begin) * kLossChunk;
    const float s2 = 2.0f * lv.scale;
    float acc = 0.0f;
    const bool vec = e0 + kLossChunk <= lv.n &&
                     ((reinterpret_cast<uintptr_t>(lv.image) | reinterpret_cast<uintptr_t>(lv.target) |
                       reinterpret_cast<uintptr_t>(lv.dimage)) & 15u) == 0;
    if (vec) {
        const float4 *im = reinterpret_cast<const float4 *>(lv.image + e0);
        const float4 *tg = reinterpret_cast<const float4 *>(lv.target + e0);
        float4 *dm = reinterpret_cast<float4 *>(lv.dimage + e0);
        float4 x[4], t[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            x[r] = __ldg(&im[threadIdx.x + r * kBlock]);
            t[r] = tg[threadIdx.x + r * kBlock];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float4 d = make_float4(x[r].x - t[r].x, x[r].y - t[r].y, x[r].z - t[r].z, x[r].w - t[r].w);
            acc = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, acc))));
            dm[threadIdx.x + r * kBlock] = make_float4(s2 * d.x, s2 * d.y, s2 * d.z, s2 * d.w);
        }
    } else {
        for (int r = 0; r < kLossChunk / kBlock; ++r) {
            const size_t e = e0 + threadIdx.x + (size_t)r * kBlock;
            if (e < lv.n) {
                const float d = lv.image[e] - lv.target[e];
                acc = fmaf(d, d, acc);
                lv.dimage[e] = s2 * d;
            }
        }
    }
    __shared__ float s_part[kBlock / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < kBlock / 32 ? s_part[threadIdx.x] : 0.0f;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicAdd(lv.loss, (double)v * (double)lv.scale);
    }
}

}  // namespace

int render_bwd_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_render_bwd, kBlock, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

void launch_render_bwd(const RenderBwdArgs &a, int grid, cudaStream_t s)
{
    if (grid > 0) k_render_bwd<<<grid, kBlock, 0, s>>>(a);
}

int launch_preprocess_bwd(const PreprocessBwdArgs &a_in, int grid, int max_sh_degree, cudaStream_t s)
{
    PreprocessBwdArgs a = a_in;
    a.sh_stride = 3 * (max_sh_degree + 1) * (max_sh_degree + 1) * kBlock;
    const int smem = 2 * a.sh_stride * (int)sizeof(float);
    if (grid <= 0) return 0;
    if (cudaFuncSetAttribute(k_preprocess_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -1;
    k_preprocess_bwd<<<grid, kBlock, smem, s>>>(a);
    return 0;
}

void launch_loss_l2(const LossView *views, int num_views, uint32_t grid, cudaStream_t s)
{
    if (grid > 0 && num_views > 0) k_loss_l2<<<grid, kBlock, 0, s>>>(views, num_views);
}

}  // namespace rara
