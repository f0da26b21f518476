// Steps (c)+(d): per-tile front-to-back compositing with the RaRa decay weight.
//
// One 256-thread block per 16x16 tile, one pixel per thread. The tile's depth-sorted
// list is walked in batches of 256: each thread gathers one splat record (and, for a
// cutoff Gaussian, its ray-tracing record) into shared memory, then every pixel walks the
// batch. A pixel stops at the first Gaussian that would take its transmittance below
// 1e-4; the block stops once all of its pixels have stopped.
//
// Decay weight (Eq. 4-8, Eq. 11, Algorithm 1 step 2), evaluated in the unit-sphere frame
// of the ellipsoid M = k R S without forming t1, t2 or t_p explicitly:
//   local ray   u(tau) = -G + tau V,  V = G + p,  p = P (dx, dy)   (tau = 1 at the centre
//               depth for the central ray; dx, dy = pixel offset from the projected centre)
//   chord       the closest point to the origin is c = p - (p.V / V.V) V (the component of
//               p orthogonal to V: no cancellation between the large G and the small p);
//               the ray meets the sphere iff |c| < 1, at tau_mid -/+ h with
//               tau_mid = G.V / V.V and h = sqrt(1 - |c|^2) / |V|
//   in front    t1 > 0  <=>  G.V > 0 and (G.V)^2 > (1 - |c|^2) V.V
//   plane       s(u) = d_ep + m . u with m = M^T n, linear along the ray:
//               s1,2 = d_ep + m.c -/+ sqrt(1 - |c|^2) (m.V) / |V|
//   weight      both >= 0: 1; both < 0: 0; otherwise the visible share of the chord,
//               max(s1, s2) / |s2 - s1|  (= (t2 - t_p)/(t2 - t1) or (t_p - t1)/(t2 - t1)).
#include "rara_internal.cuh"

namespace rara {

namespace {

__device__ __forceinline__ float rara_weight(const float4 c0, const float4 c1, const float4 c2, const float4 c3,
                                             float dx, float dy)
{
    // p = P (dx, dy), V = G + p
    const float p0 = fmaf(c1.x, dx, c2.x * dy);
    const float p1 = fmaf(c1.y, dx, c2.y * dy);
    const float p2 = fmaf(c1.z, dx, c2.z * dy);
    const float V0 = c0.x + p0, V1 = c0.y + p1, V2 = c0.z + p2;
    const float VV = fmaf(V0, V0, fmaf(V1, V1, V2 * V2));
    const float pV = fmaf(p0, V0, fmaf(p1, V1, p2 * V2));
    const float f = pV / VV;
    const float e0 = fmaf(-f, V0, p0), e1 = fmaf(-f, V1, p1), e2 = fmaf(-f, V2, p2);
    const float cc = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
    if (cc >= 1.0f) return 1.0f;                    // misses or grazes: keep rasterization
    const float h2 = 1.0f - cc;
    const float GV = fmaf(c0.x, V0, fmaf(c0.y, V1, c0.z * V2));
    if (!(GV > 0.0f && GV * GV > h2 * VV)) return 1.0f;  // camera inside or behind
    const float mc = fmaf(c1.w, e0, fmaf(c2.w, e1, c3.x * e2));
    const float mV = fmaf(c1.w, V0, fmaf(c2.w, V1, c3.x * V2));
    const float smid = c0.w + mc;
    const float half = sqrtf(h2) * mV * rsqrtf(VV);
    const float s1 = smid - half, s2 = smid + half;
    const bool v1 = s1 >= 0.0f, v2 = s2 >= 0.0f;
    if (v1 && v2) return 1.0f;
    if (!v1 && !v2) return 0.0f;
    return fminf(1.0f, fmaxf(s1, s2) / fabsf(s2 - s1));
}

__global__ void __launch_bounds__(kBlock) k_render(RenderArgs a)
{
    __shared__ float4 s_r0[kBlock], s_r1[kBlock], s_r2[kBlock];
    __shared__ float4 s_c0[kBlock], s_c1[kBlock], s_c2[kBlock], s_c3[kBlock];

    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * kTile + (threadIdx.x / kTile);
    const bool inside = px < a.W && py < a.H;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const int2 range = a.ranges[tile];

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    bool done = !inside;
    uint32_t last = 0;
    uint32_t evaluated = 0, walked = 0, cut_evaluated = 0;

    for (int base = range.x; base < range.y; base += kBlock) {
        if (__syncthreads_count(done) == kBlock) break;
        const int k = base + threadIdx.x;
        if (k < range.y) {
            const uint32_t g = __ldg(&a.pair_vals[k]);
            const SplatRec rec = a.rec[g];
            s_r0[threadIdx.x] = rec.r0;
            s_r1[threadIdx.x] = rec.r1;
            s_r2[threadIdx.x] = rec.r2;
            if (rec.r2.y != 0.0f) {
                const CutRec c = a.cut[g];
                s_c0[threadIdx.x] = c.c0;
                s_c1[threadIdx.x] = c.c1;
                s_c2[threadIdx.x] = c.c2;
                s_c3[threadIdx.x] = c.c3;
            }
        }
        __syncthreads();
        if (!done) {
            const int cnt = min(kBlock, range.y - base);
            int j = 0;
            for (; j < cnt; ++j) {
                const float4 r0 = s_r0[j];
                const float dx = pxf - r0.x, dy = pyf - r0.y;
                const float4 r1 = s_r1[j];
                const float q = fmaf(dx, fmaf(r0.z, dx, 2.0f * r0.w * dy), r1.x * dy * dy);
                if (q > kSupportQ) continue;
                ++evaluated;
                const float4 r2 = s_r2[j];
                float alpha = r1.y * __expf(-0.5f * q);
                if (r2.y != 0.0f) {
                    alpha *= rara_weight(s_c0[j], s_c1[j], s_c2[j], s_c3[j], dx, dy);
                    ++cut_evaluated;
                }
                alpha = fminf(kAlphaMax, alpha);
                if (alpha < kAlphaMin) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < kTMin) { done = true; break; }
                const float wgt = alpha * T;
                C0 = fmaf(r1.z, wgt, C0);
                C1 = fmaf(r1.w, wgt, C1);
                C2 = fmaf(r2.x, wgt, C2);
                T = Tn;
                last = (uint32_t)(base - range.x + j + 1);
            }
            walked += (uint32_t)min(j + 1, cnt);
        }
    }

    if (inside) {
        const size_t p = (size_t)py * a.W + px;
        const size_t plane = (size_t)a.W * a.H;
        a.image[p] = fmaf(T, a.bg[0], C0);
        a.image[plane + p] = fmaf(T, a.bg[1], C1);
        a.image[2 * plane + p] = fmaf(T, a.bg[2], C2);
        if (a.final_T) a.final_T[p] = T;
        if (a.n_contrib) a.n_contrib[p] = last;
    }
    unsigned long long ev = evaluated, wk = walked, ce = cut_evaluated;
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
        wk += __shfl_xor_sync(0xffffffffu, wk, o);
        ce += __shfl_xor_sync(0xffffffffu, ce, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ev) atomicAdd(&a.counters->n_evaluated, ev);
        if (wk) atomicAdd(&a.counters->n_walked, wk);
        if (ce) atomicAdd(&a.counters->n_cut_evaluated, ce);
    }
}

}  // namespace

void launch_render(const RenderArgs &a, int num_tiles, cudaStream_t s)
{
    if (num_tiles > 0) k_render<<<num_tiles, kBlock, 0, s>>>(a);
}

}  // namespace rara
