// Per-pixel pieces of the render shared by the forward and the backward kernels, so the
// backward recomputes exactly what the forward computed.
#pragma once

#include "rara_internal.cuh"

namespace rara {

// q(dx, dy) = a dx^2 + 2 b dx dy + c dy^2 of a splat with conic (a, b, c), given b2 = 2 b.
__device__ __forceinline__ float splat_q(float a, float b2, float c, float dx, float dy)
{
    return fmaf(dx, fmaf(a, dx, b2 * dy), c * dy * dy);
}

constexpr float kHalfLog2e = 0.72134752044448170f;  // log2(e) / 2
constexpr float kLog2_255 = 7.99435343685885793f;   // -log2(kAlphaMin)

// 2^x (the special function unit's base-2 exponential).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// alpha0 = opacity exp(-q/2) (Eq. 10 without the normalisation) from log2(opacity).
__device__ __forceinline__ float splat_alpha0(float q, float lo)
{
    return ex2_approx(fmaf(q, -kHalfLog2e, lo));
}

// Per-pixel quantities of the ray through pixel offset (dx, dy) in the unit-sphere frame
// of a cutoff Gaussian (the local ray is -G + tau V, V = G + p, p = P (dx, dy)), from the
// staged form of its CutRec (stage_cut):
//   Gp = G.p, pp = p.p, VV = V.V = G.G + 2 Gp + pp, GV = G.V = G.G + Gp,
//   uu = |p x V|^2 = |dx A + dy B|^2 = A.A dx^2 + 2 A.B dx dy + B.B dy^2 (p x V = p x G, so
//        no difference of the large G and the small p enters), cc = uu / V.V, the squared
//        distance of the ray from the centre
struct RayTerms {
    float Gp, pp, VV, rVV, GV, cc, uu;
};

__device__ __forceinline__ RayTerms ray_terms(const float4 c0, const float4 c1, const float4 c2, const float4 c3,
                                              float dx, float dy)
{
    RayTerms t;
    t.Gp = fmaf(c0.y, dx, c0.z * dy);
    const float yy = dy * dy;
    t.pp = fmaf(dx, fmaf(c1.x, dx, c1.y * dy), c1.z * yy);
    t.uu = fmaf(dx, fmaf(c2.z, dx, c2.w * dy), c3.x * yy);
    t.VV = c0.x + fmaf(2.0f, t.Gp, t.pp);
    t.rVV = __fdividef(1.0f, t.VV);
    t.cc = __fmul_rn(t.uu, t.rVV);
    t.GV = c0.x + t.Gp;
    return t;
}

// The ray meets the unit sphere with both roots in front of the camera. The roots of
// |-G + tau V|^2 = 1 are real iff cc < 1 (|u|^2 < V.V), their sum is 2 G.V / V.V and their
// product (G.G - 1) / V.V, so both are positive iff G.V > 0 and G.G > 1. (Equivalently
// (G.V)^2 > (1 - cc) V.V: by Lagrange's identity (G.V)^2 = G.G V.V - |u|^2.) G.G > 1 is a
// property of the Gaussian, not of the ray: the preprocess gives the Gaussians with
// G.G <= 1 no weight (kWeightNone), so only the two per-ray conditions remain here.
__device__ __forceinline__ bool ray_hits_front(const RayTerms &t)
{
    return t.uu < t.VV && t.GV > 0.0f;
}

// Decay weight (Eq. 4-8, Eq. 11) of a Gaussian that the plane splits (kWeightSplit): the ray
// meets the unit sphere iff cc < 1, in front iff G.V > 0 and (G.V)^2 > (1 - cc) V.V; the
// plane s(u) = d_ep + m.u is linear along the chord, with values at its ends
//   s1,2 = s_mid -/+ h,  s_mid = d_ep + m.c,  h = sqrt(1 - cc) (m.V) / |V|,
// where c is the chord's midpoint, m.c = m.p - (p.V / V.V)(m.V). w = 1 if both ends are on
// the visible side, 0 if both are not, else the visible share max(s1, s2) / |s2 - s1|
// (together: clamp(1/2 + s_mid / (2 |h|), 0, 1)).
// Products that feed a sum are written with __fmul_rn so the forward (rara_weight) and the
// backward (rara_weight_terms, which also keeps the intermediate values for the weight's
// gradient) round identically.
struct SplitTerms {
    RayTerms t;
    float mp, mV, v;  // m.p, m.V and the unclamped share 1/2 + s_mid / (2 H)
    bool hit;
};

__device__ __forceinline__ float rara_weight_terms(const float4 c0, const float4 c1, const float4 c2, const float4 c3,
                                                   float dx, float dy, SplitTerms &s)
{
    // Every lane evaluates the whole expression and the cases are selected at the end, so a
    // warp whose pixels fall into different cases does not diverge; the values are the ones
    // the case-by-case form gives (the unselected ones may be NaN and are never used).
    s.t = ray_terms(c0, c1, c2, c3, dx, dy);
    s.hit = ray_hits_front(s.t);
    s.mp = fmaf(c2.x, dx, c2.y * dy);
    s.mV = c1.w + s.mp;
    // With H = |h| the chord's ends are s_mid -/+ H and the visible share is
    // (s_mid + H) / (2 H) = 1/2 + s_mid / (2 H), which reaches 1 (or 0) exactly when both ends
    // are on the visible (or the invisible) side: clamped to [0, 1] it is w in every case.
    // Multiplied through by V.V: s_mid / H = num / sqrt(den2) with
    //   num = (d_ep + m.p) V.V - (G.p + p.p) m.V,  den2 = (V.V - |u|^2) (m.V)^2.
    const float num = fmaf(c0.w + s.mp, s.t.VV, -__fmul_rn(s.t.Gp + s.t.pp, s.mV));
    const float den2 = __fmul_rn(s.t.VV - s.t.uu, __fmul_rn(s.mV, s.mV));
    s.v = fmaf(__fmul_rn(num, rsqrtf(den2)), 0.5f, 0.5f);
    return s.hit ? __saturatef(s.v) : 1.0f;  // a ray that misses, grazes or starts inside keeps rasterization
}

// The forward's form of rara_weight_terms: the same operations in the same order (so the same
// value), without keeping the terms (the render kernel schedules this form slightly faster).
__device__ __forceinline__ float rara_weight(const float4 c0, const float4 c1, const float4 c2, const float4 c3,
                                             float dx, float dy)
{
    const RayTerms t = ray_terms(c0, c1, c2, c3, dx, dy);
    const bool hit = ray_hits_front(t);
    const float mp = fmaf(c2.x, dx, c2.y * dy);
    const float mV = c1.w + mp;
    const float num = fmaf(c0.w + mp, t.VV, -__fmul_rn(t.Gp + t.pp, mV));
    const float den2 = __fmul_rn(t.VV - t.uu, __fmul_rn(mV, mV));
    const float w = __saturatef(fmaf(__fmul_rn(num, rsqrtf(den2)), 0.5f, 0.5f));
    return hit ? w : 1.0f;
}

// Decay weight of a Gaussian that several planes of a convex clip volume split
// (kWeightMulti): the share of the chord inside every half-space (Eq. 11 with the chord
// clipped by each plane, Eq. 8 per plane). Along the chord, with x in [-1, 1] from one end
// to the other, plane k is s_mid,k + x h_k, visible for x >= -g_k when h_k > 0 and for
// x <= g_k' = -(-g_k) when h_k < 0, with g_k = s_mid,k / |h_k| (rara_weight's ratio, here
// num_k / (sqrt(V.V - |u|^2) |m_k.V|)). The visible part is [lo, hi] = the intersection of
// those intervals with [-1, 1]; w = (hi - lo) / 2, clamped at 0. A plane with m_k.V = 0 is
// parallel to the ray: g_k = +-inf keeps everything or nothing by the sign of s, and the
// padding entries (1, 0, 0, 0) of a CutExtra keep everything. The planes are the CutRec's
// (c0.w, c1.w, c2.x, c2.y) and x[0..2].
__device__ __forceinline__ float rara_weight_multi(const float4 c0, const float4 c1, const float4 c2, const float4 c3,
                                                   const CutExtra &x, float dx, float dy)
{
    const RayTerms t = ray_terms(c0, c1, c2, c3, dx, dy);
    const bool hit = ray_hits_front(t);
    const float rs = rsqrtf(t.VV - t.uu);  // NaN when the ray misses; then w = 1 below
    const float GT = t.Gp + t.pp;
    float lo = -1.0f, hi = 1.0f;
    auto clip = [&](float dep, float mG, float mPx, float mPy) {
        const float mp = fmaf(mPx, dx, mPy * dy);
        const float mV = mG + mp;
        const float num = fmaf(dep + mp, t.VV, -__fmul_rn(GT, mV));
        const float g = __fmul_rn(num, rs) / fabsf(mV);
        if (mV >= 0.0f) lo = fmaxf(lo, -g);
        else hi = fminf(hi, g);
    };
    clip(c0.w, c1.w, c2.x, c2.y);
#pragma unroll
    for (int k = 0; k < 3; ++k) clip(x.p[k].x, x.p[k].y, x.p[k].z, x.p[k].w);
    const float w = __saturatef(0.5f * (hi - lo));
    return hit ? w : 1.0f;
}

// The weight of a Gaussian wholly on the invisible side of the plane (kWeightHidden): 0 when
// the ray hits the ellipsoid in front of the camera, else 1 (rara_weight's hit test).
__device__ __forceinline__ float rara_weight_hidden(const float4 c0, const float4 c1, const float4 c2,
                                                    const float4 c3, float dx, float dy)
{
    return ray_hits_front(ray_terms(c0, c1, c2, c3, dx, dy)) ? 0.0f : 1.0f;
}

// Decay weight of a slot with weight mode `mode` (kWeightSplit or kWeightHidden).
__device__ __forceinline__ float decay_weight(float mode, const float4 c0, const float4 c1, const float4 c2,
                                              const float4 c3, float dx, float dy)
{
    return mode == kWeightSplit ? rara_weight(c0, c1, c2, c3, dx, dy) : rara_weight_hidden(c0, c1, c2, c3, dx, dy);
}

// decay_weight for lanes that may hold entries of different modes (kWeightNone gives 1):
// both cases are evaluated and selected, with the same values as decay_weight.
__device__ __forceinline__ float decay_weight_any(float mode, const float4 c0, const float4 c1, const float4 c2,
                                                  const float4 c3, float dx, float dy)
{
    const float ws = rara_weight(c0, c1, c2, c3, dx, dy);
    const float wh = rara_weight_hidden(c0, c1, c2, c3, dx, dy);
    return mode == kWeightSplit ? ws : (mode == kWeightHidden ? wh : 1.0f);
}

// Minimum of q(dx, dy) = a dx^2 + 2 b dx dy + c dy^2 over the box [ax, bx] x [ay, by] of
// offsets from the projected centre. q is convex, so when the centre lies outside the box
// the minimum is on an edge, at the edge's 1D minimiser clamped to the edge
// (dx* = nba dy on a horizontal edge, dy* = nbc dx on a vertical one).
__device__ __forceinline__ float box_min_q(float ax, float bx, float ay, float by, float a, float b2, float c,
                                           float nba, float nbc)
{
    if (ax <= 0.0f && bx >= 0.0f && ay <= 0.0f && by >= 0.0f) return 0.0f;
    float best;
    {
        const float dx = fminf(bx, fmaxf(ax, nba * ay));
        best = splat_q(a, b2, c, dx, ay);
    }
    {
        const float dx = fminf(bx, fmaxf(ax, nba * by));
        best = fminf(best, splat_q(a, b2, c, dx, by));
    }
    {
        const float dy = fminf(by, fmaxf(ay, nbc * ax));
        best = fminf(best, splat_q(a, b2, c, ax, dy));
    }
    {
        const float dy = fminf(by, fmaxf(ay, nbc * bx));
        best = fminf(best, splat_q(a, b2, c, bx, dy));
    }
    return best;
}

// Margin of the rectangle test over the float32 rounding of the minimum.
constexpr float kCullMargin = 1.0001f;

// Shared-memory staging of one batch of list entries, as the per-pixel loops read them:
//   s0 = (mean2d.x, mean2d.y, conic.a, 2 conic.b)
//   s1 = (conic.c, log2(opacity), q_cut, decay-weight mode)
//   s2 = (rgb.r, rgb.g, rgb.b, opacity)
//   nb = (-b/a, -b/c), the rectangle test's line minimisers
//   c0..c3 = a cutoff entry's CutRec in the staged form of stage_cut
// q_cut = min(9, the q at which alpha0 = opacity exp(-q/2) falls to 1/255, plus a margin
// over its float32 rounding): a pixel with q > q_cut is outside the 3-sigma support or has
// alpha0 < 1/255, so it is skipped before the exponential; alpha0 itself is still compared
// with 1/255 afterwards, so q_cut only saves work and never decides.
// D entries per batch (the blend batch depth: 128, 256 or 512; 120 bytes per entry).
template <int D>
struct StageT {
    float4 s0[D], s1[D], s2[D];
    float2 nb[D];
    float4 c0[D], c1[D], c2[D], c3[D];
};
using Stage = StageT<kBlock>;

// Staged form of a CutRec: the quadratic forms p.p and |dx A + dy B|^2 in (dx, dy) take
// their coefficients directly,
//   c0 = (G.G, G.Px, G.Py, d_ep), c1 = (Px.Px, 2 Px.Py, Py.Py, m.G),
//   c2 = (m.Px, m.Py, A.A, 2 A.B), c3 = (B.B, 0, 0, 0).
template <int D>
__device__ __forceinline__ void stage_cut(StageT<D> &st, int i, const CutRec &c)
{
    const float ax = c.c2.z, ay = c.c2.w, az = c.c3.x, bx = c.c3.y, by = c.c3.z, bz = c.c3.w;
    st.c0[i] = c.c0;
    st.c1[i] = make_float4(c.c1.x, 2.0f * c.c1.y, c.c1.z, c.c1.w);
    st.c2[i] = make_float4(c.c2.x, c.c2.y, fmaf(ax, ax, fmaf(ay, ay, az * az)),
                           2.0f * fmaf(ax, bx, fmaf(ay, by, az * bz)));
    st.c3[i] = make_float4(fmaf(bx, bx, fmaf(by, by, bz * bz)), 0.0f, 0.0f, 0.0f);
}

// q_cut of a splat from log2(opacity) (see Stage).
__device__ __forceinline__ float splat_qcut(float lo)
{
    return fminf(kSupportQ, fmaf(lo + kLog2_255, 1.0f / kHalfLog2e, 1e-4f));
}

template <int D>
__device__ __forceinline__ void stage_splat(StageT<D> &st, int i, const SplatRec &rec)
{
    const float lo = __log2f(rec.r1.y);
    st.s0[i] = make_float4(rec.r0.x, rec.r0.y, rec.r0.z, 2.0f * rec.r0.w);
    st.s1[i] = make_float4(rec.r1.x, lo, splat_qcut(lo), rec.r2.y);
    st.s2[i] = make_float4(rec.r1.z, rec.r1.w, rec.r2.x, rec.r1.y);
    st.nb[i] = make_float2(rec.r2.z, rec.r2.w);
}

// A cutoff Gaussian wholly on the invisible side (kWeightHidden) has w = 0, hence alpha = 0,
// at every pixel whose ray hits its ellipsoid in front of the camera. With the camera outside
// the ellipsoid those pixels form a convex region of the image (the central projection of the
// ellipsoid's part in front of the camera), and so do the pixels whose rays pass within
// sqrt(0.999) of its centre (in the unit-sphere frame) with G.V above a margin. If the four
// corners of a box of pixel centres (offsets [ax, bx] x [ay, by] from the projected centre)
// lie in that smaller region, every pixel of the box does, and its float32 hit test
// (|u|^2 < V.V and G.V > 0, ray_hits_front; margins 1e-3 V.V and 1e-4 (G.G + |G.p|), far
// above the rounding) cannot fail: the entry is nothing to the box.
template <int D>
__device__ __forceinline__ bool hidden_covers_box(const StageT<D> &st, int j, float ax, float bx, float ay, float by)
{
    const float4 c0 = st.c0[j], c1 = st.c1[j], c2 = st.c2[j], c3 = st.c3[j];
    if (!(c0.x >= 1.001f)) return false;  // camera outside the ellipsoid, with a margin
    bool all = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const RayTerms t = ray_terms(c0, c1, c2, c3, k & 1 ? bx : ax, k & 2 ? by : ay);
        all = all && t.cc <= 0.999f && t.GV >= 1e-4f * (c0.x + fabsf(t.Gp));
    }
    return all;
}

// Exact rectangle test of staged entry j against the box [rx0, rx1] x [ry0, ry1] of pixel
// centres: whether some pixel of the box can have q <= q_cut and, for a Gaussian wholly on
// the invisible side, can miss its ellipsoid (elsewhere its alpha is 0).
template <int D>
__device__ __forceinline__ bool entry_reaches(const StageT<D> &st, int j, float rx0, float rx1, float ry0, float ry1)
{
    const float4 s0 = st.s0[j];
    const float4 s1 = st.s1[j];
    const float2 nb = st.nb[j];
    const float ax = rx0 - s0.x, bx = rx1 - s0.x, ay = ry0 - s0.y, by = ry1 - s0.y;
    const bool reach = box_min_q(ax, bx, ay, by, s0.z, s0.w, s1.x, nb.x, nb.y) <= s1.z * kCullMargin;
    return reach && !(s1.w == kWeightHidden && hidden_covers_box(st, j, ax, bx, ay, by));
}

}  // namespace rara
