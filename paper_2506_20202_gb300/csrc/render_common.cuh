// Per-pixel pieces of the render shared by the forward and the backward kernels, so the
// backward recomputes exactly what the forward computed.
#pragma once

#include "rara_internal.cuh"

namespace rara {

// q(dx, dy) = a dx^2 + 2 b dx dy + c dy^2 of a splat with conic (a, b, c).
__device__ __forceinline__ float splat_q(float a, float b, float c, float dx, float dy)
{
    return fmaf(dx, fmaf(a, dx, 2.0f * b * dy), c * dy * dy);
}

// Per-pixel quantities of the ray through pixel offset (dx, dy) in the unit-sphere frame
// of a cutoff Gaussian (the local ray is -G + tau V, V = G + p, p = P (dx, dy)), from the
// products stored in its CutRec:
//   Gp = G.p, pp = p.p, VV = V.V = G.G + 2 Gp + pp, GV = G.V = G.G + Gp,
//   cc = |p x V|^2 / V.V = |dx A + dy B|^2 / V.V, the squared distance of the ray from the
//        centre (a sum of squares: no cancellation between the large G and the small p)
struct RayTerms {
    float Gp, pp, VV, rVV, GV, cc, u0, u1, u2;
};

__device__ __forceinline__ RayTerms ray_terms(const float4 c0, const float4 c1, const float4 c2, const float4 c3,
                                              float dx, float dy)
{
    RayTerms t;
    t.Gp = fmaf(c0.y, dx, c0.z * dy);
    t.pp = fmaf(dx, fmaf(c1.x, dx, 2.0f * c1.y * dy), c1.z * dy * dy);
    t.u0 = fmaf(c2.z, dx, c3.y * dy);
    t.u1 = fmaf(c2.w, dx, c3.z * dy);
    t.u2 = fmaf(c3.x, dx, c3.w * dy);
    const float uu = fmaf(t.u0, t.u0, fmaf(t.u1, t.u1, t.u2 * t.u2));
    t.VV = c0.x + fmaf(2.0f, t.Gp, t.pp);
    t.rVV = __fdividef(1.0f, t.VV);
    t.cc = __fmul_rn(uu, t.rVV);
    t.GV = c0.x + t.Gp;
    return t;
}

// Decay weight (Eq. 4-8, Eq. 11) of a Gaussian that the plane splits (kWeightSplit): the ray
// meets the unit sphere iff cc < 1, in front iff G.V > 0 and (G.V)^2 > (1 - cc) V.V; the
// plane s(u) = d_ep + m.u is linear along the chord, with values at its ends
//   s1,2 = s_mid -/+ h,  s_mid = d_ep + m.c,  h = sqrt(1 - cc) (m.V) / |V|,
// where c is the chord's midpoint, m.c = m.p - (p.V / V.V)(m.V). w = 1 if both ends are on
// the visible side, 0 if both are not, else the visible share max(s1, s2) / |s2 - s1|.
// Products that feed a sum are written with __fmul_rn so the forward and the backward,
// which re-evaluates this function, round identically.
__device__ __forceinline__ float rara_weight(const float4 c0, const float4 c1, const float4 c2, const float4 c3,
                                             float dx, float dy)
{
    const RayTerms t = ray_terms(c0, c1, c2, c3, dx, dy);
    if (t.cc >= 1.0f) return 1.0f;                    // misses or grazes: keep rasterization
    const float h2 = 1.0f - t.cc;
    if (!(t.GV > 0.0f && t.GV * t.GV > h2 * t.VV)) return 1.0f;  // camera inside or behind
    const float mp = fmaf(c2.x, dx, c2.y * dy);
    const float mV = c1.w + mp;
    const float f = __fmul_rn(t.Gp + t.pp, t.rVV);
    const float smid = c0.w + fmaf(-f, mV, mp);
    const float half = __fmul_rn(__fmul_rn(__fmul_rn(h2, rsqrtf(h2)), mV), rsqrtf(t.VV));
    const float s1 = smid - half, s2 = smid + half;
    const bool v1 = s1 >= 0.0f, v2 = s2 >= 0.0f;
    if (v1 && v2) return 1.0f;
    if (!v1 && !v2) return 0.0f;
    return fminf(1.0f, __fdividef(fmaxf(s1, s2), fabsf(s2 - s1)));
}

// The weight of a Gaussian wholly on the invisible side of the plane (kWeightHidden): 0 when
// the ray hits the ellipsoid in front of the camera, else 1 (rara_weight's hit test).
__device__ __forceinline__ float rara_weight_hidden(const float4 c0, const float4 c1, const float4 c2,
                                                    const float4 c3, float dx, float dy)
{
    const RayTerms t = ray_terms(c0, c1, c2, c3, dx, dy);
    if (t.cc >= 1.0f) return 1.0f;
    const float h2 = 1.0f - t.cc;
    return (t.GV > 0.0f && t.GV * t.GV > h2 * t.VV) ? 0.0f : 1.0f;
}

// Decay weight of a slot with weight mode `mode` (kWeightSplit or kWeightHidden).
__device__ __forceinline__ float decay_weight(float mode, const float4 c0, const float4 c1, const float4 c2,
                                              const float4 c3, float dx, float dy)
{
    return mode == kWeightSplit ? rara_weight(c0, c1, c2, c3, dx, dy) : rara_weight_hidden(c0, c1, c2, c3, dx, dy);
}

// Minimum of q(dx, dy) = a dx^2 + 2 b dx dy + c dy^2 over the box [ax, bx] x [ay, by] of
// offsets from the projected centre. q is convex, so when the centre lies outside the box
// the minimum is on an edge, at the edge's 1D minimiser clamped to the edge
// (dx* = nba dy on a horizontal edge, dy* = nbc dx on a vertical one).
__device__ __forceinline__ float box_min_q(float ax, float bx, float ay, float by, float a, float b, float c,
                                           float nba, float nbc)
{
    if (ax <= 0.0f && bx >= 0.0f && ay <= 0.0f && by >= 0.0f) return 0.0f;
    float best;
    {
        const float dx = fminf(bx, fmaxf(ax, nba * ay));
        best = fmaf(dx, fmaf(a, dx, 2.0f * b * ay), c * ay * ay);
    }
    {
        const float dx = fminf(bx, fmaxf(ax, nba * by));
        best = fminf(best, fmaf(dx, fmaf(a, dx, 2.0f * b * by), c * by * by));
    }
    {
        const float dy = fminf(by, fmaxf(ay, nbc * ax));
        best = fminf(best, fmaf(ax, fmaf(a, ax, 2.0f * b * dy), c * dy * dy));
    }
    {
        const float dy = fminf(by, fmaxf(ay, nbc * bx));
        best = fminf(best, fmaf(bx, fmaf(a, bx, 2.0f * b * dy), c * dy * dy));
    }
    return best;
}

constexpr float kCullQ = kSupportQ * 1.0001f;  // margin over float32 rounding of the test

// Shared-memory staging of one batch of list entries.
struct Stage {
    float4 r0[kBlock], r1[kBlock], r2[kBlock];
    float4 c0[kBlock], c1[kBlock], c2[kBlock], c3[kBlock];
};

}  // namespace rara
