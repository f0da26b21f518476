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
    const float f = __fdividef(pV, VV);
    const float e0 = fmaf(-f, V0, p0), e1 = fmaf(-f, V1, p1), e2 = fmaf(-f, V2, p2);
    const float cc = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
    if (cc >= 1.0f) return 1.0f;                    // misses or grazes: keep rasterization
    const float h2 = 1.0f - cc;
    const float GV = fmaf(c0.x, V0, fmaf(c0.y, V1, c0.z * V2));
    if (!(GV > 0.0f && GV * GV > h2 * VV)) return 1.0f;  // camera inside or behind
    const float mc = fmaf(c1.w, e0, fmaf(c2.w, e1, c3.x * e2));
    const float mV = fmaf(c1.w, V0, fmaf(c2.w, V1, c3.x * V2));
    const float smid = c0.w + mc;
    // __fmul_rn keeps the compiler from fusing this product into s1 / s2, so the forward and
    // the backward (which re-evaluates this function) round identically.
    const float half = __fmul_rn(sqrtf(h2) * mV, rsqrtf(VV));
    const float s1 = smid - half, s2 = smid + half;
    const bool v1 = s1 >= 0.0f, v2 = s2 >= 0.0f;
    if (v1 && v2) return 1.0f;
    if (!v1 && !v2) return 0.0f;
    return fminf(1.0f, __fdividef(fmaxf(s1, s2), fabsf(s2 - s1)));
}

// The weight of a Gaussian wholly on the invisible side of the plane (kWeightHidden): 0 when
// the ray hits the ellipsoid in front of the camera, else 1. The hit test is rara_weight's.
__device__ __forceinline__ float rara_weight_hidden(const float4 c0, const float4 c1, const float4 c2, float dx,
                                                    float dy)
{
    const float p0 = fmaf(c1.x, dx, c2.x * dy);
    const float p1 = fmaf(c1.y, dx, c2.y * dy);
    const float p2 = fmaf(c1.z, dx, c2.z * dy);
    const float V0 = c0.x + p0, V1 = c0.y + p1, V2 = c0.z + p2;
    const float VV = fmaf(V0, V0, fmaf(V1, V1, V2 * V2));
    const float pV = fmaf(p0, V0, fmaf(p1, V1, p2 * V2));
    const float f = __fdividef(pV, VV);
    const float e0 = fmaf(-f, V0, p0), e1 = fmaf(-f, V1, p1), e2 = fmaf(-f, V2, p2);
    const float cc = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
    if (cc >= 1.0f) return 1.0f;
    const float h2 = 1.0f - cc;
    const float GV = fmaf(c0.x, V0, fmaf(c0.y, V1, c0.z * V2));
    return (GV > 0.0f && GV * GV > h2 * VV) ? 0.0f : 1.0f;
}

// Decay weight of a slot with weight mode `mode` (kWeightSplit or kWeightHidden).
__device__ __forceinline__ float decay_weight(float mode, const float4 c0, const float4 c1, const float4 c2,
                                              const float4 c3, float dx, float dy)
{
    return mode == kWeightSplit ? rara_weight(c0, c1, c2, c3, dx, dy) : rara_weight_hidden(c0, c1, c2, dx, dy);
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
