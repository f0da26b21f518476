// Step (a): per-Gaussian classification, projection and SH colour, for every view of a
// batch, and the compaction of the rendered (view, Gaussian) slots.
//
// Preprocess: one thread per Gaussian and loop over the views of its scene. Loads are
// planar (one coalesced 128-byte line per warp per attribute plane). Per slot the kernel
// writes the label and tiles-touched count, and for rendered slots the 48-byte splat record,
// the tile rectangle, the depth key and the 64-byte ray-tracing record (cutoff only).
// Compaction: rendered slots in slot order (view, then Gaussian index), placed by a chained
// scan across blocks so the order is deterministic.
#include "chained_scan.cuh"
#include "rara_internal.cuh"
#include "render_common.cuh"
#include "sh.cuh"

namespace rara {

namespace {

__device__ __forceinline__ float dot3(const float a[3], const float b[3])
{
    return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float out[3])
{
    out[0] = fmaf(a[1], b[2], -a[2] * b[1]);
    out[1] = fmaf(a[2], b[0], -a[0] * b[2]);
    out[2] = fmaf(a[0], b[1], -a[1] * b[0]);
}

// r0 x + r1 y + r2 z + t in doubled float32 precision, rounded once: the compensated dot
// product "Dot2" of Ogita, Rump and Oishi (Accurate sum and dot product, SIAM J. Sci.
// Comput. 26(6), 2005), with each product split exactly by an FMA (p + e = a b) and each
// sum by Knuth's TwoSum (s + e = a + b); the rounding errors are added up and folded in
// at the end. Every operation is explicitly rounded, so no contraction changes it.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float dot2_depth(float r0, float r1, float r2, float t, float x, float y, float z)
{
    const float p0 = __fmul_rn(r0, x), e0 = fmaf(r0, x, -p0);
    const float p1 = __fmul_rn(r1, y), e1 = fmaf(r1, y, -p1);
    const float p2 = __fmul_rn(r2, z), e2 = fmaf(r2, z, -p2);
    float s, f0, f1, f2;
    two_sum(p0, p1, s, f0);
    two_sum(s, p2, s, f1);
    two_sum(s, t, s, f2);
    const float err = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, f0)), __fadd_rn(f1, f2));
    return __fadd_rn(s, err);
}

// One-dimensional bulk copies (TMA) of the block's SH coefficient slices into shared memory,
// completed on an mbarrier. The planar layout makes the unit's slice of each coefficient
// plane one contiguous run of floats; a bulk copy needs both addresses 16-byte aligned and a
// size that is a multiple of 16 bytes, which holds when the scene size is a multiple of 4 and
// the array is 16-byte aligned (bulk_sh_ok).
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Waits for phase 0 of the mbarrier, at most kSpinLimit polls; false if it gave up.
__device__ __forceinline__ bool mbar_wait0(uint64_t *bar)
{
    for (int spin = 0; spin < kSpinLimit; ++spin) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar))
            : "memory");
        if (done) return true;
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ bool bulk_sh_ok(const float *sh, int n)
{
    return (n & 3) == 0 && ((uintptr_t)sh & 15u) == 0;
}

// Colour along the unit direction (x, y, z): sum_k sh_k Y_k + 0.5, clamped at 0. The
// thread's coefficients are staged in shared memory, s_sh[(k * 3 + c) * kBlock + thread].
__device__ __forceinline__ void sh_colour(const float *s_sh, int degree, float x, float y, float z, float rgb[3])
{
    float basis[16];
    sh_basis(degree, x, y, z, basis);
    const int kmax = sh_count(degree);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < kmax) acc = fmaf(s_sh[(k * 3 + c) * kBlock + threadIdx.x], basis[k], acc);
        rgb[c] = fmaxf(acc + 0.5f, 0.0f);
    }
}

constexpr int kViewChunk = 16;  // views staged in shared memory at a time

// The camera's part of a rendered slot: rectangle, splat-record terms, colour and depth key.
// ntiles = 0 when the projection culls the Gaussian (centre behind the near plane, singular 2D
// covariance, no tile of the image in its rectangle).
struct Proj {
    uint32_t ntiles;
    uint2 rect;
    float4 r0;            // (mean2d.x, mean2d.y, conic.a, conic.b)
    float r1x;            // conic.c
    float rgb0, rgb1, rgb2;
    float nbc, nba;       // b / c and b / a of the dilated covariance (the record's line minimisers)
    float depth;
};
constexpr int kProjWords = 14;

// Eq. 9-10 for one Gaussian and camera: Sigma2 = (J W M)(J W M)^T + 0.3 I with M = R S and J
// the affine approximation of the projection at the centre (x/z, y/z clamped); the tile
// rectangle of the q <= 9 ellipse; the SH colour at normalize(mu - e); the depth key.
__device__ __forceinline__ void project(Proj &pj, const ViewDev &vw, const CamDev &cam, float mx, float my, float mz,
                                        const float Rg[9], const float sg[3], const float *s_sh, int sh_degree,
                                        Counters *counters)
{
    pj.ntiles = 0;
    const float tx = fmaf(cam.R[0], mx, fmaf(cam.R[1], my, fmaf(cam.R[2], mz, cam.t[0])));
    const float ty = fmaf(cam.R[3], mx, fmaf(cam.R[4], my, fmaf(cam.R[5], mz, cam.t[1])));
    const float tz = fmaf(cam.R[6], mx, fmaf(cam.R[7], my, fmaf(cam.R[8], mz, cam.t[2])));
    if (!(tz > kNearZ)) return;
    const float itz = 1.0f / tz;
    const float limx = 1.3f * (0.5f * cam.W / cam.fx), limy = 1.3f * (0.5f * cam.H / cam.fy);
    const float txz = fminf(limx, fmaxf(-limx, tx * itz));
    const float tyz = fminf(limy, fmaxf(-limy, ty * itz));
    const float J00 = cam.fx * itz, J02 = -cam.fx * txz * itz;
    const float J11 = cam.fy * itz, J12 = -cam.fy * tyz * itz;
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T0[k] = fmaf(J00, cam.R[k], J02 * cam.R[6 + k]);
        T1[k] = fmaf(J11, cam.R[3 + k], J12 * cam.R[6 + k]);
    }
    float A0[3], A1[3];  // rows of J W R S
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        A0[k] = (T0[0] * Rg[k] + T0[1] * Rg[3 + k] + T0[2] * Rg[6 + k]) * sg[k];
        A1[k] = (T1[0] * Rg[k] + T1[1] * Rg[3 + k] + T1[2] * Rg[6 + k]) * sg[k];
    }
    const float a0 = A0[0] * A0[0] + A0[1] * A0[1] + A0[2] * A0[2];
    const float b0 = A0[0] * A1[0] + A0[1] * A1[1] + A0[2] * A1[2];
    const float c0 = A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2];
    // det((A A^T) + 0.3 I) = |A0 x A1|^2 + 0.3 (a0 + c0) + 0.09: every term is non-negative,
    // so elongated splats keep their precision.
    const float x0 = A0[1] * A1[2] - A0[2] * A1[1];
    const float x1 = A0[2] * A1[0] - A0[0] * A1[2];
    const float x2 = A0[0] * A1[1] - A0[1] * A1[0];
    const float ca = a0 + kDilation, cb = b0, cc = c0 + kDilation;
    const float det = (x0 * x0 + x1 * x1 + x2 * x2) + kDilation * (a0 + c0) + kDilation * kDilation;
    if (!(det > 0.0f)) return;
    const float idet = 1.0f / det;
    const float mx2 = fmaf(cam.fx, tx * itz, cam.cx);
    const float my2 = fmaf(cam.fy, ty * itz, cam.cy);
    // Tile rectangle: axis-aligned box of the q <= 9 ellipse; tile edges are powers of two, so
    // the products are the exact quotients
    const float hx = 3.0f * sqrtf(ca), hy = 3.0f * sqrtf(cc);
    const float itw = 1.0f / (float)vw.tile_w, ith = 1.0f / (float)vw.tile_h;
    const float fx0 = floorf((mx2 - hx) * itw), fx1 = floorf((mx2 + hx) * itw);
    const float fy0 = floorf((my2 - hy) * ith), fy1 = floorf((my2 + hy) * ith);
    const int rx0 = (int)fmaxf(0.0f, fminf((float)vw.tiles_x, fx0));
    const int rx1 = (int)fmaxf(-1.0f, fminf((float)(vw.tiles_x - 1), fx1));
    const int ry0 = (int)fmaxf(0.0f, fminf((float)vw.tiles_y, fy0));
    const int ry1 = (int)fmaxf(-1.0f, fminf((float)(vw.tiles_y - 1), fy1));
    if (!(rx0 <= rx1 && ry0 <= ry1)) return;
    pj.ntiles = (uint32_t)((rx1 - rx0 + 1) * (ry1 - ry0 + 1));
    pj.rect = make_uint2((uint32_t)rx0 | ((uint32_t)ry0 << 16), (uint32_t)rx1 | ((uint32_t)ry1 << 16));
    // colour at normalize(mu - e)
    const float ex = mx - cam.eye[0], ey = my - cam.eye[1], ez = mz - cam.eye[2];
    const float il = rsqrtf(ex * ex + ey * ey + ez * ez);
    float rgb[3];
    sh_colour(s_sh, sh_degree, ex * il, ey * il, ez * il, rgb);
    if (!isfinite(rgb[0] + rgb[1] + rgb[2])) atomicOr(&counters->status, kStatusBadInput);
    pj.r0 = make_float4(mx2, my2, cc * idet, -cb * idet);
    pj.r1x = ca * idet;
    pj.rgb0 = rgb[0];
    pj.rgb1 = rgb[1];
    pj.rgb2 = rgb[2];
    pj.nbc = cb / cc;
    pj.nba = cb / ca;
    // The sort key holds the depth rounded once from a dot product carried in doubled
    // float32 precision (dot2), i.e. the correctly rounded float32 of the exact depth except
    // within about 2^-48 of a rounding midpoint.
    pj.depth = dot2_depth(cam.R[6], cam.R[7], cam.R[8], cam.t[2], mx, my, mz);
}

// This thread's column of the projection cache (kProjWords words, stride kBlock).
__device__ __forceinline__ void store_proj(float (*c)[kBlock], const Proj &p)
{
    const int t = threadIdx.x;
    c[0][t] = __uint_as_float(p.ntiles);
    if (!p.ntiles) return;
    c[1][t] = __uint_as_float(p.rect.x); c[2][t] = __uint_as_float(p.rect.y);
    c[3][t] = p.r0.x; c[4][t] = p.r0.y; c[5][t] = p.r0.z; c[6][t] = p.r0.w;
    c[7][t] = p.r1x; c[8][t] = p.rgb0; c[9][t] = p.rgb1; c[10][t] = p.rgb2;
    c[11][t] = p.nbc; c[12][t] = p.nba; c[13][t] = p.depth;
}

__device__ __forceinline__ void load_proj(float (*c)[kBlock], Proj &p)
{
    const int t = threadIdx.x;
    p.ntiles = __float_as_uint(c[0][t]);
    if (!p.ntiles) return;
    p.rect = make_uint2(__float_as_uint(c[1][t]), __float_as_uint(c[2][t]));
    p.r0 = make_float4(c[3][t], c[4][t], c[5][t], c[6][t]);
    p.r1x = c[7][t]; p.rgb0 = c[8][t]; p.rgb1 = c[9][t]; p.rgb2 = c[10][t];
    p.nbc = c[11][t]; p.nba = c[12][t]; p.depth = c[13][t];
}

// One block = one unit of 256 Gaussians of one scene. The Gaussians' attributes are read
// once (the SH coefficients into shared memory, all loads of a thread issued together) and
// every view of the scene is processed from registers and shared memory; the views' tables
// are staged kViewChunk at a time. Per-view counts are summed per warp and per block in
// shared memory and added to the global counters once per chunk.
// One instance serves every batch, a single frame included: a view renders with the same
// instructions whatever batch it is in, so its images are the same bit for bit (two instances
// tuned for few and for many views were each free to contract the colour's multiply-adds
// differently). Its register budget is sized for 3 blocks per SM (with many views per Gaussian
// the per-view loop is arithmetic). The camera's part of each slot is kept in shared memory
// across consecutive views with the same camera (a single view has nothing to reuse).
constexpr bool CACHE = true;
__global__ void __launch_bounds__(kBlock, 3) k_preprocess(PreprocessArgs a)
{
    extern __shared__ __align__(16) float s_sh[];  // [3 (degree+1)^2][kBlock]
    __shared__ float s_pc[CACHE ? kProjWords : 1][kBlock];
    bool cam_ok = false;                            // s_pc holds this thread's slot for the view's camera
    uint32_t ukey = kNoKey;                         // one-camera batches: the depth key, once a view renders it
    uint32_t vmask = 0;                             // shared listing: the views that render it
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ ViewDev s_views[kViewChunk];
    __shared__ unsigned long long s_cnt[3][kViewChunk];
    const int lane = threadIdx.x & 31;
    const int unit = blockIdx.x;
    int si = 0;
    while (si + 1 < a.num_scenes && (int)a.scenes[si + 1].unit_begin <= unit) ++si;
    const SceneDev &sc = a.scenes[si];
    const int n = sc.n;
    const int i = (unit - (int)sc.unit_begin) * kBlock + threadIdx.x;
    const bool valid = i < n;

    float mx = 0.f, my = 0.f, mz = 0.f, s0 = 1.f, s1 = 1.f, s2 = 1.f, logit = 0.f;
    float Rg[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    bool bad = false;  // a non-finite parameter or a zero quaternion: not rendered, reported
    if (valid) {
        mx = __ldg(&sc.means[i]); my = __ldg(&sc.means[n + i]); mz = __ldg(&sc.means[2 * n + i]);
        const float l0 = __ldg(&sc.log_scales[i]), l1 = __ldg(&sc.log_scales[n + i]);
        const float l2 = __ldg(&sc.log_scales[2 * n + i]);
        s0 = expf(l0);
        s1 = expf(l1);
        s2 = expf(l2);
        logit = __ldg(&sc.logits[i]);
        // rotation of the normalised quaternion (w, x, y, z)
        float qw = __ldg(&sc.quats[i]), qx = __ldg(&sc.quats[n + i]);
        float qy = __ldg(&sc.quats[2 * n + i]), qz = __ldg(&sc.quats[3 * n + i]);
        const float qq = qw * qw + qx * qx + qy * qy + qz * qz;
        // a NaN or an infinity anywhere makes the sum non-finite (so does a sum that
        // overflows, which only inputs near the float range can cause: treated as bad too)
        bad = !isfinite(mx + my + mz + l0 + l1 + l2 + logit) || !isfinite(qq) || !(qq > 0.0f);
        if (bad) atomicOr(&a.counters->status, kStatusBadInput);
        const float qn = rsqrtf(qq);
        qw *= qn; qx *= qn; qy *= qn; qz *= qn;
        Rg[0] = 1.f - 2.f * (qy * qy + qz * qz); Rg[1] = 2.f * (qx * qy - qw * qz); Rg[2] = 2.f * (qx * qz + qw * qy);
        Rg[3] = 2.f * (qx * qy + qw * qz); Rg[4] = 1.f - 2.f * (qx * qx + qz * qz); Rg[5] = 2.f * (qy * qz - qw * qx);
        Rg[6] = 2.f * (qx * qz - qw * qy); Rg[7] = 2.f * (qy * qz + qw * qx); Rg[8] = 1.f - 2.f * (qx * qx + qy * qy);
    }
    {
        // the unit's SH coefficients: bulk copies of its slice of each plane when aligned
        const int q3 = 3 * sh_count(sc.sh_degree);
        const int first = (unit - (int)sc.unit_begin) * kBlock;
        const uint32_t bytes = (uint32_t)(min(kBlock, n - first) * (int)sizeof(float));
        bool staged = false;
        if (bulk_sh_ok(sc.sh, n)) {
            if (threadIdx.x == 0) mbar_init(&s_bar, 1);
            __syncthreads();
            if (threadIdx.x == 0) {
                mbar_expect_tx(&s_bar, bytes * (uint32_t)q3);
                for (int q = 0; q < q3; ++q)
                    bulk_copy_g2s(&s_sh[q * kBlock], sc.sh + (size_t)q * n + first, bytes, &s_bar);
            }
            staged = mbar_wait0(&s_bar);
            if (!staged) {  // report, let the copies land (bounded), then load directly
                atomicOr(&a.counters->status, kStatusLookbackTimeout);
                mbar_wait0(&s_bar);
            }
        }
        if (!staged)
            for (int q = 0; q < q3; ++q)
                s_sh[q * kBlock + threadIdx.x] = valid ? __ldg(&sc.sh[(size_t)q * n + i]) : 0.0f;
    }
    const float sg[3] = {s0, s1, s2};
    const float r = 3.0f * fmaxf(s0, fmaxf(s1, s2));
    const float op = 1.0f / (1.0f + expf(-logit));
    const int view_end = sc.view_begin + sc.view_count;

    for (int vbase = sc.view_begin; vbase < view_end; vbase += kViewChunk) {
        const int nv = min(kViewChunk, view_end - vbase);
        __syncthreads();  // the previous chunk's tables and counts are no longer read
        {
            constexpr int kWords = (int)(sizeof(ViewDev) / sizeof(uint32_t));
            const uint32_t *src = reinterpret_cast<const uint32_t *>(a.views + vbase);
            uint32_t *dst = reinterpret_cast<uint32_t *>(s_views);
            for (int t = threadIdx.x; t < nv * kWords; t += kBlock) dst[t] = __ldg(&src[t]);
            if (threadIdx.x < 3 * kViewChunk) (&s_cnt[0][0])[threadIdx.x] = 0ull;
        }
        __syncthreads();
        uint32_t cmask = 0;  // the chunk's views that label this Gaussian cutoff
        for (int vv = 0; vv < nv; ++vv) {
            const ViewDev &vw = s_views[vv];
            const PlaneDev &pl = vw.plane;
            const CamDev &cam = vw.cam;
            bool rendered = false, cutoff = false;
            uint32_t ntiles = 0;
            if (CACHE && !vw.same_cam) cam_ok = false;
            if (valid) {
                const uint32_t slot = vw.slot_base + (uint32_t)i;
                // Section 3.2 / Algorithm 1 step 1: d_ep = n.mu + d, r = 3 max(sigma)
                const float dep = fmaf(pl.n[0], mx, fmaf(pl.n[1], my, fmaf(pl.n[2], mz, pl.d)));
                int label;
                if (pl.mode == RARA_MODE_NONE) label = RARA_VISIBLE;
                else if (pl.mode == RARA_MODE_HARD) label = dep < 0.0f ? RARA_INVISIBLE : RARA_VISIBLE;
                else {
                    label = dep < -r ? RARA_INVISIBLE : (dep > r ? RARA_VISIBLE : RARA_CUTOFF);
                    if (pl.mode == RARA_MODE_RARA_ALL && label != RARA_INVISIBLE) label = RARA_CUTOFF;
                }
                if (bad) label = RARA_INVISIBLE;
                // A convex clip volume: the rule of each further plane joins the first's.
                // Invisible if behind any plane (the centre for hard clipping, the radius-r
                // sphere otherwise), visible only if in front of all of them.
                for (int e = 0; e < pl.n_extra && pl.mode != RARA_MODE_NONE; ++e) {
                    const float de = fmaf(pl.ex[e][0], mx, fmaf(pl.ex[e][1], my, fmaf(pl.ex[e][2], mz, pl.ex[e][3])));
                    if (pl.mode == RARA_MODE_HARD) {
                        if (de < 0.0f) label = RARA_INVISIBLE;
                    } else if (de < -r) {
                        label = RARA_INVISIBLE;
                    } else if (de <= r && label == RARA_VISIBLE) {
                        label = RARA_CUTOFF;
                    }
                }
                a.labels[slot] = (uint8_t)label;

                if (label != RARA_INVISIBLE) {
                    // The camera's part of the slot (projection, rectangle, colour, depth key)
                    // does not depend on the plane: with CACHE it is computed once per run of
                    // views with the same camera (a plane sweep from one viewpoint) and kept in
                    // this thread's column of the shared cache; the values are the same either way.
                    Proj pj;
                    if (!CACHE || !cam_ok) {
                        project(pj, vw, cam, mx, my, mz, Rg, sg, s_sh, sc.sh_degree, a.counters);
                        if (CACHE) {
                            store_proj(s_pc, pj);
                            cam_ok = true;
                        }
                    } else {
                        load_proj(s_pc, pj);
                    }
                    if (pj.ntiles) {
                        ntiles = pj.ntiles;
                        rendered = true;
                        cutoff = label == RARA_CUTOFF;
                        // A shared listing (one-camera batch) reads the emission record of the
                        // first view that renders the Gaussian only (its lowest view-mask bit),
                        // and so does the export of any view: the later views write none.
                        if (!a.vmask || vmask == 0u) {
                            EmitRec er;
                            er.rect = pj.rect;
                            er.mx = pj.r0.x; er.my = pj.r0.y; er.ca = pj.r0.z; er.cb = pj.r0.w; er.cc = pj.r1x;
                            er.qcut = splat_qcut(__log2f(op));
                            a.erec[slot] = er;
                        }
                        SplatRec rec;
                        rec.r0 = pj.r0;
                        rec.r1 = make_float4(pj.r1x, op, pj.rgb0, pj.rgb1);
                        float wmode = 0.0f;
                        a.depth[slot] = pj.depth;
                        ukey = __float_as_uint(pj.depth);
                    if (cutoff) cmask |= 1u << vv;  // its ray-tracing record comes after the views

                        rec.r2 = make_float4(pj.rgb2, wmode, pj.nbc, pj.nba);
                        a.rec[slot] = rec;
                    }
                }
                a.tiles[slot] = ntiles;
                const int vbit = vbase - sc.view_begin + vv;
                if (rendered && vbit < kListViews) vmask |= 1u << vbit;
            }
            // per-view counts: warp sums, then one shared-memory add per warp
            const unsigned nr = __reduce_add_sync(0xffffffffu, rendered ? 1u : 0u);
            const unsigned nc = __reduce_add_sync(0xffffffffu, cutoff ? 1u : 0u);
            unsigned long long np = ntiles;
            for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
            if (lane == 0) {
                if (nr) atomicAdd(&s_cnt[0][vv], (unsigned long long)nr);
                if (np) atomicAdd(&s_cnt[1][vv], np);
                if (nc) atomicAdd(&s_cnt[2][vv], (unsigned long long)nc);
            }
        }
        // Ray-tracing records of the cutoff slots, in rounds: every lane takes its own next
        // cutoff view of the chunk, so the record's arithmetic runs for the lanes that need it
        // instead of for every lane of a warp in which one lane is cutoff. The splat record
        // written above gets the weight mode.
        while (__any_sync(0xffffffffu, cmask != 0u)) {
            const bool has = cmask != 0u;
            const int vv = has ? __ffs(cmask) - 1 : 0;
            cmask &= cmask - 1u;
            if (has) {
                const ViewDev &vw = s_views[vv];
                const PlaneDev &pl = vw.plane;
                const CamDev &cam = vw.cam;
                const uint32_t slot = vw.slot_base + (uint32_t)i;
                const float dep = fmaf(pl.n[0], mx, fmaf(pl.n[1], my, fmaf(pl.n[2], mz, pl.d)));
                float wmode = kWeightNone;
                {
                        // the camera-space centre and the eye offset again (not cached)
                        const float tz = fmaf(cam.R[6], mx, fmaf(cam.R[7], my, fmaf(cam.R[8], mz, cam.t[2])));
                        const float ex = mx - cam.eye[0], ey = my - cam.eye[1], ez = mz - cam.eye[2];
                        // Ray-tracing record in the unit-sphere frame of M = k R S
                        // (Eq. 4): M^-1 = diag(1/(k sigma)) R^T. For the pixel ray with
                        // offset (dx, dy) from the projected centre, the local ray is
                        // o + tau V with o = -G, V = G + P (dx, dy): G = M^-1 (mu - e) and
                        // P = z M^-1 W^T[:, 0:2] diag(1/fx, 1/fy). m = M^T n carries the
                        // plane into the same frame: s(x) = d_ep + m . u for x = mu + M u.
                        const float kk = pl.k;
                        const float iks[3] = {1.0f / (kk * s0), 1.0f / (kk * s1), 1.0f / (kk * s2)};
                        float G[3], Px[3], Py[3], m[3];
                        const float sx = tz / cam.fx, sy = tz / cam.fy;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float rk0 = Rg[k], rk1 = Rg[3 + k], rk2 = Rg[6 + k];  // column k of R
                            G[k] = iks[k] * (rk0 * ex + rk1 * ey + rk2 * ez);
                            Px[k] = iks[k] * sx * (rk0 * cam.R[0] + rk1 * cam.R[1] + rk2 * cam.R[2]);
                            Py[k] = iks[k] * sy * (rk0 * cam.R[3] + rk1 * cam.R[4] + rk2 * cam.R[5]);
                            m[k] = kk * sg[k] * (rk0 * pl.n[0] + rk1 * pl.n[1] + rk2 * pl.n[2]);
                        }
                        // The plane meets the ellipsoid only if |d_ep| <= |m| (s varies by
                        // at most |m| over the unit ball). Beyond that (with a margin over
                        // rounding) every chord lies on one side: w = 1 for every ray when
                        // it is the visible side, and w = 0 for rays that hit the ellipsoid
                        // in front (1 for the others) when it is the invisible side.
                        const float mlen = sqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
                        const float bound = mlen * (1.0f + 1e-4f);
                        wmode = dep > bound ? kWeightNone : (dep < -bound ? kWeightHidden : kWeightSplit);
                        // Convex clip volume: a plane wholly in front of the ellipsoid
                        // constrains no chord and drops out; one wholly behind it hides
                        // it (w = 0 where a ray hits it in front); the splitting planes
                        // clip the chord. The first splitting plane takes the CutRec's
                        // plane terms, the others the slot's CutExtra.
                        float xs[3][4] = {};
                        int nsplit = wmode == kWeightSplit ? 1 : 0;
                        float sdep = dep;
                        for (int e = 0; e < pl.n_extra; ++e) {
                            float me[3];
#pragma unroll
                            for (int k = 0; k < 3; ++k)
                                me[k] = kk * sg[k] * (Rg[k] * pl.ex[e][0] + Rg[3 + k] * pl.ex[e][1] +
                                                      Rg[6 + k] * pl.ex[e][2]);
                            const float de = fmaf(pl.ex[e][0], mx,
                                                  fmaf(pl.ex[e][1], my, fmaf(pl.ex[e][2], mz, pl.ex[e][3])));
                            const float be = sqrtf(me[0] * me[0] + me[1] * me[1] + me[2] * me[2]) * (1.0f + 1e-4f);
                            if (de < -be) {
                                wmode = kWeightHidden;
                            } else if (de <= be) {
                                if (nsplit == 0) {
                                    sdep = de;
#pragma unroll
                                    for (int k = 0; k < 3; ++k) m[k] = me[k];
                                } else {
                                    xs[nsplit - 1][0] = de;
#pragma unroll
                                    for (int k = 0; k < 3; ++k) xs[nsplit - 1][1 + k] = me[k];
                                }
                                ++nsplit;
                            }
                        }
                        if (pl.n_extra > 0 && wmode != kWeightHidden)
                            wmode = nsplit == 0 ? kWeightNone : (nsplit == 1 ? kWeightSplit : kWeightMulti);
                        // With the camera inside (or on) the ellipsoid, G.G <= 1, the
                        // roots of every ray have product (G.G - 1) / V.V <= 0: no ray
                        // meets it twice in front, so w = 1 for every ray.
                        const float GG = dot3(G, G);
                        if (!(GG > 1.0f)) wmode = kWeightNone;
                        if (wmode != kWeightNone) {
                            // The render needs, per pixel, p = P (dx, dy) only through the
                            // dot products G.p, p.p, m.p and the cross product p x G: store
                            // the pairwise products of G, Px, Py, m and A = Px x G, B = Py x G.
                            CutRec c;
                            c.c0 = make_float4(GG, dot3(G, Px), dot3(G, Py), sdep);
                            c.c1 = make_float4(dot3(Px, Px), dot3(Px, Py), dot3(Py, Py), dot3(m, G));
                            float A[3], B[3];
                            cross3(Px, G, A);
                            cross3(Py, G, B);
                            c.c2 = make_float4(dot3(m, Px), dot3(m, Py), A[0], A[1]);
                            c.c3 = make_float4(A[2], B[0], B[1], B[2]);
                            a.cut[slot] = c;
                            if (wmode == kWeightMulti) {
                                CutExtra x;
#pragma unroll
                                for (int e = 0; e < 3; ++e) {
                                    const float *me = &xs[e][1];
                                    x.p[e] = e + 1 < nsplit
                                                 ? make_float4(xs[e][0], dot3(me, G), dot3(me, Px), dot3(me, Py))
                                                 : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
                                }
                                a.cut_x[slot] = x;
                            }
                        }
                    }
                a.rec[slot].r2.y = wmode;
            }
        }
        __syncthreads();
        if (threadIdx.x < 3 * nv) {
            const int f = threadIdx.x / nv, vv = threadIdx.x % nv;
            const unsigned long long c = s_cnt[f][vv];
            if (c) {
                ViewCounters *vc = &a.view_counters[vbase + vv];
                atomicAdd(f == 0 ? &vc->n_rendered : (f == 1 ? &vc->n_pairs : &vc->n_cutoff), c);
                atomicAdd(f == 0 ? &a.counters->n_rendered : (f == 1 ? &a.counters->n_pairs : &a.counters->n_cutoff), c);
            }
        }
    }
    // one-camera batches: the views share this Gaussian's depth, so the depth order of every
    // view is the order of the Gaussians some view renders (sorted once, then expanded per view)
    if (a.gkey && valid) a.gkey[i] = ukey;
    if (a.vmask && valid) a.vmask[i] = vmask;
}

// Compaction of rendered slots in slot order: partitions of 256 x ITEMS slots (ITEMS
// consecutive ones per thread), block prefix by warp scans, global prefix by the chained scan;
// the 8-bit digit histograms of the depth keys are accumulated on the way. Large batches take
// 16 slots per thread (fewer partitions, so fewer block barriers and look-backs), small ones
// 4 (more partitions to spread over the SMs).
constexpr int kCompactItemsLarge = 16, kCompactItemsSmall = 4;
constexpr uint32_t kCompactLargeSlots = 1u << 23;
constexpr int kExpandItems = 4;

template <int ITEMS>
__global__ void __launch_bounds__(kBlock) k_compact(CompactArgs a)
{
    __shared__ uint32_t s_hist[4][256];
    __shared__ unsigned s_part;
    __shared__ unsigned s_warp[kBlock / 32];
    __shared__ unsigned long long s_prefix;
    for (int t = threadIdx.x; t < 4 * 256; t += kBlock) (&s_hist[0][0])[t] = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t parts = (a.num_slots + kBlock * ITEMS - 1) / (kBlock * ITEMS);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_part = atomicAdd(&a.counters->ticket[kTicketCompact], 1u);
        __syncthreads();
        const uint32_t part = s_part;
        if (part >= parts) break;
        const uint32_t first = part * (kBlock * ITEMS) + threadIdx.x * ITEMS;
        uint32_t key[ITEMS];
        bool flag[ITEMS];
        unsigned cnt = 0;
        // the thread's consecutive items: 16-byte loads when all are in range (the arrays are
        // 256-byte aligned and first is a multiple of ITEMS), else one by one
        uint32_t tk[ITEMS], dk[ITEMS];
        const bool whole = first + ITEMS <= a.num_slots;
        const uint32_t *src0 = a.gkey ? a.gkey : a.tiles;
#pragma unroll
        for (int q = 0; q < ITEMS / 4; ++q) {
            uint4 t = make_uint4(0u, 0u, 0u, 0u), d = make_uint4(0u, 0u, 0u, 0u);
            if (whole) {
                t = __ldg(reinterpret_cast<const uint4 *>(src0 + first) + q);
                if (!a.gkey) d = __ldg(reinterpret_cast<const uint4 *>(a.depth + first) + q);
            }
            tk[4 * q] = t.x; tk[4 * q + 1] = t.y; tk[4 * q + 2] = t.z; tk[4 * q + 3] = t.w;
            dk[4 * q] = d.x; dk[4 * q + 1] = d.y; dk[4 * q + 2] = d.z; dk[4 * q + 3] = d.w;
        }
        if (!whole) {
#pragma unroll
            for (int r = 0; r < ITEMS; ++r) {
                const uint32_t slot = first + r;
                tk[r] = slot < a.num_slots ? src0[slot] : (a.gkey ? kNoKey : 0u);
                dk[r] = !a.gkey && slot < a.num_slots ? __float_as_uint(a.depth[slot]) : 0u;
            }
        }
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            if (a.gkey) {   // tk: the Gaussian's depth key, or kNoKey
                flag[r] = tk[r] != kNoKey;
                key[r] = flag[r] ? tk[r] : 0u;
            } else {        // tk: the slot's tile count; dk: its depth bits
                flag[r] = tk[r] != 0u;
                key[r] = flag[r] ? dk[r] : 0u;
            }
            if (flag[r]) {
                ++cnt;
                atomicAdd(&s_hist[0][key[r] & 0xffu], 1u);
                atomicAdd(&s_hist[1][(key[r] >> 8) & 0xffu], 1u);
                atomicAdd(&s_hist[2][(key[r] >> 16) & 0xffu], 1u);
                atomicAdd(&s_hist[3][key[r] >> 24], 1u);
            }
        }
        unsigned incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const unsigned w = lane < kBlock / 32 ? s_warp[lane] : 0u;
            unsigned wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += v;
            }
            const unsigned total = __shfl_sync(0xffffffffu, wi, 31);
            if (lane < kBlock / 32) s_warp[lane] = wi - w;
            const unsigned long long prefix =
                warp_chained_prefix(a.lookback, (int)part, total, &a.counters->status, a.spin_limit);
            if (lane == 0) {
                s_prefix = prefix;
                if (a.gkey && part == parts - 1) a.counters->n_union = prefix + total;  // all compacted
            }
        }
        __syncthreads();
        unsigned long long pos = s_prefix + s_warp[warp] + incl - cnt;
#pragma unroll
        for (int r = 0; r < ITEMS; ++r)
            if (flag[r]) {
                a.keys[pos] = key[r];
                a.vals[pos] = first + r;
                ++pos;
            }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * 256; t += kBlock) {
        const uint32_t v = (&s_hist[0][0])[t];
        if (v) atomicAdd(&a.hist[kHistDepth * 256 + t], v);
    }
    // view passes of the depth sort (several views): digit histograms of the view index of
    // the rendered slots (its low and high byte), and the views' first slots
    if (blockIdx.x == 0 && a.num_views > 1 && !a.gkey) {
        for (int v = threadIdx.x; v < a.num_views; v += kBlock) {
            a.seg_base[v] = a.views[v].slot_base;
            const uint32_t nr = (uint32_t)a.view_counters[v].n_rendered;
            if (nr) {
                atomicAdd(&a.hist[kHistView * 256 + (v & 0xff)], nr);
                atomicAdd(&a.hist[(kHistView + 1) * 256 + (v >> 8)], nr);
            }
        }
    }
}

// One-camera batches: expansion of the depth-sorted Gaussians into every view's rendered
// slots (see ExpandArgs): partitions of 1024 virtual elements (4 per thread, consecutive),
// block prefix by warp scans, global prefix by the chained scan, as in the compaction.
__global__ void __launch_bounds__(kBlock) k_expand(ExpandArgs a)
{
    __shared__ unsigned s_part;
    __shared__ unsigned s_warp[kBlock / 32];
    __shared__ unsigned long long s_prefix;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool in_b = a.counters->depth_in_b != 0u;
    const uint32_t *sorted = in_b ? a.sorted_b : a.sorted_a;
    uint32_t *out = in_b ? a.out_a : a.out_b;
    const uint64_t nu = a.counters->n_union;
    const uint64_t total_elems = nu * (uint64_t)a.num_views;
    const uint64_t parts = (total_elems + kBlock * kExpandItems - 1) / (kBlock * kExpandItems);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_part = atomicAdd(&a.counters->ticket[kTicketExpand], 1u);
        __syncthreads();
        const uint32_t part = s_part;
        if (part >= parts) break;
        const uint64_t first = (uint64_t)part * (kBlock * kExpandItems) + threadIdx.x * kExpandItems;
        uint32_t slot[kExpandItems];
        bool flag[kExpandItems];
        unsigned cnt = 0;
        // element e = v * nu + j: view v, the j-th Gaussian in depth order
        uint64_t v = nu ? first / nu : 0, j = first - v * nu;
#pragma unroll
        for (int r = 0; r < kExpandItems; ++r) {
            flag[r] = false;
            slot[r] = 0u;
            if (first + r < total_elems) {
                slot[r] = a.views[v].slot_base + __ldg(&sorted[j]);
                flag[r] = a.tiles[slot[r]] != 0u;
                cnt += flag[r] ? 1u : 0u;
            }
            if (++j == nu) {
                j = 0;
                ++v;
            }
        }
        unsigned incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const unsigned w = lane < kBlock / 32 ? s_warp[lane] : 0u;
            unsigned wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            const unsigned total = __shfl_sync(0xffffffffu, wi, 31);
            if (lane < kBlock / 32) s_warp[lane] = wi - w;
            const unsigned long long prefix = warp_chained_prefix(a.lookback, (int)part, total, &a.counters->status);
            if (lane == 0) s_prefix = prefix;
        }
        __syncthreads();
        unsigned long long pos = s_prefix + s_warp[warp] + incl - cnt;
        const unsigned long long cap = a.counters->n_rendered;   // the expansion lists exactly these
#pragma unroll
        for (int r = 0; r < kExpandItems; ++r)
            if (flag[r]) {
                if (pos < cap) out[pos] = slot[r];
                ++pos;
            }
    }
}

}  // namespace

void launch_expand(const ExpandArgs &a, int grid, cudaStream_t s)
{
    if (grid > 0) k_expand<<<grid, kBlock, 0, s>>>(a);
}

int preprocess_configure()
{
    const int most = 3 * 16 * kBlock * (int)sizeof(float);  // SH degree 3
    return cudaFuncSetAttribute(k_preprocess, cudaFuncAttributeMaxDynamicSharedMemorySize, most) == cudaSuccess
               ? 0
               : -1;
}

void launch_preprocess(const PreprocessArgs &a, int grid, int max_sh_degree, int max_views, cudaStream_t s)
{
    (void)max_views;
    const int smem = 3 * (max_sh_degree + 1) * (max_sh_degree + 1) * kBlock * (int)sizeof(float);
    if (grid <= 0) return;
    k_preprocess<<<grid, kBlock, smem, s>>>(a);
}

int compact_blocks_per_sm()
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_compact<kCompactItemsLarge>, kBlock, 0) != cudaSuccess ||
        b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

void launch_compact(const CompactArgs &a, int grid, cudaStream_t s)
{
    if (grid <= 0) return;
    if (a.num_slots >= kCompactLargeSlots) k_compact<kCompactItemsLarge><<<grid, kBlock, 0, s>>>(a);
    else k_compact<kCompactItemsSmall><<<grid, kBlock, 0, s>>>(a);
}

}  // namespace rara
