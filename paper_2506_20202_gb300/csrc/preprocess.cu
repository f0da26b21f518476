// Step (a): per-Gaussian classification, projection, SH colour and compaction.
//
// One thread per Gaussian. Loads are planar (one coalesced 128-byte line per warp per
// attribute plane). The kernel writes, for every Gaussian, its label and tiles-touched
// count, and for rendered Gaussians the 48-byte splat record, the tile rectangle, the
// 64-byte ray-tracing record (cutoff only) and a compacted (depth bits, index) entry in
// index order, placed by a chained scan across blocks so the order is deterministic.
#include "chained_scan.cuh"
#include "rara_internal.cuh"

namespace rara {

namespace {

// Real spherical harmonics, orthonormal, standard (l, m) basis with positive polynomials:
// Y_{1,-1} = c1 y, Y_{1,0} = c1 z, Y_{1,1} = c1 x, etc. Coefficient index k = l*l + l + m.
constexpr float kY00 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;    // (1/2) sqrt(15 / pi)
constexpr float kY20 = 0.31539156525252005f;   // (1/4) sqrt(5 / pi)
constexpr float kY22 = 0.54627421529603959f;   // (1/4) sqrt(15 / pi)
constexpr float kY33 = 0.59004358992664352f;   // (1/4) sqrt(35 / (2 pi))
constexpr float kY32 = 2.8906114426405538f;    // (1/2) sqrt(105 / pi)
constexpr float kY31 = 0.45704579946446572f;   // (1/4) sqrt(21 / (2 pi))
constexpr float kY30 = 0.37317633259011540f;   // (1/4) sqrt(7 / pi)
constexpr float kY32b = 1.4453057213202769f;   // (1/4) sqrt(105 / pi)

__device__ __forceinline__ float shc(const float *__restrict__ sh, int n, int i, int k, int c)
{
    return __ldg(&sh[(size_t)(k * 3 + c) * n + i]);
}

__device__ void sh_colour(const float *__restrict__ sh, int n, int i, int degree, float x, float y,
                          float z, float rgb[3])
{
    float basis[16];
    basis[0] = kY00;
    int kmax = 1;
    if (degree >= 1) {
        basis[1] = kY1 * y;
        basis[2] = kY1 * z;
        basis[3] = kY1 * x;
        kmax = 4;
    }
    if (degree >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        basis[4] = kY2a * x * y;
        basis[5] = kY2a * y * z;
        basis[6] = kY20 * (3.0f * zz - 1.0f);
        basis[7] = kY2a * x * z;
        basis[8] = kY22 * (xx - yy);
        kmax = 9;
        if (degree >= 3) {
            basis[9] = kY33 * y * (3.0f * xx - yy);
            basis[10] = kY32 * x * y * z;
            basis[11] = kY31 * y * (5.0f * zz - 1.0f);
            basis[12] = kY30 * z * (5.0f * zz - 3.0f);
            basis[13] = kY31 * x * (5.0f * zz - 1.0f);
            basis[14] = kY32b * z * (xx - yy);
            basis[15] = kY33 * x * (xx - 3.0f * yy);
            kmax = 16;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < kmax) acc = fmaf(shc(sh, n, i, k, c), basis[k], acc);
        rgb[c] = fmaxf(acc + 0.5f, 0.0f);
    }
}

__global__ void __launch_bounds__(kBlock) k_preprocess(PreprocessArgs a)
{
    __shared__ unsigned s_part;
    __shared__ unsigned s_warp_cnt[kBlock / 32];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned long long s_pairs[kBlock / 32];
    __shared__ unsigned s_cut[kBlock / 32];

    if (threadIdx.x == 0) s_part = atomicAdd(&a.counters->part_counter[0], 1u);
    __syncthreads();
    const int part = (int)s_part;
    const int i = part * kBlock + threadIdx.x;
    const int n = a.n;

    bool rendered = false;
    bool cutoff = false;
    uint32_t ntiles = 0;
    float depth = 0.0f;

    if (i < n) {
        const float mx = __ldg(&a.means[i]), my = __ldg(&a.means[n + i]), mz = __ldg(&a.means[2 * n + i]);
        const float s0 = expf(__ldg(&a.log_scales[i]));
        const float s1 = expf(__ldg(&a.log_scales[n + i]));
        const float s2 = expf(__ldg(&a.log_scales[2 * n + i]));
        const PlaneDev &pl = a.plane;

        // Section 3.2 / Algorithm 1 step 1: d_ep = n.mu + d, r = 3 max(sigma)
        const float dep = fmaf(pl.n[0], mx, fmaf(pl.n[1], my, fmaf(pl.n[2], mz, pl.d)));
        const float r = 3.0f * fmaxf(s0, fmaxf(s1, s2));
        int label;
        if (pl.mode == RARA_MODE_NONE) label = RARA_VISIBLE;
        else if (pl.mode == RARA_MODE_HARD) label = dep < 0.0f ? RARA_INVISIBLE : RARA_VISIBLE;
        else {
            label = dep < -r ? RARA_INVISIBLE : (dep > r ? RARA_VISIBLE : RARA_CUTOFF);
            if (pl.mode == RARA_MODE_RARA_ALL && label != RARA_INVISIBLE) label = RARA_CUTOFF;
        }
        a.labels[i] = (uint8_t)label;

        const CamDev &cam = a.cam;
        const float tx = fmaf(cam.R[0], mx, fmaf(cam.R[1], my, fmaf(cam.R[2], mz, cam.t[0])));
        const float ty = fmaf(cam.R[3], mx, fmaf(cam.R[4], my, fmaf(cam.R[5], mz, cam.t[1])));
        const float tz = fmaf(cam.R[6], mx, fmaf(cam.R[7], my, fmaf(cam.R[8], mz, cam.t[2])));
        // The sort key holds the depth rounded once from a double-precision dot product, so
        // it is the correctly rounded float32 of the exact depth (ties order by index).
        depth = (float)fma((double)cam.R[6], (double)mx,
                           fma((double)cam.R[7], (double)my, fma((double)cam.R[8], (double)mz, (double)cam.t[2])));

        if (label != RARA_INVISIBLE && tz > kNearZ) {
            // Rotation of the normalised quaternion (w, x, y, z)
            float qw = __ldg(&a.quats[i]), qx = __ldg(&a.quats[n + i]);
            float qy = __ldg(&a.quats[2 * n + i]), qz = __ldg(&a.quats[3 * n + i]);
            const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
            qw *= qn; qx *= qn; qy *= qn; qz *= qn;
            const float Rg[9] = {
                1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
            const float sg[3] = {s0, s1, s2};

            // Eq. 9-10: Sigma2 = (J W M)(J W M)^T + 0.3 I with M = R S and J the affine
            // approximation of the projection at the centre (x/z, y/z clamped).
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
            // det((A A^T) + 0.3 I) = |A0 x A1|^2 + 0.3 (a0 + c0) + 0.09: every term is
            // non-negative, so elongated splats keep their precision.
            const float x0 = A0[1] * A1[2] - A0[2] * A1[1];
            const float x1 = A0[2] * A1[0] - A0[0] * A1[2];
            const float x2 = A0[0] * A1[1] - A0[1] * A1[0];
            const float ca = a0 + kDilation, cb = b0, cc = c0 + kDilation;
            const float det = (x0 * x0 + x1 * x1 + x2 * x2) + kDilation * (a0 + c0) + kDilation * kDilation;
            if (det > 0.0f) {
                const float idet = 1.0f / det;
                const float mx2 = fmaf(cam.fx, tx * itz, cam.cx);
                const float my2 = fmaf(cam.fy, ty * itz, cam.cy);
                // Tile rectangle: axis-aligned box of the q <= 9 ellipse
                const float hx = 3.0f * sqrtf(ca), hy = 3.0f * sqrtf(cc);
                const float inv_t = 1.0f / kTile;
                const float fx0 = floorf((mx2 - hx) * inv_t), fx1 = floorf((mx2 + hx) * inv_t);
                const float fy0 = floorf((my2 - hy) * inv_t), fy1 = floorf((my2 + hy) * inv_t);
                const int rx0 = (int)fmaxf(0.0f, fminf((float)a.tiles_x, fx0));
                const int rx1 = (int)fmaxf(-1.0f, fminf((float)(a.tiles_x - 1), fx1));
                const int ry0 = (int)fmaxf(0.0f, fminf((float)a.tiles_y, fy0));
                const int ry1 = (int)fmaxf(-1.0f, fminf((float)(a.tiles_y - 1), fy1));
                if (rx0 <= rx1 && ry0 <= ry1) {
                    ntiles = (uint32_t)((rx1 - rx0 + 1) * (ry1 - ry0 + 1));
                    rendered = true;
                    cutoff = label == RARA_CUTOFF;
                    a.rect[i] = make_uint2((uint32_t)rx0 | ((uint32_t)ry0 << 16),
                                           (uint32_t)rx1 | ((uint32_t)ry1 << 16));
                    const float op = 1.0f / (1.0f + expf(-__ldg(&a.logits[i])));
                    // colour at normalize(mu - e)
                    const float ex = mx - cam.eye[0], ey = my - cam.eye[1], ez = mz - cam.eye[2];
                    const float il = rsqrtf(ex * ex + ey * ey + ez * ez);
                    float rgb[3];
                    sh_colour(a.sh, n, i, a.sh_degree, ex * il, ey * il, ez * il, rgb);
                    SplatRec rec;
                    rec.r0 = make_float4(mx2, my2, cc * idet, -cb * idet);
                    rec.r1 = make_float4(ca * idet, op, rgb[0], rgb[1]);
                    rec.r2 = make_float4(rgb[2], cutoff ? 1.0f : 0.0f, cb / cc, cb / ca);
                    a.rec[i] = rec;
                    a.depth[i] = depth;

                    if (cutoff) {
                        // Ray-tracing record in the unit-sphere frame of M = k R S
                        // (Eq. 4): M^-1 = diag(1/(k sigma)) R^T. For the pixel ray with
                        // offset (dx, dy) from the projected centre, the local ray is
                        // o + tau V with o = -G, V = G + P (dx, dy): G = M^-1 (mu - e) and
                        // P = z M^-1 W^T[:, 0:2] diag(1/fx, 1/fy). m = M^T n carries the
                        // plane into the same frame: s(x) = d_ep + m . u for x = mu + M u.
                        const float kk = pl.k;
                        const float iks[3] = {1.0f / (kk * s0), 1.0f / (kk * s1), 1.0f / (kk * s2)};
                        float G[3], Px[3], Py[3], m[3];
                        const float cxw[3] = {cam.R[0], cam.R[1], cam.R[2]};  // camera x axis (world)
                        const float cyw[3] = {cam.R[3], cam.R[4], cam.R[5]};  // camera y axis (world)
                        const float sx = tz / cam.fx, sy = tz / cam.fy;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float rk0 = Rg[k], rk1 = Rg[3 + k], rk2 = Rg[6 + k];  // column k of R
                            G[k] = iks[k] * (rk0 * ex + rk1 * ey + rk2 * ez);
                            Px[k] = iks[k] * sx * (rk0 * cxw[0] + rk1 * cxw[1] + rk2 * cxw[2]);
                            Py[k] = iks[k] * sy * (rk0 * cyw[0] + rk1 * cyw[1] + rk2 * cyw[2]);
                            m[k] = kk * sg[k] * (rk0 * pl.n[0] + rk1 * pl.n[1] + rk2 * pl.n[2]);
                        }
                        CutRec c;
                        c.c0 = make_float4(G[0], G[1], G[2], dep);
                        c.c1 = make_float4(Px[0], Px[1], Px[2], m[0]);
                        c.c2 = make_float4(Py[0], Py[1], Py[2], m[1]);
                        c.c3 = make_float4(m[2], 0.0f, 0.0f, 0.0f);
                        a.cut[i] = c;
                    }
                }
            }
        }
        a.tiles[i] = ntiles;
    }

    // Stable compaction of rendered Gaussians: block prefix by warp ballots, global
    // prefix by the chained scan.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ballot = __ballot_sync(0xffffffffu, rendered);
    const unsigned cut_ballot = __ballot_sync(0xffffffffu, cutoff);
    unsigned long long pairs = ntiles;
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    if (lane == 0) {
        s_warp_cnt[warp] = __popc(ballot);
        s_pairs[warp] = pairs;
        s_cut[warp] = __popc(cut_ballot);
    }
    __syncthreads();
    if (warp == 0) {
        unsigned cnt = lane < kBlock / 32 ? s_warp_cnt[lane] : 0u;
        unsigned incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        if (lane < kBlock / 32) s_warp_cnt[lane] = incl - cnt;  // exclusive over warps
        const unsigned long long prefix = warp_chained_prefix(a.lookback, part, total, &a.counters->status);
        if (lane == 0) {
            s_prefix = prefix;
            unsigned long long bp = 0, bc = 0;
            for (int w = 0; w < kBlock / 32; ++w) { bp += s_pairs[w]; bc += s_cut[w]; }
            if (total) atomicAdd(&a.counters->n_rendered, (unsigned long long)total);
            if (bp) atomicAdd(&a.counters->n_pairs, bp);
            if (bc) atomicAdd(&a.counters->n_cutoff, bc);
        }
    }
    __syncthreads();
    if (rendered) {
        const unsigned long long pos = s_prefix + s_warp_cnt[warp] + __popc(ballot & ((1u << lane) - 1u));
        a.ckeys[pos] = __float_as_uint(depth);
        a.cvals[pos] = (uint32_t)i;
    }
}

}  // namespace

void launch_preprocess(const PreprocessArgs &a, int num_blocks, cudaStream_t s)
{
    if (num_blocks > 0) k_preprocess<<<num_blocks, kBlock, 0, s>>>(a);
}

}  // namespace rara
