/*
 * rara_oracle.c -- plain FP64 CPU oracle of the RaRa clipped Gaussian-splat render
 * (arXiv 2506.20202, "RaRa Clipper").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct statement of what
 * the render computes. It is called by the tests, by the oracle check in the entry-point
 * smoke test and by the benchmark's CPU-baseline leg; nothing on the product path links,
 * loads or calls it, and it shares no code with the CUDA library.
 *
 * Arithmetic is double precision throughout. The Gaussians' parameters arrive as double
 * arrays: the float32 values the GPU consumes, widened exactly, or (for finite-difference
 * gradients) any double values. Every step follows the paper's order:
 *   1. per Gaussian: covariance V = R S^2 R^T (Section 3.1), three-way classification
 *      against the plane (Section 3.2, Eq. 3; Algorithm 1 step 1), EWA projection of the
 *      covariance (Section 3.4, Eq. 9-10), colour from real spherical harmonics;
 *   2. binning: one (tile, depth) key per touched tile, stable sort (Section 3.1 "points
 *      are sorted by depth");
 *   3. per pixel: candidates in depth order, alpha from Eq. 10, for cutoff Gaussians the
 *      ray-ellipsoid chord (Eq. 4-7), ray-plane hit (Eq. 8) and decay weight (Eq. 11),
 *      opacity update and clamp (Eq. 12, Algorithm 1 step 3), front-to-back compositing
 *      (Eq. 2).
 * Readings where the paper is silent or inconsistent (all listed in the design notes):
 *   - the ray-traced ellipsoid is M = k R S with k = k_sigma (default 3, the 3-sigma
 *     support of Section 3 and the r = 3 max(sigma) of Section 3.2);
 *   - the normalisation factors of Eq. 1/9/10 are dropped: alpha0 = delta exp(-q/2);
 *   - a chord with both ends visible gets w = 1, both ends invisible w = 0; a ray that
 *     misses or grazes the ellipsoid, or starts inside or behind it, gets w = 1;
 *   - renderer conventions inherited from 3D Gaussian Splatting: 0.3 px^2 dilation,
 *     near cull at z <= 0.2, Jacobian clamp at 1.3 tan(half FOV), per-pixel support
 *     q <= 9, skip when alpha < 1/255, stop before the Gaussian that takes T below 1e-4;
 *   - pixel centres at (i + 0.5, j + 0.5); depth order by (float32(depth), index).
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INVISIBLE 0
#define ORC_VISIBLE 1
#define ORC_CUTOFF 2

#define ORC_MODE_NONE 0
#define ORC_MODE_HARD 1
#define ORC_MODE_RARA 2
#define ORC_MODE_RARA_ALL 3

/* Per-pixel event bits: the pixel's oracle sequence passed within tolerance of a
 * discontinuity of the method, so a float32 renderer may legitimately differ there. */
#define EV_Q 1u        /* q near the support bound 9 */
#define EV_ALPHA 2u    /* final alpha near 1/255 */
#define EV_T 4u        /* transmittance near the 1e-4 stop */
#define EV_GAUSS 8u    /* a candidate, or the footprint of an invisible Gaussian, near a threshold where the image jumps */
#define EV_DISC 16u    /* ray grazing a cutoff ellipsoid (discriminant near 0) */
#define EV_DEPTH 32u   /* two candidates whose float32 depths differ by a few ulp */
#define EV_T1 64u      /* camera on the surface of a cutoff ellipsoid */

/* ------------------------------------------------------------------------------------ */
/* Small linear algebra                                                                  */
/* ------------------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Rotation matrix of the normalised quaternion (w, x, y, z). */
static void quat_to_rot(double w, double x, double y, double z, double R[3][3])
{
    double nrm = sqrt(w * w + x * x + y * y + z * z);
    w /= nrm; x /= nrm; y /= nrm; z /= nrm;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

typedef struct {
    double R[3][3]; /* world -> camera rotation W */
    double t[3];
    double fx, fy, cx, cy;
    int W, H;
    double e[3];    /* camera centre in world coordinates, e = -R^T t */
} cam_t;

static void load_cam(const double *cam16, int W, int H, cam_t *c)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c->R[i][j] = cam16[i * 3 + j];
    for (int i = 0; i < 3; ++i) c->t[i] = cam16[9 + i];
    c->fx = cam16[12]; c->fy = cam16[13]; c->cx = cam16[14]; c->cy = cam16[15];
    c->W = W; c->H = H;
    for (int j = 0; j < 3; ++j) c->e[j] = -(c->R[0][j] * c->t[0] + c->R[1][j] * c->t[1] + c->R[2][j] * c->t[2]);
}

/* ------------------------------------------------------------------------------------ */
/* Real spherical harmonics, from the associated Legendre functions                       */
/* ------------------------------------------------------------------------------------ */

static double factorial(int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; }

/* Associated Legendre P_l^m(x) for m >= 0 WITHOUT the Condon-Shortley phase, by the
 * standard upward recurrences: P_m^m = (2m-1)!! (1-x^2)^{m/2}, P_{m+1}^m = x (2m+1) P_m^m,
 * (l-m) P_l^m = x (2l-1) P_{l-1}^m - (l+m-1) P_{l-2}^m. */
static double legendre_p(int l, int m, double x)
{
    double pmm = 1.0, s = sqrt(fmax(0.0, 1.0 - x * x));
    for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * s;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pl = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pl = (x * (2.0 * ll - 1.0) * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1; pm1 = pl;
    }
    return pl;
}

/* Real orthonormal SH Y_{l,m}(dir) for a unit direction: m = 0: K P_l^0(cos th);
 * m > 0: sqrt2 K P_l^m cos(m phi); m < 0: sqrt2 K P_l^|m| sin(|m| phi),
 * K = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!). */
double orc_real_sh(int l, int m, const double *dir)
{
    int am = m < 0 ? -m : m;
    double ct = dir[2];
    double phi = atan2(dir[1], dir[0]);
    double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
    double P = legendre_p(l, am, ct);
    if (m == 0) return K * P;
    if (m > 0) return sqrt(2.0) * K * P * cos(am * phi);
    return sqrt(2.0) * K * P * sin(am * phi);
}

/* Colour of Gaussian i seen along unit direction dir: sum_k sh_k Y_k(dir) + 0.5, clamped at 0. */
static void eval_colour(const double *sh, int64_t n, int64_t i, int degree, const double *dir, double rgb[3])
{
    for (int c = 0; c < 3; ++c) rgb[c] = 0.0;
    for (int l = 0; l <= degree; ++l)
        for (int m = -l; m <= l; ++m) {
            int k = l * l + l + m;
            double y = orc_real_sh(l, m, dir);
            for (int c = 0; c < 3; ++c) rgb[c] += sh[(int64_t)(k * 3 + c) * n + i] * y;
        }
    for (int c = 0; c < 3; ++c) rgb[c] = fmax(rgb[c] + 0.5, 0.0);
}

/* ------------------------------------------------------------------------------------ */
/* Step 1: per-Gaussian classification and projection                                    */
/* ------------------------------------------------------------------------------------ */

/*
 * Outputs, per Gaussian i (caller-allocated):
 *   label[i]      0 invisible, 1 visible, 2 cutoff (Section 3.2; mode variants below)
 *   culled[i]     1 if not rendered: invisible, z <= 0.2, singular 2D covariance, or no tile
 *                 (the projection fields below are still filled for invisible Gaussians)
 *   depth[i]      camera-space z of the centre
 *   mean2d[2i..]  projected centre (pixels)
 *   cov2d[3i..]   dilated 2D covariance (a, b, c) = [[a, b], [b, c]]
 *   conic[3i..]   inverse of cov2d, same packing
 *   rect[4i..]    inclusive tile rectangle (tx0, ty0, tx1, ty1)
 *   tiles[i]      number of tiles in the rectangle (0 when culled)
 *   rgb[3i..], opacity[i], d_ep[i], radius[i] (= 3 max sigma)
 *   margin_class[i]  distance of d_ep to the nearest label threshold (world units)
 *   margin_gauss[i]  distance to the nearest threshold across which the image is
 *                    discontinuous: the near cull (z); for hard clipping the centre test;
 *                    for the three-way rule the invisible threshold d_ep = -r of every
 *                    plane (and, with k_sigma > 3, the visible threshold d_ep = +r too)
 *   margin_rect[i]   distance (pixels) of the rectangle bounds to the nearest tile edge
 * Modes: NONE labels all visible; HARD labels invisible iff d_ep < 0 (centre test);
 * RARA is the paper's three-way rule; RARA_ALL uses the three-way rule but ray-traces
 * every non-invisible Gaussian (label cutoff for all of them).
 * plane4 holds nplanes >= 1 planes (n, d), four doubles each; the visible region is the
 * intersection of their visible sides (a convex clip volume). The three-way rule then
 * reads: invisible if the Gaussian's sphere of radius r lies wholly behind some plane
 * (d_ep,k < -r for some k), visible if it lies wholly in front of all of them (d_ep,k > r
 * for every k), cutoff otherwise; hard clipping: invisible iff the centre is behind some
 * plane. With one plane these are the rules above. d_ep[i] reports the first plane's.
 */
int orc_preprocess(int64_t n, const double *means, const double *log_scales, const double *quats,
                   const double *opacity_logits, const double *sh, int sh_degree,
                   const double *cam16, int W, int H, const double *plane4, int nplanes, double k_sigma,
                   int mode, int tile_w, int tile_h,
                   uint8_t *label, uint8_t *culled, double *depth, double *mean2d, double *cov2d,
                   double *conic, int32_t *rect, int32_t *tiles, double *rgb, double *opacity,
                   double *d_ep, double *radius, double *margin_class, double *margin_gauss,
                   double *margin_rect)
{
    cam_t cam;
    load_cam(cam16, W, H, &cam);
    const int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
    const double pn[3] = {plane4[0], plane4[1], plane4[2]}, pd = plane4[3];
    const double limx = 1.3 * (0.5 * W / cam.fx), limy = 1.3 * (0.5 * H / cam.fy);

    for (int64_t i = 0; i < n; ++i) {
        double mu[3] = {means[i], means[n + i], means[2 * n + i]};
        double sig[3] = {exp(log_scales[i]), exp(log_scales[n + i]), exp(log_scales[2 * n + i])};

        /* Section 3.2 / Algorithm 1 step 1: signed distance of the centre and r = 3 max sigma. */
        double dep = dot3(pn, mu) + pd;
        double smax = fmax(sig[0], fmax(sig[1], sig[2]));
        double r = 3.0 * smax;
        d_ep[i] = dep;
        radius[i] = r;
        int lab;
        double mc = INFINITY;   /* distance to the label thresholds */
        double mg = INFINITY;   /* distance to thresholds where the image is discontinuous */
        if (mode == ORC_MODE_NONE) {
            lab = ORC_VISIBLE;
        } else if (mode == ORC_MODE_HARD) {
            int behind = 0;
            mc = INFINITY;
            for (int k = 0; k < nplanes; ++k) {
                double dk = dot3(&plane4[4 * k], mu) + plane4[4 * k + 3];
                behind = behind || dk < 0.0;
                mc = fmin(mc, fabs(dk));
            }
            lab = behind ? ORC_INVISIBLE : ORC_VISIBLE;
            mg = mc;
        } else {
            int behind = 0, front = 1;
            double m_inv = INFINITY;  /* distance to the invisible thresholds d_ep,k = -r */
            mc = INFINITY;
            for (int k = 0; k < nplanes; ++k) {
                double dk = dot3(&plane4[4 * k], mu) + plane4[4 * k + 3];
                behind = behind || dk < -r;
                front = front && dk > r;
                mc = fmin(mc, fmin(fabs(dk - r), fabs(dk + r)));
                m_inv = fmin(m_inv, fabs(dk + r));
            }
            if (behind) lab = ORC_INVISIBLE;
            else if (front) lab = ORC_VISIBLE;
            else lab = ORC_CUTOFF;
            if (mode == ORC_MODE_RARA_ALL && lab != ORC_INVISIBLE) lab = ORC_CUTOFF;
            /* Where the image jumps. At d_ep = +r (k_sigma <= 3) the traced ellipsoid lies
             * inside the radius-r sphere, so every chord is already wholly visible (w = 1)
             * when the label turns visible: no jump. At d_ep = -r it is not so: a ray that
             * hits the ellipsoid has w = 0 just before the Gaussian turns invisible, but the
             * pixels of the q <= 9 footprint whose rays miss the ellipsoid (the footprint is
             * the EWA approximation widened by the 0.3 px^2 dilation, so it reaches past the
             * ellipsoid's silhouette) keep w = 1 up to the threshold and drop to nothing
             * after it. With k_sigma > 3 the ellipsoid pokes out of the sphere and +r jumps
             * as well. */
            mg = k_sigma > 3.0 ? mc : m_inv;
        }
        label[i] = (uint8_t)lab;
        margin_class[i] = mc;

        culled[i] = 1; tiles[i] = 0;
        rect[4 * i + 0] = rect[4 * i + 1] = 0; rect[4 * i + 2] = rect[4 * i + 3] = -1;
        mean2d[2 * i] = mean2d[2 * i + 1] = 0.0;
        for (int k = 0; k < 3; ++k) { cov2d[3 * i + k] = 0.0; conic[3 * i + k] = 0.0; rgb[3 * i + k] = 0.0; }
        opacity[i] = 0.0; depth[i] = 0.0; margin_rect[i] = INFINITY;

        /* camera-space centre */
        double tc[3];
        for (int a = 0; a < 3; ++a) tc[a] = dot3(cam.R[a], mu) + cam.t[a];
        depth[i] = tc[2];
        mg = fmin(mg, fabs(tc[2] - 0.2));
        margin_gauss[i] = mg;
        if (tc[2] <= 0.2) continue;

        /* Section 3.1: V = R S^2 R^T */
        double Rg[3][3], V[3][3];
        quat_to_rot(quats[i], quats[n + i], quats[2 * n + i], quats[3 * n + i], Rg);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += Rg[a][k] * sig[k] * sig[k] * Rg[b][k];
                V[a][b] = s;
            }

        /* Eq. 9-10: upper-left 2x2 of J W V W^T J^T, J the affine approximation of the
         * perspective map at the centre (x/z, y/z clamped to 1.3 tan(half FOV)). */
        double tz = tc[2];
        double txz = fmin(limx, fmax(-limx, tc[0] / tz));
        double tyz = fmin(limy, fmax(-limy, tc[1] / tz));
        double J[2][3] = {{cam.fx / tz, 0.0, -cam.fx * txz / tz}, {0.0, cam.fy / tz, -cam.fy * tyz / tz}};
        double T[2][3];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) T[a][b] = J[a][0] * cam.R[0][b] + J[a][1] * cam.R[1][b] + J[a][2] * cam.R[2][b];
        double S2[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) s += T[a][k] * V[k][l] * T[b][l];
                S2[a][b] = s;
            }
        double ca = S2[0][0] + 0.3, cb = S2[0][1], cc = S2[1][1] + 0.3;
        double det = ca * cc - cb * cb;
        if (det <= 0.0) continue;
        cov2d[3 * i] = ca; cov2d[3 * i + 1] = cb; cov2d[3 * i + 2] = cc;
        conic[3 * i] = cc / det; conic[3 * i + 1] = -cb / det; conic[3 * i + 2] = ca / det;
        double mx = cam.fx * tc[0] / tz + cam.cx, my = cam.fy * tc[1] / tz + cam.cy;
        mean2d[2 * i] = mx; mean2d[2 * i + 1] = my;

        /* Tile rectangle: the axis-aligned box of the q <= 9 ellipse, |dx| <= 3 sqrt(a),
         * |dy| <= 3 sqrt(c), mapped to tile indices and clamped to the grid. */
        double hx = 3.0 * sqrt(ca), hy = 3.0 * sqrt(cc);
        double bx[2] = {mx - hx, mx + hx}, by[2] = {my - hy, my + hy};
        double fx0 = floor(bx[0] / tile_w), fx1 = floor(bx[1] / tile_w);
        double fy0 = floor(by[0] / tile_h), fy1 = floor(by[1] / tile_h);
        int tx0 = (int)fmax(0.0, fmin((double)tiles_x, fx0));
        int tx1 = (int)fmax(-1.0, fmin((double)tiles_x - 1, fx1));
        int ty0 = (int)fmax(0.0, fmin((double)tiles_y, fy0));
        int ty1 = (int)fmax(-1.0, fmin((double)tiles_y - 1, fy1));
        double mr = INFINITY;
        for (int k = 0; k < 2; ++k) {
            mr = fmin(mr, fabs(bx[k] - tile_w * nearbyint(bx[k] / tile_w)));
            mr = fmin(mr, fabs(by[k] - tile_h * nearbyint(by[k] / tile_h)));
        }
        margin_rect[i] = mr;
        if (tx0 > tx1 || ty0 > ty1) continue;
        rect[4 * i] = tx0; rect[4 * i + 1] = ty0; rect[4 * i + 2] = tx1; rect[4 * i + 3] = ty1;
        /* Invisible Gaussians keep their projection (for diagnostics) but are discarded
         * (Algorithm 1 step 1 returns alpha = 0). */
        if (lab == ORC_INVISIBLE) continue;
        tiles[i] = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
        culled[i] = 0;

        opacity[i] = 1.0 / (1.0 + exp(-opacity_logits[i]));
        double dir[3] = {mu[0] - cam.e[0], mu[1] - cam.e[1], mu[2] - cam.e[2]};
        double dl = sqrt(dot3(dir, dir));
        for (int k = 0; k < 3; ++k) dir[k] /= dl;
        double col[3];
        eval_colour(sh, n, i, sh_degree, dir, col);
        for (int k = 0; k < 3; ++k) rgb[3 * i + k] = col[k];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Step 2: binning keys                                                                  */
/* ------------------------------------------------------------------------------------ */

static uint32_t f32_bits(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

typedef struct { uint64_t key; uint32_t val; } kv_t;

static int cmp_kv(const void *a, const void *b)
{
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->val != y->val) return x->val < y->val ? -1 : 1;
    return 0;
}

/* Smallest value of q(dx, dy) = a dx^2 + 2 b dx dy + c dy^2 (a positive definite conic) over
 * the box [x0, x1] x [y0, y1] of offsets from the projected centre. q is convex: the minimum
 * is 0 when the box holds the centre, and otherwise lies on the boundary, so it is the
 * smallest of the four edge minima; along an edge q is a 1D quadratic whose vertex is
 * clamped to the edge. */
double orc_box_min_q(double a, double b, double c, double x0, double x1, double y0, double y1)
{
    if (x0 <= 0.0 && x1 >= 0.0 && y0 <= 0.0 && y1 >= 0.0) return 0.0;
    double best = INFINITY;
    const double ys[2] = {y0, y1}, xs[2] = {x0, x1};
    for (int k = 0; k < 2; ++k) {
        /* horizontal edge dy = ys[k]: q = a dx^2 + 2 b ys dx + c ys^2, vertex dx = -b ys / a */
        double dy = ys[k];
        double dx = fmin(x1, fmax(x0, -b * dy / a));
        best = fmin(best, a * dx * dx + 2.0 * b * dx * dy + c * dy * dy);
        /* vertical edge dx = xs[k]: vertex dy = -b xs / c */
        dx = xs[k];
        dy = fmin(y1, fmax(y0, -b * dx / c));
        best = fmin(best, a * dx * dx + 2.0 * b * dx * dy + c * dy * dy);
    }
    return best;
}

/* q up to which Gaussian i can blend: alpha0 = opacity exp(-q/2) >= 1/255 and q <= 9, so
 * q_cut = min(9, 2 ln(255 opacity)). Beyond it a pixel skips the Gaussian (Algorithm 1
 * step 3 skips alpha < 1/255, and the decay weight w <= 1 only lowers alpha). */
static double q_cut(double opacity)
{
    return fmin(9.0, 2.0 * log(255.0 * opacity));
}

/* Whether tile (tx, ty) lists Gaussian i: the smallest q over the rectangle spanned by the
 * tile's pixel centres (those inside the W x H image) is at most q_cut. Every pixel centre
 * of the tile lies in that rectangle, so a pixel where the Gaussian can blend is never in a
 * tile that does not list it. */
static int tile_lists(const double *mean2d, const double *conic, const double *opacity, int64_t i, int tx, int ty,
                      int W, int H, int tile_w, int tile_h)
{
    double px0 = tx * tile_w + 0.5, px1 = fmin((double)(tx + 1) * tile_w, (double)W) - 0.5;
    double py0 = ty * tile_h + 0.5, py1 = fmin((double)(ty + 1) * tile_h, (double)H) - 0.5;
    double mx = mean2d[2 * i], my = mean2d[2 * i + 1];
    double m = orc_box_min_q(conic[3 * i], conic[3 * i + 1], conic[3 * i + 2], px0 - mx, px1 - mx, py0 - my,
                             py1 - my);
    return m <= q_cut(opacity[i]);
}

/* Number of (Gaussian, tile) pairs: the tiles of each rendered Gaussian's rectangle that
 * list it (tile_lists). */
int64_t orc_count_pairs(int64_t n, const uint8_t *culled, const int32_t *rect, const double *mean2d,
                        const double *conic, const double *opacity, int W, int H, int tile_w, int tile_h)
{
    int64_t p = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (culled[i]) continue;
        for (int ty = rect[4 * i + 1]; ty <= rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx <= rect[4 * i + 2]; ++tx)
                p += tile_lists(mean2d, conic, opacity, i, tx, ty, W, H, tile_w, tile_h);
    }
    return p;
}

/* One key per listing tile: key = tile_id << 32 | bits(float32(depth)), value = Gaussian
 * index, tile_id = ty * tiles_x + tx. Sorted ascending by (key, index), which is the
 * stable sort of the index-ordered emission. ranges[2t], ranges[2t+1] = [start, end) of
 * tile t in the sorted list (zero-length when empty). */
int orc_build_keys(int64_t n, const uint8_t *culled, const int32_t *rect, const double *depth,
                   const double *mean2d, const double *conic, const double *opacity, int W, int H,
                   int tile_w, int tile_h, uint64_t *keys, uint32_t *vals, int64_t *ranges)
{
    const int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
    int64_t p = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (culled[i]) continue;
        uint32_t db = f32_bits(depth[i]);
        for (int ty = rect[4 * i + 1]; ty <= rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx <= rect[4 * i + 2]; ++tx) {
                if (!tile_lists(mean2d, conic, opacity, i, tx, ty, W, H, tile_w, tile_h)) continue;
                keys[p] = ((uint64_t)(uint32_t)(ty * tiles_x + tx) << 32) | db;
                vals[p] = (uint32_t)i;
                ++p;
            }
    }
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)(p > 0 ? p : 1));
    if (!kv) return -1;
    for (int64_t k = 0; k < p; ++k) { kv[k].key = keys[k]; kv[k].val = vals[k]; }
    qsort(kv, (size_t)p, sizeof(kv_t), cmp_kv);
    for (int64_t k = 0; k < p; ++k) { keys[k] = kv[k].key; vals[k] = kv[k].val; }
    free(kv);
    int64_t nt = (int64_t)tiles_x * tiles_y;
    for (int64_t t = 0; t < 2 * nt; ++t) ranges[t] = 0;
    for (int64_t k = 0; k < p; ++k) {
        int64_t t = (int64_t)(keys[k] >> 32);
        if (k == 0 || (int64_t)(keys[k - 1] >> 32) != t) ranges[2 * t] = k;
        if (k == p - 1 || (int64_t)(keys[k + 1] >> 32) != t) ranges[2 * t + 1] = k + 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Step 3: the RaRa decay weight for one pixel ray and one Gaussian                      */
/* ------------------------------------------------------------------------------------ */

/*
 * Algorithm 1 step 2 with Eq. 4-8 and Eq. 11. e: ray origin (camera centre), d: unit ray
 * direction, mu/Rg/sig: Gaussian centre, rotation and per-axis sigma, k_sigma: the
 * ellipsoid is M = k R S, pn/pd: plane n.x + d. Returns w in [0, 1]; the t values are
 * written to tout (t1, t2, tp) when two intersections in front of the camera exist.
 */
double orc_rara_weight_full(const double *e, const double *d, const double *mu, double Rg[3][3],
                            const double *sig, double k_sigma, const double *pn, double pd,
                            double *tout, unsigned *events, double tol_disc)
{
    /* Eq. 4: ray in the unit-sphere frame, M^-1 = diag(1/(k sigma)) R^T */
    double em[3] = {e[0] - mu[0], e[1] - mu[1], e[2] - mu[2]};
    double et[3], dt[3];
    for (int a = 0; a < 3; ++a) {
        double inv = 1.0 / (k_sigma * sig[a]);
        et[a] = inv * (Rg[0][a] * em[0] + Rg[1][a] * em[1] + Rg[2][a] * em[2]);
        dt[a] = inv * (Rg[0][a] * d[0] + Rg[1][a] * d[1] + Rg[2][a] * d[2]);
    }
    /* Eq. 5-6 coefficients */
    double A = dot3(dt, dt);
    double B = 2.0 * dot3(et, dt);
    double C = dot3(et, et) - 1.0;
    double disc = B * B - 4.0 * A * C;
    if (tout) { tout[0] = tout[1] = tout[2] = NAN; }
    if (events && fabs(disc) <= tol_disc * 4.0 * A) {
        /* A grazing ray is a discontinuity of w only when the tangent point is on the
         * invisible side (w jumps between ~0 and the miss value 1). */
        double tm = -B / (2.0 * A);
        double xm[3] = {e[0] + tm * d[0], e[1] + tm * d[1], e[2] + tm * d[2]};
        if (dot3(pn, xm) + pd <= 1e-6) *events |= EV_DISC;
    }
    if (disc <= 0.0) return 1.0;            /* fewer than two intersections: keep (Eq. 11) */
    /* Eq. 7 */
    double sq = sqrt(disc);
    double t1 = (-B - sq) / (2.0 * A), t2 = (-B + sq) / (2.0 * A);
    if (events && fabs(t1) <= 1e-6 * (t2 - t1)) *events |= EV_T1;
    if (!(t1 > 0.0 && t2 > 0.0)) return 1.0; /* ellipsoid behind or around the camera */
    /* Algorithm 1: chord end points and their visibility (n.x + d >= 0 is visible) */
    double x1[3], x2[3];
    for (int a = 0; a < 3; ++a) { x1[a] = e[a] + t1 * d[a]; x2[a] = e[a] + t2 * d[a]; }
    int v1 = dot3(pn, x1) + pd >= 0.0;
    int v2 = dot3(pn, x2) + pd >= 0.0;
    /* Eq. 8 */
    double nd = dot3(pn, d);
    double tp = nd != 0.0 ? -(dot3(pn, e) + pd) / nd : NAN;
    if (tout) { tout[0] = t1; tout[1] = t2; tout[2] = tp; }
    if (v1 && v2) return 1.0;               /* whole chord visible */
    if (!v1 && !v2) return 0.0;             /* whole chord invisible: L_vis = 0 */
    /* Eq. 11: L_vis / (L_vis + L_invis), the chord split at the plane hit t_p */
    double lvis = v1 ? (tp - t1) : (t2 - tp);
    double w = lvis / (t2 - t1);
    return fmin(1.0, fmax(0.0, w));
}

/*
 * The decay weight against a convex clip volume: the intersection of the half-spaces
 * n_k.x + d_k >= 0, k < K (planes[4k..4k+3] = n_k, d_k). The paper clips by one plane and
 * names other clipping primitives as an extension wherever a ray-primitive intersection is
 * available (Discussion, Limitations); for a convex volume Eq. 11 keeps its meaning: w is
 * the share of the chord [t1, t2] (Eq. 4-7) that lies inside the volume. Each plane is
 * linear along the ray, s_k(t) = (n_k.e + d_k) + t (n_k.d), so its visible part of the
 * chord is one interval (Eq. 8 gives its end t_p); the visible part of the chord is their
 * intersection, and w = its length / (t2 - t1). Rays that meet the ellipsoid fewer than
 * twice in front of the camera keep w = 1, as for one plane.
 */
double orc_rara_weight_volume(const double *e, const double *d, const double *mu, double Rg[3][3],
                              const double *sig, double k_sigma, const double *planes, int nplanes,
                              unsigned *events, double tol_disc)
{
    double em[3] = {e[0] - mu[0], e[1] - mu[1], e[2] - mu[2]};
    double et[3], dt[3];
    for (int a = 0; a < 3; ++a) {
        double inv = 1.0 / (k_sigma * sig[a]);
        et[a] = inv * (Rg[0][a] * em[0] + Rg[1][a] * em[1] + Rg[2][a] * em[2]);
        dt[a] = inv * (Rg[0][a] * d[0] + Rg[1][a] * d[1] + Rg[2][a] * d[2]);
    }
    double A = dot3(dt, dt);
    double B = 2.0 * dot3(et, dt);
    double C = dot3(et, et) - 1.0;
    double disc = B * B - 4.0 * A * C;
    if (events && fabs(disc) <= tol_disc * 4.0 * A) {
        /* grazing ray: w jumps between the miss value 1 and ~0 when the tangent point is
         * outside the volume (on or behind one of its planes) */
        double tm = -B / (2.0 * A);
        double xm[3] = {e[0] + tm * d[0], e[1] + tm * d[1], e[2] + tm * d[2]};
        for (int k = 0; k < nplanes; ++k)
            if (dot3(&planes[4 * k], xm) + planes[4 * k + 3] <= 1e-6) *events |= EV_DISC;
    }
    if (disc <= 0.0) return 1.0;
    double sq = sqrt(disc);
    double t1 = (-B - sq) / (2.0 * A), t2 = (-B + sq) / (2.0 * A);
    if (events && fabs(t1) <= 1e-6 * (t2 - t1)) *events |= EV_T1;
    if (!(t1 > 0.0 && t2 > 0.0)) return 1.0;
    double lo = t1, hi = t2;
    for (int k = 0; k < nplanes; ++k) {
        const double *pk = &planes[4 * k];
        double a0 = dot3(pk, e) + pk[3];  /* s_k at t = 0 */
        double b = dot3(pk, d);           /* ds_k / dt */
        if (b > 0.0) lo = fmax(lo, -a0 / b);       /* visible for t >= t_p */
        else if (b < 0.0) hi = fmin(hi, -a0 / b);  /* visible for t <= t_p */
        else if (a0 < 0.0) return 0.0;             /* parallel, chord wholly behind it */
    }
    return hi > lo ? (hi - lo) / (t2 - t1) : 0.0;
}

/* ctypes-friendly wrapper of the volume weight (quaternion (w,x,y,z), sigma). */
double orc_rara_weight_vol(const double *e, const double *d, const double *mu, const double *quat,
                           const double *sig, double k_sigma, const double *planes, int nplanes)
{
    double Rg[3][3];
    quat_to_rot(quat[0], quat[1], quat[2], quat[3], Rg);
    double dn = sqrt(dot3(d, d));
    double du[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    return orc_rara_weight_volume(e, du, mu, Rg, sig, k_sigma, planes, nplanes, NULL, 0.0);
}

/* ctypes-friendly wrapper: quaternion (w,x,y,z) and log-free sigma. */
double orc_rara_weight(const double *e, const double *d, const double *mu, const double *quat,
                       const double *sig, double k_sigma, const double *plane4, double *tout)
{
    double Rg[3][3];
    quat_to_rot(quat[0], quat[1], quat[2], quat[3], Rg);
    double dn = sqrt(dot3(d, d));
    double du[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    return orc_rara_weight_full(e, du, mu, Rg, sig, k_sigma, plane4, plane4[3], tout, NULL, 0.0);
}

/* Colour evaluation exposed for tests (coefficients for one Gaussian, [(L+1)^2 * 3]). */
void orc_sh_colour(int degree, const double *coeffs, const double *dir, double *rgb)
{
    double dn = sqrt(dot3(dir, dir));
    double du[3] = {dir[0] / dn, dir[1] / dn, dir[2] / dn};
    eval_colour(coeffs, 1, 0, degree, du, rgb);
}

/* ------------------------------------------------------------------------------------ */
/* Step 4: per-pixel compositing                                                         */
/* ------------------------------------------------------------------------------------ */

typedef struct { float depth; uint32_t idx; } cand_t;

static int cmp_cand(const void *a, const void *b)
{
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

static int f32_ulp_close(float a, float b, int ulps)
{
    int32_t ia, ib;
    memcpy(&ia, &a, 4); memcpy(&ib, &b, 4);
    int32_t dlt = ia > ib ? ia - ib : ib - ia;
    return dlt <= ulps;
}

/*
 * Render. bg[3]: background colour. Binned mode when keys/vals/ranges are non-NULL: the
 * pixel walks its tile's sorted list; brute mode otherwise: the pixel gathers every
 * rendered Gaussian and sorts by (float32(depth), index). Both apply the same per-pixel
 * rule, so they agree exactly. tol[7] = {q (relative), alpha (relative), T (relative),
 * 1 - b^2 (absolute), Gaussian threshold margin, position (pixels), depth ulps (0 = equal
 * float32 depths only, which both sides order by index)} for the event bits. Only rows [row_begin, row_end) are rendered (the others are left as
 * passed in). Outputs: image [3, H, W] planar, final_T [H, W], n_contrib [H, W]
 * (1 + list position of the last blended Gaussian in binned mode, the count of walked
 * candidates in brute mode), events [H, W].
 */
int orc_render(int64_t n, const double *means, const double *log_scales, const double *quats,
               const uint8_t *label, const uint8_t *culled, const double *depth,
               const double *mean2d, const double *conic, const double *rgb, const double *opacity,
               const double *margin_gauss,
               const double *cam16, int W, int H, const double *plane4, int nplanes, double k_sigma,
               int tile_w, int tile_h, const double *bg,
               const uint64_t *keys, const uint32_t *vals, const int64_t *ranges,
               const double *tol, int nthreads, int row_begin, int row_end,
               double *image, double *final_T, int32_t *n_contrib, uint8_t *events)
{
    cam_t cam;
    load_cam(cam16, W, H, &cam);
    const int tiles_x = (W + tile_w - 1) / tile_w;
    const double pn[3] = {plane4[0], plane4[1], plane4[2]}, pd = plane4[3];
    const int binned = keys != NULL && vals != NULL && ranges != NULL;
    const double tol_q = tol[0], tol_a = tol[1], tol_T = tol[2], tol_disc = tol[3], tol_g = tol[4];
    const double tol_pos = tol[5];
    const int tol_ulps = (int)tol[6];
    (void)keys;

    /* brute-mode candidate list, in (float32 depth, index) order for the whole frame */
    cand_t *all = NULL;
    int64_t nall = 0;
    if (!binned) {
        all = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
        if (!all) return -1;
        for (int64_t i = 0; i < n; ++i)
            if (!culled[i]) { all[nall].depth = (float)depth[i]; all[nall].idx = (uint32_t)i; ++nall; }
        qsort(all, (size_t)nall, sizeof(cand_t), cmp_cand);
    }

    /* Gaussians labelled invisible within tol_g of a threshold where the image jumps: a
     * float32 renderer may label them cutoff and blend them, so every pixel of their
     * q <= 9 footprint is flagged (they are in no tile list, so the walk below never sees
     * them). Their projection fields are filled by the preprocess. */
    int64_t *haz = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t nhaz = 0;
    if (!haz) { free(all); return -1; }
    for (int64_t i = 0; i < n; ++i)
        if (label[i] == ORC_INVISIBLE && margin_gauss[i] <= tol_g && conic[3 * i] > 0.0 && conic[3 * i + 2] > 0.0)
            haz[nhaz++] = i;

    if (row_begin < 0) row_begin = 0;
    if (row_end > H) row_end = H;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int py = row_begin; py < row_end; ++py) {
        for (int px = 0; px < W; ++px) {
            const double pxc = px + 0.5, pyc = py + 0.5;
            /* ProjectRay / CameraOrigin (Algorithm 1): ray through the pixel centre */
            double dcam[3] = {(pxc - cam.cx) / cam.fx, (pyc - cam.cy) / cam.fy, 1.0};
            double dw[3];
            for (int a = 0; a < 3; ++a) dw[a] = cam.R[0][a] * dcam[0] + cam.R[1][a] * dcam[1] + cam.R[2][a] * dcam[2];
            double dn = sqrt(dot3(dw, dw));
            for (int a = 0; a < 3; ++a) dw[a] /= dn;

            int64_t start, end;
            if (binned) {
                int64_t t = (int64_t)(py / tile_h) * tiles_x + (px / tile_w);
                start = ranges[2 * t]; end = ranges[2 * t + 1];
            } else {
                start = 0; end = nall;
            }
            double T = 1.0, C[3] = {0.0, 0.0, 0.0};
            int32_t last = 0;
            unsigned ev = 0;
            for (int64_t h = 0; h < nhaz; ++h) {
                const int64_t i = haz[h];
                double dx = pxc - mean2d[2 * i], dy = pyc - mean2d[2 * i + 1];
                double q = conic[3 * i] * dx * dx + 2.0 * conic[3 * i + 1] * dx * dy + conic[3 * i + 2] * dy * dy;
                double tq = tol_q * 9.0 + 6.0 * tol_pos * sqrt(fabs(conic[3 * i]) + fabs(conic[3 * i + 2]));
                if (q <= 9.0 + tq) ev |= EV_GAUSS;
            }
            float prev_depth = 0.0f;
            int have_prev = 0;
            for (int64_t k = start; k < end; ++k) {
                uint32_t i = binned ? vals[k] : all[k].idx;
                double dx = pxc - mean2d[2 * i], dy = pyc - mean2d[2 * i + 1];
                double q = conic[3 * i] * dx * dx + 2.0 * conic[3 * i + 1] * dx * dy + conic[3 * i + 2] * dy * dy;
                /* q near 9: relative conic error plus a position error tol_pos (pixels)
                 * amplified by the splat's inverse size, dq ~ 2 sqrt(q) |conic|^(1/2) dpos */
                double tq = tol_q * 9.0 + 6.0 * tol_pos * sqrt(fabs(conic[3 * i]) + fabs(conic[3 * i + 2]));
                if (fabs(q - 9.0) <= tq) ev |= EV_Q;
                if (q > 9.0) continue;            /* outside the 3-sigma support */
                if (margin_gauss[i] <= tol_g) ev |= EV_GAUSS;
                float fd = (float)depth[i];
                if (tol_ulps > 0 && have_prev && fd != prev_depth && f32_ulp_close(fd, prev_depth, tol_ulps))
                    ev |= EV_DEPTH;
                prev_depth = fd; have_prev = 1;
                /* Eq. 10 with the normalisation dropped */
                double a0 = opacity[i] * exp(-0.5 * q);
                double w = 1.0;
                if (label[i] == ORC_CUTOFF) {
                    double mu[3] = {means[i], means[n + i], means[2 * n + i]};
                    double sig[3] = {exp(log_scales[i]), exp(log_scales[n + i]), exp(log_scales[2 * n + i])};
                    double Rg[3][3];
                    quat_to_rot(quats[i], quats[n + i], quats[2 * n + i], quats[3 * n + i], Rg);
                    if (nplanes == 1)
                        w = orc_rara_weight_full(cam.e, dw, mu, Rg, sig, k_sigma, pn, pd, NULL, &ev, tol_disc);
                    else
                        w = orc_rara_weight_volume(cam.e, dw, mu, Rg, sig, k_sigma, plane4, nplanes, &ev,
                                                   tol_disc);
                }
                /* Eq. 12 and Algorithm 1 step 3 */
                double alpha = fmin(0.99, a0 * w);
                if (fabs(alpha - 1.0 / 255.0) <= tol_a / 255.0) ev |= EV_ALPHA;
                if (alpha < 1.0 / 255.0) continue;
                double Tn = T * (1.0 - alpha);
                if (fabs(Tn - 1e-4) <= tol_T * 1e-4) ev |= EV_T;
                if (Tn < 1e-4) break;
                /* Eq. 2 */
                for (int c = 0; c < 3; ++c) C[c] += rgb[3 * i + c] * alpha * T;
                T = Tn;
                last = (int32_t)(k - start + 1);
            }
            size_t p = (size_t)py * W + px;
            for (int c = 0; c < 3; ++c) image[(size_t)c * H * W + p] = C[c] + T * bg[c];
            final_T[p] = T;
            n_contrib[p] = last;
            events[p] = (uint8_t)ev;
        }
    }
    free(haz);
    free(all);
    return 0;
}
