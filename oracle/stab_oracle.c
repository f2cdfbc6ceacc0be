/*
 * stab_oracle.c -- plain, slow, single-threaded CPU oracle of the stabiliser's
 * per-frame hot path (arXiv 1701.03572).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product path (the CUDA
 * library under paper_1701_03572_gb300/) never does, and shares no code, header,
 * table or constant with it.
 *
 * Precision: FP64, except where a floating-point result is turned into an
 * integer decision (the corner score that orders top-K, the inlier test of the
 * robust fit, the warp's rounded output byte).  There both sides take the
 * decision in FP32 with the same IEEE operation sequence (no contraction: the
 * file is compiled with -ffp-contract=off and fused operations are written as
 * fmaf), so the decision is reproducible bit for bit.
 *
 * Every loop follows the definition in the order the paper states it; no
 * blocking, fusion or reordering.  Readings of silent or ambiguous passages are
 * stated where they are used.
 *
 * Threads: the library the tests load is built without OpenMP and runs on one
 * thread.  Loops whose iterations are independent (image rows, features) carry
 * an OpenMP pragma that takes effect only in the separate timing build
 * (-fopenmp), which the benchmark uses to time the oracle on all host cores;
 * each iteration computes exactly what it computes alone, so both builds give
 * the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int reflect101(int i, int n)
{
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * n - 2 - i;
    }
    return i;
}

static int clampi(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

/* ------------------------------------------------------------------------ */
/* Luma of interleaved RGB (the paper tracks on gray frames; it does not state
 * the conversion).  Reading: integer BT.601 weights 77/150/29 (sum 256),
 * rounded half up. */
void or_luma(const uint8_t *rgb, int w, int h, int pitch, uint8_t *out, int out_pitch)
{
#pragma omp parallel for
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            const uint8_t *p = rgb + (size_t)y * pitch + 3 * x;
            out[(size_t)y * out_pitch + x] = (uint8_t)((77 * p[0] + 150 * p[1] + 29 * p[2] + 128) >> 8);
        }
}

/* ------------------------------------------------------------------------ */
/* One REDUCE step of the Gaussian pyramid (Sec. 3.2, Burt & Adelson's
 * generating kernel with a = 0.375, i.e. w = [1 4 6 4 1] / 16 in each axis):
 *   out(x, y) = round( sum_{i,j=-2..2} w_i w_j in(2x+i, 2y+j) )
 * Readings: reflect-101 border; rounding half up ((sum + 128) >> 8 on the
 * integer sum of weights 256); output size ((w+1)/2, (h+1)/2). */
void or_pyr_down(const uint8_t *src, int w, int h, int sp, uint8_t *dst, int dp)
{
    static const int k5[5] = {1, 4, 6, 4, 1};
    int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
#pragma omp parallel for
    for (int y = 0; y < h2; ++y)
        for (int x = 0; x < w2; ++x) {
            long s = 0;
            for (int j = -2; j <= 2; ++j)
                for (int i = -2; i <= 2; ++i)
                    s += (long)k5[i + 2] * k5[j + 2] *
                         src[(size_t)reflect101(2 * y + j, h) * sp + reflect101(2 * x + i, w)];
            dst[(size_t)y * dp + x] = (uint8_t)((s + 128) >> 8);
        }
}

/* ------------------------------------------------------------------------ */
/* Shi-Tomasi structure tensor (Sec. 3.1, Eq. 2): the 2x2 matrix of summed
 * gradient products over a window; R = min(lambda1, lambda2).
 * Readings: unnormalised 3x3 Sobel gradients, unweighted 3x3 box window (the
 * text allows a rectangular window), exact integer sums. */
static int sobel_x(const uint8_t *I, int pitch, int x, int y)
{
#define P(xx, yy) ((int)I[(size_t)(yy) * pitch + (xx)])
    return (P(x + 1, y - 1) + 2 * P(x + 1, y) + P(x + 1, y + 1)) -
           (P(x - 1, y - 1) + 2 * P(x - 1, y) + P(x - 1, y + 1));
}
static int sobel_y(const uint8_t *I, int pitch, int x, int y)
{
    return (P(x - 1, y + 1) + 2 * P(x, y + 1) + P(x + 1, y + 1)) -
           (P(x - 1, y - 1) + 2 * P(x, y - 1) + P(x + 1, y - 1));
#undef P
}

/* Tensor entries a = sum gx^2, b = sum gx gy, c = sum gy^2 at pixel (x, y);
 * needs 2 <= x < w-2, 2 <= y < h-2. */
void or_structure(const uint8_t *I, int pitch, int x, int y, int32_t abc[3])
{
    int32_t a = 0, b = 0, c = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int gx = sobel_x(I, pitch, x + dx, y + dy);
            int gy = sobel_y(I, pitch, x + dx, y + dy);
            a += gx * gx;
            b += gx * gy;
            c += gy * gy;
        }
    abc[0] = a; abc[1] = b; abc[2] = c;
}

/* min eigenvalue of [[a, b], [b, c]] in the FP32 sequence both sides use for
 * ranking: lambda_min = 2 det / (tr + sqrt(disc)), with det, disc exact in
 * int64 (the cancellation-free form of (tr - sqrt(disc)) / 2). */
float or_lambda32(int32_t a, int32_t b, int32_t c)
{
    int64_t tr = (int64_t)a + c;
    if (tr == 0) return 0.0f;
    int64_t det = (int64_t)a * c - (int64_t)b * b;
    int64_t d = (int64_t)a - c;
    int64_t disc = d * d + 4 * (int64_t)b * b;
    float num = (float)(2 * det);
    float den = (float)tr + sqrtf((float)disc);
    return num / den;
}

/* Same eigenvalue in FP64 (for the pins). */
double or_lambda64(int32_t a, int32_t b, int32_t c)
{
    double tr = (double)a + c;
    if (tr == 0) return 0.0;
    double det = (double)a * c - (double)b * b;
    double d = (double)a - c;
    return 2.0 * det / (tr + sqrt(d * d + 4.0 * (double)b * b));
}

/* Response map over a rectangle (for tests): lam[(y-y0)*(x1-x0) + (x-x0)]. */
void or_response(const uint8_t *I, int pitch, int x0, int y0, int x1, int y1, float *lam32, double *lam64)
{
#pragma omp parallel for
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            int32_t t[3];
            or_structure(I, pitch, x, y, t);
            size_t o = (size_t)(y - y0) * (x1 - x0) + (x - x0);
            if (lam32) lam32[o] = or_lambda32(t[0], t[1], t[2]);
            if (lam64) lam64[o] = or_lambda64(t[0], t[1], t[2]);
        }
}

typedef struct { float lam; int32_t idx; } cand_t;

static int cand_cmp(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->lam > b->lam) return -1;
    if (a->lam < b->lam) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

/* Corner detection on the reduced region of interest (Sec. 3.1): Shi-Tomasi
 * score at every ROI pixel, 3x3 non-maximum suppression, relative quality
 * threshold, strongest K first (the paper fixes only the count).
 * Readings: ROI = [x0, x1) x [y0, y1) (its size is not stated; callers pass a
 * margin); a pixel survives if its (score, -raster index) key beats all eight
 * neighbours (neighbours outside the ROI included, so the ROI must keep 3 px
 * from the border); the threshold is q * (max ROI score) in FP32, strict;
 * order by score descending, ties by raster index ascending.
 * Returns the number of points written (<= K); *n_cand = candidates before the
 * cut; -1 on a bad ROI. */
int or_detect(const uint8_t *I, int w, int h, int pitch, int x0, int y0, int x1, int y1, float q, int K,
              float *pts, float *lam_out, int *n_cand)
{
    if (x0 < 3 || y0 < 3 || x1 > w - 3 || y1 > h - 3 || x1 <= x0 || y1 <= y0 || K < 0) return -1;
    int ew = x1 - x0 + 2, eh = y1 - y0 + 2; /* ROI plus one ring */
    float *lam = (float *)malloc(sizeof(float) * (size_t)ew * eh);
    or_response(I, pitch, x0 - 1, y0 - 1, x1 + 1, y1 + 1, lam, NULL);
#define L(xx, yy) lam[(size_t)((yy) - (y0 - 1)) * ew + ((xx) - (x0 - 1))]
    float mx = 0.0f;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x)
            if (L(x, y) > mx) mx = L(x, y);
    float thr = q * mx;
    cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (size_t)(x1 - x0) * (y1 - y0) + sizeof(cand_t));
    int n = 0;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            float v = L(x, y);
            if (!(v > thr)) continue;
            int idx = y * w + x, keep = 1;
            for (int dy = -1; dy <= 1 && keep; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy) continue;
                    float u = L(x + dx, y + dy);
                    int uidx = (y + dy) * w + (x + dx);
                    if (!(v > u || (v == u && idx < uidx))) { keep = 0; break; }
                }
            if (keep) { c[n].lam = v; c[n].idx = idx; ++n; }
        }
#undef L
    qsort(c, (size_t)n, sizeof(cand_t), cand_cmp);
    int m = n < K ? n : K;
    for (int i = 0; i < m; ++i) {
        pts[2 * i] = (float)(c[i].idx % w);
        pts[2 * i + 1] = (float)(c[i].idx / w);
        if (lam_out) lam_out[i] = c[i].lam;
    }
    if (n_cand) *n_cand = n;
    free(c);
    free(lam);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Pyramidal Lucas-Kanade (Sec. 3.2, Eq. 3-6 and the coarse-to-fine scheme of
 * Bouguet cited there), one feature.
 * Readings: gradients are central differences (I(x+1) - I(x-1)) / 2 at integer
 * pixels with replicated borders, sampled between pixels by bilinear
 * interpolation (replicated border taps); window (2r+1)^2 at integer offsets
 * around the point; lost if the window's smallest normalised G eigenvalue is
 * below min_eig at any level; stop when |eta| < eps; the result must lie in the
 * level-0 image. */
typedef struct {
    const uint8_t *img;
    int w, h, pitch;
} plane_t;

static double px_at(const plane_t *P, int x, int y)
{
    return (double)P->img[(size_t)clampi(y, 0, P->h - 1) * P->pitch + clampi(x, 0, P->w - 1)];
}
static double gx_at(const plane_t *P, int x, int y) { return 0.5 * (px_at(P, x + 1, y) - px_at(P, x - 1, y)); }
static double gy_at(const plane_t *P, int x, int y) { return 0.5 * (px_at(P, x, y + 1) - px_at(P, x, y - 1)); }

/* The I, Ix, Iy planes of one level as the tracker defines them (central
 * differences with replicated borders), FP64. */
void or_grad_planes(const uint8_t *img, int w, int h, int pitch, double *I, double *Ix, double *Iy)
{
    plane_t P = {img, w, h, pitch};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            I[(size_t)y * w + x] = px_at(&P, x, y);
            Ix[(size_t)y * w + x] = gx_at(&P, x, y);
            Iy[(size_t)y * w + x] = gy_at(&P, x, y);
        }
}

/* bilinear sample of f (one of px_at, gx_at, gy_at) at (x, y); the base is
 * clamped far outside the image, where every tap is a border replica anyway */
static double bilin(const plane_t *P, double (*f)(const plane_t *, int, int), double x, double y)
{
    double lo = -64.0, hx = P->w + 64.0, hy = P->h + 64.0;
    x = x < lo ? lo : (x > hx ? hx : x);
    y = y < lo ? lo : (y > hy ? hy : y);
    double fx = floor(x), fy = floor(y);
    double ax = x - fx, ay = y - fy;
    int x0 = (int)fx, y0 = (int)fy;
    return (1 - ax) * (1 - ay) * f(P, x0, y0) + ax * (1 - ay) * f(P, x0 + 1, y0) +
           (1 - ax) * ay * f(P, x0, y0 + 1) + ax * ay * f(P, x0 + 1, y0 + 1);
}

/* Track u from pyramid I to pyramid J.  Returns 1 if tracked. */
static int lk_one(const plane_t *I, const plane_t *J, int L, double ux, double uy, int r, int max_iters,
                  double eps, double min_eig, double *vx, double *vy, int *iters, double *lam_min)
{
    int n = (2 * r + 1) * (2 * r + 1);
    double *T = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double gx = 0.0, gy = 0.0, dx = 0.0, dy = 0.0;
    int ok = 1, it_total = 0;
    for (int l = L - 1; l >= 0 && ok; --l) {
        double px = ldexp(ux, -l), py = ldexp(uy, -l);
        double Gxx = 0, Gxy = 0, Gyy = 0;
        int k = 0;
        for (int j = -r; j <= r; ++j)
            for (int i = -r; i <= r; ++i, ++k) {
                double t = bilin(&I[l], px_at, px + i, py + j);
                double tx = bilin(&I[l], gx_at, px + i, py + j);
                double ty = bilin(&I[l], gy_at, px + i, py + j);
                T[3 * k] = t; T[3 * k + 1] = tx; T[3 * k + 2] = ty;
                Gxx += tx * tx; Gxy += tx * ty; Gyy += ty * ty;
            }
        double lam = 0.5 * ((Gxx + Gyy) - sqrt((Gxx - Gyy) * (Gxx - Gyy) + 4.0 * Gxy * Gxy));
        double D = Gxx * Gyy - Gxy * Gxy;
        if (lam_min && lam / n < lam_min[0]) { lam_min[0] = lam / n; lam_min[1] = (Gxx + Gyy) / n; }
        if (!(lam / n >= min_eig) || !(D > 0)) { ok = 0; break; }
        double nx = 0.0, ny = 0.0;
        for (int it = 0; it < max_iters; ++it) {
            double qx = px + gx + nx, qy = py + gy + ny;
            double bx = 0.0, by = 0.0;
            k = 0;
            for (int j = -r; j <= r; ++j)
                for (int i = -r; i <= r; ++i, ++k) {
                    double e = T[3 * k] - bilin(&J[l], px_at, qx + i, qy + j);
                    bx += e * T[3 * k + 1];
                    by += e * T[3 * k + 2];
                }
            double ex = (Gyy * bx - Gxy * by) / D;
            double ey = (Gxx * by - Gxy * bx) / D;
            nx += ex; ny += ey;
            ++it_total;
            if (ex * ex + ey * ey < eps * eps) break;
        }
        if (l > 0) { gx = 2.0 * (gx + nx); gy = 2.0 * (gy + ny); }
        else { dx = gx + nx; dy = gy + ny; }
    }
    free(T);
    *vx = ux + dx; *vy = uy + dy;
    if (iters) *iters += it_total;
    if (!ok) return 0;
    return (*vx >= 0.0 && *vx <= I[0].w - 1 && *vy >= 0.0 && *vy <= I[0].h - 1);
}

/* Forward tracking plus forward-backward weeding (Sec. 4.1: flow consistency
 * in the backward direction).  Pyramids are given level by level (pointer,
 * width, height, pitch).  Reading: the backward pass starts from the forward
 * result with a zero guess; a pair is kept when both passes track and the
 * round trip ends within fb_thresh of the start.
 * Outputs (n each): fwd xy (2n), back xy (2n), fb error, status (1 kept),
 * status of the forward pass alone, and (when lam_min is not NULL, 2n) the
 * smallest normalised eigenvalue lambda_min(G) / (2r+1)^2 met at any level of
 * either pass -- the quantity the loss test compares with min_eig -- with the
 * normalised trace of that G, reported so that a caller can tell a decision
 * taken close to that threshold and how finely the eigenvalue is resolved.
 * Returns the number kept. */
int or_track(const uint8_t *const *pyrI, const uint8_t *const *pyrJ, const int *lw, const int *lh,
             const int *lp, int L, const float *pts, int n, int r, int max_iters, double eps, double min_eig,
             double fb_thresh, double *fwd, double *back, double *fb_err, uint8_t *status, uint8_t *status_fwd,
             int *iters, double *lam_min)
{
    plane_t I[16], J[16];
    if (L < 1 || L > 16) return -1;
    for (int l = 0; l < L; ++l) {
        I[l].img = pyrI[l]; J[l].img = pyrJ[l];
        I[l].w = J[l].w = lw[l]; I[l].h = J[l].h = lh[l]; I[l].pitch = J[l].pitch = lp[l];
    }
    int kept = 0;
    if (iters) *iters = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : kept)
    for (int k = 0; k < n; ++k) {
        double ux = pts[2 * k], uy = pts[2 * k + 1], vx, vy, bx, by;
        double *lm = lam_min ? &lam_min[2 * k] : NULL;
        int itk = 0;
        if (lm) { lm[0] = HUGE_VAL; lm[1] = 0.0; }
        int s1 = lk_one(I, J, L, ux, uy, r, max_iters, eps, min_eig, &vx, &vy, &itk, lm);
        int s2 = s1 ? lk_one(J, I, L, vx, vy, r, max_iters, eps, min_eig, &bx, &by, &itk, lm) : 0;
        if (iters) {
#pragma omp atomic
            *iters += itk;
        }
        if (!s1) { bx = ux; by = uy; }
        double e = sqrt((bx - ux) * (bx - ux) + (by - uy) * (by - uy));
        fwd[2 * k] = vx; fwd[2 * k + 1] = vy;
        back[2 * k] = bx; back[2 * k + 1] = by;
        fb_err[k] = s2 ? e : -1.0;
        status_fwd[k] = (uint8_t)s1;
        status[k] = (uint8_t)(s1 && s2 && e <= fb_thresh);
        kept += status[k];
    }
    return kept;
}

/* ------------------------------------------------------------------------ */
/* Counter-based generator for the fit's samples: SplitMix64 (Steele, Lea and
 * Flood, OOPSLA 2014; the 64-bit finaliser published with it), used as a hash
 * of a counter: value(x) = the first output of a SplitMix64 generator whose
 * state is x. */
uint64_t or_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Sample pair of hypothesis h (of frame t) among n points: i = r0 mod n,
 * j = r1 mod (n-1), skipping i. */
void or_sample_pair(uint64_t seed, int t, int h, int n, int *i, int *j)
{
    uint64_t base = seed ^ ((uint64_t)(uint32_t)t << 32) ^ ((uint64_t)(uint32_t)h << 8);
    uint64_t r0 = or_splitmix64(base ^ 0ULL), r1 = or_splitmix64(base ^ 1ULL);
    int a = (int)(r0 % (uint64_t)n);
    int b = (int)(r1 % (uint64_t)(n - 1));
    if (b >= a) b += 1;
    *i = a; *j = b;
}

/* Two-point model (Sec. 4: similarity = rotation, scale, translation; rigid
 * = similarity with scale 1) through points (si, di), (sj, dj) in centred
 * coordinates, in the FP32 operation order both sides use.  Returns 0 when the
 * sample is degenerate (|sj - si| < 1 px). Model: d = [a -b; b a] s + t. */
static int two_point(const float *si, const float *sj, const float *di, const float *dj, int rigid, float m[4])
{
    float vsx = sj[0] - si[0], vsy = sj[1] - si[1];
    float vdx = dj[0] - di[0], vdy = dj[1] - di[1];
    float nn = fmaf(vsx, vsx, vsy * vsy);
    if (!(nn >= 1.0f)) return 0;
    float dot = fmaf(vsx, vdx, vsy * vdy);
    float crs = fmaf(vsx, vdy, -(vsy * vdx));
    float a, b;
    if (rigid) {
        float r = sqrtf(fmaf(dot, dot, crs * crs));
        if (!(r > 0.0f)) return 0;
        a = dot / r; b = crs / r;
    } else {
        a = dot / nn; b = crs / nn;
    }
    float msx = 0.5f * (si[0] + sj[0]), msy = 0.5f * (si[1] + sj[1]);
    float mdx = 0.5f * (di[0] + dj[0]), mdy = 0.5f * (di[1] + dj[1]);
    m[0] = a; m[1] = b;
    m[2] = mdx - fmaf(a, msx, -(b * msy));
    m[3] = mdy - fmaf(b, msx, a * msy);
    return 1;
}

static int is_inlier(const float m[4], const float *s, const float *d, float tau2)
{
    float px = fmaf(m[0], s[0], fmaf(-m[1], s[1], m[2]));
    float py = fmaf(m[1], s[0], fmaf(m[0], s[1], m[3]));
    float ex = d[0] - px, ey = d[1] - py;
    return fmaf(ex, ex, ey * ey) < tau2;
}

/* Robust rigid / similarity fit (Sec. 4 and 4.1, Eq. 7 restricted to the 3-
 * and 4-degree-of-freedom models).  src, dst: n points in pixel coordinates
 * (FP32, the precision the tracker returns).  Readings: the paper does not say
 * how outliers surviving the backward check are handled; H hypotheses from
 * two-point samples are scored by their inlier count (strict residual < tau
 * px, FP32), the first best wins, and Eq. 7 is solved in closed form on its
 * inliers (FP64): with centred sums A = sum x.y, B = sum x cross y,
 * theta = atan2(B, A), s = sqrt(A^2 + B^2) / sum |x|^2 (1 for rigid),
 * t = mean(dst) - s R mean(src).  Coordinates are centred on the image centre.
 * out = (tx, ty, theta, log s).  flags bit 0 = skipped (fewer than min_pts
 * pairs or no valid hypothesis: identity, Sec. 4.1 "stabilization is skipped").
 * Returns the inlier count of the refit set. */
int or_fit(const float *src, const float *dst, int n, int w, int h, int rigid, int H, uint64_t seed, int t,
           float tau, int min_pts, double out[4], int *best_h, double *rms, uint8_t *inlier_mask, int *flags)
{
    float cx = 0.5f * (float)(w - 1), cy = 0.5f * (float)(h - 1);
    out[0] = out[1] = out[2] = out[3] = 0.0;
    *best_h = -1; *rms = 0.0; *flags = 0;
    if (inlier_mask) memset(inlier_mask, 0, (size_t)(n > 0 ? n : 0));
    int need = min_pts > 2 ? min_pts : 2;
    if (n < need) { *flags = 1; return 0; }
    float *s = (float *)malloc(sizeof(float) * 4 * (size_t)n), *d = s + 2 * n;
    for (int k = 0; k < n; ++k) {
        s[2 * k] = src[2 * k] - cx; s[2 * k + 1] = src[2 * k + 1] - cy;
        d[2 * k] = dst[2 * k] - cx; d[2 * k + 1] = dst[2 * k + 1] - cy;
    }
    float tau2 = tau * tau;
    int best = -1, best_score = -1;
    float bm[4] = {0, 0, 0, 0};
    for (int hh = 0; hh < H; ++hh) {
        int i, j;
        float m[4];
        or_sample_pair(seed, t, hh, n, &i, &j);
        if (!two_point(&s[2 * i], &s[2 * j], &d[2 * i], &d[2 * j], rigid, m)) continue;
        int score = 0;
        for (int k = 0; k < n; ++k) score += is_inlier(m, &s[2 * k], &d[2 * k], tau2);
        if (score > best_score) { best_score = score; best = hh; memcpy(bm, m, sizeof(bm)); }
    }
    if (best < 0 || best_score < 2) { free(s); *flags = 1; return 0; }
    *best_h = best;
    double mus[2] = {0, 0}, mud[2] = {0, 0};
    int ni = 0;
    for (int k = 0; k < n; ++k)
        if (is_inlier(bm, &s[2 * k], &d[2 * k], tau2)) {
            if (inlier_mask) inlier_mask[k] = 1;
            mus[0] += s[2 * k]; mus[1] += s[2 * k + 1];
            mud[0] += d[2 * k]; mud[1] += d[2 * k + 1];
            ++ni;
        }
    mus[0] /= ni; mus[1] /= ni; mud[0] /= ni; mud[1] /= ni;
    double A = 0, B = 0, Sxx = 0;
    for (int k = 0; k < n; ++k)
        if (is_inlier(bm, &s[2 * k], &d[2 * k], tau2)) {
            double x0 = s[2 * k] - mus[0], x1 = s[2 * k + 1] - mus[1];
            double y0 = d[2 * k] - mud[0], y1 = d[2 * k + 1] - mud[1];
            A += x0 * y0 + x1 * y1;
            B += x0 * y1 - x1 * y0;
            Sxx += x0 * x0 + x1 * x1;
        }
    if (!(Sxx > 0.0)) { free(s); *flags = 1; *best_h = -1; if (inlier_mask) memset(inlier_mask, 0, (size_t)n); return 0; }
    double th = atan2(B, A);
    double sc = rigid ? 1.0 : sqrt(A * A + B * B) / Sxx;
    double c = cos(th), sn = sin(th);
    double tx = mud[0] - sc * (c * mus[0] - sn * mus[1]);
    double ty = mud[1] - sc * (sn * mus[0] + c * mus[1]);
    double e2 = 0;
    for (int k = 0; k < n; ++k)
        if (is_inlier(bm, &s[2 * k], &d[2 * k], tau2)) {
            double px = sc * (c * s[2 * k] - sn * s[2 * k + 1]) + tx;
            double py = sc * (sn * s[2 * k] + c * s[2 * k + 1]) + ty;
            e2 += (d[2 * k] - px) * (d[2 * k] - px) + (d[2 * k + 1] - py) * (d[2 * k + 1] - py);
        }
    *rms = sqrt(e2 / ni);
    out[0] = tx; out[1] = ty; out[2] = th; out[3] = log(sc);
    free(s);
    return ni;
}

/* ------------------------------------------------------------------------ */
/* Full 6-degree-of-freedom affine model of Eq. 7-8: d = A s + t with a 2x2
 * matrix A, fitted like the 3/4-DOF models (hypotheses from minimal samples,
 * inlier count, closed-form least squares on the winner's inliers).  Eq. 8
 * needs three non-degenerate pairs for the six unknowns.
 *
 * Sample triple of hypothesis h: i and j as for the pair, k = r2 mod (n-2)
 * stepped past the smaller and then the larger of i, j (uniform over the
 * remaining points). */
void or_sample_triple(uint64_t seed, int t, int h, int n, int *i, int *j, int *k)
{
    uint64_t base = seed ^ ((uint64_t)(uint32_t)t << 32) ^ ((uint64_t)(uint32_t)h << 8);
    uint64_t r2 = or_splitmix64(base ^ 2ULL);
    or_sample_pair(seed, t, h, n, i, j);
    int lo = *i < *j ? *i : *j, hi = *i < *j ? *j : *i;
    int c = (int)(r2 % (uint64_t)(n - 2));
    if (c >= lo) c += 1;
    if (c >= hi) c += 1;
    *k = c;
}

/* Exact affine map through three pairs (centred coordinates) in the FP32
 * operation order both sides use: with u1 = sj - si, u2 = sk - si,
 * v1 = dj - di, v2 = dk - di, A [u1 u2] = [v1 v2], so A = [v1 v2] adj / det
 * (det = u1 x u2) and t = di - A si.  Degenerate when |det| < 1 px^2 (twice the
 * triangle's area).  m = (a00, a01, a10, a11, tx, ty). */
static int three_point(const float *si, const float *sj, const float *sk, const float *di, const float *dj,
                       const float *dk, float m[6])
{
    float u1x = sj[0] - si[0], u1y = sj[1] - si[1], u2x = sk[0] - si[0], u2y = sk[1] - si[1];
    float v1x = dj[0] - di[0], v1y = dj[1] - di[1], v2x = dk[0] - di[0], v2y = dk[1] - di[1];
    float det = fmaf(u1x, u2y, -(u1y * u2x));
    if (!(fabsf(det) >= 1.0f)) return 0;
    m[0] = fmaf(v1x, u2y, -(v2x * u1y)) / det;
    m[1] = fmaf(v2x, u1x, -(v1x * u2x)) / det;
    m[2] = fmaf(v1y, u2y, -(v2y * u1y)) / det;
    m[3] = fmaf(v2y, u1x, -(v1y * u2x)) / det;
    m[4] = di[0] - fmaf(m[0], si[0], m[1] * si[1]);
    m[5] = di[1] - fmaf(m[2], si[0], m[3] * si[1]);
    return 1;
}

static int is_inlier_affine(const float m[6], const float *s, const float *d, float tau2)
{
    float px = fmaf(m[0], s[0], fmaf(m[1], s[1], m[4]));
    float py = fmaf(m[2], s[0], fmaf(m[3], s[1], m[5]));
    float ex = d[0] - px, ey = d[1] - py;
    return fmaf(ex, ex, ey * ey) < tau2;
}

/* Robust affine fit.  Arguments as or_fit; out = (a00, a01, a10, a11, tx, ty)
 * in centred coordinates.  Least squares of Eq. 7 on the inliers (FP64): with
 * centred x = s - mean(s), y = d - mean(d), Sxx = sum x x^T, Syx = sum y x^T,
 * A = Syx Sxx^-1 and t = mean(d) - A mean(s); skipped when Sxx is singular. */
int or_fit_affine(const float *src, const float *dst, int n, int w, int h, int H, uint64_t seed, int t, float tau,
                  int min_pts, double out[6], int *best_h, double *rms, uint8_t *inlier_mask, int *flags)
{
    float cx = 0.5f * (float)(w - 1), cy = 0.5f * (float)(h - 1);
    for (int k = 0; k < 6; ++k) out[k] = 0.0;
    out[0] = out[3] = 1.0;
    *best_h = -1; *rms = 0.0; *flags = 0;
    if (inlier_mask) memset(inlier_mask, 0, (size_t)(n > 0 ? n : 0));
    int need = min_pts > 3 ? min_pts : 3;
    if (n < need) { *flags = 1; return 0; }
    float *s = (float *)malloc(sizeof(float) * 4 * (size_t)n), *d = s + 2 * n;
    for (int k = 0; k < n; ++k) {
        s[2 * k] = src[2 * k] - cx; s[2 * k + 1] = src[2 * k + 1] - cy;
        d[2 * k] = dst[2 * k] - cx; d[2 * k + 1] = dst[2 * k + 1] - cy;
    }
    float tau2 = tau * tau;
    int best = -1, best_score = -1;
    float bm[6] = {0, 0, 0, 0, 0, 0};
    for (int hh = 0; hh < H; ++hh) {
        int i, j, kk;
        float m[6];
        or_sample_triple(seed, t, hh, n, &i, &j, &kk);
        if (!three_point(&s[2 * i], &s[2 * j], &s[2 * kk], &d[2 * i], &d[2 * j], &d[2 * kk], m)) continue;
        int score = 0;
        for (int k = 0; k < n; ++k) score += is_inlier_affine(m, &s[2 * k], &d[2 * k], tau2);
        if (score > best_score) { best_score = score; best = hh; memcpy(bm, m, sizeof(bm)); }
    }
    if (best < 0 || best_score < 3) { free(s); *flags = 1; return 0; }
    *best_h = best;
    double mus[2] = {0, 0}, mud[2] = {0, 0};
    int ni = 0;
    for (int k = 0; k < n; ++k)
        if (is_inlier_affine(bm, &s[2 * k], &d[2 * k], tau2)) {
            if (inlier_mask) inlier_mask[k] = 1;
            mus[0] += s[2 * k]; mus[1] += s[2 * k + 1];
            mud[0] += d[2 * k]; mud[1] += d[2 * k + 1];
            ++ni;
        }
    mus[0] /= ni; mus[1] /= ni; mud[0] /= ni; mud[1] /= ni;
    double Sxx[2][2] = {{0, 0}, {0, 0}}, Syx[2][2] = {{0, 0}, {0, 0}};
    for (int k = 0; k < n; ++k)
        if (is_inlier_affine(bm, &s[2 * k], &d[2 * k], tau2)) {
            double x[2] = {s[2 * k] - mus[0], s[2 * k + 1] - mus[1]};
            double y[2] = {d[2 * k] - mud[0], d[2 * k + 1] - mud[1]};
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) {
                    Sxx[r][c] += x[r] * x[c];
                    Syx[r][c] += y[r] * x[c];
                }
        }
    double D = Sxx[0][0] * Sxx[1][1] - Sxx[0][1] * Sxx[1][0];
    if (!(D > 0.0)) {
        free(s); *flags = 1; *best_h = -1;
        if (inlier_mask) memset(inlier_mask, 0, (size_t)n);
        for (int k = 0; k < 6; ++k) out[k] = 0.0;
        out[0] = out[3] = 1.0;
        return 0;
    }
    double inv[2][2] = {{Sxx[1][1] / D, -Sxx[0][1] / D}, {-Sxx[1][0] / D, Sxx[0][0] / D}};
    double A[2][2];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) A[r][c] = Syx[r][0] * inv[0][c] + Syx[r][1] * inv[1][c];
    double tx = mud[0] - (A[0][0] * mus[0] + A[0][1] * mus[1]);
    double ty = mud[1] - (A[1][0] * mus[0] + A[1][1] * mus[1]);
    double e2 = 0;
    for (int k = 0; k < n; ++k)
        if (is_inlier_affine(bm, &s[2 * k], &d[2 * k], tau2)) {
            double px = A[0][0] * s[2 * k] + A[0][1] * s[2 * k + 1] + tx;
            double py = A[1][0] * s[2 * k] + A[1][1] * s[2 * k + 1] + ty;
            e2 += (d[2 * k] - px) * (d[2 * k] - px) + (d[2 * k + 1] - py) * (d[2 * k + 1] - py);
        }
    *rms = sqrt(e2 / ni);
    out[0] = A[0][0]; out[1] = A[0][1]; out[2] = A[1][0]; out[3] = A[1][1]; out[4] = tx; out[5] = ty;
    free(s);
    return ni;
}

/* Closed-form least squares of Eq. 7 restricted to a similarity or rigid
 * model, on all n given pairs (centred coordinates; FP64).  Used for pins. */
void or_ls_similarity(const double *src, const double *dst, int n, int rigid, double out[4])
{
    double mus[2] = {0, 0}, mud[2] = {0, 0};
    for (int k = 0; k < n; ++k) {
        mus[0] += src[2 * k]; mus[1] += src[2 * k + 1];
        mud[0] += dst[2 * k]; mud[1] += dst[2 * k + 1];
    }
    mus[0] /= n; mus[1] /= n; mud[0] /= n; mud[1] /= n;
    double A = 0, B = 0, Sxx = 0;
    for (int k = 0; k < n; ++k) {
        double x0 = src[2 * k] - mus[0], x1 = src[2 * k + 1] - mus[1];
        double y0 = dst[2 * k] - mud[0], y1 = dst[2 * k + 1] - mud[1];
        A += x0 * y0 + x1 * y1;
        B += x0 * y1 - x1 * y0;
        Sxx += x0 * x0 + x1 * x1;
    }
    double th = atan2(B, A);
    double sc = rigid ? 1.0 : sqrt(A * A + B * B) / Sxx;
    double c = cos(th), sn = sin(th);
    out[0] = mud[0] - sc * (c * mus[0] - sn * mus[1]);
    out[1] = mud[1] - sc * (sn * mus[0] + c * mus[1]);
    out[2] = th;
    out[3] = log(sc);
}

/* ------------------------------------------------------------------------ */
/* Averaging-window smoothing (Sec. 5.1): accumulate the per-frame parameters
 * into a trajectory C, average C over a window of W frames, and correct each
 * frame's parameters by the difference: m'_t = m_t + (S_t - C_t).
 * Readings: m (T x 4) with m_0 = 0 (frame 0 has no predecessor);
 * C_t = sum_{k<=t} m_k; S_t = mean of C_k for k in
 * [t - floor((W-1)/2), t + ceil((W-1)/2)] clipped to [0, T-1]; parameters are
 * averaged component-wise (theta and log s additively). */
void or_smooth(const double *m, int T, int W, double *C, double *S, double *mp)
{
    for (int t = 0; t < T; ++t)
        for (int c = 0; c < 4; ++c) C[4 * t + c] = (t ? C[4 * (t - 1) + c] : 0.0) + m[4 * t + c];
    int before = (W - 1) / 2, after = W / 2;
    for (int t = 0; t < T; ++t) {
        int lo = t - before < 0 ? 0 : t - before;
        int hi = t + after > T - 1 ? T - 1 : t + after;
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int k = lo; k <= hi; ++k) acc += C[4 * k + c];
            S[4 * t + c] = acc / (hi - lo + 1);
            mp[4 * t + c] = m[4 * t + c] + (S[4 * t + c] - C[4 * t + c]);
        }
    }
}

/* Inverse mapping of the compensating warp for parameters m (Sec. 5.1: the
 * frame is warped by the corrected similarity; the output pixel p takes the
 * source at M(m)^-1 p).  In pixel coordinates with c the image centre:
 * q = c + (1/s) R(-theta) (p - c - t).
 *
 * Composition crop (Sec. 5.1, last paragraph: the warped frame is cropped and
 * resized to hide the unfilled border; the paper fixes no amount): a zoom z
 * about the centre, so output pixel p shows the compensated frame at
 * c + (p - c) / z.  The two maps are composed here as 3x3 matrices in FP64,
 * Minv = W Z^-1 with W the warp inverse above and Z^-1 the zoom's inverse;
 * z = 1 leaves W unchanged.  Minv = [a00 a01 b0 a10 a11 b1] (FP32). */
void or_warp_inverse(const double m[4], int w, int h, double zoom, float Minv[6])
{
    double cx = 0.5 * (w - 1), cy = 0.5 * (h - 1);
    double is = exp(-m[3]), c = cos(m[2]), sn = sin(m[2]);
    double a00 = is * c, a01 = is * sn, a10 = -is * sn, a11 = is * c;
    double ux = cx + m[0], uy = cy + m[1];
    double W[3][3] = {{a00, a01, cx - (a00 * ux + a01 * uy)}, {a10, a11, cy - (a10 * ux + a11 * uy)}, {0, 0, 1}};
    double iz = 1.0 / zoom;
    double Zi[3][3] = {{iz, 0, cx - iz * cx}, {0, iz, cy - iz * cy}, {0, 0, 1}};
    double P[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            P[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) P[i][j] += W[i][k] * Zi[k][j];
        }
    Minv[0] = (float)P[0][0]; Minv[1] = (float)P[0][1]; Minv[2] = (float)P[0][2];
    Minv[3] = (float)P[1][0]; Minv[4] = (float)P[1][1]; Minv[5] = (float)P[1][2];
}

/* Compensating bilinear warp (Sec. 5.1, final step).  out(p) = bilinear(src,
 * Minv p), taps outside the image read 0, rounded half up and clamped; C
 * interleaved channels.  The output byte is a quantised decision, so the FP32
 * operation order is fixed: q = fma(a0, x, fma(a1, y, a2)); v = two lerps in x
 * then one in y, each fma(f, hi - lo, lo). */
void or_warp(const uint8_t *src, int w, int h, int C, int sp, const float M[6], uint8_t *dst, int dp)
{
#pragma omp parallel for
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            float xf = (float)x, yf = (float)y;
            float qx = fmaf(M[0], xf, fmaf(M[1], yf, M[2]));
            float qy = fmaf(M[3], xf, fmaf(M[4], yf, M[5]));
            int inside = (qx > -1.0f && qx < (float)w && qy > -1.0f && qy < (float)h);
            float fx0 = 0, fy0 = 0, ax = 0, ay = 0;
            int x0 = 0, y0 = 0;
            if (inside) {
                fx0 = floorf(qx); fy0 = floorf(qy);
                ax = qx - fx0; ay = qy - fy0;
                x0 = (int)fx0; y0 = (int)fy0;
            }
            for (int c = 0; c < C; ++c) {
                uint8_t o = 0;
                if (inside) {
#define TAP(xx, yy) (((xx) >= 0 && (xx) < w && (yy) >= 0 && (yy) < h) ? (float)src[(size_t)(yy) * sp + (size_t)(xx) * C + c] : 0.0f)
                    float p00 = TAP(x0, y0), p01 = TAP(x0 + 1, y0), p10 = TAP(x0, y0 + 1), p11 = TAP(x0 + 1, y0 + 1);
#undef TAP
                    float top = fmaf(ax, p01 - p00, p00);
                    float bot = fmaf(ax, p11 - p10, p10);
                    float v = fmaf(ay, bot - top, top);
                    float r = floorf(v + 0.5f);
                    o = (uint8_t)(r < 0.0f ? 0 : (r > 255.0f ? 255 : (int)r));
                }
                dst[(size_t)y * dp + (size_t)x * C + c] = o;
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Photometric Charbonnier objective of the warp and its adjoint (direct
 * refinement of the similarity by Gauss-Newton; the model is the one of
 * Sec. 4, the warp the one of Sec. 5.1):
 *   L(theta) = sum_{p in Omega} sqrt(r_p^2 + eps^2),  r_p = I_t(W(p)) - I_prev(p),
 *   W(p) = c + s R(th) (p - c) + (tx, ty),  theta = (tx, ty, th, log s).
 * I_t is read by bilinear interpolation with zero outside; Omega is the inner
 * rectangle [margin, w - margin) x [margin, h - margin).  Outputs (each may be
 * NULL): dtheta (4), dIt (w*h, d L / d I_t), dIp (w*h), the IRLS Gauss-Newton
 * system Hm (4x4) and g (4): weights 1/sqrt(r^2 + eps^2), H = sum w J^T J,
 * g = sum w J^T r.  Returns L. */
double or_charb(const float *It, const float *Ip, int w, int h, int margin, const double th[4], double eps,
                double *dtheta, double *dIt, double *dIp, double *Hm, double *g)
{
    double cx = 0.5 * (w - 1), cy = 0.5 * (h - 1);
    double s = exp(th[3]), c = cos(th[2]), sn = sin(th[2]);
    double L = 0;
    if (dtheta) memset(dtheta, 0, 4 * sizeof(double));
    if (dIt) memset(dIt, 0, sizeof(double) * (size_t)w * h);
    if (dIp) memset(dIp, 0, sizeof(double) * (size_t)w * h);
    if (Hm) memset(Hm, 0, 16 * sizeof(double));
    if (g) memset(g, 0, 4 * sizeof(double));
    for (int y = margin; y < h - margin; ++y)
        for (int x = margin; x < w - margin; ++x) {
            double dx = x - cx, dy = y - cy;
            double rx = c * dx - sn * dy, ry = sn * dx + c * dy; /* R d */
            double Wx = cx + s * rx + th[0], Wy = cy + s * ry + th[1];
            double fx = floor(Wx), fy = floor(Wy);
            double ax = Wx - fx, ay = Wy - fy;
            int x0 = (int)fx, y0 = (int)fy;
#define TAPF(xx, yy) (((xx) >= 0 && (xx) < w && (yy) >= 0 && (yy) < h) ? (double)It[(size_t)(yy) * w + (xx)] : 0.0)
            double p00 = TAPF(x0, y0), p01 = TAPF(x0 + 1, y0), p10 = TAPF(x0, y0 + 1), p11 = TAPF(x0 + 1, y0 + 1);
#undef TAPF
            double v = (1 - ax) * (1 - ay) * p00 + ax * (1 - ay) * p01 + (1 - ax) * ay * p10 + ax * ay * p11;
            double gxv = (1 - ay) * (p01 - p00) + ay * (p11 - p10);
            double gyv = (1 - ax) * (p10 - p00) + ax * (p11 - p01);
            double r = v - (double)Ip[(size_t)y * w + x];
            double rho = sqrt(r * r + eps * eps);
            L += rho;
            double psi = r / rho;
            /* dW/dtheta: tx -> (1,0); ty -> (0,1); th -> s R' d = s(-ry, rx); log s -> s R d */
            double J[4] = {gxv, gyv, s * (-ry * gxv + rx * gyv), s * (rx * gxv + ry * gyv)};
            if (dtheta)
                for (int a = 0; a < 4; ++a) dtheta[a] += psi * J[a];
            if (dIt) {
                double wt[4] = {(1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay};
                int tx_[4] = {x0, x0 + 1, x0, x0 + 1}, ty_[4] = {y0, y0, y0 + 1, y0 + 1};
                for (int q = 0; q < 4; ++q)
                    if (tx_[q] >= 0 && tx_[q] < w && ty_[q] >= 0 && ty_[q] < h)
                        dIt[(size_t)ty_[q] * w + tx_[q]] += psi * wt[q];
            }
            if (dIp) dIp[(size_t)y * w + x] -= psi;
            if (Hm || g) {
                double wgt = 1.0 / rho;
                for (int a = 0; a < 4; ++a) {
                    if (g) g[a] += wgt * J[a] * r;
                    if (Hm)
                        for (int b = 0; b < 4; ++b) Hm[4 * a + b] += wgt * J[a] * J[b];
                }
            }
        }
    return L;
}
