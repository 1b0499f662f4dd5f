/*
 * gf_oracle.c -- plain FP64 CPU oracle for the Fast Guided Filter
 * (K. He and J. Sun, "Fast Guided Filter", arXiv:1505.00996, 2015).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load this library.  The GPU library never links, includes or calls it, and the two
 * share no code: no headers, no helpers, no tables.
 *
 * What it computes, in double precision, one step at a time and in the paper's order:
 *   - Algorithm 2 (fast guided filter): subsample I and p by s, box statistics at radius r', variance and
 *     covariance, the coefficients a and b of Eq. (2)-(3), box means of a and b, bilinear upsampling of
 *     those means, and the output q = mean_a .* I + mean_b of Eq. (4) on the full-resolution guidance.
 *   - Algorithm 1 (guided filter), coded separately with its own box filter (a summed-area table), so that
 *     "Algorithm 2 with s = 1 equals Algorithm 1" is a check between two codings.
 *   - The adjoint (backward pass) of Algorithm 2, written operator by operator as scatters of the forward
 *     maps (the paper has no backward pass; it is the exact derivative of the forward above).
 *   - The detail-enhancement application of the paper's Fig. 2: q + k (I - q), the guide's detail layer
 *     I - q amplified by k over the filtered base layer q.
 *
 * Readings of points the paper leaves open (each is a parameter of the tests):
 *   R1 box mean: f_mean(x, r)_k = (1/|w_k n Omega|) * sum of x over the window w_k of radius r clipped to
 *      the image (border windows are normalised by their in-image pixel count).
 *   R2 nearest subsample: low-res (j, i) takes full-res (floor((j + 1/2) s), floor((i + 1/2) s)), clamped
 *      to the last row / column.
 *   R3 bilinear subsample: half-pixel centres, no antialiasing: source y = (j + 1/2) s - 1/2 clamped to
 *      [0, H - 1], bilinear between floor(y) and floor(y) + 1 (clamped), likewise x.
 *   R4 box subsample (not in the paper; used by the trainable-layer workload): mean of the s x s block,
 *      clipped to the image.
 *   R5 low-res size: h = ceil(H / s), w = ceil(W / s); coordinates use the ratio s exactly.
 *   R6 low-res radius r' = r / s rounded half up, raised to 1 when r >= 1 (s = 1 gives r' = r); a caller
 *      may pass r' explicitly.
 *   R7 bilinear upsample: full-res (Y, X) samples the low-res map at ((Y + 1/2)/s - 1/2, (X + 1/2)/s - 1/2),
 *      each coordinate clamped to [0, h - 1] / [0, w - 1].
 *   R8 channels: the guide has CI = 1 channel shared by all C channels of p, or CI = C channels with
 *      channel c guiding channel c; each channel of p is filtered independently.
 *   R9 eps is added to var(I) as given (no rescaling); R10 q is not clamped.
 *   R12 colour guide (the guided filter's colour form, which the paper cites but does not restate): with a
 *      3-channel guide the model in each window is q = a^T I + b with a 3-vector a, a = (Sigma + eps U)^-1
 *      cov_Ip and b = mean_p - a^T mean_I, Sigma being the 3 x 3 covariance of the guide in the window and
 *      cov_Ip the covariance of each guide channel with p; Algorithm 2's subsample and upsample steps wrap it
 *      unchanged, and q = mean_a^T I + mean_b on the full-resolution guide.
 *   R13 a non-integer ratio s (a rational sn / sd > 1, e.g. 5/2): the same coordinate maps R2, R3, R5-R7, R11
 *      with that s, evaluated exactly as ratios of integers; the box subsample needs an integer s.
 *   R11 antialiased bilinear subsample (a fourth mode; the paper names only "bilinear", and this is the
 *      form a shrinking resize takes when it low-passes first): a triangle filter of half-width s centred
 *      on the low-res pixel centre, so source pixel x has weight max(0, 1 - |x + 1/2 - (i + 1/2) s| / s)
 *      along each axis; taps outside the image are dropped and the remaining weights renormalised.
 *
 * Layout: all images are dense row-major planes; a batch is N x channels x rows x cols.
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -o libgforacle.so gf_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { GFO_SUB_NEAREST = 0, GFO_SUB_BILINEAR = 1, GFO_SUB_BOX = 2, GFO_SUB_BILINEAR_AA = 3 };

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }
static int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static double dclamp(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* The ratio s is a rational sn / sd (sd = 1 for the integer ratios of Algorithm 2; R13 reads a non-integer
 * ratio the same way), so every coordinate below is a ratio of integers and every floor, clamp and weight
 * is decided exactly. */

/* R6: r' from r and s (Algorithm 2 sets r' = r/s). */
int gfo_lowres_radius_q(int r, int sn, int sd)
{
    if (sn == sd) return r;
    int rl = (int)((2LL * r * sd + sn) / (2LL * sn)); /* floor(r/s + 1/2) */
    if (r >= 1 && rl < 1) rl = 1;
    return rl;
}
int gfo_lowres_radius(int r, int s) { return gfo_lowres_radius_q(r, s, 1); }

/* R5: h = ceil(H / s), w = ceil(W / s). */
void gfo_lowres_shape_q(int H, int W, int sn, int sd, int *h, int *w)
{
    *h = (int)(((long long)H * sd + sn - 1) / sn);
    *w = (int)(((long long)W * sd + sn - 1) / sn);
}
void gfo_lowres_shape(int H, int W, int s, int *h, int *w) { gfo_lowres_shape_q(H, W, s, 1, h, w); }

/* One bilinear tap pair along an axis (R3/R7): position t on an axis of length n, clamped. */
static void axis_taps(double t, int n, int *i0, int *i1, double *f)
{
    t = dclamp(t, 0.0, (double)(n - 1));
    int a = (int)floor(t);
    *i0 = a;
    *i1 = imin(a + 1, n - 1);
    *f = t - (double)a;
}

/* A bilinear tap pair at the position num / den (a ratio of integers) on an axis of length n, clamped. */
static void axis_taps_q(long long num, long long den, int n, int *i0, int *i1, double *f)
{
    if (num <= 0) { *i0 = *i1 = 0; *f = 0.0; return; }
    long long q = num / den;
    if (q >= n - 1) { *i0 = *i1 = n - 1; *f = 0.0; return; }
    *i0 = (int)q;
    *i1 = (int)q + 1;
    *f = (double)(num - q * den) / (double)den;
}

/* R11: triangle weight of source pixel x for low-res pixel i at ratio s = sn / sd:
 * max(0, 1 - |x + 1/2 - (i + 1/2) s| / s) = max(0, 2 sn - |(2x + 1) sd - (2i + 1) sn|) / (2 sn). */
static double aa_weight(int x, int i, int sn, int sd)
{
    long long d = (2LL * x + 1) * sd - (2LL * i + 1) * sn;
    long long num = 2LL * sn - (d < 0 ? -d : d);
    return num > 0 ? (double)num / (2.0 * sn) : 0.0;
}

/* f_subsample(x, s), Algorithm 2 first step; modes R2/R3/R4/R11 at ratio s = sn / sd (box mode: integer s
 * only).  y is ceil(H/s) x ceil(W/s). */
void gfo_subsample_q(const double *x, int H, int W, int sn, int sd, int mode, double *y)
{
    int h, w;
    gfo_lowres_shape_q(H, W, sn, sd, &h, &w);
    for (int j = 0; j < h; ++j) {
        for (int i = 0; i < w; ++i) {
            double v = 0.0;
            if (mode == GFO_SUB_NEAREST) { /* floor((j + 1/2) s) */
                int sy = iclamp((int)(((2LL * j + 1) * sn) / (2LL * sd)), 0, H - 1);
                int sx = iclamp((int)(((2LL * i + 1) * sn) / (2LL * sd)), 0, W - 1);
                v = x[(size_t)sy * W + sx];
            } else if (mode == GFO_SUB_BILINEAR) { /* (j + 1/2) s - 1/2 = ((2j + 1) sn - sd) / (2 sd) */
                int y0, y1, x0, x1;
                double fy, fx;
                axis_taps_q((2LL * j + 1) * sn - sd, 2LL * sd, H, &y0, &y1, &fy);
                axis_taps_q((2LL * i + 1) * sn - sd, 2LL * sd, W, &x0, &x1, &fx);
                double top = (1.0 - fx) * x[(size_t)y0 * W + x0] + fx * x[(size_t)y0 * W + x1];
                double bot = (1.0 - fx) * x[(size_t)y1 * W + x0] + fx * x[(size_t)y1 * W + x1];
                v = (1.0 - fy) * top + fy * bot;
            } else if (mode == GFO_SUB_BILINEAR_AA) {
                /* every source pixel within s of the centre, weighted, over the sum of the weights used */
                double acc = 0.0, wsum = 0.0;
                int ya = (int)(((long long)j * sn) / sd) - (sn + sd - 1) / sd - 1;
                int xa = (int)(((long long)i * sn) / sd) - (sn + sd - 1) / sd - 1;
                int span = 3 * ((sn + sd - 1) / sd) + 3; /* covers (i + 1/2) s +- s */
                for (int yy = imax(0, ya); yy <= imin(H - 1, ya + span); ++yy) {
                    double wy = aa_weight(yy, j, sn, sd);
                    if (wy == 0.0) continue;
                    for (int xx = imax(0, xa); xx <= imin(W - 1, xa + span); ++xx) {
                        double wx = aa_weight(xx, i, sn, sd);
                        if (wx == 0.0) continue;
                        acc += wy * wx * x[(size_t)yy * W + xx];
                        wsum += wy * wx;
                    }
                }
                v = acc / wsum;
            } else { /* GFO_SUB_BOX (integer s = sn, sd = 1) */
                int ya = j * sn, yb = imin((j + 1) * sn, H);
                int xa = i * sn, xb = imin((i + 1) * sn, W);
                double acc = 0.0;
                for (int yy = ya; yy < yb; ++yy)
                    for (int xx = xa; xx < xb; ++xx) acc += x[(size_t)yy * W + xx];
                v = acc / (double)((yb - ya) * (xb - xa));
            }
            y[(size_t)j * w + i] = v;
        }
    }
}
void gfo_subsample(const double *x, int H, int W, int s, int mode, double *y) { gfo_subsample_q(x, H, W, s, 1, mode, y); }

/* Sum of x over the clipped window of radius r around every pixel (no normalisation).  Separable:
 * the sum over a rectangle is the sum over its rows of the sums over its columns. */
void gfo_box_sum(const double *x, int h, int w, int r, double *y)
{
    double *t = (double *)malloc(sizeof(double) * (size_t)h * w);
    for (int j = 0; j < h; ++j) {
        for (int i = 0; i < w; ++i) {
            double acc = 0.0;
            for (int ii = imax(0, i - r); ii <= imin(w - 1, i + r); ++ii) acc += x[(size_t)j * w + ii];
            t[(size_t)j * w + i] = acc;
        }
    }
    for (int j = 0; j < h; ++j) {
        for (int i = 0; i < w; ++i) {
            double acc = 0.0;
            for (int jj = imax(0, j - r); jj <= imin(h - 1, j + r); ++jj) acc += t[(size_t)jj * w + i];
            y[(size_t)j * w + i] = acc;
        }
    }
    free(t);
}

/* Number of in-image pixels of the clipped window of radius r centred at (j, i) (R1). */
static double window_count(int j, int i, int h, int w, int r)
{
    int ny = imin(h - 1, j + r) - imax(0, j - r) + 1;
    int nx = imin(w - 1, i + r) - imax(0, i - r) + 1;
    return (double)ny * (double)nx;
}

/* f_mean(x, r) with R1 border normalisation. */
void gfo_box_mean(const double *x, int h, int w, int r, double *y)
{
    gfo_box_sum(x, h, w, r, y);
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) y[(size_t)j * w + i] /= window_count(j, i, h, w, r);
}

/* f_mean(x, r) by brute force: a double loop over every clipped window (tiny images only). */
void gfo_box_mean_bruteforce(const double *x, int h, int w, int r, double *y)
{
    for (int j = 0; j < h; ++j) {
        for (int i = 0; i < w; ++i) {
            double acc = 0.0;
            int n = 0;
            for (int jj = j - r; jj <= j + r; ++jj) {
                for (int ii = i - r; ii <= i + r; ++ii) {
                    if (jj < 0 || jj >= h || ii < 0 || ii >= w) continue;
                    acc += x[(size_t)jj * w + ii];
                    ++n;
                }
            }
            y[(size_t)j * w + i] = acc / (double)n;
        }
    }
}

static void box_mean_mode(const double *x, int h, int w, int r, int brute, double *y)
{
    if (brute)
        gfo_box_mean_bruteforce(x, h, w, r, y);
    else
        gfo_box_mean(x, h, w, r, y);
}

/* f_upsample(x, s) to H x W, bilinear (R7); Algorithm 2 upsampling step.  Full-res X samples
 * (X + 1/2) / s - 1/2 = ((2X + 1) sd - sn) / (2 sn). */
void gfo_upsample_q(const double *x, int h, int w, int sn, int sd, int H, int W, double *y)
{
    for (int Y = 0; Y < H; ++Y) {
        int y0, y1;
        double fy;
        axis_taps_q((2LL * Y + 1) * sd - sn, 2LL * sn, h, &y0, &y1, &fy);
        for (int X = 0; X < W; ++X) {
            int x0, x1;
            double fx;
            axis_taps_q((2LL * X + 1) * sd - sn, 2LL * sn, w, &x0, &x1, &fx);
            double top = (1.0 - fx) * x[(size_t)y0 * w + x0] + fx * x[(size_t)y0 * w + x1];
            double bot = (1.0 - fx) * x[(size_t)y1 * w + x0] + fx * x[(size_t)y1 * w + x1];
            y[(size_t)Y * W + X] = (1.0 - fy) * top + fy * bot;
        }
    }
}
void gfo_upsample(const double *x, int h, int w, int s, int H, int W, double *y)
{
    gfo_upsample_q(x, h, w, s, 1, H, W, y);
}

/*
 * Algorithm 2 (fast guided filter) for a batch.
 *   I: N x CI x H x W guide (CI = 1 or C, R8);  p: N x C x H x W, or N x C x h x w when p_lowres != 0.
 *   q: N x C x H x W output.  r_low: the low-res radius r' (R6 is applied by the caller).
 * Optional outputs (NULL to skip), all N x C x h x w:
 *   a_out, b_out      -- Eq. (2), (3) at every low-res window;
 *   ma_out, mb_out    -- the box means of a and b before upsampling;
 *   stats_out         -- N x C x 4 x h x w: mean_I, corr_I, mean_p, corr_Ip (Algorithm 2 box step).
 * Returns 0, or -1 on invalid arguments.
 */
int gfo_fast_guided_filter_q(const double *I, const double *p, int N, int CI, int C, int H, int W, int r_low,
                             double eps, int sn, int sd, int mode, int p_lowres, int brute, double *q, double *a_out,
                             double *b_out, double *ma_out, double *mb_out, double *stats_out)
{
    if (N < 1 || C < 1 || H < 1 || W < 1 || sd < 1 || sn < sd || r_low < 0 || !(eps >= 0.0)) return -1;
    if (mode < GFO_SUB_NEAREST || mode > GFO_SUB_BILINEAR_AA) return -1;
    if (mode == GFO_SUB_BOX && sn % sd != 0) return -1; /* box blocks need an integer ratio */
    if (CI != 1 && CI != C) return -1;
    if (sn % sd == 0) { sn /= sd; sd = 1; }
    int h, w;
    gfo_lowres_shape_q(H, W, sn, sd, &h, &w);
    size_t n = (size_t)h * w, NF = (size_t)H * W;
    double *Il = malloc(sizeof(double) * n), *pl = malloc(sizeof(double) * n);
    double *II = malloc(sizeof(double) * n), *Ip = malloc(sizeof(double) * n);
    double *mean_I = malloc(sizeof(double) * n), *mean_p = malloc(sizeof(double) * n);
    double *corr_I = malloc(sizeof(double) * n), *corr_Ip = malloc(sizeof(double) * n);
    double *a = malloc(sizeof(double) * n), *b = malloc(sizeof(double) * n);
    double *mean_a = malloc(sizeof(double) * n), *mean_b = malloc(sizeof(double) * n);
    double *up_a = malloc(sizeof(double) * NF), *up_b = malloc(sizeof(double) * NF);

    for (int bn = 0; bn < N; ++bn) {
        for (int c = 0; c < C; ++c) {
            const double *Ig = I + ((size_t)bn * CI + (CI == 1 ? 0 : c)) * NF;
            /* step 1: I' = f_subsample(I, s), p' = f_subsample(p, s), r' = r/s */
            gfo_subsample_q(Ig, H, W, sn, sd, mode, Il);
            if (p_lowres)
                memcpy(pl, p + ((size_t)bn * C + c) * n, sizeof(double) * n);
            else
                gfo_subsample_q(p + ((size_t)bn * C + c) * NF, H, W, sn, sd, mode, pl);
            /* step 2: box means of I', p', I'.*I', I'.*p' */
            for (size_t k = 0; k < n; ++k) {
                II[k] = Il[k] * Il[k];
                Ip[k] = Il[k] * pl[k];
            }
            box_mean_mode(Il, h, w, r_low, brute, mean_I);
            box_mean_mode(pl, h, w, r_low, brute, mean_p);
            box_mean_mode(II, h, w, r_low, brute, corr_I);
            box_mean_mode(Ip, h, w, r_low, brute, corr_Ip);
            /* steps 3-4: var, cov, then a (Eq. 2) and b (Eq. 3) */
            for (size_t k = 0; k < n; ++k) {
                double var_I = corr_I[k] - mean_I[k] * mean_I[k];
                double cov_Ip = corr_Ip[k] - mean_I[k] * mean_p[k];
                a[k] = cov_Ip / (var_I + eps);
                b[k] = mean_p[k] - a[k] * mean_I[k];
            }
            /* step 5: box means of a and b */
            box_mean_mode(a, h, w, r_low, brute, mean_a);
            box_mean_mode(b, h, w, r_low, brute, mean_b);
            /* step 6: bilinear upsample to the original size */
            gfo_upsample_q(mean_a, h, w, sn, sd, H, W, up_a);
            gfo_upsample_q(mean_b, h, w, sn, sd, H, W, up_b);
            /* step 7: q = mean_a .* I + mean_b on the full-resolution guide (Eq. 4) */
            double *qc = q + ((size_t)bn * C + c) * NF;
            for (size_t k = 0; k < NF; ++k) qc[k] = up_a[k] * Ig[k] + up_b[k];

            size_t off = ((size_t)bn * C + c) * n;
            if (a_out) memcpy(a_out + off, a, sizeof(double) * n);
            if (b_out) memcpy(b_out + off, b, sizeof(double) * n);
            if (ma_out) memcpy(ma_out + off, mean_a, sizeof(double) * n);
            if (mb_out) memcpy(mb_out + off, mean_b, sizeof(double) * n);
            if (stats_out) {
                double *st = stats_out + ((size_t)bn * C + c) * 4 * n;
                memcpy(st + 0 * n, mean_I, sizeof(double) * n);
                memcpy(st + 1 * n, corr_I, sizeof(double) * n);
                memcpy(st + 2 * n, mean_p, sizeof(double) * n);
                memcpy(st + 3 * n, corr_Ip, sizeof(double) * n);
            }
        }
    }
    free(Il); free(pl); free(II); free(Ip); free(mean_I); free(mean_p); free(corr_I); free(corr_Ip);
    free(a); free(b); free(mean_a); free(mean_b); free(up_a); free(up_b);
    return 0;
}

int gfo_fast_guided_filter(const double *I, const double *p, int N, int CI, int C, int H, int W, int r_low,
                           double eps, int s, int mode, int p_lowres, int brute, double *q, double *a_out,
                           double *b_out, double *ma_out, double *mb_out, double *stats_out)
{
    if (s < 1) return -1;
    return gfo_fast_guided_filter_q(I, p, N, CI, C, H, W, r_low, eps, s, 1, mode, p_lowres, brute, q, a_out, b_out,
                                    ma_out, mb_out, stats_out);
}

/* ---- Algorithm 1 (guided filter), coded separately ------------------------------------------------ */

/* Mean over clipped windows through a summed-area table: S(j, i) = sum of x over rows < j, cols < i. */
static void sat_box_mean(const double *x, int h, int w, int r, double *y)
{
    size_t pw = (size_t)w + 1;
    double *S = calloc(((size_t)h + 1) * pw, sizeof(double));
    for (int j = 0; j < h; ++j) {
        double row = 0.0;
        for (int i = 0; i < w; ++i) {
            row += x[(size_t)j * w + i];
            S[(size_t)(j + 1) * pw + (i + 1)] = S[(size_t)j * pw + (i + 1)] + row;
        }
    }
    for (int j = 0; j < h; ++j) {
        int ja = imax(0, j - r), jb = imin(h - 1, j + r) + 1;
        for (int i = 0; i < w; ++i) {
            int ia = imax(0, i - r), ib = imin(w - 1, i + r) + 1;
            double sum = S[(size_t)jb * pw + ib] - S[(size_t)ja * pw + ib] - S[(size_t)jb * pw + ia] +
                         S[(size_t)ja * pw + ia];
            y[(size_t)j * w + i] = sum / (double)((jb - ja) * (ib - ia));
        }
    }
    free(S);
}

/* Algorithm 1 on one H x W guide and one H x W input. */
int gfo_guided_filter(const double *I, const double *p, int H, int W, int r, double eps, double *q)
{
    if (H < 1 || W < 1 || r < 0 || !(eps >= 0.0)) return -1;
    size_t n = (size_t)H * W;
    double *t = malloc(sizeof(double) * n);
    double *mI = malloc(sizeof(double) * n), *mp = malloc(sizeof(double) * n);
    double *cI = malloc(sizeof(double) * n), *cIp = malloc(sizeof(double) * n);
    double *a = malloc(sizeof(double) * n), *b = malloc(sizeof(double) * n);
    sat_box_mean(I, H, W, r, mI);
    sat_box_mean(p, H, W, r, mp);
    for (size_t k = 0; k < n; ++k) t[k] = I[k] * I[k];
    sat_box_mean(t, H, W, r, cI);
    for (size_t k = 0; k < n; ++k) t[k] = I[k] * p[k];
    sat_box_mean(t, H, W, r, cIp);
    for (size_t k = 0; k < n; ++k) {
        double var = cI[k] - mI[k] * mI[k];
        double cov = cIp[k] - mI[k] * mp[k];
        a[k] = cov / (var + eps);
        b[k] = mp[k] - a[k] * mI[k];
    }
    sat_box_mean(a, H, W, r, mI); /* reuse buffers: mean_a, mean_b */
    sat_box_mean(b, H, W, r, mp);
    for (size_t k = 0; k < n; ++k) q[k] = mI[k] * I[k] + mp[k];
    free(t); free(mI); free(mp); free(cI); free(cIp); free(a); free(b);
    return 0;
}

/* ---- Adjoint of Algorithm 2 ----------------------------------------------------------------------- */

/* Transpose of f_mean (R1): for every window k, spread y_k / n_k over the pixels of the window. */
static void box_mean_T(const double *y, int h, int w, int r, int brute, double *out)
{
    size_t n = (size_t)h * w;
    if (brute) {
        memset(out, 0, sizeof(double) * n);
        for (int j = 0; j < h; ++j)
            for (int i = 0; i < w; ++i) {
                double v = y[(size_t)j * w + i] / window_count(j, i, h, w, r);
                for (int jj = imax(0, j - r); jj <= imin(h - 1, j + r); ++jj)
                    for (int ii = imax(0, i - r); ii <= imin(w - 1, i + r); ++ii) out[(size_t)jj * w + ii] += v;
            }
        return;
    }
    /* Same map, gathered: pixel i receives the sum of y_k / n_k over the windows k that contain it,
     * which (windows are symmetric) are the k inside the window of radius r around i. */
    double *z = malloc(sizeof(double) * n);
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) z[(size_t)j * w + i] = y[(size_t)j * w + i] / window_count(j, i, h, w, r);
    gfo_box_sum(z, h, w, r, out);
    free(z);
}

/* Transpose of f_subsample: every low-res value is spread back with the weights the forward map used. */
static void subsample_T(const double *y, int H, int W, int s, int mode, double *x)
{
    int h, w;
    gfo_lowres_shape(H, W, s, &h, &w);
    memset(x, 0, sizeof(double) * (size_t)H * W);
    for (int j = 0; j < h; ++j) {
        for (int i = 0; i < w; ++i) {
            double g = y[(size_t)j * w + i];
            if (mode == GFO_SUB_NEAREST) {
                int sy = iclamp((int)floor((j + 0.5) * s), 0, H - 1);
                int sx = iclamp((int)floor((i + 0.5) * s), 0, W - 1);
                x[(size_t)sy * W + sx] += g;
            } else if (mode == GFO_SUB_BILINEAR) {
                int y0, y1, x0, x1;
                double fy, fx;
                axis_taps((j + 0.5) * s - 0.5, H, &y0, &y1, &fy);
                axis_taps((i + 0.5) * s - 0.5, W, &x0, &x1, &fx);
                x[(size_t)y0 * W + x0] += (1.0 - fy) * (1.0 - fx) * g;
                x[(size_t)y0 * W + x1] += (1.0 - fy) * fx * g;
                x[(size_t)y1 * W + x0] += fy * (1.0 - fx) * g;
                x[(size_t)y1 * W + x1] += fy * fx * g;
            } else {
                int ya = j * s, yb = imin((j + 1) * s, H);
                int xa = i * s, xb = imin((i + 1) * s, W);
                double v = g / (double)((yb - ya) * (xb - xa));
                for (int yy = ya; yy < yb; ++yy)
                    for (int xx = xa; xx < xb; ++xx) x[(size_t)yy * W + xx] += v;
            }
        }
    }
}

/* Transpose of f_upsample: every full-res value is spread to its four low-res taps. */
static void upsample_T(const double *Y, int h, int w, int s, int H, int W, double *y)
{
    memset(y, 0, sizeof(double) * (size_t)h * w);
    for (int Yi = 0; Yi < H; ++Yi) {
        int y0, y1;
        double fy;
        axis_taps((Yi + 0.5) / (double)s - 0.5, h, &y0, &y1, &fy);
        for (int X = 0; X < W; ++X) {
            int x0, x1;
            double fx;
            axis_taps((X + 0.5) / (double)s - 0.5, w, &x0, &x1, &fx);
            double g = Y[(size_t)Yi * W + X];
            y[(size_t)y0 * w + x0] += (1.0 - fy) * (1.0 - fx) * g;
            y[(size_t)y0 * w + x1] += (1.0 - fy) * fx * g;
            y[(size_t)y1 * w + x0] += fy * (1.0 - fx) * g;
            y[(size_t)y1 * w + x1] += fy * fx * g;
        }
    }
}

/*
 * Backward pass of Algorithm 2: given gq = dL/dq (N x C x H x W), accumulate
 *   dI   (N x CI x H x W, overwritten), dp (same shape as p, overwritten), *deps (overwritten).
 * Any of dI, dp, deps may be NULL.  The chain runs the forward steps in reverse; each line names the
 * forward step it differentiates.
 */
int gfo_fast_guided_filter_backward(const double *I, const double *p, const double *gq, int N, int CI, int C,
                                    int H, int W, int r_low, double eps, int s, int mode, int p_lowres,
                                    int brute, double *dI, double *dp, double *deps)
{
    if (N < 1 || C < 1 || H < 1 || W < 1 || s < 1 || r_low < 0 || !(eps >= 0.0)) return -1;
    if (mode < GFO_SUB_NEAREST || mode > GFO_SUB_BOX) return -1; /* the adjoint covers R2-R4 */
    if (CI != 1 && CI != C) return -1;
    int h, w;
    gfo_lowres_shape(H, W, s, &h, &w);
    size_t n = (size_t)h * w, NF = (size_t)H * W;
    size_t pn = p_lowres ? n : NF;
#define ALLOC(name, cnt) double *name = malloc(sizeof(double) * (cnt))
    ALLOC(Il, n); ALLOC(pl, n); ALLOC(t, n); ALLOC(mean_I, n); ALLOC(mean_p, n); ALLOC(corr_I, n);
    ALLOC(corr_Ip, n); ALLOC(var, n); ALLOC(a, n); ALLOC(mean_a, n); ALLOC(up_a, NF);
    ALLOC(gfull, NF); ALLOC(d_ma, n); ALLOC(d_mb, n); ALLOC(da, n); ALLOC(db, n);
    ALLOC(dmI, n); ALLOC(dmp, n); ALLOC(dcI, n); ALLOC(dcIp, n); ALLOC(tI, n); ALLOC(tp, n);
    ALLOC(dIl, n); ALLOC(dpl, n); ALLOC(dfull, NF);
#undef ALLOC
    if (dI) memset(dI, 0, sizeof(double) * (size_t)N * CI * NF);
    double eps_acc = 0.0;

    for (int bn = 0; bn < N; ++bn) {
        for (int c = 0; c < C; ++c) {
            const double *Ig = I + ((size_t)bn * CI + (CI == 1 ? 0 : c)) * NF;
            const double *g = gq + ((size_t)bn * C + c) * NF;
            /* forward recomputation */
            gfo_subsample(Ig, H, W, s, mode, Il);
            if (p_lowres)
                memcpy(pl, p + ((size_t)bn * C + c) * n, sizeof(double) * n);
            else
                gfo_subsample(p + ((size_t)bn * C + c) * NF, H, W, s, mode, pl);
            box_mean_mode(Il, h, w, r_low, brute, mean_I);
            box_mean_mode(pl, h, w, r_low, brute, mean_p);
            for (size_t k = 0; k < n; ++k) t[k] = Il[k] * Il[k];
            box_mean_mode(t, h, w, r_low, brute, corr_I);
            for (size_t k = 0; k < n; ++k) t[k] = Il[k] * pl[k];
            box_mean_mode(t, h, w, r_low, brute, corr_Ip);
            for (size_t k = 0; k < n; ++k) {
                var[k] = corr_I[k] - mean_I[k] * mean_I[k];
                double cov = corr_Ip[k] - mean_I[k] * mean_p[k];
                a[k] = cov / (var[k] + eps);
            }
            box_mean_mode(a, h, w, r_low, brute, mean_a);
            gfo_upsample(mean_a, h, w, s, H, W, up_a);

            /* q = up_a .* I + up_b */
            if (dI) {
                double *dIg = dI + ((size_t)bn * CI + (CI == 1 ? 0 : c)) * NF;
                for (size_t k = 0; k < NF; ++k) dIg[k] += g[k] * up_a[k];
            }
            for (size_t k = 0; k < NF; ++k) gfull[k] = g[k] * Ig[k];
            /* up_a = U(mean_a), up_b = U(mean_b) */
            upsample_T(gfull, h, w, s, H, W, d_ma);
            upsample_T(g, h, w, s, H, W, d_mb);
            /* mean_a = B(a), mean_b = B(b) */
            box_mean_T(d_ma, h, w, r_low, brute, da);
            box_mean_T(d_mb, h, w, r_low, brute, db);
            for (size_t k = 0; k < n; ++k) {
                /* b = mean_p - a .* mean_I */
                double dmp_k = db[k];
                double da_k = da[k] - mean_I[k] * db[k];
                double dmI_k = -a[k] * db[k];
                /* a = cov / (var + eps) */
                double inv = 1.0 / (var[k] + eps);
                double dcov = da_k * inv;
                double dvar = -da_k * a[k] * inv;
                eps_acc += dvar; /* d(var + eps)/d eps = 1 */
                /* var = corr_I - mean_I.^2 ;  cov = corr_Ip - mean_I .* mean_p */
                dcI[k] = dvar;
                dmI_k += -2.0 * mean_I[k] * dvar;
                dcIp[k] = dcov;
                dmI_k += -mean_p[k] * dcov;
                dmp_k += -mean_I[k] * dcov;
                dmI[k] = dmI_k;
                dmp[k] = dmp_k;
            }
            /* mean_I = B(I'), mean_p = B(p'), corr_I = B(I'.*I'), corr_Ip = B(I'.*p') */
            box_mean_T(dmI, h, w, r_low, brute, dIl);
            box_mean_T(dmp, h, w, r_low, brute, dpl);
            box_mean_T(dcI, h, w, r_low, brute, tI);
            box_mean_T(dcIp, h, w, r_low, brute, tp);
            for (size_t k = 0; k < n; ++k) {
                dIl[k] += 2.0 * Il[k] * tI[k] + pl[k] * tp[k];
                dpl[k] += Il[k] * tp[k];
            }
            /* I' = f_subsample(I), p' = f_subsample(p) */
            if (dI) {
                double *dIg = dI + ((size_t)bn * CI + (CI == 1 ? 0 : c)) * NF;
                subsample_T(dIl, H, W, s, mode, dfull);
                for (size_t k = 0; k < NF; ++k) dIg[k] += dfull[k];
            }
            if (dp) {
                double *dpc = dp + ((size_t)bn * C + c) * pn;
                if (p_lowres)
                    memcpy(dpc, dpl, sizeof(double) * n);
                else
                    subsample_T(dpl, H, W, s, mode, dpc);
            }
        }
    }
    if (deps) *deps = eps_acc;
    free(Il); free(pl); free(t); free(mean_I); free(mean_p); free(corr_I); free(corr_Ip); free(var);
    free(a); free(mean_a); free(up_a); free(gfull); free(d_ma); free(d_mb); free(da); free(db);
    free(dmI); free(dmp); free(dcI); free(dcIp); free(tI); free(tp); free(dIl); free(dpl); free(dfull);
    return 0;
}

/* Detail enhancement (Fig. 2 application: the smoothed base layer q plus k times the detail layer I - q).
 * q: N x C x H x W; I: N x CI x H x W (channel c uses guide channel c, or channel 0 when CI = 1). */
int gfo_detail_enhance(const double *I, const double *q, int N, int CI, int C, int H, int W, double k, double *out)
{
    if (N < 1 || C < 1 || H < 1 || W < 1 || (CI != 1 && CI != C)) return -1;
    const size_t HW = (size_t)H * W;
    for (int n = 0; n < N; ++n)
        for (int c = 0; c < C; ++c) {
            const double *Ic = I + ((size_t)n * CI + (CI == 1 ? 0 : c)) * HW;
            const double *qc = q + ((size_t)n * C + c) * HW;
            double *oc = out + ((size_t)n * C + c) * HW;
            for (size_t i = 0; i < HW; ++i) oc[i] = qc[i] + k * (Ic[i] - qc[i]);
        }
    return 0;
}

/* x = M^-1 v for a 3 x 3 matrix M by Cramer's rule.  Returns -1 if M is singular. */
static int solve3(const double M[3][3], const double v[3], double x[3])
{
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (det == 0.0) return -1;
    for (int k = 0; k < 3; ++k) {
        double A[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) A[i][j] = (j == k) ? v[i] : M[i][j];
        x[k] = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) / det;
    }
    return 0;
}

/*
 * Colour-guided fast guided filter (R12) for a batch.
 *   I: N x 3 x H x W colour guide;  p: N x C x H x W, or N x C x h x w when p_lowres != 0;  q: N x C x H x W.
 *   Optional: a_out N x C x 3 x h x w (the 3-vector a of every window), b_out N x C x h x w.
 * Returns 0, -1 on invalid arguments, -2 if some Sigma + eps U is singular.
 */
int gfo_color_guided_filter(const double *I, const double *p, int N, int C, int H, int W, int r_low, double eps,
                            int s, int mode, int p_lowres, double *q, double *a_out, double *b_out)
{
    if (N < 1 || C < 1 || H < 1 || W < 1 || s < 1 || r_low < 0 || !(eps >= 0.0)) return -1;
    if (mode < GFO_SUB_NEAREST || mode > GFO_SUB_BILINEAR_AA) return -1;
    int h, w;
    gfo_lowres_shape(H, W, s, &h, &w);
    size_t n = (size_t)h * w, NF = (size_t)H * W;
    static const int PK[6] = {0, 0, 0, 1, 1, 2}, PL[6] = {0, 1, 2, 1, 2, 2}; /* guide products rr rg rb gg gb bb */
    double *buf = malloc(sizeof(double) * (n * 27 + NF * 4));
    double *Il = buf, *mean_I = Il + 3 * n, *corr_I = mean_I + 3 * n, *pl = corr_I + 6 * n, *mean_p = pl + n;
    double *corr_Ip = mean_p + n, *a = corr_Ip + 3 * n, *b = a + 3 * n, *mean_a = b + n, *mean_b = mean_a + 3 * n;
    double *tmp = mean_b + n, *up = buf + n * 27;
    int rc = 0;
    for (int bn = 0; bn < N && rc == 0; ++bn) {
        const double *Ig = I + (size_t)bn * 3 * NF;
        /* step 1 for the guide: I' = f_subsample(I, s), channel by channel */
        for (int k = 0; k < 3; ++k) gfo_subsample(Ig + k * NF, H, W, s, mode, Il + k * n);
        /* step 2 for the guide: box means of I'_k and of every product I'_k I'_l */
        for (int k = 0; k < 3; ++k) gfo_box_mean(Il + k * n, h, w, r_low, mean_I + k * n);
        for (int m = 0; m < 6; ++m) {
            for (size_t t = 0; t < n; ++t) tmp[t] = Il[PK[m] * n + t] * Il[PL[m] * n + t];
            gfo_box_mean(tmp, h, w, r_low, corr_I + m * n);
        }
        for (int c = 0; c < C && rc == 0; ++c) {
            /* steps 1-2 for p: p' and the box means of p' and of I'_k p' */
            if (p_lowres)
                memcpy(pl, p + ((size_t)bn * C + c) * n, sizeof(double) * n);
            else
                gfo_subsample(p + ((size_t)bn * C + c) * NF, H, W, s, mode, pl);
            gfo_box_mean(pl, h, w, r_low, mean_p);
            for (int k = 0; k < 3; ++k) {
                for (size_t t = 0; t < n; ++t) tmp[t] = Il[k * n + t] * pl[t];
                gfo_box_mean(tmp, h, w, r_low, corr_Ip + k * n);
            }
            /* steps 3-4: Sigma + eps U, cov_Ip, a = (Sigma + eps U)^-1 cov_Ip, b = mean_p - a^T mean_I */
            for (size_t t = 0; t < n; ++t) {
                double M[3][3], v[3], x[3];
                for (int m = 0; m < 6; ++m) {
                    double e = corr_I[m * n + t] - mean_I[PK[m] * n + t] * mean_I[PL[m] * n + t];
                    M[PK[m]][PL[m]] = e;
                    M[PL[m]][PK[m]] = e;
                }
                for (int k = 0; k < 3; ++k) {
                    M[k][k] += eps;
                    v[k] = corr_Ip[k * n + t] - mean_I[k * n + t] * mean_p[t];
                }
                if (solve3(M, v, x) != 0) { rc = -2; break; }
                double bb = mean_p[t];
                for (int k = 0; k < 3; ++k) {
                    a[k * n + t] = x[k];
                    bb -= x[k] * mean_I[k * n + t];
                }
                b[t] = bb;
            }
            if (rc) break;
            /* step 5: box means of a (each component) and b */
            for (int k = 0; k < 3; ++k) gfo_box_mean(a + k * n, h, w, r_low, mean_a + k * n);
            gfo_box_mean(b, h, w, r_low, mean_b);
            /* steps 6-7: upsample, q = mean_a^T I + mean_b on the full-resolution guide */
            double *qc = q + ((size_t)bn * C + c) * NF;
            gfo_upsample(mean_b, h, w, s, H, W, up);
            memcpy(qc, up, sizeof(double) * NF);
            for (int k = 0; k < 3; ++k) {
                gfo_upsample(mean_a + k * n, h, w, s, H, W, up);
                for (size_t t = 0; t < NF; ++t) qc[t] += up[t] * Ig[k * NF + t];
            }
            if (a_out) memcpy(a_out + ((size_t)bn * C + c) * 3 * n, a, sizeof(double) * 3 * n);
            if (b_out) memcpy(b_out + ((size_t)bn * C + c) * n, b, sizeof(double) * n);
        }
    }
    free(buf);
    return rc;
}
