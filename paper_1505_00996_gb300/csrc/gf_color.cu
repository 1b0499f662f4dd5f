// gf_color.cu -- the colour-guided form of the fast guided filter on sm_103a.
//
// The guided filter's colour form (the paper cites it; its Algorithm 2 wraps it unchanged): with a
// 3-channel guide I, every window fits q = a^T I + b with a 3-vector a,
//     a = (Sigma + eps U)^-1 cov_Ip,   b = mean_p - a^T mean_I,
// Sigma being the 3 x 3 covariance of the subsampled guide I' in the window and cov_Ip the covariance of each
// guide channel with p'.  Then mean_a (3 maps) and mean_b are box-averaged, upsampled bilinearly, and
// q = mean_a^T I + mean_b on the full-resolution guide.
//
// Stages (the box means run in k_box_tile_x2's KIND 2 form, in gf_forward.cu, two planes per pass):
//   k_color_products  per low-res pixel: the 9 guide quantities I'_k and I'_k I'_l and, per channel of p,
//                     p' and I'_k p', all taken relative to the first sample of each plane (covariances do
//                     not change under a shift, and the smaller values keep E[xy] - E[x]E[y] accurate in
//                     FP32).  Written as two arrays A and B of K = 5 + 2C planes per image (one pad plane).
//   box means         of the 2K planes.
//   k_color_coef      per low-res pixel and channel: Sigma + eps U and cov_Ip from the means, a by the
//                     adjugate of the symmetric 3 x 3 matrix, b; written as the planes (a_r, a_b) and
//                     (a_g, b) of every channel.
//   box means         of the 4C coefficient planes.
//   k_color_output    per full-res pixel and channel: the four means interpolated bilinearly (gf.h
//                     conventions) and q = mean_a^T I + mean_b, plus the optional detail epilogue;
//                     k_color_output_s4x is its run form for s = 4, 8 on aligned rows (compile-time weights).
#include <algorithm>

#include "gf_device.cuh"
#include "gf_internal.cuh"

namespace gfk {

namespace {

constexpr int COL_NT = 256;

// Guide products in plane order: A gets rr, rg (after the three shifted guide planes), B gets rb, gg, gb, bb.
__global__ void __launch_bounds__(COL_NT) k_color_products(const float *__restrict__ Il, const float *__restrict__ pl,
                                                           float *__restrict__ QA, float *__restrict__ QB, int C,
                                                           int h, int w, size_t lps)
{
    const int n = blockIdx.y;
    const int K = 5 + 2 * C;
    const float *g = Il + (size_t)n * 3 * lps;
    const float *pp = pl + (size_t)n * C * lps;
    float *A = QA + (size_t)n * K * lps, *B = QB + (size_t)n * K * lps;
    const float s0 = g[0], s1 = g[lps], s2 = g[2 * lps];
    const size_t hw = (size_t)h * w;
    for (size_t t = (size_t)blockIdx.x * COL_NT + threadIdx.x; t < hw; t += (size_t)gridDim.x * COL_NT) {
        const float r = g[t] - s0, gg = g[lps + t] - s1, b = g[2 * lps + t] - s2;
        A[t] = r;
        A[lps + t] = gg;
        A[2 * lps + t] = b;
        A[3 * lps + t] = r * r;
        A[4 * lps + t] = r * gg;
        B[t] = r * b;
        B[lps + t] = gg * gg;
        B[2 * lps + t] = gg * b;
        B[3 * lps + t] = b * b;
        B[4 * lps + t] = 0.0f;
        for (int c = 0; c < C; ++c) {
            const float pv = pp[c * lps + t] - pp[c * lps];
            A[(5 + 2 * c) * lps + t] = pv;
            A[(6 + 2 * c) * lps + t] = r * pv;
            B[(5 + 2 * c) * lps + t] = gg * pv;
            B[(6 + 2 * c) * lps + t] = b * pv;
        }
    }
}

__global__ void __launch_bounds__(COL_NT) k_color_coef(const float *__restrict__ Il, const float *__restrict__ pl,
                                                       const float *__restrict__ MA, const float *__restrict__ MB,
                                                       float *__restrict__ AX, float *__restrict__ AY, int C, int h,
                                                       int w, size_t lps, float eps)
{
    const int n = blockIdx.y;
    const int K = 5 + 2 * C;
    const float *A = MA + (size_t)n * K * lps, *B = MB + (size_t)n * K * lps;
    const float *g = Il + (size_t)n * 3 * lps;
    const float *pp = pl + (size_t)n * C * lps;
    const float s0 = g[0], s1 = g[lps], s2 = g[2 * lps];
    const size_t hw = (size_t)h * w;
    for (size_t t = (size_t)blockIdx.x * COL_NT + threadIdx.x; t < hw; t += (size_t)gridDim.x * COL_NT) {
        const float mr = A[t], mg = A[lps + t], mb = A[2 * lps + t];  // shifted guide means
        // Sigma + eps U (symmetric)
        const float xx = A[3 * lps + t] - mr * mr + eps, xy = A[4 * lps + t] - mr * mg, xz = B[t] - mr * mb;
        const float yy = B[lps + t] - mg * mg + eps, yz = B[2 * lps + t] - mg * mb, zz = B[3 * lps + t] - mb * mb + eps;
        // adjugate (cofactors) and determinant
        const float c00 = yy * zz - yz * yz, c01 = xz * yz - xy * zz, c02 = xy * yz - xz * yy;
        const float c11 = xx * zz - xz * xz, c12 = xy * xz - xx * yz, c22 = xx * yy - xy * xy;
        const float inv_det = 1.0f / (xx * c00 + xy * c01 + xz * c02);
        for (int c = 0; c < C; ++c) {
            const float mp = A[(5 + 2 * c) * lps + t];
            const float vr = A[(6 + 2 * c) * lps + t] - mr * mp;
            const float vg = B[(5 + 2 * c) * lps + t] - mg * mp;
            const float vb = B[(6 + 2 * c) * lps + t] - mb * mp;
            const float ar = (c00 * vr + c01 * vg + c02 * vb) * inv_det;
            const float ag = (c01 * vr + c11 * vg + c12 * vb) * inv_det;
            const float ab = (c02 * vr + c12 * vg + c22 * vb) * inv_det;
            // b = mean_p - a^T mean_I with the shifts put back
            const float bb = (mp + pp[c * lps]) - ar * (mr + s0) - ag * (mg + s1) - ab * (mb + s2);
            float *ax = AX + ((size_t)n * 2 * C + 2 * c) * lps, *ay = AY + ((size_t)n * 2 * C + 2 * c) * lps;
            ax[t] = ar;
            ax[lps + t] = ab;
            ay[t] = ag;
            ay[lps + t] = bb;
        }
    }
}

template <typename T>
__device__ __forceinline__ void ld4g(const T *p, bool vec, int valid, float v[4])
{
    if constexpr (sizeof(T) == 4) {
        if (vec) {
            const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
            v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (k < valid) ? ldv(p + k) : 0.0f;
}

template <typename T>
__device__ __forceinline__ void st4g(T *p, bool vec, int valid, const float v[4])
{
    if constexpr (sizeof(T) == 4) {
        if (vec) {
            __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (k < valid) {
            if constexpr (sizeof(T) == 4) __stcs(reinterpret_cast<float *>(p) + k, v[k]);
            else p[k] = __float2half_rn(v[k]);
        }
}

// CTA = one channel of one 512-pixel-wide band of CO_R rows; the channel is the fastest-varying block index,
// so the channel CTAs of a band run side by side and read the guide through L2 once.  The low-res taps of
// the four means (mean of a_r, a_g, a_b, b) under the band are staged in shared memory; each thread owns 4
// adjacent pixels, keeps the horizontally interpolated upper and lower tap rows of the four maps in
// registers (recomputed only when the tap rows change, every s rows), and reads the three guide planes with
// 128-bit streaming loads.
constexpr int CO_NT = 128, CO_BAND = 4 * CO_NT, CO_NST = 4;

// 4 pixels from the thread's ring slot, as floats.
template <typename T>
__device__ __forceinline__ void ld4_ring(const unsigned char *p, float v[4])
{
    if constexpr (sizeof(T) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

template <typename TI, typename TQ>
__global__ void __launch_bounds__(CO_NT) k_color_output(const TI *__restrict__ I, TQ *__restrict__ q,
                                                        const float *__restrict__ MX, const float *__restrict__ MY,
                                                        int C, int H, int W, int h, int w, int s, size_t fps,
                                                        size_t lps, int R, int LCmax, int Yw0, int Yw1, float detail,
                                                        bool vec_io)
{
    extern __shared__ float tap[];  // [4 maps][LR][LCmax]
    const int c = blockIdx.x % C, band = blockIdx.x / C, n = blockIdx.z;
    const int Xb = band * CO_BAND;
    const int Yb = max((int)blockIdx.y * R, Yw0), Ye = min(min((int)blockIdx.y * R + R, H), Yw1);
    if (Yb >= Ye) return;
    int ly0, ly1, lx0, lx1, t0;
    float ft;
    up_taps(Yb, s, h, ly0, t0, ft);
    up_taps(Ye - 1, s, h, t0, ly1, ft);
    up_taps(Xb, s, w, lx0, t0, ft);
    up_taps(min(Xb + CO_BAND, W) - 1, s, w, t0, lx1, ft);
    const int LR = ly1 - ly0 + 1, LC = lx1 - lx0 + 1, tile = LR * LCmax;
    const float *mx = MX + ((size_t)n * 2 * C + 2 * c) * lps, *my = MY + ((size_t)n * 2 * C + 2 * c) * lps;
    for (int mr = 0; mr < 4 * LR; ++mr) {  // maps in order: mean of a_r (mx), a_g (my), a_b (mx + lps), b (my + lps)
        const int m = mr / LR, row = mr - m * LR;
        const float *src = ((m & 1) ? my : mx) + (m >> 1) * lps + (size_t)(ly0 + row) * w + lx0;
        float *dst = tap + m * tile + row * LCmax;
        for (int col = threadIdx.x; col < LC; col += CO_NT) cp_async4(dst + col, src + col);
    }
    cp_async_wait_all();
    __syncthreads();

    const int X0 = Xb + threadIdx.x * 4;
    if (X0 >= W) return;
    const int valid = min(4, W - X0);
    const bool vec = vec_io && (valid == 4);
    int xa[4], xb[4];
    float fx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        up_taps(min(X0 + k, W - 1), s, w, xa[k], xb[k], fx[k]);
        xa[k] -= lx0;
        xb[k] -= lx0;
    }
    // horizontally interpolated upper tap row (lo) and lower minus upper (d), per map and pixel
    float lo[4][4], d[4][4];
    auto hrow = [&](int yy, float (&o)[4][4]) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float *rp = tap + m * tile + (yy - ly0) * LCmax;
#pragma unroll
            for (int k = 0; k < 4; ++k) o[m][k] = fmaf(fx[k], rp[xb[k]] - rp[xa[k]], rp[xa[k]]);
        }
    };
    const TI *Ig = I + (size_t)n * 3 * fps + X0;
    TQ *qc = q + ((size_t)n * C + c) * fps + X0;
    // The three guide planes' 4 pixels of the next CO_NST - 1 rows are in flight at any time: each thread
    // copies them into its own slots of a shared ring (cp.async, 16 or 8 bytes) and reads back only what it
    // copied itself, so the only synchronisation is the thread's own group wait.  A thread whose 4 pixels
    // are not one aligned vector (a ragged last group, unaligned planes) loads them directly instead.
    constexpr int VB = 4 * (int)sizeof(TI);
    unsigned char *ring = reinterpret_cast<unsigned char *>(tap + 4 * tile);  // [CO_NST][3][CO_NT][VB]
    auto slot = [&](int stage, int k) { return ring + ((size_t)(stage * 3 + k) * CO_NT + threadIdx.x) * VB; };
    auto issue = [&](int u) {
        const int Y = Yb + u;
        if (vec && Y < Ye) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const TI *src = Ig + k * fps + (size_t)Y * W;
                if constexpr (VB == 16) cp_async16(slot(u % CO_NST, k), src);
                else ld_async_small<TI>(slot(u % CO_NST, k), src);
            }
        }
        cp_async_commit();  // one group per row, empty when nothing was copied, so the count stays uniform
    };
#pragma unroll
    for (int u = 0; u < CO_NST - 1; ++u) issue(u);
    float gv[3][4];
    // vertical taps walked row by row: numerator 2Y + 1 - s over 2s, quotient qt and remainder rem (gf.h, R7)
    const int den = 2 * s;
    const float inv_den = 1.0f / (float)den;
    int num = 2 * Yb + 1 - s, qt = 0, rem = 0;
    if (num > 0) { qt = num / den; rem = num - qt * den; }
    int cur_a = -1, cur_b = -1;
    for (int Y = Yb; Y < Ye; ++Y) {
        const int u = Y - Yb;
        issue(u + CO_NST - 1);
        cp_async_wait_group<CO_NST - 1>();  // this thread's copies of row u have landed
        if (vec) {
#pragma unroll
            for (int k = 0; k < 3; ++k) ld4_ring<TI>(slot(u % CO_NST, k), gv[k]);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) ld4g<TI>(Ig + k * fps + (size_t)Y * W, false, valid, gv[k]);
        }
        int ya, yb;
        float fy;
        if (num <= 0) { ya = yb = 0; fy = 0.0f; }
        else if (qt >= h - 1) { ya = yb = h - 1; fy = 0.0f; }
        else { ya = qt; yb = qt + 1; fy = (float)rem * inv_den; }
        if (ya != cur_a || yb != cur_b) {
            if (ya == cur_b) {  // the old lower row becomes the upper one
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int k = 0; k < 4; ++k) lo[m][k] += d[m][k];
            } else {
                hrow(ya, lo);
            }
            hrow(yb, d);
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int k = 0; k < 4; ++k) d[m][k] -= lo[m][k];
            cur_a = ya;
            cur_b = yb;
        }
        num += 2;
        if (num > 0) {
            if (num <= 2) { qt = num / den; rem = num - qt * den; }
            else if ((rem += 2) >= den) { rem -= den; ++qt; }
        }
        const float *ir = gv[0], *ig = gv[1], *ib = gv[2];
        float out[4];
        const size_t row = (size_t)Y * W;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            float m[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) m[k] = fmaf(fy, d[k][x], lo[k][x]);
            out[x] = fmaf(m[0], ir[x], fmaf(m[1], ig[x], fmaf(m[2], ib[x], m[3])));
        }
        if (detail != 0.0f) {  // C == 3: channel c's own guide channel is its detail source
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const float iv = (c == 0) ? ir[x] : (c == 1 ? ig[x] : ib[x]);
                out[x] = fmaf(detail, iv - out[x], out[x]);
            }
        }
        st4g<TQ>(qc + row, vec, valid, out);
    }
    cp_async_wait_all();
}

// Run form of k_color_output for s = 4, 8 on aligned rows (the guide read as whole vectors).  Run j covers
// full-res rows s j + s/2 .. s j + s/2 + s - 1, which all sample low-res rows j and j + 1 with vertical weight
// (2k + 1)/(2s) on row j + 1 for row k of the run; across a row the thread's 4 pixels sample fixed low-res
// columns with fixed weights (s = 4: 5/8, 7/8 of column i for pixels 0, 1; 1/8, 3/8 of column i + 1 for
// pixels 2, 3).  So the four means are interpolated horizontally once per run per tap row, and each output
// value costs one FMA per mean and three for q.  The tap tile is filled with clamped indices, so the image's
// edges give the clamped taps (an interpolation between equal values returns that value).  The CTA covers
// 8 runs of one channel of a 512-pixel band; the guide's three planes reach each thread through its own
// cp.async ring slots as in k_color_output.
template <typename TI, typename TQ, int S>
__global__ void __launch_bounds__(CO_NT) k_color_output_s4x(const TI *__restrict__ I, TQ *__restrict__ q,
                                                            const float *__restrict__ MX, const float *__restrict__ MY,
                                                            int C, int H, int W, int h, int w, size_t fps, size_t lps,
                                                            int LR, int LC, int Yw0, int Yw1, float detail)
{
    static_assert(S % 4 == 0, "whole 4-row groups per run");
    extern __shared__ float tap[];  // [4 maps][LR][LC]: means at low-res rows jb - 1 .. jb + NB, clamped
    constexpr int NB = 8;           // runs (low-res rows) per CTA
    const int c = blockIdx.x % C, band = blockIdx.x / C, n = blockIdx.z;
    const int jb = blockIdx.y * NB;
    const int Xb = band * CO_BAND;
    const int Yb = max(jb * S, Yw0), Ye = min(min(jb * S + NB * S, H), Yw1);  // rows written by this CTA
    if (Yb >= Ye) return;
    const int ly0 = jb - 1, lx0 = Xb / S - 1;
    const int tile = LR * LC;
    const float *mx = MX + ((size_t)n * 2 * C + 2 * c) * lps, *my = MY + ((size_t)n * 2 * C + 2 * c) * lps;
    for (int k = threadIdx.x; k < 4 * tile; k += CO_NT) {  // maps: mean of a_r (mx), a_g (my), a_b, b
        const int m = k / tile, rem = k - m * tile, row = rem / LC, col = rem - row * LC;
        const int gy = min(max(ly0 + row, 0), h - 1), gx = min(max(lx0 + col, 0), w - 1);
        cp_async4(tap + k, ((m & 1) ? my : mx) + (m >> 1) * lps + (size_t)gy * w + gx);
    }
    cp_async_wait_all();
    __syncthreads();

    const int X0 = Xb + threadIdx.x * 4;
    if (X0 >= W) return;
    const int ti = X0 / S - lx0;  // tile column of the low-res column that holds pixel X0 (>= 1)
    const int g = (S == 8) ? ((X0 >> 2) & 1) : 0;
    // horizontally interpolated tap row `tr` of the four means for the thread's 4 pixels
    auto hrow = [&](int tr, float (&o)[4][4]) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float *row = tap + m * tile + tr * LC;
            if (S == 4) {
                const float a = row[ti - 1], b = row[ti], cc = row[ti + 1];
                o[m][0] = fmaf(0.625f, b - a, a);
                o[m][1] = fmaf(0.875f, b - a, a);
                o[m][2] = fmaf(0.125f, cc - b, b);
                o[m][3] = fmaf(0.375f, cc - b, b);
            } else {
                const int lo = g ? ti : ti - 1;
                const float a = row[lo], b = row[lo + 1];
                const float f0 = g ? 0.0625f : 0.5625f;
#pragma unroll
                for (int k = 0; k < 4; ++k) o[m][k] = fmaf(f0 + 0.125f * k, b - a, a);
            }
        }
    };
    const TI *Ig = I + (size_t)n * 3 * fps + X0;
    TQ *qc = q + ((size_t)n * C + c) * fps + X0;
    constexpr int VB = 4 * (int)sizeof(TI);
    unsigned char *ring = reinterpret_cast<unsigned char *>(tap + 4 * tile);  // [CO_NST][3][CO_NT][VB]
    auto slot = [&](int stage, int k) { return ring + ((size_t)(stage * 3 + k) * CO_NT + threadIdx.x) * VB; };
    const int Ys = S * (jb - 1) + S / 2;  // first row of the first run
    constexpr int NROWS = (NB + 1) * S;   // rows of the NB + 1 runs
    auto issue = [&](int u) {  // row Ys + u of the walk
        const int Y = Ys + u;
        if (u < NROWS && Y >= Yb && Y < Ye) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const TI *src = Ig + k * fps + (size_t)Y * W;
                if constexpr (VB == 16) cp_async16(slot(u % CO_NST, k), src);
                else ld_async_small<TI>(slot(u % CO_NST, k), src);
            }
        }
        cp_async_commit();  // one group per row, empty when nothing was copied, so the count stays uniform
    };
#pragma unroll
    for (int u = 0; u < CO_NST - 1; ++u) issue(u);
    float lo[4][4], d[4][4];
    hrow(0, lo);  // low-res row jb - 1
    for (int t = 0; t <= NB; ++t) {
        // run t samples tile rows t, t + 1: the previous run's lower row becomes the upper one
        if (t > 0) {
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int x = 0; x < 4; ++x) lo[m][x] += d[m][x];
        }
        hrow(t + 1, d);
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int x = 0; x < 4; ++x) d[m][x] -= lo[m][x];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const int u = t * S + k, Y = Ys + u;
            issue(u + CO_NST - 1);
            cp_async_wait_group<CO_NST - 1>();  // this thread's copies of row u have landed
            if (Y < Yb || Y >= Ye) continue;
            float gv[3][4];
#pragma unroll
            for (int p = 0; p < 3; ++p) ld4_ring<TI>(slot(k % CO_NST, p), gv[p]);  // u % CO_NST == k % CO_NST
            const float fy = (float)(2 * k + 1) * (1.0f / (float)(2 * S));
            float out[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                float mm[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) mm[m] = fmaf(fy, d[m][x], lo[m][x]);
                out[x] = fmaf(mm[0], gv[0][x], fmaf(mm[1], gv[1][x], fmaf(mm[2], gv[2][x], mm[3])));
            }
            if (detail != 0.0f) {  // C == 3: channel c's own guide channel is its detail source
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const float iv = (c == 0) ? gv[0][x] : (c == 1 ? gv[1][x] : gv[2][x]);
                    out[x] = fmaf(detail, iv - out[x], out[x]);
                }
            }
            st4g<TQ>(qc + (size_t)Y * W, true, 4, out);
        }
    }
    cp_async_wait_all();
}

int blocks_for(size_t items) { return (int)std::min<size_t>((items + COL_NT - 1) / COL_NT, 152 * 8); }

}  // namespace

cudaError_t launch_color_products(const FwdPlan &P, cudaStream_t st)
{
    dim3 grid(blocks_for((size_t)P.h * P.w), P.N);
    k_color_products<<<grid, COL_NT, 0, st>>>(P.Il, P.pl, P.col[0], P.col[1], P.C, P.h, P.w, P.lps);
    return cudaGetLastError();
}

cudaError_t launch_color_coef(const FwdPlan &P, cudaStream_t st)
{
    dim3 grid(blocks_for((size_t)P.h * P.w), P.N);
    k_color_coef<<<grid, COL_NT, 0, st>>>(P.Il, P.pl, P.col[2], P.col[3], P.col[4], P.col[5], P.C, P.h, P.w, P.lps,
                                         P.eps);
    return cudaGetLastError();
}

cudaError_t launch_color_output(const FwdPlan &P, cudaStream_t st)
{
    const int R = 8 * P.s;
    // tap rows / columns under R rows / CO_BAND columns: at most ceil((n - 1)/s) + 2 <= ceil(n/s) + 2
    const int LR = (R + P.s - 1) / P.s + 2, LCmax = (CO_BAND + P.s - 1) / P.s + 2;
    const size_t smem = (size_t)4 * LR * LCmax * sizeof(float) + (size_t)CO_NST * 3 * CO_NT * 4 * dtype_size(P.dt_in);
    const int bands = (P.W + CO_BAND - 1) / CO_BAND;
    dim3 grid(bands * P.C, (P.H + R - 1) / R, P.N);
    // ring copies and 128-bit stores need every row of every plane on a vector boundary
    const size_t vb = 4 * dtype_size(P.dt_in);
    const bool vec_io = (P.W % 4 == 0) && (P.fps % 4 == 0) && ((uintptr_t)P.I % vb == 0) && ((uintptr_t)P.q % 16 == 0);
    cudaError_t e;
    if (vec_io && (P.s == 4 || P.s == 8)) {  // the run form
        constexpr int NB = 8;
        const int LRr = NB + 2, LCr = CO_BAND / P.s + 2;
        const size_t smem_r = (size_t)4 * LRr * LCr * sizeof(float) + (size_t)CO_NST * 3 * CO_NT * 4 * dtype_size(P.dt_in);
        dim3 grid_r(bands * P.C, (P.h + NB - 1) / NB, P.N);
#define GF_COR(TI, TQ, SS)                                                                                        \
    do {                                                                                                          \
        if ((e = opt_in_smem(k_color_output_s4x<TI, TQ, SS>, smem_r)) != cudaSuccess) return e;                  \
        k_color_output_s4x<TI, TQ, SS><<<grid_r, CO_NT, smem_r, st>>>((const TI *)P.I, (TQ *)P.q, P.col[6], P.col[7], \
                                                                     P.C, P.H, P.W, P.h, P.w, P.fps, P.lps, LRr, LCr,  \
                                                                     P.Yw0, P.Yw1, P.detail);                        \
    } while (0)
#define GF_COS(TI, TQ) do { if (P.s == 4) GF_COR(TI, TQ, 4); else GF_COR(TI, TQ, 8); } while (0)
        if (P.dt_in == F32) {
            if (P.dt_out == F32) GF_COS(float, float); else GF_COS(float, __half);
        } else {
            if (P.dt_out == F32) GF_COS(__half, float); else GF_COS(__half, __half);
        }
#undef GF_COS
#undef GF_COR
        return cudaGetLastError();
    }
#define GF_CO(TI, TQ)                                                                                            \
    do {                                                                                                         \
        if ((e = opt_in_smem(k_color_output<TI, TQ>, smem)) != cudaSuccess) return e;                          \
        k_color_output<TI, TQ><<<grid, CO_NT, smem, st>>>((const TI *)P.I, (TQ *)P.q, P.col[6], P.col[7], P.C, P.H, \
                                                          P.W, P.h, P.w, P.s, P.fps, P.lps, R, LCmax, P.Yw0,     \
                                                          P.Yw1, P.detail, vec_io);                              \
    } while (0)
    if (P.dt_in == F32) {
        if (P.dt_out == F32) GF_CO(float, float); else GF_CO(float, __half);
    } else {
        if (P.dt_out == F32) GF_CO(__half, float); else GF_CO(__half, __half);
    }
#undef GF_CO
    return cudaGetLastError();
}

}  // namespace gfk
