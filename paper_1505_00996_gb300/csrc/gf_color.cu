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
//                     conventions) and q = mean_a^T I + mean_b, plus the optional detail epilogue.
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

// Thread = 4 adjacent pixels of one row band and one channel; CTA = COL_NT threads along a row.
template <typename TI, typename TQ>
__global__ void __launch_bounds__(COL_NT) k_color_output(const TI *__restrict__ I, TQ *__restrict__ q,
                                                         const float *__restrict__ MX, const float *__restrict__ MY,
                                                         int C, int H, int W, int h, int w, int s, size_t fps,
                                                         size_t lps, int R, int Yw0, int Yw1, float detail,
                                                         bool vec_io)
{
    const int X0 = (blockIdx.x * COL_NT + threadIdx.x) * 4;
    if (X0 >= W) return;
    const int valid = min(4, W - X0);
    const int c = blockIdx.z % C, n = blockIdx.z / C;
    const int Yb = max((int)blockIdx.y * R, Yw0), Ye = min(min((int)blockIdx.y * R + R, H), Yw1);
    const bool vec = vec_io && (valid == 4);
    const float *mx = MX + ((size_t)n * 2 * C + 2 * c) * lps, *my = MY + ((size_t)n * 2 * C + 2 * c) * lps;
    const float *maps[4] = {mx, my, mx + lps, my + lps};  // mean of a_r, a_g, a_b, b
    int xa[4], xb[4];
    float fx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) up_taps(min(X0 + k, W - 1), s, w, xa[k], xb[k], fx[k]);
    const TI *Ig = I + (size_t)n * 3 * fps + X0;
    TQ *qc = q + ((size_t)n * C + c) * fps + X0;
    for (int Y = Yb; Y < Ye; ++Y) {
        int ya, yb;
        float fy;
        up_taps(Y, s, h, ya, yb, fy);
        float m[4][4];  // [map][pixel]
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float *r0 = maps[k] + (size_t)ya * w, *r1 = maps[k] + (size_t)yb * w;
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const float t0 = fmaf(fx[x], r0[xb[x]] - r0[xa[x]], r0[xa[x]]);
                const float t1 = fmaf(fx[x], r1[xb[x]] - r1[xa[x]], r1[xa[x]]);
                m[k][x] = fmaf(fy, t1 - t0, t0);
            }
        }
        float ir[4], ig[4], ib[4], out[4];
        const size_t row = (size_t)Y * W;
        ld4g<TI>(Ig + row, vec, valid, ir);
        ld4g<TI>(Ig + fps + row, vec, valid, ig);
        ld4g<TI>(Ig + 2 * fps + row, vec, valid, ib);
#pragma unroll
        for (int x = 0; x < 4; ++x) out[x] = fmaf(m[0][x], ir[x], fmaf(m[1][x], ig[x], fmaf(m[2][x], ib[x], m[3][x])));
        if (detail != 0.0f) {  // C == 3: channel c's own guide channel is its detail source
            const float *iv = (c == 0) ? ir : (c == 1 ? ig : ib);
#pragma unroll
            for (int x = 0; x < 4; ++x) out[x] = fmaf(detail, iv[x] - out[x], out[x]);
        }
        st4g<TQ>(qc + row, vec, valid, out);
    }
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
    const int R = 16;
    dim3 grid((P.W + 4 * COL_NT - 1) / (4 * COL_NT), (P.H + R - 1) / R, P.N * P.C);
    // 128-bit loads and stores need every row of every plane on a 16-byte boundary (FP32 only)
    const bool vec_io = (P.W % 4 == 0) && (P.fps % 4 == 0) && ((uintptr_t)P.I % 16 == 0) && ((uintptr_t)P.q % 16 == 0);
#define GF_CO(TI, TQ)                                                                                          \
    k_color_output<TI, TQ><<<grid, COL_NT, 0, st>>>((const TI *)P.I, (TQ *)P.q, P.col[6], P.col[7], P.C, P.H, P.W, \
                                                    P.h, P.w, P.s, P.fps, P.lps, R, P.Yw0, P.Yw1, P.detail, vec_io)
    if (P.dt_in == F32) {
        if (P.dt_out == F32) GF_CO(float, float); else GF_CO(float, __half);
    } else {
        if (P.dt_out == F32) GF_CO(__half, float); else GF_CO(__half, __half);
    }
#undef GF_CO
    return cudaGetLastError();
}

}  // namespace gfk
