// gf_backward.cu -- sm_103a kernels of the backward pass (the exact derivative) of Algorithm 2 of He and Sun,
// "Fast Guided Filter" (2015).  The paper has no backward pass; this is the adjoint of the forward chain in
// gf_forward.cu, operator by operator.  With g = dL/dq for channel c and guide channel I_g:
//
//   q = U(mean_a) .* I + U(mean_b)          -> dI += g .* U(mean_a);  dMA = U^T(g .* I);  dMB = U^T(g)
//   mean_a = B(a), mean_b = B(b)            -> da = B^T(dMA),  db = B^T(dMB)
//   b = mean_p - a .* mean_I                -> dmp = db;  da -= mean_I .* db;  dmI = -a .* db
//   a = cov / (var + eps)                   -> dcov = da / (var+eps);  dvar = -da .* a / (var+eps);  deps += sum dvar
//   var = corr_I - mean_I.^2, cov = corr_Ip - mean_I .* mean_p
//                                           -> dcII = dvar;  dcIp = dcov;  dmI -= 2 mean_I dvar + mean_p dcov;
//                                              dmp -= mean_I dcov
//   mean_I = B(I'), mean_p = B(p'), corr_I = B(I'.*I'), corr_Ip = B(I'.*p')
//                                           -> dI' = B^T(dmI) + 2 I' B^T(dcII) + p' B^T(dcIp);
//                                              dp' = B^T(dmp) + I' B^T(dcIp)
//   I' = D(I), p' = D(p)                    -> dI += D^T(dI');  dp = D^T(dp')
//
// B^T of the border-normalised box mean is B^T(y)_i = sum over windows k containing i of y_k / n_k, i.e. the
// box SUM of y ./ n (n_k: in-image pixel count of window k) -- not B itself at the borders.  U^T and D^T are
// the transposed bilinear / subsample maps, evaluated as gathers (no atomics).
//
//   k_bwd_upsample_T   dMA, dMB: per low-res tile, a horizontal gather of g.*I and g into a shared table of
//                      full-res rows x low-res columns, then a vertical gather.  k_bwd_upsample_T_w is the
//                      form for s = 4, 8 (H, W multiples of s): each lane reads one s-pixel block of a row
//                      with vector loads, the three columns it reaches are summed across lanes by warp
//                      shuffles, and each warp walks down its rows keeping three low-res row sums in registers.
//   k_bwd_box_T        B^T of 2 maps with the chain epilogue (4 maps out, per-CTA partial sums of deps), or
//                      B^T of 4 maps with the final combination into dI', dp'.  Same tiling as k_box_tile;
//                      the epilogue runs in the write-out phase, a thread per pixel, so the forward planes it
//                      reads (statistics, a, I', p') are read coalesced.
//   k_bwd_full         full-res: dI = sum_c g_c U(mean_a_c) + D^T(dI'), dp = D^T(dp'); k_bwd_full_v is its
//                      4-pixel vector form for s = 4, 8 (H, W multiples of s), where D^T is block-local.
//   k_reduce_eps       deterministic sum of the per-CTA deps partials (FP64 accumulation).
#include <algorithm>

#include "gf_device.cuh"
#include "gf_internal.cuh"

namespace gfk {

// ------------------------------------------------------------------------------------------------------
// k_bwd_upsample_T
// ------------------------------------------------------------------------------------------------------
constexpr int UT_NT = 256;
constexpr int UT_TI = 32;  // low-res columns per tile

struct UpTParams {
    const float *g;   // dL/dq, N x C x H x W
    const float *I;   // guide, N x CI x H x W
    float *dma, *dmb; // out: N x C planes of stride lps
    int C, CI, H, W, h, w, s, TJ;
    size_t lps;
};

__device__ __forceinline__ float up_weight(int X, int i, int s, int n)
{
    int i0, i1;
    float f;
    up_taps(X, s, n, i0, i1, f);
    return (i0 == i ? 1.0f - f : 0.0f) + (i1 == i ? f : 0.0f);
}

__global__ void __launch_bounds__(UT_NT) k_bwd_upsample_T(UpTParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    extern __shared__ float sm[];
    const int s = P.s, TJ = P.TJ;
    const int i0 = blockIdx.x * UT_TI, j0 = blockIdx.y * TJ;
    const int plane = blockIdx.z, n = plane / P.C, c = plane - n * P.C;
    const size_t HW = (size_t)P.H * P.W;
    const float *g = P.g + (size_t)plane * HW;
    const float *I = P.I + (size_t)(n * P.CI + (P.CI == 1 ? 0 : c)) * HW;
    const int ncand = 3 * s;                 // candidate full-res positions per low-res index
    const int Y0 = max(0, s * (j0 - 1)), Y1 = min(P.H, s * (j0 + TJ + 1));
    const int NR = Y1 - Y0;
    float *Tga = sm;                         // [NR][UT_TI] horizontal gathers of g .* I
    float *Tg = Tga + (size_t)NR * UT_TI;    // [NR][UT_TI] horizontal gathers of g
    float *wx = Tg + (size_t)NR * UT_TI;     // [UT_TI][ncand] weights of X = s(i-1) + t onto column i
    float *wy = wx + UT_TI * ncand;          // [TJ][ncand] weights of Y = s(j-1) + t onto row j
    for (int k = threadIdx.x; k < UT_TI * ncand; k += UT_NT) {
        const int il = k / ncand, t = k - il * ncand;
        const int i = i0 + il, X = s * (i - 1) + t;
        wx[k] = (i < P.w && X >= 0 && X < P.W) ? up_weight(X, i, s, P.w) : 0.0f;
    }
    for (int k = threadIdx.x; k < TJ * ncand; k += UT_NT) {
        const int jl = k / ncand, t = k - jl * ncand;
        const int j = j0 + jl, Y = s * (j - 1) + t;
        wy[k] = (j < P.h && Y >= 0 && Y < P.H) ? up_weight(Y, j, s, P.h) : 0.0f;
    }
    __syncthreads();
    // horizontal gather: T[y][i] = sum_X wx(X -> i) v(y, X)
    for (int k = threadIdx.x; k < NR * UT_TI; k += UT_NT) {
        const int yl = k / UT_TI, il = k - yl * UT_TI;
        const int i = i0 + il;
        float sga = 0.0f, sg = 0.0f;
        if (i < P.w) {
            const size_t ro = (size_t)(Y0 + yl) * P.W;
            const int xb = s * (i - 1);
            for (int t = 0; t < ncand; ++t) {
                const float wgt = wx[il * ncand + t];
                if (wgt != 0.0f) {
                    const float gv = __ldg(g + ro + xb + t);
                    sg = fmaf(wgt, gv, sg);
                    sga = fmaf(wgt, gv * __ldg(I + ro + xb + t), sga);
                }
            }
        }
        Tga[k] = sga;
        Tg[k] = sg;
    }
    __syncthreads();
    // vertical gather: dM[j][i] = sum_y wy(y -> j) T[y][i]
    for (int k = threadIdx.x; k < TJ * UT_TI; k += UT_NT) {
        const int jl = k / UT_TI, il = k - jl * UT_TI;
        const int j = j0 + jl, i = i0 + il;
        if (j >= P.h || i >= P.w) continue;
        float sa = 0.0f, sb = 0.0f;
        const int yb = s * (j - 1);
        for (int t = 0; t < ncand; ++t) {
            const float wgt = wy[jl * ncand + t];
            if (wgt != 0.0f) {
                const int yl = yb + t - Y0;
                sa = fmaf(wgt, Tga[yl * UT_TI + il], sa);
                sb = fmaf(wgt, Tg[yl * UT_TI + il], sb);
            }
        }
        const size_t o = (size_t)plane * P.lps + (size_t)j * P.w + i;
        P.dma[o] = sa;
        P.dmb[o] = sb;
    }
    pdl_trigger();
}

// Interior weights of the bilinear upsample for an even integer s: pixel t of block i lies between low-res
// columns i - 1 and i at weight f_t of column i when t < s/2 (f_t = (2t + 1 + s)/(2s)), and between i and i + 1
// at weight f_t = (2t + 1 - s)/(2s) of column i + 1 when t >= s/2.
template <int S>
__host__ __device__ constexpr float up_f(int t)
{
    return (float)(2 * t + 1 - S + (2 * t + 1 < S ? 2 * S : 0)) / (float)(2 * S);
}
// weight with which pixel t of block i + b (b = -1, 0, 1) reaches low-res index i (interior)
template <int S>
__host__ __device__ constexpr float up_wT(int b, int t)
{
    return b < 0 ? (2 * t + 1 > S ? up_f<S>(t) : 0.0f)
                 : b == 0 ? (2 * t + 1 < S ? up_f<S>(t) : 1.0f - up_f<S>(t))
                          : (2 * t + 1 < S ? 1.0f - up_f<S>(t) : 0.0f);
}

template <int N>
__device__ __forceinline__ void ld_vec(const float *p, float (&v)[N])
{
    static_assert(N == 2 || N % 4 == 0, "float2 or float4 pieces");
    if constexpr (N == 2) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p + 4 * q));
            v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
        }
    }
}

// Walking form of U^T for s = 4, 8 (H and W multiples of s, 16-byte aligned planes).  Under the bilinear
// upsample, pixel t of block i reaches low-res column i - 1 with weight up_wT(1, t) (first half only), column i
// with up_wT(0, t) and column i + 1 with up_wT(-1, t) (second half only); rows likewise.  Lane l of a warp reads
// block i = i0 - 1 + l of a full-res row with vector loads and forms its three partial sums L, M, R; column i
// then totals M_i + R_{i-1} + L_{i+1}, the neighbours' parts arriving by warp shuffles.  Lanes 0 and 31 only
// supply those parts for the tile's outer columns, so a warp produces UW_TI = 30 columns.  The warp walks down
// its TJ low-res rows keeping the row sums of rows j - 1, j, j + 1 in registers (no shared memory, no block
// barrier): after block row j is read, row j - 1 is complete and is stored.  At the image's first and last
// column (row) the upsample's taps are clamped, so the half block that would reach column -1 (or w) reaches
// the edge column with weight 1 instead: the part is folded into M there.
constexpr int UW_WARPS = 4;   // warps per CTA, each on its own TJ low-res rows
constexpr int UW_TI = 30;     // low-res columns per warp (lanes 1 .. 30)

template <int S>
__global__ void __launch_bounds__(32 * UW_WARPS) k_bwd_upsample_T_w(UpTParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    static_assert(S % 4 == 0, "whole float4 pieces per block");
    constexpr int HS = S / 2;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ja = (blockIdx.y * UW_WARPS + warp) * P.TJ;
    if (ja >= P.h) return;  // the whole warp: nothing below waits on the other warps
    const int je = min(P.h, ja + P.TJ);
    const int i = blockIdx.x * UW_TI - 1 + lane;  // the block this lane reads
    const int plane = blockIdx.z, n = plane / P.C, c = plane - n * P.C;
    const size_t HW = (size_t)P.H * P.W;
    const float *g = P.g + (size_t)plane * HW + (size_t)S * max(i, 0);
    const float *I = P.I + (size_t)(n * P.CI + (P.CI == 1 ? 0 : c)) * HW + (size_t)S * max(i, 0);
    const bool col_ok = i >= 0 && i < P.w;
    const bool first = i == 0, last = i == P.w - 1;
    const bool store = lane >= 1 && lane <= UW_TI && col_ok;
    float pa = 0.0f, pg = 0.0f, ca = 0.0f, cg = 0.0f;  // sums of low-res rows jb - 1 and jb
    for (int jb = ja - 1; jb <= je; ++jb) {
        float na = 0.0f, ng = 0.0f;                    // sums of low-res row jb + 1
        const bool blk = jb >= 0 && jb < P.h;
#pragma unroll
        for (int t = 0; t < S; ++t) {
            // block row ja - 1 gives only its second half, block row je only its first half (warp-uniform)
            if (!blk || (jb < ja && t < HS) || (jb == je && t >= HS)) continue;
            float gv[S], Iv[S];
            if (col_ok) {
                const size_t ro = (size_t)(S * jb + t) * P.W;
                ld_vec<S>(g + ro, gv);
                ld_vec<S>(I + ro, Iv);
            } else {
#pragma unroll
                for (int u = 0; u < S; ++u) gv[u] = Iv[u] = 0.0f;
            }
            float La = 0.0f, Lg = 0.0f, Ma = 0.0f, Mg = 0.0f, Ra = 0.0f, Rg = 0.0f;
#pragma unroll
            for (int u = 0; u < S; ++u) {
                const float a = gv[u] * Iv[u];
                if (u < HS) {
                    La = fmaf(up_wT<S>(1, u), a, La);
                    Lg = fmaf(up_wT<S>(1, u), gv[u], Lg);
                } else {
                    Ra = fmaf(up_wT<S>(-1, u), a, Ra);
                    Rg = fmaf(up_wT<S>(-1, u), gv[u], Rg);
                }
                Ma = fmaf(up_wT<S>(0, u), a, Ma);
                Mg = fmaf(up_wT<S>(0, u), gv[u], Mg);
            }
            if (first) { Ma += La; Mg += Lg; }
            if (last) { Ma += Ra; Mg += Rg; }
            const float Ta = Ma + __shfl_up_sync(FULL, Ra, 1) + __shfl_down_sync(FULL, La, 1);
            const float Tg = Mg + __shfl_up_sync(FULL, Rg, 1) + __shfl_down_sync(FULL, Lg, 1);
            if (t < HS) {
                pa = fmaf(up_wT<S>(1, t), Ta, pa);
                pg = fmaf(up_wT<S>(1, t), Tg, pg);
            } else {
                na = fmaf(up_wT<S>(-1, t), Ta, na);
                ng = fmaf(up_wT<S>(-1, t), Tg, ng);
            }
            ca = fmaf(up_wT<S>(0, t), Ta, ca);
            cg = fmaf(up_wT<S>(0, t), Tg, cg);
        }
        if (jb == 0) { ca += pa; cg += pg; }
        if (jb == P.h - 1) { ca += na; cg += ng; }
        if (jb - 1 >= ja && store) {  // low-res row jb - 1 has all its rows now
            const size_t o = (size_t)plane * P.lps + (size_t)(jb - 1) * P.w + i;
            P.dma[o] = pa;
            P.dmb[o] = pg;
        }
        pa = ca; pg = cg;
        ca = na; cg = ng;
    }
    pdl_trigger();
}

// ------------------------------------------------------------------------------------------------------
// k_bwd_box_T
// ------------------------------------------------------------------------------------------------------
constexpr int BB_NT = 256;
constexpr int BB_TH = 32;
constexpr int BB_TW = 64;
constexpr int BB_RV = 8;
constexpr int BB_RH = 8;
constexpr int BB_VP = BB_TH + 1;
constexpr int BB_OP = BB_TW + 1;

enum { EPI_CHAIN = 0, EPI_COMBINE = 1 };

struct BoxTParams {
    const float *in[4];  // input maps (N x C planes of stride lps each)
    float *out[4];       // output maps (N x C planes of stride lps each)
    size_t lps;
    int C, CI, h, w, r;
    float eps;
    // chain epilogue: forward statistics (dense h*w planes, 4 per (n, c)) and a (stride lps)
    const float *stats, *a;
    float *eps_partial;  // one partial sum of dvar per CTA
    // combine epilogue: I' (plane index n*CI + guide) and p' (plane index n*C + c), plane stride xps / yps
    const float *Il, *pl;
    size_t xps, yps;
};

__device__ __forceinline__ int win_count(int k, int r, int n) { return min(n - 1, k + r) - max(0, k - r) + 1; }

template <int NIN, int EPI, bool COMP, int RC = 0>
__global__ void __launch_bounds__(BB_NT) k_bwd_box_T(BoxTParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    static_assert(RC == 0 || !COMP, "a compile-time radius is for the small, uncompensated windows");
    constexpr int NOUT = (EPI == EPI_CHAIN) ? 4 : 2;
    extern __shared__ float smf[];
    __shared__ float red[BB_NT / 32];
    const int tid = threadIdx.x;
    const int h = P.h, w = P.w, r = RC > 0 ? RC : P.r;
    const int span = BB_TW + 2 * r;
    float *Vt = smf;                                 // [NIN][span][BB_VP]
    float *Ot = smf;                                 // [NIN][BB_TH][BB_OP] window sums, over Vt after phase 2
    const int x0 = blockIdx.x * BB_TW, y0 = blockIdx.y * BB_TH;
    const int plane = blockIdx.z;
    const size_t pbase = (size_t)plane * P.lps;

    // ---- phase 1: vertical sums of in ./ n (n: pixel count of the window centred at each pixel)
    for (int item = tid; item < span * (BB_TH / BB_RV); item += BB_NT) {
        const int xc = item % span, seg = item / span;
        const int gx = x0 - r + xc, ya = y0 + seg * BB_RV, vrow = seg * BB_RV;
        float S[NIN], Sc[NIN];
#pragma unroll
        for (int q = 0; q < NIN; ++q) { S[q] = 0.0f; Sc[q] = 0.0f; }
        if constexpr (RC > 0) {
            // radius known at compile time: the RV + 2 RC scaled rows of the segment's window span are requested
            // at once into registers (rows outside the image count as zero), then slid over
            if (gx >= 0 && gx < w && ya < h) {
                constexpr int NR = BB_RV + 2 * RC;
                const float inx = __fdividef(1.0f, (float)win_count(gx, RC, w));
                float v[NR][NIN];
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const int yy = ya - RC + k;
                    const bool ok = yy >= 0 && yy < h;
                    const float sc = ok ? inx * __fdividef(1.0f, (float)win_count(yy, RC, h)) : 0.0f;
                    const size_t o = pbase + (size_t)(ok ? yy : 0) * w + gx;
#pragma unroll
                    for (int q = 0; q < NIN; ++q) v[k][q] = ok ? sc * __ldg(P.in[q] + o) : 0.0f;
                }
#pragma unroll
                for (int k = 0; k <= 2 * RC; ++k)
#pragma unroll
                    for (int q = 0; q < NIN; ++q) S[q] += v[k][q];
#pragma unroll
                for (int i = 0; i < BB_RV; ++i) {
                    if (i > 0) {
#pragma unroll
                        for (int q = 0; q < NIN; ++q) S[q] = (S[q] + v[i + 2 * RC][q]) - v[i - 1][q];
                    }
#pragma unroll
                    for (int q = 0; q < NIN; ++q) Vt[((size_t)q * span + xc) * BB_VP + vrow + i] = S[q];
                }
            } else {
#pragma unroll
                for (int i = 0; i < BB_RV; ++i)
#pragma unroll
                    for (int q = 0; q < NIN; ++q) Vt[((size_t)q * span + xc) * BB_VP + vrow + i] = 0.0f;
            }
            continue;
        }
        if (gx >= 0 && gx < w && ya < h) {
            const float inx = __fdividef(1.0f, (float)win_count(gx, r, w));
            auto add_row = [&](int yy, float sign) {
                const float sc = sign * inx * __fdividef(1.0f, (float)win_count(yy, r, h));
                const size_t o = pbase + (size_t)yy * w + gx;
#pragma unroll
                for (int q = 0; q < NIN; ++q) {
                    const float v = sc * __ldg(P.in[q] + o);
                    if (COMP) {
                        const float t = S[q] + v;
                        Sc[q] += (fabsf(S[q]) >= fabsf(v)) ? ((S[q] - t) + v) : ((v - t) + S[q]);
                        S[q] = t;
                    } else {
                        S[q] += v;
                    }
                }
            };
            for (int yy = max(0, ya - r); yy <= min(h - 1, ya + r); ++yy) add_row(yy, 1.0f);
#pragma unroll
            for (int i = 0; i < BB_RV; ++i) {
                const int y = ya + i;
                if (i > 0) {
                    if (y + r < h) add_row(y + r, 1.0f);
                    if (y - r - 1 >= 0) add_row(y - r - 1, -1.0f);
                }
#pragma unroll
                for (int q = 0; q < NIN; ++q) Vt[((size_t)q * span + xc) * BB_VP + vrow + i] = S[q] + Sc[q];
            }
        } else {
#pragma unroll
            for (int i = 0; i < BB_RV; ++i)
#pragma unroll
                for (int q = 0; q < NIN; ++q) Vt[((size_t)q * span + xc) * BB_VP + vrow + i] = 0.0f;
        }
    }
    __syncthreads();

    // ---- phase 2: horizontal sums, one row segment per thread; the sums wait in registers until every thread
    // has read the column sums, then go to a staging tile over them
    static_assert(BB_TH * (BB_TW / BB_RH) <= BB_NT, "one phase-2 item per thread");
    float O[NIN][BB_RH];
    {
        const int yr = tid % BB_TH, seg = tid / BB_TH;
        const int y = y0 + yr, xa = seg * BB_RH;
        const bool item = tid < BB_TH * (BB_TW / BB_RH) && y < h && x0 + xa < w;
        if (item) {
            float S[NIN], Sc[NIN];
#pragma unroll
            for (int q = 0; q < NIN; ++q) { S[q] = 0.0f; Sc[q] = 0.0f; }
            auto vacc = [&](int col, float sign) {
#pragma unroll
                for (int q = 0; q < NIN; ++q) {
                    const float v = sign * Vt[((size_t)q * span + col) * BB_VP + yr];
                    if (COMP) {
                        const float t = S[q] + v;
                        Sc[q] += (fabsf(S[q]) >= fabsf(v)) ? ((S[q] - t) + v) : ((v - t) + S[q]);
                        S[q] = t;
                    } else {
                        S[q] += v;
                    }
                }
            };
            for (int k = 0; k <= 2 * r; ++k) vacc(xa + k, 1.0f);
#pragma unroll
            for (int i = 0; i < BB_RH; ++i) {
                if (x0 + xa + i >= w) break;
                if (i > 0) {
                    vacc(xa + i + 2 * r, 1.0f);
                    vacc(xa + i - 1, -1.0f);
                }
#pragma unroll
                for (int q = 0; q < NIN; ++q) O[q][i] = S[q] + Sc[q];
            }
        }
        __syncthreads();  // every column sum has been read
        if (item) {
#pragma unroll
            for (int i = 0; i < BB_RH; ++i) {
                if (x0 + xa + i >= w) break;
#pragma unroll
                for (int q = 0; q < NIN; ++q) Ot[(q * BB_TH + yr) * BB_OP + xa + i] = O[q][i];
            }
        }
    }
    __syncthreads();

    // ---- phase 3: the epilogue, thread per output pixel (coalesced reads of the forward planes and writes)
    float eps_acc = 0.0f;
    const int n = plane / P.C, c = plane - n * P.C;
    for (int idx = tid; idx < BB_TH * BB_TW; idx += BB_NT) {
        const int yr = idx / BB_TW, xt = idx - yr * BB_TW;
        const int y = y0 + yr, x = x0 + xt;
        if (y >= h || x >= w) continue;
        const size_t pix = (size_t)y * w + x;
        float t[NIN];
#pragma unroll
        for (int q = 0; q < NIN; ++q) t[q] = Ot[(q * BB_TH + yr) * BB_OP + xt];
        float o[NOUT];
        if (EPI == EPI_CHAIN) {
            const float da0 = t[0], db = t[1];  // B^T(dMA), B^T(dMB)
            const size_t ps = (size_t)h * w;
            const float *st = P.stats + (size_t)plane * 4 * ps + pix;
            const float mI = st[0], cI = st[ps], mp = st[2 * ps];
            const float a = P.a[pbase + pix];
            const float var = fmaxf(cI - mI * mI, 0.0f);
            const float inv = 1.0f / (var + P.eps);
            const float da = da0 - mI * db;          // through b = mean_p - a mean_I
            const float dcov = da * inv;              // through a = cov / (var + eps)
            const float dvar = -da * a * inv;
            eps_acc += dvar;
            o[0] = -a * db - 2.0f * mI * dvar - mp * dcov;  // d mean_I
            o[1] = dvar;                                    // d corr_I
            o[2] = dcov;                                    // d corr_Ip
            o[3] = db - mI * dcov;                          // d mean_p
        } else {
            const float tmI = t[0], tcII = t[1], tcIp = t[2], tmp = t[3];
            const float Iv = P.Il[(size_t)(n * P.CI + (P.CI == 1 ? 0 : c)) * P.xps + pix];
            const float pv = P.pl[(size_t)plane * P.yps + pix];
            o[0] = tmI + 2.0f * Iv * tcII + pv * tcIp;  // dI'
            o[1] = tmp + Iv * tcIp;                     // dp'
        }
#pragma unroll
        for (int q = 0; q < NOUT; ++q) P.out[q][pbase + pix] = o[q];
    }
    if (EPI == EPI_CHAIN) {
        // deterministic CTA reduction of the deps contributions
        for (int off = 16; off > 0; off >>= 1) eps_acc += __shfl_xor_sync(0xffffffffu, eps_acc, off);
        if ((tid & 31) == 0) red[tid >> 5] = eps_acc;
        __syncthreads();
        if (tid == 0) {
            float tt = 0.0f;
            for (int k = 0; k < BB_NT / 32; ++k) tt += red[k];
            P.eps_partial[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tt;
        }
    }
    pdl_trigger();
}

// ------------------------------------------------------------------------------------------------------
// k_bwd_full
// ------------------------------------------------------------------------------------------------------
constexpr int BF_NT = 256;

struct FullParams {
    const float *g;            // N x C x H x W
    const float *ma;           // mean_a, N x C planes of stride lps
    const float *dIl, *dpl;    // dI', dp' per channel, N x C planes of stride lps
    float *dI;                 // N x CI x H x W
    float *dp;                 // N x C x H x W, or NULL when p is low-res
    int C, CI, H, W, h, w, s, mode;
    size_t lps;
};

// Weights with which full-res index Y receives from low-res indices j in {Y/s - 1, Y/s, Y/s + 1} under the
// transposed subsample (the gather form of D^T).
__device__ __forceinline__ void sub_adjoint(int Y, int s, int H, int h, int mode, int j[3], float wgt[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int jj = Y / s - 1 + k;
        j[k] = min(max(jj, 0), h - 1);
        float wv = 0.0f;
        if (jj >= 0 && jj < h) {
            if (mode == GF_SUB_BOX && s > 1) {
                const int a = jj * s, b = min(a + s, H);
                wv = (Y >= a && Y < b) ? 1.0f / (float)(b - a) : 0.0f;
            } else {
                int t0, t1;
                float f;
                sub_taps(jj, s, H, mode, t0, t1, f);
                wv = (t0 == Y ? 1.0f - f : 0.0f) + (t1 == Y ? f : 0.0f);
            }
        }
        wgt[k] = wv;
    }
}

__global__ void __launch_bounds__(BF_NT) k_bwd_full(FullParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    const int X = blockIdx.x * BF_NT + threadIdx.x, Y = blockIdx.y, n = blockIdx.z;
    if (X >= P.W) return;
    const size_t HW = (size_t)P.H * P.W, pix = (size_t)Y * P.W + X;
    int ya, yb, xa, xb;
    float fy, fx;
    up_taps(Y, P.s, P.h, ya, yb, fy);
    up_taps(X, P.s, P.w, xa, xb, fx);
    int jy[3], ix[3];
    float wy[3], wx[3];
    sub_adjoint(Y, P.s, P.H, P.h, P.mode, jy, wy);
    sub_adjoint(X, P.s, P.W, P.w, P.mode, ix, wx);
    float dI_shared = 0.0f;
    for (int c = 0; c < P.C; ++c) {
        const size_t lp = (size_t)(n * P.C + c) * P.lps;
        const float *ma = P.ma + lp;
        const float A0 = fmaf(fx, __ldg(ma + (size_t)ya * P.w + xb) - __ldg(ma + (size_t)ya * P.w + xa), __ldg(ma + (size_t)ya * P.w + xa));
        const float A1 = fmaf(fx, __ldg(ma + (size_t)yb * P.w + xb) - __ldg(ma + (size_t)yb * P.w + xa), __ldg(ma + (size_t)yb * P.w + xa));
        const float A = fmaf(fy, A1 - A0, A0);                        // U(mean_a)
        const float gv = __ldg(P.g + (size_t)(n * P.C + c) * HW + pix);
        float tI = 0.0f, tp = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (wy[a] == 0.0f) continue;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (wx[b] == 0.0f) continue;
                const size_t o = lp + (size_t)jy[a] * P.w + ix[b];
                const float wv = wy[a] * wx[b];
                tI = fmaf(wv, __ldg(P.dIl + o), tI);
                if (P.dp) tp = fmaf(wv, __ldg(P.dpl + o), tp);
            }
        }
        const float dIc = fmaf(gv, A, tI);                            // direct term + D^T(dI')
        if (P.CI == 1) dI_shared += dIc;
        else P.dI[(size_t)(n * P.CI + c) * HW + pix] = dIc;
        if (P.dp) P.dp[(size_t)(n * P.C + c) * HW + pix] = tp;        // D^T(dp')
    }
    if (P.CI == 1) P.dI[(size_t)n * HW + pix] = dI_shared;
    pdl_trigger();
}

// Vector form of k_bwd_full for s = 4, 8 with H and W multiples of s and 16-byte aligned planes.  Then every
// transposed-subsample weight of a full-res pixel comes from its own s x s block -- the block's mean (box),
// its centre pixel (nearest) or its central 2 x 2 (bilinear at even s) -- with weight wsub(Y mod s) *
// wsub(X mod s).  A thread owns 4 adjacent pixels of one row, all in one block: it reads g as float4, takes
// the block's dI', dp' once, and writes dI (and dp) as float4.
template <int S, int MODE>
__global__ void __launch_bounds__(BF_NT) k_bwd_full_v(FullParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    static_assert(S % 4 == 0, "4 adjacent pixels in one block");
    const int X0 = 4 * (blockIdx.x * BF_NT + threadIdx.x), Y = blockIdx.y, n = blockIdx.z;
    if (X0 >= P.W) return;
    const size_t HW = (size_t)P.H * P.W, pix = (size_t)Y * P.W + X0;
    int ya, yb;
    float fy;
    up_taps(Y, S, P.h, ya, yb, fy);
    // The 4 pixels' bilinear taps: pixel t of block i (t < s/2) lies between low-res columns i - 1 and i,
    // pixel t >= s/2 between i and i + 1, at weight fx of the right one; at the image's first and last block
    // the clamped column indices give the clamped taps (a lerp between equal values returns that value).
    const int ib = X0 / S, t0 = X0 - ib * S;
    const int cl = max(ib - 1, 0), cr = min(ib + 1, P.w - 1);
    bool lo[4];
    float fx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int t = t0 + k;
        lo[k] = 2 * t + 1 < S;
        fx[k] = (float)(2 * t + 1 - S + (lo[k] ? 2 * S : 0)) * (1.0f / (float)(2 * S));
    }
    auto wsub = [](int t) -> float {
        if (MODE == GF_SUB_BOX) return 1.0f / (float)S;
        if (MODE == GF_SUB_NEAREST) return t == S / 2 ? 1.0f : 0.0f;
        return (t == S / 2 - 1 || t == S / 2) ? 0.5f : 0.0f;  // bilinear, even s
    };
    const float wy = wsub(Y % S);
    float wx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) wx[k] = wsub((X0 + k) % S);
    const size_t blk = (size_t)(Y / S) * P.w + X0 / S;  // the block's low-res pixel
    float4 shared = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int c = 0; c < P.C; ++c) {
        const size_t lp = (size_t)(n * P.C + c) * P.lps;
        const float *ra = P.ma + lp + (size_t)ya * P.w, *rb = P.ma + lp + (size_t)yb * P.w;
        // U(mean_a): the three columns lerped vertically first, then each pixel between its two columns
        const float vl = fmaf(fy, __ldg(rb + cl) - __ldg(ra + cl), __ldg(ra + cl));
        const float vc = fmaf(fy, __ldg(rb + ib) - __ldg(ra + ib), __ldg(ra + ib));
        const float vr = fmaf(fy, __ldg(rb + cr) - __ldg(ra + cr), __ldg(ra + cr));
        float A[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float a0 = lo[k] ? vl : vc, a1 = lo[k] ? vc : vr;
            A[k] = fmaf(fx[k], a1 - a0, a0);
        }
        const float4 gv = __ldg(reinterpret_cast<const float4 *>(P.g + (size_t)(n * P.C + c) * HW + pix));
        const float tI = wy != 0.0f ? wy * __ldg(P.dIl + lp + blk) : 0.0f;  // D^T(dI') before the x weight
        const float4 dIc = make_float4(fmaf(gv.x, A[0], tI * wx[0]), fmaf(gv.y, A[1], tI * wx[1]),
                                       fmaf(gv.z, A[2], tI * wx[2]), fmaf(gv.w, A[3], tI * wx[3]));
        if (P.CI == 1) {
            shared.x += dIc.x; shared.y += dIc.y; shared.z += dIc.z; shared.w += dIc.w;
        } else {
            *reinterpret_cast<float4 *>(P.dI + (size_t)(n * P.CI + c) * HW + pix) = dIc;
        }
        if (P.dp) {
            const float tp = wy != 0.0f ? wy * __ldg(P.dpl + lp + blk) : 0.0f;  // D^T(dp')
            *reinterpret_cast<float4 *>(P.dp + (size_t)(n * P.C + c) * HW + pix) =
                make_float4(tp * wx[0], tp * wx[1], tp * wx[2], tp * wx[3]);
        }
    }
    if (P.CI == 1) *reinterpret_cast<float4 *>(P.dI + (size_t)n * HW + pix) = shared;
    pdl_trigger();
}

// ------------------------------------------------------------------------------------------------------
// k_reduce_eps
// ------------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_reduce_eps(const float *partial, int n, float *out)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    __shared__ double red[256];
    double t = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) t += (double)partial[k];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)red[0];
    pdl_trigger();
}

// ------------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------------
namespace {

template <int NIN, int EPI>
cudaError_t launch_box_T(const BoxTParams &bp, int planes, cudaStream_t st)
{
    // the staging tile of the window sums lies over the column sums: the larger of the two
    const size_t smem = std::max((size_t)NIN * (BB_TW + 2 * bp.r) * BB_VP, (size_t)NIN * BB_TH * BB_OP) * sizeof(float);
    dim3 grid((bp.w + BB_TW - 1) / BB_TW, (bp.h + BB_TH - 1) / BB_TH, planes);
    if (bp.r >= 1 && bp.r <= 4) {  // compile-time radius: every row of a column segment requested at once
        cudaError_t e = cudaSuccess;
#define GF_BT(RR)                                                                             \
    do {                                                                                      \
        if ((e = opt_in_smem(k_bwd_box_T<NIN, EPI, false, RR>, smem)) != cudaSuccess) return e; \
        launch_pdl(k_bwd_box_T<NIN, EPI, false, RR>, grid, dim3(BB_NT), smem, st, bp);                        \
    } while (0)
        switch (bp.r) {
        case 1: GF_BT(1); break;
        case 2: GF_BT(2); break;
        case 3: GF_BT(3); break;
        default: GF_BT(4); break;
        }
#undef GF_BT
        return cudaGetLastError();
    }
    if (bp.r > 16) {
        cudaError_t e = opt_in_smem(k_bwd_box_T<NIN, EPI, true>, smem);
        if (e != cudaSuccess) return e;
        launch_pdl(k_bwd_box_T<NIN, EPI, true>, grid, dim3(BB_NT), smem, st, bp);
    } else {
        cudaError_t e = opt_in_smem(k_bwd_box_T<NIN, EPI, false>, smem);
        if (e != cudaSuccess) return e;
        launch_pdl(k_bwd_box_T<NIN, EPI, false>, grid, dim3(BB_NT), smem, st, bp);
    }
    return cudaGetLastError();
}

}  // namespace

size_t bwd_eps_partials(int N, int C, int h, int w)
{
    return (size_t)N * C * ((h + BB_TH - 1) / BB_TH) * ((w + BB_TW - 1) / BB_TW);
}

cudaError_t launch_backward(const BwdPlan &B, cudaStream_t st)
{
    cudaError_t err;
    const FwdPlan &F = B.fwd;
    const int planes = F.N * F.C;
    // ---- forward recomputation: low-res planes, statistics, a, mean_a (unless a gf_filter call saved them)
    if (!B.fwd_saved && (err = launch_forward(F, st)) != cudaSuccess) return err;

    // ---- dMA = U^T(g .* I), dMB = U^T(g)
    const bool up_vec = (F.s == 4 || F.s == 8) && F.W % F.s == 0 && F.H % F.s == 0 &&
                        ((reinterpret_cast<uintptr_t>(B.dq) | reinterpret_cast<uintptr_t>(F.I)) & 15u) == 0;
    if (up_vec) {
        UpTParams up;
        up.g = B.dq; up.I = (const float *)F.I; up.dma = B.dma; up.dmb = B.dmb;
        up.C = F.C; up.CI = F.CI; up.H = F.H; up.W = F.W; up.h = F.h; up.w = F.w; up.s = F.s;
        up.TJ = 16;
        up.lps = F.lps;
        const int rows_per_cta = UW_WARPS * up.TJ;
        dim3 grid((F.w + UW_TI - 1) / UW_TI, (F.h + rows_per_cta - 1) / rows_per_cta, planes);
        if (F.s == 4)
            launch_pdl(k_bwd_upsample_T_w<4>, grid, dim3(32 * UW_WARPS), 0, st, up);
        else
            launch_pdl(k_bwd_upsample_T_w<8>, grid, dim3(32 * UW_WARPS), 0, st, up);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    } else {
        UpTParams up;
        up.g = B.dq; up.I = (const float *)F.I; up.dma = B.dma; up.dmb = B.dmb;
        up.C = F.C; up.CI = F.CI; up.H = F.H; up.W = F.W; up.h = F.h; up.w = F.w; up.s = F.s;
        up.TJ = F.s <= 8 ? 8 : (F.s <= 16 ? 4 : 2);
        up.lps = F.lps;
        const int NRmax = F.s * (up.TJ + 2);
        const size_t smem = ((size_t)2 * NRmax * UT_TI + (size_t)UT_TI * 3 * F.s + (size_t)up.TJ * 3 * F.s) * sizeof(float);
        if ((err = opt_in_smem(k_bwd_upsample_T, smem)) != cudaSuccess) return err;
        dim3 grid((F.w + UT_TI - 1) / UT_TI, (F.h + up.TJ - 1) / up.TJ, planes);
        launch_pdl(k_bwd_upsample_T, grid, dim3(UT_NT), smem, st, up);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }

    // ---- da, db = B^T(dMA), B^T(dMB) with the chain epilogue -> d mean_I, d corr_I, d corr_Ip, d mean_p
    {
        BoxTParams bp{};
        bp.in[0] = B.dma; bp.in[1] = B.dmb;
        for (int k = 0; k < 4; ++k) bp.out[k] = B.gq[k];
        bp.lps = F.lps; bp.C = F.C; bp.CI = F.CI; bp.h = F.h; bp.w = F.w; bp.r = F.r_low; bp.eps = F.eps;
        bp.stats = (const float *)F.stats; bp.a = F.a; bp.eps_partial = B.eps_partial;
        if ((err = launch_box_T<2, EPI_CHAIN>(bp, planes, st)) != cudaSuccess) return err;
    }

    // ---- dI', dp' = B^T of the four maps, combined with I', p'
    {
        BoxTParams bp{};
        for (int k = 0; k < 4; ++k) bp.in[k] = B.gq[k];
        bp.out[0] = B.dIl; bp.out[1] = B.dpl;
        bp.lps = F.lps; bp.C = F.C; bp.CI = F.CI; bp.h = F.h; bp.w = F.w; bp.r = F.r_low; bp.eps = F.eps;
        const bool sub = F.s > 1;
        bp.Il = sub ? F.Il : (const float *)F.I;
        bp.pl = sub ? F.pl : (const float *)F.p;
        bp.xps = sub ? F.lps : (size_t)F.h * F.w;
        bp.yps = sub ? F.lps : (size_t)F.h * F.w;
        if ((err = launch_box_T<4, EPI_COMBINE>(bp, planes, st)) != cudaSuccess) return err;
    }

    // ---- full resolution: dI (direct term + D^T(dI')), dp = D^T(dp')
    {
        FullParams fp;
        fp.g = B.dq; fp.ma = F.ma; fp.dIl = B.dIl; fp.dpl = B.dpl; fp.dI = B.dI;
        fp.dp = F.p_lowres ? nullptr : B.dp;
        fp.C = F.C; fp.CI = F.CI; fp.H = F.H; fp.W = F.W; fp.h = F.h; fp.w = F.w; fp.s = F.s; fp.mode = F.mode;
        fp.lps = F.lps;
        auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
        const bool vec = (F.s == 4 || F.s == 8) && F.H % F.s == 0 && F.W % F.s == 0 && F.mode != GF_SUB_BILINEAR_AA &&
                         al16(fp.g) && al16(fp.dI) && (!fp.dp || al16(fp.dp));
        if (vec) {
            dim3 grid((F.W / 4 + BF_NT - 1) / BF_NT, F.H, F.N);
#define GF_BFV(ss, m) launch_pdl(k_bwd_full_v<ss, m>, grid, dim3(BF_NT), 0, st, fp)
            if (F.s == 4) {
                if (F.mode == GF_SUB_BOX) GF_BFV(4, GF_SUB_BOX);
                else if (F.mode == GF_SUB_NEAREST) GF_BFV(4, GF_SUB_NEAREST);
                else GF_BFV(4, GF_SUB_BILINEAR);
            } else {
                if (F.mode == GF_SUB_BOX) GF_BFV(8, GF_SUB_BOX);
                else if (F.mode == GF_SUB_NEAREST) GF_BFV(8, GF_SUB_NEAREST);
                else GF_BFV(8, GF_SUB_BILINEAR);
            }
#undef GF_BFV
        } else {
            dim3 grid((F.W + BF_NT - 1) / BF_NT, F.H, F.N);
            launch_pdl(k_bwd_full, grid, dim3(BF_NT), 0, st, fp);
        }
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if (F.p_lowres) {  // p was given at low resolution: dp = dp' (dense copy out of the strided workspace)
            if ((err = cudaMemcpy2DAsync(B.dp, (size_t)F.h * F.w * sizeof(float), B.dpl, F.lps * sizeof(float),
                                         (size_t)F.h * F.w * sizeof(float), planes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                return err;
        }
    }

    // ---- deps
    if (B.d_eps) {
        const int np = (int)bwd_eps_partials(F.N, F.C, F.h, F.w);
        launch_pdl(k_reduce_eps, 1, dim3(256), 0, st, B.eps_partial, np, B.d_eps);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace gfk
