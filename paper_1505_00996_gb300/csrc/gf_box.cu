// gf_box.cu -- TMA-fed tile kernels for the box steps of Algorithm 2 (He and Sun, "Fast Guided Filter", 2015):
//
//   BK_STATS     Algorithm 2, box statistics mean_I, mean_p, corr_I, corr_Ip at radius r', fused with
//                var_I, cov_Ip and the coefficients a (Eq. 2) and b (Eq. 3);
//   BK_MEAN2     Algorithm 2, box means of a and b;
//   BK_MEAN2_OUT the box means of a and b fused with q = mean_a I + mean_b (Eq. 4).  Only at s = 1, where
//                Algorithm 2's upsample is the identity, so each output pixel needs its own mean_a, mean_b only.
//
// f_mean is the box mean over the window clipped to the image, divided by the window's in-image count.
//
// One CTA owns a 32 x 64 tile of outputs of one channel.  One thread issues two 3-D TMA loads (X and Y
// planes) of the tile plus its r' halo on every side into shared memory and all threads wait on one
// mbarrier (bounded: a wait that gives up reports FAULT_BOX_TMA and the CTA returns).  Out-of-image cells of
// a border tile are then overwritten with the shift sample, so that they add exactly zero to the shifted
// sums.  Phase 1: one thread per column walks down its column of the shared tile, carrying the vertical
// window sums of both pairs of quantities, and writes them into a column-sum buffer (CB rows at a time).  Phase 2: one
// thread per (row, 8 columns) slides the horizontal window along the column sums and applies the epilogue,
// storing straight to global memory with 128-bit stores.  Both passes are O(1) per output in r'.
//
// Sums are taken of values shifted by one sample of the tile (the tile's first output pixel), so
// E[I^2] - E[I]^2 is formed from terms near the tile's own level; pairs of quantities travel as packed FP32x2.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "gf_device.cuh"
#include "gf_internal.cuh"

namespace gfk {

namespace {

// Output rows per tile (TH) and threads per CTA: tall tiles (32 rows, 256 threads) at large radii, whose
// vertical halo of 2 r' rows they amortise; short ones (16 rows, 128 threads, about 6 CTAs per SM) at small
// radii, where the tiles' short latency chains and the CTAs' number decide.
__host__ __device__ constexpr int nt_of(int TH) { return TH == 16 ? 128 : 256; }
constexpr int BX_TW = 64;   // output columns per tile
constexpr int BX_RH = 8;    // outputs per phase-2 thread (a run of one row)

enum { BK_STATS = 0, BK_MEAN2 = 2, BK_MEAN2_OUT = 3 };

struct BoxTmaParams {
    float *out0, *out1;  // BK_STATS: a, b; BK_MEAN2: mean_a, mean_b (plane stride ops)
    size_t ops;
    int N, C, CX;        // images; Y planes per image (channels); X planes per image (1 or C)
    int h, w, r;         // plane size; radius (used when the kernel's RC < 0)
    float eps;
    float *stats;        // BK_STATS, optional: 4 dense h*w planes per (n, c) of window means (mean_I, corr_I,
                         // mean_p, corr_Ip), kept for the backward
    // BK_MEAN2_OUT (s = 1): q = mean_a I + mean_b on rows [Yw0, Yw1) of the guide I (plane stride fps, one or
    // C planes per image) into q (dtype dt_out), with the detail epilogue q + k (I - q) when detail != 0
    const float *I;
    void *q;
    size_t fps;
    int CI, Yw0, Yw1;
    float detail;
    FaultSink fault;
};

__host__ __device__ constexpr int round4(int v) { return (v + 3) & ~3; }

// Shared-memory layout of one CTA for radius r and CB column-sum rows per block.
struct BoxSmem {
    int BW, BH, span, off, VP;
    size_t x_bytes, v_off, bar_off, total;
    __host__ __device__ BoxSmem(int r, int CB, int NP, int TH)
    {
        BW = BX_TW + 2 * round4(r);  // TMA box width: starts at x0 - round4(r), a multiple of 4 columns
        BH = TH + 2 * r;
        span = BX_TW + 2 * r;        // tile columns with vertical sums (tile column -r .. 63 + r)
        off = round4(r) - r;         // box column of tile column -r
        VP = span | 1;               // column-sum pitch in float2 (odd: conflict-free column reads)
        x_bytes = ((size_t)BH * BW * sizeof(float) + 127) & ~size_t(127);
        v_off = 2 * x_bytes;
        bar_off = v_off + (size_t)NP * CB * VP * sizeof(float2);
        total = bar_off + 16;
    }
};

template <typename TQ>
__device__ __forceinline__ void store8(TQ *p, bool second, const float v[8]);
template <>
__device__ __forceinline__ void store8<float>(float *p, bool second, const float v[8])
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    if (second) reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
template <>
__device__ __forceinline__ void store8<__half>(__half *p, bool second, const float v[8])
{
    auto pack = [](float a, float b) {
        const __half2 t = __floats2half2_rn(a, b);
        return *reinterpret_cast<const unsigned *>(&t);
    };
    reinterpret_cast<uint2 *>(p)[0] = make_uint2(pack(v[0], v[1]), pack(v[2], v[3]));
    if (second) reinterpret_cast<uint2 *>(p)[1] = make_uint2(pack(v[4], v[5]), pack(v[6], v[7]));
}

template <typename TQ>
__device__ __forceinline__ void stream8(TQ *p, bool second, const float v[8]);
template <>
__device__ __forceinline__ void stream8<float>(float *p, bool second, const float v[8])
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
    if (second) __stcs(reinterpret_cast<float4 *>(p) + 1, make_float4(v[4], v[5], v[6], v[7]));
}
template <>
__device__ __forceinline__ void stream8<__half>(__half *p, bool second, const float v[8])
{
    store8<__half>(p, second, v);
}

// Phase 1 for one strip column: the vertical window sums of one column of the shared tile for the tile rows
// [b CB, (b + 1) CB), continuing S0, S1 from the previous block.  S0 sums the shifted pair (dX, dY) and, when
// NP == 2, S1 the pair (dX^2, dX dY).
template <int NP, int RC, int CB>
__device__ __forceinline__ void walk_column(float2 &S0, float2 &S1, const float *px, const float *py, int BW,
                                            float2 cs, int r, int b, float2 *vcol, int VP)
{
    auto d = [&](int t) -> float2 { return sub2(make_float2(px[t * BW], py[t * BW]), cs); };
    auto prod = [](float2 v) { return mul2(make_float2(v.x, v.x), v); };  // (dX^2, dX dY)
    float2 *vcol1 = vcol + CB * VP;
    int i0 = b * CB, first = 0;
    if (b == 0) {
        S0 = S1 = make_float2(0.0f, 0.0f);
        if constexpr (RC >= 0) {
#pragma unroll
            for (int t = 0; t <= 2 * RC; ++t) {
                const float2 v = d(t);
                S0 = add2(S0, v);
                if (NP == 2) S1 = add2(S1, prod(v));
            }
        } else {
#pragma unroll 4
            for (int t = 0; t <= 2 * r; ++t) {
                const float2 v = d(t);
                S0 = add2(S0, v);
                if (NP == 2) S1 = add2(S1, prod(v));
            }
        }
        vcol[0] = S0;
        if (NP == 2) vcol1[0] = S1;
        first = 1;
    }
#pragma unroll
    for (int k = first; k < CB; ++k) {
        const int i = i0 + k;
        const float2 e = d(i + 2 * r), l = d(i - 1);  // row entering, row leaving
        S0 = add2(S0, sub2(e, l));
        vcol[k * VP] = S0;
        if (NP == 2) {
            S1 = add2(S1, sub2(prod(e), prod(l)));
            vcol1[k * VP] = S1;
        }
    }
}

template <int KIND, int RC, int CB, int TH, typename TQ>
__global__ void __launch_bounds__(nt_of(TH), TH == 16 ? 6 : 3) k_box_tma(const __grid_constant__ CUtensorMap tmX,
                                                   const __grid_constant__ CUtensorMap tmY, BoxTmaParams P)
{
    constexpr int NP = (KIND == BK_STATS) ? 2 : 1;  // float2 pairs of window sums
    constexpr int NT = nt_of(TH);
    static_assert(TH % CB == 0 && CB * (BX_TW / BX_RH) <= NT, "column-sum blocks");
    const int r = RC >= 0 ? RC : P.r;
    const BoxSmem L(r, CB, NP, TH);
    const int BW = L.BW, BH = L.BH, VP = L.VP;
    extern __shared__ __align__(128) unsigned char sm[];
    float *Xs = reinterpret_cast<float *>(sm);
    float *Ys = reinterpret_cast<float *>(sm + L.x_bytes);
    float2 *V = reinterpret_cast<float2 *>(sm + L.v_off);  // [NP][CB][VP]
    const unsigned bar = smem_u32(sm + L.bar_off);
    const int tid = threadIdx.x;
    const int c = blockIdx.x % P.C, tx = blockIdx.x / P.C, n = blockIdx.z;
    const int x0 = tx * BX_TW, y0 = blockIdx.y * TH;
    const int plane = n * P.C + c, xplane = n * P.CX + (P.CX == 1 ? 0 : c);
    const int h = P.h, w = P.w;
    pdl_wait();  // launched with programmatic serialization: the previous kernel's planes are complete here

    // ---- phase 0: the tile and its halo, X and Y, by TMA (zeros outside the image)
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar, 2u * (unsigned)(BH * BW) * (unsigned)sizeof(float));
        tma_load_3d(Xs, &tmX, x0 - round4(r), y0 - r, xplane, bar);
        tma_load_3d(Ys, &tmY, x0 - round4(r), y0 - r, plane, bar);
    }
    const bool landed = mbar_wait(bar, 0, P.fault, FAULT_BOX_TMA);
    if (!__syncthreads_and(landed)) return;  // a wait gave up: the whole CTA leaves, its outputs unwritten

    // the shift: the tile's first output pixel (always inside the image)
    const float2 cs = make_float2(Xs[r * BW + round4(r)], Ys[r * BW + round4(r)]);
    const bool interior = (x0 - r >= 0) && (x0 + BX_TW + r <= w) && (y0 - r >= 0) && (y0 + TH + r <= h);
    if (!interior) {  // out-of-image cells take the shift, so their shifted values are exactly zero
        const int t_lo = r - y0, t_hi = h - y0 + r, u_lo = round4(r) - x0, u_hi = w - x0 + round4(r);
        for (int idx = tid; idx < BH * BW; idx += NT) {
            const int t = idx / BW, u = idx - t * BW;
            if (t < t_lo || t >= t_hi || u < u_lo || u >= u_hi) {
                Xs[idx] = cs.x;
                Ys[idx] = cs.y;
            }
        }
        __syncthreads();
    }

    // one walker per strip column carries both pairs
    const bool walker = tid < L.span;
    const float *px = Xs + L.off + tid, *py = Ys + L.off + tid;
    float2 *vcol = V + tid;
    float2 S0w = make_float2(0.0f, 0.0f), S1w = make_float2(0.0f, 0.0f);

    // the guide pixels of this thread's outputs (s = 1 output form): requested before the sums, which hide
    // their latency; one block of CB = 32 rows there
    float iv[8];
    const int p_yr = tid % CB, p_xa = (tid / CB) * BX_RH;
    if (KIND == BK_MEAN2_OUT && tid < CB * (BX_TW / BX_RH)) {
        const int y = y0 + p_yr, x = x0 + p_xa;
        if (y < h && x < w && y >= P.Yw0 && y < P.Yw1) {
            const float *Ip = P.I + (size_t)(n * P.CI + (P.CI == 1 ? 0 : c)) * P.fps + (size_t)y * w + x;
            const float4 u = __ldcs(reinterpret_cast<const float4 *>(Ip));
            const float4 v = (x + 4 < w) ? __ldcs(reinterpret_cast<const float4 *>(Ip) + 1)
                                         : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            iv[0] = u.x; iv[1] = u.y; iv[2] = u.z; iv[3] = u.w;
            iv[4] = v.x; iv[5] = v.y; iv[6] = v.z; iv[7] = v.w;
        }
    }

    const float n_full = (float)((2 * r + 1) * (2 * r + 1));
    const float inv_full = 1.0f / n_full;
    const int nblocks = TH / CB;
    for (int b = 0; b < nblocks; ++b) {
        // ---- phase 1: vertical window sums of the block's rows
        if (walker) walk_column<NP, RC, CB>(S0w, S1w, px, py, BW, cs, r, b, vcol, VP);
        __syncthreads();

        // ---- phase 2: horizontal window sums along 8 outputs of one row, epilogue, store
        if (tid < CB * (BX_TW / BX_RH)) {
            const int yr = tid % CB, seg = tid / CB;
            const int y = y0 + b * CB + yr, xa = seg * BX_RH, x = x0 + xa;
            bool live = (y < h) && (x < w);
            if (KIND == BK_MEAN2_OUT) live = live && (y >= P.Yw0) && (y < P.Yw1);
            if (live) {
                const bool second = (x + 4 < w);
                const float2 *v0 = V + yr * VP + xa;
                const float2 *v1 = v0 + CB * VP;
                float2 S0 = make_float2(0.0f, 0.0f), S1 = make_float2(0.0f, 0.0f);
                if constexpr (RC >= 0) {
#pragma unroll
                    for (int k = 0; k <= 2 * RC; ++k) {
                        S0 = add2(S0, v0[k]);
                        if (NP == 2) S1 = add2(S1, v1[k]);
                    }
                } else {
#pragma unroll 4
                    for (int k = 0; k <= 2 * r; ++k) {
                        S0 = add2(S0, v0[k]);
                        if (NP == 2) S1 = add2(S1, v1[k]);
                    }
                }
                const int ny = min(h - 1, y + r) - max(0, y - r) + 1;
                float o0[8], o1[8];
                const bool with_stats = (KIND == BK_STATS) && P.stats != nullptr;
                float wst[(KIND == BK_STATS && TH == 16) ? 4 : 1][8];
#pragma unroll
                for (int j = 0; j < BX_RH; ++j) {
                    if (j > 0) {
                        S0 = add2(S0, sub2(v0[j + 2 * r], v0[j - 1]));
                        if (NP == 2) S1 = add2(S1, sub2(v1[j + 2 * r], v1[j - 1]));
                    }
                    float inv = inv_full;
                    if (!interior) {
                        const int xx = x + j;
                        const int nx = min(w - 1, xx + r) - max(0, xx - r) + 1;
                        inv = __fdividef(1.0f, (float)(nx * ny));
                    }
                    const float2 m0 = mul2(S0, make_float2(inv, inv));
                    if (KIND == BK_STATS) {
                        const float2 m1 = mul2(S1, make_float2(inv, inv));
                        // var_I and cov_Ip; a one-sample window (r' = 0) has both exactly 0 (Eq. 2 then gives a = 0),
                        // where the shifted sums would leave the rounding of the square, amplified by 1 / eps
                        const float var = r ? fmaxf(fmaf(-m0.x, m0.x, m1.x), 0.0f) : 0.0f;
                        const float cov = r ? fmaf(-m0.x, m0.y, m1.y) : 0.0f;
                        const float a = __fdividef(cov, var + P.eps);            // a, Eq. (2)
                        o0[j] = a;
                        o1[j] = (m0.y + cs.y) - a * (m0.x + cs.x);               // b, Eq. (3)
                        if (with_stats) {  // the window means the backward reads
                            const float st4[4] = {m0.x + cs.x,                                  // mean_I
                                                  m1.x + cs.x * (2.0f * m0.x + cs.x),           // corr_I
                                                  m0.y + cs.y,                                  // mean_p
                                                  m1.y + cs.x * m0.y + cs.y * m0.x + cs.x * cs.y};  // corr_Ip
                            if constexpr (TH == 16) {  // kept for 128-bit stores after the run
#pragma unroll
                                for (int k = 0; k < 4; ++k) wst[k][j] = st4[k];
                            } else if (x + j < w) {    // tall tiles (large radii): stored at once, fewer registers
                                const size_t ps = (size_t)h * w;
                                float *stp = P.stats + (size_t)plane * 4 * ps + (size_t)y * w + x + j;
#pragma unroll
                                for (int k = 0; k < 4; ++k) stp[k * ps] = st4[k];
                            }
                        }
                    } else {
                        o0[j] = m0.x + cs.x;  // mean_a
                        o1[j] = m0.y + cs.y;  // mean_b
                    }
                }
                if (KIND == BK_MEAN2_OUT) {
                    float qv[8];
#pragma unroll
                    for (int j = 0; j < BX_RH; ++j) {
                        qv[j] = fmaf(o0[j], iv[j], o1[j]);  // Eq. (4)
                        if (P.detail != 0.0f) qv[j] = fmaf(P.detail, iv[j] - qv[j], qv[j]);
                    }
                    stream8<TQ>((TQ *)P.q + (size_t)plane * P.fps + (size_t)y * w + x, second, qv);
                } else {
                    const size_t o = (size_t)plane * P.ops + (size_t)y * w + x;
                    store8<float>(P.out0 + o, second, o0);
                    store8<float>(P.out1 + o, second, o1);
                    if constexpr (KIND == BK_STATS && TH == 16) {
                        if (with_stats) {
                            const size_t ps = (size_t)h * w;
                            float *st = P.stats + (size_t)plane * 4 * ps + (size_t)y * w + x;
#pragma unroll
                            for (int k = 0; k < 4; ++k) store8<float>(st + k * ps, second, wst[k]);
                        }
                    }
                }
            }
        }
        if (b + 1 < nblocks) __syncthreads();  // the column sums are rewritten by the next block
    }
    pdl_trigger();  // this CTA's outputs are written: the next kernel may be scheduled
}

}  // namespace

namespace {

// Column-sum rows per block: the whole tile height, except for the statistics at r' > 8, whose two pairs of
// column sums would otherwise keep the CTA above 74 KB of shared memory (three CTAs per SM).
// Tile height and column-sum rows per block: tall tiles above r' = 8, with two blocks of 16 rows for the
// statistics (two pairs of column sums would otherwise keep the CTA above 74 KB of shared memory, three CTAs per
// SM); 16-row tiles, one block, up to r' = 8.
constexpr int th_of(int r) { return r > 8 ? 32 : 16; }
constexpr int cb_of(int r, int NP) { return (r > 8 && NP == 2) ? 16 : th_of(r); }

template <int KIND, int RC, int CB, int TH, typename TQ>
cudaError_t launch_one(const CUtensorMap &mx, const CUtensorMap &my, const BoxTmaParams &P, int r, cudaStream_t st)
{
    const size_t smem = BoxSmem(r, CB, KIND == BK_STATS ? 2 : 1, TH).total;
    cudaError_t e = opt_in_smem(k_box_tma<KIND, RC, CB, TH, TQ>, smem);
    if (e != cudaSuccess) return e;
    // the channel is the fastest block index: the channel CTAs of a tile share its guide tile through L2
    const dim3 grid(P.C * ((P.w + BX_TW - 1) / BX_TW), (P.h + TH - 1) / TH, P.N);
    if ((e = launch_pdl(k_box_tma<KIND, RC, CB, TH, TQ>, grid, dim3(nt_of(TH)), smem, st, mx, my, P)) != cudaSuccess)
        return e;
    return cudaGetLastError();
}

// The radius as a compile-time constant for the common radii (s = 4 and 8 at the paper's figure radii,
// serving's r' <= 8, s = 1 at r = 8 and 16, the feathering figure's r' = 15), else at run time.
template <int KIND, typename TQ>
cudaError_t launch_kind(const CUtensorMap &mx, const CUtensorMap &my, const BoxTmaParams &P, cudaStream_t st)
{
    constexpr int NP = KIND == BK_STATS ? 2 : 1;
    const int r = P.r;
#define GF_BOX_R(RR) launch_one<KIND, RR, cb_of(RR, NP), th_of(RR), TQ>(mx, my, P, r, st)
    switch (r) {
    case 1: return GF_BOX_R(1);
    case 2: return GF_BOX_R(2);
    case 3: return GF_BOX_R(3);
    case 4: return GF_BOX_R(4);
    case 5: return GF_BOX_R(5);
    case 6: return GF_BOX_R(6);
    case 7: return GF_BOX_R(7);
    case 8: return GF_BOX_R(8);
    case 15: return GF_BOX_R(15);
    case 16: return GF_BOX_R(16);
    default: break;
    }
#undef GF_BOX_R
    if (r <= 8) return launch_one<KIND, -1, cb_of(8, NP), th_of(8), TQ>(mx, my, P, r, st);
    return launch_one<KIND, -1, cb_of(16, NP), th_of(16), TQ>(mx, my, P, r, st);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

bool box_tma_supported(const BoxTmaJob &J)
{
    if (J.r < 0 || J.r > 16 || J.w % 4 != 0 || J.xps % 4 != 0 || J.yps % 4 != 0) return false;
    if (!aligned16(J.X) || !aligned16(J.Y)) return false;
    if (J.kind == BOX_JOB_MEANS_OUTPUT) {
        if (!aligned16(J.I) || !aligned16(J.q) || J.fps % 4 != 0) return false;
        if (J.dt_out != F32 && J.dt_out != F16) return false;
    } else if (!aligned16(J.out0) || !aligned16(J.out1) || J.ops % 4 != 0 || (J.stats && !aligned16(J.stats))) {
        return false;
    }
    if (getenv("GF_NO_TMA_BOX") != nullptr) return false;  // the per-thread-load box kernels instead (tests)
    CUtensorMap probe;
    return encode_tmap_3d(&probe, F32, J.X, J.w, J.h, 1, J.xps, 64, 32);
}

cudaError_t launch_box_tma(const BoxTmaJob &J, cudaStream_t st)
{
    const BoxSmem L(J.r, 32, 1, th_of(J.r));
    CUtensorMap mx, my;
    if (!encode_tmap_3d(&mx, F32, J.X, J.w, J.h, J.N * J.CX, J.xps, L.BW, L.BH) ||
        !encode_tmap_3d(&my, F32, J.Y, J.w, J.h, J.N * J.C, J.yps, L.BW, L.BH))
        return cudaErrorInvalidValue;
    BoxTmaParams P{};
    P.out0 = J.out0;
    P.out1 = J.out1;
    P.ops = J.ops;
    P.N = J.N;
    P.C = J.C;
    P.CX = J.CX;
    P.h = J.h;
    P.w = J.w;
    P.r = J.r;
    P.eps = J.eps;
    P.stats = J.stats;
    P.I = J.I;
    P.q = J.q;
    P.fps = J.fps;
    P.CI = J.CI;
    P.Yw0 = J.Yw0;
    P.Yw1 = J.Yw1;
    P.detail = J.detail;
    P.fault = J.fault;
    switch (J.kind) {
    case BOX_JOB_STATS: return launch_kind<BK_STATS, float>(mx, my, P, st);
    case BOX_JOB_MEANS: return launch_kind<BK_MEAN2, float>(mx, my, P, st);
    default:
        if (J.dt_out == F16) return launch_kind<BK_MEAN2_OUT, __half>(mx, my, P, st);
        return launch_kind<BK_MEAN2_OUT, float>(mx, my, P, st);
    }
}

}  // namespace gfk
