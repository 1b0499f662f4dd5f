// gf_forward.cu -- sm_103a kernels of the fast guided filter forward pass (Algorithm 2 of He and Sun,
// "Fast Guided Filter", 2015) and the host launcher that chains them.
//
//   k_subsample / k_subsample_vec
//                 Algorithm 2 first step: I' = f_subsample(I, s), p' = f_subsample(p, s) into FP32 low-res
//                 planes (nearest, bilinear or box; see gf.h for the conventions).  Each thread produces a
//                 column of low-res pixels so that all of its full-res loads are in flight together; the
//                 _vec form reads aligned FP32 rows with 64/128-bit loads for s = 2, 4, 8.
//   k_box_tile    KIND 0/1: the box statistics of I', p', I'.*I', I'.*p' at radius r' fused with the
//                 variance/covariance and the coefficients a (Eq. 2) and b (Eq. 3).
//                 KIND 2: the box means of a and b.
//                 One CTA owns a 32 x 64 tile of outputs of one channel.  Phase 1: each thread slides a
//                 vertical window down a segment of one column (loads straight from global memory, sums in
//                 registers) and writes the column sums into a transposed shared tile.  Phase 2: each thread
//                 slides a horizontal window along a segment of one row of that tile and applies the
//                 epilogue.  Phase 3 writes the tile out coalesced.  Work per pixel is O(1) in r'.
//   k_upsample_output_s4x / k_upsample_output
//                 Algorithm 2 last two steps fused: bilinear upsampling of mean_a, mean_b (never written at
//                 full resolution) and q = mean_a .* I + mean_b (Eq. 4) on the full-resolution guide.  A CTA
//                 stages the low-res taps of its 512-pixel-wide band in shared memory; each thread owns 4
//                 adjacent columns, reads I with 128-bit streaming loads (several rows in flight) and
//                 writes q once with streaming stores.  The _s4x form (s = 4, 8) walks the rows in the
//                 s-row runs that share one pair of low-res tap rows, with the vertical weights as
//                 compile-time constants: three FMAs per output value.
//   k_output_s1   the s = 1 form of the last step (no resampling).
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "gf_device.cuh"
#include "gf_internal.cuh"

namespace gfk {

// ------------------------------------------------------------------------------------------------------
// k_subsample
// ------------------------------------------------------------------------------------------------------
constexpr int SUB_NT = 128;      // threads per CTA (one low-res column each)
constexpr int SUB_NT_VEC = 256;  // the same for the aligned FP32 nearest/bilinear kernel (measured best)
constexpr int SUB_JB = 4;    // low-res rows per thread

struct SubJob {
    const void *src;
    float *dst;
    int planes, H, W, s;
    size_t sps, dps;  // source / destination plane strides (elements)
    int sn, sd;       // the ratio as sn / sd (s = sn, sd = 1 for an integer ratio)
};
struct SubParams {
    SubJob job[2];
    int h, w, mode;
    float scale;  // result multiplier: k on the uint8 path (exact integers J = k * value), else 1
    unsigned *clear_word;  // the call's fault word, zeroed by the first thread (the chain's first kernel)
};

// The first thread of the chain's first kernel zeroes the call's fault word; the kernels after it, which
// may report into it, start only once this kernel has finished.
__device__ __forceinline__ void clear_call_fault(unsigned *word)
{
    if (word && (blockIdx.x | blockIdx.y | blockIdx.z | threadIdx.x) == 0) *word = 0u;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(SUB_NT) k_subsample(SubParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    clear_call_fault(P.clear_word);
    const int i = blockIdx.x * SUB_NT + threadIdx.x;
    const int j0 = blockIdx.y * SUB_JB;
    if (i >= P.w) return;
    int z = blockIdx.z;
    const SubJob &J = (z < P.job[0].planes) ? P.job[0] : P.job[1];
    if (z >= P.job[0].planes) z -= P.job[0].planes;
    const T *src = (const T *)J.src + (size_t)z * J.sps;
    float v[SUB_JB];
#pragma unroll
    for (int u = 0; u < SUB_JB; ++u) {
        const int j = min(j0 + u, P.h - 1);
        v[u] = subsample_one<T, MODE>(src, J.H, J.W, J.s, J.sn, J.sd, j, i);
    }
    float *dst = J.dst + (size_t)z * J.dps + i;
#pragma unroll
    for (int u = 0; u < SUB_JB; ++u)
        if (j0 + u < P.h) dst[(size_t)(j0 + u) * P.w] = v[u] * P.scale;
    pdl_trigger();
}

// Antialiased bilinear subsample: along each axis, source pixel x weighs n(x) = 2s - |2x + 1 - (2i + 1)s|
// (twice s times the triangle weight) for low-res pixel i, over the 2s (even s) or 2s - 1 (odd s) taps with
// n > 0 that lie in the image, divided by the sum of those n.  Each thread owns one low-res column and
// SUB_JB consecutive low-res rows; it walks the source rows they cover once, forming the horizontal
// weighted sum of each row and adding it to the (at most two) low-res rows whose taps include that row.
template <typename T>
__global__ void __launch_bounds__(SUB_NT) k_subsample_aa(SubParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    clear_call_fault(P.clear_word);
    const int i = blockIdx.x * SUB_NT + threadIdx.x;
    const int j0 = blockIdx.y * SUB_JB;
    if (i >= P.w) return;
    int z = blockIdx.z;
    const SubJob &J = (z < P.job[0].planes) ? P.job[0] : P.job[1];
    if (z >= P.job[0].planes) z -= P.job[0].planes;
    const T *src = (const T *)J.src + (size_t)z * J.sps;
    float *dst = J.dst + (size_t)z * J.dps + i;
    const int H = J.H, W = J.W, sn = J.sn, sd = J.sd;
    if (J.s == 1) {  // a low-res p given by the caller: copied
        for (int u = 0; u < SUB_JB && j0 + u < P.h; ++u) dst[(size_t)(j0 + u) * P.w] = ldv(src + (size_t)(j0 + u) * W + i);
        return;
    }
    // Weight numerator of source index t for low-res index k: 2 sn - |(2t + 1) sd - (2k + 1) sn| (over 2 sn);
    // positive for t in [lo(k), hi(k)]: (2t + 1) sd strictly within 2 sn of (2k + 1) sn.
    auto wnum = [&](int t, int k) { return 2 * sn - abs((2 * t + 1) * sd - (2 * k + 1) * sn); };
    auto lo_of = [&](int k) { return floor_div((2 * k + 1) * sn - 2 * sn - sd, 2 * sd) + 1; };
    auto hi_of = [&](int k) { return -floor_div(-((2 * k + 1) * sn + 2 * sn - sd), 2 * sd) - 1; };
    const int xa = max(0, lo_of(i)), xb = min(W - 1, hi_of(i));
    int nx = 0;
    for (int x = xa; x <= xb; ++x) nx += wnum(x, i);
    const int jl = min(j0 + SUB_JB, P.h) - 1;  // last low-res row of the block
    const int ya = max(0, lo_of(j0)), yb = min(H - 1, hi_of(jl));
    float acc[SUB_JB];
#pragma unroll
    for (int u = 0; u < SUB_JB; ++u) acc[u] = 0.0f;
    for (int y = ya; y <= yb; ++y) {
        const T *row = src + (size_t)y * W;
        float hs = 0.0f;
        for (int x = xa; x <= xb; ++x) hs = fmaf((float)wnum(x, i), ldv(row + x), hs);
#pragma unroll
        for (int u = 0; u < SUB_JB; ++u) {
            const int ny = wnum(y, j0 + u);
            if (ny > 0) acc[u] = fmaf((float)ny, hs, acc[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < SUB_JB; ++u) {
        const int j = j0 + u;
        if (j >= P.h) break;
        const int ja = max(0, lo_of(j)), jb = min(H - 1, hi_of(j));
        int ny = 0;
        for (int y = ja; y <= jb; ++y) ny += wnum(y, j);
        dst[(size_t)j * P.w] = acc[u] / ((float)nx * (float)ny) * P.scale;
    }
    pdl_trigger();
}

// Aligned FP32 fast path of the box and antialiased subsamples for s = 2, 4, 8 with H and W multiples of s.
// Thread = one low-res column i, SUB_JB low-res rows.  Each source row is read once per thread as vectors:
// the s-column chunk of block i (box), or the three chunks i-1, i, i+1 (antialiased: taps S i - S/2 + k,
// k = 0 .. 2S-1, weight 2S - |2k + 1 - 2S|; chunks outside the image are skipped and their weights left out
// of the normalisation -- S^2/4 on each side).  Neighbouring threads share chunks through L1.
template <int S>
__device__ __forceinline__ void ld_chunk(const float *p, float (&v)[S])
{
    if constexpr (S == 2) {
        const float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int q = 0; q < S / 4; ++q) {
            const float4 t = __ldcs(reinterpret_cast<const float4 *>(p) + q);
            v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
        }
    }
}

template <int MODE, int S>
__global__ void __launch_bounds__(SUB_NT) k_subsample_wide(SubParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    clear_call_fault(P.clear_word);
    const int i = blockIdx.x * SUB_NT + threadIdx.x;
    const int j0 = blockIdx.y * SUB_JB;
    if (i >= P.w) return;
    int z = blockIdx.z;
    const SubJob &J = (z < P.job[0].planes) ? P.job[0] : P.job[1];
    if (z >= P.job[0].planes) z -= P.job[0].planes;
    const float *src = (const float *)J.src + (size_t)z * J.sps;
    float *dst = J.dst + (size_t)z * J.dps + i;
    const int H = J.H, W = J.W;
    if (J.s == 1) {  // a low-res p given by the caller: copied
        for (int u = 0; u < SUB_JB && j0 + u < P.h; ++u) dst[(size_t)(j0 + u) * P.w] = src[(size_t)(j0 + u) * W + i];
        return;
    }
    float acc[SUB_JB];
#pragma unroll
    for (int u = 0; u < SUB_JB; ++u) acc[u] = 0.0f;
    if constexpr (MODE == GF_SUB_BOX) {
#pragma unroll
        for (int u = 0; u < SUB_JB; ++u) {
            if (j0 + u >= P.h) break;
#pragma unroll
            for (int k = 0; k < S; ++k) {
                float v[S];
                ld_chunk<S>(src + (size_t)(S * (j0 + u) + k) * W + S * i, v);
#pragma unroll
                for (int x = 0; x < S; ++x) acc[u] += v[x];
            }
        }
#pragma unroll
        for (int u = 0; u < SUB_JB; ++u)
            if (j0 + u < P.h) dst[(size_t)(j0 + u) * P.w] = acc[u] * (1.0f / (float)(S * S));
    } else {  // antialiased bilinear
        const bool has_l = i > 0, has_r = S * (i + 1) < W;
        const int jl = min(j0 + SUB_JB, P.h) - 1;
        const int ya = max(0, S * j0 - S / 2), yb = min(H - 1, S * jl + 3 * S / 2 - 1);
        for (int y = ya; y <= yb; ++y) {
            const float *row = src + (size_t)y * W + S * i;
            float l[S], m[S], r[S];
            ld_chunk<S>(row, m);
#pragma unroll
            for (int x = 0; x < S; ++x) { l[x] = 0.0f; r[x] = 0.0f; }
            if (has_l) ld_chunk<S>(row - S, l);
            if (has_r) ld_chunk<S>(row + S, r);
            // taps k = 0 .. 2S-1 are columns S i - S/2 + k: the last S/2 of chunk l, all of m, the first S/2 of r
            float hs = 0.0f;
#pragma unroll
            for (int k = 0; k < 2 * S; ++k) {
                const int c = k - S / 2;  // column offset from S i
                const float v = (c < 0) ? l[S + c] : (c < S ? m[c] : r[c - S]);
                hs = fmaf((float)(2 * S - abs(2 * k + 1 - 2 * S)), v, hs);
            }
#pragma unroll
            for (int u = 0; u < SUB_JB; ++u) {
                const int t = y - (S * (j0 + u) - S / 2);  // tap index of row y for low-res row j0 + u
                if (t >= 0 && t < 2 * S) acc[u] = fmaf((float)(2 * S - abs(2 * t + 1 - 2 * S)), hs, acc[u]);
            }
        }
        const float nx = (float)(2 * S * S - (has_l ? 0 : S * S / 4) - (has_r ? 0 : S * S / 4));
#pragma unroll
        for (int u = 0; u < SUB_JB; ++u) {
            const int j = j0 + u;
            if (j >= P.h) break;
            const float ny = (float)(2 * S * S - (j > 0 ? 0 : S * S / 4) - (S * (j + 1) < H ? 0 : S * S / 4));
            dst[(size_t)j * P.w] = acc[u] / (nx * ny);
        }
    }
    pdl_trigger();
}

// The two source columns a bilinear sample at ratio S reads (S/2 - 1 and S/2 of the block; the sample
// twice for nearest, column S/2), from one aligned vector load of the block's first S (S <= 4) or 8 (S = 8:
// columns 3 and 4) values.  FP32, FP16 (converted) or uint8 (raw byte values, as ldv gives them).
template <typename T, int S, int MODE>
__device__ __forceinline__ float2 ld_block_pair(const T *rp)
{
    float v0, v1;  // columns S/2 - 1 and S/2
    if constexpr (sizeof(T) == 4) {
        if constexpr (S == 2) {
            const float2 t = __ldcs(reinterpret_cast<const float2 *>(rp));
            v0 = t.x; v1 = t.y;
        } else if constexpr (S == 4) {
            const float4 t = __ldcs(reinterpret_cast<const float4 *>(rp));
            v0 = t.y; v1 = t.z;
        } else {
            const float4 b = __ldcs(reinterpret_cast<const float4 *>(rp + 4));
            v1 = b.x;
            v0 = (MODE == GF_SUB_BILINEAR) ? __ldcs(reinterpret_cast<const float4 *>(rp)).w : b.x;
        }
    } else if constexpr (sizeof(T) == 2) {
        if constexpr (S == 2) {
            const unsigned t = __ldcs(reinterpret_cast<const unsigned *>(rp));
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&t));
            v0 = f.x; v1 = f.y;
        } else if constexpr (S == 4) {
            const uint2 t = __ldcs(reinterpret_cast<const uint2 *>(rp));
            const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
            const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
            v0 = lo.y; v1 = hi.x;
        } else {
            const uint4 t = __ldcs(reinterpret_cast<const uint4 *>(rp));
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));  // columns 2, 3
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.z));  // columns 4, 5
            v0 = a.y; v1 = b.x;
        }
    } else {
        if constexpr (S == 2) {
            const unsigned short t = __ldcs(reinterpret_cast<const unsigned short *>(rp));
            v0 = (float)(t & 0xffu); v1 = (float)(t >> 8);
        } else if constexpr (S == 4) {
            const unsigned t = __ldcs(reinterpret_cast<const unsigned *>(rp));
            v0 = (float)((t >> 8) & 0xffu); v1 = (float)((t >> 16) & 0xffu);
        } else {
            const uint2 t = __ldcs(reinterpret_cast<const uint2 *>(rp));
            v0 = (float)(t.x >> 24); v1 = (float)(t.y & 0xffu);
        }
    }
    return MODE == GF_SUB_BILINEAR ? make_float2(v0, v1) : make_float2(v1, v1);
}

// Aligned fast path of k_subsample (nearest / bilinear) for s = 2, 4, 8 with H and W multiples of s (so no
// sample is clamped): the one or two source columns of a low-res pixel are read with one vector load per
// source row (two for FP32 at s = 8).
template <typename T, int MODE, int S>
__global__ void __launch_bounds__(SUB_NT_VEC) k_subsample_vec(SubParams P)
{
    pdl_wait();  // launched with programmatic serialization: the previous call's kernels are complete here
    clear_call_fault(P.clear_word);
    constexpr int JB = (S == 8) ? 1 : 2;  // low-res rows per thread: short threads, many of them (measured best)
    const int i = blockIdx.x * SUB_NT_VEC + threadIdx.x;
    const int j0 = blockIdx.y * JB;
    if (i >= P.w) return;
    int z = blockIdx.z;
    const SubJob &J = (z < P.job[0].planes) ? P.job[0] : P.job[1];
    if (z >= P.job[0].planes) z -= P.job[0].planes;
    const T *src = (const T *)J.src + (size_t)z * J.sps;
    const int W = J.W;
    auto row_val = [&](int y) { return ld_block_pair<T, S, MODE>(src + (size_t)y * W + (size_t)i * S); };
    float2 top[JB], bot[JB];
#pragma unroll
    for (int u = 0; u < JB; ++u) {
        const int j = min(j0 + u, P.h - 1);
        if (MODE == GF_SUB_BILINEAR) {
            top[u] = row_val(S * j + S / 2 - 1);
            bot[u] = row_val(S * j + S / 2);
        } else {
            top[u] = row_val(S * j + S / 2);
        }
    }
    float *dst = J.dst + (size_t)z * J.dps + i;
#pragma unroll
    for (int u = 0; u < JB; ++u) {
        if (j0 + u >= P.h) break;
        float v;
        if (MODE == GF_SUB_BILINEAR)
            v = 0.5f * (0.5f * top[u].x + 0.5f * top[u].y) + 0.5f * (0.5f * bot[u].x + 0.5f * bot[u].y);
        else
            v = top[u].x;
        dst[(size_t)(j0 + u) * P.w] = v * P.scale;
    }
    pdl_trigger();  // the next kernel may be scheduled once every CTA is here
}

// ------------------------------------------------------------------------------------------------------
// k_box_tile
// ------------------------------------------------------------------------------------------------------
constexpr int BT_NT_MAX = 320;  // largest CTA (the launch sizes it to the phase-1 work, a multiple of 32)
constexpr int BT_TH = 32;   // output rows per tile
constexpr int BT_TW = 64;   // output columns per tile
constexpr int BT_VP = BT_TH + 1;  // pitch of the transposed column-sum tile (odd: no bank conflicts)
constexpr int BT_OP = BT_TW + 1;  // pitch of the output staging tile

enum { KIND_STATS_F = 0, KIND_STATS_INT = 1, KIND_MEAN2 = 2 };

struct BoxParams {
    const void *X, *Y;  // KIND 0/1: guide I' and input p' planes; KIND 2: a and b planes
    size_t xps, yps;    // plane strides (elements)
    int CX, C;          // X planes per image (1 or C), Y planes per image (C)
    float *out0, *out1; // KIND 0/1: a, b.  KIND 2: mean of X, mean of Y.
    size_t ops;         // output plane stride
    void *stats;        // optional, KIND 0/1: 4 dense h*w planes per (n, c)
    int h, w, r;
    float eps;
    float int_scale;    // KIND 1: 255 * k (values are integers J = int_scale * I')
};

inline size_t box_tile_smem(int nq, int r)
{
    return ((size_t)nq * (BT_TW + 2 * r) * BT_VP + 2 * BT_TH * BT_OP) * sizeof(float);
}

// Window-sum accumulation.  With COMP the sum is Neumaier-compensated (s + c carries it to about one
// rounding of its value); used for large radii, where a window holds hundreds of terms.  For r' <= 16 the
// shifted FP32 sums of at most a few dozen terms stay well inside the error budget without it.
template <bool COMP>
__device__ __forceinline__ void kadd(float &s, float &c, float v)
{
    if (COMP) {
        const float t = s + v;
        c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    } else {
        s += v;
    }
}

template <int KIND>
struct Quant {
    static constexpr int NQ = (KIND == KIND_MEAN2) ? 2 : 4;
    // the quantities whose window sums the kernel needs, from one (X, Y) sample
    __device__ __forceinline__ static void of(float x, float y, float cx, float cy, float *q)
    {
        if (KIND == KIND_MEAN2) {
            q[0] = x - cx;
            q[1] = y - cy;
        } else {
            const float dx = x - cx, dy = y - cy;
            q[0] = dx; q[1] = dx * dx; q[2] = dy; q[3] = dx * dy;
        }
    }
    __device__ __forceinline__ static void of_int(float x, float y, uint32_t *q)
    {
        const uint32_t J = (uint32_t)x, Pv = (uint32_t)y;
        q[0] = J; q[1] = J * J; q[2] = Pv; q[3] = J * Pv;
    }
};

template <typename T, int KIND, bool COMP, int BT_RV, int BT_RH>
__global__ void __launch_bounds__(BT_NT_MAX) k_box_tile(BoxParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    const int BT_NT = blockDim.x;
    using Q = Quant<KIND>;
    constexpr int NQ = Q::NQ;
    constexpr bool INT = (KIND == KIND_STATS_INT);
    extern __shared__ float smf[];
    const int tid = threadIdx.x;
    const int h = P.h, w = P.w, r = P.r;
    const int span = BT_TW + 2 * r;
    float *Vt = smf;                        // [NQ][span][BT_VP] column sums, transposed
    uint32_t *Vu = reinterpret_cast<uint32_t *>(smf);
    float *Ot = smf + (size_t)NQ * span * BT_VP;  // [2][BT_TH][BT_OP] outputs
    const int x0 = blockIdx.x * BT_TW, y0 = blockIdx.y * BT_TH;
    const int plane = blockIdx.z;  // n * C + c
    const int n = plane / P.C, c = plane - n * P.C;
    const T *Xp = (const T *)P.X + (size_t)(n * P.CX + (P.CX == 1 ? 0 : c)) * P.xps;
    const T *Yp = (const T *)P.Y + (size_t)plane * P.yps;

    auto xval = [&](int y, int x) -> float { return ldv(Xp + (size_t)y * w + x); };
    auto yval = [&](int y, int x) -> float { return ldv(Yp + (size_t)y * w + x); };
    // shift of the float sums: one sample of the tile, so that the sums of squares stay small
    float cx = 0.0f, cy = 0.0f;
    if (!INT) {
        cx = xval(y0, x0);
        cy = yval(y0, x0);
    }

    // ---- phase 1: vertical window sums of every tile column (halo columns included)
    constexpr int NSEG_V = BT_TH / BT_RV;
    for (int item = tid; item < span * NSEG_V; item += BT_NT) {
        const int xc = item % span, seg = item / span;
        const int gx = x0 - r + xc;
        const int ya = y0 + seg * BT_RV;
        const int vrow = seg * BT_RV;
        if (gx < 0 || gx >= w || ya >= h) {
#pragma unroll
            for (int i = 0; i < BT_RV; ++i)
#pragma unroll
                for (int q = 0; q < NQ; ++q) Vt[((size_t)q * span + xc) * BT_VP + vrow + i] = 0.0f;
            continue;
        }
        float S[NQ], Sc[NQ];
        uint32_t U[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) { S[q] = 0.0f; Sc[q] = 0.0f; U[q] = 0u; }
        auto add_row = [&](int yy, bool sub) {
            const float xv = xval(yy, gx), yv = yval(yy, gx);
            if (INT) {
                uint32_t qv[4];
                Q::of_int(xv, yv, qv);
#pragma unroll
                for (int q = 0; q < NQ; ++q) U[q] = sub ? U[q] - qv[q] : U[q] + qv[q];
            } else {
                float qv[NQ];
                Q::of(xv, yv, cx, cy, qv);
#pragma unroll
                for (int q = 0; q < NQ; ++q) kadd<COMP>(S[q], Sc[q], sub ? -qv[q] : qv[q]);
            }
        };
        const int lo = max(0, ya - r), hi = min(h - 1, ya + r);
#pragma unroll 4
        for (int yy = lo; yy <= hi; ++yy) add_row(yy, false);
#pragma unroll
        for (int i = 0; i < BT_RV; ++i) {
            const int y = ya + i;
            if (i > 0) {
                if (y + r < h) add_row(y + r, false);
                if (y - r - 1 >= 0) add_row(y - r - 1, true);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const size_t vi = ((size_t)q * span + xc) * BT_VP + vrow + i;
                if (INT) Vu[vi] = U[q];
                else Vt[vi] = S[q] + Sc[q];
            }
        }
    }
    __syncthreads();

    // ---- phase 2: horizontal window sums along each tile row, then the epilogue
    constexpr int NSEG_H = BT_TW / BT_RH;
    for (int item = tid; item < BT_TH * NSEG_H; item += BT_NT) {
        const int yr = item % BT_TH, seg = item / BT_TH;
        const int y = y0 + yr;
        const int xa = seg * BT_RH;
        if (y >= h || x0 + xa >= w) continue;
        const int ny = min(h - 1, y + r) - max(0, y - r) + 1;
        float S[NQ], Sc[NQ];
        uint32_t U[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) { S[q] = 0.0f; Sc[q] = 0.0f; U[q] = 0u; }
        auto vget = [&](int q, int col) -> size_t { return ((size_t)q * span + col) * BT_VP + yr; };
        // window of tile column xa covers span columns [xa, xa + 2r]; out-of-image columns hold zeros
        for (int k = 0; k <= 2 * r; ++k) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (INT) U[q] += Vu[vget(q, xa + k)];
                else kadd<COMP>(S[q], Sc[q], Vt[vget(q, xa + k)]);
            }
        }
#pragma unroll
        for (int i = 0; i < BT_RH; ++i) {
            const int xt = xa + i, x = x0 + xt;
            if (x >= w) break;
            if (i > 0) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    if (INT) {
                        U[q] += Vu[vget(q, xt + 2 * r)];
                        U[q] -= Vu[vget(q, xt - 1)];
                    } else {
                        kadd<COMP>(S[q], Sc[q], Vt[vget(q, xt + 2 * r)]);
                        kadd<COMP>(S[q], Sc[q], -Vt[vget(q, xt - 1)]);
                    }
                }
            }
            const int nx = min(w - 1, x + r) - max(0, x - r) + 1;
            const int cnt = nx * ny;
            float o0, o1;
            if (KIND == KIND_STATS_F) {
                const float inv = __fdividef(1.0f, (float)cnt);
                const float mI = (S[0] + Sc[0]) * inv, mp = (S[2] + Sc[2]) * inv;  // shifted means
                const float eII = (S[1] + Sc[1]) * inv, eIp = (S[3] + Sc[3]) * inv;
                // var_I, cov_Ip: exactly 0 for a one-sample window (r' = 0), where Eq. 2 gives a = 0
                const float var = r ? fmaxf(eII - mI * mI, 0.0f) : 0.0f;
                const float cov = r ? eIp - mI * mp : 0.0f;
                o0 = __fdividef(cov, var + P.eps);             // a, Eq. (2)
                o1 = (mp + cy) - o0 * (mI + cx);               // b, Eq. (3)
                if (P.stats) {
                    const size_t ps = (size_t)h * w;
                    float *st = (float *)P.stats + (size_t)plane * 4 * ps + (size_t)y * w + x;
                    st[0] = mI + cx;
                    st[ps] = eII + cx * (2.0f * mI + cx);
                    st[2 * ps] = mp + cy;
                    st[3 * ps] = eIp + cx * mp + cy * mI + cx * cy;
                }
            } else if (KIND == KIND_STATS_INT) {
                const long long nn = cnt;
                // exact integer numerators of var and cov, scaled by n^2 (255k)^2
                const long long vnum = nn * (long long)U[1] - (long long)U[0] * (long long)U[0];
                const long long cnum = nn * (long long)U[3] - (long long)U[0] * (long long)U[2];
                const float den = (float)vnum + P.eps * ((float)nn * (float)nn) * (P.int_scale * P.int_scale);
                o0 = __fdividef((float)cnum, den);                                              // a, Eq. (2)
                o1 = __fdividef((float)U[2] - o0 * (float)U[0], (float)cnt * P.int_scale);      // b, Eq. (3)
                if (P.stats) {
                    const size_t ps = (size_t)h * w;
                    uint32_t *st = (uint32_t *)P.stats + (size_t)plane * 4 * ps + (size_t)y * w + x;
                    st[0] = U[0]; st[ps] = U[1]; st[2 * ps] = U[2]; st[3 * ps] = U[3];
                }
            } else {
                const float inv = __fdividef(1.0f, (float)cnt);
                o0 = (S[0] + Sc[0]) * inv + cx;
                o1 = (S[1] + Sc[1]) * inv + cy;
            }
            Ot[yr * BT_OP + xt] = o0;
            Ot[BT_TH * BT_OP + yr * BT_OP + xt] = o1;
        }
    }
    __syncthreads();

    // ---- phase 3: coalesced write of the tile
    const size_t obase = (size_t)plane * P.ops;
    for (int idx = tid; idx < BT_TH * BT_TW; idx += BT_NT) {
        const int yr = idx / BT_TW, xt = idx - yr * BT_TW;
        const int y = y0 + yr, x = x0 + xt;
        if (y < h && x < w) {
            P.out0[obase + (size_t)y * w + x] = Ot[yr * BT_OP + xt];
            P.out1[obase + (size_t)y * w + x] = Ot[BT_TH * BT_OP + yr * BT_OP + xt];
        }
    }
    pdl_trigger();
}

// Packed form of k_box_tile for the FP32 kinds (KIND 0 and 2) at r' <= 16: the window sums travel as float2
// pairs -- (dx, dy) and (dx^2, dx dy) for the statistics, (a, b) for the means -- through registers, a float2
// column-sum tile (64-bit shared accesses) and the sliding updates, so every add, subtract and product
// covers two quantities in one f32x2 instruction.  Same tiling, phases and epilogue as k_box_tile.
template <typename T, int KIND, int BT_RV, int BT_RH, int RC = 0>
__global__ void __launch_bounds__(BT_NT_MAX) k_box_tile_x2(BoxParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    constexpr int NP = (KIND == KIND_MEAN2) ? 1 : 2;  // float2 pairs
    // uint8 input (KIND 1): the samples are integers J, P <= 1020 and J^2, J P <= 1020^2 < 2^24, so the
    // unshifted FP32 column sums of at most 2 r' + 2 <= 10 rows are exact; they are staged as uint32 and the
    // horizontal sums and the variance and covariance numerators are exact integers (r' <= 4 only).
    constexpr bool INT = (KIND == KIND_STATS_INT);
    static_assert(!INT || (RC > 0 && RC <= 4), "the integer form needs a compile-time r' <= 4");
    extern __shared__ float smf[];
    const int BT_NT = blockDim.x;
    const int tid = threadIdx.x;
    const int h = P.h, w = P.w;
    const int r = RC > 0 ? RC : P.r;  // compile-time for the common small radii
    const int span = BT_TW + 2 * r;
    float2 *Vt = reinterpret_cast<float2 *>(smf);           // [NP][span][BT_VP]
    float *Ot = smf + (size_t)2 * NP * span * BT_VP;         // [2][BT_TH][BT_OP]
    float *St = Ot + 2 * BT_TH * BT_OP;                      // [4][BT_TH][BT_OP] window statistics (P.stats only)
    const int x0 = blockIdx.x * BT_TW, y0 = blockIdx.y * BT_TH;
    const int plane = blockIdx.z;
    const int n = plane / P.C, c = plane - n * P.C;
    const T *Xp = (const T *)P.X + (size_t)(n * P.CX + (P.CX == 1 ? 0 : c)) * P.xps;
    const T *Yp = (const T *)P.Y + (size_t)plane * P.yps;
    const float2 shift = INT ? make_float2(0.0f, 0.0f)
                             : make_float2(ldv(Xp + (size_t)y0 * w + x0), ldv(Yp + (size_t)y0 * w + x0));
    uint2 *Vu = reinterpret_cast<uint2 *>(smf);  // INT: the same tile as uint32 pairs

    // ---- phase 1: vertical window sums
    constexpr int NSEG_V = BT_TH / BT_RV;
    for (int item = tid; item < span * NSEG_V; item += BT_NT) {
        const int xc = item % span, seg = item / span;
        const int gx = x0 - r + xc;
        const int ya = y0 + seg * BT_RV, vrow = seg * BT_RV;
        float2 S[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) S[k] = make_float2(0.0f, 0.0f);
        if constexpr (RC > 0) {
            // radius known at compile time: the RV + 2 RC rows of the segment's window span are requested at
            // once into registers; rows outside the image contribute nothing
            constexpr int NR = BT_RV + 2 * RC;
            float2 v[NR];
            bool ok[NR];
            if (gx >= 0 && gx < w && ya < h) {
                const T *xc_p = Xp + gx, *yc_p = Yp + gx;
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const int yy = ya - RC + k;
                    ok[k] = (yy >= 0) && (yy < h);
                    v[k] = ok[k] ? make_float2(ldv(xc_p + yy * w), ldv(yc_p + yy * w)) : shift;
                }
                auto acc = [&](int k, bool sub) {
                    const float2 d = sub2(v[k], shift);  // zero for rows outside the image
                    if (sub) S[0] = sub2(S[0], d); else S[0] = add2(S[0], d);
                    if (NP == 2) {
                        const float2 pr = mul2(make_float2(d.x, d.x), d);  // (dx^2, dx dy)
                        if (sub) S[NP - 1] = sub2(S[NP - 1], pr); else S[NP - 1] = add2(S[NP - 1], pr);
                    }
                };
#pragma unroll
                for (int k = 0; k <= 2 * RC; ++k) acc(k, false);
#pragma unroll
                for (int i = 0; i < BT_RV; ++i) {
                    if (i > 0) {
                        acc(i + 2 * RC, false);
                        acc(i - 1, true);
                    }
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const size_t vi = ((size_t)k * span + xc) * BT_VP + vrow + i;
                        if (INT) Vu[vi] = make_uint2(__float2uint_rn(S[k].x), __float2uint_rn(S[k].y));
                        else Vt[vi] = S[k];
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < BT_RV; ++i)
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const size_t vi = ((size_t)k * span + xc) * BT_VP + vrow + i;
                        if (INT) Vu[vi] = make_uint2(0u, 0u);
                        else Vt[vi] = S[k];
                    }
            }
            continue;
        }
        if (gx >= 0 && gx < w && ya < h) {
            const T *xc_p = Xp + gx, *yc_p = Yp + gx;
            auto row = [&](int yy, bool sub) {
                const int off = yy * w;
                const float2 d = sub2(make_float2(ldv(xc_p + off), ldv(yc_p + off)), shift);
                if (sub) S[0] = sub2(S[0], d); else S[0] = add2(S[0], d);
                if (NP == 2) {
                    const float2 pr = mul2(make_float2(d.x, d.x), d);  // (dx^2, dx dy)
                    if (sub) S[NP - 1] = sub2(S[NP - 1], pr); else S[NP - 1] = add2(S[NP - 1], pr);
                }
            };
            const int lo = max(0, ya - r), hi = min(h - 1, ya + r);
#pragma unroll 4
            for (int yy = lo; yy <= hi; ++yy) row(yy, false);
#pragma unroll
            for (int i = 0; i < BT_RV; ++i) {
                const int y = ya + i;
                if (i > 0) {
                    if (y + r < h) row(y + r, false);
                    if (y - r - 1 >= 0) row(y - r - 1, true);
                }
#pragma unroll
                for (int k = 0; k < NP; ++k) Vt[((size_t)k * span + xc) * BT_VP + vrow + i] = S[k];
            }
        } else {
#pragma unroll
            for (int i = 0; i < BT_RV; ++i)
#pragma unroll
                for (int k = 0; k < NP; ++k) Vt[((size_t)k * span + xc) * BT_VP + vrow + i] = S[k];
        }
    }
    __syncthreads();

    // ---- phase 2: horizontal window sums and the epilogue
    constexpr int NSEG_H = BT_TW / BT_RH;
    const size_t kstride = (size_t)span * BT_VP;  // between the pair planes of Vt
    for (int item = tid; item < BT_TH * NSEG_H; item += BT_NT) {
        const int yr = item % BT_TH, seg = item / BT_TH;
        const int y = y0 + yr, xa = seg * BT_RH;
        if (y >= h || x0 + xa >= w) continue;
        const int ny = min(h - 1, y + r) - max(0, y - r) + 1;
        const float2 *col = Vt + yr;  // column k of pair plane q at col[q * kstride + k * BT_VP]
        const uint2 *ucol = Vu + yr;
        float2 S[NP];
        uint2 U[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) { S[k] = make_float2(0.0f, 0.0f); U[k] = make_uint2(0u, 0u); }
#pragma unroll
        for (int k = 0; k <= 2 * r; ++k) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                if (INT) {
                    const uint2 t = ucol[q * kstride + (size_t)(xa + k) * BT_VP];
                    U[q].x += t.x; U[q].y += t.y;
                } else {
                    S[q] = add2(S[q], col[q * kstride + (size_t)(xa + k) * BT_VP]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < BT_RH; ++i) {
            const int xt = xa + i, x = x0 + xt;
            if (x >= w) break;
            if (i > 0) {
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    if (INT) {
                        const uint2 a = ucol[q * kstride + (size_t)(xt + 2 * r) * BT_VP];
                        const uint2 b = ucol[q * kstride + (size_t)(xt - 1) * BT_VP];
                        U[q].x = U[q].x + a.x - b.x;
                        U[q].y = U[q].y + a.y - b.y;
                    } else {
                        S[q] = sub2(add2(S[q], col[q * kstride + (size_t)(xt + 2 * r) * BT_VP]),
                                    col[q * kstride + (size_t)(xt - 1) * BT_VP]);
                    }
                }
            }
            const int nx = min(w - 1, x + r) - max(0, x - r) + 1;
            const float inv = __fdividef(1.0f, (float)(nx * ny));
            float o0, o1;
            if (INT) {
                // exact integer numerators of var and cov (n^2 (255 k)^2 times them), as k_box_tile forms them
                const long long nn = nx * ny;
                const long long vnum = nn * (long long)U[1].x - (long long)U[0].x * (long long)U[0].x;
                const long long cnum = nn * (long long)U[1].y - (long long)U[0].x * (long long)U[0].y;
                const float den = (float)vnum + P.eps * ((float)nn * (float)nn) * (P.int_scale * P.int_scale);
                o0 = __fdividef((float)cnum, den);                                                   // a, Eq. (2)
                o1 = __fdividef((float)U[0].y - o0 * (float)U[0].x, (float)(nx * ny) * P.int_scale);  // b, Eq. (3)
                if (P.stats) {  // the integer window sums, staged as bit patterns
                    const int so = yr * BT_OP + xt;
                    St[so] = __uint_as_float(U[0].x);
                    St[BT_TH * BT_OP + so] = __uint_as_float(U[1].x);
                    St[2 * BT_TH * BT_OP + so] = __uint_as_float(U[0].y);
                    St[3 * BT_TH * BT_OP + so] = __uint_as_float(U[1].y);
                }
            } else if (KIND == KIND_STATS_F) {
                const float mI = S[0].x * inv, mp = S[0].y * inv;    // shifted means
                const float eII = S[1].x * inv, eIp = S[1].y * inv;
                // var_I, cov_Ip: exactly 0 for a one-sample window (r' = 0), where Eq. 2 gives a = 0
                const float var = r ? fmaxf(eII - mI * mI, 0.0f) : 0.0f;
                const float cov = r ? eIp - mI * mp : 0.0f;
                o0 = __fdividef(cov, var + P.eps);                 // a, Eq. (2)
                o1 = (mp + shift.y) - o0 * (mI + shift.x);         // b, Eq. (3)
                if (P.stats) {  // staged, written as coalesced rows in phase 3
                    const float cx = shift.x, cy = shift.y;
                    const int so = yr * BT_OP + xt;
                    St[so] = mI + cx;
                    St[BT_TH * BT_OP + so] = eII + cx * (2.0f * mI + cx);
                    St[2 * BT_TH * BT_OP + so] = mp + cy;
                    St[3 * BT_TH * BT_OP + so] = eIp + cx * mp + cy * mI + cx * cy;
                }
            } else {
                o0 = S[0].x * inv + shift.x;
                o1 = S[0].y * inv + shift.y;
            }
            Ot[yr * BT_OP + xt] = o0;
            Ot[BT_TH * BT_OP + yr * BT_OP + xt] = o1;
        }
    }
    __syncthreads();

    // ---- phase 3: coalesced write of the tile
    const size_t obase = (size_t)plane * P.ops;
    for (int idx = tid; idx < BT_TH * BT_TW; idx += BT_NT) {
        const int yr = idx / BT_TW, xt = idx - yr * BT_TW;
        const int y = y0 + yr, x = x0 + xt;
        if (y < h && x < w) {
            P.out0[obase + (size_t)y * w + x] = Ot[yr * BT_OP + xt];
            P.out1[obase + (size_t)y * w + x] = Ot[BT_TH * BT_OP + yr * BT_OP + xt];
            if (KIND != KIND_MEAN2 && P.stats) {  // FP32 statistics, or the uint32 window sums (KIND 1)
                const size_t ps = (size_t)h * w;
                uint32_t *st = (uint32_t *)P.stats + (size_t)plane * 4 * ps + (size_t)y * w + x;
#pragma unroll
                for (int q = 0; q < 4; ++q) st[q * ps] = __float_as_uint(St[q * BT_TH * BT_OP + yr * BT_OP + xt]);
            }
        }
    }
    pdl_trigger();
}

// ------------------------------------------------------------------------------------------------------
// k_upsample_output / k_output_s1
// ------------------------------------------------------------------------------------------------------
constexpr int UP_NT = 128;            // threads per CTA, 4 columns each
constexpr int UP_NST = 4;             // quads of I rows in the s = 4, 8 kernel's shared ring
constexpr int UP_BAND = UP_NT * 4;    // full-res columns per CTA

struct UpParams {
    const void *I;
    const float *ma, *mb;
    void *q;
    int C, CI, H, W, h, w, s, R, CG;  // R: full-res rows per CTA; CG: channel groups per image
    size_t lps;                       // low-res plane stride
    int LRmax, LCmax;                 // staged low-res tile bounds (rows, columns)
    float detail;                     // detail gain k: output q + k (I - q) (0: q itself)
    int sn, sd;                       // the ratio as sn / sd (generic kernel; s = sn, sd = 1 if integer)
    size_t fps;                       // plane stride of the full-res I and q (elements)
    int Yw0, Yw1;                     // rows written: [Yw0, Yw1) of the H rows
    FaultSink fault;                  // the TMA-fed form's bounded waits
};

template <typename T>
__device__ __forceinline__ void ld4(const T *p, bool vec, int valid, float v[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float *p, bool vec, int valid, float v[4])
{
    if (vec) {
        const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (k < valid) ? __ldcs(p + k) : 0.0f;
    }
}
template <>
__device__ __forceinline__ void ld4<__half>(const __half *p, bool vec, int valid, float v[4])
{
    if (vec) {
        const uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
        const __half2 lo = *reinterpret_cast<const __half2 *>(&t.x), hi = *reinterpret_cast<const __half2 *>(&t.y);
        const float2 a = __half22float2(lo), b = __half22float2(hi);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (k < valid) ? __half2float(p[k]) : 0.0f;
    }
}
template <>
__device__ __forceinline__ void ld4<uint8_t>(const uint8_t *p, bool vec, int valid, float v[4])
{
    if (vec) {
        const uint32_t t = __ldcs(reinterpret_cast<const unsigned int *>(p));
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = u8_unit((t >> (8 * k)) & 0xffu);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (k < valid) ? u8_unit(p[k]) : 0.0f;
    }
}

template <typename TI, typename TQ, int CC, bool VEC>
__global__ void __launch_bounds__(UP_NT) k_upsample_output(UpParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    extern __shared__ float tap[];  // [CC][2][LRmax][LCmax] low-res tap tile (mean_a, mean_b)
    const int Xb = blockIdx.x * UP_BAND;
    const int Yb = max(blockIdx.y * P.R, P.Yw0), Ye = min(min(blockIdx.y * P.R + P.R, P.H), P.Yw1);
    if (Yb >= Ye) return;  // the whole CTA is outside the written rows
    const int n = blockIdx.z / P.CG, c0 = (blockIdx.z - n * P.CG) * CC;
    const int ncc = min(CC, P.C - c0);
    const size_t HW = P.fps;

    // low-res rows / columns this CTA samples
    int ly0, ly1, lx0, lx1, t0, t1;
    float ft;
    up_taps_q(Yb, P.sn, P.sd, P.h, ly0, t0, ft);
    up_taps_q(Ye - 1, P.sn, P.sd, P.h, t0, ly1, ft);
    up_taps_q(Xb, P.sn, P.sd, P.w, lx0, t1, ft);
    up_taps_q(min(Xb + UP_BAND, P.W) - 1, P.sn, P.sd, P.w, t1, lx1, ft);
    const int LR = ly1 - ly0 + 1, LC = lx1 - lx0 + 1;
    const int tile = P.LRmax * P.LCmax;
    for (int mr = 0; mr < CC * 2 * LR; ++mr) {  // (map, row) pairs; mc = cc * 2 + map
        const int mc = mr / LR, row = mr - mc * LR;
        const int c = min(c0 + (mc >> 1), P.C - 1);
        const float *src = ((mc & 1) ? P.mb : P.ma) + (size_t)(n * P.C + c) * P.lps + (size_t)(ly0 + row) * P.w + lx0;
        float *dst = tap + mc * tile + row * P.LCmax;
        for (int col = threadIdx.x; col < LC; col += UP_NT) cp_async4(dst + col, src + col);
    }
    cp_async_wait_all();
    __syncthreads();

    const int X0 = Xb + threadIdx.x * 4;
    if (X0 >= P.W) return;
    const int valid = min(4, P.W - X0);
    const bool vec = VEC && (valid == 4);

    const TI *Ig[CC];
    TQ *Qp[CC];
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
        const int c = min(c0 + cc, P.C - 1);
        Qp[cc] = (TQ *)P.q + (size_t)(n * P.C + c) * HW;
        Ig[cc] = (const TI *)P.I + (size_t)(n * P.CI + (P.CI == 1 ? 0 : c)) * HW;
    }

    int xa[4], xb[4];
    float fx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        up_taps_q(min(X0 + k, P.W - 1), P.sn, P.sd, P.w, xa[k], xb[k], fx[k]);
        xa[k] -= lx0;
        xb[k] -= lx0;
    }

    // horizontally interpolated tap rows: slot 0 = upper tap row, slot 1 = lower tap row
    float ha[CC][2][4], hb[CC][2][4];
    int cur0 = -1, cur1 = -1;
    auto load_row = [&](int yy, int slot) {
#pragma unroll
        for (int cc = 0; cc < CC; ++cc) {
            const float *ra = tap + (cc * 2) * tile + (yy - ly0) * P.LCmax;
            const float *rb = ra + tile;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float a0 = ra[xa[k]], a1 = ra[xb[k]];
                const float b0 = rb[xa[k]], b1 = rb[xb[k]];
                ha[cc][slot][k] = fmaf(fx[k], a1 - a0, a0);
                hb[cc][slot][k] = fmaf(fx[k], b1 - b0, b0);
            }
        }
    };

    for (int Yg = Yb; Yg < Ye; Yg += 4) {
        float iv[4][4];
        if (P.CI == 1) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (Yg + u < Ye) ld4<TI>(Ig[0] + (size_t)(Yg + u) * P.W + X0, vec, valid, iv[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int Y = Yg + u;
            if (Y >= Ye) break;
            int ya, yb;
            float fy;
            up_taps_q(Y, P.sn, P.sd, P.h, ya, yb, fy);
            if (ya != cur0) {
                if (ya == cur1) {
#pragma unroll
                    for (int cc = 0; cc < CC; ++cc)
#pragma unroll
                        for (int k = 0; k < 4; ++k) { ha[cc][0][k] = ha[cc][1][k]; hb[cc][0][k] = hb[cc][1][k]; }
                } else {
                    load_row(ya, 0);
                }
                cur0 = ya;
                cur1 = -1;
            }
            if (yb != cur1) {
                if (yb == cur0) {
#pragma unroll
                    for (int cc = 0; cc < CC; ++cc)
#pragma unroll
                        for (int k = 0; k < 4; ++k) { ha[cc][1][k] = ha[cc][0][k]; hb[cc][1][k] = hb[cc][0][k]; }
                } else {
                    load_row(yb, 1);
                }
                cur1 = yb;
            }
#pragma unroll
            for (int cc = 0; cc < CC; ++cc) {
                if (cc >= ncc) break;
                float ivc[4];
                if (P.CI == 1) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) ivc[k] = iv[u][k];
                } else {
                    ld4<TI>(Ig[cc] + (size_t)Y * P.W + X0, vec, valid, ivc);
                }
                float out[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float A = fmaf(fy, ha[cc][1][k] - ha[cc][0][k], ha[cc][0][k]);  // upsampled mean_a
                    const float B = fmaf(fy, hb[cc][1][k] - hb[cc][0][k], hb[cc][0][k]);  // upsampled mean_b
                    out[k] = fmaf(A, ivc[k], B);                                           // Eq. (4)
                }
                detail_epilogue(P.detail, ivc, out);
                st4<TQ>(Qp[cc] + (size_t)Y * P.W + X0, vec, valid, out);
            }
        }
    }
    pdl_trigger();
}

// s = 4 or 8, 4-aligned rows (one guide channel for all of p, or one per channel).  Full-res row S*j + S/2 + k (k = 0 .. S-1) samples low-res
// rows j and j+1 with weight (2k + 1)/(2S) on row j+1, so the rows are walked in such S-row runs: one pair of
// horizontally interpolated tap rows (and their difference) serves the whole run.  Columns: pixels 4t .. 4t+3
// sample low-res columns i-1, i, i+1 (S = 4) or one adjacent pair of them (S = 8) with fixed weights.  Taps
// beyond the image are clamped copies, which gives the same value as clamping the sample position.
// One channel per CTA; the channel is the fastest-varying block index, so with one guide channel the CTAs
// of one band of I run side by side and share I through L2.
template <typename TI, typename TQ, int S>
__global__ void __launch_bounds__(UP_NT, 8) k_upsample_output_s4x(UpParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    extern __shared__ float tap[];  // [2][LRmax][LCmax]: mean_a, mean_b at low-res rows jb-1 .. jb+nb, clamped
    const int nb = P.R / S;         // low-res rows (bands) per CTA
    const int jb = blockIdx.y * nb;
    const int c = blockIdx.x % P.C, band = blockIdx.x / P.C;
    const int n = blockIdx.z;
    const int Xb = band * UP_BAND;
    const int Yb = max(jb * S, P.Yw0), Ye = min(min(jb * S + P.R, P.H), P.Yw1);  // rows written by this CTA
    if (Yb >= Ye) return;
    const int ly0 = jb - 1, lx0 = Xb / S - 1;
    const int LR = P.LRmax, LC = P.LCmax, tile = LR * LC;
    {
        // asynchronous fill of the tap tile; each thread owns at most two tile columns
        const int c0 = threadIdx.x, c1 = threadIdx.x + UP_NT;
        const int g0 = min(max(lx0 + c0, 0), P.w - 1), g1 = min(max(lx0 + c1, 0), P.w - 1);
        const float *pa = P.ma + (size_t)(n * P.C + c) * P.lps, *pb = P.mb + (size_t)(n * P.C + c) * P.lps;
        for (int row = 0; row < LR; ++row) {
            const size_t go = (size_t)min(max(ly0 + row, 0), P.h - 1) * P.w;
            float *da = tap + row * LC, *db = da + tile;
            if (c0 < LC) { cp_async4(da + c0, pa + go + g0); cp_async4(db + c0, pb + go + g0); }
            if (c1 < LC) { cp_async4(da + c1, pa + go + g1); cp_async4(db + c1, pb + go + g1); }
        }
        cp_async_wait_all();
        __syncthreads();
    }

    const int X0 = Xb + threadIdx.x * 4;
    if (X0 >= P.W) return;
    const int ti = X0 / S - lx0;  // tile column of the low-res column that holds pixel X0 (>= 1)
    const int g = (S == 8) ? ((X0 >> 2) & 1) : 0;

    // horizontally interpolated tap row `tr` for the thread's 4 pixels, both maps
    auto hrow = [&](int tr, float (&o)[2][4]) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
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

    const size_t HW = P.fps;
    const TI *Ip = (const TI *)P.I + (size_t)(n * P.CI + (P.CI == 1 ? 0 : c)) * HW + X0;
    TQ *Qp = (TQ *)P.q + (size_t)(n * P.C + c) * HW + X0;

    // Run j covers full-res rows S*j + S/2 .. S*j + S/2 + S - 1 and samples low-res rows j and j+1 (tile
    // rows t and t+1 for t = j - jb + 1).  Runs are walked in quads of 4 rows.  The I values of the next
    // UP_NST - 1 quads are in flight at any time: each thread copies its own 4 pixels of every row into its
    // slots of a shared ring with 16-byte cp.async and reads back only what it copied itself, so the only
    // synchronisation is the thread's own cp.async group wait.
    constexpr int QPR = S / 4;  // quads per run
    constexpr int VB = 4 * (int)sizeof(TI);  // bytes of one row's 4 pixels
    const int nquads = (nb + 1) * QPR;
    unsigned char *ring = reinterpret_cast<unsigned char *>(tap + 2 * tile);  // [UP_NST][4 rows][UP_NT][VB]
    auto slot = [&](int stage, int k) { return ring + ((size_t)(stage * 4 + k) * UP_NT + threadIdx.x) * VB; };
    auto issue_quad = [&](int u) {
        if (u < nquads) {
            const int Yq = S * (jb - 1 + u / QPR) + S / 2 + 4 * (u % QPR);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int Y = Yq + k;
                if (Y >= Yb && Y < Ye) {
                    if (VB == 16) cp_async16(slot(u % UP_NST, k), Ip + (size_t)Y * P.W);
                    else ld_async_small<TI>(slot(u % UP_NST, k), Ip + (size_t)Y * P.W);
                }
            }
        }
        cp_async_commit();  // one group per quad, empty past the end, so the group count stays uniform
    };
    float lo[2][4], d[2][4];
    hrow(0, lo);  // low-res row jb - 1
#pragma unroll
    for (int u = 0; u < UP_NST - 1; ++u) issue_quad(u);
    for (int u = 0; u < nquads; ++u) {
        issue_quad(u + UP_NST - 1);
        cp_async_wait_group<UP_NST - 1>();  // this thread's copies of quad u have landed
        const int t = u / QPR, sub = u % QPR;
        const int Yq = S * (jb - 1 + t) + S / 2 + 4 * sub;
        if (Yq >= Ye) break;
        if (sub == 0) {
            if (t > 0) {  // the previous run's lower tap row becomes this run's upper one
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                    for (int x = 0; x < 4; ++x) lo[m][x] += d[m][x];
            }
            hrow(t + 1, d);
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int x = 0; x < 4; ++x) d[m][x] -= lo[m][x];
        }
        const float fy0 = (S == 4) ? 0.125f : (sub ? 0.5625f : 0.0625f);  // (8 sub + 1) / (2S)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int Y = Yq + k;
            if (Y < Yb || Y >= Ye) continue;
            float iv[4];
            ld4_shared<TI>(slot(u % UP_NST, k), iv);
            const float fy = fy0 + (float)k / (float)S;
            float out[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const float A = fmaf(fy, d[0][x], lo[0][x]);  // upsampled mean_a
                const float B = fmaf(fy, d[1][x], lo[1][x]);  // upsampled mean_b
                out[x] = fmaf(A, iv[x], B);                   // Eq. (4)
            }
            detail_epilogue(P.detail, iv, out);
            st4<TQ>(Qp + (size_t)Y * P.W, true, 4, out);
        }
    }
    cp_async_wait_all();
    pdl_trigger();
}

template <typename TI, typename TQ, int CC, bool VEC>
__global__ void __launch_bounds__(UP_NT) k_output_s1(UpParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    const int X0 = (blockIdx.x * UP_NT + threadIdx.x) * 4;
    if (X0 >= P.W) return;
    const int valid = min(4, P.W - X0);
    const bool vec = VEC && (valid == 4);
    const int Yb = max(blockIdx.y * P.R, P.Yw0), Ye = min(min(blockIdx.y * P.R + P.R, P.H), P.Yw1);
    const int n = blockIdx.z / P.CG, c0 = (blockIdx.z - n * P.CG) * CC;
    const int ncc = min(CC, P.C - c0);
    const size_t HW = P.fps;
    for (int Y = Yb; Y < Ye; ++Y) {
        float iv[4];
        if (P.CI == 1) ld4<TI>((const TI *)P.I + (size_t)n * HW + (size_t)Y * P.W + X0, vec, valid, iv);
        float A[CC][4], B[CC][4];
#pragma unroll
        for (int cc = 0; cc < CC; ++cc) {
            if (cc >= ncc) break;
            const size_t lo = (size_t)(n * P.C + c0 + cc) * P.lps + (size_t)Y * P.W + X0;
            ld4<float>(P.ma + lo, vec, valid, A[cc]);
            ld4<float>(P.mb + lo, vec, valid, B[cc]);
        }
#pragma unroll
        for (int cc = 0; cc < CC; ++cc) {
            if (cc >= ncc) break;
            const int c = c0 + cc;
            if (P.CI != 1) ld4<TI>((const TI *)P.I + (size_t)(n * P.CI + c) * HW + (size_t)Y * P.W + X0, vec, valid, iv);
            float out[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) out[k] = fmaf(A[cc][k], iv[k], B[cc][k]);  // Eq. (4), s = 1
            detail_epilogue(P.detail, iv, out);
            st4<TQ>((TQ *)P.q + (size_t)(n * P.C + c) * HW + (size_t)Y * P.W + X0, vec, valid, out);
        }
    }
    pdl_trigger();
}

// ------------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------------
cudaError_t opt_in_smem(const void *func, size_t smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;  // (kernel, device) -> bytes opted in
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = done[{func, dev}];
    if (smem <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) have = smem;
    return e;
}

namespace {

struct StageTimer {
    cudaEvent_t *ev;
    cudaStream_t st;
    int k = 0;
    void before() { if (ev && k < GF_MAX_STAGES) cudaEventRecord(ev[2 * k], st); }
    void after() { if (ev && k < GF_MAX_STAGES) cudaEventRecord(ev[2 * k + 1], st); ++k; }
};

template <typename T>
void launch_sub_t(const SubParams &sp, dim3 grid, cudaStream_t st)
{
    switch (sp.mode) {
    case GF_SUB_NEAREST: launch_pdl(k_subsample<T, GF_SUB_NEAREST>, grid, dim3(SUB_NT), 0, st, sp); break;
    case GF_SUB_BILINEAR: launch_pdl(k_subsample<T, GF_SUB_BILINEAR>, grid, dim3(SUB_NT), 0, st, sp); break;
    case GF_SUB_BOX: launch_pdl(k_subsample<T, GF_SUB_BOX>, grid, dim3(SUB_NT), 0, st, sp); break;
    default: launch_pdl(k_subsample_aa<T>, grid, dim3(SUB_NT), 0, st, sp); break;
    }
}

template <typename T, int KIND, bool COMP, int RV, int RH>
cudaError_t launch_box_v(const BoxParams &bp, int planes, cudaStream_t st)
{
    const int nq = (KIND == KIND_MEAN2) ? 2 : 4;
    const size_t smem = box_tile_smem(nq, bp.r);
    cudaError_t e = opt_in_smem(k_box_tile<T, KIND, COMP, RV, RH>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((bp.w + BT_TW - 1) / BT_TW, (bp.h + BT_TH - 1) / BT_TH, planes);
    // one phase-1 item (column segment) per thread when it fits; phase 2 needs BT_TH * BT_TW / RH <= 256
    const int items = (BT_TW + 2 * bp.r) * (BT_TH / RV);
    const int nt = std::min(BT_NT_MAX, std::max(256, (items + 31) / 32 * 32));
    launch_pdl(k_box_tile<T, KIND, COMP, RV, RH>, grid, dim3(nt), smem, st, bp);
    return cudaGetLastError();
}

// Segment lengths grow with the radius (a segment pays 2r'+1 loads to open its window); compensated
// sums for windows of more than 33 x 33 terms.
template <typename T, int KIND, int RV, int RH, int RC = 0>
cudaError_t launch_box_x2(const BoxParams &bp, int planes, cudaStream_t st)
{
    const int nq = (KIND == KIND_MEAN2) ? 2 : 4;
    // plus the staging tile of the four window statistics when they are an output
    const size_t smem = box_tile_smem(nq, bp.r) +
                        ((KIND != KIND_MEAN2 && bp.stats) ? (size_t)4 * BT_TH * BT_OP * sizeof(float) : 0);
    cudaError_t e = opt_in_smem(k_box_tile_x2<T, KIND, RV, RH, RC>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((bp.w + BT_TW - 1) / BT_TW, (bp.h + BT_TH - 1) / BT_TH, planes);
    const int items = (BT_TW + 2 * bp.r) * (BT_TH / RV);
    const int nt = std::min(BT_NT_MAX, std::max(256, (items + 31) / 32 * 32));
    launch_pdl(k_box_tile_x2<T, KIND, RV, RH, RC>, grid, dim3(nt), smem, st, bp);
    return cudaGetLastError();
}

template <typename T, int KIND>
cudaError_t launch_box_t(const BoxParams &bp, int planes, cudaStream_t st)
{
    if constexpr (KIND == KIND_STATS_INT && std::is_same<T, float>::value) {
        switch (bp.r) {  // exact FP32 column sums staged as integers (k_box_tile_x2), r' <= 4
        case 1: return launch_box_x2<T, KIND, 8, 8, 1>(bp, planes, st);
        case 2: return launch_box_x2<T, KIND, 8, 8, 2>(bp, planes, st);
        case 3: return launch_box_x2<T, KIND, 8, 8, 3>(bp, planes, st);
        case 4: return launch_box_x2<T, KIND, 8, 8, 4>(bp, planes, st);
        default: break;
        }
    }
    if constexpr (KIND != KIND_STATS_INT) {
        switch (bp.r) {  // common small radii with the radius known at compile time
        case 1: return launch_box_x2<T, KIND, 8, 8, 1>(bp, planes, st);
        case 2: return launch_box_x2<T, KIND, 8, 8, 2>(bp, planes, st);
        case 3: return launch_box_x2<T, KIND, 8, 8, 3>(bp, planes, st);
        case 4: return launch_box_x2<T, KIND, 8, 8, 4>(bp, planes, st);
        default: break;
        }
        if (bp.r <= 8) return launch_box_x2<T, KIND, 8, 8>(bp, planes, st);
        if (bp.r <= 16) return launch_box_x2<T, KIND, 16, 16>(bp, planes, st);
        return launch_box_v<T, KIND, true, 16, 16>(bp, planes, st);
    }
    if (bp.r <= 8) return launch_box_v<T, KIND, false, 8, 8>(bp, planes, st);
    if (bp.r <= 16) return launch_box_v<T, KIND, false, 16, 16>(bp, planes, st);
    return launch_box_v<T, KIND, true, 16, 16>(bp, planes, st);
}

template <typename TI, typename TQ>
void launch_up_t(UpParams up, int N, int CC, bool vec, cudaStream_t st)
{
    const bool s1 = (up.s == 1);
    const int bands = (up.W + UP_BAND - 1) / UP_BAND;
    if (s1) {
        dim3 grid(bands, (up.H + up.R - 1) / up.R, N * up.CG);
#define GF_S1(cc, v) launch_pdl(k_output_s1<TI, TQ, cc, v>, grid, dim3(UP_NT), 0, st, up)
        if (CC == 3) { if (vec) GF_S1(3, true); else GF_S1(3, false); }
        else { if (vec) GF_S1(1, true); else GF_S1(1, false); }
#undef GF_S1
        return;
    }
    if (vec && up.sd == 1 && (up.s == 4 || up.s == 8)) {
        // the guide streamed by TMA when the tensor map can describe it; else the per-thread cp.async ring
        constexpr int DT_IN = sizeof(TI) == 4 ? F32 : (sizeof(TI) == 2 ? F16 : U8);
        constexpr int DT_OUT = sizeof(TQ) == 4 ? F32 : F16;
        if (output_tma_ok(up.I, DT_IN, up.W, up.fps) &&
            launch_output_tma(up.I, up.ma, up.mb, up.q, N, up.C, up.CI, up.H, up.W, up.h, up.w, up.s, up.lps, up.fps,
                              up.Yw0, up.Yw1, up.detail, DT_IN, DT_OUT, up.fault, st) == cudaSuccess)
            return;
        up.R = 8 * up.s;  // 8 low-res rows per CTA
        up.LRmax = up.R / up.s + 2;
        up.LCmax = UP_BAND / up.s + 2;
        up.LCmax = (up.LCmax + 1) & ~1;  // 2 * LRmax * LCmax floats is then a multiple of 16 bytes
        dim3 grid(bands * up.C, (up.H + up.R - 1) / up.R, N);
        const size_t smem = (size_t)2 * up.LRmax * up.LCmax * sizeof(float) + (size_t)UP_NST * 4 * UP_NT * 4 * sizeof(TI);
        if (up.s == 4) launch_pdl(k_upsample_output_s4x<TI, TQ, 4>, grid, dim3(UP_NT), smem, st, up);
        else launch_pdl(k_upsample_output_s4x<TI, TQ, 8>, grid, dim3(UP_NT), smem, st, up);
        return;
    }
    up.LRmax = (up.R * up.sd + up.sn - 1) / up.sn + 2;  // ceil(R / s) + 2 tap rows under R full-res rows
    up.LCmax = (UP_BAND * up.sd + up.sn - 1) / up.sn + 2;
    dim3 grid(bands, (up.H + up.R - 1) / up.R, N * up.CG);
    const size_t smem = (size_t)CC * 2 * up.LRmax * up.LCmax * sizeof(float);
#define GF_UP(cc, v)                                                                 \
    do {                                                                             \
        if (opt_in_smem(k_upsample_output<TI, TQ, cc, v>, smem) == cudaSuccess)      \
            launch_pdl(k_upsample_output<TI, TQ, cc, v>, grid, dim3(UP_NT), smem, st, up);         \
    } while (0)
    if (CC == 3) { if (vec) GF_UP(3, true); else GF_UP(3, false); }
    else { if (vec) GF_UP(1, true); else GF_UP(1, false); }
#undef GF_UP
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// FP32 input at s = 2, 4, 8 (bilinear or nearest, full-res p) whose rows are 16-byte aligned and whose size
// is a multiple of s: every subsample reads one or two whole vectors per source row and nothing is clamped.
// The box and antialiased modes' fast path: FP32, s = 2, 4, 8, H and W multiples of s, aligned planes.
// (The whole-plane stride is H * W of the whole image, a multiple of 4 floats, so every plane is aligned.)
bool aligned_fp32_wide_subsample(const FwdPlan &P)
{
    return (P.dt_in == F32) && (P.mode == GF_SUB_BOX || P.mode == GF_SUB_BILINEAR_AA) && P.sd == 1 &&
           (P.s == 2 || P.s == 4 || P.s == 8) && (P.H % P.s == 0) && (P.W % P.s == 0) && (P.W % 4 == 0) &&
           aligned16(P.I) && (P.p_lowres || aligned16(P.p));  // a low-res p is only copied
}

bool aligned_vec_subsample(const FwdPlan &P)
{
    // every row of every plane starts on a 16-byte boundary: 16-byte aligned planes, W a multiple of 16 bytes
    const size_t rowb = (size_t)P.W * dtype_size(P.dt_in);
    return !P.p_lowres && (P.mode == GF_SUB_NEAREST || P.mode == GF_SUB_BILINEAR) && P.sd == 1 &&
           (P.s == 2 || P.s == 4 || P.s == 8) && (P.H % P.s == 0) && (P.W % P.s == 0) && (rowb % 16 == 0) &&
           ((P.fps * dtype_size(P.dt_in)) % 16 == 0) && aligned16(P.I) && aligned16(P.p);
}

}  // namespace

// The TMA-fed box kernels (gf_box.cu) take every box step whose planes they accept (FP32 planes with rows of a
// multiple of 4 floats, r' <= 16, no window statistics kept for the backward).  Measured on one GB300 against
// the per-thread-load kernels: 12 MP at s = 1 (r = 16) 0.45 against 0.90 ms per call; at s = 4 (r' = 4) the
// statistics 13.9 against 17.1 us and the box means 12.1 against 12.9 us (two images in flight: 178 k against
// 177 k MP/s); the feathering figure's r' = 15 at s = 4 38 against 47 us.
static bool box_tma_pays(int, int) { return true; }
// The column-strip kernels (gf_strip.cu) take the box steps at large radii, where the tiles' 2r halo rows and
// columns cost more than their outputs; on large planes, whose long segments amortise the window opening; and
// for three channels of one gray guide at r' = 4 (a compile-time radius of the strip kernels), where one strip
// CTA forms the guide's sums once for the three.  Measured on the 12 MP scene: s = 1 calls at r = 4 / 8 / 12
// take 246 / 287 / 305 us with strips against 291 / 335 / 482 us with tiles; at s = 4 (r' = 4, gray guide, 3
// channels) two images in flight take 64.4-64.6 against 67.1 us per image; at s = 8 (r' = 2) 251 k against
// 261 k MP/s, with a depthwise guide or r' = 1 the strips lost 1-4 %, and at the run-time radii r' = 5, 6 (s =
// 10/3, 5/2, one image at a time) 1.5-3 %, so the tiles keep those.  GF_STRIP_MIN_R (read per call) replaces
// the rule by r >= its value, so that tests and measurements can send any radius through either form.
static bool strip_pays(int r, int h, int w, bool gray3)
{
    if (const char *e = getenv("GF_STRIP_MIN_R")) return r >= atoi(e);
    return r >= 9 || (long long)h * w >= (2LL << 20) || (gray3 && r == 4);
}

bool s1_means_output_form(const Resolved &R)
{
    return R.s == 1 && R.sd == 1 && !R.color && !R.fused && !R.dense_lowres && !R.p_lowres && !R.saved_forward &&
           R.dt_in == F32 &&
           (R.dt_out == F32 || R.dt_out == F16) && R.W % 4 == 0 && R.r_low <= 16;
}

// Whether a call with this geometry takes the subsample and the box statistics as one kernel (k_box_strip_sub),
// given 16-byte aligned planes and no window statistics asked for (gf_opts.stats_out).
static bool sub_strip_form(const Resolved &R)
{
    return !R.color && !R.fused && !R.saved_forward && !R.int_stats &&
           strip_sub_geometry(R.C, R.CI, R.H, R.W, R.h, R.w, R.s, R.sd, R.mode, R.r_low, R.dt_in, R.p_lowres);
}

int forward_kernel_count(const Resolved &R)
{
    if (R.fused) return 1;
    if (R.color) return 6;
    if (R.s > 1) return sub_strip_form(R) ? 3 : 4;
    return s1_means_output_form(R) ? 2 : 3;
}

namespace {

// The colour-guide form after the subsample: products, their box means, the 3 x 3 solves, the box means of
// the coefficients, and the output (kernels in gf_color.cu).
cudaError_t launch_color_chain(const FwdPlan &P0, float *pl, StageTimer &tm, cudaStream_t st)
{
    FwdPlan P = P0;
    P.pl = pl;  // I' itself when the call is self-guided
    cudaError_t err;
    const int K = 5 + 2 * P.C;
    auto box_pairs = [&](float *X, float *Y, float *oX, float *oY, int per_image) {
        BoxTmaJob J{};
        J.kind = BOX_JOB_MEANS;
        J.X = X; J.Y = Y;
        J.xps = J.yps = J.ops = P.lps;
        J.N = P.N; J.C = J.CX = per_image;
        J.h = P.h; J.w = P.w; J.r = P.r_low;
        J.out0 = oX; J.out1 = oY;
        J.fault = P.fault;
        if (strip_pays(P.r_low, P.h, P.w, P.CI == 1 && P.C % 3 == 0) && strip_box_supported(J)) return launch_strip_box(J, st);
        if (box_tma_pays(P.s, P.r_low) && box_tma_supported(J)) return launch_box_tma(J, st);
        BoxParams bp{};
        bp.X = X; bp.Y = Y;
        bp.xps = bp.yps = bp.ops = P.lps;
        bp.CX = bp.C = per_image;
        bp.out0 = oX; bp.out1 = oY;
        bp.h = P.h; bp.w = P.w; bp.r = P.r_low;
        return launch_box_t<float, KIND_MEAN2>(bp, P.N * per_image, st);
    };
    tm.before();
    err = launch_color_products(P, st);
    tm.after();
    if (err != cudaSuccess) return err;
    tm.before();
    err = box_pairs(P.col[0], P.col[1], P.col[2], P.col[3], K);
    tm.after();
    if (err != cudaSuccess) return err;
    tm.before();
    err = launch_color_coef(P, st);
    tm.after();
    if (err != cudaSuccess) return err;
    tm.before();
    err = box_pairs(P.col[4], P.col[5], P.col[6], P.col[7], 2 * P.C);
    tm.after();
    if (err != cudaSuccess || P.skip_output) return err;
    tm.before();
    err = launch_color_output(P, st);
    tm.after();
    return err;
}

}  // namespace

cudaError_t launch_forward(const FwdPlan &P, cudaStream_t st)
{
    StageTimer tm{P.events, st};
    cudaError_t err;
    // The call's fault word starts at zero (kernels whose bounded waits give up OR their bit into it): the
    // first kernel of the chain zeroes it (the single fused kernel, or the subsample), else a memset does.
    const bool fused_call = P.fused && !P.skip_output && !P.need_lowres;
    unsigned *clear_word = P.clear_fault ? P.fault.call : nullptr;
    if (clear_word && !fused_call && !(P.s > 1 || P.color) &&
        (err = cudaMemsetAsync(clear_word, 0, sizeof(unsigned), st)) != cudaSuccess)
        return err;
    if (fused_call) {  // the whole filter in one kernel
        tm.before();
        err = launch_fused(P, st);
        tm.after();
        return err;
    }
    const int planesNC = P.N * P.C;

    // ---- Algorithm 2, first step: subsample I and p (skipped at s = 1)
    const void *Xsrc = P.I, *Ysrc = P.p;
    int src_dt = P.dt_in;
    // A self-guided call (p is I, one guide channel per channel) subsamples once and uses I' as p'; the
    // backward keeps its own p' plane, so its forward recomputation subsamples both.
    const bool self_guided = (P.I == P.p) && (P.CI == P.C) && !P.p_lowres && !P.need_lowres;
    // The subsample and the box statistics as one kernel (k_box_strip_sub) where it takes the call: then I', p'
    // are never written, so not when they are kept for the backward or the window statistics are asked for.
    SubStripJob SJ{};
    bool sub_strip = false;
    if (!P.color && !P.need_lowres && !P.stats && !P.int_stats &&
        strip_sub_geometry(P.C, P.CI, P.H, P.W, P.h, P.w, P.s, P.sd, P.mode, P.r_low, P.dt_in, P.p_lowres)) {
        SJ.I = (const float *)P.I; SJ.p = (const float *)P.p; SJ.fps = P.fps;
        SJ.N = P.N; SJ.C = P.C; SJ.H = P.H; SJ.W = P.W; SJ.h = P.h; SJ.w = P.w; SJ.s = P.s; SJ.mode = P.mode;
        SJ.r = P.r_low; SJ.eps = P.eps;
        SJ.a = P.a; SJ.b = P.b; SJ.ops = P.lps;
        SJ.clear_word = clear_word;
        SJ.fault = P.fault;
        sub_strip = strip_sub_supported(SJ);
    }
    if ((P.s > 1 || P.color) && !sub_strip) {  // the colour stages read low-res planes only, so s = 1 copies
        SubParams sp;
        sp.h = P.h; sp.w = P.w; sp.mode = P.mode;
        // uint8 path: carry the subsampled values as exact integers J = k * (value in 1/255 units)
        sp.scale = P.int_stats ? P.int_scale / 255.0f : 1.0f;
        sp.clear_word = clear_word;
        sp.job[0] = SubJob{P.I, P.Il, P.N * P.CI, P.H, P.W, P.s, P.fps, P.lps, P.sn, P.sd};
        if (!P.p_lowres)
            sp.job[1] = SubJob{P.p, P.pl, planesNC, P.H, P.W, P.s, P.fps, P.lps, P.sn, P.sd};
        else  // a low-res p is only copied into the FP32 workspace
            sp.job[1] = SubJob{P.p, P.pl, planesNC, P.h, P.w, 1, P.lpin, P.lps, 1, 1};
        const int nz = P.N * P.CI + (self_guided ? 0 : planesNC);
        const bool vec_ok = aligned_vec_subsample(P);
        tm.before();
        if (vec_ok) {
            const int jb = (P.s == 8) ? 1 : 2;
            dim3 grid((P.w + SUB_NT_VEC - 1) / SUB_NT_VEC, (P.h + jb - 1) / jb, nz);
#define GF_SV(m, ss)                                                                       \
    do {                                                                                   \
        if (P.dt_in == F32) launch_pdl(k_subsample_vec<float, m, ss>, grid, dim3(SUB_NT_VEC), 0, st, sp);    \
        else if (P.dt_in == F16) launch_pdl(k_subsample_vec<__half, m, ss>, grid, dim3(SUB_NT_VEC), 0, st, sp); \
        else launch_pdl(k_subsample_vec<uint8_t, m, ss>, grid, dim3(SUB_NT_VEC), 0, st, sp);                \
    } while (0)
            if (P.mode == GF_SUB_BILINEAR) {
                if (P.s == 2) GF_SV(GF_SUB_BILINEAR, 2); else if (P.s == 4) GF_SV(GF_SUB_BILINEAR, 4); else GF_SV(GF_SUB_BILINEAR, 8);
            } else {
                if (P.s == 2) GF_SV(GF_SUB_NEAREST, 2); else if (P.s == 4) GF_SV(GF_SUB_NEAREST, 4); else GF_SV(GF_SUB_NEAREST, 8);
            }
#undef GF_SV
        } else if (aligned_fp32_wide_subsample(P)) {
            dim3 grid((P.w + SUB_NT - 1) / SUB_NT, (P.h + SUB_JB - 1) / SUB_JB, nz);
#define GF_SW(m, ss) launch_pdl(k_subsample_wide<m, ss>, grid, dim3(SUB_NT), 0, st, sp)
            if (P.mode == GF_SUB_BOX) {
                if (P.s == 2) GF_SW(GF_SUB_BOX, 2); else if (P.s == 4) GF_SW(GF_SUB_BOX, 4); else GF_SW(GF_SUB_BOX, 8);
            } else {
                if (P.s == 2) GF_SW(GF_SUB_BILINEAR_AA, 2);
                else if (P.s == 4) GF_SW(GF_SUB_BILINEAR_AA, 4);
                else GF_SW(GF_SUB_BILINEAR_AA, 8);
            }
#undef GF_SW
        } else {
            dim3 grid((P.w + SUB_NT - 1) / SUB_NT, (P.h + SUB_JB - 1) / SUB_JB, nz);
            if (P.dt_in == F32) launch_sub_t<float>(sp, grid, st);
            else if (P.dt_in == F16) launch_sub_t<__half>(sp, grid, st);
            else launch_sub_t<uint8_t>(sp, grid, st);
        }
        tm.after();
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        Xsrc = P.Il;
        Ysrc = self_guided ? P.Il : P.pl;
        src_dt = F32;
    }

    if (P.color) return launch_color_chain(P, self_guided ? P.Il : P.pl, tm, st);

    // ---- Algorithm 2, box statistics + var/cov + coefficients a, b (Eq. 2-3)
    if (sub_strip) {
        tm.before();
        err = launch_strip_sub(SJ, st);
        tm.after();
        if (err != cudaSuccess) return err;
    } else {
        BoxParams bp{};
        bp.X = Xsrc; bp.Y = Ysrc;
        const bool lowres_src = (P.s > 1);
        bp.xps = lowres_src ? P.lps : P.fps;  // s = 1: I and p themselves (h = H, w = W)
        bp.yps = lowres_src ? P.lps : (P.p_lowres ? P.lpin : P.fps);
        bp.CX = P.CI; bp.C = P.C;
        bp.out0 = P.a; bp.out1 = P.b; bp.ops = P.lps;
        bp.stats = P.stats;
        bp.h = P.h; bp.w = P.w; bp.r = P.r_low; bp.eps = P.eps;
        bp.int_scale = P.int_scale;
        BoxTmaJob J{};
        J.kind = BOX_JOB_STATS;
        J.X = (const float *)Xsrc; J.Y = (const float *)Ysrc;
        J.xps = bp.xps; J.yps = bp.yps;
        J.N = P.N; J.C = P.C; J.CX = P.CI;
        J.h = P.h; J.w = P.w; J.r = P.r_low; J.eps = P.eps;
        J.out0 = P.a; J.out1 = P.b; J.ops = P.lps;
        J.stats = P.int_stats ? nullptr : (float *)P.stats;
        J.fault = P.fault;
        const bool fp32 = !P.int_stats && src_dt == F32;
        const bool strip = fp32 && strip_pays(P.r_low, P.h, P.w, P.CI == 1 && P.C % 3 == 0) && strip_box_supported(J);
        const bool tma = !strip && fp32 && box_tma_pays(P.s, P.r_low) && box_tma_supported(J);
        tm.before();
        if (strip) {
            err = launch_strip_box(J, st);
        } else if (tma) {
            err = launch_box_tma(J, st);
        } else if (P.int_stats) {
            if (src_dt == F32) err = launch_box_t<float, KIND_STATS_INT>(bp, planesNC, st);
            else err = launch_box_t<uint8_t, KIND_STATS_INT>(bp, planesNC, st);
        } else {
            if (src_dt == F32) err = launch_box_t<float, KIND_STATS_F>(bp, planesNC, st);
            else err = launch_box_t<__half, KIND_STATS_F>(bp, planesNC, st);
        }
        tm.after();
        if (err != cudaSuccess) return err;
    }

    // ---- s = 1: the upsample is the identity, so the box means of a and b and the output are one kernel
    if (P.s == 1 && !P.skip_output && !P.need_lowres && !P.lowres_out && !P.color && P.dt_in == F32 &&
        (P.dt_out == F32 || P.dt_out == F16)) {
        BoxTmaJob J{};
        J.kind = BOX_JOB_MEANS_OUTPUT;
        J.X = P.a; J.Y = P.b;
        J.xps = J.yps = P.lps;
        J.N = P.N; J.C = J.CX = P.C;
        J.h = P.h; J.w = P.w; J.r = P.r_low;
        J.I = (const float *)P.I; J.q = P.q; J.fps = P.fps; J.CI = P.CI;
        J.Yw0 = P.Yw0; J.Yw1 = P.Yw1; J.dt_out = P.dt_out; J.detail = P.detail;
        J.fault = P.fault;
        const bool strip = strip_pays(P.r_low, P.h, P.w, P.CI == 1 && P.C % 3 == 0) && strip_box_supported(J);
        if (strip || box_tma_supported(J)) {
            tm.before();
            err = strip ? launch_strip_box(J, st) : launch_box_tma(J, st);
            tm.after();
            return err;
        }
    }

    // ---- Algorithm 2, box means of a and b
    {
        BoxTmaJob J{};
        J.kind = BOX_JOB_MEANS;
        J.X = P.a; J.Y = P.b;
        J.xps = J.yps = J.ops = P.lps;
        J.N = P.N; J.C = J.CX = P.C;
        J.h = P.h; J.w = P.w; J.r = P.r_low;
        J.out0 = P.ma; J.out1 = P.mb;
        J.fault = P.fault;
        tm.before();
        if (strip_pays(P.r_low, P.h, P.w, P.CI == 1 && P.C % 3 == 0) && strip_box_supported(J)) {
            err = launch_strip_box(J, st);
        } else if (box_tma_pays(P.s, P.r_low) && box_tma_supported(J)) {
            err = launch_box_tma(J, st);
        } else {
            BoxParams bp{};
            bp.X = P.a; bp.Y = P.b;
            bp.xps = P.lps; bp.yps = P.lps;
            bp.CX = P.C; bp.C = P.C;
            bp.out0 = P.ma; bp.out1 = P.mb; bp.ops = P.lps;
            bp.h = P.h; bp.w = P.w; bp.r = P.r_low;
            err = launch_box_t<float, KIND_MEAN2>(bp, planesNC, st);
        }
        tm.after();
        if (err != cudaSuccess) return err;
    }

    if (P.skip_output) return cudaSuccess;

    // ---- Algorithm 2, bilinear upsample of mean_a, mean_b fused with q = mean_a .* I + mean_b
    {
        UpParams up{};
        up.fault = P.fault;
        up.I = P.I; up.ma = P.ma; up.mb = P.mb; up.q = P.q;
        up.detail = P.detail;
        up.sn = P.sn;
        up.sd = P.sd;
        up.fps = P.fps;
        up.Yw0 = P.Yw0;
        up.Yw1 = P.Yw1;
        up.C = P.C; up.CI = P.CI; up.H = P.H; up.W = P.W; up.h = P.h; up.w = P.w; up.s = P.s;
        up.lps = P.lps;
        const int CC = (P.C % 3 == 0) ? 3 : 1;
        up.CG = P.C / CC;
        const bool s1 = (P.s == 1);
        up.R = s1 ? 8 : std::max(8, 4 * P.s);
        // 4-wide vector accesses need every row of every plane to start on the vector boundary
        const bool vec = (P.W % 4 == 0) && aligned16(P.I) && aligned16(P.q) &&
                         (!s1 || ((P.lps % 4 == 0) && aligned16(P.ma) && aligned16(P.mb)));
        tm.before();
        if (P.dt_in == F32) {
            if (P.dt_out == F32) launch_up_t<float, float>(up, P.N, CC, vec, st);
            else launch_up_t<float, __half>(up, P.N, CC, vec, st);
        } else if (P.dt_in == F16) {
            if (P.dt_out == F32) launch_up_t<__half, float>(up, P.N, CC, vec, st);
            else launch_up_t<__half, __half>(up, P.N, CC, vec, st);
        } else {
            if (P.dt_out == F32) launch_up_t<uint8_t, float>(up, P.N, CC, vec, st);
            else launch_up_t<uint8_t, __half>(up, P.N, CC, vec, st);
        }
        tm.after();
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace gfk
