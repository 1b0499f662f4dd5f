// gf_strip.cu -- column-strip kernels for the box steps at large radii (He and Sun, "Fast Guided Filter", 2015):
//
//   SK_STATS     Algorithm 2 (Algorithm 1 at s = 1), box statistics mean_I, mean_p, corr_I, corr_Ip at radius r,
//                fused with var_I, cov_Ip and the coefficients a (Eq. 2) and b (Eq. 3);
//   SK_MEAN2     box means of a and b;
//   SK_MEAN2_OUT box means of a and b fused with q = mean_a I + mean_b (Eq. 4), at s = 1 only, where the
//                upsample is the identity;
// and k_box_strip_sub (further down), Algorithm 2's subsample and statistics in one kernel, its rows fed by TMA.
//
// f_mean is the box mean over the window clipped to the image, divided by the window's in-image count.
//
// One CTA owns a strip of 128 output columns over a segment of rows, of one plane or, when one guide plane
// serves three channels, of all three (the guide's sums are then formed once per pixel).  Phase 1: one thread
// per strip column (the 128 columns and the r halo on each side: 160 threads at r = 16) carries the vertical
// window sums down the segment, adding the row that enters the window and subtracting the row that leaves it,
// both read straight from global memory (the leaving row was read 2r + 1 rows earlier, so it comes from L2)
// and requested a block ahead, and writes the sums of a block of 10 rows to shared memory.  Phase 2: every
// thread takes a run of 8 outputs of one row of the block; the 16 runs of a row share the sums of whole
// 8-column blocks, each run slides its window along the column sums, applies the epilogue and stores with
// 128-bit stores.  A window is opened once per segment, not per tile, and both phases keep all threads busy,
// which the tile form (gf_box.cu) cannot at large radii: its 2r halo rows and columns cost more there than the
// outputs themselves.
//
// Statistics are taken of values shifted by one sample of the segment (its first output pixel), so
// E[I^2] - E[I]^2 is formed from terms near the local level; pairs of quantities travel as packed FP32x2.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "gf_device.cuh"
#include "gf_internal.cuh"

namespace gfk {

namespace {

constexpr int SP_TW = 128;                      // output columns per strip
constexpr int SP_NT = 160;                      // threads: walkers (128 + 2r <= 160), then the runs
constexpr int SP_RUN = 8;                       // outputs per phase-2 run
constexpr int SP_CB = SP_NT / (SP_TW / SP_RUN); // rows per block: 10
constexpr int SP_RMAX = (SP_NT - SP_TW) / 2;    // 16
// Longest segment: the running sums carry the rounding of every row added and subtracted, so a window is
// reopened (with a new shift) at least every 160 rows.
constexpr int SP_SEG_MAX = 16 * SP_CB;

enum { SK_STATS = 0, SK_MEAN2 = 2, SK_MEAN2_OUT = 3 };

struct StripParams {
    const float *X, *Y;  // SK_STATS: guide planes (CX per image) and input planes (C per image); else a and b
    size_t xps, yps;     // plane strides (elements); rows are w elements apart
    int C, CX;           // channels per image; guide planes per image (1 or C)
    int groups;          // CTAs across the channels of one image (C / NY)
    int h, w, r;         // plane size; radius (used when the kernel's RC < 0)
    int ylo, yhi, seg;   // output rows [ylo, yhi), seg rows per CTA (a multiple of SP_CB)
    int seg_order;       // the grid's rows take the segments in the order (k mod seg_order, k / seg_order)
    float eps;
    float *out0, *out1;  // SK_STATS: a, b; SK_MEAN2: mean_a, mean_b (plane stride ops)
    size_t ops;
    int stream_out;      // the outputs are stored with the streaming (evict-first) policy
    // SK_MEAN2_OUT: q = mean_a I + mean_b into q (dtype TQ, plane stride fps), the guide I with CI planes per
    // image (plane stride fps); the detail epilogue q + k (I - q) when detail != 0
    const float *I;
    void *q;
    size_t fps;
    int CI;
    float detail;
};

// Pairs of window sums carried per column: statistics of NY channels sharing one guide carry (dX, dY_c) and
// (dX^2, dX dY_c) -- 2 pairs for one channel, 4 for three; box means carry (a, b).
__host__ __device__ constexpr int nq_of(int KIND, int NY) { return KIND == SK_STATS ? (NY == 1 ? 2 : 4) : 1; }
// Column sums of the block are double-buffered (one barrier per block) where they are small enough to leave
// room for four CTAs per SM.
__host__ __device__ constexpr bool db_of(int NQ) { return NQ <= 2; }

// Shared-memory index of column c.  float4 elements (NQ >= 2): the low three bits XOR-swizzled by c / 8, so the
// 8 runs read by a quarter-warp fall on distinct banks.  float2 elements (NQ == 1): two pads per 8 columns, so
// each even / odd pair of columns is one aligned 16-byte word and the runs of a quarter-warp (10 float2 apart)
// again fall on distinct banks.
__host__ __device__ constexpr int vp_of(int NQ) { return NQ == 1 ? SP_NT + 2 * (SP_NT / 8) : SP_NT; }
__device__ __forceinline__ int vidx4(int c) { return c ^ ((c >> 3) & 7); }
__device__ __forceinline__ int vidx2(int c) { return c + 2 * (c >> 3); }

// Bytes of shared memory of one CTA.
// The block sums shared by the runs of a row: [SP_CB rows][SP_NT / 8 blocks] of NQ float2 (as NQ / 2 float4
// arrays when NQ >= 2).
constexpr int SP_NBLK = SP_NT / 8;
__host__ __device__ constexpr size_t bsum_bytes(int NQ) { return (size_t)SP_CB * SP_NBLK * 8 * NQ; }
// The column-sum pitch at a compile-time radius r <= 8: just the 128 + 2r walker columns, in whole 8-column
// blocks for the float4 swizzle; for float2, past the padded index of the last column and 8 mod 16.  Rows then
// keep the bank offset of the full pitch (0 banks for float4, 16 for float2), and the smaller CTAs fit beside
// other kernels' CTAs on an SM.  Larger and run-time radii keep the pitch of r = 16.
__host__ __device__ constexpr int vp2_need(int RC) { return (SP_TW + 2 * RC - 1) + 2 * ((SP_TW + 2 * RC - 1) >> 3) + 1; }
__host__ __device__ constexpr int vp_rc(int NQ, int RC)
{
    return (RC < 0 || RC > 8) ? vp_of(NQ)
                              : (NQ == 1 ? vp2_need(RC) + (24 - vp2_need(RC) % 16) % 16
                                         : ((SP_TW + 2 * RC + 7) & ~7));
}
__host__ __device__ constexpr size_t buf_bytes_rc(int NQ, int RC)
{
    return (size_t)SP_CB * vp_rc(NQ, RC) * (NQ == 1 ? 8 : 16) * (NQ == 1 ? 1 : NQ / 2);
}
__host__ __device__ constexpr size_t strip_smem_rc(int NQ, int RC)
{
    return (size_t)(db_of(NQ) ? 2 : 1) * buf_bytes_rc(NQ, RC) + bsum_bytes(NQ);
}

// One strip column's sources: the planes it reads (statistics: the guide, then NY inputs; box means: a, b),
// offset to the column, and for the statistics the shift subtracted from each.
template <int KIND, int NY>
struct Column {
    static constexpr int NS = (KIND == SK_STATS) ? 1 + NY : 2;
    static constexpr int NQ = nq_of(KIND, NY);
    const float *p[NS];
    float c[NS];
    int w;
    __device__ __forceinline__ void load(int t, float v[NS]) const
    {
#pragma unroll
        for (int k = 0; k < NS; ++k) v[k] = __ldg(p[k] + t * w);
    }
    // the pairs one row contributes to the window sums
    __device__ __forceinline__ void pairs(const float v[NS], float2 q[NQ]) const
    {
        if constexpr (KIND != SK_STATS) {
            q[0] = make_float2(v[0], v[1]);
        } else if constexpr (NY == 1) {
            const float2 d = sub2(make_float2(v[0], v[1]), make_float2(c[0], c[1]));
            q[0] = d;
            q[1] = mul2(make_float2(d.x, d.x), d);  // (dX^2, dX dY)
        } else {
            const float2 d0 = sub2(make_float2(v[0], v[1]), make_float2(c[0], c[1]));
            const float2 d1 = sub2(make_float2(v[2], v[3]), make_float2(c[2], c[3]));
            const float2 xx = make_float2(d0.x, d0.x);
            q[0] = d0;            // (dX, dY_0)
            q[1] = d1;            // (dY_1, dY_2)
            q[2] = mul2(xx, d0);  // (dX^2, dX dY_0)
            q[3] = mul2(xx, d1);  // (dX dY_1, dX dY_2)
        }
    }
    __device__ __forceinline__ void add_row(int t, float2 S[NQ]) const
    {
        float v[NS];
        float2 q[NQ];
        load(t, v);
        pairs(v, q);
#pragma unroll
        for (int k = 0; k < NQ; ++k) S[k] = add2(S[k], q[k]);
    }
};

// Column sums of one row of a block into shared memory (walker column j).
template <int NQ, int VP = vp_of(NQ)>
__device__ __forceinline__ void put_sums(unsigned char *buf, int k, int j, const float2 S[NQ])
{
    if constexpr (NQ == 1) {
        reinterpret_cast<float2 *>(buf)[k * VP + vidx2(j)] = S[0];
    } else {
        float4 *VA = reinterpret_cast<float4 *>(buf);
        VA[k * VP + vidx4(j)] = make_float4(S[0].x, S[0].y, S[1].x, S[1].y);
        if constexpr (NQ == 4) VA[(SP_CB + k) * VP + vidx4(j)] = make_float4(S[2].x, S[2].y, S[3].x, S[3].y);
    }
}
// The rows one walker column reads for a block of output rows yb .. yb + SP_CB - 1: row yb + k + r enters the
// window of output row yb + k and row yb + k - r leaves it after.  They are requested one block ahead (fetch
// right after the previous block's column sums are written), so the loads are in flight during phase 2.  A row
// outside the image reads as the shift value, whose shifted pair is exactly zero.  The three-channel statistics
// (four planes) request their leaving rows ahead only at the radii 15 and 16 (PL), where a batch of 80 values a
// thread and two CTAs per SM pay; elsewhere they read those rows when they use them, at three CTAs per SM.
template <int KIND, int NY, bool PL>
struct RowBatch {
    static constexpr int NS = Column<KIND, NY>::NS;
    static constexpr bool PRE_L = (NS <= 2) || PL;  // the leaving rows too
    float e[SP_CB][NS], l[PRE_L ? SP_CB : 1][NS];
    __device__ __forceinline__ static float ld_row(const Column<KIND, NY> &col, int t, int h, int k)
    {
        return (t >= 0 && t < h) ? __ldg(col.p[k] + t * col.w) : col.c[k];
    }
    template <bool CHECK>
    __device__ __forceinline__ void fetch_rows(const Column<KIND, NY> &col, int yb, int r, int h)
    {
#pragma unroll
        for (int k = 0; k < SP_CB; ++k) {
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                e[k][q] = CHECK ? ld_row(col, yb + k + r, h, q) : __ldg(col.p[q] + (yb + k + r) * col.w);
                if constexpr (PRE_L)
                    l[k][q] = CHECK ? ld_row(col, yb + k - r, h, q) : __ldg(col.p[q] + (yb + k - r) * col.w);
            }
        }
    }
    __device__ __forceinline__ void fetch(const Column<KIND, NY> &col, int yb, int r, int h)
    {
        if (yb - r >= 0 && yb + SP_CB - 1 + r < h) fetch_rows<false>(col, yb, r, h);
        else fetch_rows<true>(col, yb, r, h);
    }
};

// Phase 1 of one block for one walker column: the vertical window sums of rows yb .. yb + SP_CB - 1 from the
// batch fetched for them.  S holds the sums of rows [yb - r, yb + r - 1] (clipped to the image) on entry and is
// carried on to the next block.
template <int KIND, int NY, bool PL, int VP>
__device__ __forceinline__ void walk_block(const Column<KIND, NY> &col, const RowBatch<KIND, NY, PL> &B,
                                           float2 (&S)[nq_of(KIND, NY)], int yb, int r, int h, unsigned char *buf,
                                           int j)
{
    constexpr int NQ = nq_of(KIND, NY);
    constexpr int NS = Column<KIND, NY>::NS;
#pragma unroll
    for (int k = 0; k < SP_CB; ++k) {
        float2 qe[NQ], ql[NQ];
        col.pairs(B.e[k], qe);
        if constexpr (RowBatch<KIND, NY, PL>::PRE_L) {
            col.pairs(B.l[k], ql);
        } else {
            float vl[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) vl[q] = RowBatch<KIND, NY, PL>::ld_row(col, yb + k - r, h, q);
            col.pairs(vl, ql);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) S[q] = add2(S[q], qe[q]);
        put_sums<NQ, VP>(buf, k, j, S);
#pragma unroll
        for (int q = 0; q < NQ; ++q) S[q] = sub2(S[q], ql[q]);
    }
}

template <typename TQ>
__device__ __forceinline__ void store4q(TQ *p, const float v[4]);
template <>
__device__ __forceinline__ void store4q<float>(float *p, const float v[4])
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}
template <>
__device__ __forceinline__ void store4q<__half>(__half *p, const float v[4])
{
    const __half2 lo = __floats2half2_rn(v[0], v[1]), hi = __floats2half2_rn(v[2], v[3]);
    *reinterpret_cast<uint2 *>(p) =
        make_uint2(*reinterpret_cast<const unsigned *>(&lo), *reinterpret_cast<const unsigned *>(&hi));
}


// Phase-2 reads of one run: the column sums of walker columns c0 + i (c0 = 8 g) of row k of a block.
//   float2 layout (NQ == 1): column c at c + 2 (c / 8), i.e. 10 g + i + 2 (i / 8) -- a constant offset from the
//   run's base, each even / odd pair of columns one aligned 16-byte word;
//   float4 layout (NQ >= 2): column c at c ^ ((c / 8) mod 8).  A run's own 8-column block is read slot by slot,
//   lane g taking slot (e + g) mod 8 at step e (8 distinct banks across a quarter-warp), since a block sum does
//   not depend on the order; single columns take the swizzle: one XOR and one address per read.
template <int NQ, int VP = vp_of(NQ)>
struct RunReader {
    const float4 *pair2;  // NQ == 1: the run's base (column pairs c0 + i, c0 + i + 1 for even i)
    const float4 *row4;   // NQ >= 2: the block's row
    int pg;
    __device__ __forceinline__ RunReader(const unsigned char *buf, int k, int g) : pg(g)
    {
        pair2 = reinterpret_cast<const float4 *>(reinterpret_cast<const float2 *>(buf) + k * VP + 10 * g);
        row4 = reinterpret_cast<const float4 *>(buf) + k * VP;
    }
    // NQ == 1: columns c0 + i and c0 + i + 1 (i even) as (a, b, a', b')
    __device__ __forceinline__ float4 pair_at(int i) const { return pair2[(i + 2 * (i >> 3)) >> 1]; }
    // The windows of the run's outputs from the sums of whole 8-column blocks, which the 16 runs of a row (lanes
    // of one half-warp) share through this row's block sums `bs`: a run sums its own block (whose columns leave
    // its windows) and reads the other full blocks' sums, then only single columns of the block or two that its
    // windows' right ends cross.  Output j's window is walker columns c0 + j .. c0 + j + 2r: n = 2r + 1 columns,
    // for j = 0 nb full blocks and rem columns of block nb (relative to the run's own block).  Blocks 16 .. 19
    // (the strip's right halo) are no run's own block: the run nb blocks to their left sums them.  Every lane of
    // the warp calls these (they synchronise the warp), live run or not; `bs` is next written after the block
    // barrier that follows the next phase 1.
    //
    // NQ == 1: all 8 window sums W at once; the own block's columns stay in registers, the entering columns
    // n .. n + 6 are the 4 column pairs from n - 1.
    template <int RC>
    __device__ __forceinline__ void windows8_shared(int r, float2 *bs, float2 W[SP_RUN]) const
    {
        const int n = 2 * (RC >= 0 ? RC : r) + 1, nb = n >> 3, rem = n & 7;
        float2 own[8];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            const float4 q = pair_at(i);
            own[i] = make_float2(q.x, q.y);
            own[i + 1] = make_float2(q.z, q.w);
        }
        const float2 b_own = add2(add2(add2(own[0], own[1]), add2(own[2], own[3])),
                                  add2(add2(own[4], own[5]), add2(own[6], own[7])));
        bs[pg] = b_own;
        if (pg + nb >= SP_TW / 8 && pg + nb < SP_NBLK) {
            float2 f = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                const float4 q = pair_at(8 * nb + i);
                f = add2(f, add2(make_float2(q.x, q.y), make_float2(q.z, q.w)));
            }
            bs[pg + nb] = f;
        }
        __syncwarp();
        float2 w0 = nb >= 1 ? b_own : make_float2(0.0f, 0.0f);
        for (int d = 1; d < nb; ++d) w0 = add2(w0, bs[pg + d]);
        for (int c = 0; c < rem; c += 2) {
            const float4 q = pair_at(8 * nb + c);
            w0 = add2(w0, make_float2(q.x, q.y));
            if (c + 1 < rem) w0 = add2(w0, make_float2(q.z, q.w));
        }
        float4 ep[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) ep[t] = pair_at(n - 1 + 2 * t);
        W[0] = w0;
#pragma unroll
        for (int j = 1; j < SP_RUN; ++j) {
            const float4 q = ep[j >> 1];  // column n + j - 1 = (n - 1) + j
            const float2 e = (j & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
            W[j] = add2(W[j - 1], sub2(e, own[j - 1]));
        }
    }
    __device__ __forceinline__ void add_at(const float4 *p, float2 T[NQ]) const
    {
        const float4 a = p[0];
        T[0] = add2(T[0], make_float2(a.x, a.y));
        T[1] = add2(T[1], make_float2(a.z, a.w));
        if constexpr (NQ == 4) {
            const float4 b = p[SP_CB * VP];
            T[2] = add2(T[2], make_float2(b.x, b.y));
            T[3] = add2(T[3], make_float2(b.z, b.w));
        }
    }
    __device__ __forceinline__ void get_at(const float4 *p, float2 u[NQ]) const
    {
        const float4 a = p[0];
        u[0] = make_float2(a.x, a.y);
        u[1] = make_float2(a.z, a.w);
        if constexpr (NQ == 4) {
            const float4 b = p[SP_CB * VP];
            u[2] = make_float2(b.x, b.y);
            u[3] = make_float2(b.z, b.w);
        }
    }
    // column c0 + i through the swizzle
    __device__ __forceinline__ const float4 *col4(int i) const
    {
        const int blk = pg + (i >> 3);
        return row4 + 8 * blk + ((i & 7) ^ (blk & 7));
    }
    // NQ >= 2: T = the first window's sums (the slides re-read single columns: the own block's columns would take
    // 8 NQ registers).  bA / bB hold pairs 0-1 and 2-3 of this row's block sums.
    template <int RC>
    __device__ __forceinline__ void window_shared(int r, float4 *bA, float4 *bB, float2 T[NQ]) const
    {
        const int n = 2 * (RC >= 0 ? RC : r) + 1, nb = n >> 3, rem = n & 7;
        auto block_sum = [&](int blk, float2 B[NQ]) {  // slot (e + g) mod 8 at step e: distinct banks per quarter-warp
#pragma unroll
            for (int q = 0; q < NQ; ++q) B[q] = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int e = 0; e < 8; ++e) add_at(row4 + 8 * blk + ((e + pg) & 7), B);
        };
        auto put = [&](int m, const float2 B[NQ]) {
            bA[m] = make_float4(B[0].x, B[0].y, B[1].x, B[1].y);
            if constexpr (NQ == 4) bB[m] = make_float4(B[2].x, B[2].y, B[3].x, B[3].y);
        };
        float2 Bo[NQ];
        block_sum(pg, Bo);
        put(pg, Bo);
        if (pg + nb >= SP_TW / 8 && pg + nb < SP_NBLK) {
            float2 Bf[NQ];
            block_sum(pg + nb, Bf);
            put(pg + nb, Bf);
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NQ; ++q) T[q] = nb >= 1 ? Bo[q] : make_float2(0.0f, 0.0f);
        for (int d = 1; d < nb; ++d) {
            const float4 a = bA[pg + d];
            T[0] = add2(T[0], make_float2(a.x, a.y));
            T[1] = add2(T[1], make_float2(a.z, a.w));
            if constexpr (NQ == 4) {
                const float4 b = bB[pg + d];
                T[2] = add2(T[2], make_float2(b.x, b.y));
                T[3] = add2(T[3], make_float2(b.z, b.w));
            }
        }
        for (int c = 0; c < rem; ++c) add_at(col4(8 * nb + c), T);
    }
    // the window of output j from that of output j - 1: column c0 + j + 2r enters, c0 + j - 1 leaves
    template <int RC>
    __device__ __forceinline__ void slide(int j, int r, float2 T[NQ]) const
    {
        const int rr = RC >= 0 ? RC : r;
        if constexpr (NQ >= 2) {
            float2 ua[NQ], ub[NQ];
            get_at(col4(j + 2 * rr), ua);
            get_at(col4(j - 1), ub);
#pragma unroll
            for (int q = 0; q < NQ; ++q) T[q] = add2(T[q], sub2(ua[q], ub[q]));
        }
    }
};

// Whether the three-channel statistics request their leaving rows a block ahead: at the compile-time radii 15 and
// 16 (12 MP, s = 1, r = 16: 158 us against 164 us).  At r' = 4 one call alone also gains, but with other images'
// kernels in flight on other streams the 168-register CTAs leave them less room (190.4 k -> 186.1 k MP/s), and the
// run-time radius form loses (r = 12: 179 us against 175 us).
__host__ __device__ constexpr bool pl_of(int NQ, int RC) { return NQ == 4 && (RC == 15 || RC == 16); }
// Phase 2 of one block for one thread: the horizontal windows of its run (row pk of the block: outputs ox .. ox + 7 of
// output row y) from the column sums in buf, the epilogue and the 128-bit stores.  bs holds the block sums the
// runs of a row share.  Every one of the CTA's 160 threads calls it, live run or not (the block sums synchronise
// each half-warp).  shift: the values subtracted from every plane (statistics); iv: the guide under the run
// (box means + output).
template <int KIND, int NY, int RC, typename TQ, int VP = vp_of(nq_of(KIND, NY))>
__device__ __forceinline__ void run_block(const StripParams &P, const unsigned char *buf, unsigned char *bs,
                                          const float (&shift)[Column<KIND, NY>::NS], const float (&iv)[8], int y,
                                          bool live, int pk, int pg, int ox, int r, int h, int w, int n, int grp,
                                          bool second, bool x_interior, float inv_full)
{
    constexpr int NQ = nq_of(KIND, NY);
    const RunReader<NQ, VP> rd(buf, pk, pg);
    float2 W8[NQ == 1 ? SP_RUN : 1];
    float2 T[NQ];
    {
        if constexpr (NQ == 1) {
            rd.template windows8_shared<RC>(r, reinterpret_cast<float2 *>(bs) + pk * SP_NBLK, W8);
        } else {
            float4 *bA = reinterpret_cast<float4 *>(bs) + pk * SP_NBLK;
            rd.template window_shared<RC>(r, bA, bA + SP_CB * SP_NBLK, T);
        }
    }
    if (live) {
        const bool interior = x_interior && (y - r >= 0) && (y + r < h);
        const int ny = min(h - 1, y + r) - max(0, y - r) + 1;
        // output rows of this run
        constexpr int NO = (KIND == SK_STATS) ? 2 * NY : (KIND == SK_MEAN2 ? 2 : 1);
        float *dst0[NO / 2 > 0 ? NO / 2 : 1], *dst1[NO / 2 > 0 ? NO / 2 : 1];
        TQ *dq = nullptr;
        if constexpr (KIND == SK_MEAN2_OUT) {
            dq = (TQ *)P.q + (size_t)(n * P.C + grp) * P.fps + (size_t)y * w + ox;
        } else {
#pragma unroll
            for (int k = 0; k < NO / 2; ++k) {
                const size_t off = (size_t)(n * P.C + grp * (NO / 2) + k) * P.ops + (size_t)y * w + ox;
                dst0[k] = P.out0 + off;
                dst1[k] = P.out1 + off;
            }
        }
        auto run = [&](auto border_tag) {
            constexpr bool BORDER = decltype(border_tag)::value;
            float o[NO][4];
#pragma unroll
            for (int j = 0; j < SP_RUN; ++j) {
                if constexpr (NQ == 1) T[0] = W8[j];
                else if (j > 0) rd.template slide<RC>(j, r, T);
                float inv = inv_full;
                if constexpr (BORDER) {
                    const int xx = ox + j;
                    const int nx = min(w - 1, xx + r) - max(0, xx - r) + 1;
                    inv = __fdividef(1.0f, (float)(nx * ny));
                }
                const float2 iv2 = make_float2(inv, inv);
                const int jj = j & 3;
                if constexpr (KIND == SK_STATS) {
                    const float2 m0 = mul2(T[0], iv2);
                    if constexpr (NY == 1) {
                        const float2 m1 = mul2(T[1], iv2);
                        // var_I, cov_Ip; exactly 0 for a one-sample window (r = 0), as in the tile kernels
                        const float var = r ? fmaxf(fmaf(-m0.x, m0.x, m1.x), 0.0f) : 0.0f;
                        const float cov = r ? fmaf(-m0.x, m0.y, m1.y) : 0.0f;
                        const float a = __fdividef(cov, var + P.eps);            // a, Eq. (2)
                        o[0][jj] = a;
                        o[1][jj] = (m0.y + shift[1]) - a * (m0.x + shift[0]);    // b, Eq. (3)
                    } else {
                        const float2 m1 = mul2(T[1], iv2), m2 = mul2(T[2], iv2), m3 = mul2(T[3], iv2);
                        const float var = r ? fmaxf(fmaf(-m0.x, m0.x, m2.x), 0.0f) : 0.0f;
                        const float rv = __fdividef(1.0f, var + P.eps);
                        const float mx = m0.x + shift[0];
                        const float my[3] = {m0.y, m1.x, m1.y}, mxy[3] = {m2.y, m3.x, m3.y};
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float cov = r ? fmaf(-m0.x, my[k], mxy[k]) : 0.0f;
                            const float a = cov * rv;                             // a, Eq. (2)
                            o[2 * k][jj] = a;
                            o[2 * k + 1][jj] = (my[k] + shift[1 + k]) - a * mx;   // b, Eq. (3)
                        }
                    }
                } else if constexpr (KIND == SK_MEAN2) {
                    o[0][jj] = T[0].x * inv;  // mean_a
                    o[1][jj] = T[0].y * inv;  // mean_b
                } else {
                    o[0][jj] = fmaf(T[0].x * inv, iv[j], T[0].y * inv);  // Eq. (4)
                }
                if (jj == 3 && (j == 3 || second)) {  // a float4 of every output plane
                    const int xs = j - 3;
                    if constexpr (KIND == SK_MEAN2_OUT) {
                        if (P.detail != 0.0f) {
#pragma unroll
                            for (int e = 0; e < 4; ++e) o[0][e] = fmaf(P.detail, iv[xs + e] - o[0][e], o[0][e]);
                        }
                        store4q<TQ>(dq + xs, o[0]);
                    } else {
#pragma unroll
                        for (int k = 0; k < NO / 2; ++k) {
                            const float4 va = make_float4(o[2 * k][0], o[2 * k][1], o[2 * k][2], o[2 * k][3]);
                            const float4 vb =
                                make_float4(o[2 * k + 1][0], o[2 * k + 1][1], o[2 * k + 1][2], o[2 * k + 1][3]);
                            if (P.stream_out) {  // planes larger than L2: streamed
                                __stcs(reinterpret_cast<float4 *>(dst0[k] + xs), va);
                                __stcs(reinterpret_cast<float4 *>(dst1[k] + xs), vb);
                            } else {             // small planes stay in L2 for the next kernel
                                *reinterpret_cast<float4 *>(dst0[k] + xs) = va;
                                *reinterpret_cast<float4 *>(dst1[k] + xs) = vb;
                            }
                        }
                    }
                }
            }
        };
        if (interior) run(std::false_type{});
        else run(std::true_type{});
    }
}

// The segment of grid row p (of n): the rows take the segments in the order (k mod m, k / m).  With m the waves
// of resident CTAs an image's grid fills, segment k + 1 then starts in the wave after segment k's, about when
// segment k ends, so the 2r rows that open its window (the last ones segment k read) are still in L2.
__device__ __forceinline__ int seg_of(int p, int n, int m)
{
    for (int j = 0; j < m - 1; ++j) {
        const int c = (n - j + m - 1) / m;  // segments k < n with k mod m == j
        if (p < c) return j + m * p;
        p -= c;
    }
    return (m - 1) + m * p;
}

// CTAs per SM the registers are sized for: four; three for the three-channel statistics, whose batch of entering
// rows (four planes) needs the registers of a 3-CTA split (two where the batch holds the leaving rows too), and for
// the box means + output, which also holds the next block's guide row.
__host__ __device__ constexpr int minb_of(int KIND, int NQ, int RC)
{
    return pl_of(NQ, RC) ? 2 : ((NQ == 4 || KIND == SK_MEAN2_OUT) ? 3 : 4);
}

template <int KIND, int NY, int RC, typename TQ>
__global__ void __launch_bounds__(SP_NT, minb_of(KIND, nq_of(KIND, NY), RC)) k_box_strip(StripParams P)
{
    constexpr int NQ = nq_of(KIND, NY);
    constexpr bool PL = pl_of(NQ, RC);
    constexpr int VP = vp_rc(NQ, RC);  // column-sum pitch
    constexpr int NS = Column<KIND, NY>::NS;
    constexpr int NBUF = db_of(NQ) ? 2 : 1;
    const int r = RC >= 0 ? RC : P.r;
    const int h = P.h, w = P.w, tid = threadIdx.x;
    const int grp = blockIdx.x % P.groups, sx = blockIdx.x / P.groups, n = blockIdx.z;
    const int x0 = sx * SP_TW;
    const int y0 = P.ylo + seg_of(blockIdx.y, gridDim.y, P.seg_order) * P.seg, yend = min(y0 + P.seg, P.yhi);
    extern __shared__ __align__(16) unsigned char sm[];
    pdl_wait();  // launched with programmatic serialization: the previous kernel's planes are complete here

    // ---- this CTA's planes; for the statistics, the shift: every plane's value at the first output pixel
    const float *base[NS];
    if constexpr (KIND == SK_STATS) {
        base[0] = P.X + (size_t)(n * P.CX + (P.CX == 1 ? 0 : grp * NY)) * P.xps;
#pragma unroll
        for (int k = 0; k < NY; ++k) base[1 + k] = P.Y + (size_t)(n * P.C + grp * NY + k) * P.yps;
    } else {
        base[0] = P.X + (size_t)(n * P.C + grp) * P.xps;
        base[1] = P.Y + (size_t)(n * P.C + grp) * P.yps;
    }
    Column<KIND, NY> col;
    col.w = w;
    const int xc = x0 - r + tid;  // this thread's walker column
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        col.p[k] = base[k] + xc;
        col.c[k] = (KIND == SK_STATS) ? __ldg(base[k] + (size_t)y0 * w + x0) : 0.0f;
    }
    const bool walker = tid < SP_TW + 2 * r;
    const bool colok = walker && xc >= 0 && xc < w;

    // ---- the window of the segment's first row, less its last row: rows [y0 - r, y0 + r - 1]
    float2 S[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) S[q] = make_float2(0.0f, 0.0f);
    if (colok) {
        if (RC >= 0 && y0 - r >= 0 && y0 + r <= h) {
#pragma unroll
            for (int i = 0; i < 2 * (RC > 0 ? RC : 0); ++i) col.add_row(y0 - r + i, S);
        } else {
            for (int t = max(y0 - r, 0); t < min(y0 + r, h); ++t) col.add_row(t, S);
        }
    }

    // ---- phase-2 task: run g (outputs x0 + 8g .. + 7) of row k of each block
    const int pk = tid >> 4, pg = tid & 15;
    const int ox = x0 + pg * SP_RUN;
    const bool second = ox + 4 < w;
    const float inv_full = 1.0f / (float)((2 * r + 1) * (2 * r + 1));
    const bool x_interior = (ox - r >= 0) && (ox + SP_RUN - 1 + r < w);

    const int nblocks = (yend - y0 + SP_CB - 1) / SP_CB;
    // SK_MEAN2_OUT: the guide under this thread's run of output row y, requested a block ahead of its use
    float ivn[8];
    auto load_guide = [&](int yg, float (&dst)[8]) {
        if (yg < yend && ox < w) {
            const float *Ip = P.I + (size_t)(n * P.CI + (P.CI == 1 ? 0 : grp)) * P.fps + (size_t)yg * w + ox;
            const float4 u = __ldcs(reinterpret_cast<const float4 *>(Ip));
            const float4 v = second ? __ldcs(reinterpret_cast<const float4 *>(Ip) + 1)
                                    : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            dst[0] = u.x; dst[1] = u.y; dst[2] = u.z; dst[3] = u.w;
            dst[4] = v.x; dst[5] = v.y; dst[6] = v.z; dst[7] = v.w;
        }
    };
    if constexpr (KIND == SK_MEAN2_OUT) load_guide(y0 + pk, ivn);
    RowBatch<KIND, NY, PL> B;
    if (colok) B.fetch(col, y0, r, h);
    for (int b = 0; b < nblocks; ++b) {
        const int yb = y0 + b * SP_CB;
        unsigned char *buf = sm + (NBUF == 2 ? (size_t)(b & 1) * buf_bytes_rc(NQ, RC) : 0);
        // ---- phase 1: vertical window sums of the block's rows; then the next block's rows are requested
        if (colok) {
            walk_block<KIND, NY, PL, VP>(col, B, S, yb, r, h, buf, tid);
            if (b + 1 < nblocks) B.fetch(col, yb + SP_CB, r, h);
        } else if (walker) {  // a column outside the image contributes nothing
            const float2 Z[NQ] = {};
#pragma unroll 1
            for (int k = 0; k < SP_CB; ++k) put_sums<NQ, VP>(buf, k, tid, Z);
        }
        __syncthreads();

        // ---- phase 2: horizontal window sums along a run of 8 outputs, epilogue, 128-bit stores
        const int y = yb + pk;
        const bool live = (y < yend) && (ox < w);
        float iv[8];
        if constexpr (KIND == SK_MEAN2_OUT) {  // this block's guide row; the next block's is requested now
#pragma unroll
            for (int e = 0; e < 8; ++e) iv[e] = ivn[e];
            if (b + 1 < nblocks) load_guide(y + SP_CB, ivn);
        }
        run_block<KIND, NY, RC, TQ, VP>(P, buf, sm + NBUF * buf_bytes_rc(NQ, RC), col.c, iv, y, live, pk, pg, ox, r, h, w, n,
                                    grp, second, x_interior, inv_full);
        if (NBUF == 1 && b + 1 < nblocks) __syncthreads();  // the column sums are rewritten by the next block
    }
    pdl_trigger();  // this CTA's outputs are written: the next kernel may be scheduled
}

// ------------------------------------------------------------------------------------------------------
// k_box_strip_sub: Algorithm 2's first two steps in one kernel, for a gray guide serving three channels (the
// statistics of k_box_strip<SK_STATS, 3>) at s = 4 or 8 with nearest or bilinear subsampling.  The low-res
// samples are never written: a producer warp streams, for each low-res row t of the CTA's strip, the full-res
// rows the samples read (S t + S/2 - 1 and S t + S/2 for bilinear, S t + S/2 for nearest) of the guide and the
// three input planes into a ring of shared-memory stages by TMA (4-D view: column, row within the S-row block,
// block, plane; S boxes of 128 + 2r full-res columns per plane, 128 / S + 2r / S walker columns each).  Each walker forms its
// column's sample of the four planes from the stage (the subsample's arithmetic), adds it to the window sums,
// and keeps it in a ring of the last 2r + 1 samples of its column in shared memory, from which the leaving row
// is taken.  Phase 2 (the runs, the epilogue of Eq. 2-3) is k_box_strip's, on column sums of pitch 128 + 2r.
// At s = 4 two CTAs fit an SM (two stages each); at s = 8 one (three stages).
//
// Waits are bounded like the TMA output kernel's: a wait that gives up reports FAULT_BOX_TMA and the thread
// stops waiting (its results are not valid; the call reports the fault); the producer drains its loads before
// the CTA exits.
// ------------------------------------------------------------------------------------------------------
constexpr int SS_NT = SP_NT + 32;  // the 160 walkers / runs, then one producer warp

__host__ __device__ constexpr int ss_nph(int MODE) { return MODE == GF_SUB_BILINEAR ? 2 : 1; }
// walker columns (the column-sum pitch) and the full-res columns of one box: 128 + 2r
__host__ __device__ constexpr int ss_vp(int r) { return SP_TW + 2 * r; }
// bytes of one box (its nph rows) as loaded, and as laid out (128-byte aligned starts)
__host__ __device__ constexpr int ss_box_bytes(int MODE, int r) { return ss_nph(MODE) * ss_vp(r) * 4; }
__host__ __device__ constexpr int ss_box_pitch(int MODE, int r) { return (ss_box_bytes(MODE, r) + 127) / 128 * 128; }
// one ring stage: the sampled full-res rows of one low-res row, 4 planes x S boxes
__host__ __device__ constexpr int ss_stage_bytes(int S, int MODE, int r) { return 4 * S * ss_box_pitch(MODE, r); }
__host__ __device__ constexpr int ss_nst(int S) { return S == 4 ? 2 : 3; }  // stages (low-res rows in flight)
// column sums (pitch 128 + 2r) and block sums, the sample ring, the stages, the full / empty mbarriers
__host__ __device__ constexpr size_t ss_sums_bytes(int r) { return (size_t)SP_CB * ss_vp(r) * 32; }
__host__ __device__ constexpr size_t ss_smem(int S, int MODE, int r)
{
    return ss_sums_bytes(r) + bsum_bytes(4) + (size_t)(2 * r + 1) * ss_vp(r) * 16 +
           (size_t)ss_nst(S) * ss_stage_bytes(S, MODE, r) + (size_t)2 * ss_nst(S) * 8;
}

struct SubStripParams {
    StripParams P;  // X, Y unused; h, w low-res; CX = 1, groups = C / 3
    int H, W;       // full-res plane size
    unsigned *clear_word;
    FaultSink fault;
};

// The bilinear (or nearest) sample of one plane from its two (one) stage rows: the walker's S-column block
// starts at float `c` of each row, rows BW floats apart.
template <int S, int MODE, int BW>
__device__ __forceinline__ float stage_sample(const float *row, int c)
{
    if constexpr (MODE == GF_SUB_BILINEAR) {
        float t0, t1, b0, b1;  // columns S/2 - 1, S/2 of the two rows
        if constexpr (S == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(row + c);
            const float4 b = *reinterpret_cast<const float4 *>(row + BW + c);
            t0 = t.y; t1 = t.z; b0 = b.y; b1 = b.z;
        } else {
            t0 = row[c + S / 2 - 1]; t1 = row[c + S / 2];
            b0 = row[BW + c + S / 2 - 1]; b1 = row[BW + c + S / 2];
        }
        return 0.5f * (0.5f * t0 + 0.5f * t1) + 0.5f * (0.5f * b0 + 0.5f * b1);
    } else {
        return row[c + S / 2];
    }
}
// The same sample straight from global memory (the CTA's shift; the row pointer is that of block row 0).
template <int S, int MODE>
__device__ __forceinline__ float global_sample(const float *blk, int W)
{
    if constexpr (MODE == GF_SUB_BILINEAR) {
        const float *t = blk + (size_t)(S / 2 - 1) * W, *b = t + W;
        return 0.5f * (0.5f * __ldg(t + S / 2 - 1) + 0.5f * __ldg(t + S / 2)) +
               0.5f * (0.5f * __ldg(b + S / 2 - 1) + 0.5f * __ldg(b + S / 2));
    } else {
        return __ldg(blk + (size_t)(S / 2) * W + S / 2);
    }
}

template <int S, int MODE, int RC>
__global__ void __launch_bounds__(SS_NT, S == 4 ? 2 : 1)
    k_box_strip_sub(const __grid_constant__ CUtensorMap tmI, const __grid_constant__ CUtensorMap tmP,
                    const __grid_constant__ SubStripParams Q)
{
    constexpr int NY = 3, NQ = 4, NST = ss_nst(S);
    constexpr int VP = ss_vp(RC);                         // walker columns; full-res columns of a box
    constexpr int STAGE = ss_stage_bytes(S, MODE, RC);
    constexpr int BOXF = ss_box_pitch(MODE, RC) / 4;      // floats from one box to the next
    constexpr int STAGE_TX = 4 * S * ss_box_bytes(MODE, RC);  // bytes the loads of one stage bring
    constexpr int WPB = VP / S;                           // walker columns per box
    constexpr int R = 2 * RC + 1;                         // sample ring rows
    static_assert(VP % 8 == 0 && VP % S == 0 && VP <= 256, "box geometry");
    static_assert((ss_sums_bytes(RC) + bsum_bytes(4) + (size_t)R * VP * 16) % 128 == 0, "stages start 128-byte aligned");
    const StripParams &P = Q.P;
    const int r = RC, h = P.h, w = P.w, tid = threadIdx.x;
    const int grp = blockIdx.x % P.groups, sx = blockIdx.x / P.groups, n = blockIdx.z;
    const int x0 = sx * SP_TW;
    const int y0 = P.ylo + seg_of(blockIdx.y, gridDim.y, P.seg_order) * P.seg, yend = min(y0 + P.seg, P.yhi);
    const int tstart = max(y0 - r, 0), tend = min(yend + r, h);  // the low-res rows streamed, in order
    extern __shared__ __align__(128) unsigned char smx[];
    unsigned char *bsx = smx + ss_sums_bytes(RC);                          // block sums of phase 2
    float4 *ring = reinterpret_cast<float4 *>(bsx + bsum_bytes(NQ));      // [R][VP]: (I, p0, p1, p2) samples
    unsigned char *stages = reinterpret_cast<unsigned char *>(ring + R * VP);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(stages + (size_t)NST * STAGE);
    const unsigned full0 = smem_u32(bars), empty0 = smem_u32(bars + NST);
    pdl_wait();  // launched with programmatic serialization: the previous call's kernels are complete here
    // the call's fault word starts at zero; a wait gives up only after FaultSink::limit polls, long after this
    // CTA (the first scheduled) has run this line
    if (Q.clear_word && (blockIdx.x | blockIdx.y | blockIdx.z | tid) == 0) *Q.clear_word = 0u;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, SP_NT / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();

    const int plane_I = n, plane_p = n * P.C + grp * NY;
    if (tid >= SP_NT) {  // ---- producer warp: one lane streams the rows
        if (tid == SP_NT) {
            const int xf = S * (x0 - r);  // first full-res column of box 0 (a multiple of 4: 16-byte aligned)
            int issued = 0;
            for (int u = 0; u < tend - tstart; ++u) {
                const int st = u % NST;
                if (u >= NST && !mbar_wait(empty0 + 8 * st, ((u / NST) - 1) & 1, Q.fault, FAULT_BOX_TMA)) break;
                const unsigned fb = full0 + 8 * st;
                mbar_expect_tx(fb, STAGE_TX);
                float *dst = reinterpret_cast<float *>(stages + (size_t)st * STAGE);
                const int t = tstart + u;
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int k = 0; k < S; ++k)
                        tma_load_4d(dst + (q * S + k) * BOXF, q == 0 ? (const void *)&tmI : (const void *)&tmP,
                                    xf + VP * k, MODE == GF_SUB_BILINEAR ? S / 2 - 1 : S / 2, t,
                                    q == 0 ? plane_I : plane_p + q - 1, fb);
                issued = u + 1;
            }
            // every load issued has landed before the CTA may exit
            for (int u = max(0, issued - NST); u < issued; ++u)
                mbar_wait(full0 + 8 * (u % NST), (u / NST) & 1, Q.fault, FAULT_BOX_TMA);
        }
        pdl_trigger();
        return;
    }

    // ---- the shift: every plane's sample at the first output pixel (y0, x0)
    Column<SK_STATS, NY> col;
    {
        const size_t off = (size_t)S * y0 * Q.W + (size_t)S * x0;
        col.c[0] = global_sample<S, MODE>(P.X + (size_t)plane_I * P.xps + off, Q.W);
#pragma unroll
        for (int k = 0; k < NY; ++k) col.c[1 + k] = global_sample<S, MODE>(P.Y + (size_t)(plane_p + k) * P.yps + off, Q.W);
    }
    const int xc = x0 - r + tid;  // this thread's walker column
    const bool walker = tid < SP_TW + 2 * r;
    const bool colok = walker && xc >= 0 && xc < w;
    const int lane = tid & 31, wbox = tid / WPB, wcol = S * (tid % WPB);
    const float4 shift4 = make_float4(col.c[0], col.c[1], col.c[2], col.c[3]);
    bool waiting = true;  // false once a wait gave up
    // the samples of low-res row t at this column, kept in the ring; rows outside the image read as the shift
    auto enter = [&](int t) -> float4 {
        float4 v = shift4;
        if (t >= tstart && t < tend) {
            const int u = t - tstart, st = u % NST;
            if (waiting && !mbar_wait(full0 + 8 * st, (u / NST) & 1, Q.fault, FAULT_BOX_TMA)) waiting = false;
            if (waiting && colok) {
                const float *sb = reinterpret_cast<const float *>(stages + (size_t)st * STAGE) + wbox * BOXF;
                v.x = stage_sample<S, MODE, VP>(sb, wcol);
                v.y = stage_sample<S, MODE, VP>(sb + S * BOXF, wcol);
                v.z = stage_sample<S, MODE, VP>(sb + 2 * S * BOXF, wcol);
                v.w = stage_sample<S, MODE, VP>(sb + 3 * S * BOXF, wcol);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * st);
        }
        if (walker) ring[((t + R) % R) * VP + tid] = v;
        return v;
    };
    auto add = [&](float2 (&S2)[NQ], const float4 &v, bool sub) {
        const float vv[4] = {v.x, v.y, v.z, v.w};
        float2 q[NQ];
        col.pairs(vv, q);
#pragma unroll
        for (int k = 0; k < NQ; ++k) S2[k] = sub ? sub2(S2[k], q[k]) : add2(S2[k], q[k]);
    };

    // ---- the window of the segment's first row, less its last row: rows [y0 - r, y0 + r - 1]
    float2 Sw[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) Sw[q] = make_float2(0.0f, 0.0f);
#pragma unroll 1
    for (int t = y0 - r; t < y0 + r; ++t) add(Sw, enter(t), false);

    const int pk = tid >> 4, pg = tid & 15;
    const int ox = x0 + pg * SP_RUN;
    const bool second = ox + 4 < w;
    const float inv_full = 1.0f / (float)((2 * r + 1) * (2 * r + 1));
    const bool x_interior = (ox - r >= 0) && (ox + SP_RUN - 1 + r < w);
    const int nblocks = (yend - y0 + SP_CB - 1) / SP_CB;
    const float iv[8] = {};
    for (int b = 0; b < nblocks; ++b) {
        const int yb = y0 + b * SP_CB;
        // ---- phase 1: row yb + k + r enters the window of output row yb + k, row yb + k - r leaves after
#pragma unroll 1
        for (int k = 0; k < SP_CB; ++k) {
            add(Sw, enter(yb + k + r), false);
            if (walker) {
                put_sums<NQ, VP>(smx, k, tid, Sw);
                add(Sw, ring[((yb + k - r + R) % R) * VP + tid], true);
            }
        }
        asm volatile("bar.sync 1, %0;\n" ::"r"(SP_NT) : "memory");  // walkers / runs only
        // ---- phase 2
        const int y = yb + pk;
        run_block<SK_STATS, NY, RC, float, VP>(P, smx, bsx, col.c, iv, y, (y < yend) && (ox < w), pk, pg, ox, r, h, w,
                                               n, grp, second, x_interior, inv_full);
        if (b + 1 < nblocks) asm volatile("bar.sync 1, %0;\n" ::"r"(SP_NT) : "memory");
    }
    pdl_trigger();
}

// SMs of the current device (cached per device ordinal).
int sm_count()
{
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    const int slot = dev < 64 ? dev : 63;
    int n = cached[slot].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        if (dev < 64) cached[slot].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Rows per CTA (at most SP_SEG_MAX): the segment length that minimises (waves of CTAs) x (rows a CTA walks, its 2r opening rows
// included) for `tasks` CTAs per segment row and `resident` CTAs on the GPU at once.
int segment_rows(int rows, int r, long long tasks, long long resident)
{
    const int max_seg = min(((rows + SP_CB - 1) / SP_CB) * SP_CB, SP_SEG_MAX);
    int best = max_seg;
    long long best_cost = -1;
    for (int seg = SP_CB; seg <= max_seg; seg += SP_CB) {
        const long long nseg = (rows + seg - 1) / seg;
        const long long waves = (tasks * nseg + resident - 1) / resident;
        const long long cost = waves * (seg + 2 * r);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = seg;
        }
    }
    return best;
}

template <int KIND, int NY, int RC, typename TQ>
cudaError_t launch_strip(StripParams P, int N, cudaStream_t st)
{
    auto kern = k_box_strip<KIND, NY, RC, TQ>;
    constexpr size_t smem = strip_smem_rc(nq_of(KIND, NY), RC);
    cudaError_t e = opt_in_smem(kern, smem);
    if (e != cudaSuccess) return e;
    static std::atomic<int> per_sm_cached{0};  // CTAs per SM of this instantiation
    int per_sm = per_sm_cached.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SP_NT, smem)) != cudaSuccess) return e;
        per_sm = per_sm > 0 ? per_sm : 1;
        per_sm_cached.store(per_sm, std::memory_order_relaxed);
    }
    const int strips = (P.w + SP_TW - 1) / SP_TW;
    const long long tasks = (long long)strips * P.groups * N;
    const long long resident = (long long)per_sm * sm_count();
    P.seg = segment_rows(P.yhi - P.ylo, P.r, tasks, resident);
    const int nseg = (P.yhi - P.ylo + P.seg - 1) / P.seg;
    const long long waves = ((long long)strips * P.groups * nseg + resident - 1) / resident;  // of one image
    P.seg_order = (int)std::min<long long>(std::max<long long>(waves, 1), nseg);
    const dim3 grid((unsigned)(strips * P.groups), (unsigned)nseg, (unsigned)N);
    if ((e = launch_pdl(kern, grid, dim3(SP_NT), smem, st, P)) != cudaSuccess) return e;
    return cudaGetLastError();
}

// The radius as a compile-time constant at r = 16 (s = 1 at the paper's 12 MP figure radius) and 15 (the
// feathering figure's r' at s = 4), else at run time.
template <int KIND, int NY, typename TQ>
cudaError_t launch_radius(const StripParams &P, int N, cudaStream_t st)
{
    if (P.r == 16) return launch_strip<KIND, NY, 16, TQ>(P, N, st);
    if (P.r == 15) return launch_strip<KIND, NY, 15, TQ>(P, N, st);
    if (P.r == 4) return launch_strip<KIND, NY, 4, TQ>(P, N, st);
    return launch_strip<KIND, NY, -1, TQ>(P, N, st);
}

bool aligned16s(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

bool strip_box_supported(const BoxTmaJob &J)
{
    if (J.r < 1 || J.r > SP_RMAX || J.w % 4 != 0 || J.stats != nullptr) return false;
    if ((long long)J.h * J.w >= (1LL << 31) || J.h > 65535 * SP_CB || J.N > 65535 || J.N < 1) return false;
    if ((long long)((J.w + SP_TW - 1) / SP_TW) * J.C >= (1LL << 31)) return false;
    if (J.kind == BOX_JOB_MEANS_OUTPUT) {
        if (!aligned16s(J.I) || !aligned16s(J.q) || J.fps % 4 != 0) return false;
        if (J.dt_out != F32 && J.dt_out != F16) return false;
        if (J.Yw0 < 0 || J.Yw1 > J.h || J.Yw0 >= J.Yw1) return false;
    } else if (!aligned16s(J.out0) || !aligned16s(J.out1) || J.ops % 4 != 0) {
        return false;
    }
    return getenv("GF_NO_STRIP_BOX") == nullptr;  // the tile kernels instead (tests)
}

cudaError_t launch_strip_box(const BoxTmaJob &J, cudaStream_t st)
{
    StripParams P{};
    P.X = J.X;
    P.Y = J.Y;
    P.xps = J.xps;
    P.yps = J.yps;
    P.C = J.C;
    P.CX = J.CX;
    P.h = J.h;
    P.w = J.w;
    P.r = J.r;
    P.ylo = 0;
    P.yhi = J.h;
    P.eps = J.eps;
    P.out0 = J.out0;
    P.out1 = J.out1;
    P.ops = J.ops;
    // outputs larger than half of L2 do not stay there for the next kernel anyway
    P.stream_out = (double)J.N * J.C * J.h * J.w * 2 * sizeof(float) > 64e6;
    P.I = J.I;
    P.q = J.q;
    P.fps = J.fps;
    P.CI = J.CI;
    P.detail = J.detail;
    switch (J.kind) {
    case BOX_JOB_STATS:
        if (J.CX == 1 && J.C % 3 == 0) {  // one guide plane for three channels: its sums formed once
            P.groups = J.C / 3;
            return launch_radius<SK_STATS, 3, float>(P, J.N, st);
        }
        P.groups = J.C;
        return launch_radius<SK_STATS, 1, float>(P, J.N, st);
    case BOX_JOB_MEANS:
        P.groups = J.C;
        return launch_radius<SK_MEAN2, 1, float>(P, J.N, st);
    default:
        P.groups = J.C;
        P.ylo = J.Yw0;
        P.yhi = J.Yw1;
        if (J.dt_out == F16) return launch_radius<SK_MEAN2_OUT, 1, __half>(P, J.N, st);
        return launch_radius<SK_MEAN2_OUT, 1, float>(P, J.N, st);
    }
}

namespace {

template <int S, int MODE, int RC>
cudaError_t launch_ss(const CUtensorMap &mI, const CUtensorMap &mP, SubStripParams Q, int N, cudaStream_t st)
{
    auto kern = k_box_strip_sub<S, MODE, RC>;
    constexpr size_t smem = ss_smem(S, MODE, RC);
    cudaError_t e = opt_in_smem(kern, smem);
    if (e != cudaSuccess) return e;
    static std::atomic<int> per_sm_cached{0};
    int per_sm = per_sm_cached.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SS_NT, smem)) != cudaSuccess) return e;
        per_sm = per_sm > 0 ? per_sm : 1;
        per_sm_cached.store(per_sm, std::memory_order_relaxed);
    }
    StripParams &P = Q.P;
    const int strips = (P.w + SP_TW - 1) / SP_TW;
    const long long tasks = (long long)strips * P.groups * N;
    const long long resident = (long long)per_sm * sm_count();
    P.seg = segment_rows(P.yhi - P.ylo, RC, tasks, resident);
    const int nseg = (P.yhi - P.ylo + P.seg - 1) / P.seg;
    const long long waves = ((long long)strips * P.groups * nseg + resident - 1) / resident;
    P.seg_order = (int)std::min<long long>(std::max<long long>(waves, 1), nseg);
    const dim3 grid((unsigned)(strips * P.groups), (unsigned)nseg, (unsigned)N);
    if ((e = launch_pdl(kern, grid, dim3(SS_NT), smem, st, mI, mP, Q)) != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

bool strip_sub_geometry(int C, int CI, int H, int W, int h, int w, int s, int sd, int mode, int r_low, int dt_in,
                        bool p_lowres)
{
    if (!getenv("GF_SUB_STRIP")) return false;
    return dt_in == F32 && !p_lowres && sd == 1 && (s == 4 || s == 8) &&
           (mode == GF_SUB_BILINEAR || mode == GF_SUB_NEAREST) && CI == 1 && C % 3 == 0 && H == s * h &&
           W == s * w && W % 4 == 0 && w % 4 == 0 && r_low == 4 && (long long)H * W < (1LL << 31) &&
           h <= 65535 * SP_CB;
}

bool strip_sub_supported(const SubStripJob &J)
{
    return strip_sub_geometry(J.C, 1, J.H, J.W, J.h, J.w, J.s, 1, J.mode, J.r, F32, false) && J.N >= 1 &&
           J.N <= 65535 && aligned16s(J.I) && aligned16s(J.p) && J.fps % 4 == 0 && aligned16s(J.a) &&
           aligned16s(J.b) && J.ops % 4 == 0 && (long long)((J.w + SP_TW - 1) / SP_TW) * (J.C / 3) < (1LL << 31);
}

cudaError_t launch_strip_sub(const SubStripJob &J, cudaStream_t st)
{
    const int nph = J.mode == GF_SUB_BILINEAR ? 2 : 1;
    CUtensorMap mI, mP;
    if (!encode_tmap_sampled_rows(&mI, J.I, J.W, J.s, J.h, J.N, J.fps, ss_vp(J.r), nph) ||
        !encode_tmap_sampled_rows(&mP, J.p, J.W, J.s, J.h, J.N * J.C, J.fps, ss_vp(J.r), nph))
        return cudaErrorInvalidValue;
    SubStripParams Q{};
    StripParams &P = Q.P;
    P.X = J.I;
    P.Y = J.p;
    P.xps = P.yps = J.fps;
    P.C = J.C;
    P.CX = 1;
    P.groups = J.C / 3;
    P.h = J.h;
    P.w = J.w;
    P.r = J.r;
    P.ylo = 0;
    P.yhi = J.h;
    P.eps = J.eps;
    P.out0 = J.a;
    P.out1 = J.b;
    P.ops = J.ops;
    P.stream_out = (double)J.N * J.C * J.h * J.w * 2 * sizeof(float) > 64e6;
    Q.H = J.H;
    Q.W = J.W;
    Q.clear_word = J.clear_word;
    Q.fault = J.fault;
    if (J.s == 4) {
        return J.mode == GF_SUB_BILINEAR ? launch_ss<4, GF_SUB_BILINEAR, 4>(mI, mP, Q, J.N, st)
                                         : launch_ss<4, GF_SUB_NEAREST, 4>(mI, mP, Q, J.N, st);
    }
    return J.mode == GF_SUB_BILINEAR ? launch_ss<8, GF_SUB_BILINEAR, 4>(mI, mP, Q, J.N, st)
                                     : launch_ss<8, GF_SUB_NEAREST, 4>(mI, mP, Q, J.N, st);
}

}  // namespace gfk
