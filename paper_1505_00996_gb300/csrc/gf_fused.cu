// gf_fused.cu -- the whole of Algorithm 2 in one kernel, for small images.
//
// Below a few megapixels the four-kernel chain is dominated by per-kernel fixed costs (launch, ramp-up,
// tail: several microseconds each) rather than by bytes.  k_fgf_fused runs every step of Algorithm 2 for
// one output tile in one CTA, recomputing the halo instead of exchanging it:
//   tile       TH x TW full-resolution output pixels of one channel;
//   T          the low-res taps those pixels sample (gf.h upsampling convention);
//   A = T +- r' the a, b the box means over T need;
//   L = A +- r' the subsampled I', p' the statistics over A need (all regions clipped to the image, so
//              every window is the image's own clipped window and the result is the whole-image result).
// Steps, each a pass over a shared-memory region with a barrier between:
//   1. I', p' at L from the full-resolution planes (any subsample mode, integer or rational ratio);
//   2. vertical window sums of I', p', I'^2, I'p' (shifted by one sample) for the rows of A;
//   3. horizontal sums, then Eq. 2-3: a, b at A;
//   4-5. the box means of a and b over T (vertical, then horizontal);
//   6. bilinear upsampling from T and q = mean_a I + mean_b (+ the detail epilogue) for the tile.
// Windows are summed directly (2r' + 1 terms), which is cheap at the radii small images use.
#include <algorithm>

#include "gf_device.cuh"
#include "gf_internal.cuh"

namespace gfk {

namespace {

constexpr int FU_NT = 256;

struct FusedParams {
    const void *I, *p;
    void *q;
    int C, CI, H, W, h, w, s, sn, sd, r, mode;
    float eps, detail;
    size_t fps, lpin;  // plane strides: full-res I, p, q; a low-res p given by the caller
    bool p_lowres;
    int TH, TW;        // full-res tile
    int Yw0, Yw1;      // rows written
    unsigned *clear_word;  // the call's fault word: zeroed by the first thread (this is the call's only kernel)
};

// The whole filter for output tile (bx, by) of plane bz = n C + c (one CTA; sm: the CTA's shared memory).
template <typename TI, typename TQ, int MODE>
__device__ __forceinline__ void fused_tile(const FusedParams &P, int bx, int by, int bz, float *sm)
{
    const int tid = threadIdx.x;
    if (P.clear_word && (bx | by | bz | tid) == 0) *P.clear_word = 0u;
    const int n = bz / P.C, c = bz - n * P.C;
    const int X0 = bx * P.TW, X1 = min(X0 + P.TW, P.W);  // columns [X0, X1)
    const int Ya = max(by * P.TH, P.Yw0), Yb = min(min(by * P.TH + P.TH, P.H), P.Yw1);
    if (Ya >= Yb) return;
    const int h = P.h, w = P.w, r = P.r;
    // regions in low-res coordinates, inclusive bounds
    int ty0, ty1, tx0, tx1, t;
    float f;
    up_taps_q(Ya, P.sn, P.sd, h, ty0, t, f);
    up_taps_q(Yb - 1, P.sn, P.sd, h, t, ty1, f);
    up_taps_q(X0, P.sn, P.sd, w, tx0, t, f);
    up_taps_q(X1 - 1, P.sn, P.sd, w, t, tx1, f);
    const int ay0 = max(0, ty0 - r), ay1 = min(h - 1, ty1 + r), ax0 = max(0, tx0 - r), ax1 = min(w - 1, tx1 + r);
    const int ly0 = max(0, ay0 - r), ly1 = min(h - 1, ay1 + r), lx0 = max(0, ax0 - r), lx1 = min(w - 1, ax1 + r);
    const int Th = ty1 - ty0 + 1, Tw = tx1 - tx0 + 1, Ah = ay1 - ay0 + 1, Aw = ax1 - ax0 + 1;
    const int Lh = ly1 - ly0 + 1, Lw = lx1 - lx0 + 1;
    float *Ls = sm;                    // [2][Lh][Lw]  I', p'
    float *V = Ls + 2 * Lh * Lw;       // [4][Ah][Lw]  vertical sums of dI, dp, dI^2, dI dp
    float *AB = V + 4 * Ah * Lw;       // [2][Ah][Aw]  a, b
    float *Vm = AB + 2 * Ah * Aw;      // [2][Th][Aw]  vertical sums of a, b (shifted)
    float *M = Vm + 2 * Th * Aw;       // [2][Th][Tw]  mean_a, mean_b

    const size_t HW = P.fps;
    const TI *Ig = (const TI *)P.I + (size_t)(n * P.CI + (P.CI == 1 ? 0 : c)) * HW;
    const TI *pg = (const TI *)P.p + (size_t)(n * P.C + c) * (P.p_lowres ? P.lpin : HW);

    // 1. subsample I and p at L
    for (int idx = tid; idx < Lh * Lw; idx += FU_NT) {
        const int jj = ly0 + idx / Lw, ii = lx0 + idx % Lw;
        float vi, vp;
        if constexpr (MODE == GF_SUB_BILINEAR_AA) {
            vi = (P.s == 1) ? ldv(Ig + (size_t)jj * P.W + ii) : subsample_aa_one(Ig, P.H, P.W, P.sn, P.sd, jj, ii);
            vp = P.p_lowres ? ldv(pg + (size_t)jj * w + ii)
                            : ((P.s == 1) ? ldv(pg + (size_t)jj * P.W + ii) : subsample_aa_one(pg, P.H, P.W, P.sn, P.sd, jj, ii));
        } else {
            vi = subsample_one<TI, MODE>(Ig, P.H, P.W, P.s, P.sn, P.sd, jj, ii);
            vp = P.p_lowres ? ldv(pg + (size_t)jj * w + ii) : subsample_one<TI, MODE>(pg, P.H, P.W, P.s, P.sn, P.sd, jj, ii);
        }
        Ls[idx] = vi;
        Ls[Lh * Lw + idx] = vp;
    }
    __syncthreads();
    const float sI = Ls[0], sp = Ls[Lh * Lw];  // shifts: E[x^2] - E[x]^2 then does not cancel badly in FP32

    // 2. vertical window sums for the rows of A, every column of L
    for (int idx = tid; idx < Ah * Lw; idx += FU_NT) {
        const int ja = ay0 + idx / Lw, col = idx % Lw;
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        for (int k = max(0, ja - r); k <= min(h - 1, ja + r); ++k) {
            const float di = Ls[(k - ly0) * Lw + col] - sI, dp = Ls[Lh * Lw + (k - ly0) * Lw + col] - sp;
            s0 += di;
            s1 += dp;
            s2 = fmaf(di, di, s2);
            s3 = fmaf(di, dp, s3);
        }
        V[idx] = s0;
        V[Ah * Lw + idx] = s1;
        V[2 * Ah * Lw + idx] = s2;
        V[3 * Ah * Lw + idx] = s3;
    }
    __syncthreads();

    // 3. horizontal sums and Eq. (2)-(3) at A
    for (int idx = tid; idx < Ah * Aw; idx += FU_NT) {
        const int ja = ay0 + idx / Aw, ia = ax0 + idx % Aw;
        const int ka = max(0, ia - r), kb = min(w - 1, ia + r);
        const float *v0 = V + (ja - ay0) * Lw - lx0;
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        for (int k = ka; k <= kb; ++k) {
            s0 += v0[k];
            s1 += v0[Ah * Lw + k];
            s2 += v0[2 * Ah * Lw + k];
            s3 += v0[3 * Ah * Lw + k];
        }
        const float inv = 1.0f / (float)((min(h - 1, ja + r) - max(0, ja - r) + 1) * (kb - ka + 1));
        const float mI = s0 * inv, mp = s1 * inv, eII = s2 * inv, eIp = s3 * inv;  // shifted means
        // var_I, cov_Ip: exactly 0 for a one-sample window (r' = 0), where Eq. 2 gives a = 0
        const float var = r ? fmaxf(eII - mI * mI, 0.0f) : 0.0f, cov = r ? eIp - mI * mp : 0.0f;
        const float a = cov / (var + P.eps);  // Eq. (2)
        AB[idx] = a;
        AB[Ah * Aw + idx] = (mp + sp) - a * (mI + sI);  // Eq. (3)
    }
    __syncthreads();
    const float sa = AB[0], sb = AB[Ah * Aw];

    // 4. vertical sums of a, b for the rows of T, every column of A
    for (int idx = tid; idx < Th * Aw; idx += FU_NT) {
        const int jt = ty0 + idx / Aw, col = idx % Aw;
        float s0 = 0.0f, s1 = 0.0f;
        for (int k = max(0, jt - r); k <= min(h - 1, jt + r); ++k) {
            s0 += AB[(k - ay0) * Aw + col] - sa;
            s1 += AB[Ah * Aw + (k - ay0) * Aw + col] - sb;
        }
        Vm[idx] = s0;
        Vm[Th * Aw + idx] = s1;
    }
    __syncthreads();

    // 5. horizontal sums: mean_a, mean_b at T
    for (int idx = tid; idx < Th * Tw; idx += FU_NT) {
        const int jt = ty0 + idx / Tw, it = tx0 + idx % Tw;
        const int ka = max(0, it - r), kb = min(w - 1, it + r);
        const float *v0 = Vm + (jt - ty0) * Aw - ax0;
        float s0 = 0.0f, s1 = 0.0f;
        for (int k = ka; k <= kb; ++k) {
            s0 += v0[k];
            s1 += v0[Th * Aw + k];
        }
        const float inv = 1.0f / (float)((min(h - 1, jt + r) - max(0, jt - r) + 1) * (kb - ka + 1));
        M[idx] = fmaf(s0, inv, sa);
        M[Th * Tw + idx] = fmaf(s1, inv, sb);
    }
    __syncthreads();

    // 6. upsample and Eq. (4) for the tile, 4 adjacent pixels per item
    const int qw = (X1 - X0 + 3) / 4;
    TQ *qp = (TQ *)P.q + (size_t)(n * P.C + c) * HW;
    for (int item = tid; item < (Yb - Ya) * qw; item += FU_NT) {
        const int Y = Ya + item / qw, Xq = X0 + 4 * (item % qw);
        int ya, yb;
        float fy;
        up_taps_q(Y, P.sn, P.sd, h, ya, yb, fy);
        const float *ra = M + (ya - ty0) * Tw - tx0, *rb = M + (yb - ty0) * Tw - tx0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int X = Xq + k;
            if (X >= X1) break;
            int xa, xb;
            float fx;
            up_taps_q(X, P.sn, P.sd, w, xa, xb, fx);
            const float ta = fmaf(fx, ra[xb] - ra[xa], ra[xa]), tb = fmaf(fx, rb[xb] - rb[xa], rb[xa]);
            const float ua = fmaf(fx, ra[Th * Tw + xb] - ra[Th * Tw + xa], ra[Th * Tw + xa]);
            const float ub = fmaf(fx, rb[Th * Tw + xb] - rb[Th * Tw + xa], rb[Th * Tw + xa]);
            const float A = fmaf(fy, tb - ta, ta), B = fmaf(fy, ub - ua, ua);  // upsampled mean_a, mean_b
            const float iv = ldv(Ig + (size_t)Y * P.W + X);
            float out = fmaf(A, iv, B);  // Eq. (4)
            if (P.detail != 0.0f) out = fmaf(P.detail, iv - out, out);
            if constexpr (sizeof(TQ) == 4) qp[(size_t)Y * P.W + X] = out;
            else qp[(size_t)Y * P.W + X] = __float2half_rn(out);
        }
    }
}

template <typename TI, typename TQ, int MODE>
__global__ void __launch_bounds__(FU_NT) k_fgf_fused(FusedParams P)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    extern __shared__ float sm[];
    fused_tile<TI, TQ, MODE>(P, blockIdx.x, blockIdx.y, blockIdx.z, sm);
    pdl_trigger();
}

// The tile-queue form: one launch for the tiles of up to FUSED_QUEUE_MAX requests of the same storage types
// and subsample mode, each with its own descriptor (sizes, strides, r', s, eps, pointers, tile shape).  CTA t
// takes tile t - start[k] of request k, the k with start[k] <= t < start[k + 1]; each tile is computed exactly
// as the request's own launch computes it, so a request's output does not depend on what it was batched with.
struct FusedQueue {
    int n;
    int start[FUSED_QUEUE_MAX + 1];
    int gx[FUSED_QUEUE_MAX], gy[FUSED_QUEUE_MAX];  // the request's tile columns and rows
    FusedParams p[FUSED_QUEUE_MAX];
};

template <typename TI, typename TQ, int MODE>
__global__ void __launch_bounds__(FU_NT) k_fgf_fused_queue(const __grid_constant__ FusedQueue Q)
{
    pdl_wait();  // launched with programmatic serialization: earlier kernels are complete here
    extern __shared__ float sm[];
    const int t = blockIdx.x;
    int k = 0;
    while (k + 1 < Q.n && t >= Q.start[k + 1]) ++k;
    const int local = t - Q.start[k], gx = Q.gx[k], gy = Q.gy[k];
    fused_tile<TI, TQ, MODE>(Q.p[k], local % gx, (local / gx) % gy, local / (gx * gy), sm);
    pdl_trigger();
}

// Upper bounds of the region sizes for a TH x TW tile (low-res rows / columns), and the shared memory.
struct FusedShape {
    int TH, TW;
    size_t smem;
};

size_t fused_smem(int TH, int TW, int sn, int sd, int r)
{
    const long long th = ((long long)(TH - 1) * sd + sn - 1) / sn + 2, tw = ((long long)(TW - 1) * sd + sn - 1) / sn + 2;
    const long long ah = th + 2 * r, aw = tw + 2 * r, lh = ah + 2 * r, lw = aw + 2 * r;
    return (size_t)(2 * lh * lw + 4 * ah * lw + 2 * ah * aw + 2 * th * aw + 2 * th * tw) * sizeof(float);
}

constexpr size_t FUSED_SMEM_MAX = 100 * 1024;

// The tile: the largest candidate whose regions fit FUSED_SMEM_MAX, made smaller while the grid would give
// fewer than two CTAs per SM (small images: the halo recomputation then costs less than idle SMs).
bool fused_shape(int sn, int sd, int r, long long H, long long W, long long planes, FusedShape &S)
{
    static const int cand[][2] = {{32, 128}, {16, 128}, {16, 64}, {16, 32}, {8, 32}};
    bool found = false;
    for (const auto &t : cand) {
        const size_t b = fused_smem(t[0], t[1], sn, sd, r);
        if (b > FUSED_SMEM_MAX) continue;
        S = {t[0], t[1], b};
        found = true;
        const long long ctas = ((H + t[0] - 1) / t[0]) * ((W + t[1] - 1) / t[1]) * planes;
        if (ctas >= 2 * 152) break;
    }
    return found;
}

}  // namespace

bool fused_supported(const Resolved &R, bool intermediates)
{
    FusedShape S;
    return !R.color && !R.int_stats && !intermediates && fused_shape(R.sn, R.sd, R.r_low, R.H, R.W, 1, S);
}

namespace {

// The kernel's descriptor of a plan, with the plan's tile shape.
FusedParams fused_params(const FwdPlan &P, const FusedShape &S)
{
    FusedParams F;
    F.I = P.I; F.p = P.p; F.q = P.q;
    F.C = P.C; F.CI = P.CI; F.H = P.H; F.W = P.W; F.h = P.h; F.w = P.w;
    F.s = P.s; F.sn = P.sn; F.sd = P.sd; F.r = P.r_low; F.mode = P.mode;
    F.eps = P.eps; F.detail = P.detail;
    F.fps = P.fps; F.lpin = P.lpin; F.p_lowres = P.p_lowres;
    F.TH = S.TH; F.TW = S.TW;
    F.Yw0 = P.Yw0; F.Yw1 = P.Yw1;
    F.clear_word = P.clear_fault ? P.fault.call : nullptr;
    return F;
}

}  // namespace

cudaError_t launch_fused_queue(const FwdPlan *plans, int n, cudaStream_t st)
{
    if (n < 1 || n > FUSED_QUEUE_MAX) return cudaErrorInvalidValue;
    FusedQueue Q{};
    Q.n = n;
    size_t smem = 0;
    long long total = 0;
    for (int k = 0; k < n; ++k) {
        const FwdPlan &P = plans[k];
        if (P.dt_in != plans[0].dt_in || P.dt_out != plans[0].dt_out || P.mode != plans[0].mode)
            return cudaErrorInvalidValue;
        FusedShape S;
        if (!fused_shape(P.sn, P.sd, P.r_low, P.H, P.W, (long long)P.N * P.C, S)) return cudaErrorInvalidValue;
        Q.p[k] = fused_params(P, S);
        Q.gx[k] = (P.W + S.TW - 1) / S.TW;
        Q.gy[k] = (P.H + S.TH - 1) / S.TH;
        Q.start[k] = (int)total;
        total += (long long)Q.gx[k] * Q.gy[k] * P.N * P.C;
        smem = std::max(smem, S.smem);
    }
    if (total < 1 || total >= (1LL << 31)) return cudaErrorInvalidValue;
    Q.start[n] = (int)total;
    const FwdPlan &P0 = plans[0];
    cudaError_t e;
#define GF_FQ(TI, TQ, M)                                                                     \
    do {                                                                                     \
        if ((e = opt_in_smem(k_fgf_fused_queue<TI, TQ, M>, smem)) != cudaSuccess) return e;  \
        launch_pdl(k_fgf_fused_queue<TI, TQ, M>, (unsigned)total, dim3(FU_NT), smem, st, Q);               \
    } while (0)
#define GF_FQ_MODE(TI, TQ)                                                                   \
    do {                                                                                     \
        switch (P0.mode) {                                                                   \
        case GF_SUB_NEAREST: GF_FQ(TI, TQ, GF_SUB_NEAREST); break;                           \
        case GF_SUB_BILINEAR: GF_FQ(TI, TQ, GF_SUB_BILINEAR); break;                         \
        case GF_SUB_BOX: GF_FQ(TI, TQ, GF_SUB_BOX); break;                                   \
        default: GF_FQ(TI, TQ, GF_SUB_BILINEAR_AA); break;                                   \
        }                                                                                    \
    } while (0)
    if (P0.dt_in == F32) {
        if (P0.dt_out == F32) GF_FQ_MODE(float, float); else GF_FQ_MODE(float, __half);
    } else {
        if (P0.dt_out == F32) GF_FQ_MODE(__half, float); else GF_FQ_MODE(__half, __half);
    }
#undef GF_FQ_MODE
#undef GF_FQ
    return cudaGetLastError();
}

cudaError_t launch_fused(const FwdPlan &P, cudaStream_t st)
{
    FusedShape S;
    if (!fused_shape(P.sn, P.sd, P.r_low, P.H, P.W, (long long)P.N * P.C, S)) return cudaErrorInvalidValue;
    const FusedParams F = fused_params(P, S);
    dim3 grid((P.W + S.TW - 1) / S.TW, (P.H + S.TH - 1) / S.TH, P.N * P.C);
    cudaError_t e;
#define GF_FU(TI, TQ, M)                                                                     \
    do {                                                                                     \
        if ((e = opt_in_smem(k_fgf_fused<TI, TQ, M>, S.smem)) != cudaSuccess) return e;      \
        launch_pdl(k_fgf_fused<TI, TQ, M>, grid, dim3(FU_NT), S.smem, st, F);                              \
    } while (0)
#define GF_FU_MODE(TI, TQ)                                                                   \
    do {                                                                                     \
        switch (P.mode) {                                                                    \
        case GF_SUB_NEAREST: GF_FU(TI, TQ, GF_SUB_NEAREST); break;                           \
        case GF_SUB_BILINEAR: GF_FU(TI, TQ, GF_SUB_BILINEAR); break;                         \
        case GF_SUB_BOX: GF_FU(TI, TQ, GF_SUB_BOX); break;                                   \
        default: GF_FU(TI, TQ, GF_SUB_BILINEAR_AA); break;                                   \
        }                                                                                    \
    } while (0)
    if (P.dt_in == F32) {
        if (P.dt_out == F32) GF_FU_MODE(float, float); else GF_FU_MODE(float, __half);
    } else {
        if (P.dt_out == F32) GF_FU_MODE(__half, float); else GF_FU_MODE(__half, __half);
    }
#undef GF_FU_MODE
#undef GF_FU
    return cudaGetLastError();
}

}  // namespace gfk
