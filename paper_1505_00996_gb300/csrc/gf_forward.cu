// gf_forward.cu -- sm_103a kernels of the fast guided filter forward pass (Algorithm 2 of He and Sun,
// "Fast Guided Filter", 2015) and the host launcher that chains them.
//
//   k_subsample   Algorithm 2 first step: I' = f_subsample(I, s), p' = f_subsample(p, s) into FP32 low-res
//                 planes (nearest, bilinear or box; see gf.h for the conventions).
//   k_sweep       KIND 0/1: the box statistics of I', p', I'.*I', I'.*p' at radius r' fused with the
//                 variance/covariance and the coefficients a (Eq. 2) and b (Eq. 3).
//                 KIND 2: the box means of a and b.
//                 One CTA owns a strip of output columns and a run of rows; it sweeps down the rows keeping
//                 compensated running column sums in registers (O(1) work per pixel for any r'), then does
//                 the horizontal window sums from shared memory with sliding sums.
//   k_upsample_output
//                 Algorithm 2 last two steps fused: bilinear upsampling of mean_a, mean_b (never written at
//                 full resolution) and q = mean_a .* I + mean_b (Eq. 4) on the full-resolution guide.  Each
//                 thread owns 4 adjacent columns and a run of rows, reads I once and writes q once with
//                 128-bit streaming accesses, and caches the horizontally interpolated low-res rows.
#include <algorithm>

#include "gf_internal.cuh"

namespace gfk {

// ------------------------------------------------------------------------------------------------------
// element loads
// ------------------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float ldv(const T *p);
template <>
__device__ __forceinline__ float ldv<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldv<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <>
__device__ __forceinline__ float ldv<uint8_t>(const uint8_t *p) { return (float)__ldg(p); }

// ------------------------------------------------------------------------------------------------------
// k_subsample
// ------------------------------------------------------------------------------------------------------
struct SubJob {
    const void *src;
    float *dst;
    int planes, H, W, s;
    size_t sps, dps;  // source / destination plane strides (elements)
};
struct SubParams {
    SubJob job[2];
    int h, w, mode;
    float scale;  // result multiplier: k on the uint8 path (exact integers J = k * value), else 1
};

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_subsample(SubParams P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= P.w) return;
    int z = blockIdx.z;
    const SubJob &J = (z < P.job[0].planes) ? P.job[0] : P.job[1];
    if (z >= P.job[0].planes) z -= P.job[0].planes;
    const T *src = (const T *)J.src + (size_t)z * J.sps;
    const int H = J.H, W = J.W, s = J.s;
    float v;
    if (MODE == GF_SUB_NEAREST || s == 1) {
        const int sy = min(((2 * j + 1) * s) >> 1, H - 1);  // floor((j + 1/2) s)
        const int sx = min(((2 * i + 1) * s) >> 1, W - 1);
        v = ldv(src + (size_t)sy * W + sx);
    } else if (MODE == GF_SUB_BILINEAR) {
        // source coordinate (j + 1/2) s - 1/2 = ((2j+1)s - 1) / 2, clamped to [0, H-1]
        const int ny = (2 * j + 1) * s - 1, nx = (2 * i + 1) * s - 1;
        int y0 = ny >> 1, x0 = nx >> 1;
        float fy = (ny & 1) ? 0.5f : 0.0f, fx = (nx & 1) ? 0.5f : 0.0f;
        if (y0 >= H - 1) { y0 = H - 1; fy = 0.0f; }
        if (x0 >= W - 1) { x0 = W - 1; fx = 0.0f; }
        const int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
        const T *r0 = src + (size_t)y0 * W, *r1 = src + (size_t)y1 * W;
        const float top = (1.0f - fx) * ldv(r0 + x0) + fx * ldv(r0 + x1);
        const float bot = (1.0f - fx) * ldv(r1 + x0) + fx * ldv(r1 + x1);
        v = (1.0f - fy) * top + fy * bot;
    } else {  // box: mean of the s x s block clipped to the image
        const int ya = j * s, yb = min(ya + s, H), xa = i * s, xb = min(xa + s, W);
        float acc = 0.0f;
        for (int yy = ya; yy < yb; ++yy)
            for (int xx = xa; xx < xb; ++xx) acc += ldv(src + (size_t)yy * W + xx);
        v = acc / (float)((yb - ya) * (xb - xa));
    }
    J.dst[(size_t)z * J.dps + (size_t)j * P.w + i] = v * P.scale;
}

// ------------------------------------------------------------------------------------------------------
// k_sweep
// ------------------------------------------------------------------------------------------------------
constexpr int SW_NT = 128;  // threads per CTA
constexpr int SW_D = 4;     // rows whose loads are issued together

enum { KIND_STATS_F = 0, KIND_STATS_INT = 1, KIND_MEAN2 = 2 };

struct SweepParams {
    const void *X, *Y;  // KIND 0/1: guide I' and input p' planes; KIND 2: a and b planes
    size_t xps, yps;    // plane strides (elements)
    int CX, C;          // X planes per image (1 or C), Y planes per image (C)
    float *out0, *out1; // KIND 0/1: a, b.  KIND 2: mean of X, mean of Y.
    size_t ops;         // output plane stride
    void *stats;        // optional, KIND 0/1: 4 dense h*w planes per (n, c)
    int h, w, r, TW, TH, G;
    float eps;
    float int_scale;    // KIND 1: 255 * k (values are integers J = int_scale * I')
};

// Neumaier-compensated accumulation: s + c carries the running sum to about one rounding of its value,
// however many rows have entered and left the window.
__device__ __forceinline__ void kadd(float &s, float &c, float v)
{
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
}

template <typename T, int KIND, int COLS>
__global__ void __launch_bounds__(SW_NT) k_sweep(SweepParams P)
{
    constexpr int NQ = (KIND == KIND_MEAN2) ? 2 : 4;
    constexpr int SPANMAX = SW_NT * COLS;
    extern __shared__ float smf[];
    uint32_t *smu = reinterpret_cast<uint32_t *>(smf);

    const int tid = threadIdx.x;
    const int h = P.h, w = P.w, r = P.r;
    const int x0 = blockIdx.x * P.TW;
    const int y0 = blockIdx.y * P.TH;
    const int plane = blockIdx.z;  // n * C + c
    const int n = plane / P.C, c = plane - n * P.C;
    const T *Xp = (const T *)P.X + (size_t)(n * P.CX + (P.CX == 1 ? 0 : c)) * P.xps;
    const T *Yp = (const T *)P.Y + (size_t)plane * P.yps;
    const int y_end = min(y0 + P.TH, h);
    const int nout = min(P.TW, w - x0);
    const int xs = x0 - r;          // global column of span index 0
    const int span = nout + 2 * r;  // <= SPANMAX (host guarantees)

    // shift for the float statistics: one value of the tile, so that sums of squares stay small
    float cx = 0.0f, cy = 0.0f;
    if (KIND != KIND_STATS_INT) {
        cx = ldv(Xp + (size_t)y0 * w + x0);
        cy = ldv(Yp + (size_t)y0 * w + x0);
    }

    float V[COLS][NQ], Vc[COLS][NQ];
    uint32_t U[COLS][NQ];
#pragma unroll
    for (int k = 0; k < COLS; ++k)
#pragma unroll
        for (int q = 0; q < NQ; ++q) { V[k][q] = 0.0f; Vc[k][q] = 0.0f; U[k][q] = 0u; }

    int colx[COLS];
    bool colv[COLS];
#pragma unroll
    for (int k = 0; k < COLS; ++k) {
        const int j = tid + k * SW_NT;
        colx[k] = xs + j;
        colv[k] = (j < span) && (colx[k] >= 0) && (colx[k] < w);
    }

    const int t_begin = y0 - r, t_end = y_end + r;
    const int t_add_min = max(0, y0 - r);
    constexpr int D = (COLS > 2) ? 1 : SW_D;

    for (int tg = t_begin; tg < t_end; tg += D) {
        // ---- issue the loads of D rows entering and D rows leaving the window
        float xn[D][COLS], yn[D][COLS], xo[D][COLS], yo[D][COLS];
#pragma unroll
        for (int u = 0; u < D; ++u) {
            const int t = tg + u, to = t - 2 * r - 1;
            const bool addv = (t >= 0) && (t < h) && (t < t_end);
            const bool subv = (to >= t_add_min) && (to < h) && (t < t_end);
#pragma unroll
            for (int k = 0; k < COLS; ++k) {
                xn[u][k] = yn[u][k] = xo[u][k] = yo[u][k] = 0.0f;
                if (colv[k] && addv) {
                    xn[u][k] = ldv(Xp + (size_t)t * w + colx[k]);
                    yn[u][k] = ldv(Yp + (size_t)t * w + colx[k]);
                }
                if (colv[k] && subv) {
                    xo[u][k] = ldv(Xp + (size_t)to * w + colx[k]);
                    yo[u][k] = ldv(Yp + (size_t)to * w + colx[k]);
                }
            }
        }
        // ---- process them one row at a time
#pragma unroll
        for (int u = 0; u < D; ++u) {
            const int t = tg + u;
            if (t >= t_end) break;  // uniform over the CTA
            const int to = t - 2 * r - 1;
            const bool addv = (t >= 0) && (t < h);
            const bool subv = (to >= t_add_min) && (to < h);
#pragma unroll
            for (int k = 0; k < COLS; ++k) {
                if (KIND == KIND_STATS_INT) {
                    if (addv) {
                        const uint32_t J = (uint32_t)xn[u][k], Pv = (uint32_t)yn[u][k];
                        U[k][0] += J; U[k][1] += J * J; U[k][2] += Pv; U[k][3] += J * Pv;
                    }
                    if (subv) {
                        const uint32_t J = (uint32_t)xo[u][k], Pv = (uint32_t)yo[u][k];
                        U[k][0] -= J; U[k][1] -= J * J; U[k][2] -= Pv; U[k][3] -= J * Pv;
                    }
                } else if (KIND == KIND_STATS_F) {
                    if (addv && colv[k]) {
                        const float dx = xn[u][k] - cx, dy = yn[u][k] - cy;
                        kadd(V[k][0], Vc[k][0], dx);
                        kadd(V[k][1], Vc[k][1], dx * dx);
                        kadd(V[k][2], Vc[k][2], dy);
                        kadd(V[k][3], Vc[k][3], dx * dy);
                    }
                    if (subv && colv[k]) {
                        const float dx = xo[u][k] - cx, dy = yo[u][k] - cy;
                        kadd(V[k][0], Vc[k][0], -dx);
                        kadd(V[k][1], Vc[k][1], -(dx * dx));
                        kadd(V[k][2], Vc[k][2], -dy);
                        kadd(V[k][3], Vc[k][3], -(dx * dy));
                    }
                } else {
                    if (addv && colv[k]) {
                        kadd(V[k][0], Vc[k][0], xn[u][k] - cx);
                        kadd(V[k][1], Vc[k][1], yn[u][k] - cy);
                    }
                    if (subv && colv[k]) {
                        kadd(V[k][0], Vc[k][0], -(xo[u][k] - cx));
                        kadd(V[k][1], Vc[k][1], -(yo[u][k] - cy));
                    }
                }
            }
            const int yrow = t - r;  // output row whose vertical window is now complete
            if (yrow < y0) continue; // uniform
            // ---- stage the column sums of this row in shared memory
#pragma unroll
            for (int k = 0; k < COLS; ++k) {
                const int j = tid + k * SW_NT;
                if (j < span) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        if (KIND == KIND_STATS_INT)
                            smu[q * SPANMAX + j] = colv[k] ? U[k][q] : 0u;
                        else
                            smf[q * SPANMAX + j] = colv[k] ? (V[k][q] + Vc[k][q]) : 0.0f;
                    }
                }
            }
            __syncthreads();
            // ---- horizontal window sums: G adjacent output columns per thread, sliding
            const int ny = min(h - 1, yrow + r) - max(0, yrow - r) + 1;
            const size_t orow = (size_t)plane * P.ops + (size_t)yrow * w;
            for (int base = tid * P.G; base < nout; base += SW_NT * P.G) {
                const int xb = x0 + base;
                float Sf[NQ];
                uint32_t Su[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) { Sf[q] = 0.0f; Su[q] = 0u; }
                const int lo = max(0, xb - r), hi = min(w - 1, xb + r);
                for (int xc = lo; xc <= hi; ++xc) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        if (KIND == KIND_STATS_INT) Su[q] += smu[q * SPANMAX + xc - xs];
                        else Sf[q] += smf[q * SPANMAX + xc - xs];
                    }
                }
                const int gmax = min(P.G, nout - base);
                for (int g = 0; g < gmax; ++g) {
                    const int xg = xb + g;
                    if (g > 0) {
                        const int ad = xg + r, rm = xg - r - 1;
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            if (KIND == KIND_STATS_INT) {
                                if (ad < w) Su[q] += smu[q * SPANMAX + ad - xs];
                                if (rm >= 0) Su[q] -= smu[q * SPANMAX + rm - xs];
                            } else {
                                if (ad < w) Sf[q] += smf[q * SPANMAX + ad - xs];
                                if (rm >= 0) Sf[q] -= smf[q * SPANMAX + rm - xs];
                            }
                        }
                    }
                    const int nx = min(w - 1, xg + r) - max(0, xg - r) + 1;
                    const int cnt = nx * ny;
                    const size_t oi = orow + xg;
                    if (KIND == KIND_STATS_F) {
                        const float inv = 1.0f / (float)cnt;
                        const float mI = Sf[0] * inv, mp = Sf[2] * inv;   // shifted means
                        const float eII = Sf[1] * inv, eIp = Sf[3] * inv;
                        const float var = fmaxf(eII - mI * mI, 0.0f);     // Algorithm 2: var_I
                        const float cov = eIp - mI * mp;                  // Algorithm 2: cov_Ip
                        const float a = cov / (var + P.eps);              // Eq. (2)
                        const float b = (mp + cy) - a * (mI + cx);        // Eq. (3)
                        P.out0[oi] = a;
                        P.out1[oi] = b;
                        if (P.stats) {
                            float *st = (float *)P.stats + (size_t)plane * 4 * h * w + (size_t)yrow * w + xg;
                            const size_t ps = (size_t)h * w;
                            st[0] = mI + cx;
                            st[ps] = eII + cx * (2.0f * mI + cx);
                            st[2 * ps] = mp + cy;
                            st[3 * ps] = eIp + cx * mp + cy * mI + cx * cy;
                        }
                    } else if (KIND == KIND_STATS_INT) {
                        const long long nn = cnt;
                        // exact integer numerators of var and cov (times n^2 (255k)^2)
                        const long long vnum = nn * (long long)Su[1] - (long long)Su[0] * (long long)Su[0];
                        const long long cnum = nn * (long long)Su[3] - (long long)Su[0] * (long long)Su[2];
                        const float den = (float)vnum + P.eps * ((float)nn * (float)nn) * (P.int_scale * P.int_scale);
                        const float a = (float)cnum / den;                                        // Eq. (2)
                        const float b = ((float)Su[2] - a * (float)Su[0]) / ((float)cnt * P.int_scale); // Eq. (3)
                        P.out0[oi] = a;
                        P.out1[oi] = b;
                        if (P.stats) {
                            uint32_t *st = (uint32_t *)P.stats + (size_t)plane * 4 * h * w + (size_t)yrow * w + xg;
                            const size_t ps = (size_t)h * w;
                            st[0] = Su[0]; st[ps] = Su[1]; st[2 * ps] = Su[2]; st[3 * ps] = Su[3];
                        }
                    } else {
                        const float inv = 1.0f / (float)cnt;
                        P.out0[oi] = Sf[0] * inv + cx;
                        P.out1[oi] = Sf[1] * inv + cy;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------------------------------------
// k_upsample_output
// ------------------------------------------------------------------------------------------------------
constexpr int UP_NT = 128;

struct UpParams {
    const void *I;
    const float *ma, *mb;
    void *q;
    int C, CI, H, W, h, w, s, R, CG;  // CG: channel groups per image
    size_t lps;                       // low-res plane stride
};

// Upsampling taps along one axis: full-res index X samples position (X + 1/2)/s - 1/2 = (2X + 1 - s)/(2s),
// clamped to [0, n-1].  Integer arithmetic keeps the taps exact.
__device__ __forceinline__ void up_taps(int X, int s, int n, int &i0, int &i1, float &f)
{
    const int num = 2 * X + 1 - s, den = 2 * s;
    if (num <= 0) { i0 = 0; i1 = 0; f = 0.0f; return; }
    const int qt = num / den, rem = num - qt * den;
    if (qt >= n - 1) { i0 = n - 1; i1 = n - 1; f = 0.0f; return; }
    i0 = qt; i1 = qt + 1; f = (float)rem / (float)den;
}

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
        for (int k = 0; k < 4; ++k) v[k] = (float)((t >> (8 * k)) & 0xffu) / 255.0f;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (k < valid) ? (float)p[k] / 255.0f : 0.0f;
    }
}

template <typename T>
__device__ __forceinline__ void st4(T *p, bool vec, int valid, const float v[4]);
template <>
__device__ __forceinline__ void st4<float>(float *p, bool vec, int valid, const float v[4])
{
    if (vec) {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < valid) __stcs(p + k, v[k]);
    }
}
template <>
__device__ __forceinline__ void st4<__half>(__half *p, bool vec, int valid, const float v[4])
{
    if (vec) {
        const __half2 lo = __floats2half2_rn(v[0], v[1]), hi = __floats2half2_rn(v[2], v[3]);
        uint2 t;
        t.x = *reinterpret_cast<const uint32_t *>(&lo);
        t.y = *reinterpret_cast<const uint32_t *>(&hi);
        __stcs(reinterpret_cast<uint2 *>(p), t);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < valid) p[k] = __float2half_rn(v[k]);
    }
}

template <typename TI, typename TQ, int CC, bool VEC, bool S1>
__global__ void __launch_bounds__(UP_NT) k_upsample_output(UpParams P)
{
    const int gx = blockIdx.x * UP_NT + threadIdx.x;
    const int X0 = gx * 4;
    if (X0 >= P.W) return;
    const int valid = min(4, P.W - X0);
    const bool vec = VEC && (valid == 4);
    const int Yb = blockIdx.y * P.R, Ye = min(Yb + P.R, P.H);
    const int n = blockIdx.z / P.CG, c0 = (blockIdx.z - n * P.CG) * CC;
    const size_t HW = (size_t)P.H * P.W;

    const float *MA[CC], *MB[CC];
    TQ *Q[CC];
    const TI *Ig[CC];
#pragma unroll
    for (int cc = 0; cc < CC; ++cc) {
        const int c = min(c0 + cc, P.C - 1);
        MA[cc] = P.ma + (size_t)(n * P.C + c) * P.lps;
        MB[cc] = P.mb + (size_t)(n * P.C + c) * P.lps;
        Q[cc] = (TQ *)P.q + (size_t)(n * P.C + c) * HW;
        Ig[cc] = (const TI *)P.I + (size_t)(n * P.CI + (P.CI == 1 ? 0 : c)) * HW;
    }
    const int ncc = min(CC, P.C - c0);

    if constexpr (S1) {
        // s = 1: no resampling, mean_a and mean_b are already full resolution
        for (int Y = Yb; Y < Ye; ++Y) {
            float iv[4];
            if (P.CI == 1) ld4<TI>(Ig[0] + (size_t)Y * P.W + X0, vec, valid, iv);
#pragma unroll
            for (int cc = 0; cc < CC; ++cc) {
                if (cc >= ncc) break;
                if (P.CI != 1) ld4<TI>(Ig[cc] + (size_t)Y * P.W + X0, vec, valid, iv);
                float A[4], B[4], out[4];
                ld4<float>(MA[cc] + (size_t)Y * P.W + X0, vec, valid, A);
                ld4<float>(MB[cc] + (size_t)Y * P.W + X0, vec, valid, B);
#pragma unroll
                for (int k = 0; k < 4; ++k) out[k] = fmaf(A[k], iv[k], B[k]);
                st4<TQ>(Q[cc] + (size_t)Y * P.W + X0, vec, valid, out);
            }
        }
    } else {
    int xa[4], xb[4];
    float fx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) up_taps(min(X0 + k, P.W - 1), P.s, P.w, xa[k], xb[k], fx[k]);

    // horizontally interpolated low-res rows: slot 0 = upper tap row, slot 1 = lower tap row
    float ha[CC][2][4], hb[CC][2][4];
    int cur0 = -1, cur1 = -1;
    auto load_row = [&](int yy, int slot) {
#pragma unroll
        for (int cc = 0; cc < CC; ++cc) {
            const float *ra = MA[cc] + (size_t)yy * P.w, *rb = MB[cc] + (size_t)yy * P.w;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float a0 = __ldg(ra + xa[k]), a1 = __ldg(ra + xb[k]);
                const float b0 = __ldg(rb + xa[k]), b1 = __ldg(rb + xb[k]);
                ha[cc][slot][k] = fmaf(fx[k], a1 - a0, a0);
                hb[cc][slot][k] = fmaf(fx[k], b1 - b0, b0);
            }
        }
    };

    for (int Y = Yb; Y < Ye; ++Y) {
        int ya, yb;
        float fy;
        up_taps(Y, P.s, P.h, ya, yb, fy);
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
        float iv[4];
        if (P.CI == 1) ld4<TI>(Ig[0] + (size_t)Y * P.W + X0, vec, valid, iv);
#pragma unroll
        for (int cc = 0; cc < CC; ++cc) {
            if (cc >= ncc) break;
            if (P.CI != 1) ld4<TI>(Ig[cc] + (size_t)Y * P.W + X0, vec, valid, iv);
            float out[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float A = fmaf(fy, ha[cc][1][k] - ha[cc][0][k], ha[cc][0][k]);  // upsampled mean_a
                const float B = fmaf(fy, hb[cc][1][k] - hb[cc][0][k], hb[cc][0][k]);  // upsampled mean_b
                out[k] = fmaf(A, iv[k], B);                                            // Eq. (4)
            }
            st4<TQ>(Q[cc] + (size_t)Y * P.W + X0, vec, valid, out);
        }
    }
    }
}

// ------------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------------
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
    case GF_SUB_NEAREST: k_subsample<T, GF_SUB_NEAREST><<<grid, 256, 0, st>>>(sp); break;
    case GF_SUB_BILINEAR: k_subsample<T, GF_SUB_BILINEAR><<<grid, 256, 0, st>>>(sp); break;
    default: k_subsample<T, GF_SUB_BOX><<<grid, 256, 0, st>>>(sp); break;
    }
}

int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Tile geometry of a sweep launch.
void sweep_geometry(int h, int w, int r, int planes, int &cols, int &TW, int &TH, int &G, dim3 &grid)
{
    cols = (32 + 2 * r <= SW_NT * 2) ? 2 : 8;
    const int spanmax = SW_NT * cols;
    TW = std::min(128, spanmax - 2 * r);
    TW = std::min(TW, ((w + 31) / 32) * 32);
    G = (r <= 1) ? 1 : std::min(16, next_pow2(r));
    const int strips = (w + TW - 1) / TW;
    const int target = 152 * 8;
    int chunks = std::max(1, (target + strips * planes - 1) / (strips * planes));
    TH = (h + chunks - 1) / chunks;
    TH = std::max(TH, std::max(8, 2 * r));
    TH = std::min(TH, h);
    chunks = (h + TH - 1) / TH;
    grid = dim3(strips, chunks, planes);
}

template <typename T, int KIND>
cudaError_t launch_sweep_t(SweepParams sp, int planes, cudaStream_t st)
{
    int cols, TW, TH, G;
    dim3 grid;
    sweep_geometry(sp.h, sp.w, sp.r, planes, cols, TW, TH, G, grid);
    sp.TW = TW; sp.TH = TH; sp.G = G;
    const int nq = (KIND == KIND_MEAN2) ? 2 : 4;
    const size_t smem = (size_t)nq * SW_NT * cols * sizeof(float);
    if (cols == 2)
        k_sweep<T, KIND, 2><<<grid, SW_NT, smem, st>>>(sp);
    else
        k_sweep<T, KIND, 8><<<grid, SW_NT, smem, st>>>(sp);
    return cudaGetLastError();
}

template <typename TI, typename TQ>
void launch_up_t(const UpParams &up, int N, int CC, bool vec, bool s1, cudaStream_t st)
{
    const int groups = (up.W + 3) / 4;
    dim3 grid((groups + UP_NT - 1) / UP_NT, (up.H + up.R - 1) / up.R, N * up.CG);
#define GF_UP(cc, v, one) k_upsample_output<TI, TQ, cc, v, one><<<grid, UP_NT, 0, st>>>(up)
    if (CC == 3) {
        if (vec) { if (s1) GF_UP(3, true, true); else GF_UP(3, true, false); }
        else { if (s1) GF_UP(3, false, true); else GF_UP(3, false, false); }
    } else {
        if (vec) { if (s1) GF_UP(1, true, true); else GF_UP(1, true, false); }
        else { if (s1) GF_UP(1, false, true); else GF_UP(1, false, false); }
    }
#undef GF_UP
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

cudaError_t launch_forward(const FwdPlan &P, cudaStream_t st)
{
    StageTimer tm{P.events, st};
    cudaError_t err;
    const int planesNC = P.N * P.C;

    // ---- Algorithm 2, first step: subsample I and p (skipped at s = 1)
    const void *Xsrc = P.I, *Ysrc = P.p;
    int src_dt = P.dt_in;
    if (P.s > 1 || P.p_lowres) {
        SubParams sp;
        sp.h = P.h; sp.w = P.w; sp.mode = P.mode;
        sp.scale = 1.0f;
        // uint8 path: carry the subsampled values as exact integers J = k * (value in 1/255 units)
        if (P.int_stats) sp.scale = P.int_scale / 255.0f;
        int nz = 0;
        if (P.s > 1) {
            sp.job[0] = SubJob{P.I, P.Il, P.N * P.CI, P.H, P.W, P.s, (size_t)P.H * P.W, P.lps};
            nz = P.N * P.CI;
            if (!P.p_lowres) {
                sp.job[1] = SubJob{P.p, P.pl, planesNC, P.H, P.W, P.s, (size_t)P.H * P.W, P.lps};
                nz += planesNC;
            } else {
                sp.job[1] = SubJob{P.p, P.pl, planesNC, P.h, P.w, 1, (size_t)P.h * P.w, P.lps};
                nz += planesNC;
            }
        } else {
            // s = 1 with a low-res p is the same grid: nothing to resample
            sp.job[0] = SubJob{P.p, P.pl, 0, P.h, P.w, 1, (size_t)P.h * P.w, P.lps};
            sp.job[1] = sp.job[0];
            nz = 0;
        }
        if (nz > 0) {
            dim3 grid((P.w + 255) / 256, P.h, nz);
            tm.before();
            if (P.dt_in == F32) launch_sub_t<float>(sp, grid, st);
            else if (P.dt_in == F16) launch_sub_t<__half>(sp, grid, st);
            else launch_sub_t<uint8_t>(sp, grid, st);
            tm.after();
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            Xsrc = P.Il;
            Ysrc = P.pl;
            src_dt = F32;
        }
    }

    // ---- Algorithm 2, box statistics + var/cov + coefficients a, b (Eq. 2-3)
    {
        SweepParams sp{};
        sp.X = Xsrc; sp.Y = Ysrc;
        const bool lowres_src = (src_dt == F32 && (P.s > 1));
        sp.xps = lowres_src ? P.lps : (size_t)P.h * P.w;
        sp.yps = lowres_src ? P.lps : (size_t)P.h * P.w;
        sp.CX = P.CI; sp.C = P.C;
        sp.out0 = P.a; sp.out1 = P.b; sp.ops = P.lps;
        sp.stats = P.stats;
        sp.h = P.h; sp.w = P.w; sp.r = P.r_low; sp.eps = P.eps;
        sp.int_scale = P.int_scale;
        tm.before();
        if (P.int_stats) {
            if (src_dt == F32) err = launch_sweep_t<float, KIND_STATS_INT>(sp, planesNC, st);
            else err = launch_sweep_t<uint8_t, KIND_STATS_INT>(sp, planesNC, st);
        } else {
            if (src_dt == F32) err = launch_sweep_t<float, KIND_STATS_F>(sp, planesNC, st);
            else err = launch_sweep_t<__half, KIND_STATS_F>(sp, planesNC, st);
        }
        tm.after();
        if (err != cudaSuccess) return err;
    }

    // ---- Algorithm 2, box means of a and b
    {
        SweepParams sp{};
        sp.X = P.a; sp.Y = P.b;
        sp.xps = P.lps; sp.yps = P.lps;
        sp.CX = P.C; sp.C = P.C;
        sp.out0 = P.ma; sp.out1 = P.mb; sp.ops = P.lps;
        sp.h = P.h; sp.w = P.w; sp.r = P.r_low;
        tm.before();
        err = launch_sweep_t<float, KIND_MEAN2>(sp, planesNC, st);
        tm.after();
        if (err != cudaSuccess) return err;
    }

    // ---- Algorithm 2, bilinear upsample of mean_a, mean_b fused with q = mean_a .* I + mean_b
    {
        UpParams up;
        up.I = P.I; up.ma = P.ma; up.mb = P.mb; up.q = P.q;
        up.C = P.C; up.CI = P.CI; up.H = P.H; up.W = P.W; up.h = P.h; up.w = P.w; up.s = P.s;
        up.lps = P.lps;
        const int CC = (P.C % 3 == 0) ? 3 : 1;
        up.CG = P.C / CC;
        const bool s1 = (P.s == 1);
        up.R = s1 ? 8 : 4 * P.s;
        // 4-wide vector accesses need every row of every plane to start on the vector boundary
        const bool vec = (P.W % 4 == 0) && aligned16(P.I) && aligned16(P.q) &&
                         (!s1 || ((P.lps % 4 == 0) && aligned16(P.ma) && aligned16(P.mb)));
        tm.before();
        if (P.dt_in == F32) {
            if (P.dt_out == F32) launch_up_t<float, float>(up, P.N, CC, vec, s1, st);
            else launch_up_t<float, __half>(up, P.N, CC, vec, s1, st);
        } else if (P.dt_in == F16) {
            if (P.dt_out == F32) launch_up_t<__half, float>(up, P.N, CC, vec, s1, st);
            else launch_up_t<__half, __half>(up, P.N, CC, vec, s1, st);
        } else {
            if (P.dt_out == F32) launch_up_t<uint8_t, float>(up, P.N, CC, vec, s1, st);
            else launch_up_t<uint8_t, __half>(up, P.N, CC, vec, s1, st);
        }
        tm.after();
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace gfk
