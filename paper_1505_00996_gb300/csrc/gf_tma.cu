// gf_tma.cu -- the s = 4, 8 upsample-and-output kernel with the guide streamed by the Tensor Memory
// Accelerator (Algorithm 2, last two steps: bilinear upsampling of mean_a, mean_b and q = mean_a I + mean_b).
//
// Same work split and arithmetic as k_upsample_output_s4x (one channel of one 512-pixel band per CTA, rows
// walked in the s-row runs that share a pair of low-res tap rows, 4 pixels per consumer thread), but the
// rows of I reach shared memory as 2-D TMA tiles instead of per-thread copies:
//   warp 4 (producer)  one lane issues, for each quad of 4 rows, two cp.async.bulk.tensor loads of a
//                      256-column x 4-row box into a ring stage, arming the stage's "full" mbarrier with
//                      the bytes to expect; before reusing a stage it waits on the stage's "empty" barrier;
//   warps 0-3          wait on "full", read their 4 pixels of the 4 rows, write q (128-bit streaming
//                      stores), and release the stage with one arrival per warp on "empty".
// Out-of-image rows and columns of a box read as zeros and are never used.  Every wait is bounded: after
// FaultSink::limit failed polls a thread reports FAULT_OUTPUT_TMA (the call's fault word and the device's
// sticky word, gf_kernel_faults) and leaves its loop; the producer then drains the loads it issued
// (bounded again) before the CTA exits.  If that drain gives up too, a load may still be landing in the
// CTA's shared memory when it exits; the call's fault word says so and the call's output is not valid.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <map>
#include <mutex>

#include "gf_device.cuh"
#include "gf_internal.cuh"

namespace gfk {

__device__ unsigned g_wait_faults;  // sticky OR of the FAULT_* bits of every call on this device

namespace {

constexpr int TO_CONS = 128;            // consumer threads (4 warps), 4 pixels each
constexpr int TO_NT = TO_CONS + 32;     // plus one producer warp
constexpr int TO_BAND = 4 * TO_CONS;    // 512 columns per CTA
constexpr int TO_BOX_X = 256;           // TMA box: 256 columns x 4 rows (a box dimension is at most 256)
constexpr int TO_NST = 6;               // ring stages (quads of rows in flight; 6 measured best with two images in flight)

struct TmaOutParams {
    const float *ma, *mb;
    void *q;
    int C, CI, H, W, h, w, R, LRmax, LCmax, Yw0, Yw1;
    size_t lps, fps;
    float detail;
    FaultSink fault;
    int skip_first;  // test hook (gf_opts.test_wait_fault): the producer never issues its first stage
};

template <typename TI, typename TQ, int S>
__global__ void __launch_bounds__(TO_NT, 4) k_output_tma(const __grid_constant__ CUtensorMap tmI, TmaOutParams P)
{
    extern __shared__ __align__(128) unsigned char sm[];
    pdl_wait();  // launched with programmatic serialization: mean_a, mean_b are complete here
    constexpr int ES = (int)sizeof(TI);
    constexpr int BOX_BYTES = TO_BOX_X * 4 * ES;  // one 256 x 4 box
    constexpr int STAGE = 2 * BOX_BYTES;          // 512 columns x 4 rows
    const int nb = P.R / S, jb = blockIdx.y * nb;
    const int c = blockIdx.x % P.C, band = blockIdx.x / P.C, n = blockIdx.z;
    const int Xb = band * TO_BAND;
    const int Yb = max(jb * S, P.Yw0), Ye = min(min(jb * S + P.R, P.H), P.Yw1);
    if (Yb >= Ye) return;  // uniform over the CTA
    const int ly0 = jb - 1, lx0 = Xb / S - 1;
    const int LR = P.LRmax, LC = P.LCmax, tile = LR * LC;
    float *tap = reinterpret_cast<float *>(sm + TO_NST * STAGE);  // [2][LR][LC]
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(tap + 2 * tile);  // full[NST], empty[NST]
    const unsigned full0 = smem_u32(bars), empty0 = smem_u32(bars + TO_NST);
    constexpr int QPR = S / 4;
    // quads (4-row groups of the runs) this CTA uses: those starting above Ye
    const int nquads_all = (nb + 1) * QPR;
    int nquads = 0;
    while (nquads < nquads_all && S * (jb - 1 + nquads / QPR) + S / 2 + 4 * (nquads % QPR) < Ye) ++nquads;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TO_NST; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, TO_CONS / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();

    // waits for data and for free stages (shortened by the test hook); the drain keeps the full limit
    FaultSink fw = P.fault;
    if (P.skip_first) fw.limit = INJECT_LIMIT;
    if (threadIdx.x >= TO_CONS) {  // ---- producer warp
        if (threadIdx.x == TO_CONS) {
            const int plane = n * P.CI + (P.CI == 1 ? 0 : c);
            int issued = 0;
            int first = 0;
            if (P.skip_first) {  // test hook: stage 0 is never filled, so the consumers' first wait runs out
                first = 1;
            }
            for (int u = first; u < nquads; ++u) {
                const int st = u % TO_NST;
                if (u >= TO_NST && !mbar_wait(empty0 + 8 * st, ((u / TO_NST) - 1) & 1, fw, FAULT_OUTPUT_TMA))
                    break;
                const unsigned fb = full0 + 8 * st;
                mbar_expect_tx(fb, STAGE);
                const int y = S * (jb - 1 + u / QPR) + S / 2 + 4 * (u % QPR);  // may be < 0: zero fill
#pragma unroll
                for (int k = 0; k < 2; ++k) tma_load_3d(sm + st * STAGE + k * BOX_BYTES, &tmI, Xb + k * TO_BOX_X, y, plane, fb);
                issued = u + 1;
            }
            // drain: every load issued has landed before the CTA may exit (the consumers waited on all of
            // them unless a wait gave up)
            for (int u = max(first, issued - TO_NST); u < issued; ++u)
                mbar_wait(full0 + 8 * (u % TO_NST), (u / TO_NST) & 1, P.fault, FAULT_OUTPUT_TMA);
        }
        return;
    }

    // ---- consumers: the tap tile (cp.async with clamped coordinates), then the rows
    {
        const int c0 = threadIdx.x, c1 = threadIdx.x + TO_CONS;
        const int g0 = min(max(lx0 + c0, 0), P.w - 1), g1 = min(max(lx0 + c1, 0), P.w - 1);
        const float *pa = P.ma + (size_t)(n * P.C + c) * P.lps, *pb = P.mb + (size_t)(n * P.C + c) * P.lps;
        for (int row = 0; row < LR; ++row) {
            const size_t go = (size_t)min(max(ly0 + row, 0), P.h - 1) * P.w;
            float *da = tap + row * LC, *db = da + tile;
            if (c0 < LC) { cp_async4(da + c0, pa + go + g0); cp_async4(db + c0, pb + go + g0); }
            if (c1 < LC) { cp_async4(da + c1, pa + go + g1); cp_async4(db + c1, pb + go + g1); }
        }
        cp_async_wait_all();
        asm volatile("bar.sync 1, %0;\n" ::"r"(TO_CONS) : "memory");  // consumers only
    }
    const int X0 = Xb + threadIdx.x * 4;
    const bool active = X0 < P.W;  // threads past the image still take part in the barriers
    const int ti = X0 / S - lx0;
    const int g = (S == 8) ? ((X0 >> 2) & 1) : 0;
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
    TQ *Qp = (TQ *)P.q + (size_t)(n * P.C + c) * P.fps + X0;
    // the thread's 4 pixels inside a stage: box threadIdx / 64, column 4 (threadIdx % 64)
    const int box = threadIdx.x / (TO_BOX_X / 4), bcol = 4 * (threadIdx.x % (TO_BOX_X / 4));
    float lo[2][4], d[2][4];
    if (active) hrow(0, lo);
    const int lane = threadIdx.x & 31;
    for (int u = 0; u < nquads; ++u) {
        const int st = u % TO_NST;
        if (!mbar_wait(full0 + 8 * st, (u / TO_NST) & 1, fw, FAULT_OUTPUT_TMA)) break;
        const int t = u / QPR, sub = u % QPR;
        const int Yq = S * (jb - 1 + t) + S / 2 + 4 * sub;
        if (active) {
            if (sub == 0) {
                if (t > 0) {
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
            const float fy0 = (S == 4) ? 0.125f : (sub ? 0.5625f : 0.0625f);
            const unsigned char *sbase = sm + st * STAGE + box * BOX_BYTES + bcol * ES;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int Y = Yq + k;
                if (Y < Yb || Y >= Ye) continue;
                float iv[4];
                ld4_shared<TI>(sbase + k * TO_BOX_X * ES, iv);
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
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * st);
    }
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;
using CtxGetCurrentFn = PFN_cuCtxGetCurrent_v4000;

template <typename F>
F driver_fn(const char *name, int version)
{
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        p = nullptr;
    return reinterpret_cast<F>(p);
}

EncodeFn encode_fn()
{
    static EncodeFn fn = driver_fn<EncodeFn>("cuTensorMapEncodeTiled", 12000);
    return fn;
}

}  // namespace

bool encode_tmap_3d(CUtensorMap *map, int dt, const void *base, int w, int h, int planes, size_t plane_stride,
                    int box_w, int box_h)
{
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const size_t es = dtype_size(dt);
    const CUtensorMapDataType dtype = dt == F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                      : (dt == F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
    const cuuint64_t dims[3] = {(cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)w * es, (cuuint64_t)plane_stride * es};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1}, estr[3] = {1, 1, 1};
    return enc(map, dtype, 3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The rows a subsample at ratio S reads, as a 4-D FP32 tensor (column, row within the S-row block, block,
// plane): dims (W, S, h, planes) for planes of H = S h rows of W floats, plane_stride floats apart.  A box is
// box_w columns of nph consecutive rows of one block: the two rows a bilinear sample reads (nph = 2), or the
// one of a nearest sample.
bool encode_tmap_sampled_rows(CUtensorMap *map, const float *base, int W, int S, int h, int planes,
                              size_t plane_stride, int box_w, int nph)
{
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)W, (cuuint64_t)S, (cuuint64_t)h, (cuuint64_t)planes};
    const cuuint64_t strides[3] = {(cuuint64_t)W * 4, (cuuint64_t)S * W * 4, (cuuint64_t)plane_stride * 4};
    const cuuint32_t box[4] = {(cuuint32_t)box_w, (cuuint32_t)nph, 1, 1}, estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The sticky word's device address, looked up once per CUDA context (a context made after cudaDeviceReset
// gets its own lookup, so no stale address is used).
unsigned *sticky_fault_word()
{
    static CtxGetCurrentFn get_ctx = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent", 4000);
    static std::mutex mu;
    static std::map<void *, unsigned *> cache;
    CUcontext ctx = nullptr;
    if (!get_ctx) return nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) {
        void *probe = nullptr;  // the runtime makes the device's primary context current for this lookup
        if (cudaGetSymbolAddress(&probe, g_wait_faults) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find((void *)ctx);
    if (it != cache.end()) return it->second;
    void *addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_wait_faults) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cache[(void *)ctx] = (unsigned *)addr;
    return (unsigned *)addr;
}

bool output_tma_ok(const void *I, int dt_in, int W, size_t fps)
{
    const size_t es = dtype_size(dt_in);
    return encode_fn() != nullptr && ((uintptr_t)I % 16 == 0) && ((size_t)W * es) % 16 == 0 && (fps * es) % 16 == 0 &&
           getenv("GF_NO_TMA") == nullptr;
}

cudaError_t launch_output_tma(const void *I, const float *ma, const float *mb, void *q, int N, int C, int CI, int H,
                              int W, int h, int w, int s, size_t lps, size_t fps, int Yw0, int Yw1, float detail,
                              int dt_in, int dt_out, const FaultSink &fault, cudaStream_t st)
{
    const size_t es = dtype_size(dt_in);
    CUtensorMap map;
    if (!encode_tmap_3d(&map, dt_in, I, W, H, N * CI, fps, TO_BOX_X, 4)) return cudaErrorInvalidValue;
    TmaOutParams P;
    P.ma = ma; P.mb = mb; P.q = q;
    P.C = C; P.CI = CI; P.H = H; P.W = W; P.h = h; P.w = w;
    P.R = 8 * s;
    P.LRmax = P.R / s + 2;
    P.LCmax = ((TO_BAND / s + 2) + 1) & ~1;
    P.Yw0 = Yw0; P.Yw1 = Yw1;
    P.lps = lps; P.fps = fps;
    P.detail = detail;
    P.fault = fault;
    P.skip_first = fault.inject ? 1 : 0;
    const int bands = (W + TO_BAND - 1) / TO_BAND;
    dim3 grid(bands * C, (H + P.R - 1) / P.R, N);
    const size_t smem = (size_t)TO_NST * 2 * TO_BOX_X * 4 * es + (size_t)2 * P.LRmax * P.LCmax * sizeof(float) +
                        2 * TO_NST * sizeof(unsigned long long);
    cudaError_t e;
#define GF_TO(TI, TQ, SS)                                                                  \
    do {                                                                                   \
        if ((e = opt_in_smem(k_output_tma<TI, TQ, SS>, smem)) != cudaSuccess) return e;    \
        if ((e = launch_pdl(k_output_tma<TI, TQ, SS>, grid, dim3(TO_NT), smem, st, map, P)) != cudaSuccess) \
            return e;                                                                      \
    } while (0)
#define GF_TO_S(TI, TQ) do { if (s == 4) GF_TO(TI, TQ, 4); else GF_TO(TI, TQ, 8); } while (0)
    if (dt_in == F32) {
        if (dt_out == F32) GF_TO_S(float, float); else GF_TO_S(float, __half);
    } else if (dt_in == F16) {
        if (dt_out == F32) GF_TO_S(__half, float); else GF_TO_S(__half, __half);
    } else {
        if (dt_out == F32) GF_TO_S(uint8_t, float); else GF_TO_S(uint8_t, __half);
    }
#undef GF_TO_S
#undef GF_TO
    return cudaGetLastError();
}

cudaError_t read_kernel_faults(unsigned *flags, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(flags, g_wait_faults, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_wait_faults, &zero, sizeof(unsigned));
    }
    return e;
}

}  // namespace gfk
