// gf_device.cuh -- device helpers shared by the forward and backward kernels: typed loads, the
// resampling tap arithmetic of the library's conventions (see gf.h), and cp.async.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gf.h"
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

// 4-byte asynchronous global -> shared copy (sm_80+ cp.async): many can be in flight per thread, and
// they complete without holding registers.
__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gmem_src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// 16-byte form (L2 only, both addresses 16-byte aligned), and per-thread group bookkeeping.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
// 8-byte (FP16) and 4-byte (uint8) forms of a ring copy of 4 pixels.
template <typename T>
__device__ __forceinline__ void ld_async_small(void *smem_dst, const T *gmem_src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    if (sizeof(T) == 2)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ------------------------------------------------------------------------------------------------------
// mbarrier and TMA (cp.async.bulk.tensor) helpers.  Every wait is bounded: after FaultSink::limit failed
// polls the waiting thread ORs `bit` into the call's fault word (and the device's sticky word) and gives
// up, so a kernel whose data never arrives returns instead of hanging.
// ------------------------------------------------------------------------------------------------------

__device__ __forceinline__ void report_fault(const FaultSink &f, unsigned bit)
{
    if (f.call) atomicOr(f.call, bit);
    if (f.sticky) atomicOr(f.sticky, bit);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Programmatic dependent launch.  A kernel launched with the programmatic stream serialization attribute
// (launch_pdl) may be scheduled while the kernel before it in the stream is still finishing; pdl_wait returns
// once that kernel has completed and its memory operations are visible, so such a kernel calls it before it
// touches global memory (without the attribute it returns at once).  pdl_trigger lets the next kernel be
// scheduled once every CTA of this one has called it or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false (and the fault reported) when it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, const FaultSink &f, unsigned bit)
{
    for (unsigned it = 0; it < f.limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    report_fault(f, bit);
    return false;
}
// One 3-D tiled TMA load (box at element coordinates x, y, z; x * element size a multiple of 16 bytes)
// into shared memory, completing on `bar` with its byte count.
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int x, int y, int z, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// One 4-D tiled TMA load (box at element coordinates x, y, z, v; x * element size a multiple of 16 bytes).
__device__ __forceinline__ void tma_load_4d(void *dst, const void *tmap, int x, int y, int z, int v, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x), "r"(y), "r"(z), "r"(v), "r"(bar)
        : "memory");
}

// Upsampling taps along one axis at ratio s = sn / sd: full-res index X samples position
// (X + 1/2)/s - 1/2 = ((2X + 1) sd - sn)/(2 sn), clamped to [0, n-1].  Integer arithmetic keeps the taps exact.
__device__ __forceinline__ void up_taps_q(int X, int sn, int sd, int n, int &i0, int &i1, float &f)
{
    const int num = (2 * X + 1) * sd - sn, den = 2 * sn;
    if (num <= 0) { i0 = 0; i1 = 0; f = 0.0f; return; }
    const int qt = num / den, rem = num - qt * den;
    if (qt >= n - 1) { i0 = n - 1; i1 = n - 1; f = 0.0f; return; }
    i0 = qt; i1 = qt + 1; f = (float)rem / (float)den;
}
__device__ __forceinline__ void up_taps(int X, int s, int n, int &i0, int &i1, float &f) { up_taps_q(X, s, 1, n, i0, i1, f); }

// floor(a / b) for b > 0 and any sign of a.
__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Subsampling taps along one axis for low-res index j (Algorithm 2 first step, gf.h conventions): the
// full-res positions t0, t1 that the sample reads and the weight f of t1 (nearest: t0 = t1, f = 0).  Box mode
// is handled by the callers (it averages a whole block).
__device__ __forceinline__ void sub_taps(int j, int s, int n, int mode, int &t0, int &t1, float &f)
{
    if (mode == GF_SUB_NEAREST || s == 1) {
        t0 = t1 = min(((2 * j + 1) * s) >> 1, n - 1);
        f = 0.0f;
        return;
    }
    const int nn = (2 * j + 1) * s - 1;  // twice the source coordinate
    t0 = nn >> 1;
    f = (nn & 1) ? 0.5f : 0.0f;
    if (t0 >= n - 1) { t0 = n - 1; f = 0.0f; }
    t1 = min(t0 + 1, n - 1);
}

// Packed FP32 pairs (sm_100+ add/sub/mul .f32x2): one instruction for both lanes of a float2.
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 r;
    asm("{ .reg .b64 ra, rb, rc; mov.b64 ra, {%2, %3}; mov.b64 rb, {%4, %5}; add.rn.f32x2 rc, ra, rb; mov.b64 {%0, %1}, rc; }"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{ .reg .b64 ra, rb, rc; mov.b64 ra, {%2, %3}; mov.b64 rb, {%4, %5}; sub.rn.f32x2 rc, ra, rb; mov.b64 {%0, %1}, rc; }"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 r;
    asm("{ .reg .b64 ra, rb, rc; mov.b64 ra, {%2, %3}; mov.b64 rb, {%4, %5}; mul.rn.f32x2 rc, ra, rb; mov.b64 {%0, %1}, rc; }"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// The source taps of a bilinear sample at ratio sn / sd: position ((2j + 1) sn - sd) / (2 sd), clamped.
__device__ __forceinline__ void sub_bilinear_taps(int j, int sn, int sd, int n, int &t0, float &f)
{
    const int num = (2 * j + 1) * sn - sd, den = 2 * sd;
    t0 = num / den;  // num >= 0 since sn >= sd
    f = (float)(num - t0 * den) / (float)den;
    if (t0 >= n - 1) { t0 = n - 1; f = 0.0f; }
}

template <typename T, int MODE>
__device__ __forceinline__ float subsample_one(const T *src, int H, int W, int s, int sn, int sd, int j, int i)
{
    if (MODE == GF_SUB_NEAREST || s == 1) {
        const int sy = min(((2 * j + 1) * sn) / (2 * sd), H - 1);  // floor((j + 1/2) s)
        const int sx = min(((2 * i + 1) * sn) / (2 * sd), W - 1);
        return ldv(src + (size_t)sy * W + sx);
    } else if (MODE == GF_SUB_BILINEAR) {
        // source coordinate (j + 1/2) s - 1/2, clamped to [0, H-1]
        int y0, x0;
        float fy, fx;
        sub_bilinear_taps(j, sn, sd, H, y0, fy);
        sub_bilinear_taps(i, sn, sd, W, x0, fx);
        const int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
        const T *r0 = src + (size_t)y0 * W, *r1 = src + (size_t)y1 * W;
        const float top = (1.0f - fx) * ldv(r0 + x0) + fx * ldv(r0 + x1);
        const float bot = (1.0f - fx) * ldv(r1 + x0) + fx * ldv(r1 + x1);
        return (1.0f - fy) * top + fy * bot;
    } else {  // box: mean of the s x s block clipped to the image
        const int ya = j * s, yb = min(ya + s, H), xa = i * s, xb = min(xa + s, W);
        float acc = 0.0f;
        for (int yy = ya; yy < yb; ++yy)
            for (int xx = xa; xx < xb; ++xx) acc += ldv(src + (size_t)yy * W + xx);
        return acc / (float)((yb - ya) * (xb - xa));
    }
}


// Antialiased bilinear sample (triangle filter of half-width s = sn / sd, renormalised over the taps inside
// the image) of low-res pixel (j, i), computed directly: for one-off samples (the fused kernel); the
// subsample kernels walk rows instead.
template <typename T>
__device__ __forceinline__ float subsample_aa_one(const T *src, int H, int W, int sn, int sd, int j, int i)
{
    auto wnum = [&](int t, int k) { return 2 * sn - abs((2 * t + 1) * sd - (2 * k + 1) * sn); };
    auto lo_of = [&](int k) { return max(0, floor_div((2 * k + 1) * sn - 2 * sn - sd, 2 * sd) + 1); };
    auto hi_of = [&](int k, int n) { return min(n - 1, -floor_div(-((2 * k + 1) * sn + 2 * sn - sd), 2 * sd) - 1); };
    const int ya = lo_of(j), yb = hi_of(j, H), xa = lo_of(i), xb = hi_of(i, W);
    float acc = 0.0f;
    int ny = 0, nx = 0;
    for (int x = xa; x <= xb; ++x) nx += wnum(x, i);
    for (int y = ya; y <= yb; ++y) {
        const int wy = wnum(y, j);
        ny += wy;
        const T *row = src + (size_t)y * W;
        float hs = 0.0f;
        for (int x = xa; x <= xb; ++x) hs = fmaf((float)wnum(x, i), ldv(row + x), hs);
        acc = fmaf((float)wy, hs, acc);
    }
    return acc / ((float)nx * (float)ny);
}

// Detail-enhancement epilogue (the application of the paper's Fig. 2): q + k (I - q), the guide's detail
// I - q scaled by k on top of the filtered image.  k = 0 leaves q as it is.
__device__ __forceinline__ void detail_epilogue(float k, const float iv[4], float out[4])
{
    if (k != 0.0f) {
#pragma unroll
        for (int x = 0; x < 4; ++x) out[x] = fmaf(k, iv[x] - out[x], out[x]);
    }
}

// A uint8 sample as a value on [0, 1]: b / 255, formed as the exact float of b times the rounded reciprocal
// of 255 -- within one unit in the last place of the quotient, without a division per pixel.
__device__ __forceinline__ float u8_unit(uint32_t b) { return (float)b * (1.0f / 255.0f); }

// 4 pixels of I from the thread's shared ring slot, as floats.
template <typename T>
__device__ __forceinline__ void ld4_shared(const void *p, float v[4]);
template <>
__device__ __forceinline__ void ld4_shared<float>(const void *p, float v[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld4_shared<__half>(const void *p, float v[4])
{
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <>
__device__ __forceinline__ void ld4_shared<uint8_t>(const void *p, float v[4])
{
    const uint32_t t = *reinterpret_cast<const uint32_t *>(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = u8_unit((t >> (8 * k)) & 0xffu);
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

}  // namespace gfk
