// gf_device.cuh -- device helpers shared by the forward and backward kernels: typed loads, the
// resampling tap arithmetic of the library's conventions (see gf.h), and cp.async.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gf.h"

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

}  // namespace gfk
