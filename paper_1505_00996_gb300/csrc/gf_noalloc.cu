// gf_noalloc.cu -- gf_filter_noalloc: the forward filter for callers that cannot allocate device memory.
//
// Some callers have no way to call cudaMalloc: a plugin that runs inside a host application which owns
// every device allocation through its own pool or budget, code that must not take the allocator's locks
// or trigger its implicit synchronisation on a latency-critical path, or a C caller that has no context
// object to own an arena.  For them this file keeps the filter's scratch (the low-res planes I', p', a,
// b, mean_a, mean_b) in one fixed array that the CUDA module itself provides on every device that loads
// the library.  The caller still passes I, p and q; nothing here allocates or frees device memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <string>

#include "gf_internal.cuh"

namespace {

// Largest scratch one call may use: 64 MiB (a 12 MP, 3-channel call at s = 4 needs about 48 MB).
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

// The scratch itself.  Every GPU that loads this library holds it until the process exits.  In host code
// `g_noalloc_scratch` names a host-side stand-in, not device memory: host code must only pass the address
// that cudaGetSymbolAddress returns for the current device (see scratch_for_current_context).
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
std::map<CUcontext, void *> g_scratch_ptr;  // the array's device address in each CUDA context

// The current CUDA context (the device's primary context once the runtime has made it current).
CUcontext current_context()
{
    static PFN_cuCtxGetCurrent_v4000 get_ctx = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    }();
    CUcontext ctx = nullptr;
    if (get_ctx && get_ctx(&ctx) == CUDA_SUCCESS) return ctx;
    return nullptr;
}

// Device address of the scratch in the current context, looked up once per context: a context made after
// cudaDeviceReset (which invalidates the old address) gets a lookup of its own.
gf_status scratch_for_current_context(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        gf_set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return GF_ECUDA;
    }
    CUcontext ctx = current_context();
    if (!ctx) {
        void *probe = nullptr;  // the runtime makes the device's primary context current for this lookup
        e = cudaGetSymbolAddress(&probe, g_noalloc_scratch);
        ctx = current_context();
        if (e != cudaSuccess || !ctx) {
            gf_set_error("gf_filter_noalloc: no CUDA context is current on device " + std::to_string(dev));
            return GF_ECUDA;
        }
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    auto it = g_scratch_ptr.find(ctx);
    if (it == g_scratch_ptr.end()) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            gf_set_error(std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
            return GF_ECUDA;
        }
        it = g_scratch_ptr.emplace(ctx, ptr).first;
    }
    *out = it->second;
    return GF_OK;
}

}  // namespace

extern "C" gf_status gf_filter_noalloc(const void *I, const void *p, void *q, int H, int W, int C, int r, float eps,
                                       int s, gf_subsample_mode mode, const gf_opts *opts, void *cuda_stream)
{
    gfk::NvtxRange range("gf_filter_noalloc");
    if (!I || !p || !q) {
        gf_set_error("I, p and q must be device pointers");
        return GF_EINVAL;
    }
    if (opts && (opts->workspace || opts->saved_forward)) {
        gf_set_error("gf_filter_noalloc uses its static scratch; opts->workspace and saved_forward must be unset");
        return GF_EINVAL;
    }
    gfk::Resolved R;
    gf_status st = gfk::resolve(H, W, C, r, eps, s, (int)mode, opts, R);
    if (st != GF_OK) return st;
    const gfk::Layout L = gfk::layout_of(R, opts);
    if (L.total > kNoAllocScratchBytes) {
        gf_set_error("gf_filter_noalloc: this call needs " + std::to_string(L.total) +
                     " bytes of scratch; the static scratch holds " + std::to_string(kNoAllocScratchBytes) +
                     " bytes (use gf_filter with a context or a caller workspace)");
        return GF_EINVAL;
    }
    void *base = nullptr;
    st = scratch_for_current_context(&base);
    if (st != GF_OK) return st;
    char *ws = (char *)base;

    // Every low-res plane is written by the kernel that produces it before any kernel reads it; the call's
    // fault word, the one part of the scratch that must start at zero, is zeroed by the call itself.
    const gfk::FwdPlan P = gfk::make_plan(R, L, I, p, q, ws, opts);
    cudaError_t e = gfk::launch_forward(P, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        gf_set_error(std::string("kernel launch in gf_filter_noalloc: ") + cudaGetErrorString(e));
        return GF_ECUDA;
    }
    return GF_OK;
}
