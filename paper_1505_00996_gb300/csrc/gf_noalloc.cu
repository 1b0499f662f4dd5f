// gf_noalloc.cu -- gf_filter_noalloc: the forward filter for callers that cannot allocate device memory.
//
// Some callers have no way to call cudaMalloc: a plugin that runs inside a host application which owns
// every device allocation through its own pool or budget, code that must not take the allocator's locks
// or trigger its implicit synchronisation on a latency-critical path, or a C caller that has no context
// object to own an arena.  For them this file keeps the filter's scratch (the low-res planes I', p', a,
// b, mean_a, mean_b) in one fixed array that the CUDA module itself provides on every device that loads
// the library.  The caller still passes I, p and q; nothing here allocates or frees device memory.
#include <mutex>
#include <string>

#include "gf_internal.cuh"

namespace {

// Largest scratch one call may use: 64 MiB (a 12 MP, 3-channel call at s = 4 needs about 48 MB).
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

// The scratch itself.  Every GPU that loads this library holds it until the process exits.  In host code
// `g_noalloc_scratch` names a host-side stand-in, not device memory: host code must only pass the address
// that cudaGetSymbolAddress returns for the current device (see scratch_for_current_device).
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
gf_status scratch_for_current_device(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        gf_set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return GF_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        gf_set_error("gf_filter_noalloc supports device ordinals below 64");
        return GF_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            gf_set_error(std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
            return GF_ECUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
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
    st = scratch_for_current_device(&base);
    if (st != GF_OK) return st;
    char *ws = (char *)base;

    // Every low-res plane is written by the kernel that produces it before any kernel reads it, so no part
    // of the shared scratch has to start at zero.
    const gfk::FwdPlan P = gfk::make_plan(R, L, I, p, q, ws, opts);
    cudaError_t e = gfk::launch_forward(P, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        gf_set_error(std::string("kernel launch in gf_filter_noalloc: ") + cudaGetErrorString(e));
        return GF_ECUDA;
    }
    return GF_OK;
}
