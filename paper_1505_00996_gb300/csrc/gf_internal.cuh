// gf_internal.cuh -- types and launcher declarations shared by the libgf translation units.
// Nothing here is part of the public ABI (include/gf.h is).
#pragma once

#include <utility>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gf.h"

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define GF_HAVE_NVTX 1
#endif

namespace gfk {

// A named NVTX range around one entry-point call or serving launch, for timeline profilers; without a
// profiler attached the push and pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name)
    {
#ifdef GF_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~NvtxRange()
    {
#ifdef GF_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Fault bits of the kernels with bounded waits (FaultSink).
enum : unsigned { FAULT_OUTPUT_TMA = 1u, FAULT_BOX_TMA = 2u };

// Where a kernel with bounded waits reports a wait that gave up: the fault word of its call (in the call's
// scratch, cleared when the call starts) and the device's sticky word (gf_kernel_faults).  Either may be
// NULL.  `limit` is the number of polls before a wait gives up.  `inject` (tests of the timeout path only,
// gf_opts.test_wait_fault) makes the TMA output kernel's producer leave its first stage unfilled and gives
// that kernel's waits for data and for free stages INJECT_LIMIT polls, so that its consumers' first wait runs
// out; waits for copies already issued (the producer's drain, the box kernels' tile loads) keep `limit`, so
// no CTA leaves while a copy into its shared memory may still be landing.
constexpr unsigned WAIT_LIMIT = 1u << 20;
constexpr unsigned INJECT_LIMIT = 256;
struct FaultSink {
    unsigned *call = nullptr;
    unsigned *sticky = nullptr;
    unsigned limit = WAIT_LIMIT;
    unsigned inject = 0;
};

// Element type of an input plane.
enum DType { F32 = GF_F32, F16 = GF_F16, U8 = GF_U8 };

// Largest low-res radius r' the box kernels support (their shared tile grows with r').
constexpr int MAX_LOWRES_RADIUS = 128;

inline size_t dtype_size(int dt) { return dt == F32 ? 4 : (dt == F16 ? 2 : 1); }

// Low-res planes in the workspace start on 256-byte boundaries.
inline size_t plane_stride_f32(size_t elems) { return (elems + 63) & ~size_t(63); }

// Everything one forward call needs, resolved on the host.
struct FwdPlan {
    int N, C, CI, H, W, h, w, s, r_low, mode;
    int sn = 1, sd = 1;  // the ratio as sn / sd; s = sn when sd = 1, else ceil(sn / sd) (sizes launches only)
    float eps;
    int dt_in, dt_out;
    bool p_lowres;
    // inputs / outputs (device)
    const void *I, *p;
    void *q;
    // low-res planes (FP32, plane stride `lps` elements)
    size_t lps;
    float *Il, *pl;      // subsampled guide (N*CI planes) and input (N*C planes); NULL when not needed
    float *a, *b;        // N*C planes each
    float *ma, *mb;      // N*C planes each
    void *stats;         // optional N*C*4 planes (dense h*w each)
    bool int_stats;      // exact integer window sums (uint8 input)
    float int_scale;     // 255 * k: J = int_scale * I' (uint8 path)
    cudaEvent_t *events; // 2*GF_MAX_STAGES or NULL
    float detail = 0.0f; // detail gain of the output epilogue (0: plain q)
    // colour guide (CI = 3 used jointly): the scratch planes of gf_color.cu -- products A, B; their means;
    // the coefficient planes (a_r, a_b), (a_g, b); their means.  K = 5 + 2C planes per image in each of the
    // first four, 2C in each of the last four.
    bool color = false;
    float *col[8] = {};
    bool fused = false;  // the whole filter in one kernel (gf_fused.cu)
    size_t fps = 0;      // plane stride (elements) of the full-res I, p and q (H * W of the whole image)
    size_t lpin = 0;     // plane stride of a low-res p given by the caller (h * w of the whole image)
    int Yw0 = 0, Yw1 = 0;  // output rows written, [Yw0, Yw1) of the H rows the plan covers
    bool lowres_out = false;   // a, b, mean_a or mean_b are caller outputs (no fusion may skip them)
    FaultSink fault;           // where kernels with bounded waits report a wait that gave up
    bool clear_fault = true;   // the call zeroes its fault word first (false: keep accumulating into it)
    bool skip_output = false;  // stop after the low-res stages (the backward's forward recomputation)
    bool need_lowres = false;  // keep I', p' in the workspace (no fused subsample); the backward reads them
};

// Everything one backward call needs (gf_backward.cu).  `fwd` describes the forward recomputation; it must
// write the window statistics (fwd.stats), a, mean_a and the low-res I', p' into the workspace.
struct BwdPlan {
    FwdPlan fwd;
    bool fwd_saved = false;  // the workspace already holds fwd's low-res planes (gf_opts.saved_forward)
    const float *dq;      // dL/dq, N x C x H x W
    float *dI, *dp;       // outputs: N x CI x H x W; like p (full or low resolution)
    float *d_eps;         // device scalar or NULL
    float *dma, *dmb;     // U^T(g .* I), U^T(g): N x C planes of stride fwd.lps
    float *gq[4];         // d mean_I, d corr_I, d corr_Ip, d mean_p
    float *dIl, *dpl;     // dI', dp'
    float *eps_partial;   // bwd_eps_partials() floats
};
size_t bwd_eps_partials(int N, int C, int h, int w);
cudaError_t launch_backward(const BwdPlan &B, cudaStream_t stream);

// Serving loop (gf_serve.cu).
struct Server;
double now_seconds();
Server *server_create(int device, size_t budget);
void server_destroy(Server *s);
gf_status server_config(Server *s, int slots, size_t queue_limit);
gf_status server_submit(Server *s, const gf_request *req, uint64_t *ticket);
gf_status server_poll(Server *s, uint64_t ticket, int64_t timeout_us, gf_result *out);
gf_status server_cancel(Server *s, uint64_t ticket);
gf_status server_stats(Server *s, gf_serve_stats *out);
gf_status server_pause(Server *s, int paused);
gf_status server_graphs(Server *s, int enable);
gf_status server_queue(Server *s, int enable);

// A forward call's arguments, checked and resolved on the host (gf_api.cu).
struct Resolved {
    int N, C, CI, H, W, h, w, s, r_low, mode, dt_in, dt_out;
    int sn, sd;  // the ratio s = sn / sd (sd = 1 for an integer ratio; then s = sn)
    bool p_lowres, dense_lowres, int_stats;
    float eps, int_scale;
    float detail;  // detail gain (gf_opts.detail_gain)
    bool color;    // colour guide (gf_opts.color_guide)
    bool fused;    // one fused kernel (gf_opts.fused, resolved)
    bool saved_forward;  // gf_opts.saved_forward: the low-res planes stay in the backward's workspace
    size_t lps;  // low-res plane stride in floats
    // Row band (gf_opts.row_begin / row_end): H and h above are those of the band of complete s-row blocks
    // that is filtered; it starts at full-res row row0 of the whole image, and the output rows written are
    // [Yw0, Yw1) of the band.  Without a row range: row0 = 0, Yw0 = 0, Yw1 = H.
    int row0, Yw0, Yw1;
    size_t fps, lpin;  // plane strides of the whole image's full-res planes and of a caller's low-res p
};
// Check every argument of a forward call and derive its geometry (no CUDA call).  On error the thread's
// gf_last_error() message is set.
gf_status resolve(int H, int W, int C, int r, float eps, int s, int mode, const gf_opts *o, Resolved &R);

// Byte offsets of a forward call's low-res planes in its scratch.
struct Layout {
    size_t off_Il, off_pl, off_a, off_b, off_ma, off_mb, off_fault, total;
    size_t off_col[8];  // colour-guide planes (FwdPlan::col)
};
Layout layout_of(const Resolved &R, const gf_opts *o);

// The forward plan of a call: geometry from R, the caller's buffers (advanced to the first row of the
// filtered band), scratch planes carved from ws as L says, optional outputs and events from opts.
FwdPlan make_plan(const Resolved &R, const Layout &L, const void *I, const void *p, void *q, char *ws,
                  const gf_opts *opts);

// Opt kernel `func` in to `smem` bytes of dynamic shared memory on the current device when that is above the
// 48 KB default.  Thread-safe; the attribute is set once per kernel, device and larger size.
cudaError_t opt_in_smem(const void *func, size_t smem);
// Launch with the programmatic stream serialization attribute: the kernel (which calls pdl_wait before any
// global memory access) may be scheduled while the previous kernel in the stream finishes.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
template <typename F>
cudaError_t opt_in_smem(F *func, size_t smem) { return opt_in_smem(reinterpret_cast<const void *>(func), smem); }

// Kernels one forward call launches for these arguments (host-side, assuming 16-byte aligned buffers).
int forward_kernel_count(const Resolved &R);
// Whether an s = 1 call takes the box means of a and b fused with the output (the identity upsample lets
// each output pixel use its own means): FP32 input, FP32 or FP16 output, rows a multiple of 4 pixels, a
// radius the TMA box kernels take, no low-res outputs.  Alignment and TMA availability are checked at launch.
bool s1_means_output_form(const Resolved &R);
// Fault word of a forward call: ws + off_fault, plus the device's sticky word; the test hook of
// gf_opts.test_wait_fault.
FaultSink call_fault_sink(char *ws, const Layout &L, const gf_opts *opts);

// The TMA-fed s = 4, 8 output kernel (gf_tma.cu): whether it takes these buffers, its launch, and the
// bounded-wait fault bits its kernels record.
bool output_tma_ok(const void *I, int dt_in, int W, size_t fps);
cudaError_t launch_output_tma(const void *I, const float *ma, const float *mb, void *q, int N, int C, int CI, int H,
                              int W, int h, int w, int s, size_t lps, size_t fps, int Yw0, int Yw1, float detail,
                              int dt_in, int dt_out, const FaultSink &fault, cudaStream_t st);
cudaError_t read_kernel_faults(unsigned *flags, bool clear);
// Device address of the current device's sticky fault word (NULL if it cannot be had).
unsigned *sticky_fault_word();
// A 3-D tiled tensor map over `planes` planes of h rows of w elements of type dt (F32, F16, U8), row pitch
// w elements, plane pitch plane_stride elements, box box_w x box_h x 1, zeros outside; false when the
// encoder is unavailable or rejects the arguments (the caller then takes a path without TMA).
bool encode_tmap_3d(CUtensorMap *map, int dt, const void *base, int w, int h, int planes, size_t plane_stride,
                    int box_w, int box_h);

// The TMA-fed box kernels (gf_box.cu): Algorithm 2's box statistics + coefficients, the box means of a and b,
// and (s = 1) the box means fused with the output.  FP32 planes whose rows are 16-byte aligned, r' <= 16.
enum { BOX_JOB_STATS = 0, BOX_JOB_MEANS = 2, BOX_JOB_MEANS_OUTPUT = 3 };
struct BoxTmaJob {
    int kind;
    const float *X, *Y;  // STATS: guide planes (N * CX) and input planes (N * C); MEANS*: a and b (N * C each)
    size_t xps, yps;     // plane strides (elements)
    int N, C, CX, h, w, r;
    float eps;
    float *out0, *out1;  // STATS: a, b; MEANS: mean_a, mean_b
    size_t ops;
    float *stats;        // STATS, optional: the FP32 window means of the backward (4 dense h*w planes per plane)
    // MEANS_OUTPUT: the full-res guide I (CI planes per image, FP32, plane stride fps), the output q (dt_out),
    // the rows [Yw0, Yw1) written, the detail gain
    const float *I;
    void *q;
    size_t fps;
    int CI, Yw0, Yw1, dt_out;
    float detail;
    FaultSink fault;
};
bool box_tma_supported(const BoxTmaJob &J);
cudaError_t launch_box_tma(const BoxTmaJob &J, cudaStream_t st);
// The column-strip box kernels (gf_strip.cu) for radii 1..16: whether they take the job (FP32 planes, rows a
// multiple of 4 outputs, 16-byte aligned outputs, no window statistics kept), and their launch.
bool strip_box_supported(const BoxTmaJob &J);
cudaError_t launch_strip_box(const BoxTmaJob &J, cudaStream_t st);
// 4-D tensor map of the full-res rows a subsample at ratio S reads (gf_tma.cu): dims (W, S, h, planes), box
// box_w columns x nph rows of one S-row block.  False when the encoder is unavailable or rejects it.
bool encode_tmap_sampled_rows(CUtensorMap *map, const float *base, int W, int S, int h, int planes,
                              size_t plane_stride, int box_w, int nph);
// Algorithm 2's first two steps in one kernel (gf_strip.cu): the nearest or bilinear subsample of a gray guide
// and three channels of p per group, fed by TMA, and the box statistics + coefficients a, b of the samples.
// FP32 full-res planes (plane stride fps), H = s h and W = s w, s = 4 or 8; a, b as for BOX_JOB_STATS.
struct SubStripJob {
    const float *I, *p;  // N guide planes, N * C input planes
    size_t fps;
    int N, C, H, W, h, w, s, mode, r;
    float eps;
    float *a, *b;
    size_t ops;
    unsigned *clear_word;  // the call's fault word, zeroed by the kernel (the first of the chain), or NULL
    FaultSink fault;
};
// Whether the geometry takes the fused form (no pointer checked); and whether these buffers do.
bool strip_sub_geometry(int C, int CI, int H, int W, int h, int w, int s, int sd, int mode, int r_low, int dt_in,
                        bool p_lowres);
bool strip_sub_supported(const SubStripJob &J);
cudaError_t launch_strip_sub(const SubStripJob &J, cudaStream_t st);

// The single-kernel form (gf_fused.cu): whether it can run these arguments, and its launch.
bool fused_supported(const Resolved &R, bool intermediates);
cudaError_t launch_fused(const FwdPlan &P, cudaStream_t st);
// The tile-queue form of the single kernel: one launch for the tiles of n <= FUSED_QUEUE_MAX fused plans with
// the same input and output storage types and subsample mode (each plan's output exactly its own launch's).
constexpr int FUSED_QUEUE_MAX = 16;
cudaError_t launch_fused_queue(const FwdPlan *plans, int n, cudaStream_t st);

// Colour-guide stages (gf_color.cu).
cudaError_t launch_color_products(const FwdPlan &P, cudaStream_t st);
cudaError_t launch_color_coef(const FwdPlan &P, cudaStream_t st);
cudaError_t launch_color_output(const FwdPlan &P, cudaStream_t st);

// Launch the forward chain on `stream`.  Returns cudaSuccess or the first launch error.
cudaError_t launch_forward(const FwdPlan &P, cudaStream_t stream);

}  // namespace gfk

// Thread-local error message used by every entry point.
void gf_set_error(const std::string &msg);
