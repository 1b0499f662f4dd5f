// gf_api.cu -- the extern "C" entry points of libgf.so declared in include/gf.h: argument checking,
// the context and its scratch arena, and the host-buffer wrapper.  All arithmetic runs in the kernels of
// gf_forward.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstdint>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "gf_internal.cuh"

static thread_local std::string g_last_error;

void gf_set_error(const std::string &msg) { g_last_error = msg; }

struct gf_ctx {
    int device = 0;
    size_t budget = 0;
    std::mutex mu;
    void *arena = nullptr;  // scratch for calls without a caller workspace
    size_t arena_bytes = 0;
    void *stage = nullptr;  // device copies of host buffers (gf_filter_host)
    size_t stage_bytes = 0;
    // gf_filter_host's strip pipeline: one call at a time per context, two copy streams of its own
    std::mutex host_mu;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    std::vector<cudaEvent_t> host_ev;
    gfk::Server *server = nullptr;  // serving loop, created with the context, started on first submit
};

namespace {

gf_status fail(gf_status st, const std::string &msg)
{
    gf_set_error(msg);
    return st;
}

gf_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(GF_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// Grow a device buffer to at least `need` bytes.  Growing waits for the device so that no queued kernel
// still reads the old buffer.
gf_status grow(void **buf, size_t *have, size_t need, const char *what)
{
    if (*have >= need) return GF_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize before growing scratch");
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    size_t bytes = need + need / 8;
    e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GF_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes for " + what +
                                   " failed: " + cudaGetErrorString(e));
    }
    *have = bytes;
    return GF_OK;
}

int lowres_radius_q(int r, int sn, int sd)
{
    if (sn == sd) return r;
    int rl = (int)((2LL * r * sd + sn) / (2LL * sn));  // r/s rounded half up
    if (r >= 1 && rl < 1) rl = 1;
    return rl;
}
int lowres_radius(int r, int s) { return lowres_radius_q(r, s, 1); }

int gcd_int(int a, int b)
{
    while (b) { const int t = a % b; a = b; b = t; }
    return a;
}

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

}  // namespace

namespace gfk {

// Check every argument of a forward call and derive its geometry.  No CUDA call.
gf_status resolve(int H, int W, int C, int r, float eps, int s, int mode, const gf_opts *o, Resolved &R)
{
    gf_opts def;
    gf_opts_init(&def);
    if (!o) o = &def;
    if (H < 1 || W < 1 || C < 1) return fail(GF_EINVAL, "H, W and C must be >= 1");
    if (s < 1) return fail(GF_EINVAL, "subsampling ratio s must be >= 1");
    if (r < 0) return fail(GF_EINVAL, "radius r must be >= 0");
    if (!(eps >= 0.0f) || !isfinite(eps)) return fail(GF_EINVAL, "eps must be finite and >= 0");
    if (mode < GF_SUB_NEAREST || mode > GF_SUB_BILINEAR_AA) return fail(GF_EINVAL, "unknown subsample mode");
    if (o->batch < 1) return fail(GF_EINVAL, "batch must be >= 1");
    const int CI = o->guide_channels == 0 ? 1 : o->guide_channels;
    R.color = o->color_guide != 0;
    if (R.color) {
        if (CI != 3) return fail(GF_EINVAL, "a colour guide has guide_channels = 3");
        if (o->dtype_in == GF_U8) return fail(GF_EINVAL, "a colour guide takes FP32 or FP16 input");
        if (o->a_out || o->b_out || o->mean_a_out || o->mean_b_out || o->stats_out)
            return fail(GF_EINVAL, "a colour guide does not produce the low-res intermediates");
        if (o->detail_gain != 0.0f && C != 3) return fail(GF_EINVAL, "detail_gain with a colour guide needs C = 3");
    } else if (CI != 1 && CI != C) {
        return fail(GF_EINVAL, "guide_channels must be 1 or C");
    }
    if (o->dtype_in < GF_F32 || o->dtype_in > GF_U8) return fail(GF_EINVAL, "unknown dtype_in");
    if (o->dtype_out != GF_F32 && o->dtype_out != GF_F16) return fail(GF_EINVAL, "dtype_out must be GF_F32 or GF_F16");
    if ((long long)H * W > (1LL << 31) - 1) return fail(GF_EINVAL, "H * W must be < 2^31");
    // the ratio: the integer s, or s_num / s_den in lowest terms (R13)
    int sn = s, sd = 1;
    if (o->s_num != 0 || o->s_den != 0) {
        if (o->s_num < 1 || o->s_den < 1 || o->s_num < o->s_den)
            return fail(GF_EINVAL, "s_num / s_den must be a ratio >= 1");
        const int g = gcd_int(o->s_num, o->s_den);
        sn = o->s_num / g;
        sd = o->s_den / g;
    }
    if (sd != 1) {
        if (mode == GF_SUB_BOX) return fail(GF_EINVAL, "box subsampling needs an integer ratio");
        if (o->dtype_in == GF_U8) return fail(GF_EINVAL, "uint8 input needs an integer ratio");
        if (R.color) return fail(GF_EINVAL, "the colour guide needs an integer ratio");
        if (o->row_begin != 0 || o->row_end != 0) return fail(GF_EINVAL, "a row range needs an integer ratio");
        // the kernels form (2X + 1) sd - sn and (2j + 3) sn in 32-bit integers
        if ((2LL * std::max(H, W) + 1) * sd + sn > INT32_MAX || (2LL * std::max(H, W) + 3) * sn > INT32_MAX)
            return fail(GF_EINVAL, "s_num, s_den too large for the image size");
    }
    R.N = o->batch; R.C = C; R.CI = CI; R.H = H; R.W = W; R.mode = mode;
    R.sn = sn;
    R.sd = sd;
    R.s = (sn + sd - 1) / sd;  // = s for an integer ratio; sizes launches otherwise
    R.h = (int)(((long long)H * sd + sn - 1) / sn);
    R.w = (int)(((long long)W * sd + sn - 1) / sn);
    R.r_low = o->r_low >= 0 ? o->r_low : lowres_radius_q(r, sn, sd);
    if (R.r_low > gfk::MAX_LOWRES_RADIUS) return fail(GF_EINVAL, "low-res radius r' > 128 is not supported");
    R.eps = eps;
    if (!isfinite(o->detail_gain)) return fail(GF_EINVAL, "detail_gain must be finite");
    R.detail = o->detail_gain;
    R.dt_in = o->dtype_in;
    R.dt_out = o->dtype_out;
    R.saved_forward = o->saved_forward != 0;
    R.p_lowres = o->p_lowres != 0;
    R.int_stats = (o->dtype_in == GF_U8);
    R.int_scale = 255.0f;
    if (R.int_stats) {
        if ((mode == GF_SUB_BOX || mode == GF_SUB_BILINEAR_AA) && s > 1)
            return fail(GF_EINVAL, "uint8 input supports nearest or bilinear subsampling");
        if (R.p_lowres) return fail(GF_EINVAL, "uint8 input does not support a low-res p");
        const int k = (mode == GF_SUB_BILINEAR && s > 1 && (s % 2 == 0)) ? 4 : 1;
        R.int_scale = 255.0f * (float)k;
        // window sums of J*J and J*P must fit in 32 bits: (2r'+1)^2 (255k)^2 <= 2^32 - 1
        const double side = 2.0 * R.r_low + 1.0, top = 255.0 * k;
        if (side * side * top * top > 4294967295.0)
            return fail(GF_EINVAL, "uint8 input: (2r'+1)^2 * (255k)^2 exceeds 32-bit window sums");
    }
    R.row0 = 0;
    R.Yw0 = 0;
    R.Yw1 = H;
    R.fps = (size_t)H * W;
    R.lpin = (size_t)R.h * R.w;
    if (o->row_begin != 0 || o->row_end != 0) {
        if (o->row_begin < 0 || o->row_end > H || o->row_begin >= o->row_end)
            return fail(GF_EINVAL, "row range must satisfy 0 <= row_begin < row_end <= H");
        if (o->a_out || o->b_out || o->mean_a_out || o->mean_b_out || o->stats_out)
            return fail(GF_EINVAL, "a row range does not produce the low-res intermediates");
        // Output row Y samples low-res rows floor((Y + 1/2)/s - 1/2) and the one below (clamped, R7); those
        // box means need a, b within r' of them, which need statistics within r' more.  Keeping 2 r' low-res
        // rows beyond the tap rows keeps every window that could end at the band's cut out of the result.
        auto tap_row = [&](int Y) { return (int)std::floor((2.0 * Y + 1.0 - s) / (2.0 * s)); };
        const int lo = std::max(0, tap_row(o->row_begin));
        const int hi = std::min(R.h - 1, tap_row(o->row_end - 1) + (s > 1 ? 1 : 0));
        // An antialiased subsample also reads s/2 rows into the neighbouring blocks, so the band's edge
        // low-res rows are themselves inexact: one more row of margin on each side.
        const int m = 2 * R.r_low + ((mode == GF_SUB_BILINEAR_AA && s > 1) ? 1 : 0);
        const int c0 = std::max(0, lo - m), c1 = std::min(R.h, hi + m + 1);
        R.row0 = s * c0;
        R.H = std::min(H, s * c1) - R.row0;  // complete s-row blocks, or the image's own last rows
        R.h = c1 - c0;
        R.Yw0 = o->row_begin - R.row0;
        R.Yw1 = o->row_end - R.row0;
    }
    if (R.h > 65535) return fail(GF_EINVAL, "low-res height ceil(H/s) must be <= 65535");
    // the single fused kernel: forced, automatic for small images, or off
    {
        const bool inter = o->a_out || o->b_out || o->mean_a_out || o->mean_b_out || o->stats_out;
        const bool ok = gfk::fused_supported(R, inter);
        if (o->fused > 0 && !ok)
            return fail(GF_EINVAL, "the fused kernel does not take these arguments (colour guide, uint8, "
                                   "intermediate outputs or too large a radius)");
        // automatic: subsampled calls up to GF_FUSED_AUTO_PIXELS pixel-channels, where the single kernel was
        // measured faster than the chain (at s = 1 its direct window sums lose).  Its cost grows with the halo
        // each tile recomputes, so the pixel-channels are weighed by (1 + r'/4)^2 against 2.1 GF_FUSED_AUTO_PIXELS
        // (measured crossings: r' = 2 between 896^2 and 1024^2 single-channel images, r' = 4 near 600 x 800)
        const double pc = (double)R.N * C * H * W, grow = 1.0 + R.r_low / 4.0;
        R.fused = ok && (o->fused > 0 || (o->fused == 0 && R.s > 1 && pc <= GF_FUSED_AUTO_PIXELS &&
                                          pc * grow * grow <= 2.1 * GF_FUSED_AUTO_PIXELS));
    }
    const long long planes = (long long)R.N * (R.CI + C);
    if (planes > 65535) return fail(GF_EINVAL, "batch * (guide channels + C) must be <= 65535");
    R.dense_lowres = (o->a_out || o->b_out || o->mean_a_out || o->mean_b_out);
    R.lps = R.dense_lowres ? (size_t)R.h * R.w : gfk::plane_stride_f32((size_t)R.h * R.w);
    return GF_OK;
}

FwdPlan make_plan(const Resolved &R, const Layout &L, const void *I, const void *p, void *q, char *ws,
                  const gf_opts *opts)
{
    FwdPlan P;
    P.N = R.N; P.C = R.C; P.CI = R.CI; P.H = R.H; P.W = R.W; P.h = R.h; P.w = R.w; P.s = R.s;
    P.r_low = R.r_low; P.mode = R.mode; P.eps = R.eps; P.dt_in = R.dt_in; P.dt_out = R.dt_out;
    P.sn = R.sn; P.sd = R.sd;
    P.p_lowres = R.p_lowres;
    const size_t row_off = (size_t)R.row0 * R.W;  // first element of the filtered band in each plane
    P.I = (const char *)I + row_off * dtype_size(R.dt_in);
    P.p = (const char *)p + (R.p_lowres ? (size_t)(R.row0 / R.s) * R.w : row_off) * dtype_size(R.dt_in);
    P.q = q ? (void *)((char *)q + row_off * dtype_size(R.dt_out)) : nullptr;
    P.fps = R.fps;
    P.lpin = R.lpin;
    P.Yw0 = R.Yw0;
    P.Yw1 = R.Yw1;
    P.lps = R.lps;
    const bool sub = R.s > 1 || R.p_lowres || R.color;
    P.Il = sub ? (float *)(ws + L.off_Il) : nullptr;
    P.pl = sub ? (float *)(ws + L.off_pl) : nullptr;
    P.color = R.color;
    for (int k = 0; k < 8; ++k) P.col[k] = R.color ? (float *)(ws + L.off_col[k]) : nullptr;
    P.a = (opts && opts->a_out) ? opts->a_out : (float *)(ws + L.off_a);
    P.b = (opts && opts->b_out) ? opts->b_out : (float *)(ws + L.off_b);
    P.ma = (opts && opts->mean_a_out) ? opts->mean_a_out : (float *)(ws + L.off_ma);
    P.mb = (opts && opts->mean_b_out) ? opts->mean_b_out : (float *)(ws + L.off_mb);
    P.stats = opts ? opts->stats_out : nullptr;
    P.int_stats = R.int_stats;
    P.int_scale = R.int_scale;
    P.events = (opts && opts->kernel_events) ? (cudaEvent_t *)opts->kernel_events : nullptr;
    P.detail = R.detail;
    P.fused = R.fused;
    P.lowres_out = R.dense_lowres;
    P.fault = call_fault_sink(ws, L, opts);
    return P;
}

FaultSink call_fault_sink(char *ws, const Layout &L, const gf_opts *opts)
{
    FaultSink f;
    f.call = (unsigned *)(ws + L.off_fault);
    f.sticky = sticky_fault_word();
    if (opts && opts->test_wait_fault) f.inject = 1;
    return f;
}

Layout layout_of(const Resolved &R, const gf_opts *o)
{
    const size_t pb = R.lps * sizeof(float);
    const size_t nc = (size_t)R.N * R.C * pb;
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off += (bytes + 255) & ~size_t(255); return at; };
    // the call's fault word first, at the same place in every layout (the strips of one host call share it)
    L.off_fault = take(sizeof(unsigned));
    const bool sub = R.s > 1 || R.p_lowres || R.color;
    L.off_Il = take(sub ? (size_t)R.N * R.CI * pb : 0);
    L.off_pl = take(sub ? nc : 0);
    const bool gray = !R.color;
    L.off_a = take((o && o->a_out) || !gray ? 0 : nc);
    L.off_b = take((o && o->b_out) || !gray ? 0 : nc);
    L.off_ma = take((o && o->mean_a_out) || !gray ? 0 : nc);
    L.off_mb = take((o && o->mean_b_out) || !gray ? 0 : nc);
    for (int k = 0; k < 8; ++k)  // colour guide: 4 arrays of 5 + 2C planes per image, then 4 of 2C
        L.off_col[k] = take(R.color ? (size_t)R.N * (k < 4 ? 5 + 2 * R.C : 2 * R.C) * pb : 0);
    L.total = off;
    return L;
}

// Scratch of a backward call: the forward planes, the dense window statistics, and the adjoint planes.
struct BwdLayout {
    Layout fwd;
    size_t off_stats, off_dma, off_dmb, off_gq[4], off_dIl, off_dpl, off_eps, total;
};

BwdLayout bwd_layout_of(const Resolved &R)
{
    BwdLayout B;
    B.fwd = layout_of(R, nullptr);
    size_t off = B.fwd.total;
    auto take = [&](size_t bytes) { size_t at = off; off += (bytes + 255) & ~size_t(255); return at; };
    const size_t nc = (size_t)R.N * R.C * R.lps * sizeof(float);
    B.off_stats = take((size_t)R.N * R.C * 4 * R.h * R.w * sizeof(float));
    B.off_dma = take(nc);
    B.off_dmb = take(nc);
    for (int k = 0; k < 4; ++k) B.off_gq[k] = take(nc);
    B.off_dIl = take(nc);
    B.off_dpl = take(nc);
    B.off_eps = take(bwd_eps_partials(R.N, R.C, R.h, R.w) * sizeof(float));
    B.total = off;
    return B;
}

// Extra checks of a backward call (FP32 only; launch-grid limits of the full-resolution kernel).
gf_status check_backward(const Resolved &R)
{
    if (R.dt_in != GF_F32 || R.dt_out != GF_F32) return fail(GF_EINVAL, "the backward pass takes FP32 I, p and dq");
    if (R.H > 65535) return fail(GF_EINVAL, "the backward pass needs H <= 65535");
    if (R.N > 65535) return fail(GF_EINVAL, "the backward pass needs batch <= 65535");
    if (R.detail != 0.0f) return fail(GF_EINVAL, "detail_gain is forward only");
    if (R.mode == GF_SUB_BILINEAR_AA && R.s > 1) return fail(GF_EINVAL, "antialiased subsampling is forward only");
    if (R.Yw1 - R.Yw0 != R.H) return fail(GF_EINVAL, "a row range is forward only");
    if (R.color) return fail(GF_EINVAL, "the colour guide is forward only");
    if (R.sd != 1) return fail(GF_EINVAL, "a non-integer ratio is forward only");
    return GF_OK;
}

}  // namespace gfk

using gfk::Layout;
using gfk::Resolved;
using gfk::layout_of;
using gfk::resolve;
using gfk::BwdLayout;
using gfk::bwd_layout_of;
using gfk::check_backward;

namespace {

// gf_filter on device buffers.  clear_fault = false leaves the call's fault word as it was, so that the strips
// of one gf_filter_host call accumulate into one word.
gf_status filter_device(gf_ctx *ctx, const void *I, const void *p, void *q, int H, int W, int C, int r, float eps,
                        int s, gf_subsample_mode mode, const gf_opts *opts, void *cuda_stream, bool clear_fault)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    if (!I || !p || !q) return fail(GF_EINVAL, "I, p and q must be device pointers");
    Resolved R;
    gf_status st = resolve(H, W, C, r, eps, s, (int)mode, opts, R);
    if (st != GF_OK) return st;
    if (opts && opts->saved_forward) {
        // the forward of a later gf_filter_backward: its low-res planes stay in the backward's workspace layout
        if ((st = check_backward(R)) != GF_OK) return st;
        if (opts->a_out || opts->b_out || opts->mean_a_out || opts->mean_b_out || opts->stats_out)
            return fail(GF_EINVAL, "saved_forward does not produce low-res intermediate outputs");
        if (!opts->workspace) return fail(GF_EINVAL, "saved_forward needs opts->workspace (gf_backward_workspace_size bytes)");
        R.lps = gfk::plane_stride_f32((size_t)R.h * R.w);
        const BwdLayout BL = bwd_layout_of(R);
        if (opts->workspace_bytes < BL.total)
            return fail(GF_EINVAL, "saved_forward: workspace_bytes is smaller than gf_backward_workspace_size()");
        DeviceGuard guard(ctx->device);
        char *ws = (char *)opts->workspace;
        gfk::FwdPlan P = gfk::make_plan(R, BL.fwd, I, p, q, ws, nullptr);
        P.stats = ws + BL.off_stats;
        P.need_lowres = true;
        P.events = opts->kernel_events ? (cudaEvent_t *)opts->kernel_events : nullptr;
        P.clear_fault = clear_fault;
        cudaError_t e = gfk::launch_forward(P, (cudaStream_t)cuda_stream);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch in gf_filter");
        return GF_OK;
    }
    const Layout L = layout_of(R, opts);

    DeviceGuard guard(ctx->device);
    std::unique_lock<std::mutex> lock(ctx->mu, std::defer_lock);
    char *ws = nullptr;
    if (opts && opts->workspace) {
        if (opts->workspace_bytes < L.total)
            return fail(GF_EINVAL, "workspace_bytes is smaller than gf_workspace_size()");
        ws = (char *)opts->workspace;
    } else {
        lock.lock();
        st = grow(&ctx->arena, &ctx->arena_bytes, L.total, "the scratch arena");
        if (st != GF_OK) return st;
        ws = (char *)ctx->arena;
    }

    gfk::FwdPlan P = gfk::make_plan(R, L, I, p, q, ws, opts);
    P.clear_fault = clear_fault;
    cudaError_t e = gfk::launch_forward(P, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch in gf_filter");
    return GF_OK;
}

// After a synchronous host call: the fault word of its scratch (offset 0 of the context arena or of the
// caller's workspace) is read back; a bounded wait inside a kernel that gave up makes the call GF_EWAIT.
gf_status check_call_faults(gf_ctx *ctx, const gf_opts *opts)
{
    const void *ws = (opts && opts->workspace) ? opts->workspace : ctx->arena;
    if (!ws) return GF_OK;
    unsigned word = 0;
    cudaError_t e = cudaMemcpy(&word, ws, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the call's fault word");
    if (word != 0) {
        char bits[16];
        snprintf(bits, sizeof(bits), "0x%x", word);
        return fail(GF_EWAIT, std::string("a kernel gave up a bounded wait (fault bits ") + bits +
                                  "): the output is incomplete");
    }
    return GF_OK;
}

// Host-buffer pipeline (gf_filter_host on large images): the output rows are cut into strips; the input rows
// each strip's band needs are copied in on one stream, the strip is filtered on the caller's stream as a
// row-range call (the same rows as the whole-image call up to FP32 rounding order), and its output rows are
// copied out on a third stream, so uploads, filtering and downloads of different strips overlap.
constexpr int HOST_MAX_STRIPS = 8;  // measured at 12 MP: 8 strips 1.15 ms, 16: 1.24 ms, 32: 1.47 ms
constexpr size_t HOST_PIPE_MIN_BYTES = size_t(8) << 20;  // below this the copies are too short to overlap

// Strip boundaries Y[0] = 0 < ... < Y[K] = H (multiples of 8 s), K >= 2; or K < 2 when the call keeps the
// single copy-in / filter / copy-out sequence (small, low-res p, colour guide, non-integer ratio, single
// fused kernel, low-res outputs, its own row range or kernel events).
int host_strips(const Resolved &R, const gf_opts *o, size_t host_bytes, std::vector<int> &Y)
{
    Y.clear();
    if (host_bytes < HOST_PIPE_MIN_BYTES) return 0;
    if (R.sd != 1 || R.color || R.p_lowres || R.fused || R.dense_lowres) return 0;
    if (o && (o->row_begin || o->row_end || o->stats_out || o->kernel_events || o->saved_forward)) return 0;
    const int align = 8 * R.s;
    const int K = std::min(HOST_MAX_STRIPS, R.H / (64 * R.s));
    if (K < 2) return 0;
    const int rows = (R.H + K - 1) / K;
    const int step = (rows + align - 1) / align * align;
    for (int y = 0; y < R.H; y += step) Y.push_back(y);
    Y.push_back(R.H);
    return (int)Y.size() - 1;
}

gf_status host_pipeline(gf_ctx *ctx, const Resolved &R, const std::vector<int> &Y, const void *I_host,
                        const void *p_host, void *q_host, char *dI, char *dp, char *dq, int r, float eps, int s,
                        gf_subsample_mode mode, const gf_opts *opts, cudaStream_t stream)
{
    const int K = (int)Y.size() - 1;
    const int H = R.H, W = R.W, C = R.C;
    gf_opts so;
    if (opts) so = *opts; else gf_opts_init(&so);
    // the input rows each strip reads (its band), and the scratch the largest band needs
    std::vector<int> band_end(K);
    size_t ws_need = 0;
    for (int k = 0; k < K; ++k) {
        so.row_begin = Y[k];
        so.row_end = Y[k + 1];
        Resolved Rk;
        gf_status st = resolve(H, W, C, r, eps, s, (int)mode, &so, Rk);
        if (st != GF_OK) return st;
        band_end[k] = std::max(Rk.row0 + Rk.H, k > 0 ? band_end[k - 1] : 0);
        ws_need = std::max(ws_need, layout_of(Rk, &so).total);
    }
    cudaError_t e;
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        if (!so.workspace) {
            gf_status st = grow(&ctx->arena, &ctx->arena_bytes, ws_need, "the scratch arena");
            if (st != GF_OK) return st;
        }
        if (!ctx->copy_in) {
            if ((e = cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "creating the host-call copy streams");
        }
        while (ctx->host_ev.size() < size_t(2 * HOST_MAX_STRIPS + 2)) {
            cudaEvent_t ev;
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "creating the host-call events");
            ctx->host_ev.push_back(ev);
        }
    }
    cudaEvent_t *ev = ctx->host_ev.data();  // [0] start, [1 + k] strip k's input, [1 + K + k] strip k's output
    const size_t ein = gfk::dtype_size(R.dt_in), eout = gfk::dtype_size(R.dt_out);
    const size_t plane = (size_t)H * W;
    const int in_planes = R.N * R.CI, p_planes = R.N * C;
    // Nearest and bilinear subsampling read p only through the subsample, which takes rows s j + o and
    // s j + o + 1 (o = floor((s - 1) / 2)) of block j, clamped to the last row: only those rows of p are
    // uploaded (half of p at s = 4, a quarter at s = 8).  The other rows of the staging copy are never read.
    const bool sampled_p = (R.mode == GF_SUB_NEAREST || R.mode == GF_SUB_BILINEAR) && s >= 3;
    const int o = (s - 1) / 2;
    gf_status result = GF_OK;
    auto check = [&](cudaError_t err, const char *what) {
        if (err != cudaSuccess && result == GF_OK) result = cuda_fail(err, what);
        return result == GF_OK;
    };
    // the copies start after the work already queued on the caller's stream
    bool ok = check(cudaEventRecord(ev[0], stream), "cudaEventRecord") &&
              check(cudaStreamWaitEvent(ctx->copy_in, ev[0], 0), "cudaStreamWaitEvent") &&
              check(cudaStreamWaitEvent(ctx->copy_out, ev[0], 0), "cudaStreamWaitEvent");
    int copied = 0;  // input rows [0, copied) of every plane are queued
    for (int k = 0; ok && k < K; ++k) {
        if (band_end[k] > copied) {
            const size_t off = (size_t)copied * W, n = (size_t)(band_end[k] - copied) * W;
            for (int pl = 0; ok && pl < in_planes; ++pl)
                ok = check(cudaMemcpyAsync(dI + (pl * plane + off) * ein, (const char *)I_host + (pl * plane + off) * ein,
                                           n * ein, cudaMemcpyHostToDevice, ctx->copy_in), "cudaMemcpyAsync of I rows");
            if (!sampled_p) {
                for (int pl = 0; ok && pl < p_planes; ++pl)
                    ok = check(cudaMemcpyAsync(dp + (pl * plane + off) * ein, (const char *)p_host + (pl * plane + off) * ein,
                                               n * ein, cudaMemcpyHostToDevice, ctx->copy_in), "cudaMemcpyAsync of p rows");
            } else {
                // rows s j + o and s j + o + 1 of each whole s-row block (copied starts on a block), and every
                // row of a partial last block (its samples may be clamped to row H - 1)
                const int whole = (band_end[k] == H ? H / s : band_end[k] / s) - copied / s;
                const size_t bpitch = (size_t)s * W * ein;
                for (int pl = 0; ok && whole > 0 && pl < p_planes; ++pl) {
                    const size_t at = (pl * plane + (size_t)(copied + o) * W) * ein;
                    ok = check(cudaMemcpy2DAsync(dp + at, bpitch, (const char *)p_host + at, bpitch, 2 * (size_t)W * ein,
                                                 whole, cudaMemcpyHostToDevice, ctx->copy_in), "cudaMemcpy2DAsync of p rows");
                }
                const int tail0 = std::max(copied, H / s * s);
                if (band_end[k] == H && tail0 < H) {
                    const size_t t_off = (size_t)tail0 * W, t_n = (size_t)(H - tail0) * W;
                    for (int pl = 0; ok && pl < p_planes; ++pl)
                        ok = check(cudaMemcpyAsync(dp + (pl * plane + t_off) * ein,
                                                   (const char *)p_host + (pl * plane + t_off) * ein, t_n * ein,
                                                   cudaMemcpyHostToDevice, ctx->copy_in), "cudaMemcpyAsync of p rows");
                }
            }
            copied = band_end[k];
        }
        ok = ok && check(cudaEventRecord(ev[1 + k], ctx->copy_in), "cudaEventRecord") &&
             check(cudaStreamWaitEvent(stream, ev[1 + k], 0), "cudaStreamWaitEvent");
        if (!ok) break;
        so.row_begin = Y[k];
        so.row_end = Y[k + 1];
        gf_status st = filter_device(ctx, dI, dp, dq, H, W, C, r, eps, s, mode, &so, stream, k == 0);
        if (st != GF_OK) {
            result = st;
            break;
        }
        ok = check(cudaEventRecord(ev[1 + K + k], stream), "cudaEventRecord") &&
             check(cudaStreamWaitEvent(ctx->copy_out, ev[1 + K + k], 0), "cudaStreamWaitEvent");
        const size_t off = (size_t)Y[k] * W, n = (size_t)(Y[k + 1] - Y[k]) * W;
        for (int pl = 0; ok && pl < p_planes; ++pl)
            ok = check(cudaMemcpyAsync((char *)q_host + (pl * plane + off) * eout, dq + (pl * plane + off) * eout,
                                       n * eout, cudaMemcpyDeviceToHost, ctx->copy_out), "cudaMemcpyAsync of q rows");
    }
    // drain all three streams (also after an error, so that no copy into the staging buffers is left in flight)
    cudaError_t e1 = cudaStreamSynchronize(ctx->copy_in);
    cudaError_t e2 = cudaStreamSynchronize(ctx->copy_out);
    cudaError_t e3 = cudaStreamSynchronize(stream);
    check(e1, "cudaStreamSynchronize of the copy-in stream");
    check(e2, "cudaStreamSynchronize of the copy-out stream");
    check(e3, "cudaStreamSynchronize");
    if (result == GF_OK) result = check_call_faults(ctx, opts);
    return result;
}

}  // namespace

extern "C" {

void gf_opts_init(gf_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->batch = 1;
    o->guide_channels = 1;
    o->r_low = -1;
    o->dtype_in = GF_F32;
    o->dtype_out = GF_F32;
}

int gf_abi_version(void) { return GF_ABI_VERSION; }

const char *gf_last_error(void) { return g_last_error.c_str(); }

gf_status gf_lowres_geometry(int H, int W, int s, int r, int r_low, int *h, int *w, int *r_prime)
{
    if (H < 1 || W < 1 || s < 1 || r < 0) return fail(GF_EINVAL, "H, W, s must be >= 1 and r >= 0");
    if (h) *h = (H + s - 1) / s;
    if (w) *w = (W + s - 1) / s;
    if (r_prime) *r_prime = r_low >= 0 ? r_low : lowres_radius(r, s);
    return GF_OK;
}

gf_status gf_workspace_size(int H, int W, int C, int s, const gf_opts *opts, size_t *bytes)
{
    if (!bytes) return fail(GF_EINVAL, "bytes is NULL");
    Resolved R;
    gf_status st = resolve(H, W, C, 0, 0.0f, s, GF_SUB_BILINEAR, opts, R);
    if (st != GF_OK) return st;
    *bytes = layout_of(R, opts).total;
    return GF_OK;
}

gf_status gf_create(gf_ctx **out, int device, size_t hbm_budget_bytes, unsigned flags)
{
    if (!out) return fail(GF_EINVAL, "out is NULL");
    *out = nullptr;
    if (flags != 0) return fail(GF_EINVAL, "flags must be 0");
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(GF_EINVAL, "no such CUDA device");
    gf_ctx *c = new gf_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    c->server = gfk::server_create(device, hbm_budget_bytes);
    *out = c;
    return GF_OK;
}

gf_status gf_destroy(gf_ctx *ctx)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    gfk::server_destroy(ctx->server);
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        if (ctx->arena) cudaFree(ctx->arena);
        if (ctx->stage) cudaFree(ctx->stage);
        if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
        if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
        for (cudaEvent_t ev : ctx->host_ev) cudaEventDestroy(ev);
    }
    delete ctx;
    return GF_OK;
}

gf_status gf_filter(gf_ctx *ctx, const void *I, const void *p, void *q, int H, int W, int C, int r, float eps, int s,
                    gf_subsample_mode mode, const gf_opts *opts, void *cuda_stream)
{
    gfk::NvtxRange range("gf_filter");
    return filter_device(ctx, I, p, q, H, W, C, r, eps, s, mode, opts, cuda_stream, true);
}

gf_status gf_filter_host(gf_ctx *ctx, const void *I_host, const void *p_host, void *q_host, int H, int W, int C,
                         int r, float eps, int s, gf_subsample_mode mode, const gf_opts *opts, void *cuda_stream)
{
    gfk::NvtxRange range("gf_filter_host");
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    if (!I_host || !p_host || !q_host) return fail(GF_EINVAL, "I, p and q must be host pointers");
    Resolved R;
    gf_status st = resolve(H, W, C, r, eps, s, (int)mode, opts, R);
    if (st != GF_OK) return st;
    const size_t esz = gfk::dtype_size(R.dt_in);
    const size_t plane = (size_t)R.H * R.W;
    const size_t bI = (size_t)R.N * R.CI * plane * esz;
    const size_t bp = (size_t)R.N * R.C * (R.p_lowres ? (size_t)R.h * R.w : plane) * esz;
    const size_t bq = (size_t)R.N * R.C * plane * gfk::dtype_size(R.dt_out);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    DeviceGuard guard(ctx->device);
    std::lock_guard<std::mutex> host_lock(ctx->host_mu);  // the staging buffers serve one host call at a time
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    char *base;
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        st = grow(&ctx->stage, &ctx->stage_bytes, al(bI) + al(bp) + al(bq), "host-call staging");
        if (st != GF_OK) return st;
        base = (char *)ctx->stage;
    }
    char *dI = base, *dp = base + al(bI), *dq = base + al(bI) + al(bp);
    std::vector<int> Y;
    if (host_strips(R, opts, bI + bp + bq, Y) >= 2)
        return host_pipeline(ctx, R, Y, I_host, p_host, q_host, dI, dp, dq, r, eps, s, mode, opts, stream);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dI, I_host, bI, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync of I");
    if ((e = cudaMemcpyAsync(dp, p_host, bp, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync of p");
    st = gf_filter(ctx, dI, dp, dq, H, W, C, r, eps, s, mode, opts, cuda_stream);
    if (st != GF_OK) return st;
    if ((e = cudaMemcpyAsync(q_host, dq, bq, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync of q");
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return check_call_faults(ctx, opts);
}

int gf_host_strips(int H, int W, int C, int s, gf_subsample_mode mode, const gf_opts *opts, int *row_starts)
{
    Resolved R;
    if (resolve(H, W, C, 0, 0.0f, s, (int)mode, opts, R) != GF_OK) return -1;
    const size_t plane = (size_t)R.H * R.W;
    const size_t bytes = (size_t)R.N * (R.CI + R.C) * plane * gfk::dtype_size(R.dt_in) +
                         (size_t)R.N * R.C * plane * gfk::dtype_size(R.dt_out);
    std::vector<int> Y;
    const int K = host_strips(R, opts, bytes, Y);
    if (K < 2) return 1;
    if (row_starts)
        for (int k = 0; k <= K; ++k) row_starts[k] = Y[k];
    return K;
}

gf_status gf_backward_workspace_size(int H, int W, int C, int s, const gf_opts *opts, size_t *bytes)
{
    if (!bytes) return fail(GF_EINVAL, "bytes is NULL");
    Resolved R;
    gf_status st = resolve(H, W, C, 0, 0.0f, s, GF_SUB_BILINEAR, opts, R);
    if (st != GF_OK) return st;
    R.lps = gfk::plane_stride_f32((size_t)R.h * R.w);
    *bytes = bwd_layout_of(R).total;
    return GF_OK;
}

gf_status gf_filter_backward(gf_ctx *ctx, const void *I, const void *p, const void *dq, void *dI, void *dp, float *d_eps,
                             int H, int W, int C, int r, float eps, int s, gf_subsample_mode mode, const gf_opts *opts,
                             void *cuda_stream)
{
    gfk::NvtxRange range("gf_filter_backward");
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    if (!I || !p || !dq || !dI || !dp) return fail(GF_EINVAL, "I, p, dq, dI and dp must be device pointers");
    Resolved R;
    gf_status st = resolve(H, W, C, r, eps, s, (int)mode, opts, R);
    if (st != GF_OK) return st;
    if ((st = check_backward(R)) != GF_OK) return st;
    R.lps = gfk::plane_stride_f32((size_t)R.h * R.w);  // optional low-res outputs are not produced here
    const BwdLayout L = bwd_layout_of(R);

    DeviceGuard guard(ctx->device);
    std::unique_lock<std::mutex> lock(ctx->mu, std::defer_lock);
    char *ws = nullptr;
    const bool saved = opts && opts->saved_forward;
    if (saved && !opts->workspace) return fail(GF_EINVAL, "saved_forward needs the workspace the forward filled");
    if (opts && opts->workspace) {
        if (opts->workspace_bytes < L.total)
            return fail(GF_EINVAL, "workspace_bytes is smaller than gf_backward_workspace_size()");
        ws = (char *)opts->workspace;
    } else {
        lock.lock();
        st = grow(&ctx->arena, &ctx->arena_bytes, L.total, "the scratch arena");
        if (st != GF_OK) return st;
        ws = (char *)ctx->arena;
    }

    gfk::BwdPlan B;
    B.fwd_saved = saved;
    B.fwd = gfk::make_plan(R, L.fwd, I, p, nullptr, ws, nullptr);
    gfk::FwdPlan &P = B.fwd;
    P.stats = ws + L.off_stats;
    P.skip_output = true;
    P.need_lowres = true;
    B.dq = (const float *)dq;
    B.dI = (float *)dI;
    B.dp = (float *)dp;
    B.d_eps = d_eps;
    B.dma = (float *)(ws + L.off_dma);
    B.dmb = (float *)(ws + L.off_dmb);
    for (int k = 0; k < 4; ++k) B.gq[k] = (float *)(ws + L.off_gq[k]);
    B.dIl = (float *)(ws + L.off_dIl);
    B.dpl = (float *)(ws + L.off_dpl);
    B.eps_partial = (float *)(ws + L.off_eps);
    cudaError_t e = gfk::launch_backward(B, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch in gf_filter_backward");
    return GF_OK;
}

double gf_clock(void) { return gfk::now_seconds(); }

gf_status gf_serve_config(gf_ctx *ctx, int slots, size_t queue_limit)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    return gfk::server_config(ctx->server, slots, queue_limit);
}

gf_status gf_submit(gf_ctx *ctx, const gf_request *req, uint64_t *ticket)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    DeviceGuard guard(ctx->device);
    return gfk::server_submit(ctx->server, req, ticket);
}

gf_status gf_poll(gf_ctx *ctx, uint64_t ticket, int64_t timeout_us, gf_result *out)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    return gfk::server_poll(ctx->server, ticket, timeout_us, out);
}

gf_status gf_cancel(gf_ctx *ctx, uint64_t ticket)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    return gfk::server_cancel(ctx->server, ticket);
}

gf_status gf_serve_graphs(gf_ctx *ctx, int enable)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    return gfk::server_graphs(ctx->server, enable);
}

gf_status gf_serve_tile_queue(gf_ctx *ctx, int enable)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    return gfk::server_queue(ctx->server, enable);
}

gf_status gf_serve_pause(gf_ctx *ctx, int paused)
{
    if (!ctx) return fail(GF_EINVAL, "ctx is NULL");
    return gfk::server_pause(ctx->server, paused);
}

gf_status gf_serve_stats_get(gf_ctx *ctx, gf_serve_stats *out)
{
    if (!ctx || !out) return fail(GF_EINVAL, "ctx and out must not be NULL");
    return gfk::server_stats(ctx->server, out);
}

gf_status gf_kernel_faults(int device, unsigned *flags, int clear)
{
    if (!flags) return fail(GF_EINVAL, "flags is NULL");
    DeviceGuard guard(device);
    cudaError_t e = gfk::read_kernel_faults(flags, clear != 0);
    if (e != cudaSuccess) return cuda_fail(e, "reading the kernel fault bits");
    return GF_OK;
}

gf_status gf_row_band(int H, int W, int s, int r, int r_low, gf_subsample_mode mode, int row_begin, int row_end,
                      int *row0, int *rows)
{
    if (!row0 || !rows) return fail(GF_EINVAL, "row0 and rows must not be NULL");
    gf_opts o;
    gf_opts_init(&o);
    o.r_low = r_low;
    o.row_begin = row_begin;
    o.row_end = row_end;
    Resolved R;
    gf_status st = resolve(H, W, 1, r, 0.0f, s, (int)mode, &o, R);
    if (st != GF_OK) return st;
    *row0 = R.row0;
    *rows = R.H;
    return GF_OK;
}

int gf_filter_kernel_count(int H, int W, int C, int s, gf_subsample_mode mode, const gf_opts *opts)
{
    Resolved R;
    if (resolve(H, W, C, 0, 0.0f, s, (int)mode, opts, R) != GF_OK) return -1;
    return gfk::forward_kernel_count(R);
}

}  // extern "C"
