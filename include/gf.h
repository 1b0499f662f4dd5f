/*
 * gf.h -- C ABI of the GB300 (sm_103a) fast guided filter library, libgf.so.
 *
 * Method: K. He and J. Sun, "Fast Guided Filter" (arXiv:1505.00996, 2015).  The library evaluates
 * Algorithm 2 of the paper: subsample the guide I and the input p by a ratio s, compute the box
 * statistics of I', p', I'.*I', I'.*p' at the low-res radius r', form the coefficients a (Eq. 2) and
 * b (Eq. 3), box-average them, bilinearly upsample the averages, and output q = mean_a .* I + mean_b
 * (Eq. 4) on the FULL-resolution guide.  With s = 1 the same call is the guided filter of Algorithm 1.
 *
 * Conventions (the paper leaves these open; the library and its tests fix them):
 *   - f_mean(x, r): mean over the window of radius r clipped to the image, divided by the number of
 *     in-image pixels of that window.
 *   - Low-res size h = ceil(H/s), w = ceil(W/s); r' = r/s rounded half up and raised to 1 when r >= 1
 *     (s = 1 gives r' = r), unless gf_opts.r_low >= 0 sets r' directly.  r' <= 128 is supported.
 *   - Nearest subsample takes full-res (floor((j+1/2)s), floor((i+1/2)s)); bilinear subsample and
 *     upsample use half-pixel centres without antialiasing, with coordinates clamped to the image;
 *     box subsample (not in the paper) averages each s x s block clipped to the image; antialiased
 *     bilinear subsample weights source pixel x by max(0, 1 - |x + 1/2 - (i + 1/2) s| / s) along each
 *     axis (a triangle filter of half-width s) and renormalises over the taps inside the image.
 *   - I has 1 channel (shared by every channel of p) or C channels (channel c guides channel c).
 *
 * Memory: every image pointer is caller-owned DEVICE memory, dense row-major planes, batch-major
 * (N x channels x rows x cols).  The library never frees caller memory.  Calls are asynchronous on the
 * caller's CUDA stream (a cudaStream_t passed as void*, NULL = legacy default stream) unless stated.
 *
 * Errors: every entry point returns a gf_status.  Argument errors return GF_EINVAL before anything is
 * launched; gf_last_error() then returns a message for the calling thread.  GF_ECUDA reports a failed
 * CUDA call (launch or allocation); the message names it.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GF_ABI_VERSION 5
#define GF_MAX_STAGES 8 /* kernel stages one gf_filter call can launch (for gf_opts.kernel_events) */
#define GF_FUSED_AUTO_PIXELS (1 << 20) /* gf_opts.fused = 0 runs the single kernel up to N*C*H*W pixels */

typedef enum gf_status {
    GF_OK = 0,
    GF_PENDING = 1,     /* gf_poll: the request has not finished yet */
    GF_EINVAL = -1,     /* invalid argument; nothing was launched */
    GF_ENOMEM = -2,     /* a device allocation failed or the request can never fit the memory budget */
    GF_ECUDA = -3,      /* a CUDA runtime call failed */
    GF_ETIMEOUT = -4,   /* gf_poll: not finished within the timeout */
    GF_EBUSY = -5,      /* the serving queue is full */
    GF_ECANCELED = -6,  /* the request was cancelled */
    GF_ENOTFOUND = -7,  /* unknown ticket */
    GF_EWAIT = -8       /* a bounded wait inside a kernel gave up (its data never arrived): the output of
                           the call or request is incomplete */
} gf_status;

typedef enum gf_subsample_mode {
    GF_SUB_NEAREST = 0,
    GF_SUB_BILINEAR = 1,
    GF_SUB_BOX = 2,
    GF_SUB_BILINEAR_AA = 3  /* antialiased bilinear; float input, forward only */
} gf_subsample_mode;

typedef enum gf_dtype { GF_F32 = 0, GF_F16 = 1, GF_U8 = 2 } gf_dtype;

typedef struct gf_ctx gf_ctx;

/*
 * Options of one filter call.  Fill with gf_opts_init() and change what you need.
 *   batch           N >= 1 images.
 *   guide_channels  CI: 1 (one gray guide for all channels of p) or C (depthwise guide).  0 means 1.
 *   r_low           >= 0: the low-res radius r'; < 0: derive r' from r and s (see above).
 *   p_lowres        nonzero: p is already at low resolution (N x C x h x w) and is not subsampled.
 *   dtype_in        storage of I and p: GF_F32, GF_F16 (FP32 arithmetic), or GF_U8 (values k/255;
 *                   window sums are exact integers; nearest or bilinear subsample only).
 *   dtype_out       storage of q: GF_F32 or GF_F16 (GF_U8 input always gives GF_F32 or GF_F16 out).
 *   a_out, b_out, mean_a_out, mean_b_out
 *                   optional device buffers (FP32, N x C x h x w) that receive a, b of Eq. (2)-(3) and
 *                   their box means before upsampling.  NULL skips them.
 *   stats_out       optional device buffer, N x C x 4 x h x w: for float input the window means
 *                   mean_I, corr_I, mean_p, corr_Ip (FP32); for GF_U8 input the exact window SUMS
 *                   (uint32) of J, J*J, P, J*P where J, P are the subsampled values in units of 1/(255k),
 *                   k = 4 for bilinear subsampling at even s and 1 otherwise.
 *   workspace, workspace_bytes
 *                   optional caller-owned device scratch of at least gf_workspace_size() bytes; NULL
 *                   makes the call use (and grow) the context's own arena.
 *   kernel_events   optional array of 2*GF_MAX_STAGES cudaEvent_t (as void*): event 2k is recorded
 *                   before and 2k+1 after the k-th kernel the call launches (unused ones untouched).
 *   detail_gain     k (finite; default 0): the output becomes q + k (I - q) instead of q, with I the
 *                   guide channel of each output channel -- with p = I, the detail enhancement of the
 *                   paper's Fig. 2 (k = 5 there).  Applied in the output kernel; forward only
 *                   (gf_filter_backward returns GF_EINVAL for k != 0).
 *   row_begin, row_end
 *                   0 <= row_begin < row_end <= H: compute and write only output rows [row_begin, row_end)
 *                   of every plane of q (other rows of q are left untouched); 0, 0 = all rows.  I, p and q
 *                   still describe the whole image.  The call filters the band of complete s-row blocks
 *                   that reaches 2 r' low-res rows beyond the tap rows of the range (the rows whose clipped
 *                   windows could differ from the whole image's are never used), so each strip equals the
 *                   same rows of the whole-image call up to FP32 rounding order.  This is how one image is
 *                   split across GPUs: each filters its own rows from the (replicated) input, and no data
 *                   is exchanged.  Not combined with a_out, b_out, mean_a_out, mean_b_out or stats_out;
 *                   forward only.
 *   s_num, s_den    0, 0: the call's integer ratio s.  Otherwise the ratio is s_num / s_den >= 1 (for
 *                   example 5 / 2), replacing s: the same coordinate maps with that s, decided exactly in
 *                   integer arithmetic; h = ceil(H s_den / s_num).  A non-integer ratio takes nearest,
 *                   bilinear or antialiased subsampling, FP32 or FP16 storage, a gray or depthwise guide,
 *                   no row range; forward only.
 *   fused           0: run the whole filter as one kernel (each CTA recomputes its halo) for a subsampled
 *                   call (s > 1) on a small image (N*C*H*W <= GF_FUSED_AUTO_PIXELS, and N*C*H*W weighed by
 *                   (1 + r'/4)^2 for the halo at most 2.1 GF_FUSED_AUTO_PIXELS), where the four-kernel
 *                   chain is dominated by per-kernel fixed costs; 1: always (GF_EINVAL where unsupported);
 *                   -1: never.  The single
 *                   kernel takes FP32 or FP16 storage, a gray or depthwise guide, any subsample mode and
 *                   ratio, r' up to what fits its tiles in shared memory, and no low-res intermediate outputs.
 *   saved_forward   nonzero, with a workspace of at least gf_backward_workspace_size() bytes: gf_filter
 *                   also keeps the forward's low-res planes (I', p', the window statistics, a, the box
 *                   means) in that workspace, laid out as gf_filter_backward reads them, and
 *                   gf_filter_backward given the same workspace and flag skips recomputing them.  The
 *                   backward call must use the same arguments and inputs as the forward that saved them,
 *                   with no other call on that workspace in between (not checked).  Takes what the
 *                   backward takes (FP32, nearest / bilinear / box, integer ratio, no row range, detail
 *                   gain or colour guide) and no low-res intermediate outputs; GF_EINVAL otherwise.
 *   color_guide     nonzero: I has guide_channels = 3 channels used jointly as a colour guide for every
 *                   channel of p (the guided filter's colour form, which the paper cites): per window
 *                   a = (Sigma + eps U)^-1 cov_Ip with Sigma the 3 x 3 covariance of I', b = mean_p - a^T
 *                   mean_I, and q = mean_a^T I + mean_b.  FP32 or FP16 storage; forward only; no low-res
 *                   intermediate outputs; detail_gain needs C = 3 (channel c's detail is I_c - q_c).
 *   test_wait_fault nonzero (tests of the timeout path only): the TMA-fed output kernel leaves the first
 *                   stage of its ring unfilled and every bounded wait of the call gives up after 256 polls,
 *                   so the consumers' first wait runs out; the kernel records GF_EWAIT in the call's fault
 *                   word and returns with q incomplete.  No GPU fault is made.
 */
typedef struct gf_opts {
    int batch;
    int guide_channels;
    int r_low;
    int p_lowres;
    gf_dtype dtype_in;
    gf_dtype dtype_out;
    float *a_out;
    float *b_out;
    float *mean_a_out;
    float *mean_b_out;
    void *stats_out;
    void *workspace;
    size_t workspace_bytes;
    void **kernel_events;
    float detail_gain;
    int row_begin;
    int row_end;
    int color_guide;
    int s_num;
    int s_den;
    int fused;
    int saved_forward;
    int test_wait_fault;
} gf_opts;

/* Default options: batch 1, gray guide, derived r', full-res p, FP32 in and out, nothing optional. */
void gf_opts_init(gf_opts *opts);

/* ABI version of the loaded library (GF_ABI_VERSION it was built with). */
int gf_abi_version(void);

/* Message describing the last error returned to the calling thread ("" if none).  Owned by the
 * library; valid until the next call on the same thread. */
const char *gf_last_error(void);

/* Low-res geometry of a call: h = ceil(H/s), w = ceil(W/s), and the radius r' used on that grid
 * (Algorithm 2 sets r' = r/s).  Host-only; returns GF_EINVAL for H, W, s < 1 or r < 0. */
gf_status gf_lowres_geometry(int H, int W, int s, int r, int r_low, int *h, int *w, int *r_prime);

/* The band of rows a call restricted to output rows [row_begin, row_end) filters (gf_opts.row_begin /
 * row_end): full-res rows [*row0, *row0 + *rows) of I and p -- the only input rows it reads (rows
 * [*row0 / s, (*row0 + *rows + s - 1) / s) of a low-res p).  r_low < 0 derives r' from r.  Host-only;
 * GF_EINVAL for invalid arguments. */
gf_status gf_row_band(int H, int W, int s, int r, int r_low, gf_subsample_mode mode, int row_begin, int row_end,
                      int *row0, int *rows);

/* Fault bits the library's kernels recorded on `device` since the last clear, over all calls (host call;
 * synchronous copy from the device).  Bit 0: a bounded wait of the TMA-fed output kernel gave up; bit 1:
 * one of the TMA-fed box kernels (the kernel stopped early; the output of that call is incomplete).
 * clear != 0 resets them.  GF_ECUDA if the copy fails.  Besides these device-wide bits, every call keeps
 * a fault word of its own in its scratch, zeroed when the call starts: gf_filter_host and the serving loop
 * read it after the call and report GF_EWAIT when it is set. */
gf_status gf_kernel_faults(int device, unsigned *flags, int clear);

/* Number of kernels one gf_filter call with these arguments launches (host-only; -1 for invalid
 * arguments): 1 when the single fused kernel runs (gf_opts.fused); else 4 when s > 1 (subsample,
 * statistics + coefficients, box means of a and b, upsample + output), 3 when the subsample and the
 * statistics run as one kernel (opt-in with the environment variable GF_SUB_STRIP=1: FP32, s = 4 or 8,
 * nearest or bilinear, a gray guide for C a multiple of 3, r' = 4, which this count learns from
 * opts->r_low; 16-byte aligned planes and no stats_out assumed); at s = 1, 2 (statistics, then the box
 * means fused with the output; rows a multiple of 4 pixels) or 3; 6 with a colour guide (subsample,
 * products, box means, coefficients, box means, upsample + output). */
int gf_filter_kernel_count(int H, int W, int C, int s, gf_subsample_mode mode, const gf_opts *opts);

/* Bytes of device scratch one gf_filter call with these arguments needs (host-only). */
gf_status gf_workspace_size(int H, int W, int C, int s, const gf_opts *opts, size_t *bytes);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device memory the serving loop
 * holds for admitted requests' scratch (0 = 2 GiB).  flags: reserved, 0.
 * The context owns a growable scratch arena and the serving state; it does not own any stream. */
gf_status gf_create(gf_ctx **out, int device, size_t hbm_budget_bytes, unsigned flags);

/* Wait for the context's own in-flight work, then free everything it owns. */
gf_status gf_destroy(gf_ctx *ctx);

/*
 * Fast guided filter, Algorithm 2 (and Algorithm 1 when s = 1).
 *   I: N x CI x H x W guide; p: N x C x H x W input (N x C x h x w if opts->p_lowres);
 *   q: N x C x H x W output, dtype opts->dtype_out.  All device pointers, dense.
 *   r >= 0 full-res radius; eps >= 0 regulariser added to var(I) (data on the [0,1] scale for the
 *   paper's eps values); s >= 1 subsampling ratio; mode: subsample mode.
 *   opts may be NULL (defaults).  cuda_stream: the stream the kernels run on.
 *   Size limits (GF_EINVAL otherwise): H * W < 2^31, ceil(H/s) <= 65535, batch * (CI + C) <= 65535,
 *   r' <= 128; uint8 input also needs (2r'+1)^2 (255k)^2 < 2^32 (k = 4 for bilinear at even s, else 1).
 * Without a caller workspace the call uses the context arena; growing it is synchronous, and two
 * calls that share a context arena must not run concurrently on different streams.
 * Returns GF_OK once the kernels are enqueued.
 */
gf_status gf_filter(gf_ctx *ctx, const void *I, const void *p, void *q, int H, int W, int C, int r, float eps,
                    int s, gf_subsample_mode mode, const gf_opts *opts, void *cuda_stream);

/*
 * Same filter on HOST buffers: copies I and p to the device, filters, copies q back and waits for all of
 * it.  Staging memory comes from the context.  Host buffers may be pageable or pinned (pinned is faster:
 * only pinned copies overlap).  Synchronous; one gf_filter_host call at a time per context (a second
 * caller waits).  Work already queued on cuda_stream runs first.
 * Large images (gf_host_strips() > 1) are pipelined: the output rows are cut into strips, each strip is
 * filtered as a row-range call (gf_opts.row_begin / row_end) as soon as the input rows of its band are on
 * the device, and its output rows are copied back while later strips are uploaded and filtered (two copy
 * streams owned by the context).  Each strip equals the same rows of the whole-image call up to FP32
 * rounding order.  With nearest or bilinear subsampling at s >= 3 only the rows of p that the subsample
 * reads are uploaded (rows s j + (s - 1) / 2 and the next of every s-row block, and a partial last block
 * whole): half of p at s = 4, a quarter at s = 8.
 * Returns GF_EWAIT (q incomplete) when a kernel of the call gave up a bounded wait.
 */
gf_status gf_filter_host(gf_ctx *ctx, const void *I_host, const void *p_host, void *q_host, int H, int W, int C,
                         int r, float eps, int s, gf_subsample_mode mode, const gf_opts *opts, void *cuda_stream);

/* The strips gf_filter_host pipelines a call with these arguments in (host-only): returns K >= 2 and, if
 * row_starts is not NULL, writes its K + 1 boundaries 0 = Y_0 < Y_1 < ... < Y_K = H (multiples of 8 s;
 * up to 8 strips, at least 64 s rows each); returns 1 when the call is not pipelined (under 8 MiB of
 * host data, a low-res p, a colour guide, a non-integer ratio, the single fused kernel, low-res outputs,
 * its own row range or kernel events), -1 for invalid arguments.  row_starts holds at least 9 ints. */
int gf_host_strips(int H, int W, int C, int s, gf_subsample_mode mode, const gf_opts *opts, int *row_starts);

/*
 * Backward pass of gf_filter: the exact derivative of Algorithm 2 (the paper gives none; it is derived by
 * the chain rule through every step, with the transposed box mean sum_{k: i in w_k} y_k / n_k at borders).
 *   dq: dL/dq, N x C x H x W.  Outputs (overwritten): dI (N x CI x H x W), dp (same shape as p: full
 *   resolution, or N x C x h x w when opts->p_lowres), and, if d_eps is not NULL, the device scalar
 *   dL/d eps (summed over every channel, pixel and batch element).  All FP32 (opts->dtype_in and dtype_out
 *   must be GF_F32); the other arguments are those of the forward call.  The forward statistics are
 *   recomputed, unless opts->saved_forward names a workspace a gf_filter call filled (see gf_opts).
 *   Scratch: the context arena, or opts->workspace of gf_backward_workspace_size() bytes.
 *   Size limits: those of gf_filter, and H <= 65535, batch <= 65535 (GF_EINVAL otherwise).
 *   Asynchronous on cuda_stream; deterministic (no atomics).
 */
gf_status gf_backward_workspace_size(int H, int W, int C, int s, const gf_opts *opts, size_t *bytes);
gf_status gf_filter_backward(gf_ctx *ctx, const void *I, const void *p, const void *dq, void *dI, void *dp, float *d_eps,
                             int H, int W, int C, int r, float eps, int s, gf_subsample_mode mode, const gf_opts *opts,
                             void *cuda_stream);

/* ---- Serving: continuous batching of filter requests -------------------------------------------------
 *
 * gf_submit queues a request and returns at once with a ticket.  A scheduler thread owned by the context
 * admits queued requests in arrival order as soon as one of its stream slots is free and the request's
 * low-res scratch fits in the context's HBM budget (gf_create's hbm_budget_bytes; 0 means 2 GiB), taken
 * from one device arena the context allocates on the first submit.  Admitted requests run on separate
 * streams, so requests that arrive while others are on the GPU overlap with them.  gf_poll returns the
 * outcome.  The per-pixel arithmetic is that of gf_filter, so a request's q is the same whether it ran alone
 * or among others.  I, p and q stay caller-owned and must remain valid until gf_poll reports a terminal
 * status (GF_OK, GF_ECANCELED or an error).  Times are seconds on gf_clock().  A request whose inputs are
 * still being written by work on another stream names an event recorded after that work (ready_event); its
 * kernels then wait for the event on the GPU.  A request whose kernel gave up a bounded wait (its data
 * never arrived) is reported GF_EWAIT, not GF_OK.
 */
typedef struct gf_request {
    const void *I, *p;  /* device inputs, as for gf_filter */
    void *q;            /* device output */
    int H, W, C, r;
    float eps;
    int s;
    gf_subsample_mode mode;
    gf_opts opts;       /* batch, guide_channels, r_low, p_lowres, dtype_in/out, fused, test_wait_fault;
                           other fields are ignored */
    void *user;         /* caller's tag, returned in gf_result */
    void *ready_event;  /* optional cudaEvent_t (as void*): the request's kernels wait for the work recorded in
                           it when gf_submit is called (record it after the work that writes I and p; the
                           event may be re-recorded or destroyed once gf_submit returns).  NULL: none */
} gf_request;

typedef struct gf_result {
    gf_status status;   /* GF_OK, GF_ECANCELED, or the error the request failed with */
    uint64_t ticket;
    void *user;
    double t_submit, t_admit, t_done;  /* gf_clock() at submission, admission and completion on the GPU */
    size_t scratch_bytes;              /* the request's HBM footprint in the serving arena */
} gf_result;

typedef struct gf_serve_stats {
    int queued, running, slots;
    size_t budget_bytes, scratch_in_use;
    long long launches;        /* requests launched so far */
    long long graph_launches;  /* of which through their bucket's CUDA graph (gf_serve_graphs) */
    long long queue_launches;  /* tile-queue launches (gf_serve_tile_queue) */
    long long queue_requests;  /* requests those launches carried */
    double launch_seconds;     /* host time the scheduler spent enqueuing them (kernels and bookkeeping) */
} gf_serve_stats;

/* Monotonic clock of the serving timestamps, in seconds. */
double gf_clock(void);

/* Stream slots (concurrent requests, default 4, at most 64) and queue limit (default 4096) of the serving
 * loop.  Only before the first gf_submit on the context (GF_EBUSY afterwards). */
gf_status gf_serve_config(gf_ctx *ctx, int slots, size_t queue_limit);

/* Per-bucket CUDA graphs for the serving launches: enable = 1 replays the launch sequence of a request
 * through an executable graph shared by the requests of its bucket on its slot (the same kernels: storage
 * types, channels, ratio, subsample mode, r', single-kernel or chain form, alignment classes), captured and
 * updated to the request's sizes and buffers; 0 (the default) launches every request's work directly, which
 * costs less host time per request on a GB300 host (18 us against 28-34 us for capture, update and graph
 * launch).  Only before the first gf_submit on the context (GF_EBUSY afterwards). */
gf_status gf_serve_graphs(gf_ctx *ctx, int enable);

/* The tile queue for the serving launches (one launch for requests of mixed sizes): enable = 1 (the
 * default) admits, once every other slot is taken, the requests that gf_filter would run as its single kernel
 * (small images, no colour guide) and that stand next to each other at the head of the queue with the same
 * storage types and subsample mode together onto the last slot, up to 16, and runs them as ONE launch of that
 * kernel's tile-queue form: a grid over
 * their (request, tile) items with one descriptor per request.  Every request keeps its own scratch, fault
 * word, completion and result, bit for bit its solo result.  0 launches every request on its own.  Only
 * before the first gf_submit on the context (GF_EBUSY afterwards). */
gf_status gf_serve_tile_queue(gf_ctx *ctx, int enable);

/* Queue a request.  GF_EINVAL for bad arguments, GF_ENOMEM if its scratch can never fit the budget,
 * GF_EBUSY if the queue is full; otherwise GF_OK and *ticket. */
gf_status gf_submit(gf_ctx *ctx, const gf_request *req, uint64_t *ticket);

/* Outcome of a request.  timeout_us = 0: check and return GF_PENDING if not finished; > 0: wait at most that
 * long, then GF_ETIMEOUT; < 0: wait until it finishes.  On a terminal status the result is written to *out
 * (if not NULL) and the ticket is retired: GF_OK, GF_ECANCELED, or the request's error.  GF_ENOTFOUND for an
 * unknown or already retired ticket. */
gf_status gf_poll(gf_ctx *ctx, uint64_t ticket, int64_t timeout_us, gf_result *out);

/* Cancel a request that is still queued (GF_OK); GF_EBUSY once it has been admitted to the GPU. */
gf_status gf_cancel(gf_ctx *ctx, uint64_t ticket);

/* Hold (paused != 0) or resume admission.  Held requests stay queued (and cancellable); requests already on
 * the GPU run to completion.  Lets a host drain or stage work. */
gf_status gf_serve_pause(gf_ctx *ctx, int paused);

/* Queue depth, running requests and scratch in use of the serving loop. */
gf_status gf_serve_stats_get(gf_ctx *ctx, gf_serve_stats *out);

/*
 * gf_filter without any device allocation.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- a plugin whose host application owns every device allocation
 * through its own pool or budget, code that must not take the allocator's locks or its implicit
 * synchronisation on a latency-critical path, or a C caller with no context object to own an arena.
 *
 * Same arguments and results as gf_filter (no ctx; opts->workspace must be NULL).  The scratch is one
 * fixed array of 64 MiB compiled into the library, which every GPU that loads the library holds until the
 * process exits; a call whose scratch (gf_workspace_size) exceeds 64 MiB returns GF_EINVAL with a message
 * (a 12 MP, 3-channel FP32 call at s = 4 needs about 48 MB; s = 1 at that size does not fit).  Runs on the
 * current CUDA device.  The first call in each CUDA context looks up that context's address of the array
 * (a context made after cudaDeviceReset gets its own lookup); make that first call before any stream
 * capture.  Every call shares the one array, which keeps the last call's contents (the filter writes each
 * scratch plane before reading it, and zeroes the call's fault word itself): calls whose kernels overlap
 * on the GPU -- on different streams, or from different threads -- race on it and must be serialised by
 * the caller.  No cudaMalloc, cudaFree or other allocating call is made.
 */
gf_status gf_filter_noalloc(const void *I, const void *p, void *q, int H, int W, int C, int r, float eps, int s,
                            gf_subsample_mode mode, const gf_opts *opts, void *cuda_stream);

/*
 * Environment variables read by the library (none is needed in normal use):
 *   GF_NO_TMA       set: the s = 4, 8 output step uses its per-thread cp.async form instead of the
 *                   TMA-fed kernel (same results; for comparing the two and for drivers without
 *                   cuTensorMapEncodeTiled).  Read at every call.
 *   GF_FAULT        "launch:K": the serving loop's launch attempt number K (counting from 0) launches
 *                   nothing and fails its request with GF_ECUDA (host-side fault injection for tests of
 *                   the error path; no GPU fault is made).  Read when the context is created.
 *
 * Timeline profilers: gf_filter, gf_filter_host, gf_filter_backward, gf_filter_noalloc and each serving
 * launch push an NVTX range named after the call ("gf_filter", ..., "gf_serve launch") for its host-side
 * duration; without a profiler attached the ranges cost nothing.
 */

#ifdef __cplusplus
}
#endif

#endif /* GF_H */
