// gf_serve.cu -- the serving loop behind gf_submit / gf_poll / gf_cancel: continuous batching of fast guided
// filter requests of mixed sizes on one GPU.
//
// Requests enter a FIFO queue.  A scheduler thread per context admits the head of the queue as soon as a
// stream slot is free and the request's low-res scratch (its HBM footprint: the I', p', a, b, mean_a,
// mean_b planes) fits in the context's budget; the scratch comes from one device arena carved by a
// first-fit allocator.  Each admitted request runs the forward kernels on its slot's stream, so requests
// that arrive while others are on the GPU overlap with them on the device.  A host callback enqueued after
// the kernels timestamps the completion and wakes the scheduler, which frees the slot and the scratch and
// admits more work.  The per-pixel arithmetic does not depend on what else is running, so a request's
// result is the same alone and in a mix.
//
// Failure handling: a failed launch marks its request GF_ECUDA and the loop carries on; the environment
// variable GF_FAULT=launch:<k> makes the k-th admitted launch report failure without launching anything
// (used by the tests); waits in gf_poll are bounded by the caller's timeout.  After a request's kernels its
// slot stream copies the request's fault word (the bounded waits inside the kernels) to pinned host memory
// ahead of the completion callback, and the scheduler reports a request whose word is set as GF_EWAIT.
// A request's ready_event is waited for on the slot stream before its kernels, so inputs that another
// stream is still writing are complete when they are read.
//
// Per-bucket CUDA graphs (off unless gf_serve_graphs turns them on): requests whose launch sequence has the
// same kernels -- the same bucket: storage types, channels, ratio, subsample mode, r', the single-kernel or
// chain form, the alignment classes that pick the vector and TMA kernels -- on the same slot share one
// executable graph.  The first request of a bucket on a slot is launched directly; later ones are captured
// on the slot stream, folded into the bucket's executable with cudaGraphExecUpdate (new grid sizes, pointers
// and arguments) and launched with one cudaGraphLaunch.  An executable is only updated once its previous
// launch has finished (its last node is the completion callback that frees the slot).  Measured on a GB300
// host (Grace) with the 512-request FP16 mix: capture, update and graph launch cost 28-34 us of host time per
// request against 18 us for launching the same work directly, at the same throughput, so direct launches are
// the default.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gf_internal.cuh"

namespace gfk {

double now_seconds()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

namespace {

// First-fit allocator over [0, size) with coalescing free list; offsets are 256-byte aligned.
class ArenaAllocator {
public:
    explicit ArenaAllocator(size_t size = 0) { reset(size); }
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
        size_ = size;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                in_use_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~size_t(255);
        in_use_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t in_use() const { return in_use_; }

private:
    std::map<size_t, size_t> free_;  // offset -> length
    size_t size_ = 0, in_use_ = 0;
};

enum ReqState { QUEUED, RUNNING, DONE, FAILED, CANCELED };

struct Request {
    uint64_t ticket;
    gf_request req;
    Resolved R;
    Layout L;
    ReqState state = QUEUED;
    gf_status status = GF_OK;
    size_t off = 0;
    int slot = -1;
    double t_submit = 0, t_admit = 0;
    std::atomic<double> t_done{0.0};
    std::atomic<int> finished{0};  // set by the stream callback
    struct Server *srv = nullptr;
    cudaEvent_t ready = nullptr;   // the caller's inputs are complete at this event (owned copy; may be NULL)
};

}  // namespace

struct Server {
    int device = 0;
    size_t budget = 0;
    int nslots = 4;
    size_t queue_limit = 4096;
    void *arena = nullptr;
    ArenaAllocator alloc;
    std::vector<cudaStream_t> streams;
    std::vector<uint64_t> slot_owner;  // ticket running on each slot, 0 = free
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false, started = false;
    std::thread thread;
    long long launches = 0, fault_launch = -1;
    bool paused = false;  // admission held (requests stay queued)
    unsigned *fault_host = nullptr;  // pinned, one word per slot: the fault word of the request on that slot
    cudaStream_t ready_stream = nullptr;  // where a request's ready event is captured at submission
    bool use_graphs = false;
    std::map<std::string, cudaGraphExec_t> graphs;  // bucket + slot -> executable graph
    std::map<std::string, int> seen;                // buckets launched once directly on a slot
    long long launched = 0;          // requests enqueued, how many through a graph, the host time spent
    long long graph_launched = 0;
    double launch_seconds = 0.0;
};

namespace {

// Stream callback after a request's kernels (and its fault-word copy).  It takes the server's lock before
// publishing completion, so the scheduler cannot retire the request -- after which gf_poll may free it --
// while the callback still uses it.  No CUDA call is made here.
void CUDART_CB on_done(void *arg)
{
    Request *r = static_cast<Request *>(arg);
    Server *s = r->srv;
    std::lock_guard<std::mutex> lock(s->mu);
    r->t_done.store(now_seconds());
    r->finished.store(1, std::memory_order_release);
    s->cv_sched.notify_all();
}

// The bucket of a request on a slot: everything that decides which kernels its launch sequence has.
std::string bucket_of(const Request &r, int slot)
{
    const Resolved &R = r.R;
    auto a16 = [](const void *p) { return (int)((reinterpret_cast<uintptr_t>(p) & 15u) == 0); };
    char key[256];
    snprintf(key, sizeof(key), "%d|%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d|%d %d %d %d %d|%d %d %d", slot, R.N, R.C,
             R.CI, R.s, R.sn, R.sd, R.mode, R.dt_in, R.dt_out, R.r_low, (int)R.fused, (int)R.color, (int)R.p_lowres,
             (int)(R.detail != 0.0f), (int)(r.req.opts.test_wait_fault != 0), R.W % 16, R.W % R.s, R.H % R.s,
             R.w % 4, (int)(r.req.I == r.req.p), a16(r.req.I), a16(r.req.p), a16(r.req.q));
    return key;
}

// Enqueue the request's work on its slot.  Called WITHOUT the server lock: the completion callback of an
// earlier request takes that lock, and no CUDA call may wait on a callback that waits on us.  Touches only the
// request, its slot's fault word and the scheduler's own graph tables.  Returns the launch status;
// *launched_some tells whether any work was enqueued before a failure, *via_graph whether it went through the
// bucket's graph.
gf_status launch_request(Server *s, Request &r, bool *launched_some, bool *via_graph)
{
    NvtxRange range("gf_serve launch");
    *launched_some = false;
    *via_graph = false;
    if (s->fault_launch >= 0 && s->launches++ == s->fault_launch) {  // injected: nothing is launched
        gf_set_error("injected launch failure (GF_FAULT)");
        return GF_ECUDA;
    }
    char *ws = (char *)s->arena + r.off;
    const FwdPlan P = make_plan(r.R, r.L, r.req.I, r.req.p, r.req.q, ws, &r.req.opts);
    cudaStream_t st = s->streams[r.slot];
    cudaError_t e = cudaSuccess;
    if (r.ready) {
        e = cudaStreamWaitEvent(st, r.ready, 0);  // the inputs are complete
        cudaEventDestroy(r.ready);                 // released once the wait has been resolved
        r.ready = nullptr;
    }
    if (e != cudaSuccess) {
        gf_set_error(std::string("serving launch: waiting for the request's ready event: ") + cudaGetErrorString(e));
        return GF_ECUDA;
    }
    *launched_some = true;
    s->fault_host[r.slot] = 0;
    // the request's work: its kernels, the copy of its fault word, the completion callback
    auto enqueue = [&]() {
        cudaError_t err = launch_forward(P, st);
        if (err == cudaSuccess && P.fault.call)
            err = cudaMemcpyAsync(&s->fault_host[r.slot], P.fault.call, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaLaunchHostFunc(st, on_done, &r);
        return err;
    };
    bool done = false;
    if (s->use_graphs) {
        const std::string key = bucket_of(r, r.slot);
        if (s->seen[key]++ > 0) {  // not the bucket's first request on this slot: through its graph
            cudaGraph_t g = nullptr;
            cudaError_t ec = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (ec == cudaSuccess) {
                ec = enqueue();
                cudaError_t ee = cudaStreamEndCapture(st, &g);
                if (ec == cudaSuccess) ec = ee;
            }
            if (ec == cudaSuccess && g) {
                cudaGraphExec_t &exec = s->graphs[key];
                if (exec) {
                    cudaGraphExecUpdateResultInfo info;
                    if (cudaGraphExecUpdate(exec, g, &info) != cudaSuccess) {  // not the same kernels after all
                        cudaGetLastError();
                        cudaGraphExecDestroy(exec);
                        exec = nullptr;
                    }
                }
                if (!exec) ec = cudaGraphInstantiate(&exec, g, 0);
                if (ec == cudaSuccess) {
                    ec = cudaGraphLaunch(exec, st);
                    done = (ec == cudaSuccess);
                    *via_graph = done;
                } else {
                    exec = nullptr;
                }
            }
            if (g) cudaGraphDestroy(g);
            if (!done) cudaGetLastError();  // nothing of the request was enqueued: launch it directly
        }
    }
    if (!done) e = enqueue();
    if (e != cudaSuccess) {
        gf_set_error(std::string("serving launch: ") + cudaGetErrorString(e));
        return GF_ECUDA;
    }
    return GF_OK;
}

void scheduler(Server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    std::vector<std::shared_ptr<Request>> admitted;
    while (true) {
        // retire finished requests: free their slot and scratch
        for (int k = 0; k < s->nslots; ++k) {
            const uint64_t t = s->slot_owner[k];
            if (!t) continue;
            auto &r = *s->reqs[t];
            if (r.finished.load(std::memory_order_acquire)) {
                r.state = DONE;
                if (s->fault_host[k] != 0) {  // a kernel of the request gave up a bounded wait: q is incomplete
                    r.state = FAILED;
                    r.status = GF_EWAIT;
                }
                s->alloc.release(r.off, r.L.total);
                s->slot_owner[k] = 0;
                s->cv_done.notify_all();
            }
        }
        // admit from the head of the queue while a slot is free and the scratch fits
        admitted.clear();
        while (!s->paused && !s->queue.empty()) {
            const uint64_t t = s->queue.front();
            auto it = s->reqs.find(t);
            if (it == s->reqs.end() || it->second->state != QUEUED) {
                s->queue.pop_front();
                continue;
            }
            Request &r = *it->second;
            int slot = -1;
            for (int k = 0; k < s->nslots; ++k)
                if (!s->slot_owner[k]) { slot = k; break; }
            if (slot < 0) break;
            size_t off;
            if (!s->alloc.alloc(r.L.total, &off)) break;  // wait for memory to free up
            s->queue.pop_front();
            r.off = off;
            r.slot = slot;
            r.t_admit = now_seconds();
            r.state = RUNNING;
            s->slot_owner[slot] = t;
            admitted.push_back(it->second);
        }
        // launch them with the lock released (their state is RUNNING: nothing else touches them meanwhile)
        if (!admitted.empty()) {
            struct Outcome {
                gf_status st;
                bool via_graph;
            };
            std::vector<Outcome> outcome(admitted.size());
            lock.unlock();
            double launch_s = 0.0;
            for (size_t k = 0; k < admitted.size(); ++k) {
                Request &r = *admitted[k];
                bool launched_some = false;
                const double t0 = now_seconds();
                outcome[k].st = launch_request(s, r, &launched_some, &outcome[k].via_graph);
                launch_s += now_seconds() - t0;
                if (outcome[k].st != GF_OK && launched_some) {
                    // work of the request may still be running: wait for it before the scratch is reused
                    cudaStreamSynchronize(s->streams[r.slot]);
                    cudaGetLastError();
                }
            }
            lock.lock();
            s->launched += (long long)admitted.size();
            s->launch_seconds += launch_s;
            for (size_t k = 0; k < admitted.size(); ++k) {
                Request &r = *admitted[k];
                s->graph_launched += outcome[k].via_graph ? 1 : 0;
                if (outcome[k].st == GF_OK) continue;
                r.state = FAILED;
                r.status = outcome[k].st;
                r.t_done.store(now_seconds());
                s->alloc.release(r.off, r.L.total);
                s->slot_owner[r.slot] = 0;
                s->cv_done.notify_all();
            }
            continue;  // requests may have finished meanwhile: retire and admit again before waiting
        }
        bool running = false;
        for (int k = 0; k < s->nslots; ++k) running |= (s->slot_owner[k] != 0);
        if (s->stop && !running) break;
        s->cv_sched.wait_for(lock, std::chrono::milliseconds(50));
    }
}

gf_status server_start(Server *s)
{
    if (s->started) return GF_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaError_t e = cudaMalloc(&s->arena, s->budget);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(prev);
        s->arena = nullptr;
        gf_set_error(std::string("serving arena of ") + std::to_string(s->budget) + " bytes: " + cudaGetErrorString(e));
        return GF_ENOMEM;
    }
    e = cudaHostAlloc((void **)&s->fault_host, sizeof(unsigned) * s->nslots, cudaHostAllocPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->arena);
        s->arena = nullptr;
        s->fault_host = nullptr;
        cudaSetDevice(prev);
        gf_set_error(std::string("serving fault words (pinned host memory): ") + cudaGetErrorString(e));
        return GF_ENOMEM;
    }
    for (int k = 0; k < s->nslots; ++k) s->fault_host[k] = 0;
    s->alloc.reset(s->budget);
    s->streams.resize(s->nslots);
    s->slot_owner.assign(s->nslots, 0);
    for (int k = 0; k < s->nslots; ++k) cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&s->ready_stream, cudaStreamNonBlocking);
    cudaSetDevice(prev);
    s->thread = std::thread(scheduler, s);
    s->started = true;
    return GF_OK;
}

}  // namespace

Server *server_create(int device, size_t budget)
{
    Server *s = new Server();
    s->device = device;
    s->budget = budget ? budget : (size_t(2) << 30);
    if (const char *f = getenv("GF_FAULT")) {
        if (strncmp(f, "launch:", 7) == 0) s->fault_launch = atoll(f + 7);
    }
    return s;
}

void server_destroy(Server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        for (auto &kv : s->reqs)
            if (kv.second->state == QUEUED) kv.second->state = CANCELED;
        s->queue.clear();
        s->cv_sched.notify_all();
    }
    if (s->thread.joinable()) s->thread.join();
    if (s->started) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(s->device);
        for (auto st : s->streams) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        if (s->ready_stream) cudaStreamDestroy(s->ready_stream);
        for (auto &kv : s->graphs)
            if (kv.second) cudaGraphExecDestroy(kv.second);
        if (s->arena) cudaFree(s->arena);
        if (s->fault_host) cudaFreeHost(s->fault_host);
        cudaSetDevice(prev);
    }
    for (auto &kv : s->reqs)
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    delete s;
}

gf_status server_config(Server *s, int slots, size_t queue_limit)
{
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->started) {
        gf_set_error("gf_serve_config must be called before the first gf_submit");
        return GF_EBUSY;
    }
    if (slots < 1 || slots > 64) {
        gf_set_error("slots must be in [1, 64]");
        return GF_EINVAL;
    }
    s->nslots = slots;
    if (queue_limit) s->queue_limit = queue_limit;
    return GF_OK;
}

gf_status server_submit(Server *s, const gf_request *req, uint64_t *ticket)
{
    if (!req || !ticket) {
        gf_set_error("req and ticket must not be NULL");
        return GF_EINVAL;
    }
    if (!req->I || !req->p || !req->q) {
        gf_set_error("request I, p and q must be device pointers");
        return GF_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->req = *req;
    r->req.opts.workspace = nullptr;
    r->req.opts.kernel_events = nullptr;
    r->req.opts.a_out = r->req.opts.b_out = r->req.opts.mean_a_out = r->req.opts.mean_b_out = nullptr;
    r->req.opts.stats_out = nullptr;
    gf_status st = resolve(req->H, req->W, req->C, req->r, req->eps, req->s, (int)req->mode, &r->req.opts, r->R);
    if (st != GF_OK) return st;
    r->L = layout_of(r->R, &r->req.opts);
    r->srv = s;
    std::lock_guard<std::mutex> lock(s->mu);
    if (r->L.total > s->budget) {
        gf_set_error("request scratch of " + std::to_string(r->L.total) + " bytes can never fit the serving budget of " +
                     std::to_string(s->budget) + " bytes");
        return GF_ENOMEM;
    }
    if (s->queue.size() >= s->queue_limit) {
        gf_set_error("serving queue is full");
        return GF_EBUSY;
    }
    if ((st = server_start(s)) != GF_OK) return st;
    if (req->ready_event) {
        // capture the caller's event as it stands now: an event of our own completes with it
        cudaError_t e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->ready_stream, (cudaEvent_t)req->ready_event, 0);
        if (e == cudaSuccess) e = cudaEventRecord(r->ready, s->ready_stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (r->ready) cudaEventDestroy(r->ready);
            gf_set_error(std::string("request ready_event: ") + cudaGetErrorString(e));
            return GF_ECUDA;
        }
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_seconds();
    s->reqs[r->ticket] = r;
    s->queue.push_back(r->ticket);
    *ticket = r->ticket;
    s->cv_sched.notify_all();
    return GF_OK;
}

gf_status server_poll(Server *s, uint64_t ticket, int64_t timeout_us, gf_result *out)
{
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        gf_set_error("unknown ticket");
        return GF_ENOTFOUND;
    }
    std::shared_ptr<Request> r = it->second;
    auto terminal = [&] { return r->state == DONE || r->state == FAILED || r->state == CANCELED; };
    if (!terminal() && timeout_us != 0) {
        if (timeout_us < 0)
            s->cv_done.wait(lock, terminal);
        else
            s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), terminal);
    }
    if (!terminal()) return timeout_us == 0 ? GF_PENDING : GF_ETIMEOUT;
    if (out) {
        out->status = r->state == CANCELED ? GF_ECANCELED : r->status;
        out->ticket = r->ticket;
        out->user = r->req.user;
        out->t_submit = r->t_submit;
        out->t_admit = r->t_admit;
        out->t_done = r->t_done.load();
        out->scratch_bytes = r->L.total;
    }
    const gf_status st = r->state == CANCELED ? GF_ECANCELED : r->status;
    if (r->ready) {  // never launched (cancelled)
        cudaEventDestroy(r->ready);
        r->ready = nullptr;
    }
    s->reqs.erase(it);  // a terminal result is delivered once
    if (st != GF_OK)
        gf_set_error(st == GF_ECANCELED ? "request was cancelled"
                     : st == GF_EWAIT   ? "request failed: a kernel gave up a bounded wait (q is incomplete)"
                                        : "request failed");
    return st;
}

gf_status server_cancel(Server *s, uint64_t ticket)
{
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        gf_set_error("unknown ticket");
        return GF_ENOTFOUND;
    }
    if (it->second->state != QUEUED) {
        gf_set_error("request is already running or finished");
        return GF_EBUSY;
    }
    it->second->state = CANCELED;
    s->cv_done.notify_all();
    return GF_OK;
}

gf_status server_graphs(Server *s, int enable)
{
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->started) {
        gf_set_error("gf_serve_graphs must be called before the first gf_submit");
        return GF_EBUSY;
    }
    s->use_graphs = enable != 0;
    return GF_OK;
}

gf_status server_pause(Server *s, int paused)
{
    std::lock_guard<std::mutex> lock(s->mu);
    s->paused = paused != 0;
    s->cv_sched.notify_all();
    return GF_OK;
}

gf_status server_stats(Server *s, gf_serve_stats *out)
{
    std::lock_guard<std::mutex> lock(s->mu);
    out->queued = 0;
    out->running = 0;
    for (auto &kv : s->reqs) {
        if (kv.second->state == QUEUED) ++out->queued;
        if (kv.second->state == RUNNING) ++out->running;
    }
    out->budget_bytes = s->budget;
    out->scratch_in_use = s->alloc.in_use();
    out->slots = s->nslots;
    out->launches = s->launched;
    out->graph_launches = s->graph_launched;
    out->launch_seconds = s->launch_seconds;
    return GF_OK;
}

}  // namespace gfk
