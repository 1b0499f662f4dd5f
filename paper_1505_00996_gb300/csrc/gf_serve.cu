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
// Tile queue (on unless gf_serve_tile_queue turns it off): when every slot is taken, requests small enough for
// the single-kernel form (gf_filter's fused path) that stand next to each other at the head of the queue and
// share storage types and subsample mode are admitted together onto the last free slot, up to 16 at a time,
// and run as ONE launch of the single kernel's tile-queue form: a grid over the (request, tile) items with per-request descriptors.  Each
// keeps its own scratch, fault word and completion callback, and each tile is computed exactly as the
// request's own launch computes it, so batching changes no result.
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
    size_t in_use() const { return in_use_; }

private:
    std::map<size_t, size_t> free_;  // offset -> length
    size_t in_use_ = 0;
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
    int bindex = 0;                // position in its slot's batch (its fault word's index)
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
    std::vector<uint64_t> slot_owner;  // first ticket running on each slot, 0 = free
    std::vector<std::vector<uint64_t>> slot_batch;  // every ticket running on each slot (tile-queue batches)
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false, started = false;
    std::thread thread;
    long long launches = 0, fault_launch = -1;
    bool paused = false;  // admission held (requests stay queued)
    unsigned *fault_host = nullptr;  // pinned, FUSED_QUEUE_MAX words per slot: the fault words of its requests
    cudaStream_t ready_stream = nullptr;  // where a request's ready event is captured at submission
    bool use_graphs = false;
    bool use_queue = true;           // tile-queue batches of single-kernel requests
    std::map<std::string, cudaGraphExec_t> graphs;  // bucket + slot -> executable graph
    std::map<std::string, int> seen;                // buckets launched once directly on a slot
    long long launched = 0;          // requests enqueued, how many through a graph, the host time spent
    long long graph_launched = 0;
    long long queue_launches = 0, queue_requests = 0;  // tile-queue launches and the requests they carried
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
    unsigned *fault_word = &s->fault_host[(size_t)r.slot * FUSED_QUEUE_MAX + r.bindex];
    *fault_word = 0;
    // the request's work: its kernels, the copy of its fault word, the completion callback
    auto enqueue = [&]() {
        cudaError_t err = launch_forward(P, st);
        if (err == cudaSuccess && P.fault.call)
            err = cudaMemcpyAsync(fault_word, P.fault.call, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
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

// Whether a request can join a tile-queue batch, and the key a batch's requests share (the kernel's template).
bool queueable(const Server *s, const Request &r)
{
    return s->use_queue && r.R.fused && !r.R.color && r.req.opts.test_wait_fault == 0;
}
long long queue_key(const Request &r) { return (long long)r.R.dt_in * 10000 + r.R.dt_out * 100 + r.R.mode; }

// Enqueue a tile-queue batch (requests of one slot, in admission order) as one launch.  Like launch_request:
// called without the server lock, touching only the batch's requests and their slot's fault words.  An
// injected failure (GF_FAULT) fails its own request, which then stays out of the launch.  Fills st[k] for each
// request; *launched_some tells whether any work was enqueued.
void launch_batch(Server *s, Request *const *b, int n, gf_status *st, bool *launched_some)
{
    NvtxRange range("gf_serve launch batch");
    *launched_some = false;
    const int slot = b[0]->slot;
    cudaStream_t stream = s->streams[slot];
    FwdPlan plans[FUSED_QUEUE_MAX];
    Request *in[FUSED_QUEUE_MAX];
    int m = 0;
    for (int k = 0; k < n; ++k) {
        Request &r = *b[k];
        st[k] = GF_OK;
        if (s->fault_launch >= 0 && s->launches++ == s->fault_launch) {  // injected: this request is left out
            st[k] = GF_ECUDA;
            continue;
        }
        if (r.ready) {
            const cudaError_t e = cudaStreamWaitEvent(stream, r.ready, 0);
            cudaEventDestroy(r.ready);
            r.ready = nullptr;
            if (e != cudaSuccess) {
                st[k] = GF_ECUDA;
                continue;
            }
            *launched_some = true;
        }
        s->fault_host[(size_t)slot * FUSED_QUEUE_MAX + r.bindex] = 0;
        plans[m] = make_plan(r.R, r.L, r.req.I, r.req.p, r.req.q, (char *)s->arena + r.off, &r.req.opts);
        in[m++] = &r;
    }
    if (m == 0) return;
    cudaError_t e = launch_fused_queue(plans, m, stream);
    if (e == cudaSuccess) *launched_some = true;
    for (int k = 0; k < m && e == cudaSuccess; ++k) {
        Request &r = *in[k];
        if (plans[k].fault.call)
            e = cudaMemcpyAsync(&s->fault_host[(size_t)slot * FUSED_QUEUE_MAX + r.bindex], plans[k].fault.call,
                                sizeof(unsigned), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(stream, on_done, &r);
    }
    if (e != cudaSuccess) {
        gf_set_error(std::string("serving launch (tile queue): ") + cudaGetErrorString(e));
        for (int k = 0; k < n; ++k)
            if (st[k] == GF_OK && !b[k]->finished.load()) st[k] = GF_ECUDA;
    }
}

void scheduler(Server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    std::vector<std::shared_ptr<Request>> admitted;
    while (true) {
        // retire finished requests (their scratch is freed); a slot is free once all of its batch is retired
        for (int k = 0; k < s->nslots; ++k) {
            if (!s->slot_owner[k]) continue;
            bool all = true;
            for (const uint64_t t : s->slot_batch[k]) {
                auto it = s->reqs.find(t);  // a retired request may have been polled and erased already
                if (it == s->reqs.end()) continue;
                auto &r = *it->second;
                if (r.state != RUNNING) continue;  // retired already (or failed at launch)
                if (!r.finished.load(std::memory_order_acquire)) {
                    all = false;
                    continue;
                }
                r.state = DONE;
                if (s->fault_host[(size_t)k * FUSED_QUEUE_MAX + r.bindex] != 0) {  // a bounded wait gave up
                    r.state = FAILED;
                    r.status = GF_EWAIT;
                }
                s->alloc.release(r.off, r.L.total);
                s->cv_done.notify_all();
            }
            if (all) {
                s->slot_owner[k] = 0;
                s->slot_batch[k].clear();
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
            r.bindex = 0;
            r.t_admit = now_seconds();
            r.state = RUNNING;
            s->slot_owner[slot] = t;
            s->slot_batch[slot].assign(1, t);
            admitted.push_back(it->second);
            // the tile queue: the requests right behind it that take the same single-kernel launch join its slot,
            // when no other slot is free for them (under light load every request keeps a slot of its own)
            if (!queueable(s, r)) continue;
            bool other_free = false;
            for (int k = 0; k < s->nslots; ++k) other_free |= (!s->slot_owner[k]);
            if (other_free) continue;
            while ((int)s->slot_batch[slot].size() < FUSED_QUEUE_MAX && !s->queue.empty()) {
                const uint64_t t2 = s->queue.front();
                auto it2 = s->reqs.find(t2);
                if (it2 == s->reqs.end() || it2->second->state != QUEUED) {
                    s->queue.pop_front();
                    continue;
                }
                Request &r2 = *it2->second;
                if (!queueable(s, r2) || queue_key(r2) != queue_key(r)) break;
                size_t off2;
                if (!s->alloc.alloc(r2.L.total, &off2)) break;
                s->queue.pop_front();
                r2.off = off2;
                r2.slot = slot;
                r2.bindex = (int)s->slot_batch[slot].size();
                r2.t_admit = now_seconds();
                r2.state = RUNNING;
                s->slot_batch[slot].push_back(t2);
                admitted.push_back(it2->second);
            }
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
            long long qlaunches = 0, qrequests = 0;
            for (size_t k = 0; k < admitted.size();) {
                Request &r = *admitted[k];
                size_t e = k + 1;  // the slot's batch: the admitted requests with the same slot, in order
                while (e < admitted.size() && admitted[e]->slot == r.slot) ++e;
                bool launched_some = false;
                const double t0 = now_seconds();
                if (e - k == 1) {
                    outcome[k].st = launch_request(s, r, &launched_some, &outcome[k].via_graph);
                } else {
                    Request *b[FUSED_QUEUE_MAX];
                    gf_status st[FUSED_QUEUE_MAX];
                    for (size_t j = k; j < e; ++j) b[j - k] = admitted[j].get();
                    launch_batch(s, b, (int)(e - k), st, &launched_some);
                    for (size_t j = k; j < e; ++j) outcome[j] = {st[j - k], false};
                    ++qlaunches;
                    qrequests += (long long)(e - k);
                }
                launch_s += now_seconds() - t0;
                bool failed = false;
                for (size_t j = k; j < e; ++j) failed |= (outcome[j].st != GF_OK);
                if (failed && launched_some) {
                    // work of the slot may still be running: wait for it before failed requests' scratch is reused
                    cudaStreamSynchronize(s->streams[r.slot]);
                    cudaGetLastError();
                }
                k = e;
            }
            lock.lock();
            s->launched += (long long)admitted.size();
            s->queue_launches += qlaunches;
            s->queue_requests += qrequests;
            s->launch_seconds += launch_s;
            for (size_t k = 0; k < admitted.size(); ++k) {
                Request &r = *admitted[k];
                s->graph_launched += outcome[k].via_graph ? 1 : 0;
                if (outcome[k].st == GF_OK) continue;
                r.state = FAILED;
                r.status = outcome[k].st;
                r.t_done.store(now_seconds());
                s->alloc.release(r.off, r.L.total);
                s->cv_done.notify_all();
            }
            // a slot none of whose requests is running any more is free (the retire pass covers the rest)
            for (size_t k = 0; k < admitted.size(); ++k) {
                const int slot = admitted[k]->slot;
                if (!s->slot_owner[slot]) continue;
                bool any = false;
                for (const uint64_t t : s->slot_batch[slot]) {
                    auto it = s->reqs.find(t);
                    any |= (it != s->reqs.end() && it->second->state == RUNNING);
                }
                if (!any) {
                    s->slot_owner[slot] = 0;
                    s->slot_batch[slot].clear();
                }
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
    e = cudaHostAlloc((void **)&s->fault_host, sizeof(unsigned) * s->nslots * FUSED_QUEUE_MAX, cudaHostAllocPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->arena);
        s->arena = nullptr;
        s->fault_host = nullptr;
        cudaSetDevice(prev);
        gf_set_error(std::string("serving fault words (pinned host memory): ") + cudaGetErrorString(e));
        return GF_ENOMEM;
    }
    for (int k = 0; k < s->nslots * FUSED_QUEUE_MAX; ++k) s->fault_host[k] = 0;
    s->alloc.reset(s->budget);
    s->streams.resize(s->nslots);
    s->slot_owner.assign(s->nslots, 0);
    s->slot_batch.assign(s->nslots, {});
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
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (r->L.total > s->budget) {
            gf_set_error("request scratch of " + std::to_string(r->L.total) +
                         " bytes can never fit the serving budget of " + std::to_string(s->budget) + " bytes");
            return GF_ENOMEM;
        }
        if ((st = server_start(s)) != GF_OK) return st;  // the first request: nothing is running yet
    }
    // The ready event is captured with the lock released: completion callbacks take the lock, and no CUDA
    // call is made while holding what a callback may be waiting for.
    if (req->ready_event) {
        // capture the caller's event as it stands now: an event of our own completes with it
        cudaError_t e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->ready_stream, (cudaEvent_t)req->ready_event, 0);
        if (e == cudaSuccess) e = cudaEventRecord(r->ready, s->ready_stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (r->ready) cudaEventDestroy(r->ready);
            r->ready = nullptr;
            gf_set_error(std::string("request ready_event: ") + cudaGetErrorString(e));
            return GF_ECUDA;
        }
    }
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->queue.size() >= s->queue_limit) {
        lock.unlock();
        if (r->ready) cudaEventDestroy(r->ready);
        r->ready = nullptr;
        gf_set_error("serving queue is full");
        return GF_EBUSY;
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
    cudaEvent_t unused_ready = r->ready;  // never launched (cancelled): destroyed below, outside the lock
    r->ready = nullptr;
    s->reqs.erase(it);  // a terminal result is delivered once
    lock.unlock();
    if (unused_ready) cudaEventDestroy(unused_ready);
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

gf_status server_queue(Server *s, int enable)
{
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->started) {
        gf_set_error("gf_serve_tile_queue must be called before the first gf_submit");
        return GF_EBUSY;
    }
    s->use_queue = enable != 0;
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
    out->queue_launches = s->queue_launches;
    out->queue_requests = s->queue_requests;
    out->launch_seconds = s->launch_seconds;
    return GF_OK;
}

}  // namespace gfk
