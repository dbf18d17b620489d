// rcm_server.cu -- serving: ordering requests of mixed sizes admitted under an HBM budget and run
// concurrently on the GPU (continuous batching). The paper orders one matrix at a time; this
// subsystem only multiplies independent instances of the same method with the same tie rules.
//
//  * Admission: every request needs one contiguous region of a device arena allocated once at
//    server creation (budget bytes): its CSR (when given in host memory), its output (when the
//    caller's buffer is in host memory), a status word and the workspace of the ordering.
//    Requests are admitted in arrival order whenever a region and an in-flight slot are free; a
//    request larger than the whole budget is refused at submission (RCM_ERR_TOO_LARGE).
//  * Execution: each admitted request gets its own stream. Requests below kServeClusterMin
//    vertices run as a batch of one graph: the validation and sorted-row kernels, then the batched
//    executor with one CTA (Engine<true>, rcm_batch.cu). Larger ones run the persistent engine of
//    rcm_order (Engine<false>) launched as one thread-block cluster, whose CTAs the hardware
//    schedules together, so wide levels spread over several SMs. Requests that arrive while
//    others are on the GPU start as soon as they are admitted and run side by side.
//  * Completion: a host function enqueued after the result copy marks the request done, records
//    its completion time and frees its region and slot; a worker thread admits waiting requests.
//  * Failure: after a kernel fault the context is unusable and host functions behind the fault
//    never run. While requests run, the worker polls their streams; a stream error finishes every
//    running and waiting request with that error (and later submissions fail), so waiters return.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rcm_batch.cuh"
#include "rcm_host.hpp"
#include "rcm_internal.cuh"
#include "rcm_single.cuh"

namespace rcm {

// Requests of at least this many vertices run on a cluster of kServeClusterBlocks CTAs by default
// (see the header comment); the rest on one CTA of the batched executor. A cluster holds whole SMs
// (one 512-thread CTA each) through levels that leave them mostly idle, while a single CTA takes a
// third of an SM: on GB300, ordering a 1M-vertex 2D grid took 18 ms on a cluster of 6 and 32 ms on
// one CTA, about ten times the SM time. So clusters pay off only for the largest requests, whose
// latency they cut most. Measured on the 2,000 req/s trace (4,000 requests, pool of 256):
// clusters of 4 from 512k vertices 1,863/s, p50 27 ms, p99 159 ms; clusters of 6 from 256k
// vertices 1,789/s, 60 / 205 ms; no clusters 1,103/s, 688 / 1,519 ms.
constexpr long long kServeClusterMin = 1LL << 19;
constexpr int kServeClusterBlocks = 4;

// Arena bytes of one request: the staged CSR and result when they are in host memory, a 256-byte
// header holding the graph offsets {0, n} of a batch of one, and the larger of the two executors'
// workspaces (so the size is plain arithmetic on n and nnz).
static size_t request_bytes(long long n, long long nnz, bool stage_in, bool stage_out) {
    const size_t N = (size_t)std::max(n, 1LL), E = (size_t)std::max(nnz, 1LL);
    size_t o = 0;
    auto take = [&](size_t b) { o = align_up(o + b, 256); };
    if (stage_in) {
        take(sizeof(int) * (N + 1));
        take(sizeof(int) * E);
    }
    if (stage_out) take(sizeof(int) * N);
    take(256);  // graph offsets
    const long long n1 = std::max(n, 1LL), e0 = std::max(nnz, 0LL);
    return o + std::max(batch_layout(n1, e0).total, single_layout(n1, e0).total);
}

// First-fit allocator over [0, size) with coalescing (host-side bookkeeping of the arena).
class ArenaAlloc {
   public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

   private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, peak_ = 0;
};

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Server;

struct Request {
    uint64_t ticket;
    int n;
    long long nnz;
    const int* rowptr;
    const int* colidx;
    int* perm;
    bool in_host, out_host;
    bool out_pageable = false;   // result copied to pageable memory by the copier thread
    int* staged_perm = nullptr;  // the result inside the request's region (host outputs)
    size_t off = 0, bytes = 0;
    int slot = -1;
    int state = 0;  // 0 waiting, 1 running, 2 done
    bool orphan = false;  // finished by the failure path: its host function may still be pending
    rcm_status status = RCM_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    Server* srv = nullptr;
};

struct Server {
    int device = 0;
    size_t budget = 0;
    char* arena = nullptr;
    ArenaAlloc alloc;
    int max_inflight = 0;
    std::vector<cudaStream_t> streams;
    struct SlotHost* h_slots = nullptr;  // pinned, one per slot
    std::vector<Request*> slot_req;  // running request of each slot
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> waiting;
    std::unordered_map<uint64_t, Request*> reqs;
    std::vector<double> latencies;
    std::thread worker;
    // results bound for pageable host memory: copied by this thread (a synchronous copy would
    // stall the worker), which then completes the request
    std::thread copier;
    std::deque<Request*> to_copy;
    std::condition_variable ccv;
    bool copier_stop = false;
    cudaStream_t copy_stream = nullptr;
    bool stop = false;
    uint64_t next_ticket = 1;
    long long submitted = 0, completed = 0, failed = 0, cancelled = 0;
    int running = 0, max_running = 0;
    cudaError_t broken = cudaSuccess;  // first stream error seen: the context is unusable
    long long cluster_min = kServeClusterMin;  // -1: never
    int cluster_blocks = kServeClusterBlocks;
    int debug_fail_after = 0;                  // test hook (rcm_server_options)
    bool trace = false;                // RCM_TRACE_ERRORS set: failed requests are reported on stderr
};

// Pinned host words of one slot: the graph offsets copied in, the status word copied out.
struct alignas(64) SlotHost {
    long long goff[2];
    int status;
};

// Marks a running request done and frees its region and slot (caller holds the lock).
static void complete_locked(Server* s, Request* r) {
    s->slot_req[r->slot] = nullptr;
    r->t_done = now_s();
    r->state = 2;
    s->alloc.release(r->off, r->bytes);
    s->free_slots.push_back(r->slot);
    s->running--;
    s->completed++;
    if (r->status != RCM_OK) s->failed++;
    s->latencies.push_back(r->t_done - r->t_submit);
    s->cv.notify_all();
}

static void CUDART_CB on_request_done(void* p) {
    Request* r = (Request*)p;
    Server* s = r->srv;
    std::lock_guard<std::mutex> g(s->mu);
    if (r->state == 2) return;  // already finished by the failure path
    const int bits = *(const volatile int*)&s->h_slots[r->slot].status;
    r->status = r->status != RCM_OK ? r->status : status_from_bits(bits);
    if (s->trace && r->status != RCM_OK)
        std::fprintf(stderr, "rcm server: request %llu (n=%d, nnz=%lld) failed with device status bits %d\n",
                     (unsigned long long)r->ticket, r->n, r->nnz, bits);
    if (r->out_pageable && r->status == RCM_OK) {
        s->to_copy.push_back(r);  // the copier moves the result, then completes the request
        s->ccv.notify_one();
        return;
    }
    complete_locked(s, r);
}

static void copier_loop(Server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->ccv.wait(lk, [&] { return !s->to_copy.empty() || s->copier_stop; });
        if (s->to_copy.empty()) break;  // stopping, nothing left
        Request* r = s->to_copy.front();
        s->to_copy.pop_front();
        if (r->state == 2) continue;  // finished by the failure path meanwhile
        lk.unlock();
        cudaError_t e = cudaMemcpyAsync(r->perm, r->staged_perm, sizeof(int) * (size_t)r->n, cudaMemcpyDeviceToHost,
                                        s->copy_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
        lk.lock();
        if (r->state == 2) continue;
        if (e != cudaSuccess) r->status = cuda_status(e);
        complete_locked(s, r);
    }
}

// Enqueue the work of an admitted request on its slot's stream (caller holds no lock).
static rcm_status launch_request(Server* s, Request* r) {
    cudaStream_t st = s->streams[r->slot];
    char* base = s->arena + r->off;
    size_t o = 0;
    auto take = [&](size_t b) {
        char* p = base + o;
        o = align_up(o + b, 256);
        return p;
    };
    const size_t N = (size_t)std::max(r->n, 1), E = (size_t)std::max(r->nnz, 1LL);
    const int* rowptr = r->rowptr;
    const int* colidx = r->colidx;
    int* perm = r->perm;
    cudaError_t e = cudaSuccess;
    if (r->in_host) {
        int* d_rp = (int*)take(sizeof(int) * (N + 1));
        int* d_ci = (int*)take(sizeof(int) * E);
        e = cudaMemcpyAsync(d_rp, r->rowptr, sizeof(int) * ((size_t)r->n + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && r->nnz > 0)
            e = cudaMemcpyAsync(d_ci, r->colidx, sizeof(int) * (size_t)r->nnz, cudaMemcpyHostToDevice, st);
        rowptr = d_rp;
        colidx = d_ci;
    }
    if (r->out_host) perm = (int*)take(sizeof(int) * N);
    long long* d_goff = (long long*)take(256);
    char* ws = base + o;  // the workspace takes the rest of the region
    SlotHost* hs = &s->h_slots[r->slot];
    hs->status = 0;
    const int* status_dev = nullptr;
    if (s->cluster_min >= 0 && r->n >= s->cluster_min && single_cluster_max() > 0) {
        const SingleLayout L = single_layout(r->n, r->nnz);
        rcm_options o{};
        o.cluster = 1;
        o.grid_blocks = s->cluster_blocks;
        SingleLaunch sl;
        const rcm_status ls = single_launch(r->n, r->nnz, o, &sl);
        if (ls != RCM_OK) return ls;
        if (e == cudaSuccess) e = enqueue_single(r->n, r->nnz, rowptr, colidx, perm, ws, L, sl, nullptr, st);
        status_dev = (const int*)(ws + L.ctl + offsetof(Ctl, status));
    } else {
        const BatchLayout L = batch_layout(std::max(r->n, 1), std::max(r->nnz, 0LL));
        hs->goff[0] = 0;
        hs->goff[1] = r->n;
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_goff, hs->goff, sizeof(hs->goff), cudaMemcpyHostToDevice, st);
        const BatchTuning t;
        if (!batch_prepare(t)) return RCM_ERR_CUDA;
        if (e == cudaSuccess) e = enqueue_batch(1, r->n, (int)r->nnz, d_goff, nullptr, rowptr, colidx, perm, ws, L, t, st);
        status_dev = (const int*)(ws + L.ctl + offsetof(Ctl, status));
    }
    r->staged_perm = perm;
    if (e == cudaSuccess && r->out_host && !r->out_pageable)
        e = cudaMemcpyAsync(r->perm, perm, sizeof(int) * (size_t)r->n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs->status, status_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_request_done, r);
    return e == cudaSuccess ? RCM_OK : cuda_status(e);
}

// Finishes every running and waiting request with the stream error e (caller holds the lock).
// Running requests stay allocated: a host function of theirs that is already waiting for the
// lock returns without touching anything else once it sees them done.
static void fail_all(Server* s, cudaError_t e) {
    s->broken = e;
    const rcm_status st = cuda_status(e);
    const double t = now_s();
    for (int i = 0; i < s->max_inflight; ++i) {
        Request* r = s->slot_req[i];
        if (!r) continue;
        s->slot_req[i] = nullptr;
        r->status = st;
        r->state = 2;
        r->orphan = true;
        r->t_done = t;
        s->running--;
        s->completed++;
        s->failed++;
    }
    for (Request* r : s->waiting) {
        r->status = st;
        r->state = 2;
        r->t_done = t;
        s->completed++;
        s->failed++;
    }
    s->waiting.clear();
    s->cv.notify_all();
}

// Polls the streams of running requests; a stream error means a fault on the device (caller
// holds the lock, which is released around the queries).
static void check_streams(Server* s, std::unique_lock<std::mutex>& lk) {
    std::vector<int> slots;
    for (int i = 0; i < s->max_inflight; ++i)
        if (s->slot_req[i]) slots.push_back(i);
    lk.unlock();
    cudaError_t bad = cudaSuccess;
    for (int i : slots) {
        const cudaError_t e = cudaStreamQuery(s->streams[i]);
        if (e != cudaSuccess && e != cudaErrorNotReady) {
            bad = e;
            break;
        }
    }
    lk.lock();
    if (bad != cudaSuccess && s->broken == cudaSuccess) fail_all(s, bad);
}

static void worker_loop(Server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // admit waiting requests in arrival order while a region and a slot are free
        std::vector<Request*> admit;
        while (!s->waiting.empty() && !s->free_slots.empty()) {
            Request* r = s->waiting.front();
            size_t off;
            if (!s->alloc.alloc(r->bytes, &off)) break;
            s->waiting.pop_front();
            r->off = off;
            r->slot = s->free_slots.back();
            s->free_slots.pop_back();
            s->slot_req[r->slot] = r;
            r->state = 1;
            r->t_start = now_s();
            s->running++;
            s->max_running = std::max(s->max_running, s->running);
            admit.push_back(r);
        }
        if (!admit.empty()) {
            lk.unlock();
            for (Request* r : admit) {
                const rcm_status st = launch_request(s, r);
                if (st != RCM_OK) {
                    // nothing reached the GPU for this request, or part of it did: wait for its
                    // stream, then release it as failed
                    cudaStreamSynchronize(s->streams[r->slot]);
                    std::lock_guard<std::mutex> g(s->mu);
                    if (r->state == 2) continue;  // finished by the failure path meanwhile
                    s->slot_req[r->slot] = nullptr;
                    r->status = st;
                    r->state = 2;
                    r->t_done = now_s();
                    s->alloc.release(r->off, r->bytes);
                    s->free_slots.push_back(r->slot);
                    s->running--;
                    s->completed++;
                    s->failed++;
                    s->cv.notify_all();
                }
            }
            lk.lock();
            continue;
        }
        if (s->stop && s->waiting.empty() && s->running == 0) break;
        if (s->running > 0 && s->broken == cudaSuccess) {
            s->cv.wait_for(lk, std::chrono::milliseconds(20));
            check_streams(s, lk);
            if (s->debug_fail_after > 0 && s->completed >= s->debug_fail_after && s->running > 0 &&
                s->broken == cudaSuccess)
                fail_all(s, cudaErrorLaunchFailure);
        } else {
            s->cv.wait(lk);
        }
    }
}

}  // namespace rcm

using namespace rcm;

struct rcm_server {
    Server s;
};

extern "C" {

size_t rcm_request_bytes(int32_t n, int64_t nnz, int32_t host_csr, int32_t host_out) {
    if (n < 0 || nnz < 0) return 0;
    return request_bytes(n, nnz, host_csr != 0, host_out != 0);
}

rcm_status rcm_server_create(size_t hbm_budget_bytes, int32_t max_inflight, rcm_server** out) {
    return rcm_server_create_ex(hbm_budget_bytes, max_inflight, nullptr, out);
}

rcm_status rcm_server_create_ex(size_t hbm_budget_bytes, int32_t max_inflight, const rcm_server_options* opts,
                                rcm_server** out) {
    if (!out || hbm_budget_bytes == 0 || max_inflight <= 0 || max_inflight > 4096) return RCM_ERR_INVALID_ARG;
    *out = nullptr;
    if (opts && (opts->cluster_min_vertices < -1 || opts->cluster_blocks < 0 || opts->cluster_blocks > 16 ||
                 opts->cluster_blocks == 1 || opts->debug_fail_after < 0))
        return RCM_ERR_INVALID_ARG;
    rcm_server* srv = new (std::nothrow) rcm_server();
    if (!srv) return RCM_ERR_OOM;
    Server& s = srv->s;
    cudaGetDevice(&s.device);
    device_info();
    s.budget = align_up(hbm_budget_bytes, 256);
    cudaError_t e = cudaMalloc((void**)&s.arena, s.budget);
    if (e != cudaSuccess) {
        delete srv;
        return cuda_status(e);
    }
    e = cudaHostAlloc((void**)&s.h_slots, sizeof(SlotHost) * (size_t)max_inflight, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaFree(s.arena);
        delete srv;
        return cuda_status(e);
    }
    s.alloc.reset(s.budget);
    s.max_inflight = max_inflight;
    if (opts) {
        s.cluster_min = opts->cluster_min_vertices == 0 ? kServeClusterMin : opts->cluster_min_vertices;
        s.cluster_blocks = opts->cluster_blocks == 0 ? kServeClusterBlocks : opts->cluster_blocks;
        s.debug_fail_after = opts->debug_fail_after;
    }
    s.slot_req.assign(max_inflight, nullptr);
    s.trace = std::getenv("RCM_TRACE_ERRORS") != nullptr;
    s.streams.resize(max_inflight);
    for (int i = 0; i < max_inflight && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&s.streams[i], cudaStreamNonBlocking);
        s.free_slots.push_back(max_inflight - 1 - i);
    }
    if (e != cudaSuccess) {
        for (cudaStream_t st : s.streams)
            if (st) cudaStreamDestroy(st);
        cudaFreeHost(s.h_slots);
        cudaFree(s.arena);
        delete srv;
        return cuda_status(e);
    }
    e = cudaStreamCreateWithFlags(&s.copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (cudaStream_t st : s.streams)
            if (st) cudaStreamDestroy(st);
        cudaFreeHost(s.h_slots);
        cudaFree(s.arena);
        delete srv;
        return cuda_status(e);
    }
    s.worker = std::thread(worker_loop, &s);
    s.copier = std::thread(copier_loop, &s);
    *out = srv;
    return RCM_OK;
}

rcm_status rcm_submit(rcm_server* srv, int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                      int32_t* perm_out, uint64_t* ticket) {
    if (!srv || !ticket || n < 0 || nnz < 0 || nnz >= 0x7fffffffLL) return RCM_ERR_INVALID_ARG;
    if (n > 0 && (!rowptr || !perm_out || (nnz > 0 && !colidx))) return RCM_ERR_INVALID_ARG;
    Server& s = srv->s;
    auto is_device = [](const void* p) {
        cudaPointerAttributes at;
        if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    };
    Request* r = new (std::nothrow) Request();
    if (!r) return RCM_ERR_OOM;
    r->n = n;
    r->nnz = nnz;
    r->rowptr = rowptr;
    r->colidx = colidx;
    r->perm = perm_out;
    r->in_host = !is_device(rowptr);
    r->out_host = !is_device(perm_out);
    if (r->out_host) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, perm_out) != cudaSuccess) {
            cudaGetLastError();
            r->out_pageable = true;
        } else {
            r->out_pageable = at.type != cudaMemoryTypeHost;
        }
    }
    r->bytes = request_bytes(n, nnz, r->in_host, r->out_host);
    r->srv = &s;
    r->t_submit = now_s();
    std::lock_guard<std::mutex> g(s.mu);
    if (s.stop) {
        delete r;
        return RCM_ERR_INVALID_ARG;
    }
    if (s.broken != cudaSuccess) {
        delete r;
        return cuda_status(s.broken);
    }
    if (r->bytes > s.budget) {
        delete r;
        return RCM_ERR_TOO_LARGE;
    }
    r->ticket = s.next_ticket++;
    s.submitted++;
    if (n == 0) {  // nothing to order
        r->state = 2;
        r->t_start = r->t_done = r->t_submit;
        s.completed++;
        s.latencies.push_back(0.0);
    } else {
        s.waiting.push_back(r);
        s.cv.notify_all();
    }
    s.reqs[r->ticket] = r;
    *ticket = r->ticket;
    return RCM_OK;
}

static rcm_status finish(Server& s, std::unordered_map<uint64_t, Request*>::iterator it) {
    Request* r = it->second;
    const rcm_status st = r->status;
    s.reqs.erase(it);
    if (!r->orphan) delete r;  // an orphan's host function may still hold it (see fail_all)
    return st;
}

rcm_status rcm_poll(rcm_server* srv, uint64_t ticket) {
    if (!srv) return RCM_ERR_INVALID_ARG;
    Server& s = srv->s;
    std::lock_guard<std::mutex> g(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return RCM_ERR_UNKNOWN_TICKET;
    if (it->second->state != 2) return RCM_ERR_NOT_READY;
    return finish(s, it);
}

rcm_status rcm_wait(rcm_server* srv, uint64_t ticket) {
    if (!srv) return RCM_ERR_INVALID_ARG;
    Server& s = srv->s;
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return RCM_ERR_UNKNOWN_TICKET;
    // wait until the request is done, or until another thread consumed the ticket
    s.cv.wait(lk, [&] {
        auto jt = s.reqs.find(ticket);
        return jt == s.reqs.end() || jt->second->state == 2;
    });
    it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return RCM_ERR_UNKNOWN_TICKET;
    return finish(s, it);
}

rcm_status rcm_cancel(rcm_server* srv, uint64_t ticket) {
    if (!srv) return RCM_ERR_INVALID_ARG;
    Server& s = srv->s;
    std::lock_guard<std::mutex> g(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return RCM_ERR_UNKNOWN_TICKET;
    Request* r = it->second;
    if (r->state != 0) return RCM_ERR_NOT_READY;
    s.waiting.erase(std::find(s.waiting.begin(), s.waiting.end(), r));
    s.cancelled++;
    s.reqs.erase(it);
    delete r;
    return RCM_OK;
}

rcm_status rcm_server_info(rcm_server* srv, rcm_server_stats* out) {
    if (!srv || !out) return RCM_ERR_INVALID_ARG;
    Server& s = srv->s;
    std::lock_guard<std::mutex> g(s.mu);
    out->submitted = s.submitted;
    out->completed = s.completed;
    out->failed = s.failed;
    out->cancelled = s.cancelled;
    out->waiting = (int64_t)s.waiting.size();
    out->running = s.running;
    out->max_running = s.max_running;
    out->arena_bytes = (int64_t)s.budget;
    out->arena_peak_bytes = (int64_t)s.alloc.peak();
    std::vector<double> v = s.latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
    out->latency_p50_s = pct(0.50);
    out->latency_p99_s = pct(0.99);
    out->latency_max_s = v.empty() ? 0.0 : v.back();
    return RCM_OK;
}

rcm_status rcm_server_destroy(rcm_server* srv) {
    if (!srv) return RCM_ERR_INVALID_ARG;
    Server& s = srv->s;
    {
        std::lock_guard<std::mutex> g(s.mu);
        // requests that never started are dropped; running ones finish first
        for (Request* r : s.waiting) {
            s.reqs.erase(r->ticket);
            delete r;
        }
        s.waiting.clear();
        s.stop = true;
        s.cv.notify_all();
    }
    if (s.worker.joinable()) s.worker.join();  // returns once no request is running or waiting
    {
        std::lock_guard<std::mutex> g(s.mu);
        s.copier_stop = true;
        s.ccv.notify_all();
    }
    if (s.copier.joinable()) s.copier.join();
    if (s.copy_stream) cudaStreamDestroy(s.copy_stream);
    for (cudaStream_t st : s.streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto& kv : s.reqs)
        if (!kv.second->orphan) delete kv.second;
    s.reqs.clear();
    cudaFreeHost(s.h_slots);
    cudaFree(s.arena);
    delete srv;
    return RCM_OK;
}

}  // extern "C"
