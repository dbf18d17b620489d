// rcm_server.cu -- serving: ordering requests of mixed sizes admitted under an HBM budget and run
// concurrently on the GPU (continuous batching). The paper orders one matrix at a time; this
// subsystem only multiplies independent instances of the same method with the same tie rules.
//
//  * Admission: every request needs one contiguous region of a device arena allocated once at
//    server creation (budget bytes): its CSR (when given in host memory), its output (when the
//    caller's buffer is in host memory), a status word and the workspace of the ordering.
//    Requests are admitted in arrival order whenever a region and an in-flight slot are free; a
//    request larger than the whole budget is refused at submission (RCM_ERR_TOO_LARGE).
//  * Execution: each admitted request gets its own stream and one kernel launch of a single CTA
//    that validates and preprocesses the pattern and runs the whole ordering (Engine<true>), so
//    requests that arrive while others are on the GPU start as soon as they are admitted and run
//    side by side on different SMs.
//  * Completion: a host function enqueued after the result copy marks the request done, records
//    its completion time and frees its region and slot; a worker thread admits waiting requests.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rcm_engine.cuh"
#include "rcm_host.hpp"
#include "rcm_internal.cuh"
#include "rcm_prep.cuh"

namespace rcm {

constexpr int kReqThreads = 256;

// Device buffers of one request (all inside its arena region, or the caller's device memory).
struct ReqDesc {
    int n;
    int nnz;
    const int* rowptr;
    const int* colidx;
    int* perm;
    int* deg;
    unsigned long long* claim;
    int* vis;
    int* pool4;   // queues / offsets; scratch of the long-row sorter during preprocessing
    int* bigrows;
    int* adj;
    int4* ell;
    int* status;
};

// One CTA orders one request: validation + degrees, sorted rows, then the engine.
__global__ void __launch_bounds__(kReqThreads, 2) k_rcm_request(ReqDesc r) {
    extern __shared__ unsigned long long s_keys[];  // kBigRowSmem keys for long rows
    __shared__ EngineSmem smem;
    __shared__ int s_nbig, s_m;
    const int n = r.n;
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    const int nnz = r.rowptr[n];
    if (threadIdx.x == 0 && (r.rowptr[0] != 0 || nnz != r.nnz)) atomicOr(r.status, kErrBadCsr);
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        int d = 0;
        if (!row_degree(n, nnz, r.rowptr, r.colidx, v, d)) atomicOr(r.status, kErrBadCsr);
        else if (r.rowptr[v + 1] - r.rowptr[v] > kSmallRowMax) r.bigrows[atomicAdd(&s_nbig, 1)] = v;
        r.deg[v] = d;
        r.claim[v] = kClaimNone;
        r.vis[v] = 0;
    }
    __syncthreads();
    if (ld_volatile(r.status) & kErrBadCsr) return;
    for (int v = threadIdx.x; v < n; v += blockDim.x)
        if (r.rowptr[v + 1] - r.rowptr[v] <= kSmallRowMax) sort_small_row(v, r.rowptr, r.colidx, r.deg, r.adj, r.ell);
    const int nbig = s_nbig;
    for (int i = 0; i < nbig; ++i) {
        const int v = r.bigrows[i];
        int P = 1;
        while (P < r.deg[v]) P <<= 1;
        sort_big_row_cta(v, r.rowptr, r.colidx, r.deg, r.adj, r.ell,
                         P <= kBigRowSmem ? s_keys : (unsigned long long*)r.pool4, &s_m);
    }
    __syncthreads();
    EngineArgs a;
    a.n = n;
    a.v0 = 0;
    a.rowptr = r.rowptr;
    a.ell = r.ell;
    a.adj = r.adj;
    a.deg = r.deg;
    a.claim = r.claim;
    a.vis = r.vis;
    a.qa = r.pool4;
    a.qb = r.pool4 + n;
    a.boff = r.pool4 + 2 * (size_t)n;
    a.perm = r.perm;
    a.ctl = nullptr;
    a.status = r.status;
    a.narrow_thr = 0x7fffffff;
    a.fused = 1;
    a.obits = claim_order_bits(n);
    a.profile = 0;
    a.limit_ns = 0;
    a.cc_parent = a.cc_size = a.cc_roots = a.cc_gidx = nullptr;
    a.cc_key = a.cc_gkey = nullptr;
    a.cc_tab = nullptr;
    a.cc_cap = 0;
    a.cc_big = 0;
    Engine<true> e;
    e.init(a, &smem);
    e.run();
}

// Bytes of the request region: inputs/outputs that must be staged, status word, workspace.
static size_t request_bytes(long long n, long long nnz, bool stage_in, bool stage_out) {
    const size_t N = (size_t)std::max(n, 1LL), E = (size_t)std::max(nnz, 1LL);
    size_t o = 0;
    auto take = [&](size_t b) { o = align_up(o + b, 256); };
    if (stage_in) {
        take(sizeof(int) * (N + 1));
        take(sizeof(int) * E);
    }
    if (stage_out) take(sizeof(int) * N);
    take(256);                                  // status word
    take(sizeof(int) * N);                      // deg
    take(sizeof(unsigned long long) * N);       // claim
    take(sizeof(int) * N);                      // vis
    take(sizeof(int) * 4 * N);                  // pool4
    take(sizeof(int) * N);                      // bigrows
    take(sizeof(int) * E);                      // adj
    take(sizeof(int4) * 2 * N);                 // ell
    return o;
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
    size_t off = 0, bytes = 0;
    int slot = -1;
    int state = 0;  // 0 waiting, 1 running, 2 done
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
    int* h_status = nullptr;  // pinned, one word per slot
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> waiting;
    std::unordered_map<uint64_t, Request*> reqs;
    std::vector<double> latencies;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    long long submitted = 0, completed = 0, failed = 0, cancelled = 0;
    int running = 0, max_running = 0;
    cudaError_t worker_error = cudaSuccess;
};

static void CUDART_CB on_request_done(void* p) {
    Request* r = (Request*)p;
    Server* s = r->srv;
    std::lock_guard<std::mutex> g(s->mu);
    const int bits = *(volatile int*)&s->h_status[r->slot];
    r->status = r->status != RCM_OK ? r->status : status_from_bits(bits);
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
    ReqDesc d;
    d.n = r->n;
    d.nnz = (int)r->nnz;
    d.rowptr = rowptr;
    d.colidx = colidx;
    d.perm = perm;
    d.status = (int*)take(256);
    d.deg = (int*)take(sizeof(int) * N);
    d.claim = (unsigned long long*)take(sizeof(unsigned long long) * N);
    d.vis = (int*)take(sizeof(int) * N);
    d.pool4 = (int*)take(sizeof(int) * 4 * N);
    d.bigrows = (int*)take(sizeof(int) * N);
    d.adj = (int*)take(sizeof(int) * E);
    d.ell = (int4*)take(sizeof(int4) * 2 * N);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.status, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        k_rcm_request<<<1, kReqThreads, sizeof(unsigned long long) * kBigRowSmem, st>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && r->out_host)
        e = cudaMemcpyAsync(r->perm, perm, sizeof(int) * (size_t)r->n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s->h_status[r->slot], d.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_request_done, r);
    return e == cudaSuccess ? RCM_OK : cuda_status(e);
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
        s->cv.wait(lk);
    }
}

}  // namespace rcm

using namespace rcm;

struct rcm_server {
    Server s;
};

extern "C" {

rcm_status rcm_server_create(size_t hbm_budget_bytes, int32_t max_inflight, rcm_server** out) {
    if (!out || hbm_budget_bytes == 0 || max_inflight <= 0 || max_inflight > 4096) return RCM_ERR_INVALID_ARG;
    *out = nullptr;
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
    e = cudaHostAlloc((void**)&s.h_status, sizeof(int) * (size_t)max_inflight, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaFree(s.arena);
        delete srv;
        return cuda_status(e);
    }
    e = cudaFuncSetAttribute(k_rcm_request, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kBigRowSmem));
    s.alloc.reset(s.budget);
    s.max_inflight = max_inflight;
    s.streams.resize(max_inflight);
    for (int i = 0; i < max_inflight && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&s.streams[i], cudaStreamNonBlocking);
        s.free_slots.push_back(max_inflight - 1 - i);
    }
    if (e != cudaSuccess) {
        for (cudaStream_t st : s.streams)
            if (st) cudaStreamDestroy(st);
        cudaFreeHost(s.h_status);
        cudaFree(s.arena);
        delete srv;
        return cuda_status(e);
    }
    s.worker = std::thread(worker_loop, &s);
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
    r->bytes = request_bytes(n, nnz, r->in_host, r->out_host);
    r->srv = &s;
    r->t_submit = now_s();
    std::lock_guard<std::mutex> g(s.mu);
    if (s.stop) {
        delete r;
        return RCM_ERR_INVALID_ARG;
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
    delete r;
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
    if (s.worker.joinable()) s.worker.join();
    for (cudaStream_t st : s.streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto& kv : s.reqs) delete kv.second;
    s.reqs.clear();
    cudaFreeHost(s.h_status);
    cudaFree(s.arena);
    delete srv;
    return RCM_OK;
}

}  // extern "C"
