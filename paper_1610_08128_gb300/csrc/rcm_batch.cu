// rcm_batch.cu -- batched ordering: G independent graphs stacked block-diagonally, ordered in one
// persistent launch. Each CTA pops graphs from a device work queue and runs the whole ordering of
// a graph with CTA barriers only (Engine<true>), so thousands of small graphs overlap on the GPU
// with no per-graph launch and no grid-wide barrier. The paper orders one matrix at a time; the
// batch only multiplies independent instances of the same method, with the same tie rules.
#include <algorithm>
#include <mutex>

#include "rcm_batch.cuh"
#include "rcm_cc.cuh"
#include "rcm_engine.cuh"
#include "rcm_host.hpp"
#include "rcm_internal.cuh"
#include "rcm_prep.cuh"

namespace rcm {

constexpr int kBatchSortCap = 2048;  // component tables sorted in shared memory up to this size

// CTAs per SM the batched executor is compiled for: many graphs are small, so occupancy matters
// more than registers (256 threads: 3 per SM at 80 registers measured faster than 4 at 64).
template <int kThreads>
constexpr int batch_min_blocks() { return kThreads >= 512 ? 2 : kThreads >= 256 ? 3 : 5; }

template <int kThreads>
__global__ void __launch_bounds__(kThreads, batch_min_blocks<kThreads>()) k_rcm_batch(BatchArgs b) {
    __shared__ EngineSmem smem;
    __shared__ int s_item;
    __shared__ unsigned long long s_sort[kBatchSortCap + kBatchSortCap / 2];
    if (ld_volatile(&b.ctl->status) & kErrBadCsr) return;
    Engine<true> e;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&b.ctl->work_next, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= b.G) break;
        const int g = b.order ? b.order[item] : item;
        const int v0 = (int)b.goff[g];
        const int n = (int)(b.goff[g + 1] - b.goff[g]);
        if (n == 0) continue;
        EngineArgs a;
        a.n = n;
        a.v0 = v0;
        a.rowptr = b.rowptr;
        a.ell = b.ell;
        a.adj = b.adj;
        a.deg = b.deg;
        a.claim = b.claim;
        a.vis = b.vis;
        a.qa = b.qa + v0;
        a.qb = b.qb + v0;
        a.boff = b.boff + v0;
        a.perm = b.perm + v0;
        a.ctl = b.ctl;
        a.status = &b.ctl->status;
        a.diag = nullptr;
        a.narrow_thr = 0x7fffffff;
        a.obits = claim_order_bits(n);
        a.profile = 0;
        a.cc_parent = b.cc_parent;
        a.cc_size = b.cc_size;
        a.cc_key = b.cc_key;
        a.cc_roots = b.cc_roots + v0;
        a.cc_gkey = b.cc_gkey + 2 * (size_t)v0;
        a.cc_gidx = b.cc_gidx + 2 * (size_t)v0;
        a.cc_tab = b.cc_tab + v0;
        a.cc_cap = n;
        a.cc_big = 0;
        a.fused = 1;
        a.hub_auto = 0;
        a.cc_first = 0;
        a.limit_ns = 0;
        a.fkey = nullptr;  // CTA engines: top-down, level by level
        a.expand_mode = 1;
        a.bu_divisor = 16;
        a.adist = nullptr;
        a.aq = nullptr;
        a.actl = nullptr;
        a.aq_cap = 0;
        a.mid_k = 0;  // CTA engines: no middle tier
        a.mid_thr = 0;
        __syncthreads();
        e.init(a, &smem);
        e.sm_sort = s_sort;
        e.sm_sort_cap = kBatchSortCap;
        if (!e.run()) return;
        __syncthreads();
        // the segment holds global ids while running; the result is in local ids
        for (int i = threadIdx.x; i < n; i += kThreads) a.perm[i] -= v0;
        __syncthreads();
    }
}

BatchLayout batch_layout(long long n_total, long long nnz, long long G) {
    const size_t N = (size_t)std::max<long long>(n_total, 1), E = (size_t)std::max<long long>(nnz, 1);
    BatchLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.ctl = take(sizeof(Ctl));
    L.pool = take(sizeof(int) * 4 * N);
    L.deg = take(sizeof(int) * N);
    L.claim = take(sizeof(unsigned long long) * N);
    L.vis = take(sizeof(int) * N);
    L.big = take(sizeof(int) * N);
    L.adj = take(sizeof(int) * E);
    L.ell = take(sizeof(int4) * 2 * N);
    L.ccs = take(sizeof(int) * N);
    L.cck = take(sizeof(unsigned long long) * N);
    L.ccr = take(sizeof(int) * N);
    L.ccgk = take(sizeof(unsigned long long) * 2 * N);
    L.ccgi = take(sizeof(int) * 2 * N);
    L.cct = take(sizeof(int4) * N);
    L.order = take(sizeof(int) * (size_t)std::max<long long>(G, 1));
    L.total = o;
    return L;
}

std::vector<int> batch_order(const std::vector<long long>& goff) {
    const int G = (int)goff.size() - 1;
    std::vector<int> order(std::max(G, 0));
    for (int i = 0; i < G; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return goff[x + 1] - goff[x] > goff[y + 1] - goff[y]; });
    return order;
}

static std::mutex g_batch_mu;
static int g_batch_per_sm[3] = {-1, -1, -1};  // CTAs per SM of the 128-, 256- and 512-thread executor

static int batch_index(int threads) { return threads == 128 ? 0 : threads == 256 ? 1 : threads == 512 ? 2 : -1; }

static const void* batch_kernel(int threads) {
    switch (threads) {
        case 128: return (const void*)k_rcm_batch<128>;
        case 512: return (const void*)k_rcm_batch<512>;
    }
    return (const void*)k_rcm_batch<256>;
}

static int batch_blocks_per_sm(int threads) {
    const int idx = batch_index(threads);
    if (idx < 0) return 0;
    std::lock_guard<std::mutex> g(g_batch_mu);
    if (g_batch_per_sm[idx] < 0) {
        int bps = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_kernel(threads), threads, 0);
        g_batch_per_sm[idx] = bps;
        cudaFuncSetAttribute(k_sort_rows_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kBigRowSmem));
    }
    return g_batch_per_sm[idx];
}

rcm_status batch_tuning(const rcm_batch_options* o, BatchTuning* out) {
    BatchTuning t;
    if (o) {
        if (o->block_threads) t.threads = o->block_threads;
        if (o->row_sort_split) t.small_max = o->row_sort_split;
        if (o->row_order != 0 && o->row_order != 1) return RCM_ERR_INVALID_ARG;
        t.by_degree = o->row_order ? 0 : 1;
    }
    if (batch_index(t.threads) < 0 || t.small_max < 4 || t.small_max > kSmallRowMax) return RCM_ERR_INVALID_ARG;
    *out = t;
    return RCM_OK;
}

bool batch_prepare(const BatchTuning& t) {
    device_info();
    return batch_blocks_per_sm(t.threads) > 0;
}

cudaError_t enqueue_batch(int G, long long n_total, int nnz, const long long* goff, const int* order,
                          const int* rowptr, const int* colidx, int* perm, char* base, const BatchLayout& L,
                          const BatchTuning& t, cudaStream_t s) {
    const DeviceInfo& di = device_info();
    const int per_sm = batch_blocks_per_sm(t.threads);
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const long long N = std::max<long long>(n_total, 1);
    Ctl* ctl = (Ctl*)(base + L.ctl);
    int* pool4 = (int*)(base + L.pool);
    int* deg = (int*)(base + L.deg);
    unsigned long long* claim = (unsigned long long*)(base + L.claim);
    int* vis = (int*)(base + L.vis);
    int* big = (int*)(base + L.big);
    int* adj = (int*)(base + L.adj);
    int4* ell = (int4*)(base + L.ell);
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
    if (e != cudaSuccess) return e;
    const int pb = 256;
    const int pgrid = (int)std::max<long long>(1, std::min<long long>((n_total + pb - 1) / pb, (long long)di.sms * 16));
    // rows longer than small_max entries number at most nnz / (small_max + 1)
    const int big_grid = (int)std::max<long long>(1, std::min<long long>(3LL * di.sms, nnz / (t.small_max + 1)));
    // one pass over the entries checks the structure and each graph's block (G > 1) and counts degrees
    k_degree_validate<<<pgrid, pb, 0, s>>>((int)n_total, nnz, rowptr, colidx, deg, claim, vis, big, ctl, t.small_max,
                                           nullptr, nullptr, G > 1 ? goff : nullptr, G);
    k_sort_rows_small<<<pgrid, pb, 0, s>>>((int)n_total, rowptr, colidx, deg, adj, ell, ctl, t.small_max,
                                           t.by_degree);
    k_sort_rows_big<<<big_grid, kBigRowThreads, sizeof(unsigned long long) * kBigRowSmem, s>>>(
        (int)n_total, rowptr, colidx, deg, adj, ell, big, ctl, (unsigned long long*)pool4, t.by_degree);
    BatchArgs b;
    b.G = G;
    b.goff = goff;
    b.order = order;
    b.rowptr = rowptr;
    b.ell = ell;
    b.adj = adj;
    b.deg = deg;
    b.claim = claim;
    b.vis = vis;
    b.qa = pool4;
    b.qb = pool4 + N;
    b.boff = pool4 + 2 * N;
    b.perm = perm;
    b.ctl = ctl;
    b.cc_parent = pool4 + 3 * N;
    b.cc_size = (int*)(base + L.ccs);
    b.cc_key = (unsigned long long*)(base + L.cck);
    b.cc_roots = (int*)(base + L.ccr);
    b.cc_gkey = (unsigned long long*)(base + L.ccgk);
    b.cc_gidx = (int*)(base + L.ccgi);
    b.cc_tab = (int4*)(base + L.cct);
    const int blocks = (int)std::min<long long>((long long)per_sm * di.sms, std::max(G, 1));
    void* kargs[] = {&b};
    return cudaLaunchKernel(batch_kernel(t.threads), dim3(blocks), dim3(t.threads), kargs, 0, s);
}

rcm_status order_batch(int32_t G, int64_t n_total, const int64_t* goff, const int32_t* rowptr,
                       const int32_t* colidx, int32_t* perm, const rcm_batch_options* opts, cudaStream_t s) {
    BatchTuning t;
    rcm_status st = batch_tuning(opts, &t);
    if (st != RCM_OK) return st;
    if (!batch_prepare(t)) return RCM_ERR_CUDA;
    // nnz sizes the sorted-adjacency copy and the graph sizes set the work-queue order: one
    // synchronised read of rowptr[n_total] and goff
    int nnz = 0;
    std::vector<long long> goff_h((size_t)G + 1);
    cudaError_t e = cudaMemcpyAsync(&nnz, rowptr + n_total, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(goff_h.data(), goff, sizeof(long long) * goff_h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (nnz < 0) return RCM_ERR_BAD_CSR;
    const BatchLayout L = batch_layout(n_total, nnz, G);
    int* latch = stream_latch(s);
    if (!latch) return RCM_ERR_TOO_LARGE;  // every latch slot held by streams whose status is unread
    void* ws = nullptr;
    st = ws_alloc(&ws, L.total, s);
    if (st != RCM_OK) return st;
    char* base = (char*)ws;
    // pageable source: the copy returns once the data is staged, so the vector may go
    const std::vector<int> order = batch_order(goff_h);
    e = cudaMemcpyAsync(base + L.order, order.data(), sizeof(int) * (size_t)G, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = enqueue_batch(G, n_total, nnz, (const long long*)goff, (const int*)(base + L.order), rowptr, colidx,
                          perm, base, L, t, s);
    if (e == cudaSuccess) e = enqueue_latch((Ctl*)(base + L.ctl), latch, nullptr, s);
    ws_free(ws, s);
    return e == cudaSuccess ? RCM_OK : cuda_status(e);
}

// Replay plan: the batched launches for fixed buffers, captured once into a CUDA graph.
struct BatchPlan {
    void* ws = nullptr;
    Ctl* ctl = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

rcm_status batch_plan_create(int32_t G, int64_t n_total, int64_t nnz, const int64_t* goff, const int32_t* rowptr,
                             const int32_t* colidx, int32_t* perm, const rcm_batch_options* opts, BatchPlan** out) {
    BatchTuning t;
    rcm_status st = batch_tuning(opts, &t);
    if (st != RCM_OK) return st;
    if (!batch_prepare(t)) return RCM_ERR_CUDA;
    BatchPlan* p = new (std::nothrow) BatchPlan();
    if (!p) return RCM_ERR_OOM;
    const BatchLayout L = batch_layout(n_total, nnz, G);
    cudaError_t e = cudaMalloc(&p->ws, L.total);
    // work-queue order (largest graph first) from the graph offsets at creation
    std::vector<long long> goff_h((size_t)G + 1);
    if (e == cudaSuccess) e = cudaMemcpy(goff_h.data(), goff, sizeof(long long) * goff_h.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        const std::vector<int> order = batch_order(goff_h);
        e = cudaMemcpy((char*)p->ws + L.order, order.data(), sizeof(int) * (size_t)G, cudaMemcpyHostToDevice);
    }
    cudaStream_t cs = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t ee = enqueue_batch(G, n_total, (int)nnz, (const long long*)goff,
                                             (const int*)((char*)p->ws + L.order), rowptr, colidx, perm,
                                             (char*)p->ws, L, t, cs);
        e = cudaStreamEndCapture(cs, &p->graph);
        if (e == cudaSuccess) e = ee;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        if (p->ws) cudaFree(p->ws);
        delete p;
        return cuda_status(e);
    }
    p->ctl = (Ctl*)((char*)p->ws + L.ctl);
    *out = p;
    return RCM_OK;
}

rcm_status batch_plan_launch(BatchPlan* p, cudaStream_t s) {
    const cudaError_t e = cudaGraphLaunch(p->exec, s);
    return e == cudaSuccess ? RCM_OK : cuda_status(e);
}

rcm_status batch_plan_status(BatchPlan* p, cudaStream_t s) {
    int bits = 0;
    cudaError_t e = cudaMemcpyAsync(&bits, &p->ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return status_from_bits(bits);
}

void batch_plan_destroy(BatchPlan* p) {
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->ws) cudaFree(p->ws);
    delete p;
}

}  // namespace rcm

struct rcm_batch_plan {
    rcm::BatchPlan* p;
};

extern "C" {

rcm_status rcm_batch_plan_create(int32_t G, int64_t n_total, int64_t nnz, const int64_t* goff,
                                 const int32_t* rowptr, const int32_t* colidx, int32_t* perm_out,
                                 const rcm_batch_options* opts, rcm_batch_plan** out) {
    if (!out || G <= 0 || n_total <= 0 || n_total >= 0x7fffffffLL || nnz < 0 || nnz >= 0x7fffffffLL)
        return RCM_ERR_INVALID_ARG;
    if (!goff || !rowptr || !perm_out || (nnz > 0 && !colidx)) return RCM_ERR_INVALID_ARG;
    *out = nullptr;
    rcm::BatchPlan* p = nullptr;
    const rcm_status st = rcm::batch_plan_create(G, n_total, nnz, goff, rowptr, colidx, perm_out, opts, &p);
    if (st != RCM_OK) return st;
    *out = new (std::nothrow) rcm_batch_plan{p};
    if (!*out) {
        rcm::batch_plan_destroy(p);
        return RCM_ERR_OOM;
    }
    return RCM_OK;
}

rcm_status rcm_batch_plan_launch(rcm_batch_plan* plan, rcm_stream_t stream) {
    if (!plan) return RCM_ERR_INVALID_ARG;
    return rcm::batch_plan_launch(plan->p, (cudaStream_t)stream);
}

rcm_status rcm_batch_plan_status(rcm_batch_plan* plan, rcm_stream_t stream) {
    if (!plan) return RCM_ERR_INVALID_ARG;
    return rcm::batch_plan_status(plan->p, (cudaStream_t)stream);
}

rcm_status rcm_batch_plan_destroy(rcm_batch_plan* plan) {
    if (!plan) return RCM_ERR_INVALID_ARG;
    rcm::batch_plan_destroy(plan->p);
    delete plan;
    return RCM_OK;
}

}  // extern "C"
