// rcm_single.cu -- RCM ordering of one graph: the preprocessing launches (degree + validation,
// (degree, id)-sorted adjacency) and one cooperative persistent kernel that runs every sweep and
// every breadth-first level on the device (Engine<false> in rcm_engine.cuh).
#include <algorithm>
#include <mutex>

#include "rcm_host.hpp"
#include "rcm_engine.cuh"
#include "rcm_internal.cuh"
#include "rcm_prep.cuh"

namespace rcm {

template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1) k_rcm_single(EngineArgs args, int stall) {
    __shared__ EngineSmem smem;
    __shared__ int s_item;
    extern __shared__ unsigned long long s_sort[];  // component-table sort (kCompSmem entries)
    Ctl* ctl = args.ctl;
    if (ld_volatile(&ctl->status) & kErrBadCsr) return;
    if (stall && blockIdx.x == 0) return;  // test hook: the other CTAs' first wait runs out
    const int n = args.n;
    Engine<false> e;
    e.init(args, &smem);
    int Z = 0;
    if (!e.label_isolated(Z)) return;
    e.stat_add(kStIsolated, Z);
    e.stat_add(kStComponents, Z);
    int nv = Z;
    int C = -1;
    bool first = true, tried = false;
    while (nv < n) {
        if (!first && !tried && args.cc_cap > 0) {
            // more than one component: order them concurrently (one attempt)
            tried = true;
            C = e.cc_prepare(nv, s_sort, kCompSmem);
            if (C == -2) return;
            if (C > 0) break;
        }
        unsigned long long k0;
        if (!e.next_start(k0)) return;
        if (k0 == kKeyMax) {
            e.fail(kErrInternal);
            return;
        }
        int size;
        // the first component's first sweep shows whether it spans everything left
        const long long left = (first && args.cc_cap > 0) ? (long long)(n - nv) : -1;
        first = false;
        if (!e.component((int)(unsigned)(k0 & 0xffffffffu), nv, size, left)) return;
        if (size < 0) continue;  // more components: the next iteration prepares them all
        nv += size;
    }
    if (C > 0) {
        // large components on the whole grid, one after another
        for (int i = 0; i < C; ++i) {
            const int4 t = __ldcg(args.cc_tab + i);
            if (!e.tab_ok(t, nv)) {
                e.fail_at(kSiteTable, i);
                return;
            }
            if (t.z < args.cc_big) continue;
            int size;
            if (!e.component(t.x, t.y, size)) return;
            if (size != t.z) {
                e.fail(kErrInternal);
                return;
            }
        }
    }
    // statistics: CTA 0 adds the grid part; CTAs add their own parts below (ctl->stats starts at 0)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i < 8; ++i) {
            if (i == kStMaxEcc) atomicMax((unsigned long long*)&ctl->stats[i], (unsigned long long)smem.st[i]);
            else atomicAdd((unsigned long long*)&ctl->stats[i], (unsigned long long)smem.st[i]);
        }
        for (int i = 0; i < 8; ++i) ctl->phase_ns[i] = smem.prof[i];
    }
    if (C <= 0) return;
    // the other components, one per CTA (CTA barriers only)
    __syncthreads();
    Engine<true> ec;
    bool any = false;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctl->work_next, 1);
        __syncthreads();
        const int i = s_item;
        __syncthreads();
        if (i >= C) break;
        const int4 t = __ldcg(args.cc_tab + i);
        if (!e.tab_ok(t, nv)) {
            e.fail_at(kSiteTable, i);
            return;
        }
        if (t.z >= args.cc_big) continue;
        EngineArgs ca = args;
        ca.qa = args.qa + t.y;
        ca.qb = args.qb + t.y;
        ca.boff = args.boff + t.y;
        ca.narrow_thr = 0x7fffffff;
        ca.obits = claim_order_bits(t.z);
        ca.profile = 0;
        if (!any) {
            ec.init(ca, &smem);
            // visit stamps of these engines stay clear of the grid engine's (whose first sweep may
            // already have stamped the first component)
            ec.sweep_id = 1 << 24;
            any = true;
        } else {
            __syncthreads();
            if (threadIdx.x == 0) smem.args = ca;
            __syncthreads();
        }
        int size;
        if (!ec.component(t.x, t.y, size)) return;
        if (size != t.z) {
            ec.fail(kErrInternal);
            return;
        }
    }
    if (any && threadIdx.x == 0) {
        for (int i = 0; i < 8; ++i) {
            if (i == kStMaxEcc) atomicMax((unsigned long long*)&ctl->stats[i], (unsigned long long)smem.st[i]);
            else if (i != kStIsolated && i != kStGrid) atomicAdd((unsigned long long*)&ctl->stats[i], (unsigned long long)smem.st[i]);
        }
    }
}


// ------------------------------------------------------------------------------------------
// host side

// Components of at least this many vertices are ordered by the whole grid; smaller ones by one
// CTA each, concurrently.
constexpr int kComponentOnGrid = 1 << 18;

struct SingleLayout {
    size_t ctl, pool4, deg, claim, vis, bigrows, adj, ell, cc_size, cc_key, cc_roots, cc_gkey, cc_gidx, cc_tab, total;
    int cc_cap;
};

// with_cc: also the arrays of the concurrent-components pass (the fixed no-allocation workspace
// leaves them out and orders components one by one).
static SingleLayout single_layout(long long n, long long nnz, bool with_cc = true) {
    SingleLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    L.ctl = take(sizeof(Ctl));
    L.pool4 = take(sizeof(int) * 4 * (size_t)std::max(n, 1LL));  // qa | qb | boff | spare; sort scratch in prep
    L.deg = take(sizeof(int) * (size_t)std::max(n, 1LL));
    L.claim = take(sizeof(unsigned long long) * (size_t)std::max(n, 1LL));
    L.vis = take(sizeof(int) * (size_t)std::max(n, 1LL));
    L.bigrows = take(sizeof(int) * (size_t)std::max(n, 1LL));
    L.adj = take(sizeof(int) * (size_t)std::max(nnz, 1LL));
    L.ell = take(sizeof(int4) * 2 * (size_t)std::max(n, 1LL));
    L.cc_cap = with_cc ? (int)std::min<long long>(std::max(n, 1LL), kMaxComps) : 0;
    if (!with_cc) {
        L.cc_size = L.cc_key = L.cc_roots = L.cc_gkey = L.cc_gidx = L.cc_tab = 0;
        L.total = o;
        return L;
    }
    long long cap2 = 1;
    while (cap2 < L.cc_cap) cap2 <<= 1;
    L.cc_size = take(sizeof(int) * (size_t)std::max(n, 1LL));
    L.cc_key = take(sizeof(unsigned long long) * (size_t)std::max(n, 1LL));
    L.cc_roots = take(sizeof(int) * (size_t)L.cc_cap);
    L.cc_gkey = take(sizeof(unsigned long long) * (size_t)cap2);
    L.cc_gidx = take(sizeof(int) * (size_t)cap2);
    L.cc_tab = take(sizeof(int4) * (size_t)L.cc_cap);
    L.total = o;
    return L;
}

static int g_single_blocks_per_sm[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
static std::mutex g_single_mu;

static int threads_index(int threads) {
    switch (threads) {
        case 32: return 0;
        case 64: return 1;
        case 128: return 2;
        case 256: return 3;
        case 512: return 4;
        case 1024: return 5;
    }
    return -1;
}

static const void* single_kernel(int threads) {
    switch (threads) {
        case 32: return (const void*)k_rcm_single<32>;
        case 64: return (const void*)k_rcm_single<64>;
        case 128: return (const void*)k_rcm_single<128>;
        case 256: return (const void*)k_rcm_single<256>;
        case 1024: return (const void*)k_rcm_single<1024>;
    }
    return (const void*)k_rcm_single<512>;
}

constexpr int kSingleDynSmem = (int)((sizeof(unsigned long long) + sizeof(int)) * kCompSmem);

static int single_blocks_per_sm(int threads) {
    std::lock_guard<std::mutex> g(g_single_mu);
    const int idx = threads_index(threads);
    if (idx < 0) return 0;  // not a supported block size (the options check rejects it first)
    if (g_single_blocks_per_sm[idx] < 0) {
        int b = 0;
        cudaFuncSetAttribute(single_kernel(threads), cudaFuncAttributeMaxDynamicSharedMemorySize, kSingleDynSmem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, single_kernel(threads), threads, kSingleDynSmem);
        g_single_blocks_per_sm[idx] = b;
        cudaFuncSetAttribute(k_sort_rows_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kBigRowSmem));
    }
    return g_single_blocks_per_sm[idx];
}

rcm_status order_single(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                        int32_t* perm, const rcm_options* opts, long long* stats_dev, cudaEvent_t* ev,
                        cudaStream_t s) {
    const DeviceInfo& di = device_info();
    rcm_options o{};
    if (opts) o = *opts;
    const int threads = o.block_threads ? o.block_threads : 512;
    if (threads_index(threads) < 0) return RCM_ERR_INVALID_ARG;
    const int per_sm = single_blocks_per_sm(threads);
    if (per_sm <= 0) return RCM_ERR_CUDA;
    const int max_blocks = std::min(per_sm * di.sms, kMaxGridBlocks);
    int blocks = o.grid_blocks ? o.grid_blocks : di.sms;
    if (blocks < 1 || blocks > max_blocks) return RCM_ERR_INVALID_ARG;
    // claim keys: (level + 1) in the high bits, the in-level order b * slot + j in the low obits;
    // slot = (2^obits - 1) / blocks must exceed any slice size (< n)
    const int obits = claim_order_bits(n);
    const unsigned long long slot_cap = ((1ull << obits) - 1ull) / (unsigned long long)std::max(n, 1);
    if ((unsigned long long)blocks > slot_cap) blocks = (int)std::max(1ull, slot_cap);
    // narrow runs keep the frontier in a shared-memory cache of kCache ids
    int narrow = o.narrow_threshold == 0 ? 2 * threads : (o.narrow_threshold < 0 ? 0 : o.narrow_threshold);
    narrow = std::min(narrow, kCache);
    const long long limit = o.spin_limit_ns > 0 ? o.spin_limit_ns : 20000000000LL;

    const SingleLayout L = single_layout(n, nnz);
    void* ws = nullptr;
    rcm_status st = ws_alloc(&ws, L.total, s);
    if (st != RCM_OK) return st;
    char* base = (char*)ws;
    Ctl* ctl = (Ctl*)(base + L.ctl);
    int* pool4 = (int*)(base + L.pool4);
    int* deg = (int*)(base + L.deg);
    unsigned long long* claim = (unsigned long long*)(base + L.claim);
    int* vis = (int*)(base + L.vis);
    int* bigrows = (int*)(base + L.bigrows);
    int* adj = (int*)(base + L.adj);
    int4* ell = (int4*)(base + L.ell);

    cudaError_t e = cudaSuccess;
    if (ev) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess) {
        const int pb = 256;
        const int pgrid = (int)std::min<long long>((n + pb - 1) / pb, (long long)di.sms * 16);
        k_degree_validate<<<std::max(pgrid, 1), pb, 0, s>>>(n, (int)nnz, rowptr, colidx, deg, claim, vis, bigrows, ctl,
                                                           kSmallRowMax);
        k_sort_rows_small<<<std::max(pgrid, 1), pb, 0, s>>>(n, rowptr, colidx, deg, adj, ell, ctl);
        // rows longer than kSmallRowMax entries number at most nnz / (kSmallRowMax + 1)
        const int big_grid = (int)std::max<long long>(1, std::min<long long>(2LL * di.sms, nnz / (kSmallRowMax + 1)));
        k_sort_rows_big<<<big_grid, 1024, sizeof(unsigned long long) * kBigRowSmem, s>>>(
            n, rowptr, colidx, deg, adj, ell, bigrows, ctl, (unsigned long long*)pool4);
        e = cudaGetLastError();
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    }
    if (e == cudaSuccess) {
        EngineArgs args;
        args.n = n;
        args.v0 = 0;
        args.rowptr = rowptr;
        args.ell = ell;
        args.adj = adj;
        args.deg = deg;
        args.claim = claim;
        args.vis = vis;
        args.qa = pool4;
        args.qb = pool4 + n;
        args.boff = pool4 + 2 * (size_t)n;
        args.perm = perm;
        args.ctl = ctl;
        args.status = &ctl->status;
        args.diag = nullptr;
        args.narrow_thr = narrow;
        args.obits = obits;
        args.profile = o.profile_phases ? 1 : 0;
        args.cc_parent = pool4 + 3 * (size_t)n;
        args.cc_size = (int*)(base + L.cc_size);
        args.cc_key = (unsigned long long*)(base + L.cc_key);
        args.cc_roots = (int*)(base + L.cc_roots);
        args.cc_gkey = (unsigned long long*)(base + L.cc_gkey);
        args.cc_gidx = (int*)(base + L.cc_gidx);
        args.cc_tab = (int4*)(base + L.cc_tab);
        args.cc_cap = L.cc_cap;
        args.cc_big = kComponentOnGrid;
        args.fused = o.fused_sweeps >= 0 ? 1 : 0;
        args.limit_ns = limit;
        int stall = o.debug_stall_barrier ? 1 : 0;
        void* kargs[] = {&args, &stall};
        e = cudaLaunchCooperativeKernel(single_kernel(threads), dim3(blocks), dim3(threads), kargs, kSingleDynSmem, s);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    }
    if (e == cudaSuccess) e = enqueue_latch(ctl, stream_latch(s), stats_dev, s);
    ws_free(ws, s);
    return e == cudaSuccess ? RCM_OK : cuda_status(e);
}

}  // namespace rcm

namespace rcm {

// ------------------------------------------------------------------------------------------
// Ordering without any device allocation.
//
// Some callers cannot allocate device memory while they run: an application whose memory
// framework has already reserved the device memory for its own caching allocator, or a solver
// loop with a fixed memory budget set at start-up in which an allocation could fail or stall
// the device. rcm_order_noalloc serves them: the whole workspace of the single-graph path lives
// in the file-scope device array below, so the call allocates nothing. The array holds the
// workspace of a pattern of at most kNoAllocMaxN vertices and kNoAllocMaxNnz stored entries
// (about 8 MiB), and every GPU that loads this library keeps it until the process exits.

constexpr int kNoAllocMaxN = 1 << 16;
constexpr long long kNoAllocMaxNnz = 1LL << 20;

constexpr size_t noalloc_take(size_t bytes) { return (bytes + 255) / 256 * 256; }
constexpr size_t kNoAllocBytes =
    noalloc_take(sizeof(Ctl)) + noalloc_take(sizeof(int) * 4 * (size_t)kNoAllocMaxN) +
    noalloc_take(sizeof(int) * (size_t)kNoAllocMaxN) + noalloc_take(sizeof(unsigned long long) * (size_t)kNoAllocMaxN) +
    noalloc_take(sizeof(int) * (size_t)kNoAllocMaxN) + noalloc_take(sizeof(int) * (size_t)kNoAllocMaxN) +
    noalloc_take(sizeof(int) * (size_t)kNoAllocMaxNnz) + noalloc_take(sizeof(int4) * 2 * (size_t)kNoAllocMaxN);

static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

// Device address of g_noalloc_ws on the current device. In host code the symbol itself is only a
// host-side stand-in, so the address is looked up once per device (with that device current)
// and cached.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];

static rcm_status noalloc_workspace(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= 64) return RCM_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_ws);
        if (e != cudaSuccess || !p) return e != cudaSuccess ? cuda_status(e) : RCM_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return RCM_OK;
}

rcm_status order_single_noalloc(int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t* perm,
                                cudaStream_t s) {
    if (n < 0) return RCM_ERR_INVALID_ARG;
    if (n == 0) return RCM_OK;
    if (!rowptr || !perm) return RCM_ERR_INVALID_ARG;
    if (n > kNoAllocMaxN) return RCM_ERR_TOO_LARGE;
    void* ws = nullptr;
    rcm_status st = noalloc_workspace(&ws);
    if (st != RCM_OK) return st;
    // stored-entry count: one 4-byte read into host stack memory
    int nnz = 0;
    cudaError_t e = cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (nnz < 0) return RCM_ERR_BAD_CSR;
    if (nnz > kNoAllocMaxNnz) return RCM_ERR_TOO_LARGE;
    if (nnz > 0 && !colidx) return RCM_ERR_INVALID_ARG;
    const SingleLayout L = single_layout(n, nnz, false);
    if (L.total > kNoAllocBytes) return RCM_ERR_TOO_LARGE;

    const DeviceInfo& di = device_info();
    const int threads = 512;
    const int per_sm = single_blocks_per_sm(threads);
    if (per_sm <= 0) return RCM_ERR_CUDA;
    int blocks = std::min(di.sms, std::min(per_sm * di.sms, kMaxGridBlocks));
    const int obits = claim_order_bits(n);
    const unsigned long long slot_cap = ((1ull << obits) - 1ull) / (unsigned long long)std::max(n, 1);
    if ((unsigned long long)blocks > slot_cap) blocks = (int)std::max(1ull, slot_cap);

    char* base = (char*)ws;
    Ctl* ctl = (Ctl*)(base + L.ctl);
    int* pool4 = (int*)(base + L.pool4);
    int* deg = (int*)(base + L.deg);
    unsigned long long* claim = (unsigned long long*)(base + L.claim);
    int* vis = (int*)(base + L.vis);
    int* bigrows = (int*)(base + L.bigrows);
    int* adj = (int*)(base + L.adj);
    int4* ell = (int4*)(base + L.ell);
    // the array keeps the previous call's contents: the control block must start at zero; every
    // other per-vertex array is initialised by the kernels below
    e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess) {
        const int pb = 256;
        const int pgrid = (int)std::min<long long>((n + pb - 1) / pb, (long long)di.sms * 16);
        k_degree_validate<<<std::max(pgrid, 1), pb, 0, s>>>(n, (int)nnz, rowptr, colidx, deg, claim, vis, bigrows, ctl,
                                                           kSmallRowMax);
        k_sort_rows_small<<<std::max(pgrid, 1), pb, 0, s>>>(n, rowptr, colidx, deg, adj, ell, ctl);
        // rows longer than kSmallRowMax entries number at most nnz / (kSmallRowMax + 1)
        const int big_grid = (int)std::max<long long>(1, std::min<long long>(2LL * di.sms, nnz / (kSmallRowMax + 1)));
        k_sort_rows_big<<<big_grid, 1024, sizeof(unsigned long long) * kBigRowSmem, s>>>(
            n, rowptr, colidx, deg, adj, ell, bigrows, ctl, (unsigned long long*)pool4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        EngineArgs args;
        args.n = n;
        args.v0 = 0;
        args.rowptr = rowptr;
        args.ell = ell;
        args.adj = adj;
        args.deg = deg;
        args.claim = claim;
        args.vis = vis;
        args.qa = pool4;
        args.qb = pool4 + n;
        args.boff = pool4 + 2 * (size_t)n;
        args.perm = perm;
        args.ctl = ctl;
        args.status = &ctl->status;
        args.diag = nullptr;
        args.narrow_thr = std::min(2 * threads, kCache);
        args.obits = obits;
        args.profile = 0;
        args.fused = 1;
        args.limit_ns = 20000000000LL;
        args.cc_parent = args.cc_size = args.cc_roots = args.cc_gidx = nullptr;
        args.cc_key = args.cc_gkey = nullptr;
        args.cc_tab = nullptr;
        args.cc_cap = 0;
        args.cc_big = 0;
        int stall = 0;
        void* kargs[] = {&args, &stall};
        e = cudaLaunchCooperativeKernel(single_kernel(threads), dim3(blocks), dim3(threads), kargs, kSingleDynSmem, s);
    }
    // synchronous: the device-detected status is read back from the control block
    int bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return status_from_bits(bits);
}

}  // namespace rcm

extern "C" rcm_status rcm_order_noalloc(int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t* perm_out,
                                        rcm_stream_t stream) {
    return rcm::order_single_noalloc(n, rowptr, colidx, perm_out, (cudaStream_t)stream);
}
