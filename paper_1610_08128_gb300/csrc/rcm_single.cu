// rcm_single.cu -- RCM ordering of one graph, host side: workspace layout, launch shape, and the
// launches (degree + validation, (degree, id)-sorted adjacency, then one persistent kernel that
// runs every sweep and every breadth-first level on the device; see rcm_single_kernels.cuh).
#include <algorithm>
#include <mutex>

#include "rcm_host.hpp"
#include "rcm_internal.cuh"
#include "rcm_prep.cuh"
#include "rcm_single.cuh"
#include "rcm_single_kernels.cuh"

namespace rcm {

// ------------------------------------------------------------------------------------------
// host side

// Components of at least this many vertices are ordered by the whole grid; smaller ones by one
// CTA each, concurrently.
constexpr int kComponentOnGrid = 1 << 18;

// Grids of at least this many CTAs label during every sweep by default (see single_launch).
constexpr int kLabelEverySweepBlocks = 64;

// with_cc: also the arrays of the concurrent-components pass (the fixed no-allocation workspace
// leaves them out and orders components one by one).
SingleLayout single_layout(long long n, long long nnz, bool with_cc, bool with_async, bool with_fkey) {
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
    L.adist = L.actl = L.fkey = 0;
    if (with_fkey) L.fkey = take(sizeof(unsigned long long) * (size_t)std::max(n, 1LL));
    if (with_async) {
        L.adist = take(sizeof(unsigned long long) * (size_t)std::max(n, 1LL));
        L.actl = take(sizeof(AsyncCtl));
    }
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

// CTAs per SM of each kernel: widths 32..1024 top-down (0..5), 512 with asynchronous sweeps (6),
// 512 with per-level bottom-up expansion (7)
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

// async: the instantiation with asynchronous levels-only sweeps; hybrid: the one with per-level
// bottom-up expansion (both 512 threads only)
static const void* single_kernel(int threads, bool async = false, bool hybrid = false) {
    if (async) return (const void*)k_rcm_single<512, true, false>;
    if (hybrid) return (const void*)k_rcm_single<512, false, true>;
    switch (threads) {
        case 32: return (const void*)k_rcm_single<32, false, false>;
        case 64: return (const void*)k_rcm_single<64, false, false>;
        case 128: return (const void*)k_rcm_single<128, false, false>;
        case 256: return (const void*)k_rcm_single<256, false, false>;
        case 1024: return (const void*)k_rcm_single<1024, false, false>;
    }
    return (const void*)k_rcm_single<512, false, false>;
}

constexpr int kSingleDynSmem = (int)((sizeof(unsigned long long) + sizeof(int)) * kCompSmem);

static int single_blocks_per_sm(int threads, bool async = false, bool hybrid = false) {
    std::lock_guard<std::mutex> g(g_single_mu);
    if ((async || hybrid) && threads != 512) return 0;
    const int idx = async ? 6 : hybrid ? 7 : threads_index(threads);
    if (idx < 0) return 0;  // not a supported block size (the options check rejects it first)
    if (g_single_blocks_per_sm[idx] < 0) {
        int b = 0;
        const void* k = single_kernel(threads, async, hybrid);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSingleDynSmem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, threads, kSingleDynSmem);
        g_single_blocks_per_sm[idx] = b;
        cudaFuncSetAttribute(k_sort_rows_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(unsigned long long) * kBigRowSmem));
    }
    return g_single_blocks_per_sm[idx];
}

static int g_cluster_max = -1;

int single_cluster_max() {
    if (single_blocks_per_sm(512) <= 0 || single_blocks_per_sm(512, true) <= 0 ||
        single_blocks_per_sm(512, false, true) <= 0)
        return 0;
    std::lock_guard<std::mutex> g(g_single_mu);
    if (g_cluster_max < 0) {
        g_cluster_max = 0;
        const void* k = single_kernel(512);
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(single_kernel(512, true), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(single_kernel(512, false, true), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        for (int c : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(c);
            cfg.blockDim = dim3(512);
            cfg.dynamicSmemBytes = kSingleDynSmem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = c;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) == cudaSuccess && clusters > 0) {
                g_cluster_max = c;
                break;
            }
            cudaGetLastError();
        }
    }
    return g_cluster_max;
}

// CTAs of the persistent grid (threads wide) that fit the device co-resident in whole clusters of
// k CTAs, launched cooperatively: 0 if the device cannot launch such clusters. Cached per shape.
static int g_mid_fit[8][5];
static int mid_cluster_fit(int threads, bool async, bool hybrid, int k) {
    const int kidx = k == 2 ? 0 : k == 4 ? 1 : k == 8 ? 2 : k == 16 ? 3 : -1;
    const int tidx = async ? 6 : hybrid ? 7 : threads_index(threads);
    if (kidx < 0 || tidx < 0) return 0;
    std::lock_guard<std::mutex> g(g_single_mu);
    if (g_mid_fit[tidx][kidx] == 0) {
        const void* kern = single_kernel(threads, async, hybrid);
        if (k > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(k);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = kSingleDynSmem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = k;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
            cudaGetLastError();
            clusters = 0;
        }
        g_mid_fit[tidx][kidx] = clusters > 0 ? clusters * k : -1;
    }
    return std::max(g_mid_fit[tidx][kidx], 0);
}

static std::once_flag g_small_once;
static cudaError_t g_small_attr = cudaSuccess;

static const void* small_kernel(int threads) {
    switch (threads) {
        case 32: return (const void*)k_rcm_small<32>;
        case 64: return (const void*)k_rcm_small<64>;
        case 128: return (const void*)k_rcm_small<128>;
        case 256: return (const void*)k_rcm_small<256>;
    }
    return (const void*)k_rcm_small<512>;
}

// CTA width of the shared-memory executor when the caller does not choose one.
// (256 was within a few percent of the best width on 2D and 3D grids and kNN meshes of 4,000
// vertices on GB300; the best ranged from 128 on long 2D grids to 512 on many-component meshes.)
static int small_default_threads(int) { return 256; }

rcm_status single_launch(int n, long long nnz, const rcm_options& o, SingleLaunch* out) {
    const DeviceInfo& di = device_info();
    SingleLaunch sl;
    // the shared-memory CTA engine: on request, or automatically for small graphs when no option
    // shapes the persistent grid
    const bool defaults = o.grid_blocks == 0 && o.cluster == 0 && o.narrow_threshold == 0 && o.block_threads == 0 &&
                          o.debug_stall_barrier == 0;
    if (o.executor == 2 || (o.executor == 0 && defaults && n <= kSmallMaxN)) {
        if (n > kSmallMaxN) return RCM_ERR_TOO_LARGE;
        const int t = o.block_threads ? o.block_threads : small_default_threads(n);
        if (t < 32 || t > 512) return RCM_ERR_INVALID_ARG;
        std::call_once(g_small_once, [] {
            for (int w : {32, 64, 128, 256, 512})
                if (g_small_attr == cudaSuccess)
                    g_small_attr = cudaFuncSetAttribute(small_kernel(w), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)small_smem_bytes(kSmallMaxN));
        });
        if (g_small_attr != cudaSuccess) return RCM_ERR_CUDA;
        single_blocks_per_sm(512);  // sets up the preprocessing kernels' attributes
        sl.small = true;
        sl.by_degree = o.row_order ? 0 : 1;
        sl.threads = t;
        sl.blocks = 1;
        sl.fused = o.fused_sweeps < 0 ? 0 : (o.fused_sweeps == 2 ? 2 : 1);
        sl.profile = o.profile_phases ? 1 : 0;
        *out = sl;
        return RCM_OK;
    }
    sl.threads = o.block_threads ? o.block_threads : 512;
    if (threads_index(sl.threads) < 0) return RCM_ERR_INVALID_ARG;
    sl.async = o.async_sweeps > 0;
    if (sl.async && sl.threads != 512) return RCM_ERR_INVALID_ARG;
    // per-level bottom-up expansion: on request, or automatically for patterns averaging at least
    // 8 stored entries per row (low-diameter graphs, whose frontiers grow wide); otherwise the
    // top-down kernel, which carries none of its code
    if (o.expand_mode >= 2 && (sl.threads != 512 || sl.async)) return RCM_ERR_INVALID_ARG;
    sl.hybrid = o.expand_mode >= 2 ||
                (o.expand_mode == 0 && sl.threads == 512 && !sl.async && nnz >= 8LL * (long long)n);
    const int per_sm = single_blocks_per_sm(sl.threads, sl.async, sl.hybrid);
    if (per_sm <= 0) return RCM_ERR_CUDA;
    sl.cluster = o.cluster != 0;
    if (o.mid_cluster > 0 && sl.cluster) return RCM_ERR_INVALID_ARG;
    if (sl.cluster) {
        // one cluster: only the 512-thread engine is set up for it
        const int cmax = sl.threads == 512 ? single_cluster_max() : 0;
        sl.blocks = o.grid_blocks ? o.grid_blocks : cmax;
        if (cmax == 0 || sl.blocks < 1 || sl.blocks > cmax) return RCM_ERR_INVALID_ARG;
    } else {
        const int max_blocks = std::min(per_sm * di.sms, kMaxGridBlocks);
        sl.blocks = o.grid_blocks ? o.grid_blocks : di.sms;
        if (sl.blocks < 1 || sl.blocks > max_blocks) return RCM_ERR_INVALID_ARG;
        if (o.mid_cluster > 0) {
            // the middle tier: whole clusters only, as many as fit co-resident
            const int k = o.mid_cluster;
            const int fit = mid_cluster_fit(sl.threads, sl.async, sl.hybrid, k);
            sl.blocks = std::min(sl.blocks, fit) / k * k;
            if (sl.blocks < k) return RCM_ERR_INVALID_ARG;
            sl.mid_k = k;
            // each member CTA takes a level share it handles in a fraction of a round: the tier is
            // bounded by its members' throughput (about 15 ns per vertex and CTA), not by its width
            sl.mid_thr = o.mid_threshold > 0 ? o.mid_threshold : 128 * k;
        }
    }
    // claim keys: (level + 1) in the high bits, the in-level order b * slot + j in the low obits;
    // slot = (2^obits - 1) / blocks must exceed any slice size (< n). A forced width (test hook)
    // skips the clamp; the kernel then checks every level's slices itself (RCM_ERR_TOO_LARGE).
    const int natural = claim_order_bits(n);
    if (o.debug_order_bits > natural) return RCM_ERR_INVALID_ARG;
    sl.obits = o.debug_order_bits > 0 ? o.debug_order_bits : natural;
    const unsigned long long slot_cap = ((1ull << sl.obits) - 1ull) / (unsigned long long)std::max(n, 1);
    if ((unsigned long long)sl.blocks > slot_cap && o.debug_order_bits == 0) {
        if (sl.cluster) return RCM_ERR_TOO_LARGE;
        sl.blocks = (int)std::max(1ull, slot_cap);
        if (sl.mid_k > 0) {  // whole clusters, or no middle tier
            sl.blocks = sl.blocks >= sl.mid_k ? sl.blocks / sl.mid_k * sl.mid_k : sl.blocks;
            if (sl.blocks < sl.mid_k) sl.mid_k = 0;
        }
    }
    // narrow runs keep the frontier in a shared-memory cache of kCache ids
    // default switch at the CTA width: for 512-thread CTAs it beat twice the width on every graph
    // measured on GB300 (the 192^3 grid 7.40 against 7.64 ms, a 1000^2 grid 19.1 against 24.3 ms)
    int narrow = o.narrow_threshold == 0 ? sl.threads : (o.narrow_threshold < 0 ? 0 : o.narrow_threshold);
    sl.narrow = std::min(narrow, kCache);
    sl.limit_ns = o.spin_limit_ns > 0 ? o.spin_limit_ns : 20000000000LL;
    // label during every sweep by default on a wide grid: there a labelled level is cheaper than a
    // levels-only one (GB300, 152 CTAs: the 192^3 grid 7.08 against 7.43 ms, a 1000^2 grid 17.7
    // against 18.6 ms, the 1.2M-point mesh 24.5 against 25.4 ms). On a few CTAs the extra work of
    // a labelled first sweep costs more than it saves (one cluster of 6: a 100^3 grid 8.6 against
    // 6.8 ms). Asynchronous sweeps are levels-only.
    sl.fused = o.fused_sweeps < 0 ? 0 : o.fused_sweeps == 1 ? 1 : o.fused_sweeps == 2 ? 2
             : (sl.async || sl.blocks < kLabelEverySweepBlocks) ? 1 : 2;
    // hub graphs (a vertex of more than kHubDegree neighbours) take a lower switch and levels-only
    // first sweeps, decided on the device, when the caller left both at their defaults
    sl.hub_auto = o.narrow_threshold == 0 && o.fused_sweeps == 0 && !sl.async ? 1 : 0;
    sl.cc_first = o.components_first > 0 ? 1 : 0;
    sl.profile = o.profile_phases ? 1 : 0;
    sl.stall = o.debug_stall_barrier ? 1 : 0;
    sl.l2_persist = o.l2_persist > 0;
    sl.async_slots = o.debug_async_slots;
    sl.by_degree = o.row_order ? 0 : 1;
    sl.expand_mode = o.expand_mode;
    sl.bu_divisor = o.bottom_up_divisor > 0 ? o.bottom_up_divisor : 16;
    *out = sl;
    return RCM_OK;
}

// The cooperative launch of the persistent grid with [win, win + bytes) -- the claim and stamp
// arrays, which every level's atomics hit at random -- marked persisting in L2, so that the rows
// streaming through L2 do not evict them. The context's persisting-L2 limit is raised to the
// window (clamped to the device maximum) on first use.
static cudaError_t launch_grid(const void* kernel, const SingleLaunch& sl, void** kargs, char* win, size_t bytes,
                               cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sl.blocks);
    cfg.blockDim = dim3(sl.threads);
    cfg.dynamicSmemBytes = kSingleDynSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[3];
    int na = 0;
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
    if (sl.mid_k > 0) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = sl.mid_k;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    if (sl.l2_persist) {
        // [win, win + bytes) -- the claim and stamp arrays, which every level's atomics hit at
        // random -- marked persisting in L2, so that the rows streaming through L2 do not evict
        // them; the context's persisting-L2 limit is raised to the window (clamped to the device
        // maximum), and order_single puts it back after the call
        int dev = 0, max_persist = 0, max_window = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev);
        if (e != cudaSuccess) return e;
        const size_t window = std::min(bytes, (size_t)max_window);
        const size_t persist = std::min(window, (size_t)max_persist);
        size_t cur = 0;
        e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
        if (e == cudaSuccess && cur < persist) e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, persist);
        if (e != cudaSuccess) return e;
        attr[na].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[na].val.accessPolicyWindow.base_ptr = win;
        attr[na].val.accessPolicyWindow.num_bytes = window;
        attr[na].val.accessPolicyWindow.hitRatio = window ? std::min(1.0f, (float)persist / (float)window) : 0.0f;
        attr[na].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[na].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelExC(&cfg, kernel, kargs);
}

// Reads one word of every 128-byte line of [p, p + words): launched with a normal-access window
// over the range, it turns the lines that a persisting window left in L2 back into normal ones,
// so that later kernels of the caller get the whole L2 again.
__global__ void k_l2_release(const int* __restrict__ p, size_t words) {
    const size_t stride = (size_t)gridDim.x * blockDim.x * 32;
    for (size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 32; i < words; i += stride) {
        int x;
        asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(x) : "l"(p + i) : "memory");
    }
}

static cudaError_t release_persisting(const char* win, size_t bytes, cudaStream_t s) {
    int dev = 0, max_window = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    if (e != cudaSuccess) return e;
    const size_t window = std::min(bytes, (size_t)max_window);
    const size_t words = window / sizeof(int);
    const DeviceInfo& di = device_info();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max<size_t>(1, std::min<size_t>((words / 32 + 255) / 256, (size_t)di.sms * 8)));
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow.base_ptr = (void*)win;
    attr[0].val.accessPolicyWindow.num_bytes = window;
    attr[0].val.accessPolicyWindow.hitRatio = 1.0f;
    attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
    attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int* p = (const int*)win;
    void* kargs[] = {(void*)&p, (void*)&words};
    return cudaLaunchKernelExC(&cfg, (const void*)k_l2_release, kargs);
}

// The components that the persistent kernel's component table leaves to smaller engines
// (k_rcm_components): as many threads as the traversal had, in CTAs of kComponentThreads. The
// kernel reads the table's size from the control block and exits at once when there is none.
static cudaError_t launch_components(EngineArgs& args, const SingleLaunch& sl, cudaStream_t s) {
    const int blocks = std::max(1, sl.blocks * sl.threads / kComponentThreads);
    void* cargs[] = {&args};
    return cudaLaunchKernel((const void*)k_rcm_components<kComponentThreads>, dim3(blocks), dim3(kComponentThreads),
                            cargs, 0, s);
}

cudaError_t enqueue_single(int n, long long nnz, const int* rowptr, const int* colidx, int* perm, char* base,
                           const SingleLayout& L, const SingleLaunch& sl, cudaEvent_t* ev, cudaStream_t s) {
    const DeviceInfo& di = device_info();
    Ctl* ctl = (Ctl*)(base + L.ctl);
    int* pool4 = (int*)(base + L.pool4);
    int* deg = (int*)(base + L.deg);
    unsigned long long* claim = (unsigned long long*)(base + L.claim);
    int* vis = (int*)(base + L.vis);
    int* bigrows = (int*)(base + L.bigrows);
    int* adj = (int*)(base + L.adj);
    int4* ell = (int4*)(base + L.ell);
    // the asynchronous sweeps need their words in the layout; without them the sweeps run level by level
    const bool async = sl.async && !sl.small && L.adist != 0;
    unsigned long long* adist = async ? (unsigned long long*)(base + L.adist) : nullptr;
    const bool hybrid = sl.hybrid && !sl.small && !async && L.fkey != 0;
    unsigned long long* fkey = hybrid ? (unsigned long long*)(base + L.fkey) : nullptr;

    cudaError_t e = cudaSuccess;
    if (ev) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess) {
        const int pb = 256;
        const int pgrid = (int)std::min<long long>((n + pb - 1) / pb, (long long)di.sms * 16);
        k_degree_validate<<<std::max(pgrid, 1), pb, 0, s>>>(n, (int)nnz, rowptr, colidx, deg, claim, vis, bigrows, ctl,
                                                           kSmallRowMax, adist, fkey);
        k_sort_rows_small<<<std::max(pgrid, 1), pb, 0, s>>>(n, rowptr, colidx, deg, adj, ell, ctl, kSmallRowMax,
                                                           sl.by_degree);
        // rows longer than kSmallRowMax entries number at most nnz / (kSmallRowMax + 1)
        const int big_grid = (int)std::max<long long>(1, std::min<long long>(3LL * di.sms, nnz / (kSmallRowMax + 1)));
        k_sort_rows_big<<<big_grid, kBigRowThreads, sizeof(unsigned long long) * kBigRowSmem, s>>>(
            n, rowptr, colidx, deg, adj, ell, bigrows, ctl, (unsigned long long*)pool4, sl.by_degree);
        e = cudaGetLastError();
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], s);
    }
    if (e != cudaSuccess) return e;
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
    args.narrow_thr = sl.narrow;
    args.obits = sl.obits > 0 ? sl.obits : claim_order_bits(n);
    args.profile = sl.profile;
    args.fused = sl.fused;
    args.hub_auto = sl.small ? 0 : sl.hub_auto;
    args.cc_first = sl.small ? 0 : sl.cc_first;
    args.limit_ns = sl.limit_ns;
    if (L.cc_cap > 0) {
        args.cc_parent = pool4 + 3 * (size_t)n;
        args.cc_size = (int*)(base + L.cc_size);
        args.cc_key = (unsigned long long*)(base + L.cc_key);
        args.cc_roots = (int*)(base + L.cc_roots);
        args.cc_gkey = (unsigned long long*)(base + L.cc_gkey);
        args.cc_gidx = (int*)(base + L.cc_gidx);
        args.cc_tab = (int4*)(base + L.cc_tab);
    } else {
        args.cc_parent = args.cc_size = args.cc_roots = args.cc_gidx = nullptr;
        args.cc_key = args.cc_gkey = nullptr;
        args.cc_tab = nullptr;
    }
    args.cc_cap = L.cc_cap;
    args.cc_big = kComponentOnGrid;
    // work queue of the asynchronous sweeps: pool4 as 2n 64-bit slots (the level-by-level
    // frontier buffers and the union-find parents are not in use while such a sweep runs)
    args.fkey = fkey;
    args.expand_mode = sl.expand_mode;
    args.bu_divisor = sl.bu_divisor;
    args.adist = adist;
    args.aq = async ? (unsigned long long*)pool4 : nullptr;
    args.actl = async ? (AsyncCtl*)(base + L.actl) : nullptr;
    long long slots = std::min<long long>(2LL * n, 1LL << 31);
    if (sl.async_slots > 0) slots = std::min<long long>(slots, sl.async_slots);
    args.aq_cap = async ? (unsigned)slots : 0u;
    args.mid_k = sl.small ? 0 : sl.mid_k;
    args.mid_thr = args.mid_k ? sl.mid_thr : 0;
    int stall = sl.stall;
    void* kargs[] = {&args, &stall};
    if (sl.small) {
        int vo = (int)small_vis_off(n), eo = (int)small_ell_off(n);
        void* sargs[] = {&args, &vo, &eo};
        e = cudaLaunchKernel(small_kernel(sl.threads), dim3(1), dim3(sl.threads), sargs, small_smem_bytes(n), s);
    } else if (sl.cluster) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(sl.blocks);
        cfg.blockDim = dim3(sl.threads);
        cfg.dynamicSmemBytes = kSingleDynSmem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = sl.blocks;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, single_kernel(sl.threads, async, hybrid), kargs);
    } else if (sl.l2_persist || sl.mid_k > 0) {
        e = launch_grid(single_kernel(sl.threads, async, hybrid), sl, kargs, base + L.claim, L.bigrows - L.claim, s);
        if (e == cudaSuccess) e = launch_components(args, sl, s);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
        if (e == cudaSuccess && sl.l2_persist) e = release_persisting(base + L.claim, L.bigrows - L.claim, s);
        return e;
    } else {
        e = cudaLaunchCooperativeKernel(single_kernel(sl.threads, async, hybrid), dim3(sl.blocks), dim3(sl.threads), kargs,
                                        kSingleDynSmem, s);
    }
    if (e == cudaSuccess && !sl.small) e = launch_components(args, sl, s);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], s);
    return e;
}

rcm_status order_single(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                        int32_t* perm, const rcm_options* opts, long long* stats_dev, cudaEvent_t* ev,
                        cudaStream_t s) {
    rcm_options o{};
    if (opts) o = *opts;
    SingleLaunch sl;
    rcm_status st = single_launch(n, nnz, o, &sl);
    if (st != RCM_OK) return st;
    const SingleLayout L = single_layout(n, nnz, true, sl.async && !sl.small, sl.hybrid && !sl.small);
    int* latch = stream_latch(s);
    if (!latch) return RCM_ERR_TOO_LARGE;  // every latch slot held by streams whose status is unread
    // the L2 window raises the context's persisting-L2 limit for the traversal; the call waits for
    // its work and puts the previous limit back (a raised limit slows the caller's later kernels)
    const bool window = sl.l2_persist && !sl.small && !sl.cluster;
    size_t prev_limit = 0;
    if (window && cudaDeviceGetLimit(&prev_limit, cudaLimitPersistingL2CacheSize) != cudaSuccess) return RCM_ERR_CUDA;
    void* ws = nullptr;
    st = ws_alloc(&ws, L.total, s);
    if (st != RCM_OK) return st;
    char* base = (char*)ws;
    cudaError_t e = enqueue_single(n, nnz, rowptr, colidx, perm, base, L, sl, ev, s);
    if (e == cudaSuccess) e = enqueue_latch((Ctl*)(base + L.ctl), latch, stats_dev, s);
    ws_free(ws, s);
    if (window) {
        const cudaError_t e2 = cudaStreamSynchronize(s);
        const cudaError_t e3 = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, prev_limit);
        if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    }
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
//
// That first call per device is also the set-up of everything else the path needs once: CUDA
// loads device code lazily (a module when one of its kernels or variables is first used), and
// loading it takes device memory. So the set-up loads every kernel the path can launch, and the
// host-side launch attributes of both executors, before the address is cached; later calls load
// nothing. (The first launch of the row sorter may also grow the context's local memory for its
// stack frame; every call launches it, so the first call does that too.)
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];

static rcm_status noalloc_setup() {
    const void* kernels[] = {(const void*)k_degree_validate, (const void*)k_sort_rows_small,
                             (const void*)k_sort_rows_big, small_kernel(small_default_threads(0)),
                             single_kernel(512)};
    for (const void* k : kernels) {
        cudaFuncAttributes fa;
        const cudaError_t e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return cuda_status(e);
    }
    // one-time attribute set-up of the shared-memory CTA and of the persistent grid
    SingleLaunch sl;
    rcm_status st = single_launch(1, 0, rcm_options{}, &sl);
    if (st == RCM_OK) st = single_launch(kSmallMaxN + 1, 0, rcm_options{}, &sl);
    return st;
}

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
        const rcm_status st = noalloc_setup();
        if (st != RCM_OK) return st;
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
    const SingleLayout L = single_layout(n, nnz, false, false, false);
    if (L.total > kNoAllocBytes) return RCM_ERR_TOO_LARGE;

    SingleLaunch sl;
    st = single_launch(n, nnz, rcm_options{}, &sl);
    if (st != RCM_OK) return st;
    char* base = (char*)ws;
    Ctl* ctl = (Ctl*)(base + L.ctl);
    // the array keeps the previous call's contents: enqueue_single clears the control block, and
    // its kernels initialise every per-vertex array they read
    e = enqueue_single(n, nnz, rowptr, colidx, perm, base, L, sl, nullptr, s);
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
