// rcm_single_kernels.cuh -- the one-graph kernels: k_rcm_single (the persistent grid engine) and
// k_rcm_small (one CTA with the graph's traversal state in shared memory), templated on the CTA
// width. Their definitions are compiled only in the translation units that instantiate them
// (rcm_kern_*.cu, built in parallel); everyone else sees declarations and extern instantiations.
#pragma once

#include "rcm_engine.cuh"
#include "rcm_internal.cuh"

namespace rcm {

// Graphs of at most kSmallMaxN vertices: one CTA orders the whole graph with its claims, visit
// stamps and padded rows in shared memory (Engine<true, true>), so every level's row reads and
// atomics stay inside one SM instead of going to L2.
constexpr int kSmallMaxN = 4608;
constexpr int kSmallSort = 256;  // component tables sorted in shared memory up to this size

// Shared-memory layout: claims (8n bytes) at 0, stamps (4n) and then the padded rows (32n, read
// and written as 16-byte int4) each at the next 16-byte boundary.
inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
inline size_t small_vis_off(int n) { return align16(8 * (size_t)n); }
inline size_t small_ell_off(int n) { return align16(small_vis_off(n) + 4 * (size_t)n); }
inline size_t small_smem_bytes(int n) { return small_ell_off(n) + 32 * (size_t)n; }

// kAsync: the engine with asynchronous levels-only sweeps; kBottomUp: the engine that may run
// whole-grid levels bottom-up. Both are instantiated for 512 threads only.
template <int kThreads, bool kAsync, bool kBottomUp>
__global__ void __launch_bounds__(kThreads, 1) k_rcm_single(EngineArgs args, int stall);
template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1) k_rcm_small(EngineArgs args, int vis_off, int ell_off);
template <int kThreads>
__global__ void __launch_bounds__(kThreads) k_rcm_components(EngineArgs args);
constexpr int kComponentThreads = 256;  // CTA width of k_rcm_components

#ifndef RCM_KERNEL_DEFINITIONS
extern template __global__ void k_rcm_single<32, false, false>(EngineArgs, int);
extern template __global__ void k_rcm_single<64, false, false>(EngineArgs, int);
extern template __global__ void k_rcm_single<128, false, false>(EngineArgs, int);
extern template __global__ void k_rcm_single<256, false, false>(EngineArgs, int);
extern template __global__ void k_rcm_single<512, false, false>(EngineArgs, int);
extern template __global__ void k_rcm_single<1024, false, false>(EngineArgs, int);
extern template __global__ void k_rcm_single<512, true, false>(EngineArgs, int);
extern template __global__ void k_rcm_single<512, false, true>(EngineArgs, int);
extern template __global__ void k_rcm_small<32>(EngineArgs, int, int);
extern template __global__ void k_rcm_small<64>(EngineArgs, int, int);
extern template __global__ void k_rcm_small<128>(EngineArgs, int, int);
extern template __global__ void k_rcm_small<256>(EngineArgs, int, int);
extern template __global__ void k_rcm_small<512>(EngineArgs, int, int);
extern template __global__ void k_rcm_components<kComponentThreads>(EngineArgs);
#else
template <int kThreads, bool kAsync, bool kBottomUp>
__device__ __forceinline__ void single_run(const EngineArgs& args, int stall, EngineSmem& smem, int& s_item,
                                           unsigned long long* s_sort) {
    Ctl* ctl = args.ctl;
    if (ld_volatile(&ctl->status) & kErrBadCsr) return;
    if (stall && blockIdx.x == 0) return;  // test hook: the other CTAs' first wait runs out
    const int n = args.n;
    Engine<false, false, kAsync, kBottomUp> e;
    e.init(args, &smem);
    // The middle tier reads its peers' shared memory, so it runs only where the launch's clusters
    // have the shape the host asked for (a profiler that relaunches the kernel may not keep it;
    // under one, a cluster launch faulted with Xid 13 before this check). Otherwise the levels run
    // without the tier: the same result. The cluster shape is the same on every CTA.
    if (args.mid_k > 0 && cluster_size() != (unsigned)args.mid_k) {
        if (threadIdx.x == 0) {
            smem.args.mid_k = 0;
            smem.args.mid_thr = 0;
        }
        __syncthreads();
    }
    if (args.hub_auto && ld_volatile(&ctl->maxdeg) > kHubDegree) {  // the same on every CTA
        if (threadIdx.x == 0) {
            smem.args.narrow_thr = min(smem.args.narrow_thr, kHubNarrow);
            smem.args.fused = 1;
        }
        __syncthreads();
    }
    int Z = 0;
    if (!e.label_isolated(Z)) return;
    e.stat_add(kStIsolated, Z);
    e.stat_add(kStComponents, Z);
    int nv = Z;
    int C = -1;
    // with cc_first the component table is built before any sweep (no probe from the first start)
    bool first = !args.cc_first, tried = false;
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
    // statistics: CTA 0 adds the grid part; k_rcm_components adds its own (ctl->stats starts at 0)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int i = 0; i < 8; ++i) {
            if (i == kStMaxEcc) atomicMax((unsigned long long*)&ctl->stats[i], (unsigned long long)smem.st[i]);
            else atomicAdd((unsigned long long*)&ctl->stats[i], (unsigned long long)smem.st[i]);
        }
        for (int i = 0; i < 8; ++i) ctl->phase_ns[i] = smem.prof[i];
    }
    // the components smaller than the whole grid: k_rcm_components, launched after this kernel
    if (C > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->comp_count = C;
        ctl->comp_nv = nv;
    }
}

template <int kThreads, bool kAsync, bool kBottomUp>
__global__ void __launch_bounds__(kThreads, 1) k_rcm_single(EngineArgs args, int stall) {
    __shared__ EngineSmem smem;
    __shared__ int s_item;
    extern __shared__ unsigned long long s_sort[];  // component-table sort (kCompSmem entries)
    // launched in clusters for the middle tier: every CTA's exchange words are cleared before any
    // peer can read them, and no CTA leaves while a peer may still read its shared memory (every
    // path of single_run ends: all its waits are bounded)
    if (args.mid_k > 0) {
        if (threadIdx.x == 0) smem.xc_flag[0] = smem.xc_flag[1] = 0ull;
        cluster_barrier();
    }
    single_run<kThreads, kAsync, kBottomUp>(args, stall, smem, s_item, s_sort);
    if (args.mid_k > 0) cluster_barrier();
}


// The components that k_rcm_single's component table left to smaller engines: those of at most
// kTinyMax vertices one per thread, the others (below the whole-grid size) one per CTA from a work
// queue, with CTA barriers only and their levels of at most kWarpLevel vertices on warp 0. A kernel
// of its own, so that neither its engine's code nor its CTA width weighs on the persistent grid
// kernel. Exits at once when the ordering built no table.
template <int kThreads>
__global__ void __launch_bounds__(kThreads) k_rcm_components(EngineArgs args) {
    __shared__ EngineSmem smem;
    __shared__ int s_item;
    Ctl* ctl = args.ctl;
    if (ld_volatile(&ctl->status) & (kErrBadCsr | kErrInternal | kErrTimeout | kErrTooLarge)) return;
    const int C = ctl->comp_count, nv = ctl->comp_nv;  // written by the previous kernel on this stream
    if (C <= 0) return;
    Engine<true, false, false, false, true> e;
    EngineArgs first = args;
    first.narrow_thr = 0x7fffffff;
    first.profile = 0;
    e.init(first, &smem);
    // visit stamps clear of the grid engine's (whose first sweep may have stamped a component)
    e.sweep_id = 1 << 24;
    // tiny components, one per thread of the grid, all at once
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
        const int4 t = __ldcg(args.cc_tab + i);
        if (t.z > kTinyMax || t.z >= args.cc_big) continue;
        if (!e.tab_ok(t, nv)) {
            e.fail_at(kSiteTable, i);
            break;
        }
        if (!e.order_tiny(t, args.qa + t.y, ctl->stats)) break;
    }
    // the others, one per CTA
    bool any = false;
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctl->work_next, 1);
        __syncthreads();
        const int i = s_item;
        __syncthreads();
        if (i >= C) break;
        const int4 t = __ldcg(args.cc_tab + i);
        if (t.z >= args.cc_big || t.z <= kTinyMax) continue;
        if (!e.tab_ok(t, nv)) {
            e.fail_at(kSiteTable, i);
            return;
        }
        EngineArgs ca = first;
        ca.qa = args.qa + t.y;
        ca.qb = args.qb + t.y;
        ca.boff = args.boff + t.y;
        ca.obits = claim_order_bits(t.z);
        if (threadIdx.x == 0) smem.args = ca;
        __syncthreads();
        any = true;
        int size;
        if (!e.component(t.x, t.y, size)) return;
        if (size != t.z) {
            e.fail(kErrInternal);
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

// kThreads: narrow graphs (a few dozen vertices per level) run best on small CTAs, whose barriers,
// scans and reductions are cheap.
template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1) k_rcm_small(EngineArgs args, int vis_off, int ell_off) {
    extern __shared__ __align__(16) unsigned long long s_state[];
    __shared__ EngineSmem smem;
    __shared__ unsigned long long s_sort[kSmallSort + kSmallSort / 2];
    Ctl* ctl = args.ctl;
    if (ld_volatile(&ctl->status) & kErrBadCsr) return;
    const int n = args.n;
    unsigned long long* claim = s_state;
    int* vis = (int*)((char*)s_state + vis_off);
    int4* ell = (int4*)((char*)s_state + ell_off);
    for (int i = threadIdx.x; i < n; i += kThreads) {
        claim[i] = kClaimNone;
        vis[i] = 0;
        ell[2 * i] = __ldg(args.ell + 2 * (size_t)i);
        ell[2 * i + 1] = __ldg(args.ell + 2 * (size_t)i + 1);
    }
    __syncthreads();
    EngineArgs a = args;
    a.claim = claim;
    a.vis = vis;
    a.ell = ell;
    Engine<true, true> e;
    e.init(a, &smem);
    e.sm_sort = s_sort;
    e.sm_sort_cap = kSmallSort;
    e.run();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 8; ++i) ctl->stats[i] = smem.st[i];
        for (int i = 0; i < 8; ++i) ctl->phase_ns[i] = smem.prof[i];
    }
}
#endif

}  // namespace rcm
