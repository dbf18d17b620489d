// rcm_internal.cuh -- device-side building blocks shared by the library's kernels: the control
// block, timer and memory-order helpers, and block-level scan/reduce helpers. Everything here is
// this library's own code (no CUB, no cooperative-groups grid sync), so every wait can carry an
// explicit time limit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rcm.h"

namespace rcm {

constexpr int kMaxGridBlocks = 1024;
constexpr int kIntMax = 0x7fffffff;
constexpr unsigned long long kKeyMax = ~0ull;

// Device-detected error bits (latched into the per-stream status by the host).
enum : int {
    kErrBadCsr = 1,     // malformed pattern
    kErrTimeout = 2,    // a bounded wait ran out
    kErrInternal = 4,   // an index guard tripped (never expected on valid input)
    kErrTooLarge = 8,   // a size beyond a fixed capacity
};

// Sites of the index guards that report through a diagnostic word (diag[0]; diag[1] holds the
// offending value).
enum : int {
    kSiteStart = 1,   // a component start vertex or first label out of range
    kSiteTable = 2,   // a component-table entry out of range (value: its index)
    kSiteParent = 3,  // a union-find parent path left the graph (value: the vertex)
    kSiteTotal = 4,   // component sizes do not add up to the vertices left (value: the sum)
    kSiteSize = 5,    // a component's ordering reached a different size than its table entry
    kSiteLevels = 6,  // a sweep ran more levels than the graph has vertices (value: the level)
};

// One CTA's slot of the grid exchange: flag = (epoch << 32) | count, written last with release.
struct alignas(32) ExSlot {
    unsigned long long flag;
    unsigned long long key;
    unsigned long long pad[2];
};

// Control block of one ordering: counters, the exchange slots, and the traversal state that
// CTA 0 publishes after running narrow levels alone.
struct alignas(128) Ctl {
    int status;
    int maxdeg;
    int nbig;              // rows longer than the per-thread sorter handles
    int work_next;         // next work item of a dynamic queue (batched engine)
    int qtail[3];          // ring of queue / staging tails, indexed by level
    int ncomp;             // connected components (counted before the traversal)
    unsigned int arrive;   // monotone arrival counter of the grid exchange
    // state published by CTA 0 at the end of a run of narrow levels
    int pub_F;       // current frontier size (0 = traversal finished)
    int pub_cur;     // which queue holds the frontier (levels-only sweeps)
    int pub_ecc;     // levels expanded so far (eccentricity once finished)
    int pub_start;   // label of the frontier's first vertex (labelled sweeps)
    int pub_lastF;   // size of the last non-empty level when finished
    int comp_count;  // component-table entries left to k_rcm_components (0 = none)
    int comp_nv;     // first label those components may take
    int cc_open;     // vertices still unnumbered when the component table is built
    unsigned long long pub_key;    // min (degree, id) key of the last level when finished
    long long pub_reached;         // vertices reached so far (levels-only sweeps)
    long long stats[8];            // rcm_stats fields, in order
    long long phase_ns[8];         // per-phase time of CTA 0 (profile_phases)
    ExSlot slots[2][kMaxGridBlocks];  // exchange slots, double-buffered by epoch parity
};

// Counters of the asynchronous levels-only sweep (one per ordering), each hot word on its own
// 128-byte line. proc[8 b] = items CTA b has finished, a monotone count published with release.
struct alignas(128) AsyncCtl {
    unsigned int head;       // next queue slot handed out (32 per warp)
    unsigned int pad0[31];
    unsigned long long tail; // queue slots reserved by producers
    unsigned long long pad1[15];
    int flag;                // bit 0: the sweep has finished; bit 1: the queue ran full
    int pad2[31];
    unsigned int proc[kMaxGridBlocks * 8];
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- distributed shared memory of a thread-block cluster ----

// This CTA's rank inside its cluster (0 for launches without clusters).
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// CTAs in this CTA's cluster (1 for launches without clusters).
__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Hardware barrier of every thread of the cluster (all threads of all its CTAs must arrive).
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared variable in the CTA of cluster rank `rank`.
__device__ __forceinline__ unsigned dsmem_addr(const void* local, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(local)), "r"(rank));
    return r;
}

__device__ __forceinline__ unsigned long long ld_acquire_cluster_u64(unsigned dsmem) {
    unsigned long long v;
    asm volatile("ld.acquire.cluster.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(dsmem) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_dsmem_u64(unsigned dsmem) {
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(dsmem) : "memory");
    return v;
}

// Release store to this CTA's own shared memory, at cluster scope: what this thread (and, through
// a preceding CTA barrier, its CTA) wrote before becomes visible to the cluster's threads that
// acquire the word.
__device__ __forceinline__ void st_release_cluster_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.cluster.shared::cta.u64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "l"(v)
                 : "memory");
}

// Coherent (L2) load for data written by other CTAs during this kernel.
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

// Bits of a 64-bit claim key left for the in-level order once the level number (at most n + 1)
// has its own high bits.
__host__ __device__ inline int claim_order_bits(long long n) {
    int dbits = 1;
    while ((1LL << dbits) < n + 2) ++dbits;
    return 64 - dbits;
}

__device__ __forceinline__ unsigned long long pack_key(int deg, int v) {
    return ((unsigned long long)(unsigned)deg << 32) | (unsigned)v;
}

// ---- block-level helpers (blockDim.x a multiple of 32, at most 1024) ----

__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of x over the CTA in thread order; *total receives the sum. smem: 64 ints used
// as two halves; callers alternate `parity` (0, 1, 0, ...) between consecutive calls, so one
// barrier suffices: a call writes the half that the previous call did not use, and every thread
// has finished reading a half before the barrier of the next call lets anyone overwrite it.
__device__ __forceinline__ int block_excl_scan(int x, int* total, int* smem, int parity) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int* half = smem + parity * 32;
    const int incl = warp_incl_scan(x);
    if (lane == 31) half[wid] = incl;
    __syncthreads();
    // every warp scans the warp totals itself: lane l holds total l
    const int t = lane < nw ? half[lane] : 0;
    const int ti = warp_incl_scan(t);
    const int before = wid > 0 ? __shfl_sync(0xffffffffu, ti, wid - 1) : 0;
    *total = __shfl_sync(0xffffffffu, ti, 31);
    return before + incl - x;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y < x ? y : x;
    }
    return x;
}

// Min over the CTA; every thread gets the result. smem: 32 u64.
__device__ __forceinline__ unsigned long long block_min_u64(unsigned long long x, unsigned long long* smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    x = warp_min_u64(x);
    if (lane == 0) smem[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long v = lane < nw ? smem[lane] : kKeyMax;
        v = warp_min_u64(v);
        if (lane == 0) smem[0] = v;
    }
    __syncthreads();
    unsigned long long r = smem[0];
    __syncthreads();
    return r;
}

}  // namespace rcm
