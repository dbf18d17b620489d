// rcm_single.cuh -- host-side pieces of the one-graph path (the persistent engine of
// rcm_single.cu), shared by rcm_order and the serving path.
#pragma once

#include "rcm_internal.cuh"

namespace rcm {

// Byte offsets of the one-graph workspace, each 256-byte aligned; total = bytes to allocate.
// cc_cap = components the concurrent-components pass handles (0 = that pass is off and the
// component arrays are absent).
// adist / actl: the asynchronous levels-only sweeps' distance words and counters (0 = absent; the
// sweeps' work queue reuses the frontier buffers of pool4).
// fkey: the bottom-up expansion's frontier keys (0 = absent: top-down only).
struct SingleLayout {
    size_t ctl, pool4, deg, claim, vis, bigrows, adj, ell, cc_size, cc_key, cc_roots, cc_gkey, cc_gidx, cc_tab,
        adist, actl, fkey, total;
    int cc_cap;
};
// with_async: include the asynchronous sweeps' arrays (only calls that ask for those sweeps).
// with_fkey: include the bottom-up frontier keys (the fixed no-allocation workspace leaves them out).
SingleLayout single_layout(long long n, long long nnz, bool with_cc = true, bool with_async = false,
                           bool with_fkey = true);

// Launch shape of the engine.
//   small = true:    one CTA holding the graph's claims, stamps and rows in shared memory.
//   cluster = false: a cooperative grid of `blocks` CTAs (at most the co-resident limit).
//   cluster = true:  one thread-block cluster of `blocks` CTAs (2..16); the hardware schedules a
//                    cluster's CTAs together, so they are co-resident whatever else runs.
struct SingleLaunch {
    int threads = 512;
    int blocks = 0;
    bool cluster = false;
    bool small = false;          // one CTA with the graph's state in shared memory (k_rcm_small)
    int narrow = 0;              // frontier size below which CTA 0 runs levels alone
    long long limit_ns = 20000000000LL;
    int fused = 1;               // 0 = separate labelled pass, 1 = labelled sweeps 2.., 2 = every sweep labelled
    int hub_auto = 0;            // frontier switch and fusing at their defaults: lowered on hub graphs
    int cc_first = 0;            // component table before the first sweep
    int profile = 0;
    int stall = 0;
    bool async = false;          // levels-only sweeps through the asynchronous work queue
    int async_slots = 0;         // its capacity (0 = 2n)
    int by_degree = 1;           // rows in (degree, id) order; 0 = stored order (sort-free variant)
    int expand_mode = 0;         // rcm_options.expand_mode
    bool hybrid = false;         // the kernel with per-level bottom-up expansion
    int bu_divisor = 16;         // bottom-up once the frontier holds n / bu_divisor vertices
    bool l2_persist = false;     // claims and stamps marked persisting in L2 for the engine's launch
    int obits = 0;               // width of the claim keys' in-level order field (0 = from n)
    int mid_k = 0;               // middle tier: the grid is launched in clusters of mid_k CTAs (0 = off)
    int mid_thr = 0;             // middle tier: levels below this size (and not narrow) run on cluster 0
};

// Derives the launch shape from options for a graph of n vertices and nnz stored entries;
// RCM_ERR_INVALID_ARG for unsupported shapes.
rcm_status single_launch(int n, long long nnz, const rcm_options& o, SingleLaunch* out);

// Largest cluster the engine can be launched as on this device (16 or 8), 0 if none.
int single_cluster_max();

// Enqueues on s, with the workspace at base (laid out by single_layout): control-block reset,
// degrees and checks (rowptr[n] == nnz), sorted rows, then the persistent engine. ev (optional):
// three events recorded before preprocessing, before the engine and after it.
cudaError_t enqueue_single(int n, long long nnz, const int* rowptr, const int* colidx, int* perm, char* base,
                           const SingleLayout& L, const SingleLaunch& sl, cudaEvent_t* ev, cudaStream_t s);

}  // namespace rcm
