// rcm_batch.cuh -- the batched executor's arguments, its workspace layout and the enqueue step,
// shared by rcm_order_batch and the serving path (which runs each request as a batch of one).
#pragma once

#include <vector>

#include "rcm_internal.cuh"

namespace rcm {

struct BatchArgs {
    int G;
    const long long* goff;
    const int* order;  // graph of each work-queue position (largest first); null = index order
    // component tables: per-vertex arrays indexed by global id; per-graph lists at v0 (2 v0 for
    // the sort scratch)
    int* cc_parent;
    int* cc_size;
    unsigned long long* cc_key;
    int* cc_roots;
    unsigned long long* cc_gkey;
    int* cc_gidx;
    int4* cc_tab;
    const int* rowptr;
    const int4* ell;
    const int* adj;
    const int* deg;
    unsigned long long* claim;
    int* vis;
    int* qa;
    int* qb;
    int* boff;
    int* perm;
    Ctl* ctl;
};

// Byte offsets of the workspace of N vertices (all graphs together) and nnz stored entries, each
// 256-byte aligned; total = bytes to allocate.
struct BatchLayout {
    size_t ctl, pool, deg, claim, vis, big, adj, ell, ccs, cck, ccr, ccgk, ccgi, cct, order, total;
};
BatchLayout batch_layout(long long N, long long nnz, long long G = 1);

// Work-queue order of G graphs: largest first (ties by index), from the host copy of goff.
std::vector<int> batch_order(const std::vector<long long>& goff);

// Tuning of the batched path: CTA width of the executor (128, 256, 512) and the row length up to
// which one thread sorts a row (4..kSmallRowMax); every value gives the same result. by_degree = 0
// selects the sort-free variant (rows in stored order), which changes the result.
struct BatchTuning {
    int threads = 256;
    int small_max = 32;
    int by_degree = 1;
};
// RCM_OK and the tuning for the options, or RCM_ERR_INVALID_ARG.
rcm_status batch_tuning(const rcm_batch_options* o, BatchTuning* out);

// Enqueues on s, with the workspace at base (laid out by batch_layout(n_total, nnz)):
// control-block reset, structural checks (block structure when G > 1; rowptr[n_total] == nnz),
// degrees, sorted rows, then the batched engine. Device-detected errors land in the control block.
// Call batch_prepare(t) first (outside any stream capture).
// order: device, the work-queue order (G ints), or null for index order.
cudaError_t enqueue_batch(int G, long long n_total, int nnz, const long long* goff, const int* order,
                          const int* rowptr, const int* colidx, int* perm, char* base, const BatchLayout& L,
                          const BatchTuning& t, cudaStream_t s);
// One-time set-up of the kernels a tuning uses (attributes, occupancy); false on a CUDA error.
bool batch_prepare(const BatchTuning& t);

}  // namespace rcm
