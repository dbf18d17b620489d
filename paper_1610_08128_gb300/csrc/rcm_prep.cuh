// rcm_prep.cuh -- declarations of the preprocessing and bandwidth/profile kernels.
#pragma once

#include "rcm_internal.cuh"

namespace rcm {

constexpr int kSmallRowMax = 32;     // rows with at most this many stored entries: per-thread sort
constexpr int kBigRowSmem = 8192;    // rows sorted in shared memory by one CTA (64 KB of keys)
constexpr int kBigRowThreads = 256;  // CTA width of k_sort_rows_big: 8 warps
constexpr int kWarpRowMax = kBigRowSmem / (kBigRowThreads / 32);  // rows sorted by one warp (its 8 KB slice)

// Padded row of vertex v: its first 7 neighbours in (degree, id) order (-1 where absent) and its
// degree in slot 7, as two 16-byte stores (one 32-byte sector per vertex).
__device__ __forceinline__ void store_ell(int4* ell, int v, const int (&r)[8]) {
    ell[2 * (size_t)v] = make_int4(r[0], r[1], r[2], r[3]);
    ell[2 * (size_t)v + 1] = make_int4(r[4], r[5], r[6], r[7]);
}

// Bitonic sort of P (a power of two) keys held in `s` (shared or global memory) by one CTA.
__device__ __forceinline__ void bitonic_sort_cta(unsigned long long* s, int P) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool asc = (i & k) == 0;
                    unsigned long long x = s[i], y = s[ixj];
                    if ((x > y) == asc) {
                        s[i] = y;
                        s[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Bitonic sort of P (a power of two, at most kWarpRowMax) keys in `s` by one warp.
__device__ __forceinline__ void bitonic_sort_warp(unsigned long long* s, int P) {
    const int lane = threadIdx.x & 31;
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool asc = (i & k) == 0;
                    unsigned long long x = s[i], y = s[ixj];
                    if ((x > y) == asc) {
                        s[i] = y;
                        s[ixj] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Degree of row v (off-diagonal entries) with the structural checks of the row; returns false if
// the row is malformed (bad bounds or a column outside [0, n)).
__device__ __forceinline__ bool row_degree(int n, int nnz, const int* __restrict__ rowptr,
                                           const int* __restrict__ colidx, int v, int& d) {
    const int a = rowptr[v], b = rowptr[v + 1];
    d = 0;
    if (a < 0 || b < a || b > nnz) return false;
    bool ok = true;
    for (int k = a; k < b; ++k) {
        const int w = colidx[k];
        if ((unsigned)w >= (unsigned)n) ok = false;
        else if (w != v) ++d;
    }
    return ok;
}

// Sort key of neighbour w, stored at position p of its row: (degree, id), or with by_degree = 0
// (the sort-free variant) its position, which keeps the stored order.
__device__ __forceinline__ unsigned long long row_key(const int* __restrict__ deg, int w, int p, int by_degree) {
    return pack_key(by_degree ? __ldg(deg + w) : p, w);
}

__device__ __forceinline__ void cmp_swap(unsigned long long& x, unsigned long long& y) {
    const unsigned long long lo = x < y ? x : y;
    y = x < y ? y : x;
    x = lo;
}

// Rows of at most 8 stored entries (every row of the grids and meshes): keys in registers, sorted
// by Batcher's 8-input odd-even merge network (19 compare-exchanges, no indexed local array).
// Absent and diagonal entries get the largest key and sort to the end. Keys are unique, so the
// order equals the insertion sort's.
__device__ __forceinline__ void sort_row8(int v, int a, int len, const int* __restrict__ colidx,
                                          const int* __restrict__ deg, int* __restrict__ adj,
                                          int4* __restrict__ ell, int by_degree) {
    unsigned long long k[8];
    int m = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        k[i] = kKeyMax;
        if (i < len) {
            const int w = colidx[a + i];
            if (w != v) {
                k[i] = row_key(deg, w, i, by_degree);
                ++m;
            }
        }
    }
    cmp_swap(k[0], k[1]); cmp_swap(k[2], k[3]); cmp_swap(k[4], k[5]); cmp_swap(k[6], k[7]);
    cmp_swap(k[0], k[2]); cmp_swap(k[1], k[3]); cmp_swap(k[4], k[6]); cmp_swap(k[5], k[7]);
    cmp_swap(k[1], k[2]); cmp_swap(k[5], k[6]);
    cmp_swap(k[0], k[4]); cmp_swap(k[1], k[5]); cmp_swap(k[2], k[6]); cmp_swap(k[3], k[7]);
    cmp_swap(k[2], k[4]); cmp_swap(k[3], k[5]);
    cmp_swap(k[1], k[2]); cmp_swap(k[3], k[4]); cmp_swap(k[5], k[6]);
    int r[8];
#pragma unroll
    for (int i = 0; i < 7; ++i) r[i] = i < m ? (int)(unsigned)(k[i] & 0xffffffffu) : -1;
    r[7] = m;
    store_ell(ell, v, r);
    if (m > 7) {
#pragma unroll
        for (int i = 0; i < 8; ++i) adj[a + i] = (int)(unsigned)(k[i] & 0xffffffffu);
    }
}

// Sorted row of a vertex with at most kSmallRowMax stored entries, by one thread: the padded row
// and, for degree > 7, the full sorted row in adj (same offsets as the input row).
__device__ __forceinline__ void sort_small_row(int v, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                               const int* __restrict__ deg, int* __restrict__ adj,
                                               int4* __restrict__ ell, int by_degree) {
    const int a = rowptr[v], b = rowptr[v + 1];
    if (b - a <= 8) {
        sort_row8(v, a, b - a, colidx, deg, adj, ell, by_degree);
        return;
    }
    unsigned long long key[kSmallRowMax];
    int m = 0;
    for (int k = a; k < b; ++k) {
        const int w = colidx[k];
        if (w == v) continue;
        const unsigned long long x = row_key(deg, w, k - a, by_degree);
        int j = m++;
        while (j > 0 && key[j - 1] > x) {
            key[j] = key[j - 1];
            --j;
        }
        key[j] = x;
    }
    int r[8];
#pragma unroll
    for (int i = 0; i < 7; ++i) r[i] = i < m ? (int)(unsigned)(key[i] & 0xffffffffu) : -1;
    r[7] = m;
    store_ell(ell, v, r);
    if (m > 7)
        for (int i = 0; i < m; ++i) adj[a + i] = (int)(unsigned)(key[i] & 0xffffffffu);
}

// nnz: the stored-entry count the caller sized its buffers for; rowptr[n] must equal it, and no
// row is read beyond it. adist, fkey (may be null): the asynchronous sweeps' per-vertex words
// (set to ~0) and the bottom-up frontier keys (set to 0). goff (may be null): a batch of G graphs
// stacked block-diagonally; every row's entries must then stay inside its graph's block.
__global__ void k_degree_validate(int n, int nnz, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                  int* __restrict__ deg, unsigned long long* __restrict__ claim, int* __restrict__ vis,
                                  int* __restrict__ bigrows, Ctl* ctl, int small_max,
                                  unsigned long long* __restrict__ adist = nullptr,
                                  unsigned long long* __restrict__ fkey = nullptr,
                                  const long long* __restrict__ goff = nullptr, int G = 0);

// small_max (<= kSmallRowMax): rows with at most this many stored entries are sorted here, one
// thread per row; k_degree_validate lists the longer ones for k_sort_rows_big with the same value.
// by_degree: 1 = rows in (degree, id) order; 0 = stored order (the sort-free variant).
__global__ void k_sort_rows_small(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                  const int* __restrict__ deg, int* __restrict__ adj, int4* __restrict__ ell,
                                  const Ctl* ctl, int small_max, int by_degree = 1);

__global__ void k_sort_rows_big(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                const int* __restrict__ deg, int* __restrict__ adj, int4* __restrict__ ell,
                                const int* __restrict__ bigrows, const Ctl* ctl,
                                unsigned long long* __restrict__ scratch, int by_degree = 1);

__global__ void k_bw_scatter(int n, const int* __restrict__ perm, int* __restrict__ pos, int* __restrict__ err);

__global__ void k_bw_rows(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                          const int* __restrict__ perm, const int* __restrict__ pos,
                          unsigned long long* __restrict__ out);

}  // namespace rcm
