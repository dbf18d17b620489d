// rcm_prep.cu -- per-graph preprocessing kernels and the bandwidth/profile kernels.
//
//  * k_degree_validate: D[v] = number of off-diagonal entries of row v (the degree vector D that
//    Alg. 3 and Alg. 4 take as input) plus the structural checks of the pattern.
//  * k_sort_rows_small / k_sort_rows_big: every row with the diagonal dropped and the neighbours in
//    increasing (degree, id), stored as a padded 32-byte row per vertex (7 neighbours + degree) and,
//    for rows of degree > 7, as a full sorted copy. (by_degree = 0: stored order instead, for the
//    sort-free variant.) Sorting each adjacency row once replaces the
//    per-level SortPerm of Sec. IV-B: when a frontier vertex scans its sorted row, the children it
//    owns come out already in (degree, id) order, so the new level is ordered by (parent label,
//    degree, id) by a prefix sum over parents alone.
//  * k_bw_scatter / k_bw_rows: bandwidth and profile of P A P^T (Sec. II-A).
#include "rcm_prep.cuh"

namespace rcm {

__global__ void k_degree_validate(int n, int nnz, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                  int* __restrict__ deg, unsigned long long* __restrict__ claim, int* __restrict__ vis,
                                  int* __restrict__ bigrows, Ctl* ctl, int small_max,
                                  unsigned long long* __restrict__ adist, unsigned long long* __restrict__ fkey,
                                  const long long* __restrict__ goff, int G) {
    __shared__ int s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rowptr[0] != 0 || rowptr[n] != nnz || nnz < 0))
        atomicOr(&ctl->status, kErrBadCsr);
    const int stride = gridDim.x * blockDim.x;
    if (goff) {  // a batch: goff must be non-decreasing from 0 to n
        if (blockIdx.x == 0 && threadIdx.x == 0 && (goff[0] != 0 || goff[G] != n)) atomicOr(&ctl->status, kErrBadCsr);
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += stride)
            if (goff[g + 1] < goff[g]) atomicOr(&ctl->status, kErrBadCsr);
    }
    // A warp takes 32 consecutive rows. In a batch, every entry of a row must stay inside its
    // graph's block [goff[g], goff[g+1]): lane 0 finds the graph of the warp's first row (binary
    // search) and every lane steps forward from there to its own.
    const int lane = threadIdx.x & 31;
    int local_max = 0;
    for (int v0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
        const int v = v0 + lane;
        long long lo = 0, hi = n;
        if (goff) {
            int g = 0;
            if (lane == 0) {
                int l = 0, h = G - 1;
                while (l < h) {
                    const int mid = (l + h + 1) >> 1;
                    if (goff[mid] <= v0) l = mid; else h = mid - 1;
                }
                g = l;
            }
            g = __shfl_sync(0xffffffffu, g, 0);
            if (v < n) {
                while (g + 1 < G && goff[g + 1] <= v) ++g;
                lo = goff[g];
                hi = goff[g + 1];
            }
        }
        if (v >= n) continue;
        const int a = rowptr[v], b = rowptr[v + 1];
        int d = 0;
        if (a < 0 || b < a || b > nnz) {
            atomicOr(&ctl->status, kErrBadCsr);
        } else {
            for (int k = a; k < b; ++k) {
                const int w = colidx[k];
                if ((unsigned)w >= (unsigned)n || w < lo || w >= hi) {
                    atomicOr(&ctl->status, kErrBadCsr);
                } else if (w != v) {
                    ++d;
                }
            }
            if (b - a > small_max) bigrows[atomicAdd(&ctl->nbig, 1)] = v;
        }
        deg[v] = d;
        claim[v] = ~0ull;
        vis[v] = 0;
        if (adist) adist[v] = ~0ull;
        if (fkey) fkey[v] = 0;
        local_max = max(local_max, d);
    }
    atomicMax(&s_max, local_max);
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&ctl->maxdeg, s_max);
}

// Rows of at most kSmallRowMax stored entries: one thread per row (sort_small_row).
__global__ void k_sort_rows_small(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                  const int* __restrict__ deg, int* __restrict__ adj, int4* __restrict__ ell,
                                  const Ctl* ctl, int small_max, int by_degree) {
    if (ctl->status & kErrBadCsr) return;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (rowptr[v + 1] - rowptr[v] <= small_max) sort_small_row(v, rowptr, colidx, deg, adj, ell, by_degree);
}

// Sorted row of v from keys[0, m) already sorted: the full row into adj (from offset a) and the
// padded row (first 7 + degree); one thread writes the padded row.
__device__ __forceinline__ void write_sorted_row(int v, int a, int m, const unsigned long long* keys, int* adj,
                                                 int4* ell, int t, int nt) {
    for (int i = t; i < m; i += nt) adj[a + i] = (int)(unsigned)(keys[i] & 0xffffffffu);
    if (t == 0) {
        int r[8];
        for (int i = 0; i < 7; ++i) r[i] = i < m ? (int)(unsigned)(keys[i] & 0xffffffffu) : -1;
        r[7] = m;
        store_ell(ell, v, r);
    }
}

// Rows longer than the per-thread sorter (listed in bigrows), by size:
//   at most kWarpRowMax entries: one warp per row, bitonic sort in the warp's slice of shared memory
//     (the rows of scale-free graphs are mostly a few dozen entries long);
//   at most kBigRowSmem keys: one CTA per row, bitonic sort in shared memory;
//   longer: CTA 0 alone, in global scratch (scratch holds next_pow2(maxdeg) keys).
// Launched with kBigRowThreads threads and kBigRowSmem keys of dynamic shared memory.
__global__ void k_sort_rows_big(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                const int* __restrict__ deg, int* __restrict__ adj, int4* __restrict__ ell,
                                const int* __restrict__ bigrows, const Ctl* ctl,
                                unsigned long long* __restrict__ scratch, int by_degree) {
    extern __shared__ unsigned long long s_keys[];
    __shared__ int s_m;
    if (ctl->status & kErrBadCsr) return;
    const int nbig = ctl->nbig;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // one warp per row; the keys are gathered in stored order (a warp compaction skips the diagonal)
    unsigned long long* ws = s_keys + (size_t)wid * kWarpRowMax;
    for (int r = blockIdx.x * nw + wid; r < nbig; r += gridDim.x * nw) {
        const int v = bigrows[r];
        const int a = rowptr[v], b = rowptr[v + 1];
        if (b - a > kWarpRowMax) continue;
        int m = 0;
        for (int k0 = a; k0 < b; k0 += 32) {
            const int k = k0 + lane;
            const int w = k < b ? colidx[k] : v;
            const bool keep = w != v;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) ws[m + __popc(bal & ((1u << lane) - 1u))] = row_key(deg, w, k - a, by_degree);
            m += __popc(bal);
        }
        int P = 1;
        while (P < m) P <<= 1;
        for (int i = m + lane; i < P; i += 32) ws[i] = kKeyMax;
        __syncwarp();
        bitonic_sort_warp(ws, P);
        write_sorted_row(v, a, m, ws, adj, ell, lane, 32);
        __syncwarp();
    }
    __syncthreads();
    // one CTA per row
    for (int r = blockIdx.x; r < nbig; r += gridDim.x) {
        const int v = bigrows[r];
        const int a = rowptr[v], b = rowptr[v + 1];
        if (b - a <= kWarpRowMax) continue;
        const int m = deg[v];
        int P = 1;
        while (P < m) P <<= 1;
        if (P > kBigRowSmem) continue;
        if (threadIdx.x == 0) s_m = 0;
        __syncthreads();
        for (int k = a + threadIdx.x; k < b; k += blockDim.x) {
            const int w = colidx[k];
            if (w != v) s_keys[atomicAdd(&s_m, 1)] = row_key(deg, w, k - a, by_degree);
        }
        __syncthreads();
        for (int i = m + threadIdx.x; i < P; i += blockDim.x) s_keys[i] = kKeyMax;
        __syncthreads();
        bitonic_sort_cta(s_keys, P);
        write_sorted_row(v, a, m, s_keys, adj, ell, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    // rows beyond shared memory, by CTA 0 in global scratch: its threads scan the list together
    // (one entry each per round), then sort the rows found one after another
    if (blockIdx.x != 0) return;
    for (int r0 = 0; r0 < nbig; r0 += blockDim.x) {
        const int r = r0 + (int)threadIdx.x;
        const bool huge = r < nbig && deg[bigrows[r]] > kBigRowSmem;
        const int cnt = __syncthreads_count(huge);
        if (cnt == 0) continue;
        if (threadIdx.x == 0) s_m = kIntMax;
        __syncthreads();
        if (huge) atomicMin(&s_m, r);
        __syncthreads();
        // sort the first huge row of this round, then rescan from just after it
        const int rr = s_m;
        __syncthreads();
        r0 = rr + 1 - (int)blockDim.x;
        const int v = bigrows[rr];
        const int m = deg[v];
        int P = 1;
        while (P < m) P <<= 1;
        const int a = rowptr[v], b = rowptr[v + 1];
        if (threadIdx.x == 0) s_m = 0;
        __syncthreads();
        for (int k = a + threadIdx.x; k < b; k += blockDim.x) {
            const int w = colidx[k];
            if (w != v) scratch[atomicAdd(&s_m, 1)] = row_key(deg, w, k - a, by_degree);
        }
        __syncthreads();
        for (int i = m + threadIdx.x; i < P; i += blockDim.x) scratch[i] = kKeyMax;
        __syncthreads();
        bitonic_sort_cta(scratch, P);
        write_sorted_row(v, a, m, scratch, adj, ell, threadIdx.x, blockDim.x);
        __syncthreads();
    }
}

// ---- bandwidth / profile (Sec. II-A) ----

__global__ void k_bw_scatter(int n, const int* __restrict__ perm, int* __restrict__ pos, int* __restrict__ err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = perm[i];
        if ((unsigned)v >= (unsigned)n) {
            atomicOr(err, 1);
            continue;
        }
        if (atomicExch(&pos[v], i) != -1) atomicOr(err, 1);
    }
}

__global__ void k_bw_rows(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                          const int* __restrict__ perm, const int* __restrict__ pos,
                          unsigned long long* __restrict__ out /* [0] max beta, [1] sum beta */) {
    __shared__ unsigned long long s_max, s_sum;
    if (threadIdx.x == 0) { s_max = 0; s_sum = 0; }
    __syncthreads();
    unsigned long long lmax = 0, lsum = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = perm[i];
        int f = i;
        for (int k = rowptr[v]; k < rowptr[v + 1]; ++k) f = min(f, pos[colidx[k]]);
        const unsigned long long beta = (unsigned long long)(i - f);
        lmax = beta > lmax ? beta : lmax;
        lsum += beta;
    }
    atomicMax(&s_max, lmax);
    atomicAdd(&s_sum, lsum);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&out[0], s_max);
        atomicAdd(&out[1], s_sum);
    }
}

}  // namespace rcm
