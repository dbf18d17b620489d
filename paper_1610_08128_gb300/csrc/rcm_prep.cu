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
                                  unsigned long long* __restrict__ adist, unsigned long long* __restrict__ fkey) {
    __shared__ int s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rowptr[0] != 0 || rowptr[n] != nnz || nnz < 0))
        atomicOr(&ctl->status, kErrBadCsr);
    int local_max = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int a = rowptr[v], b = rowptr[v + 1];
        int d = 0;
        if (a < 0 || b < a || b > nnz) {
            atomicOr(&ctl->status, kErrBadCsr);
        } else {
            for (int k = a; k < b; ++k) {
                const int w = colidx[k];
                if ((unsigned)w >= (unsigned)n) {
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

// Rows longer than the per-thread sorter: one CTA per row, bitonic sort in shared memory for rows
// of at most kBigRowSmem entries; longer rows are sorted by CTA 0 alone in global scratch
// (scratch holds next_pow2(maxdeg) keys).
__global__ void k_sort_rows_big(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                const int* __restrict__ deg, int* __restrict__ adj, int4* __restrict__ ell,
                                const int* __restrict__ bigrows, const Ctl* ctl,
                                unsigned long long* __restrict__ scratch, int by_degree) {
    extern __shared__ unsigned long long s_keys[];
    __shared__ int s_m;
    if (ctl->status & kErrBadCsr) return;
    const int nbig = ctl->nbig;
    for (int r = blockIdx.x; r < nbig; r += gridDim.x) {
        const int v = bigrows[r];
        const int a = rowptr[v], b = rowptr[v + 1];
        const int m = deg[v];
        int P = 1;
        while (P < m) P <<= 1;
        const bool in_smem = P <= kBigRowSmem;
        if (!in_smem && blockIdx.x != 0) continue;
        unsigned long long* s = in_smem ? s_keys : scratch;
        if (threadIdx.x == 0) s_m = 0;
        __syncthreads();
        for (int k = a + threadIdx.x; k < b; k += blockDim.x) {
            const int w = colidx[k];
            if (w != v) s[atomicAdd(&s_m, 1)] = row_key(deg, w, k - a, by_degree);
        }
        __syncthreads();
        for (int i = m + threadIdx.x; i < P; i += blockDim.x) s[i] = kKeyMax;
        __syncthreads();
        bitonic_sort_cta(s, P);
        for (int i = threadIdx.x; i < m; i += blockDim.x) adj[a + i] = (int)(unsigned)(s[i] & 0xffffffffu);
        if (threadIdx.x == 0) {
            int r[8];
            for (int i = 0; i < 7; ++i) r[i] = i < m ? (int)(unsigned)(s[i] & 0xffffffffu) : -1;
            r[7] = m;
            store_ell(ell, v, r);
        }
        __syncthreads();
    }
    // Huge rows assigned to other CTAs by the stride are picked up here by CTA 0.
    if (blockIdx.x != 0) return;
    for (int r = 0; r < nbig; ++r) {
        if (r % gridDim.x == 0) continue;  // already handled above by CTA 0
        const int v = bigrows[r];
        const int m = deg[v];
        int P = 1;
        while (P < m) P <<= 1;
        if (P <= kBigRowSmem) continue;
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
        for (int i = threadIdx.x; i < m; i += blockDim.x) adj[a + i] = (int)(unsigned)(scratch[i] & 0xffffffffu);
        if (threadIdx.x == 0) {
            int r[8];
            for (int i = 0; i < 7; ++i) r[i] = i < m ? (int)(unsigned)(scratch[i] & 0xffffffffu) : -1;
            r[7] = m;
            store_ell(ell, v, r);
        }
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
