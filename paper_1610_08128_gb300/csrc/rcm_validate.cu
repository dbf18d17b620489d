// rcm_validate.cu -- rcm_validate: the pattern contract of include/rcm.h checked on the device.
//
// The ordering calls take a symmetric pattern without duplicate entries as a precondition (the
// graph of A, Sec. II-A, is undirected) and check only the CSR structure. This debugging aid
// checks all of it:
//   pass 1 (k_val_rows)     per row: bounds, columns in range, diagonal entries, the longest row;
//                           a copy of each well-formed row of at most kSmallRowMax entries sorted
//                           by column (one thread), longer rows listed;
//   pass 2 (k_val_sort_big) the listed rows sorted by a whole CTA (bitonic, shared memory, or
//                           global scratch for rows beyond kBigRowSmem entries);
//   pass 3 (k_val_entries)  per stored entry (v, w): a duplicate if it equals its predecessor in
//                           the sorted row; otherwise, off the diagonal, asymmetric unless a
//                           binary search finds v in the sorted row of w.
// Passes 2 and 3 run only when pass 1 found the rows and columns well formed.
#include <algorithm>

#include "rcm_host.hpp"
#include "rcm_internal.cuh"
#include "rcm_prep.cuh"

namespace rcm {

// Counters (u64 each): faults, the longest row, the first faulty row (a min, starting at ~0) and
// the number of long rows listed by pass 1.
enum { kVBadRows = 0, kVBadCols, kVDup, kVAsym, kVDiag, kVMaxRow, kVFirstBad, kVBig, kVCount };

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    return x;
}

// Per-thread partial counts, combined per warp before the atomics (kVFirstBad is a min, kVMaxRow
// a max, the others sums). Every thread of the grid calls this once, after its loop.
__device__ __forceinline__ void flush_counts(unsigned long long* cnt, unsigned long long (&c)[kVCount]) {
    const bool lead = (threadIdx.x & 31) == 0;
#pragma unroll
    for (int i = 0; i < kVCount; ++i) {
        unsigned long long x;
        if (i == kVFirstBad) x = warp_min_u64(c[i]);
        else if (i == kVMaxRow) x = warp_max_u64(c[i]);
        else x = warp_sum_u64(c[i]);
        if (!lead) continue;
        if (i == kVFirstBad) {
            if (x != kKeyMax) atomicMin(cnt + i, x);
        } else if (i == kVMaxRow) {
            if (x) atomicMax(cnt + i, x);
        } else if (x) {
            atomicAdd(cnt + i, x);
        }
    }
}

__global__ void k_val_rows(int n, long long nnz, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                           int* __restrict__ srt, int* __restrict__ big, unsigned long long* cnt) {
    unsigned long long c[kVCount] = {0, 0, 0, 0, 0, 0, kKeyMax, 0};
    const int stride = gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0 && rowptr[0] != 0) {
        c[kVBadRows] = 1;
        c[kVFirstBad] = 0;
    }
    // every thread runs the same number of rounds, so the warp collectives below stay converged
    for (int v0 = blockIdx.x * blockDim.x; v0 < n; v0 += stride) {
        const int v = v0 + (int)threadIdx.x;
        if (v >= n) continue;
        const long long a = rowptr[v], b = rowptr[v + 1];
        if (a < 0 || b < a || b > nnz) {
            c[kVBadRows]++;
            c[kVFirstBad] = min(c[kVFirstBad], (unsigned long long)v);
            continue;
        }
        bool ok = true;
        for (long long k = a; k < b; ++k) {
            const int w = colidx[k];
            if ((unsigned)w >= (unsigned)n) {
                c[kVBadCols]++;
                ok = false;
            } else if (w == v) {
                c[kVDiag]++;
            }
        }
        if (!ok) {
            c[kVFirstBad] = min(c[kVFirstBad], (unsigned long long)v);
            continue;
        }
        const int m = (int)(b - a);
        c[kVMaxRow] = max(c[kVMaxRow], (unsigned long long)m);
        if (m <= kSmallRowMax) {
            int r[kSmallRowMax];
            for (int i = 0; i < m; ++i) {
                const int x = colidx[a + i];
                int j = i;
                while (j > 0 && r[j - 1] > x) {
                    r[j] = r[j - 1];
                    --j;
                }
                r[j] = x;
            }
            for (int i = 0; i < m; ++i) srt[a + i] = r[i];
        } else {
            big[atomicAdd(cnt + kVBig, 1ull)] = v;
        }
    }
    flush_counts(cnt, c);
}

// Sorts rows listed in big by column, one CTA per row; rows of more than kBigRowSmem entries by
// CTA 0 alone in scratch (next_pow2(longest row) keys).
__global__ void k_val_sort_big(const int* __restrict__ rowptr, const int* __restrict__ colidx, int* __restrict__ srt,
                               const int* __restrict__ big, int nbig, unsigned long long* __restrict__ scratch) {
    extern __shared__ unsigned long long s_keys[];
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0: rows that fit in shared memory, strided over the CTAs; pass 1: the rest, CTA 0
        if (pass == 1 && blockIdx.x != 0) return;
        const int first = pass == 0 ? (int)blockIdx.x : 0;
        const int step = pass == 0 ? (int)gridDim.x : 1;
        for (int r = first; r < nbig; r += step) {
            const int v = big[r];
            const int a = rowptr[v];
            const int m = rowptr[v + 1] - a;
            int P = 1;
            while (P < m) P <<= 1;
            const bool in_smem = P <= kBigRowSmem;
            if (in_smem != (pass == 0)) continue;
            unsigned long long* s = in_smem ? s_keys : scratch;
            for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < m ? (unsigned long long)(unsigned)colidx[a + i] : kKeyMax;
            __syncthreads();
            bitonic_sort_cta(s, P);
            for (int i = threadIdx.x; i < m; i += blockDim.x) srt[a + i] = (int)(unsigned)s[i];
            __syncthreads();
        }
    }
}

__global__ void k_val_entries(int n, long long nnz, const int* __restrict__ rowptr, const int* __restrict__ srt,
                              unsigned long long* cnt) {
    unsigned long long c[kVCount] = {0, 0, 0, 0, 0, 0, kKeyMax, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k0 = (long long)blockIdx.x * blockDim.x; k0 < nnz; k0 += stride) {
        const long long k = k0 + threadIdx.x;
        if (k >= nnz) continue;
        // the row of entry k: the last r with rowptr[r] <= k (rows are well formed here)
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = lo + (hi - lo + 1) / 2;
            if (rowptr[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        const int r = lo;
        const int w = srt[k];
        if (k > rowptr[r] && srt[k - 1] == w) {
            c[kVDup]++;
            c[kVFirstBad] = min(c[kVFirstBad], (unsigned long long)r);
            continue;
        }
        if (w == r) continue;
        int x = rowptr[w], y = rowptr[w + 1];
        const int end = y;
        while (x < y) {
            const int mid = x + (y - x) / 2;
            if (srt[mid] < r) x = mid + 1;
            else y = mid;
        }
        if (x == end || srt[x] != r) {
            c[kVAsym]++;
            c[kVFirstBad] = min(c[kVFirstBad], (unsigned long long)r);
        }
    }
    flush_counts(cnt, c);
}

}  // namespace rcm

using namespace rcm;

extern "C" rcm_status rcm_validate(int32_t n, const int32_t* rowptr, const int32_t* colidx,
                                   rcm_validate_report* report, rcm_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n < 0 || !report) return RCM_ERR_INVALID_ARG;
    *report = rcm_validate_report{};
    report->first_bad_row = -1;
    if (n == 0) return RCM_OK;
    if (!rowptr) return RCM_ERR_INVALID_ARG;
    int last = 0;
    cudaError_t e = cudaMemcpyAsync(&last, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    const long long nnz = last;
    if (nnz > 0 && !colidx) return RCM_ERR_INVALID_ARG;
    const size_t b_cnt = 256;
    const size_t b_srt = align_up(sizeof(int) * (size_t)std::max(nnz, 1LL), 256);
    const size_t b_big = align_up(sizeof(int) * (size_t)n, 256);
    void* buf = nullptr;
    rcm_status st = ws_alloc(&buf, b_cnt + b_srt + b_big, s);
    if (st != RCM_OK) return st;
    unsigned long long* cnt = (unsigned long long*)buf;
    int* srt = (int*)((char*)buf + b_cnt);
    int* big = (int*)((char*)buf + b_cnt + b_srt);
    unsigned long long* scratch = nullptr;
    const DeviceInfo& di = device_info();
    const int tb = 256;
    unsigned long long h[kVCount] = {0};
    auto read_counts = [&]() {
        cudaError_t r = cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
        return r == cudaSuccess ? cudaStreamSynchronize(s) : r;
    };
    e = cudaMemsetAsync(cnt, 0, b_cnt, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt + kVFirstBad, 0xff, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        const int grid = (int)std::max<long long>(1, std::min<long long>((n + tb - 1) / tb, (long long)di.sms * 16));
        k_val_rows<<<grid, tb, 0, s>>>(n, nnz, rowptr, colidx, srt, big, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = read_counts();
    const bool structured = e == cudaSuccess && h[kVBadRows] == 0 && h[kVBadCols] == 0;
    if (structured && h[kVBig] > 0) {
        const int nbig = (int)h[kVBig];
        long long P = 1;
        while (P < (long long)h[kVMaxRow]) P <<= 1;
        if (P > kBigRowSmem) st = ws_alloc((void**)&scratch, sizeof(unsigned long long) * (size_t)P, s);
        if (st == RCM_OK) {
            const int smem = (int)(sizeof(unsigned long long) * kBigRowSmem);
            e = cudaFuncSetAttribute(k_val_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess) {
                k_val_sort_big<<<std::min(nbig, 2 * di.sms), 1024, smem, s>>>(rowptr, colidx, srt, big, nbig, scratch);
                e = cudaGetLastError();
            }
        }
    }
    if (structured && st == RCM_OK && e == cudaSuccess && nnz > 0) {
        const int grid = (int)std::max<long long>(1, std::min<long long>((nnz + tb - 1) / tb, (long long)di.sms * 32));
        k_val_entries<<<grid, tb, 0, s>>>(n, nnz, rowptr, srt, cnt);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = read_counts();
    }
    if (scratch) ws_free(scratch, s);
    ws_free(buf, s);
    if (st != RCM_OK) return st;
    if (e != cudaSuccess) return cuda_status(e);
    report->bad_rows = (int64_t)h[kVBadRows];
    report->bad_columns = (int64_t)h[kVBadCols];
    report->duplicates = structured ? (int64_t)h[kVDup] : -1;
    report->asymmetric = structured ? (int64_t)h[kVAsym] : -1;
    report->diagonal = (int64_t)h[kVDiag];
    report->max_row = (int64_t)h[kVMaxRow];
    report->first_bad_row = h[kVFirstBad] == kKeyMax ? -1 : (int64_t)h[kVFirstBad];
    const bool good = structured && h[kVDup] == 0 && h[kVAsym] == 0;
    return good ? RCM_OK : RCM_ERR_BAD_CSR;
}
