// rcm_prep.cuh -- declarations of the preprocessing and bandwidth/profile kernels.
#pragma once

#include "rcm_internal.cuh"

namespace rcm {

constexpr int kSmallRowMax = 32;     // rows with at most this many stored entries: per-thread sort
constexpr int kBigRowSmem = 8192;    // rows sorted in shared memory by one CTA (64 KB of keys)

__global__ void k_degree_validate(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                  int* __restrict__ deg, unsigned long long* __restrict__ claim, int* __restrict__ vis,
                                  int* __restrict__ bigrows, Ctl* ctl, int small_max);

__global__ void k_sort_rows_small(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                  const int* __restrict__ deg, int* __restrict__ adj, int4* __restrict__ ell,
                                  const Ctl* ctl);

__global__ void k_sort_rows_big(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                const int* __restrict__ deg, int* __restrict__ adj, int4* __restrict__ ell,
                                const int* __restrict__ bigrows, const Ctl* ctl,
                                unsigned long long* __restrict__ scratch);

__global__ void k_bw_scatter(int n, const int* __restrict__ perm, int* __restrict__ pos, int* __restrict__ err);

__global__ void k_bw_rows(int n, const int* __restrict__ rowptr, const int* __restrict__ colidx,
                          const int* __restrict__ perm, const int* __restrict__ pos,
                          unsigned long long* __restrict__ out);

}  // namespace rcm
