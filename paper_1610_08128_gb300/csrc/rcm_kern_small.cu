// rcm_kern_small.cu -- instantiates the shared-memory one-CTA kernel of rcm_single_kernels.cuh for
// every CTA width it supports (the persistent grid kernel has one translation unit per width).
#define RCM_KERNEL_DEFINITIONS
#include "rcm_single_kernels.cuh"

namespace rcm {

template __global__ void k_rcm_small<32>(EngineArgs, int, int);
template __global__ void k_rcm_small<64>(EngineArgs, int, int);
template __global__ void k_rcm_small<128>(EngineArgs, int, int);
template __global__ void k_rcm_small<256>(EngineArgs, int, int);
template __global__ void k_rcm_small<512>(EngineArgs, int, int);

}  // namespace rcm
