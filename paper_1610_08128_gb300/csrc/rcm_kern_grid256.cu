// rcm_kern_grid256.cu -- instantiates the persistent grid kernel of rcm_single_kernels.cuh for CTAs of 256 threads
// (one translation unit per width, so the widths compile in parallel).
#define RCM_KERNEL_DEFINITIONS
#include "rcm_single_kernels.cuh"

namespace rcm {

template __global__ void k_rcm_single<256, false, false>(EngineArgs, int);

}  // namespace rcm
