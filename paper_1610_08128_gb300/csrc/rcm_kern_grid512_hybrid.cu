// rcm_kern_grid512_hybrid.cu -- instantiates the persistent grid kernel of rcm_single_kernels.cuh with
// per-level top-down / bottom-up expansion, for CTAs of 512 threads.
#define RCM_KERNEL_DEFINITIONS
#include "rcm_single_kernels.cuh"

namespace rcm {

template __global__ void k_rcm_single<512, false, true>(EngineArgs, int);

}  // namespace rcm
