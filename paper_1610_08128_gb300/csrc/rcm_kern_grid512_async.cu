// rcm_kern_grid512_async.cu -- instantiates the persistent grid kernel of rcm_single_kernels.cuh with
// asynchronous levels-only sweeps, for CTAs of 512 threads.
#define RCM_KERNEL_DEFINITIONS
#include "rcm_single_kernels.cuh"

namespace rcm {

template __global__ void k_rcm_single<512, true, false>(EngineArgs, int);

}  // namespace rcm
