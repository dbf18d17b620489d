// rcm_kern_components.cu -- instantiates the component kernel of rcm_single_kernels.cuh (the
// components that the persistent grid kernel's component table leaves to smaller engines).
#define RCM_KERNEL_DEFINITIONS
#include "rcm_single_kernels.cuh"

namespace rcm {

template __global__ void k_rcm_components<kComponentThreads>(EngineArgs);

}  // namespace rcm
