// rcm_host.hpp -- host-side helpers shared by the library's entry points: CUDA error mapping,
// the per-stream error latch (host-mapped pinned words the kernels OR their error bits into),
// device properties, and stream-ordered workspace allocation.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rcm.h"

namespace rcm {

struct Ctl;

struct DeviceInfo {
    int device;
    int sms;
    int max_smem_optin;
    size_t l2_bytes;
};

// Properties of the current device (cached per device).
const DeviceInfo& device_info();

// Device pointer of the latch word of `stream` (host-mapped pinned memory, one word per stream).
int* stream_latch(cudaStream_t stream);

// Map device error bits to a status.
rcm_status status_from_bits(int bits);

// Stream-ordered allocation from the device's default pool (kept cached between calls).
rcm_status ws_alloc(void** p, size_t bytes, cudaStream_t s);
void ws_free(void* p, cudaStream_t s);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Enqueue a one-thread kernel that ORs ctl->status into the stream's latch word and, if
// stats_dev != NULL, copies ctl->stats (8 x int64) there.
cudaError_t enqueue_latch(const Ctl* ctl, int* latch, long long* stats_dev, cudaStream_t s);

rcm_status cuda_status(cudaError_t e);

}  // namespace rcm
