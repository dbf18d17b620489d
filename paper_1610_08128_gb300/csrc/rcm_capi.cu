// rcm_capi.cu -- the extern "C" entry points declared in include/rcm.h and the host helpers they
// share: device properties, the per-stream error latch, stream-ordered workspace.
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "rcm_host.hpp"
#include "rcm_internal.cuh"
#include "rcm_cc.cuh"
#include "rcm_prep.cuh"
#include "rcm_single.cuh"

namespace rcm {

rcm_status order_single(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colidx,
                        int32_t* perm, const rcm_options* opts, long long* stats_dev, cudaEvent_t* ev,
                        cudaStream_t s);
rcm_status order_batch(int32_t G, int64_t n_total, const int64_t* goff, const int32_t* rowptr,
                       const int32_t* colidx, int32_t* perm, const rcm_batch_options* opts, cudaStream_t s);

rcm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RCM_OK;
    if (e == cudaErrorMemoryAllocation) return RCM_ERR_OOM;
    return RCM_ERR_CUDA;
}

rcm_status status_from_bits(int bits) {
    if (bits & kErrBadCsr) return RCM_ERR_BAD_CSR;
    if (bits & kErrTimeout) return RCM_ERR_TIMEOUT;
    if (bits & kErrTooLarge) return RCM_ERR_TOO_LARGE;
    if (bits & kErrInternal) return RCM_ERR_CUDA;
    return RCM_OK;
}

static std::mutex g_dev_mu;
static DeviceInfo g_dev[64];
static bool g_dev_ok[64];

const DeviceInfo& device_info() {
    int d = 0;
    cudaGetDevice(&d);
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (!g_dev_ok[d & 63]) {
        DeviceInfo& di = g_dev[d & 63];
        di.device = d;
        cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, d);
        cudaDeviceGetAttribute(&di.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d);
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, d);
        di.l2_bytes = (size_t)l2;
        // keep freed workspace cached in the default pool between calls
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        g_dev_ok[d & 63] = true;
    }
    return g_dev[d & 63];
}

// ---- per-stream error latch: one host-mapped pinned word per (device, stream) ----
// A stream holds a slot from its first ordering call until rcm_stream_status reads and clears it
// (after synchronising the stream, so nothing still writes the slot); the slot is then free for
// any stream. A call on a new stream while all kLatchSlots slots are held fails before any work
// (RCM_ERR_TOO_LARGE) instead of sharing a slot with another stream.
constexpr int kLatchSlots = 4096;
static std::mutex g_latch_mu;
static int* g_latch = nullptr;  // host-mapped, portable
static std::unordered_map<unsigned long long, int> g_slot_of;
static std::vector<int> g_free_slots;
static int g_next_slot = 0;

static unsigned long long stream_key(cudaStream_t s) {
    int d = 0;
    cudaGetDevice(&d);
    return (unsigned long long)(uintptr_t)s * 64ull + (unsigned long long)d;
}

// The stream's latch word; with create, a free slot is taken for a stream that holds none.
// nullptr: no slot (not created, or all held), or the pinned words could not be allocated.
static int* latch_host(cudaStream_t s, bool create) {
    std::lock_guard<std::mutex> g(g_latch_mu);
    if (!g_latch) {
        void* p = nullptr;
        if (cudaHostAlloc(&p, sizeof(int) * kLatchSlots, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
            return nullptr;
        g_latch = (int*)p;
        for (int i = 0; i < kLatchSlots; ++i) g_latch[i] = 0;
    }
    const unsigned long long k = stream_key(s);
    auto it = g_slot_of.find(k);
    if (it != g_slot_of.end()) return g_latch + it->second;
    if (!create) return nullptr;
    int slot;
    if (!g_free_slots.empty()) {
        slot = g_free_slots.back();
        g_free_slots.pop_back();
    } else if (g_next_slot < kLatchSlots) {
        slot = g_next_slot++;
    } else {
        return nullptr;
    }
    g_latch[slot] = 0;
    g_slot_of.emplace(k, slot);
    return g_latch + slot;
}

// Reads, clears and frees the stream's slot (the stream must be synchronised); 0 if it holds none.
static int latch_take(cudaStream_t s) {
    int* h = latch_host(s, false);
    if (!h) return 0;
    std::lock_guard<std::mutex> g(g_latch_mu);
    const int bits = *(volatile int*)h;
    *(volatile int*)h = 0;
    auto it = g_slot_of.find(stream_key(s));
    if (it != g_slot_of.end()) {
        g_free_slots.push_back(it->second);
        g_slot_of.erase(it);
    }
    return bits;
}

int* stream_latch(cudaStream_t s) {
    int* h = latch_host(s, true);
    if (!h) return nullptr;
    int* d = nullptr;
    if (cudaHostGetDevicePointer((void**)&d, h, 0) != cudaSuccess) return nullptr;
    return d;
}

__global__ void k_latch(const Ctl* ctl, int* latch, long long* stats) {
    if (threadIdx.x == 0) {
        const int bits = ((const volatile Ctl*)ctl)->status;
        if (bits && latch) *(volatile int*)latch = *(volatile int*)latch | bits;
        if (stats) {
            for (int i = 0; i < 8; ++i) stats[i] = ctl->stats[i];
            for (int i = 0; i < 8; ++i) stats[8 + i] = ctl->phase_ns[i];
        }
    }
}

cudaError_t enqueue_latch(const Ctl* ctl, int* latch, long long* stats_dev, cudaStream_t s) {
    if (!latch) return cudaErrorMemoryAllocation;
    k_latch<<<1, 32, 0, s>>>(ctl, latch, stats_dev);
    return cudaGetLastError();
}

rcm_status ws_alloc(void** p, size_t bytes, cudaStream_t s) {
    device_info();  // sets the pool's release threshold once per device
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 256), s);
    return e == cudaSuccess ? RCM_OK : cuda_status(e);
}

void ws_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

static rcm_status read_nnz(int32_t n, const int32_t* rowptr, cudaStream_t s, int64_t* nnz) {
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    if (v < 0) return RCM_ERR_BAD_CSR;
    *nnz = v;
    return RCM_OK;
}

static rcm_status check_options(const rcm_options* o) {
    if (!o) return RCM_OK;
    if (o->narrow_threshold < -1 || o->grid_blocks < 0 || o->spin_limit_ns < 0 || o->nnz < 0 || o->nnz >= 0x7fffffffLL)
        return RCM_ERR_INVALID_ARG;
    const int t = o->block_threads;
    if (t && t != 32 && t != 64 && t != 128 && t != 256 && t != 512 && t != 1024) return RCM_ERR_INVALID_ARG;
    if (o->cluster != 0 && o->cluster != 1) return RCM_ERR_INVALID_ARG;
    if (o->executor < 0 || o->executor > 2) return RCM_ERR_INVALID_ARG;
    if (o->async_sweeps < -1 || o->async_sweeps > 1 || o->debug_async_slots < 0) return RCM_ERR_INVALID_ARG;
    if (o->row_order != 0 && o->row_order != 1) return RCM_ERR_INVALID_ARG;
    if (o->expand_mode < 0 || o->expand_mode > 3 || o->bottom_up_divisor < 0) return RCM_ERR_INVALID_ARG;
    if (o->fused_sweeps < -1 || o->fused_sweeps > 2 || o->l2_persist < -1 || o->l2_persist > 1) return RCM_ERR_INVALID_ARG;
    if (o->debug_order_bits < 0 || o->debug_order_bits > 63) return RCM_ERR_INVALID_ARG;
    if (o->mid_cluster != 0 && o->mid_cluster != -1 && o->mid_cluster != 2 && o->mid_cluster != 4 &&
        o->mid_cluster != 8 && o->mid_cluster != 16)
        return RCM_ERR_INVALID_ARG;
    if (o->mid_threshold < 0) return RCM_ERR_INVALID_ARG;
    if (o->components_first < -1 || o->components_first > 1) return RCM_ERR_INVALID_ARG;
    return RCM_OK;
}

}  // namespace rcm

using namespace rcm;

extern "C" {

const char* rcm_status_string(rcm_status s) {
    switch (s) {
        case RCM_OK: return "RCM_OK";
        case RCM_ERR_INVALID_ARG: return "RCM_ERR_INVALID_ARG";
        case RCM_ERR_BAD_CSR: return "RCM_ERR_BAD_CSR";
        case RCM_ERR_OOM: return "RCM_ERR_OOM";
        case RCM_ERR_TOO_LARGE: return "RCM_ERR_TOO_LARGE";
        case RCM_ERR_CUDA: return "RCM_ERR_CUDA";
        case RCM_ERR_TIMEOUT: return "RCM_ERR_TIMEOUT";
        case RCM_ERR_NOT_READY: return "RCM_ERR_NOT_READY";
        case RCM_ERR_UNKNOWN_TICKET: return "RCM_ERR_UNKNOWN_TICKET";
    }
    return "RCM_ERR_UNKNOWN";
}

size_t rcm_workspace_bytes(int32_t n, int64_t nnz) {
    if (n < 0 || nnz < 0) return 0;
    return single_layout(n, nnz).total;
}

rcm_status rcm_order_ex(int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t* perm_out,
                        const rcm_options* opts, rcm_stats* stats, rcm_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n < 0) return RCM_ERR_INVALID_ARG;
    rcm_status st = check_options(opts);
    if (st != RCM_OK) return st;
    if (n == 0) {
        if (stats) *stats = rcm_stats{};
        return RCM_OK;
    }
    if (!rowptr || !perm_out) return RCM_ERR_INVALID_ARG;
    int64_t nnz = opts ? opts->nnz : 0;
    if (nnz == 0) {
        st = read_nnz(n, rowptr, s, &nnz);
        if (st != RCM_OK) return st;
    }
    if (nnz > 0 && !colidx) return RCM_ERR_INVALID_ARG;
    long long* stats_dev = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (stats) {
        st = ws_alloc((void**)&stats_dev, 16 * sizeof(long long), s);
        if (st != RCM_OK) return st;
        cudaMemsetAsync(stats_dev, 0, 16 * sizeof(long long), s);
        for (auto& x : ev) cudaEventCreate(&x);
    }
    st = order_single(n, nnz, rowptr, colidx, perm_out, opts, stats_dev, stats ? ev : nullptr, s);
    if (stats) {
        long long h[16] = {0};
        cudaError_t e = cudaMemcpyAsync(h, stats_dev, sizeof(h), cudaMemcpyDeviceToHost, s);
        ws_free(stats_dev, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (st == RCM_OK && e != cudaSuccess) st = cuda_status(e);
        float t01 = 0.f, t12 = 0.f;
        if (st == RCM_OK) {
            cudaEventElapsedTime(&t01, ev[0], ev[1]);
            cudaEventElapsedTime(&t12, ev[1], ev[2]);
        }
        for (auto& x : ev) cudaEventDestroy(x);
        stats->prep_ms = t01;
        stats->traverse_ms = t12;
        stats->components = h[0];
        stats->sweeps = h[1];
        stats->traversals = h[2];
        stats->levels = h[3];
        stats->max_ecc = h[4];
        stats->isolated = h[5];
        stats->narrow_levels = h[6];
        stats->grid_levels = h[7];
        for (int i = 0; i < 8; ++i) stats->phase_ns[i] = h[8 + i];
        if (st == RCM_OK) st = rcm_stream_status(stream);
    }
    return st;
}

rcm_status rcm_order(int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t* perm_out,
                     rcm_stream_t stream) {
    return rcm_order_ex(n, rowptr, colidx, perm_out, nullptr, nullptr, stream);
}

rcm_status rcm_order_host(int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t* perm_out,
                          rcm_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n < 0) return RCM_ERR_INVALID_ARG;
    if (n == 0) return RCM_OK;
    if (!rowptr || !perm_out) return RCM_ERR_INVALID_ARG;
    const int64_t nnz = rowptr[n];
    if (nnz < 0 || rowptr[0] != 0) return RCM_ERR_BAD_CSR;
    if (nnz > 0 && !colidx) return RCM_ERR_INVALID_ARG;
    const size_t b_rp = align_up(sizeof(int) * ((size_t)n + 1), 256);
    const size_t b_ci = align_up(sizeof(int) * (size_t)std::max<int64_t>(nnz, 1), 256);
    const size_t b_pm = align_up(sizeof(int) * (size_t)n, 256);
    void* buf = nullptr;
    rcm_status st = ws_alloc(&buf, b_rp + b_ci + b_pm, s);
    if (st != RCM_OK) return st;
    int* d_rp = (int*)buf;
    int* d_ci = (int*)((char*)buf + b_rp);
    int* d_pm = (int*)((char*)buf + b_rp + b_ci);
    cudaError_t e = cudaMemcpyAsync(d_rp, rowptr, sizeof(int) * ((size_t)n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(d_ci, colidx, sizeof(int) * (size_t)nnz, cudaMemcpyHostToDevice, s);
    // the L2 window on the persistent grid (rcm_options.l2_persist): this call synchronises
    // anyway, which is the window's only cost (the 192^3 grid: 6.8 against 7.1 ms)
    rcm_options o{};
    o.l2_persist = 1;
    if (e == cudaSuccess) st = order_single(n, nnz, d_rp, d_ci, d_pm, &o, nullptr, nullptr, s);
    if (e == cudaSuccess && st == RCM_OK)
        e = cudaMemcpyAsync(perm_out, d_pm, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, s);
    ws_free(buf, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (st != RCM_OK) return st;
    return rcm_stream_status(stream);
}

rcm_status rcm_order_batch(int32_t G, int64_t n_total, const int64_t* goff, const int32_t* rowptr,
                           const int32_t* colidx, int32_t* perm_out, rcm_stream_t stream) {
    if (G < 0 || n_total < 0 || n_total >= 0x7fffffffLL) return RCM_ERR_INVALID_ARG;
    if (G == 0 || n_total == 0) return RCM_OK;
    if (!goff || !rowptr || !perm_out) return RCM_ERR_INVALID_ARG;
    return order_batch(G, n_total, goff, rowptr, colidx, perm_out, nullptr, (cudaStream_t)stream);
}

rcm_status rcm_order_batch_ex(int32_t G, int64_t n_total, const int64_t* goff, const int32_t* rowptr,
                              const int32_t* colidx, int32_t* perm_out, const rcm_batch_options* opts,
                              rcm_stream_t stream) {
    if (G < 0 || n_total < 0 || n_total >= 0x7fffffffLL) return RCM_ERR_INVALID_ARG;
    if (G == 0 || n_total == 0) return RCM_OK;
    if (!goff || !rowptr || !perm_out) return RCM_ERR_INVALID_ARG;
    return order_batch(G, n_total, goff, rowptr, colidx, perm_out, opts, (cudaStream_t)stream);
}

rcm_status rcm_stream_status(rcm_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return status_from_bits(latch_take(s));
}

rcm_status rcm_bandwidth_profile(int32_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* perm,
                                 int64_t* bw, int64_t* profile, rcm_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n < 0 || !bw || !profile) return RCM_ERR_INVALID_ARG;
    *bw = 0;
    *profile = 0;
    if (n == 0) return RCM_OK;
    if (!rowptr || !perm) return RCM_ERR_INVALID_ARG;
    void* buf = nullptr;
    const size_t b_pos = align_up(sizeof(int) * (size_t)n, 256);
    rcm_status st = ws_alloc(&buf, b_pos + 256, s);
    if (st != RCM_OK) return st;
    int* pos = (int*)buf;
    unsigned long long* out = (unsigned long long*)((char*)buf + b_pos);
    int* err = (int*)(out + 2);
    const DeviceInfo& di = device_info();
    const int pb = 256;
    const int grid = (int)std::max<long long>(1, std::min<long long>((n + pb - 1) / pb, (long long)di.sms * 16));
    cudaError_t e = cudaMemsetAsync(pos, 0xff, sizeof(int) * (size_t)n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, 256, s);
    if (e == cudaSuccess) {
        k_bw_scatter<<<grid, pb, 0, s>>>(n, perm, pos, err);
        e = cudaGetLastError();
    }
    unsigned long long h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && (h[2] & 0xffffffffu) != 0) {
        ws_free(buf, s);
        return RCM_ERR_INVALID_ARG;
    }
    if (e == cudaSuccess) {
        k_bw_rows<<<grid, pb, 0, s>>>(n, rowptr, colidx, perm, pos, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    ws_free(buf, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    *bw = (int64_t)h[0];
    *profile = (int64_t)h[1];
    return RCM_OK;
}

}  // extern "C"
