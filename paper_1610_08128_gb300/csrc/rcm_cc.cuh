// rcm_cc.cuh -- connected components by union-find, used to order independent components at the
// same time.
//
// Sec. III-B orders a disconnected graph by running Alg. 3 once per connected component. With the
// start rule (each component starts at the lowest-id vertex of minimum degree among the vertices
// not yet numbered), components are numbered in increasing order of their own minimum
// (degree, id) vertex, and component c receives the labels [offset_c, offset_c + size_c), where
// offset_c adds up the sizes of the components before it in that order. Knowing every
// component's key and size in advance therefore fixes every label range, and the components can
// be ordered concurrently with results identical to the sequential loop.
//
// Union-find with lock-free hooking of the larger root under the smaller: parent pointers only
// ever point to smaller ids, so every root ends as the smallest vertex id of its component.
#pragma once

#include "rcm_internal.cuh"

namespace rcm {

constexpr int kMaxComps = 1 << 20;   // components ordered concurrently at most (else one by one)
constexpr int kCompSmem = 8192;      // component tables sorted in shared memory up to this size

// Representative of v; shortens the path on the way (benign races: a shortcut always points to
// an ancestor, and parents only decrease).
__device__ __forceinline__ int cc_root(volatile int* parent, int v) {
    int cur = parent[v];
    if (cur != v) {
        int prev = v, next;
        while (cur > (next = parent[cur])) {
            parent[prev] = next;
            prev = cur;
            cur = next;
        }
    }
    return cur;
}

__device__ __forceinline__ void cc_union(int* parent, int a, int b) {
    volatile int* vp = parent;
    int ra = cc_root(vp, a), rb = cc_root(vp, b);
    while (ra != rb) {
        if (ra < rb) {
            const int old = atomicCAS(&parent[rb], rb, ra);
            if (old == rb) break;
            rb = cc_root(vp, old);
        } else {
            const int old = atomicCAS(&parent[ra], ra, rb);
            if (old == ra) break;
            ra = cc_root(vp, old);
        }
    }
}

}  // namespace rcm
