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
// an ancestor, and parents only decrease). Every id on the path must lie in [lo, hi) and every
// non-root must point to a smaller id; a path that breaks either rule (a parent entry that was
// never initialised) returns -1 without following it.
__device__ __forceinline__ int cc_root(volatile int* parent, int v, int lo, int hi) {
    int cur = parent[v];
    if (cur == v) return v;
    int prev = v;
    while (true) {
        if (cur < lo || cur >= hi) return -1;
        const int next = parent[cur];
        if (next >= cur) return next == cur ? cur : -1;
        parent[prev] = next;
        prev = cur;
        cur = next;
    }
}

// Joins the sets of a and b. Returns false if a parent path was invalid (see cc_root).
__device__ __forceinline__ bool cc_union(int* parent, int a, int b, int lo, int hi) {
    volatile int* vp = parent;
    int ra = cc_root(vp, a, lo, hi), rb = cc_root(vp, b, lo, hi);
    while (ra != rb) {
        if (ra < 0 || rb < 0) return false;
        if (ra < rb) {
            const int old = atomicCAS(&parent[rb], rb, ra);
            if (old == rb) return true;
            rb = cc_root(vp, old, lo, hi);
        } else {
            const int old = atomicCAS(&parent[ra], ra, rb);
            if (old == ra) return true;
            ra = cc_root(vp, old, lo, hi);
        }
    }
    return ra >= 0;
}

}  // namespace rcm
