// Lock-free union-find over cell indices, shared by the connectivity
// kernels.  A root is only ever linked to a smaller index, so parent chains
// strictly decrease, every find terminates, and the final root of a set is
// its smallest index; each failed CAS means another thread linked that
// root, so the retry loop makes global progress.  Both loops still carry an
// iteration cap that raises bit 2 of *err instead of spinning.
#pragma once

#include <cuda_runtime.h>

namespace cl {

constexpr int kUfMaxIter = 1 << 24;

// Root of a, walking the parent chain without writing (the final flatten
// pass: each thread then writes only its own cell's label).
__device__ __forceinline__ int uf_find(volatile int* L, int a, int* err) {
    int it = 0;
    int p = L[a];
    while (p != a) {
        a = p;
        p = L[a];
        if (++it > kUfMaxIter) { atomicOr(err, 2); break; }
    }
    return a;
}

// Root of a with path halving, for the merge pass: each visited node is
// pointed at its grandparent.  Any ancestor is a valid parent while sets
// only merge (parents stay smaller than children), and only nodes already
// seen to be non-roots are written, so the halving never races with the
// CAS that links a root.  It must not run beside the flatten pass, whose
// final root labels a late halving write could replace.
__device__ __forceinline__ int uf_find_halving(volatile int* L, int a, int* err) {
    int it = 0;
    int p = L[a];
    while (p != a) {
        const int gp = L[p];
        if (gp != p) L[a] = gp;
        a = gp;
        p = L[a];
        if (++it > kUfMaxIter) { atomicOr(err, 2); break; }
    }
    return a;
}

__device__ __forceinline__ void uf_union(int* L, int a, int b, int* err) {
    for (int it = 0; it < kUfMaxIter; ++it) {
        a = uf_find_halving(L, a, err);
        b = uf_find_halving(L, b, err);
        if (a == b) return;
        if (a < b) { int t = a; a = b; b = t; }
        int old = atomicCAS(L + a, a, b);
        if (old == a) return;
    }
    atomicOr(err, 2);
}

}  // namespace cl
