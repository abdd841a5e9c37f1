// uvwx.cuh -- parent-neighbour-child interaction lists (paper Section 2.1:
// the alternative to the size/distance acceptance test, after Cheng,
// Greengard and Rokhlin 1999), one cell or leaf at a time.  Host-and-device
// functions over the tree's arrays, so that the kernels of uvwx.cu and a
// host-compiled check run the same code.
//
// Geometry: cell c has the doubled centre C = icentre[c].xyz and the level
// l = icentre[c].w in integer units u = side / 2^21; its cube spans C +- s,
// s = 2^(21 - l), in doubled units.  Two cells are adjacent when their closed
// cubes meet (|C_a - C_b| <= s_a + s_b on every axis) and neither contains
// the other (not |C_a - C_b| <= |s_a - s_b| on every axis).
//
// Lists (W and X are taken as direct sums, so that every list is one the
// stage kernels already evaluate):
//   neighbours N(c): the adjacent cells of c's level, found among the
//     children of c's parent and of the parent's neighbours (at most 26);
//   V(c): the children of the parent's neighbours that are not adjacent to c
//     (M2L pairs, same level, at most 189);
//   U(b), b a leaf: b, the leaves among the neighbours of b and of its
//     ancestors that are adjacent to b, and the adjacent leaves inside b's
//     neighbours (P2P pairs);
//   W(b), b a leaf: the cells inside b's neighbours that are not adjacent to b
//     but whose parent is (their leaves become P2P pairs in both directions:
//     W by the direct sum on b, X = the dual of W on those leaves).
#pragma once
#include <stdint.h>
#include <vector_types.h>

namespace fmm {

constexpr int UV_NB = 26;        // neighbours of a cell at most
constexpr int UV_STACK = 192;    // descent stack per leaf (7 per level + 8 is enough for 21 levels)

struct UvTree {
    const int4* icentre;
    const int32_t* parent;
    const int32_t* child_first;
    const int32_t* child_count;
    const int32_t* nb;     // [ncell][UV_NB]
    const int32_t* nbc;    // [ncell]
};

__host__ __device__ inline int uv_iabs(int v) { return v < 0 ? -v : v; }

__host__ __device__ inline bool uv_adjacent(int4 a, int4 b) {
    const int sa = 1 << (21 - a.w), sb = 1 << (21 - b.w);
    const int dx = uv_iabs(a.x - b.x), dy = uv_iabs(a.y - b.y), dz = uv_iabs(a.z - b.z);
    const int sum = sa + sb;
    if (dx > sum || dy > sum || dz > sum) return false;
    const int dif = uv_iabs(sa - sb);
    return !(dx <= dif && dy <= dif && dz <= dif);
}

// N(c) into out[0 .. UV_NB); returns the count (more than UV_NB: an error the
// caller reports; only UV_NB are written).  Needs N(parent) done.
__host__ __device__ inline int uv_neighbours(const UvTree& T, int c, int32_t* out) {
    const int P = T.parent[c];
    if (P < 0) return 0;
    const int4 me = T.icentre[c];
    int cnt = 0;
    for (int k = -1; k < T.nbc[P]; k++) {
        const int Q = k < 0 ? P : T.nb[(int64_t)P * UV_NB + k];
        const int f = T.child_first[Q], e = f + T.child_count[Q];
        for (int x = f; x < e; x++) {
            if (x != c && uv_adjacent(me, T.icentre[x])) {
                if (cnt < UV_NB) out[cnt] = x;
                cnt++;
            }
        }
    }
    return cnt;
}

// V(c): emit(source) for every entry; returns the count
template <typename Emit>
__host__ __device__ inline int64_t uv_v_list(const UvTree& T, int c, Emit emit) {
    const int P = T.parent[c];
    if (P < 0) return 0;
    const int4 me = T.icentre[c];
    int64_t cnt = 0;
    for (int k = 0; k < T.nbc[P]; k++) {
        const int Q = T.nb[(int64_t)P * UV_NB + k];
        const int f = T.child_first[Q], e = f + T.child_count[Q];
        for (int x = f; x < e; x++)
            if (!uv_adjacent(me, T.icentre[x])) {
                emit(x);
                cnt++;
            }
    }
    return cnt;
}

// U(b) and W(b) of leaf b: emit_u(leaf), emit_w(cell).  Returns false when the
// descent stack would overflow (nothing past that point is emitted).
template <typename EmitU, typename EmitW>
__host__ __device__ inline bool uv_uw_lists(const UvTree& T, int b, EmitU emit_u, EmitW emit_w) {
    const int4 me = T.icentre[b];
    emit_u(b);
    // leaves among the neighbours of b (same level) and of its ancestors (coarser, if adjacent to b)
    for (int A = b; A >= 0; A = T.parent[A]) {
        for (int k = 0; k < T.nbc[A]; k++) {
            const int Q = T.nb[(int64_t)A * UV_NB + k];
            if (T.child_count[Q] == 0 && (A == b || uv_adjacent(T.icentre[Q], me))) emit_u(Q);
        }
    }
    // inside the neighbours that are not leaves: adjacent leaves (U), and the
    // first non-adjacent cell on every path (W); descent only through cells
    // adjacent to b
    int32_t stk[UV_STACK];
    for (int k = 0; k < T.nbc[b]; k++) {
        const int Q = T.nb[(int64_t)b * UV_NB + k];
        if (T.child_count[Q] == 0) continue;
        int sp = 0;
        for (int x = T.child_first[Q] + T.child_count[Q] - 1; x >= T.child_first[Q]; x--) stk[sp++] = x;
        while (sp > 0) {
            const int D = stk[--sp];
            if (uv_adjacent(T.icentre[D], me)) {
                const int cc = T.child_count[D];
                if (cc == 0) {
                    emit_u(D);
                } else {
                    if (sp + cc > UV_STACK) return false;
                    for (int x = T.child_first[D] + cc - 1; x >= T.child_first[D]; x--) stk[sp++] = x;
                }
            } else {
                emit_w(D);
            }
        }
    }
    return true;
}

// leaves inside cell D: the run [k0, k1) of the leaves in particle order
// (lfirst = their first particles, ascending)
__host__ __device__ inline void uv_leaf_run(const int32_t* lfirst, int nleaf, int32_t first, int32_t count, int& k0,
                                            int& k1) {
    int lo = 0, hi = nleaf;
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (lfirst[mid] < first) lo = mid + 1; else hi = mid;
    }
    k0 = lo;
    hi = nleaf;
    const int64_t end = (int64_t)first + count;
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if ((int64_t)lfirst[mid] < end) lo = mid + 1; else hi = mid;
    }
    k1 = lo;
}

}  // namespace fmm
