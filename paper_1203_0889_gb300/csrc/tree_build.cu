// tree_build.cu -- root cube, Morton keys, adaptive octree and breadth-first
// dual tree traversal on the device (paper Sections 2.1, 2.2, 4 and 5).
//
// All integer work (keys, cells, lists) is bit-exact with the CPU oracle: the
// FP64 quantisation uses explicit round-to-nearest intrinsics (no FMA
// contraction), the acceptance test compares an exact integer with one FP64
// product, and the lists are put in canonical (target, source) order by a
// radix sort.
#include <cooperative_groups.h>
#include <cub/cub.cuh>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

// ---------------------------------------------------------------------------
// allocation helpers (stream-ordered pool allocator)
// ---------------------------------------------------------------------------

template <typename T>
int dev_alloc(T** p, size_t count, fmm_tree* t, cudaStream_t st) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), st);
    if (e != cudaSuccess) {
        fmm_set_error("cudaMallocAsync(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
        return FMM_ERR_ALLOC;
    }
    if (t) t->device_bytes += (int64_t)(count * sizeof(T));
    return FMM_OK;
}
template int dev_alloc<uint64_t>(uint64_t**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<int32_t>(int32_t**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<int64_t>(int64_t**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<double>(double**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<char>(char**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<int4>(int4**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<__nv_bfloat16>(__nv_bfloat16**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<int2>(int2**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<double4_32a>(double4_32a**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<unsigned long long>(unsigned long long**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<cplx<float>>(cplx<float>**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<char2>(char2**, size_t, fmm_tree*, cudaStream_t);
template int dev_alloc<int8_t>(int8_t**, size_t, fmm_tree*, cudaStream_t);

template <typename T>
static void dev_free(T*& p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
}

// grow a device array to hold `need` elements, keeping `keep` of them
template <typename T>
static int grow(T*& p, size_t& cap, size_t need, size_t keep, cudaStream_t st) {
    if (need <= cap) return FMM_OK;
    size_t nc = std::max(need, cap * 2);
    T* q = nullptr;
    int rc = dev_alloc(&q, nc, (fmm_tree*)nullptr, st);
    if (rc) return rc;
    if (keep) FMM_CUDA_TRY(cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, st));
    dev_free(p, st);
    p = q;
    cap = nc;
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// root cube and keys
// ---------------------------------------------------------------------------

constexpr int BB_THREADS = 256;

// Block b reduces particles [blk[2b], blk[2b+1]) (one system's share).
template <typename T>
__global__ void k_bbox_partial(const T* __restrict__ pos, const int64_t* __restrict__ blk, double* part, Geometry* g) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int bad = 0;
    const int64_t i0 = blk[2 * blockIdx.x], i1 = blk[2 * blockIdx.x + 1];
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        for (int d = 0; d < 3; d++) {
            double v = (double)pos[3 * i + d];
            if (!isfinite(v)) bad = 1;
            lo[d] = fmin(lo[d], v);
            hi[d] = fmax(hi[d], v);
        }
    }
    __shared__ double s[6][BB_THREADS];
    for (int d = 0; d < 3; d++) { s[d][threadIdx.x] = lo[d]; s[3 + d][threadIdx.x] = hi[d]; }
    if (bad) g->bad = 1;
    __syncthreads();
    for (int w = BB_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int d = 0; d < 3; d++) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + w]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; k++) part[blockIdx.x * 6 + k] = s[k][0];
}

// Root cube of system s (same operation sequence as the oracle): side = longest
// extent (1 if zero), origin = (lo + hi) * 0.5 - side * 0.5, inv = 2^21 / side.
// One warp per system reduces the partials of the system's blocks
// [sblk[s], sblk[s+1]); min/max are exact, so the order does not matter.
__global__ void k_bbox_final(const double* part, const int32_t* sblk, int nsys, Geometry* gs) {
    const int sy = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (sy >= nsys) return;
    Geometry* g = gs + sy;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = sblk[sy] + lane; b < sblk[sy + 1]; b += 32)
        for (int d = 0; d < 3; d++) {
            lo[d] = fmin(lo[d], part[b * 6 + d]);
            hi[d] = fmax(hi[d], part[b * 6 + 3 + d]);
        }
    if (lane == 0 && gs[0].bad) g->bad = 1;
    for (int o = 16; o > 0; o >>= 1)
        for (int d = 0; d < 3; d++) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    if (lane != 0) return;
    double s = 0.0;
    for (int d = 0; d < 3; d++) s = fmax(s, __dsub_rn(hi[d], lo[d]));
    if (s == 0.0) s = 1.0;
    for (int d = 0; d < 3; d++) {
        g->origin[d] = __dsub_rn(__dmul_rn(__dadd_rn(lo[d], hi[d]), 0.5), __dmul_rn(s, 0.5));
        g->centre[d] = __dadd_rn(g->origin[d], __dmul_rn(s, 0.5));
    }
    g->side = s;
    g->inv = __ddiv_rn(2097152.0, s);
}

// 21 bits -> bits 0, 3, 6, ... (every third bit)
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
}
__device__ __forceinline__ int64_t compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (int64_t)v;
}

__device__ __forceinline__ uint64_t quantise(double x, double o, double inv) {
    double v = floor(__dmul_rn(__dsub_rn(x, o), inv));
    if (v < 0.0) v = 0.0;
    if (v > 2097151.0) v = 2097151.0;
    return (uint64_t)v;
}

__device__ __forceinline__ int system_of(int64_t i, const int64_t* off, int nsys) {
    int a = 0, b = nsys;   // last s with off[s] <= i
    while (b - a > 1) {
        int mid = (a + b) >> 1;
        if (off[mid] <= i) a = mid; else b = mid;
    }
    return a;
}

template <typename T>
__global__ void k_keys(const T* __restrict__ pos, int64_t n, const int64_t* __restrict__ off, int nsys,
                       const Geometry* __restrict__ gs, uint64_t* keys, int32_t* idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Geometry* g = gs + system_of(i, off, nsys);
    uint64_t kx = quantise((double)pos[3 * i], g->origin[0], g->inv);
    uint64_t ky = quantise((double)pos[3 * i + 1], g->origin[1], g->inv);
    uint64_t kz = quantise((double)pos[3 * i + 2], g->origin[2], g->inv);
    keys[i] = spread3(kx) | (spread3(ky) << 1) | (spread3(kz) << 2);
    idx[i] = (int32_t)i;
}

template <typename T>
__global__ void k_gather_pos(const T* __restrict__ pos, const int32_t* __restrict__ perm, int64_t n,
                             double* spos) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    spos[3 * i] = (double)pos[3 * j];
    spos[3 * i + 1] = (double)pos[3 * j + 1];
    spos[3 * i + 2] = (double)pos[3 * j + 2];
}

// ---------------------------------------------------------------------------
// octree, one level at a time
// ---------------------------------------------------------------------------

// Children of cell c are the distinct values of key >> shift within its
// particle range.  Eight lanes serve one cell: lane o finds the end of octant
// o (first particle whose prefix exceeds base + o) by binary search, so the
// eight searches run side by side; octant o spans [end(o-1), end(o)).
__device__ __forceinline__ int octant_end(const uint64_t* keys, int f, int e, uint64_t lim, int shift) {
    int a = f, b = e;
    while (a < b) {
        int mid = (a + b) >> 1;
        if ((keys[mid] >> shift) <= lim) a = mid + 1; else b = mid;
    }
    return a;
}

// first index in [lo, hi) whose (key >> shift) > lim (hi if none), found by
// the whole warp with 31 probes per step (all lanes call it with equal
// arguments; lanes read the result)
__device__ __forceinline__ int warp_upper_bound(const uint64_t* __restrict__ keys, int lo, int hi, uint64_t lim,
                                                int shift) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) / 32;
        const int pk = lo + (lane + 1) * step;
        const bool le_ = lane < 31 && pk < hi && (keys[pk] >> shift) <= lim;
        const int c = __popc(__ballot_sync(0xffffffffu, le_));
        const int nlo = c > 0 ? lo + c * step + 1 : lo;
        const int nhi = min(hi, lo + (c + 1) * step);
        lo = nlo;
        hi = nhi;
    }
    const bool le_ = lo + lane < hi && (keys[lo + lane] >> shift) <= lim;
    return lo + __popc(__ballot_sync(0xffffffffu, le_));
}

// Octant boundaries of the cells [lb, le) that split: ends[8 (c - lb) + o] =
// first particle above octant o.  wide = one warp per (cell, octant) with the
// 32-way search (narrow levels: few cells, long particle ranges); otherwise
// 8 lanes per cell, one binary search each.  Then nchild[c - lb] = number of
// non-empty octants.
__global__ void k_count_children(int lb, int le, int level, int leaf_size, int wide, const int32_t* first,
                                 const int32_t* count, const uint64_t* ckey, const uint64_t* keys,
                                 int32_t* ends, int32_t* nchild) {
    const int shift = 3 * (FMM_MAX_LEVEL - (level + 1));
    if (wide) {
        const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // one warp per (cell, octant)
        const int c = lb + (u >> 3), o = u & 7;
        if (c >= le) return;                                           // warp-uniform
        const int cnt = count[c];
        if (!(cnt > leaf_size && level < FMM_MAX_LEVEL)) {
            if ((threadIdx.x & 31) == 0 && o == 0) nchild[c - lb] = 0;
            return;
        }
        const int f = first[c];
        const int e = warp_upper_bound(keys, f, f + cnt, (ckey[c] << 3) + (uint64_t)o, shift);
        if ((threadIdx.x & 31) == 0) ends[u] = e;
        return;
    }
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    int c = lb + (g >> 3), o = g & 7;
    bool valid = c < le;
    int cnt = valid ? count[c] : 0;
    bool split = valid && cnt > leaf_size && level < FMM_MAX_LEVEL;
    int f = valid ? first[c] : 0;
    int end = split ? octant_end(keys, f, f + cnt, (ckey[c] << 3) + (uint64_t)o, shift) : 0;
    if (split) ends[g] = end;
    int beg = __shfl_up_sync(0xffffffffu, end, 1, 8);
    if (o == 0) beg = f;
    unsigned nonempty = __ballot_sync(0xffffffffu, split && end > beg);
    if (valid && o == 0) nchild[c - lb] = __popc((nonempty >> (threadIdx.x & 24)) & 0xffu);
}

// child counts of the wide levels (after the warp searches)
__global__ void k_count_from_ends(int lb, int le, int level, int leaf_size, const int32_t* first,
                                  const int32_t* count, const int32_t* ends, int32_t* nchild) {
    const int c = lb + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= le) return;
    const int cnt = count[c];
    if (!(cnt > leaf_size && level < FMM_MAX_LEVEL)) { nchild[c - lb] = 0; return; }
    int beg = first[c], k = 0;
    for (int o = 0; o < 8; o++) {
        const int e = ends[8 * (c - lb) + o];
        k += e > beg;
        beg = e;
    }
    nchild[c - lb] = k;
}

__global__ void k_emit_children(int lb, int le, int level, const int32_t* ends, const int32_t* nchild,
                                const int32_t* coff, int next_base, int32_t* lev, uint64_t* ckey, int32_t* first,
                                int32_t* count, int32_t* parent, int32_t* child_first, int32_t* child_count) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    int c = lb + (g >> 3), o = g & 7;
    bool valid = c < le;
    int nc = valid ? nchild[c - lb] : 0;
    int f = valid ? first[c] : 0;
    uint64_t base = valid ? (ckey[c] << 3) : 0;
    int end = nc ? ends[g] : 0;
    int beg = __shfl_up_sync(0xffffffffu, end, 1, 8);
    if (o == 0) beg = f;
    bool ne = nc && end > beg;
    unsigned m8 = (__ballot_sync(0xffffffffu, ne) >> (threadIdx.x & 24)) & 0xffu;
    if (!valid) return;
    int w = next_base + coff[c - lb];
    if (o == 0) {
        child_first[c] = nc ? w : 0;
        child_count[c] = nc;
    }
    if (!ne) return;
    w += __popc(m8 & ((1u << o) - 1u));
    lev[w] = level + 1;
    ckey[w] = base + (uint64_t)o;
    first[w] = beg;
    count[w] = end - beg;
    parent[w] = c;
}

__global__ void k_centres(int ncell, const int32_t* lev, const uint64_t* ckey, const int32_t* first,
                          const int64_t* off, int nsys, const Geometry* gs, double4_32a* centre, int4* icentre,
                          float* cu2f) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const Geometry* g = gs + system_of(first[c], off, nsys);
    cu2f[c] = (float)__ddiv_rn(g->side, 4194304.0);
    int l = lev[c];
    int64_t s = (int64_t)1 << (FMM_MAX_LEVEL - l);
    uint64_t k = ckey[c];
    double u2 = __ddiv_rn(g->side, 4194304.0);  // side / 2^22: the unit of twice a centre
    double x[3];
    int ic[3];
    for (int d = 0; d < 3; d++) {
        int64_t kc = compact3(k >> d);
        int64_t twoc = 2 * kc * s + s;
        ic[d] = (int)twoc;
        x[d] = __dadd_rn(g->origin[d], __dmul_rn((double)twoc, u2));
    }
    icentre[c] = make_int4(ic[0], ic[1], ic[2], l);
    centre[c] = make_double4_32a(x[0], x[1], x[2], __dmul_rn((double)s, __ddiv_rn(g->side, 2097152.0)));
}

// ---------------------------------------------------------------------------
// octree in one pass over the sorted keys
// ---------------------------------------------------------------------------
//
// The cell of level L that holds particle a is the run of particles sharing
// a's level-L key prefix.  It splits (Section 2.1) iff it holds more than
// S = leaf_size particles and L < FMM_MAX_LEVEL, and it holds more than S
// particles iff some window of S + 1 consecutive sorted particles containing a
// shares that prefix.  With m(s) = number of levels particles s and s + S have
// in common (-1 when they lie in different systems), M(a) = max m(s) over
// s in [a - S, a] is the deepest level whose cell around a holds more than S
// particles, so a's leaf is at level hi(a) = min(M(a) + 1, FMM_MAX_LEVEL)
// (0 when M(a) < 0).  a is the first particle of its level-L cell iff L is
// deeper than the levels it shares with particle a - 1, so the cells that
// start at a are those of levels lo(a) .. hi(a).  Counting them per level and
// block and scanning the counts places every cell in (level, position) order,
// which is (level, system, key) order.

constexpr int OCT_B = 256;                        // particles per block
constexpr int OCT_NL = FMM_MAX_LEVEL + 1;         // levels 0 .. FMM_MAX_LEVEL

// levels two keys have in common: prefixes key >> 3 (FMM_MAX_LEVEL - L) agree
// for L <= 20 - (highest differing bit) / 3, and at every level when equal
__device__ __forceinline__ int common_levels(uint64_t k1, uint64_t k2) {
    const uint64_t x = k1 ^ k2;
    return x ? 20 - (63 - __clzll((long long)x)) / 3 : FMM_MAX_LEVEL;
}

// per-block cell and leaf counts of every level of the particles of one block
__device__ __forceinline__ void oct_warp_counts(int lo, int hi, int (*wc)[2 * OCT_NL]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int L = 0; L < OCT_NL; L++) {
        const bool in = lo <= L && L <= hi;
        const unsigned mc = __ballot_sync(0xffffffffu, in);
        const unsigned ml = __ballot_sync(0xffffffffu, in && L == hi);
        if (lane == 0) { wc[w][L] = __popc(mc); wc[w][OCT_NL + L] = __popc(ml); }
    }
}

// lo(a), hi(a) of every particle; cnt[j * nb + b] = cells (j < OCT_NL) or
// leaves (j >= OCT_NL) of level j % OCT_NL starting in block b.
// Dynamic shared memory: 2 (OCT_B + S) bytes.
__global__ void __launch_bounds__(OCT_B) k_oct_levels(const uint64_t* __restrict__ keys, int64_t n,
                                                      const int64_t* __restrict__ off, int nsys, int S, int nb,
                                                      char2* __restrict__ lohi, int64_t* __restrict__ cnt) {
    extern __shared__ signed char oct_sm[];
    __shared__ int wc[OCT_B / 32][2 * OCT_NL];
    const int Lb = OCT_B + S;
    signed char* x = oct_sm;
    signed char* y = oct_sm + Lb;
    const int64_t A = (int64_t)blockIdx.x * OCT_B;
    // x[j] = m(A - S + j)
    for (int j = threadIdx.x; j < Lb; j += OCT_B) {
        const int64_t s = A - S + j;
        int v = -1;
        if (s >= 0 && s + S < n) {
            const int sy = nsys > 1 ? system_of(s, off, nsys) : 0;
            if (s + S < off[sy + 1]) v = common_levels(keys[s], keys[s + S]);
        }
        x[j] = (signed char)v;
    }
    __syncthreads();
    // doubling: after step k, x[j] = max of m over [A - S + j, A - S + j + 2^k)
    int k = 0;
    while ((2 << k) <= S + 1) k++;   // 2^k <= S + 1 < 2^(k+1)
    for (int st = 0; st < k; st++) {
        const int o = 1 << st;
        for (int j = threadIdx.x; j < Lb; j += OCT_B) y[j] = j + o < Lb ? max(x[j], x[j + o]) : x[j];
        __syncthreads();
        signed char* tmp = x;
        x = y;
        y = tmp;
    }
    const int t = threadIdx.x;
    const int64_t a = A + t;
    int lo = 1, hi = 0;   // no cell starts here
    if (a < n) {
        // window [a - S, a] = [A - S + t, A - S + t + 2^k) u [.. , A + t]
        const int M = max((int)x[t], (int)x[t + S + 1 - (1 << k)]);
        hi = M < 0 ? 0 : min(FMM_MAX_LEVEL, M + 1);
        const int sy = nsys > 1 ? system_of(a, off, nsys) : 0;
        lo = off[sy] == a ? 0 : common_levels(keys[a - 1], keys[a]) + 1;
        lohi[a] = make_char2((char)lo, (char)hi);
    }
    oct_warp_counts(lo, hi, wc);
    __syncthreads();
    if (t < 2 * OCT_NL) {
        int s = 0;
        for (int i = 0; i < OCT_B / 32; i++) s += wc[i][t];
        cnt[(int64_t)t * nb + blockIdx.x] = s;
    }
}

// hdr[L] = first cell of level L (L = 0 .. OCT_NL; hdr[OCT_NL] = cells),
// hdr[OCT_NL + 1] = leaves; the systems' root cubes follow at geo_out
__global__ void k_oct_summary(const int64_t* __restrict__ offs, const int64_t* __restrict__ cnt, int nb,
                              const Geometry* __restrict__ geom, int nsys, int64_t* hdr, Geometry* geo_out) {
    const int t = threadIdx.x;
    if (t <= OCT_NL) hdr[t] = offs[(int64_t)t * nb];
    if (t == 0) {
        const int64_t last = (int64_t)2 * OCT_NL * nb - 1;
        hdr[OCT_NL + 1] = offs[last] + cnt[last] - offs[(int64_t)OCT_NL * nb];
    }
    for (int s = t; s < nsys; s += blockDim.x) geo_out[s] = geom[s];
}

// writes level, key, first particle and count of every cell, and the leaf list
__global__ void __launch_bounds__(OCT_B) k_oct_emit(const uint64_t* __restrict__ keys, int64_t n,
                                                    const int64_t* __restrict__ off, int nsys, int nb,
                                                    const char2* __restrict__ lohi,
                                                    const int64_t* __restrict__ offs, int32_t* __restrict__ lev,
                                                    uint64_t* __restrict__ ckey, int32_t* __restrict__ first,
                                                    int32_t* __restrict__ count, int32_t* __restrict__ leaves) {
    __shared__ int wc[OCT_B / 32][2 * OCT_NL];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int64_t a = (int64_t)blockIdx.x * OCT_B + t;
    int lo = 1, hi = 0;
    if (a < n) {
        const char2 v = lohi[a];
        lo = v.x;
        hi = v.y;
    }
    oct_warp_counts(lo, hi, wc);
    __syncthreads();
    if (t < 2 * OCT_NL) {   // exclusive offsets of the warps within the block
        int s = 0;
        for (int i = 0; i < OCT_B / 32; i++) {
            const int c = wc[i][t];
            wc[i][t] = s;
            s += c;
        }
    }
    __syncthreads();
    const int64_t ncell = offs[(int64_t)OCT_NL * nb];
    const uint64_t key = a < n ? keys[a] : 0;
    int64_t se = 0;
    if (a < n && lo <= hi) se = off[(nsys > 1 ? system_of(a, off, nsys) : 0) + 1];
    const unsigned lt = (1u << lane) - 1u;
    int64_t good = a;   // last particle known to share a's prefix (the deeper level's run end - 1)
    for (int L = FMM_MAX_LEVEL; L >= 0; L--) {
        const bool in = lo <= L && L <= hi;
        const unsigned mc = __ballot_sync(0xffffffffu, in);
        const unsigned ml = __ballot_sync(0xffffffffu, in && L == hi);
        if (!in) continue;
        const int64_t idx = offs[(int64_t)L * nb + blockIdx.x] + wc[w][L] + __popc(mc & lt);
        const int shift = 3 * (FMM_MAX_LEVEL - L);
        const uint64_t pre = key >> shift;
        // end of the run sharing the prefix: gallop from the deeper run's end, then bisect
        int64_t step = 1;
        while (good + step < se && (keys[good + step] >> shift) == pre) {
            good += step;
            step <<= 1;
        }
        int64_t bad = min(good + step, se);
        while (bad - good > 1) {
            const int64_t mid = (good + bad) >> 1;
            if ((keys[mid] >> shift) == pre) good = mid; else bad = mid;
        }
        lev[idx] = L;
        ckey[idx] = pre;
        first[idx] = (int32_t)a;
        count[idx] = (int32_t)(bad - a);
        if (L == hi)
            leaves[offs[(int64_t)(OCT_NL + L) * nb + blockIdx.x] - ncell + wc[w][OCT_NL + L] + __popc(ml & lt)] =
                (int32_t)idx;
    }
}

struct LevelStarts {
    int32_t s[FMM_MAX_LEVEL + 2];
};

// first index in [lo, hi) of sorted v with v[i] >= x (hi if none)
__device__ __forceinline__ int lower_bound_i32(const int32_t* __restrict__ v, int lo, int hi, int64_t x) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// parent and children of every cell, by bisection over the first particles of
// the neighbouring levels (ordered by position within a level)
__global__ void k_oct_links(int ncell, LevelStarts ls, int S, const int32_t* __restrict__ lev,
                            const int32_t* __restrict__ first, const int32_t* __restrict__ count, int32_t* parent,
                            int32_t* child_first, int32_t* child_count) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int L = lev[c], a = first[c], n = count[c];
    // the last cell of level L - 1 whose first particle is <= a holds a
    parent[c] = L > 0 ? lower_bound_i32(first, ls.s[L - 1], ls.s[L], (int64_t)a + 1) - 1 : -1;
    int cf = 0, cc = 0;
    if (n > S && L < FMM_MAX_LEVEL) {
        cf = lower_bound_i32(first, ls.s[L + 1], ls.s[L + 2], a);
        cc = lower_bound_i32(first, cf, ls.s[L + 2], (int64_t)a + n) - cf;
    }
    child_first[c] = cf;
    child_count[c] = cc;
}

// ---------------------------------------------------------------------------
// breadth-first dual tree traversal
// ---------------------------------------------------------------------------

__global__ void k_init_roots(int nsys, const int64_t* off, int32_t* lev, uint64_t* ckey, int32_t* first,
                             int32_t* count, int32_t* parent) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    lev[s] = 0; ckey[s] = 0; first[s] = (int32_t)off[s]; count[s] = (int32_t)(off[s + 1] - off[s]); parent[s] = -1;
}

__global__ void k_init_frontier(int nsys, int2* front) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys) front[s] = make_int2(s, s);
}

struct TravCounters {
    unsigned long long nm2l, np2p, nnext;
};

// All 32 lanes call this; returns the lane's first slot of `cnt` slots.
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long* ctr, unsigned cnt) {
    const unsigned FULL = 0xffffffffu;
    unsigned lane = threadIdx.x & 31;
    unsigned v = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned t = __shfl_up_sync(FULL, v, o);
        if (lane >= (unsigned)o) v += t;
    }
    unsigned total = __shfl_sync(FULL, v, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(ctr, (unsigned long long)total);
    base = __shfl_sync(FULL, base, 31);
    return base + v - cnt;
}

// Block-wide version for three counters at once: every thread of the block
// calls it; thread t gets the first of its c[k] slots in counter k.  One global
// atomic per counter per call (the three counters are hot: every warp of the
// grid appends to them).
constexpr int TRAV_THREADS = 256;
__device__ __forceinline__ void block_reserve3(unsigned long long* ctr0, unsigned long long* ctr1,
                                               unsigned long long* ctr2, const unsigned c[3],
                                               unsigned long long slot[3]) {
    __shared__ unsigned wsum[3][TRAV_THREADS / 32];
    __shared__ unsigned long long base[3];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned v[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        v[k] = c[k];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(FULL, v[k], o);
            if (lane >= o) v[k] += t;
        }
        if (lane == 31) wsum[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int k = threadIdx.x;
        unsigned tot = 0;
        for (int w = 0; w < TRAV_THREADS / 32; w++) {
            const unsigned x = wsum[k][w];
            wsum[k][w] = tot;   // exclusive prefix over the warps
            tot += x;
        }
        unsigned long long* ctr = k == 0 ? ctr0 : (k == 1 ? ctr1 : ctr2);
        base[k] = tot ? atomicAdd(ctr, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; k++) slot[k] = base[k] + wsum[k][warp] + v[k] - c[k];
    __syncthreads();   // wsum / base are reused by the next call
}

__global__ void k_traverse(const int2* __restrict__ front, int64_t nf, const int32_t* __restrict__ lev,
                           const uint64_t* __restrict__ ckey, const int32_t* __restrict__ child_first,
                           const int32_t* __restrict__ child_count, double th2, int2* m2l, int2* p2p,
                           int2* next, TravCounters* cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool valid = i < nf;
    int action = -1, nsplit = 0, split_target = 0, ci = 0, cj = 0;
    if (valid) {
        int2 pr = front[i];
        ci = pr.x; cj = pr.y;
        int li = lev[ci], lj = lev[cj];
        int64_t si = (int64_t)1 << (FMM_MAX_LEVEL - li), sj = (int64_t)1 << (FMM_MAX_LEVEL - lj);
        uint64_t ki = ckey[ci], kj = ckey[cj];
        int64_t D2 = 0;
        for (int d = 0; d < 3; d++) {
            int64_t a = 2 * compact3(ki >> d) * si + si;
            int64_t b = 2 * compact3(kj >> d) * sj + sj;
            D2 += (a - b) * (a - b);
        }
        int64_t S = si + sj;
        bool accept = (double)(S * S) < __dmul_rn(th2, (double)D2);
        bool leaf_i = child_count[ci] == 0, leaf_j = child_count[cj] == 0;
        if (accept) action = 0;
        else if (leaf_i && leaf_j) action = 1;
        else {
            action = 2;
            split_target = leaf_j || (!leaf_i && li <= lj);
            nsplit = split_target ? child_count[ci] : child_count[cj];
        }
    }
    unsigned long long s0 = warp_reserve(&cnt->nm2l, action == 0 ? 1u : 0u);
    unsigned long long s1 = warp_reserve(&cnt->np2p, action == 1 ? 1u : 0u);
    unsigned long long s2 = warp_reserve(&cnt->nnext, (unsigned)nsplit);
    if (action == 0) m2l[s0] = make_int2(ci, cj);
    else if (action == 1) p2p[s1] = make_int2(ci, cj);
    else if (action == 2) {
        if (split_target) {
            int cf = child_first[ci];
            for (int k = 0; k < nsplit; k++) next[s2 + k] = make_int2(cf + k, cj);
        } else {
            int cf = child_first[cj];
            for (int k = 0; k < nsplit; k++) next[s2 + k] = make_int2(ci, cf + k);
        }
    }
}

struct TravState {
    // frontier sizes, rotating: round r reads front[r % 3] and appends to
    // front[(r + 1) % 3]; front[(r + 2) % 3] is cleared during round r
    unsigned long long front[3];
    unsigned long long nm2l, np2p;
    // overflow seen in round r goes to ovf[r % 2], read by every thread only at
    // the top of round r + 1 (after the barrier), so all threads decide alike
    int ovf[2], rounds;
};

// (first child, child count) of every cell, one 8-byte load in the traversal
__global__ void k_child_pack(int ncell, const int32_t* __restrict__ cf, const int32_t* __restrict__ cc, int2* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) out[c] = make_int2(cf[c], cc[c]);
}

// The multipole acceptance test on the integer centres: icentre holds twice
// each centre in units of 2^-22 of the system's side (and the level), so
// D2 = sum (2 c_i - 2 c_j)^2 and S = s_i + s_j are the same integers the
// Morton keys give.
__device__ __forceinline__ void traverse_pair(int ci, int cj, bool valid, const int4* __restrict__ icentre,
                                              const int2* __restrict__ child, double th2, int2* m2l, int2* p2p,
                                              int2* next, TravState* stt, unsigned long long* nnext, int* ovf,
                                              unsigned long long cap_m, unsigned long long cap_p,
                                              unsigned long long cap_f) {
    int action = -1, nsplit = 0, split_target = 0, cfirst = 0;
    if (valid) {
        const int4 a = icentre[ci], b = icentre[cj];
        const int2 ch_i = child[ci], ch_j = child[cj];
        const int64_t si = (int64_t)1 << (FMM_MAX_LEVEL - a.w), sj = (int64_t)1 << (FMM_MAX_LEVEL - b.w);
        const int64_t dx = (int64_t)a.x - b.x, dy = (int64_t)a.y - b.y, dz = (int64_t)a.z - b.z;
        const int64_t D2 = dx * dx + dy * dy + dz * dz;
        const int64_t S = si + sj;
        const bool accept = (double)(S * S) < __dmul_rn(th2, (double)D2);
        const bool leaf_i = ch_i.y == 0, leaf_j = ch_j.y == 0;
        if (accept) action = 0;
        else if (leaf_i && leaf_j) action = 1;
        else {
            action = 2;
            split_target = leaf_j || (!leaf_i && a.w <= b.w);
            nsplit = split_target ? ch_i.y : ch_j.y;
            cfirst = split_target ? ch_i.x : ch_j.x;
        }
    }
    const unsigned cnt[3] = {action == 0 ? 1u : 0u, action == 1 ? 1u : 0u, (unsigned)nsplit};
    unsigned long long sl[3];
    block_reserve3(&stt->nm2l, &stt->np2p, nnext, cnt, sl);
    const unsigned long long s0 = sl[0], s1 = sl[1], s2 = sl[2];
    if (action == 0) {
        if (s0 < cap_m) m2l[s0] = make_int2(ci, cj); else *ovf = 1;
    } else if (action == 1) {
        if (s1 < cap_p) p2p[s1] = make_int2(ci, cj); else *ovf = 1;
    } else if (action == 2) {
        if (s2 + nsplit > cap_f) { *ovf = 1; return; }
        if (split_target) {
            for (int k = 0; k < nsplit; k++) next[s2 + k] = make_int2(cfirst + k, cj);
        } else {
            for (int k = 0; k < nsplit; k++) next[s2 + k] = make_int2(ci, cfirst + k);
        }
    }
}

// All rounds of the breadth-first traversal in one cooperative launch, one
// grid-wide barrier per round (the frontier counters rotate, see TravState).
// Writes are checked against the buffer capacities; on overflow the kernel
// stops and reports it, and the host reruns the traversal round by round
// with growing buffers.
__global__ void k_traverse_coop(int2* fa, int2* fb, const int4* __restrict__ icentre, const int2* __restrict__ child,
                                double th2, int2* m2l, int2* p2p, TravState* stt, unsigned long long cap_m,
                                unsigned long long cap_p, unsigned long long cap_f) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long gtid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long bbase = (unsigned long long)blockIdx.x * blockDim.x;   // block-uniform loop
    for (int round = 0;; round++) {
        int2* cur = (round & 1) ? fb : fa;
        int2* nxt = (round & 1) ? fa : fb;
        const unsigned long long nf = *(volatile unsigned long long*)&stt->front[round % 3];
        // overflow of the previous round (written before the barrier only)
        const int ovf_prev = round > 0 ? *(volatile int*)&stt->ovf[(round + 1) & 1] : 0;
        if (nf == 0 || ovf_prev) {
            if (gtid == 0) stt->rounds = round;
            break;
        }
        if (gtid == 0) stt->front[(round + 2) % 3] = 0;
        unsigned long long* nnext = &stt->front[(round + 1) % 3];
        int* ovf = &stt->ovf[round & 1];
        for (unsigned long long base = bbase; base < nf; base += nthreads) {
            const unsigned long long i = base + threadIdx.x;
            const bool valid = i < nf;
            const int2 pr = valid ? cur[i] : make_int2(0, 0);
            traverse_pair(pr.x, pr.y, valid, icentre, child, th2, m2l, p2p, nxt, stt, nnext, ovf, cap_m, cap_p,
                          cap_f);
        }
        grid.sync();
    }
}

// (target, source) packed as target * 2^B + source, B = bits of the cell count,
// so the sort touches 2B bits
__global__ void k_pack_pairs(const int2* pr, int64_t np, int B, uint64_t* key) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < np) key[i] = ((uint64_t)(uint32_t)pr[i].x << B) | (uint32_t)pr[i].y;
}

__global__ void k_unpack_sources(const uint64_t* key, int64_t np, int B, int32_t* src, int32_t* tgt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    src[i] = (int32_t)(key[i] & ((1ull << B) - 1ull));
    if (tgt) tgt[i] = (int32_t)(key[i] >> B);
}

// start[c] = first list entry whose target is >= c, for c = 0..ncell
__global__ void k_csr_start(const uint64_t* key, int64_t np, int ncell, int B, int64_t* start) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    uint64_t lim = (uint64_t)c << B;
    int64_t a = 0, b = np;
    while (a < b) {
        int64_t mid = (a + b) >> 1;
        if (key[mid] < lim) a = mid + 1; else b = mid;
    }
    start[c] = a;
}

// P2P pairs join two leaves, and leaves in cell order are leaves in rank
// order, so the list sorts on (target rank, source rank): 2 bits_for(nleaf)
// bits, 32-bit keys while they fit, instead of two cell indices.
__global__ void k_leaf_rank(int nleaf, const int32_t* __restrict__ leaves, int32_t* lrank) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nleaf) lrank[leaves[i]] = i;
}
template <typename K>
__global__ void k_pack_leaf_pairs(const int2* __restrict__ pr, int64_t np, int B, const int32_t* __restrict__ lrank,
                                  K* key) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < np) key[i] = ((K)(uint32_t)lrank[pr[i].x] << B) | (K)(uint32_t)lrank[pr[i].y];
}
// sorted keys back to cells; cnt[e] = particles of the source (for the records)
template <typename K>
__global__ void k_unpack_leaf_pairs(const K* __restrict__ key, int64_t np, int B, const int32_t* __restrict__ leaves,
                                    const int32_t* __restrict__ count, int32_t* src, int32_t* tgt, int64_t* cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const K k = key[i];
    const int s = leaves[(int)(k & (((K)1 << B) - 1))];
    src[i] = s;
    tgt[i] = leaves[(int)(k >> B)];
    cnt[i] = count[s];
}
// start[c] = first entry whose target rank is at least the number of leaves
// before cell c (cells that are not leaves get empty ranges), c = 0..ncell
template <typename K>
__global__ void k_csr_start_leaf(const K* __restrict__ key, int64_t np, int ncell, int nleaf, int B,
                                 const int32_t* __restrict__ leaves, int64_t* start) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    int a = 0, b = nleaf;
    while (a < b) {
        const int mid = (a + b) >> 1;
        if (leaves[mid] < c) a = mid + 1; else b = mid;
    }
    const K lim = (K)(uint32_t)a << B;
    int64_t lo = 0, hi = np;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key[mid] < lim) lo = mid + 1; else hi = mid;
    }
    start[c] = lo;
}

// P2P records: source range and where its particles start in the target's
// concatenated source stream (exclusive prefix of counts within the target)
__global__ void k_p2p_counts(int64_t np, const int32_t* src, const int32_t* count, int64_t* cnt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < np) cnt[e] = count[src[e]];
}
__global__ void k_p2p_records(int64_t np, const int32_t* src, const int32_t* tgt, const int64_t* start,
                              const int32_t* first, const int32_t* count, const int64_t* gcum, int4* rec) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= np) return;
    int s = src[e];
    rec[e] = make_int4(first[s], count[s], (int)(gcum[e] - gcum[start[tgt[e]]]), s);
}

// P2P work items of the stage-by-stage kernel.  A leaf whose list holds more
// than R (prm.p2p_item_records) source records (a coarse leaf beside much finer ones
// can hold thousands) is split into runs of that many records, so that no
// block carries a large share of the kernel; the split leaves' items come
// first in the grid, then one item per other leaf.
__global__ void k_p2p_item_counts(int nleaf, int split_ok, int R, const int32_t* __restrict__ leaves,
                                  const int64_t* __restrict__ start, const int32_t* __restrict__ count,
                                  int32_t* nsplit, int32_t* nwhole, int64_t* nslot) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaf) return;
    const int c = leaves[i];
    const int64_t nrec = start[c + 1] - start[c];
    const int k = split_ok && nrec > R ? (int)((nrec + R - 1) / R) : 1;
    nsplit[i] = k > 1 ? k : 0;
    nwhole[i] = k > 1 ? 0 : 1;
    nslot[i] = k > 1 ? (int64_t)k * count[c] : 0;   // partial slots: items x targets
}
__global__ void k_p2p_items(int nleaf, int R, const int32_t* __restrict__ leaves, const int64_t* __restrict__ start,
                            const int32_t* __restrict__ nsplit, const int32_t* __restrict__ osplit,
                            const int32_t* __restrict__ owhole, const int64_t* __restrict__ nslot,
                            const int64_t* __restrict__ oslot, int4* items, int4* split, int32_t* nitems) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaf) return;
    const int c = leaves[i];
    const int nrec = (int)(start[c + 1] - start[c]);
    const int nsp = osplit[nleaf - 1] + nsplit[nleaf - 1];   // items of split leaves
    const int k = nsplit[i];
    if (k > 0) {
        const int64_t b = oslot[i];
        for (int j = 0; j < k; j++) {
            items[osplit[i] + j] = make_int4(c, j * R, min(R, nrec - j * R), 1 | (j == 0 ? 2 : 0));
            split[osplit[i] + j] = make_int4(k, j, (int)(uint32_t)b, (int)(b >> 32));
        }
    } else {
        items[nsp + owhole[i]] = make_int4(c, 0, nrec, 2);
    }
    if (i == nleaf - 1) {
        nitems[0] = nsp + owhole[i] + (k > 0 ? 0 : 1);
        nitems[1] = nsp;
        const int64_t ns = oslot[i] + nslot[i];   // partial slots, as two words
        nitems[2] = (int32_t)(uint32_t)ns;
        nitems[3] = (int32_t)(ns >> 32);
    }
}

__global__ void k_leaf_flags(int ncell, const int32_t* child_count, char* flag, int32_t* iota) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) { flag[c] = child_count[c] == 0; iota[c] = c; }
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// leaf index of every sorted particle (one warp per leaf)
__global__ void k_particle_leaf(int nleaf, const int32_t* __restrict__ leaves, const int32_t* __restrict__ first,
                                const int32_t* __restrict__ count, int32_t* pleaf) {
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nleaf) return;
    int c = leaves[w];
    for (int i = first[c] + lane; i < first[c] + count[c]; i += 32) pleaf[i] = c;
}

static int bits_for(int64_t v) {
    int b = 1;
    while (((int64_t)1 << b) <= v && b < 63) b++;
    return b;
}

// sort (target, source) pairs and build the CSR arrays
static int finish_list(fmm_tree* t, int2* pairs, int64_t np, int64_t** start, int32_t** src,
                       int32_t** tgt, cudaStream_t st) {
    int rc;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    if ((rc = dev_alloc(&k0, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&k1, np, nullptr, st))) return rc;
    const int B = bits_for(t->ncell);
    if (np) { k_pack_pairs<<<nblk(np, 256), 256, 0, st>>>(pairs, np, B, k0); count_launch(t); }
    size_t tmp_bytes = 0;
    int end_bit = 2 * B;
    cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, k0, k1, (int64_t)np, 0, end_bit, st);
    char* tmp = nullptr;
    if ((rc = dev_alloc(&tmp, tmp_bytes, nullptr, st))) return rc;
    if (np) { FMM_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp, tmp_bytes, k0, k1, (int64_t)np, 0, end_bit, st)); count_launch(t); }
    if ((rc = dev_alloc(src, np, t, st))) return rc;
    if ((rc = dev_alloc(start, (size_t)t->ncell + 1, t, st))) return rc;
    if (tgt && (rc = dev_alloc(tgt, np, t, st))) return rc;
    if (np) { k_unpack_sources<<<nblk(np, 256), 256, 0, st>>>(k1, np, B, *src, tgt ? *tgt : nullptr); count_launch(t); }
    k_csr_start<<<nblk(t->ncell + 1, 256), 256, 0, st>>>(k1, np, t->ncell, B, *start);
    count_launch(t);
    dev_free(tmp, st);
    dev_free(k0, st);
    dev_free(k1, st);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}


// The P2P list as CSR by target with its records (source range, offset of its
// particles in the target's source stream).  *tgt receives the target of each
// entry (freed by the caller).
template <typename K>
static int p2p_list_sorted(fmm_tree* t, int2* pairs, int64_t np, int B, int32_t* tgt, int64_t* cnt,
                           cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    K *k0 = nullptr, *k1 = nullptr;
    int32_t* lrank = nullptr;
    char* tmp = nullptr;
    if ((rc = dev_alloc((char**)&k0, sizeof(K) * (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc((char**)&k1, sizeof(K) * (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&lrank, (size_t)t->ncell, nullptr, st))) return rc;
    k_leaf_rank<<<nblk(t->nleaf, 256), 256, 0, st>>>(t->nleaf, d.leaves, lrank);
    k_pack_leaf_pairs<K><<<nblk(np, 256), 256, 0, st>>>(pairs, np, B, lrank, k0);
    size_t tb = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, tb, k0, k1, np, 0, 2 * B, st);
    if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp, tb, k0, k1, np, 0, 2 * B, st));
    k_unpack_leaf_pairs<K><<<nblk(np, 256), 256, 0, st>>>(k1, np, B, d.leaves, d.count, d.p2p_src, tgt, cnt);
    k_csr_start_leaf<K><<<nblk(t->ncell + 1, 256), 256, 0, st>>>(k1, np, t->ncell, t->nleaf, B, d.leaves,
                                                                 d.p2p_start);
    count_launch(t, 5);
    dev_free(tmp, st);
    dev_free(k0, st);
    dev_free(k1, st);
    dev_free(lrank, st);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

static int finish_p2p_list(fmm_tree* t, int2* pairs, int64_t np, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    int32_t* tgt = nullptr;
    int64_t *cnt = nullptr, *gcum = nullptr;
    char* tmp = nullptr;
    if (t->prm.flags & FMM_BUILD_FALLBACKS) {
        // the generic list (cell-index keys), counts by a separate pass
        if ((rc = finish_list(t, pairs, np, &d.p2p_start, &d.p2p_src, &tgt, st))) return rc;
        if ((rc = dev_alloc(&cnt, (size_t)np, nullptr, st))) return rc;
        if (np) { k_p2p_counts<<<nblk(np, 256), 256, 0, st>>>(np, d.p2p_src, d.count, cnt); count_launch(t); }
    } else {
        if ((rc = dev_alloc(&d.p2p_src, (size_t)np, t, st))) return rc;
        if ((rc = dev_alloc(&d.p2p_start, (size_t)t->ncell + 1, t, st))) return rc;
        if ((rc = dev_alloc(&tgt, (size_t)np, nullptr, st))) return rc;
        if ((rc = dev_alloc(&cnt, (size_t)np, nullptr, st))) return rc;
        const int B = bits_for(t->nleaf);
        if (np == 0) {
            FMM_CUDA_TRY(cudaMemsetAsync(d.p2p_start, 0, sizeof(int64_t) * ((size_t)t->ncell + 1), st));
        } else if (2 * B <= 32) {
            if ((rc = p2p_list_sorted<uint32_t>(t, pairs, np, B, tgt, cnt, st))) return rc;
        } else {
            if ((rc = p2p_list_sorted<uint64_t>(t, pairs, np, B, tgt, cnt, st))) return rc;
        }
    }
    if ((rc = dev_alloc(&gcum, (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&d.p2p_rec, (size_t)np, t, st))) return rc;
    if (np) {
        size_t sb = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, sb, cnt, gcum, np, st);
        if ((rc = dev_alloc(&tmp, sb, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, sb, cnt, gcum, np, st));
        dev_free(tmp, st);
        k_p2p_records<<<nblk(np, 256), 256, 0, st>>>(np, d.p2p_src, tgt, d.p2p_start, d.first, d.count, gcum,
                                                        d.p2p_rec);
        count_launch(t, 2);
        if (p2p_mutual(t) && (rc = build_p2p_modes(t, tgt, st))) return rc;
    }
    dev_free(cnt, st);
    dev_free(gcum, st);
    dev_free(tgt, st);
    // work items of the stage-by-stage P2P kernel; their count reaches the
    // tree's pinned words when the build synchronises
    if (t->nleaf > 0) {
        const int nl = t->nleaf;
        const int R = t->prm.p2p_item_records;
        t->p2p_items_bound = nl + (np + R - 1) / R;
        int32_t* w = nullptr;
        int64_t* w64 = nullptr;
        const size_t nb = (size_t)t->p2p_items_bound;
        if ((rc = dev_alloc(&d.p2p_items, nb, t, st))) return rc;
        if ((rc = dev_alloc(&d.p2p_split, nb, t, st))) return rc;
        if ((rc = dev_alloc(&d.p2p_arrived, nb, t, st))) return rc;
        if ((rc = dev_alloc(&d.p2p_nitems, 4, t, st))) return rc;
        if ((rc = dev_alloc(&w, (size_t)4 * nl, nullptr, st))) return rc;
        if ((rc = dev_alloc(&w64, (size_t)2 * nl, nullptr, st))) return rc;
        FMM_CUDA_TRY(cudaMemsetAsync(d.p2p_arrived, 0, sizeof(int32_t) * nb, st));
        k_p2p_item_counts<<<nblk(nl, 256), 256, 0, st>>>(nl, t->h_pin ? 1 : 0, R, d.leaves, d.p2p_start, d.count, w,
                                                          w + nl, w64);
        size_t sb = 0, sb64 = 0;
        cub::DeviceScan::ExclusiveSum(nullptr, sb, w, w + 2 * nl, nl, st);
        cub::DeviceScan::ExclusiveSum(nullptr, sb64, w64, w64 + nl, nl, st);
        if ((rc = dev_alloc(&tmp, std::max(sb, sb64), nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, sb, w, w + 2 * nl, nl, st));
        FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, sb, w + nl, w + 3 * nl, nl, st));
        FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, sb64, w64, w64 + nl, nl, st));
        k_p2p_items<<<nblk(nl, 256), 256, 0, st>>>(nl, R, d.leaves, d.p2p_start, w, w + 2 * nl, w + 3 * nl, w64, w64 + nl,
                                                    d.p2p_items, d.p2p_split, d.p2p_nitems);
        count_launch(t, 5);
        if (t->h_pin) FMM_CUDA_TRY(cudaMemcpyAsync(t->h_pin, d.p2p_nitems, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        dev_free(tmp, st);
        dev_free(w, st);
        dev_free(w64, st);
    }
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// a2 in one pass: leaf level of every particle, one scan of the per-level
// counts, then every cell and its links (the level-by-level octree serves
// FMM_BUILD_FALLBACKS).  One host round trip, which also brings back the
// root cubes.
template <class TakeGeometry>
static int build_octree_onepass(fmm_tree* t, TakeGeometry&& take_geometry, cudaStream_t st) {
    int rc;
    TreeDev& d = t->d;
    const int64_t n = t->n;
    const int nsys = t->nsys, S = t->prm.leaf_size;
    stage_begin(t, FMM_STAGE_OCTREE, st);
    const int nb = (int)((n + OCT_B - 1) / OCT_B);
    const size_t ncnt = (size_t)2 * OCT_NL * nb;
    char2* lohi = nullptr;
    int64_t *cnt = nullptr, *offs = nullptr, *hdr = nullptr;
    char* tmp = nullptr;
    auto release = [&]() {
        dev_free(tmp, st);
        dev_free(lohi, st);
        dev_free(cnt, st);
        dev_free(offs, st);
        dev_free(hdr, st);
    };
    const size_t hdr_words = 32 + (sizeof(Geometry) * (size_t)nsys + 7) / 8;
    if ((rc = dev_alloc(&lohi, (size_t)n, nullptr, st))) return rc;
    if ((rc = dev_alloc(&cnt, ncnt, nullptr, st))) return rc;
    if ((rc = dev_alloc(&offs, ncnt, nullptr, st))) return rc;
    if ((rc = dev_alloc(&hdr, hdr_words, nullptr, st))) return rc;
    k_oct_levels<<<nb, OCT_B, 2 * (OCT_B + S), st>>>(d.keys, n, d.sys_off, nsys, S, nb, lohi, cnt);
    count_launch(t);
    size_t sb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, sb, cnt, offs, (int64_t)ncnt, st);
    if ((rc = dev_alloc(&tmp, sb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, sb, cnt, offs, (int64_t)ncnt, st));
    count_launch(t);
    k_oct_summary<<<1, 128, 0, st>>>(offs, cnt, nb, d.geom, nsys, hdr, (Geometry*)(hdr + 32));
    count_launch(t);
    std::vector<int64_t> h(hdr_words);
    FMM_CUDA_TRY(cudaMemcpyAsync(h.data(), hdr, hdr_words * 8, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    if ((rc = take_geometry((const Geometry*)(h.data() + 32)))) { release(); return rc; }
    const int64_t ncell = h[OCT_NL], nleaf = h[OCT_NL + 1];
    if (ncell >= INT32_MAX) {
        release();
        fmm_set_error("fmm_build_tree: %lld cells exceed the 32-bit cell index", (long long)ncell);
        return FMM_ERR_ARG;
    }
    t->ncell = (int)ncell;
    t->nleaf = (int)nleaf;
    LevelStarts ls;
    int deepest = 0;
    for (int L = 0; L <= OCT_NL; L++) t->level_start[L] = ls.s[L] = (int32_t)h[L];
    for (int L = 0; L < OCT_NL; L++)
        if (h[L + 1] > h[L]) deepest = L;
    t->nlevel = deepest + 1;
    const size_t nc = (size_t)ncell;
    if ((rc = dev_alloc(&d.level, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.ckey, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.first, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.count, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.parent, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.child_first, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.child_count, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.leaves, nc, t, st))) return rc;
    k_oct_emit<<<nb, OCT_B, 0, st>>>(d.keys, n, d.sys_off, nsys, nb, lohi, offs, d.level, d.ckey, d.first, d.count,
                                     d.leaves);
    count_launch(t);
    k_oct_links<<<nblk((int64_t)nc, 256), 256, 0, st>>>((int)nc, ls, S, d.level, d.first, d.count, d.parent,
                                                         d.child_first, d.child_count);
    count_launch(t);
    release();
    FMM_CUDA_TRY(cudaGetLastError());
    stage_end(t, FMM_STAGE_OCTREE, st);
    return FMM_OK;
}

int build_tree_impl(fmm_tree* t, const void* pos, int pos_dtype, cudaStream_t st) {
    int rc;
    const int64_t n = t->n;
    TreeDev& d = t->d;
    const int nsys = t->nsys;
    if ((rc = dev_alloc(&d.geom, (size_t)nsys, t, st))) return rc;
    FMM_CUDA_TRY(cudaMemsetAsync(d.geom, 0, sizeof(Geometry) * nsys, st));
    if ((rc = dev_alloc(&d.status, 4, t, st))) return rc;
    FMM_CUDA_TRY(cudaMemsetAsync(d.status, 0, 4 * sizeof(int), st));
    if (n == 0) {
        t->ncell = 0; t->nlevel = 0; t->nleaf = 0;
        return FMM_OK;
    }
    if ((rc = dev_alloc(&d.sys_off, (size_t)nsys + 1, t, st))) return rc;
    FMM_CUDA_TRY(cudaMemcpyAsync(d.sys_off, t->h_sys_off.data(), sizeof(int64_t) * (nsys + 1), cudaMemcpyHostToDevice, st));
    stage_begin(t, FMM_STAGE_KEYS, st);
    // --- a1: root cube of every system, keys.  Blocks of the bounding-box
    // reduction are dealt to the systems in proportion to their size.
    std::vector<int64_t> hblk;
    std::vector<int32_t> hsblk(nsys + 1, 0);
    {
        const int64_t chunk = std::max<int64_t>(BB_THREADS * 8, (n + 1023) / 1024);
        for (int s = 0; s < nsys; s++) {
            hsblk[s] = (int32_t)(hblk.size() / 2);
            for (int64_t a = t->h_sys_off[s]; a < t->h_sys_off[s + 1]; a += chunk) {
                hblk.push_back(a);
                hblk.push_back(std::min(t->h_sys_off[s + 1], a + chunk));
            }
        }
        hsblk[nsys] = (int32_t)(hblk.size() / 2);
    }
    const int nb = hsblk[nsys];
    double* part = nullptr;
    int64_t* dblk = nullptr;
    int32_t* dsblk = nullptr;
    if ((rc = dev_alloc(&part, (size_t)nb * 6, nullptr, st))) return rc;
    if ((rc = dev_alloc(&dblk, hblk.size(), nullptr, st))) return rc;
    if ((rc = dev_alloc(&dsblk, (size_t)nsys + 1, nullptr, st))) return rc;
    FMM_CUDA_TRY(cudaMemcpyAsync(dblk, hblk.data(), sizeof(int64_t) * hblk.size(), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(dsblk, hsblk.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, st));
    if (pos_dtype == FMM_F64)
        k_bbox_partial<double><<<nb, BB_THREADS, 0, st>>>((const double*)pos, dblk, part, d.geom);
    else
        k_bbox_partial<float><<<nb, BB_THREADS, 0, st>>>((const float*)pos, dblk, part, d.geom);
    k_bbox_final<<<nblk((int64_t)nsys * 32, 128), 128, 0, st>>>(part, dsblk, nsys, d.geom);
    count_launch(t, 2);
    uint64_t* keys_in = nullptr;
    int32_t* idx_in = nullptr;
    if ((rc = dev_alloc(&keys_in, n, nullptr, st))) return rc;
    if ((rc = dev_alloc(&idx_in, n, nullptr, st))) return rc;
    if ((rc = dev_alloc(&d.keys, n, t, st))) return rc;
    if ((rc = dev_alloc(&d.perm, n, t, st))) return rc;
    if (pos_dtype == FMM_F64)
        k_keys<double><<<nblk(n, 256), 256, 0, st>>>((const double*)pos, n, d.sys_off, nsys, d.geom, keys_in, idx_in);
    else
        k_keys<float><<<nblk(n, 256), 256, 0, st>>>((const float*)pos, n, d.sys_off, nsys, d.geom, keys_in, idx_in);
    count_launch(t);
    // --- a2: stable sort of (key, input index), within each system
    size_t tmp_bytes = 0;
    char* tmp = nullptr;
    if (nsys == 1) {
        cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys_in, d.keys, idx_in, d.perm, n, 0, 63, st);
        if ((rc = dev_alloc(&tmp, tmp_bytes, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, d.keys, idx_in, d.perm, n, 0, 63, st));
    } else {
        cub::DeviceSegmentedRadixSort::SortPairs(nullptr, tmp_bytes, keys_in, d.keys, idx_in, d.perm, n, nsys,
                                                 d.sys_off, d.sys_off + 1, 0, 63, st);
        if ((rc = dev_alloc(&tmp, tmp_bytes, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceSegmentedRadixSort::SortPairs(tmp, tmp_bytes, keys_in, d.keys, idx_in, d.perm, n,
                                                              nsys, d.sys_off, d.sys_off + 1, 0, 63, st));
    }
    count_launch(t);
    dev_free(tmp, st);
    dev_free(keys_in, st);
    dev_free(idx_in, st);
    dev_free(part, st);
    dev_free(dblk, st);
    dev_free(dsblk, st);
    if ((rc = dev_alloc(&d.spos, (size_t)n * 3, t, st))) return rc;
    if (pos_dtype == FMM_F64)
        k_gather_pos<double><<<nblk(n, 256), 256, 0, st>>>((const double*)pos, d.perm, n, d.spos);
    else
        k_gather_pos<float><<<nblk(n, 256), 256, 0, st>>>((const float*)pos, d.perm, n, d.spos);
    count_launch(t);
    stage_end(t, FMM_STAGE_KEYS, st);
    // root cubes on the host; a non-finite position fails the build
    auto take_geometry = [&](const Geometry* hg) -> int {
        t->h_geom.assign((size_t)nsys * 4, 0.0);
        for (int s = 0; s < nsys; s++) {
            if (hg[s].bad) {
                fmm_set_error("fmm_build_tree: positions contain a non-finite value");
                return FMM_ERR_ARG;
            }
            for (int k = 0; k < 3; k++) t->h_geom[4 * s + k] = hg[s].origin[k];
            t->h_geom[4 * s + 3] = hg[s].side;
        }
        for (int k = 0; k < 3; k++) t->origin[k] = hg[0].origin[k];
        t->side = hg[0].side;
        return FMM_OK;
    };
    if (!(t->prm.flags & FMM_BUILD_FALLBACKS)) {
        if ((rc = build_octree_onepass(t, take_geometry, st))) return rc;
        stage_begin(t, FMM_STAGE_SETUP, st);
    } else {
        std::vector<Geometry> hg(nsys);
        FMM_CUDA_TRY(cudaMemcpyAsync(hg.data(), d.geom, sizeof(Geometry) * nsys, cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
        if ((rc = take_geometry(hg.data()))) return rc;
        // --- a2: octree, level by level
        stage_begin(t, FMM_STAGE_OCTREE, st);
        size_t cap = (size_t)std::max<int64_t>(64, 4 * n / std::max(1, t->prm.leaf_size) + 64);
        size_t c_lev = 0, c_key = 0, c_first = 0, c_count = 0, c_par = 0, c_cf = 0, c_cc = 0;
        int32_t *lev = nullptr, *first = nullptr, *count = nullptr, *par = nullptr, *cf = nullptr, *cc = nullptr;
        uint64_t* ckey = nullptr;
        auto grow_all = [&](size_t need, size_t keep) -> int {
            int r;
            if ((r = grow(lev, c_lev, need, keep, st))) return r;
            if ((r = grow(ckey, c_key, need, keep, st))) return r;
            if ((r = grow(first, c_first, need, keep, st))) return r;
            if ((r = grow(count, c_count, need, keep, st))) return r;
            if ((r = grow(par, c_par, need, keep, st))) return r;
            if ((r = grow(cf, c_cf, need, keep, st))) return r;
            if ((r = grow(cc, c_cc, need, keep, st))) return r;
            return FMM_OK;
        };
        if ((rc = grow_all(std::max(cap, (size_t)nsys + 64), 0))) return rc;
        k_init_roots<<<nblk(nsys, 128), 128, 0, st>>>(nsys, d.sys_off, lev, ckey, first, count, par);
        count_launch(t);
        int32_t *nch = nullptr, *coff = nullptr, *ends = nullptr;
        size_t c_nch = 0, c_coff = 0, c_ends = 0;
        int lb = 0, le = nsys, level = 0;
        t->level_start[0] = 0;
        while (true) {
            int width = le - lb;
            if ((rc = grow(nch, c_nch, width, 0, st))) return rc;
            if ((rc = grow(coff, c_coff, width, 0, st))) return rc;
            if ((rc = grow(ends, c_ends, (size_t)width * 8, 0, st))) return rc;
            // a narrow level (few cells, long ranges) searches with a warp per boundary
            const int wide = (int64_t)width * 8 * 32 <= (int64_t)t->num_sms * 1024 ? 1 : 0;
            k_count_children<<<nblk((int64_t)width * 8 * (wide ? 32 : 1), 128), 128, 0, st>>>(
                lb, le, level, t->prm.leaf_size, wide, first, count, ckey, d.keys, ends, nch);
            count_launch(t);
            if (wide) {
                k_count_from_ends<<<nblk(width, 128), 128, 0, st>>>(lb, le, level, t->prm.leaf_size, first, count, ends,
                                                                   nch);
                count_launch(t);
            }
            size_t sb = 0;
            cub::DeviceScan::ExclusiveSum(nullptr, sb, nch, coff, width, st);
            if ((rc = dev_alloc(&tmp, sb, nullptr, st))) return rc;
            FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, sb, nch, coff, width, st));
            count_launch(t);
            dev_free(tmp, st);
            int32_t last_off = 0, last_n = 0;
            FMM_CUDA_TRY(cudaMemcpyAsync(&last_off, coff + width - 1, 4, cudaMemcpyDeviceToHost, st));
            FMM_CUDA_TRY(cudaMemcpyAsync(&last_n, nch + width - 1, 4, cudaMemcpyDeviceToHost, st));
            FMM_CUDA_TRY(cudaStreamSynchronize(st));
            int total = last_off + last_n;
            if ((size_t)le + total > c_lev) {
                if ((rc = grow_all((size_t)le + total, (size_t)le))) return rc;
            }
            k_emit_children<<<nblk((int64_t)width * 8, 128), 128, 0, st>>>(lb, le, level, ends, nch, coff, le, lev, ckey,
                                                                          first, count, par, cf, cc);
            count_launch(t);
            t->level_start[level + 1] = le;
            if (total == 0) break;
            lb = le;
            le += total;
            level++;
        }
        dev_free(nch, st);
        dev_free(coff, st);
        dev_free(ends, st);
        stage_end(t, FMM_STAGE_OCTREE, st);
        stage_begin(t, FMM_STAGE_SETUP, st);
        t->ncell = le;
        t->nlevel = level + 1;
        for (int l = t->nlevel + 1; l <= FMM_MAX_LEVEL + 1; l++) t->level_start[l] = le;
        // move the cell table into exactly sized, tree-owned arrays
        const size_t nc = (size_t)t->ncell;
        if ((rc = dev_alloc(&d.level, nc, t, st))) return rc;
        if ((rc = dev_alloc(&d.ckey, nc, t, st))) return rc;
        if ((rc = dev_alloc(&d.first, nc, t, st))) return rc;
        if ((rc = dev_alloc(&d.count, nc, t, st))) return rc;
        if ((rc = dev_alloc(&d.parent, nc, t, st))) return rc;
        if ((rc = dev_alloc(&d.child_first, nc, t, st))) return rc;
        if ((rc = dev_alloc(&d.child_count, nc, t, st))) return rc;
        FMM_CUDA_TRY(cudaMemcpyAsync(d.level, lev, nc * 4, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(d.ckey, ckey, nc * 8, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(d.first, first, nc * 4, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(d.count, count, nc * 4, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(d.parent, par, nc * 4, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(d.child_first, cf, nc * 4, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(d.child_count, cc, nc * 4, cudaMemcpyDeviceToDevice, st));
        dev_free(lev, st); dev_free(ckey, st); dev_free(first, st); dev_free(count, st);
        dev_free(par, st); dev_free(cf, st); dev_free(cc, st);
        // leaves
        {
            char* flag = nullptr;
            int32_t *nsel = nullptr, *it = nullptr;
            if ((rc = dev_alloc(&flag, nc, nullptr, st))) return rc;
            if ((rc = dev_alloc(&it, nc, nullptr, st))) return rc;
            if ((rc = dev_alloc(&nsel, 1, nullptr, st))) return rc;
            if ((rc = dev_alloc(&d.leaves, nc, t, st))) return rc;
            k_leaf_flags<<<nblk(nc, 256), 256, 0, st>>>((int)nc, d.child_count, flag, it);
            count_launch(t);
            size_t sb = 0;
            cub::DeviceSelect::Flagged(nullptr, sb, it, flag, d.leaves, nsel, (int)nc, st);
            if ((rc = dev_alloc(&tmp, sb, nullptr, st))) return rc;
            FMM_CUDA_TRY(cub::DeviceSelect::Flagged(tmp, sb, it, flag, d.leaves, nsel, (int)nc, st));
            count_launch(t);
            int32_t h = 0;
            FMM_CUDA_TRY(cudaMemcpyAsync(&h, nsel, 4, cudaMemcpyDeviceToHost, st));
            FMM_CUDA_TRY(cudaStreamSynchronize(st));
            t->nleaf = h;
            dev_free(tmp, st); dev_free(flag, st); dev_free(nsel, st); dev_free(it, st);
        }
    }
    const size_t nc = (size_t)t->ncell;
    if ((rc = dev_alloc(&d.centre, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.icentre, nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.cu2f, nc, t, st))) return rc;
    k_centres<<<nblk(nc, 128), 128, 0, st>>>((int)nc, d.level, d.ckey, d.first, d.sys_off, nsys, d.geom, d.centre,
                                              d.icentre, d.cu2f);
    count_launch(t);
    if ((rc = dev_alloc(&d.pleaf, (size_t)n, t, st))) return rc;
    k_particle_leaf<<<nblk((int64_t)t->nleaf * 32, 256), 256, 0, st>>>(t->nleaf, d.leaves, d.first, d.count,
                                                                     d.pleaf);
    count_launch(t);

    stage_end(t, FMM_STAGE_SETUP, st);
    // --- a3: breadth-first dual traversal from (root, root)
    stage_begin(t, FMM_STAGE_LISTS, st);
    stage_begin(t, FMM_STAGE_TRAVERSAL, st);
    int2 *m2l = nullptr, *p2p = nullptr;
    int64_t nm = 0, npp = 0;
    if (t->prm.flags & FMM_LISTS_UVWX) {
        // the parent-neighbour-child lists instead of the size/distance test
        if ((rc = uvwx_lists(t, &m2l, &nm, &p2p, &npp, st))) return rc;
    } else {
        size_t c_front = 1024, c_next = 1024, c_m = 1024, c_p = 1024;
        int2 *front = nullptr, *next = nullptr;
        if ((rc = grow(front, c_front = 0, std::max<size_t>(1024, nsys), 0, st))) return rc;
        if ((rc = grow(next, c_next = 0, 1024, 0, st))) return rc;
        if ((rc = grow(m2l, c_m = 0, 1024, 0, st))) return rc;
        if ((rc = grow(p2p, c_p = 0, 1024, 0, st))) return rc;
        TravCounters* ctr = nullptr;
        if ((rc = dev_alloc(&ctr, 1, nullptr, st))) return rc;
        FMM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(TravCounters), st));
        k_init_frontier<<<nblk(nsys, 128), 128, 0, st>>>(nsys, front);
        count_launch(t);
        int64_t nf = nsys;
        const double th2 = t->prm.theta * t->prm.theta;
        {
            // one cooperative launch for every round, with buffers sized from the
            // cell count; the round-by-round loop below runs only on overflow
            const size_t nc0 = (size_t)t->ncell;
            const size_t cf = std::max<size_t>(1 << 20, 96 * nc0), cm = std::max<size_t>(1 << 22, 640 * nc0),
                         cp = std::max<size_t>(1 << 20, 160 * nc0);
            int2 *fa = nullptr, *fb = nullptr, *mm = nullptr, *pp = nullptr, *chpk = nullptr;
            TravState* stt = nullptr;
            bool ok = dev_alloc(&fa, cf, nullptr, st) == FMM_OK && dev_alloc(&fb, cf, nullptr, st) == FMM_OK &&
                      dev_alloc(&mm, cm, nullptr, st) == FMM_OK && dev_alloc(&pp, cp, nullptr, st) == FMM_OK &&
                      dev_alloc(&chpk, (size_t)t->ncell, nullptr, st) == FMM_OK &&
                      dev_alloc((char**)&stt, sizeof(TravState), nullptr, st) == FMM_OK;
            int per_sm = 0;
            if (t->prm.flags & FMM_BUILD_FALLBACKS) ok = false;
            if (ok) ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse_coop, TRAV_THREADS, 0) ==
                             cudaSuccess &&
                         per_sm > 0;
            if (ok) {
                TravState h0 = {{(unsigned long long)nsys, 0ull, 0ull}, 0ull, 0ull, {0, 0}, 0};
                FMM_CUDA_TRY(cudaMemcpyAsync(stt, &h0, sizeof(h0), cudaMemcpyHostToDevice, st));
                k_init_frontier<<<nblk(nsys, 128), 128, 0, st>>>(nsys, fa);
                k_child_pack<<<nblk(t->ncell, 256), 256, 0, st>>>(t->ncell, d.child_first, d.child_count, chpk);
                unsigned long long a_cm = cm, a_cp = cp, a_cf = cf;
                const int4* a_ic = d.icentre;
                const int2* a_ch = chpk;
                double a_th2 = th2;
                void* args[] = {&fa, &fb, &a_ic, &a_ch, &a_th2, &mm, &pp, &stt, &a_cm, &a_cp, &a_cf};
                dim3 grid(per_sm * t->num_sms), block(TRAV_THREADS);
                FMM_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_traverse_coop, grid, block, args, 0, st));
                count_launch(t, 3);
                TravState h;
                FMM_CUDA_TRY(cudaMemcpyAsync(&h, stt, sizeof(h), cudaMemcpyDeviceToHost, st));
                FMM_CUDA_TRY(cudaStreamSynchronize(st));
                if (!h.ovf[0] && !h.ovf[1]) {
                    dev_free(m2l, st); dev_free(p2p, st);
                    m2l = mm; p2p = pp; c_m = cm; c_p = cp;
                    mm = pp = nullptr;
                    nm = (int64_t)h.nm2l;
                    npp = (int64_t)h.np2p;
                    nf = 0;   // done
                }
            }
            dev_free(fa, st); dev_free(fb, st); dev_free(mm, st); dev_free(pp, st); dev_free(chpk, st);
            if (stt) cudaFreeAsync(stt, st);
        }
        while (nf > 0) {
            if ((rc = grow(next, c_next, (size_t)nf * 8, 0, st))) return rc;
            if ((rc = grow(m2l, c_m, (size_t)(nm + nf), (size_t)nm, st))) return rc;
            if ((rc = grow(p2p, c_p, (size_t)(npp + nf), (size_t)npp, st))) return rc;
            FMM_CUDA_TRY(cudaMemsetAsync(&ctr->nnext, 0, 8, st));
            k_traverse<<<nblk(nf, 256), 256, 0, st>>>(front, nf, d.level, d.ckey, d.child_first, d.child_count, th2,
                                                        m2l, p2p, next, ctr);
            count_launch(t);
            TravCounters h;
            FMM_CUDA_TRY(cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
            FMM_CUDA_TRY(cudaStreamSynchronize(st));
            nm = (int64_t)h.nm2l;
            npp = (int64_t)h.np2p;
            nf = (int64_t)h.nnext;
            std::swap(front, next);
            std::swap(c_front, c_next);
        }
        dev_free(front, st); dev_free(next, st); dev_free(ctr, st);
    }
    stage_end(t, FMM_STAGE_TRAVERSAL, st);
    t->nm2l = nm;
    t->np2p = npp;
    // The P2P list and its records go on the second stream of the evaluation's
    // far field (idle during the build), so they fill the GPU while the host
    // waits on the M2L/class grouping below; joined before the task queue.
    cudaStream_t sl = (t->hi_stream && t->ev_join_hi) ? t->hi_stream : st;
    if (sl != st) {
        FMM_CUDA_TRY(cudaEventRecord(t->ev_fork, st));
        FMM_CUDA_TRY(cudaStreamWaitEvent(sl, t->ev_fork, 0));
    }
    stage_begin(t, FMM_STAGE_P2P_LIST, sl);
    if ((rc = finish_p2p_list(t, p2p, npp, sl))) return rc;
    dev_free(p2p, sl);
    stage_end(t, FMM_STAGE_P2P_LIST, sl);
    if (sl != st) FMM_CUDA_TRY(cudaEventRecord(t->ev_join_hi, sl));
    const bool want_classes = t->prm.precision == FMM_PREC_MIXED_TC && tc_supported(t->prm.p);
    // with the tensor cores the M2L pairs are grouped by class straight from the
    // traversal output; no (target, source) order is needed on that path
    stage_begin(t, FMM_STAGE_CLASSES, st);
    if (want_classes) {
        if ((rc = build_m2l_classes(t, m2l, st))) return rc;
    } else if ((rc = finish_list(t, m2l, nm, &d.m2l_start, &d.m2l_src, nullptr, st))) {
        return rc;
    }
    dev_free(m2l, st);
    stage_end(t, FMM_STAGE_CLASSES, st);
    if (sl != st) FMM_CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join_hi, 0));
    if (queue_supported(t) && (rc = build_queue(t, st))) return rc;
    if (tc_uses_dag(t) && (rc = build_dag(t, st))) return rc;
    stage_end(t, FMM_STAGE_LISTS, st);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int set_positions_impl(fmm_tree* t, const void* pos, int pos_dtype, cudaStream_t st) {
    if (t->n == 0) return FMM_OK;
    if (pos_dtype == FMM_F64)
        k_gather_pos<double><<<nblk(t->n, 256), 256, 0, st>>>((const double*)pos, t->d.perm, t->n, t->d.spos);
    else
        k_gather_pos<float><<<nblk(t->n, 256), 256, 0, st>>>((const float*)pos, t->d.perm, t->n, t->d.spos);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

template <typename T>
__global__ void k_grad_combine(int64_t n, const T* __restrict__ q, const T* __restrict__ w, const T* __restrict__ eq,
                               const T* __restrict__ ew, T* __restrict__ dx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int d = 0; d < 3; d++) dx[3 * i + d] = -(w[i] * eq[3 * i + d] + q[i] * ew[3 * i + d]);
}

int grad_combine(fmm_tree* t, const void* q, const void* w, const void* eq, const void* ew, void* dx, int dtype,
                 cudaStream_t st) {
    if (t->n == 0 || !dx) return FMM_OK;
    if (dtype == FMM_F64)
        k_grad_combine<double><<<nblk(t->n, 256), 256, 0, st>>>(t->n, (const double*)q, (const double*)w,
                                                                 (const double*)eq, (const double*)ew, (double*)dx);
    else
        k_grad_combine<float><<<nblk(t->n, 256), 256, 0, st>>>(t->n, (const float*)q, (const float*)w,
                                                                (const float*)eq, (const float*)ew, (float*)dx);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

void free_tree_device(fmm_tree* t) {
    TreeDev& d = t->d;
    cudaStream_t st = 0;
    dev_free(d.keys, st); dev_free(d.perm, st); dev_free(d.spos, st);
    dev_free(d.level, st); dev_free(d.ckey, st); dev_free(d.first, st); dev_free(d.count, st);
    dev_free(d.parent, st); dev_free(d.child_first, st); dev_free(d.child_count, st);
    dev_free(d.centre, st); dev_free(d.icentre, st); dev_free(d.sys_off, st); dev_free(d.cu2f, st); dev_free(d.leaves, st); dev_free(d.pleaf, st);
    dev_free(d.m2l_start, st); dev_free(d.m2l_src, st); dev_free(d.p2p_start, st); dev_free(d.p2p_src, st);
    dev_free(d.geom, st); dev_free(d.status, st);
    if (d.grad_tmp) cudaFreeAsync(d.grad_tmp, st);
    d.grad_tmp = nullptr;
    dev_free(d.m2l_tgt, st); dev_free(d.p2p_rec, st); dev_free(d.p2p_items, st); dev_free(d.p2p_nitems, st);
    dev_free(d.p2p_mode, st); dev_free(d.p2p_split, st); dev_free(d.p2p_arrived, st); dev_free(d.p2p_part, st); dev_free(d.rem_count, st); dev_free(d.tc_items, st); dev_free(d.tc_block_first, st); dev_free(d.tc_item_list, st); dev_free(d.tc_tgt, st); dev_free(d.tc_src, st);
    dev_free(d.rem_start, st); dev_free(d.rem_chunks, st);
    dev_free(d.dag_cnt_init, st); dev_free(d.dag_cnt, st); dev_free(d.dag_q_init, st); dev_free(d.dag_q, st);
    dev_free(d.dag_lvl, st); dev_free(d.dag_ctr, st); dev_free(d.dag_zero_first, st);
    dev_free(d.tr_start, st); dev_free(d.tr_tgt, st); dev_free(d.q_cnt_init, st); dev_free(d.q_cnt, st);
    dev_free(d.q_init, st); dev_free(d.q_work, st); dev_free(d.q_ctr, st);
    dev_free(d.tc_keys, st);
    if (d.tc_harm) cudaFreeAsync(d.tc_harm, st);
    if (d.tc_msplit) cudaFreeAsync(d.tc_msplit, st);
    if (d.tc_lr) cudaFreeAsync(d.tc_lr, st);
    d.tc_harm = nullptr; d.tc_msplit = nullptr; d.tc_lr = nullptr;
    t->tc_tmap_ok = false;
    dev_free(d.M, st); dev_free(d.L, st); dev_free(d.xq, st); dev_free(d.near, st);
    if (d.shift_ops) cudaFreeAsync(d.shift_ops, st);
    d.shift_ops = nullptr;
}

}  // namespace fmm
