// fmm_internal.cuh -- types and helpers shared by the CUDA translation units.
//
// Coefficient storage on the device: orders m >= 0 only ("triangular"),
// complex entry (n, m) at n(n+1)/2 + m; negative orders follow from
// X_n^{-m} = (-1)^m conj(X_n^m), which holds for the solid harmonics and for
// every expansion of a real charge distribution.
//
// Expansions are stored per-level scaled (h = side of the cell):
//   multipole  Mt_n^m = M_n^m / h^n       = sum_j q_j R_n^m((x_j - c) / h)
//   local      Lt_k^l = L_k^l * h^(k+1),   phi(x) = (1/h) sum Lt_k^l R_k^l((x - c) / h)
// so that a translation between cells of sizes (h_s, h_t) depends only on the
// offset in target-cell units and on the size ratio.  Every value then stays
// inside FP32 range for any tree depth.
#pragma once
#include <cuda.h>            // CUtensorMap (a type only: no driver-API symbol is linked)
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fmm.h"

#define FMM_MAX_P 20
#define M2L_CHUNK 16   // list entries per warp in the chunked CUDA-core M2L
#define FMM_MAX_LEVEL 21

namespace fmm {

__host__ __device__ inline int tri(int n, int m) { return n * (n + 1) / 2 + m; }
__host__ __device__ inline int ntri(int p) { return (p + 1) * (p + 2) / 2; }
// row stride of expansion arrays (complex entries): rows start on 32-byte (FP32)
// or 64-byte (FP64) boundaries, so FP32 rows can take 16-byte vector atomics
__host__ __device__ inline int kstride(int p) { return (ntri(p) + 3) & ~3; }

// Real basis of an expansion truncated at degree p (tensor-core M2L): index c
// runs over, for n = 0..p, (n, 0) re, then (n, m) re, (n, m) im for m = 1..n,
// so there are (p+1)^2 of them (the imaginary parts of the m = 0 terms vanish
// for real charges and are left out).  Decoded as n | m << 8 | im << 16.
__host__ __device__ inline int real_index_decode(int c) {
    int n = 0;
    while ((n + 1) * (n + 1) <= c) n++;
    const int r = c - n * n;
    if (r == 0) return n;
    const int m = (r + 1) >> 1;
    return n | (m << 8) | ((r & 1) ? 0 : (1 << 16));
}

template <typename T>
struct cplx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cplx<T> cmk(T a, T b) { cplx<T> c; c.re = a; c.im = b; return c; }
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return cmk<T>(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return cmk<T>(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return cmk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return cmk<T>(a.re * s, a.im * s); }
template <typename T>
__device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return cmk<T>(a.re, -a.im); }
// a += b * c
template <typename T>
__device__ __forceinline__ void cfma(cplx<T>& a, cplx<T> b, cplx<T> c) {
    a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
    a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
// a += b * conj(c)
template <typename T>
__device__ __forceinline__ void cfma_cj(cplx<T>& a, cplx<T> b, cplx<T> c) {
    a.re = fma(b.re, c.re, fma(b.im, c.im, a.re));
    a.im = fma(b.im, c.re, fma(-b.re, c.im, a.im));
}

// Entry (n, m) of a triangular array for any order -n <= m <= n (zero outside).
template <typename T>
__device__ __forceinline__ cplx<T> get_sym(const cplx<T>* A, int n, int m) {
    if (m > n || -m > n) return cmk<T>(0, 0);
    if (m >= 0) return A[tri(n, m)];
    cplx<T> v = A[tri(n, -m)];
    return (m & 1) ? cmk<T>(-v.re, v.im) : cmk<T>(v.re, -v.im);
}

// Regular solid harmonics R_n^m(x, y, z), 0 <= m <= n <= p, into R (triangular).
//   R_0^0 = 1, R_m^m = R_{m-1}^{m-1} (x + iy) / (2m), R_{m+1}^m = z R_m^m,
//   (n+m)(n-m) R_n^m = (2n-1) z R_{n-1}^m - r^2 R_{n-2}^m.
template <typename T>
__device__ inline void regular_harmonics(int p, T x, T y, T z, cplx<T>* R) {
    T r2 = x * x + y * y + z * z;
    cplx<T> rmm = cmk<T>(1, 0);
    for (int m = 0; m <= p; m++) {
        if (m > 0) rmm = cscale(cmul(rmm, cmk<T>(x, y)), T(1) / T(2 * m));
        R[tri(m, m)] = rmm;
        if (m + 1 <= p) R[tri(m + 1, m)] = cscale(rmm, z);
        cplx<T> a = rmm, b = cscale(rmm, z);
        for (int n = m + 2; n <= p; n++) {
            T inv = T(1) / T((n + m) * (n - m));
            cplx<T> c = cmk<T>((T(2 * n - 1) * z * b.re - r2 * a.re) * inv,
                               (T(2 * n - 1) * z * b.im - r2 * a.im) * inv);
            R[tri(n, m)] = c;
            a = b; b = c;
        }
    }
}

// Irregular solid harmonics column m: I_n^m(x, y, z) for n = m..P, into I (triangular).
//   I_m^m = (2m-1)!! (x + iy)^m / r^{2m+1},  I_{m+1}^m = (2m+1) z I_m^m / r^2,
//   r^2 I_n^m = (2n-1) z I_{n-1}^m - (n+m-1)(n-m-1) I_{n-2}^m.
template <typename T>
__device__ inline void irregular_column(int P, int m, T x, T y, T z, cplx<T>* I) {
    T r2 = x * x + y * y + z * z;
    T inv = T(1) / r2;
    cplx<T> v = cmk<T>(T(1) / sqrt(r2), 0);
    cplx<T> w = cscale(cmk<T>(x, y), inv);
    for (int j = 1; j <= m; j++) v = cscale(cmul(v, w), T(2 * j - 1));
    I[tri(m, m)] = v;
    if (m + 1 > P) return;
    cplx<T> a = v, b = cscale(v, T(2 * m + 1) * z * inv);
    I[tri(m + 1, m)] = b;
    for (int n = m + 2; n <= P; n++) {
        T c1 = T(2 * n - 1) * z, c2 = T((n + m - 1) * (n - m - 1));
        cplx<T> c = cmk<T>((c1 * b.re - c2 * a.re) * inv, (c1 * b.im - c2 * a.im) * inv);
        I[tri(n, m)] = c;
        a = b; b = c;
    }
}

// ---------------------------------------------------------------------------
// Tree state
// ---------------------------------------------------------------------------

struct Geometry {        // device-resident root cube
    double origin[3];
    double side;
    double inv;          // 2^21 / side
    double centre[3];    // centre of the root cube (FP32 positions are relative to it)
    int bad;             // non-finite input seen
};

struct TreeDev {
    // particles (sorted order)
    uint64_t* keys = nullptr;     // [n]
    int32_t* perm = nullptr;      // [n] sorted slot -> input index
    double* spos = nullptr;       // [n*3] sorted positions (FP64)
    // cells, ordered by (level, key)
    int32_t* level = nullptr;
    uint64_t* ckey = nullptr;
    int32_t* first = nullptr;
    int32_t* count = nullptr;
    int32_t* parent = nullptr;
    int32_t* child_first = nullptr;
    int32_t* child_count = nullptr;
    double4_32a* centre = nullptr;    // (cx, cy, cz, h) in input coordinates
    int4* icentre = nullptr;      // twice the centre in units side/2^21 (exact integers), level
    int32_t* leaves = nullptr;    // [nleaf]
    int32_t* pleaf = nullptr;     // [n] leaf of each sorted particle
    // lists, CSR by target
    int64_t* m2l_start = nullptr; // [ncell+1]
    int32_t* m2l_src = nullptr;   // [nm2l]
    int64_t* p2p_start = nullptr;
    int32_t* p2p_src = nullptr;
    int32_t* m2l_tgt = nullptr;   // [nm2l] target of each list entry (class build only)
    int4* p2p_rec = nullptr;      // [np2p] (first, count, particle offset within the target's sources, source)
    // stage-by-stage P2P work items (target cell, first record - p2p_start[cell],
    // records, flags: 1 = the leaf is split over several items, 2 = the item adds
    // the leaf's own particles); leaves split into runs of prm.p2p_item_records
    // records come first.  p2p_nitems: [items, split items, partial slots (low,
    // high word)].
    // Split items: p2p_split (items of the leaf, rank, first partial slot of the
    // leaf as two words), p2p_arrived (per leaf, at its first item: blocks done,
    // back to 0 after the combine), p2p_part (4 doubles per slot: item x target)
    int4* p2p_items = nullptr;
    int32_t* p2p_nitems = nullptr;
    int8_t* p2p_mode = nullptr;     // [np2p] FMM_MUTUAL: 0 skip, 1 this direction only, 2 both leaves
    int32_t* rem_count = nullptr;   // chunks of the CUDA-core M2L (device word, copied to h_pin[4])
    int4* p2p_split = nullptr;
    int32_t* p2p_arrived = nullptr;
    double* p2p_part = nullptr;
    // tensor-core M2L (FMM_PREC_MIXED_TC): pairs grouped by translation class
    int4* tc_items = nullptr;     // [tc_nitems] (class, first pair, rows, -)
    int32_t* tc_block_first = nullptr;  // [tc_nblocks + 1] range of each tensor-core block in tc_item_list
    int32_t* tc_item_list = nullptr;    // [tc_nitems] work items, grouped by tensor-core block
    void* tc_harm = nullptr;      // [nclass][ntri(2p)] cplx<float>: irregular harmonics of each class offset
    uint64_t* tc_keys = nullptr;  // [nclass] class keys, in class order
    int32_t* tc_tgt = nullptr;    // [nm2l] targets in class order (class-less pairs last)
    int32_t* tc_src = nullptr;
    int64_t* rem_start = nullptr; // CSR of the class-less pairs by target
    int2* rem_chunks = nullptr;   // (target, first entry) chunks of at most M2L_CHUNK class-less pairs
    void* tc_msplit = nullptr;    // [ncell][hi | lo][KI] bf16 multipoles in the real basis (tc_kin)
    void* tc_lr = nullptr;        // [ncell][128] FP32 tensor-core M2L results in the real basis
    Geometry* geom = nullptr;     // [nsys] root cube of each system
    int64_t* sys_off = nullptr;   // [nsys+1] particle offsets of the systems
    float* cu2f = nullptr;        // [ncell] side/2^22 of the cell's system (FP32 P2P offsets)
    int* status = nullptr;        // device status word(s)
    // evaluation workspace
    void* M = nullptr;            // [ncell * ntri(p)] cplx<T>
    void* L = nullptr;
    void* xq = nullptr;           // sorted (x, y, z, q): double4_32a or float4
    double* near = nullptr;       // [n*4] sorted near-field (phi, gx, gy, gz)
    void* shift_ops = nullptr;    // [2][8][K2][K2] dense M2M / L2L operators per octant
    // persistent task queue (queue.cu)
    int64_t* tr_start = nullptr;  // transposed M2L list: source -> targets (CSR)
    int32_t* tr_tgt = nullptr;
    int32_t* q_cnt_init = nullptr;  // [4][ncell] initial dependency counters
    int32_t* q_cnt = nullptr;
    int32_t* q_init = nullptr;    // initial high-priority queue
    int32_t* q_work = nullptr;
    char* q_ctr = nullptr;        // queue heads / tails / done
    void* grad_tmp = nullptr;     // [n*3] field of the adjoint pass (fmm_backward)
    // task-graph evaluation of the mixed form (dag.cu)
    int32_t* dag_cnt_init = nullptr;  // [2][ncell] initial counters: children not final, L2P prerequisites
    int32_t* dag_cnt = nullptr;       // working copy
    int32_t* dag_q_init = nullptr;    // initial high-priority queue (the P2M tasks, then empty slots)
    int32_t* dag_q = nullptr;
    int32_t* dag_lvl = nullptr;       // [2][FMM_MAX_LEVEL + 1]: cells per level, final cells per level
    char* dag_ctr = nullptr;          // queue counters
    int32_t* dag_zero_first = nullptr;  // an empty item list per block (trees without tensor-core items)
};

}  // namespace fmm

struct fmm_tree {
    fmm_params prm;
    // stage timing (FMM_TIMING) and launch counts
    cudaEvent_t ev[2 * FMM_NUM_STAGES] = {};
    bool ev_used[FMM_NUM_STAGES] = {};
    bool timing = false;
    int64_t launches_build = 0, launches_eval = 0;
    // second stream of the stage-by-stage evaluation (P2P beside the far field)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // recorded on side_stream after the tensor-core class operators are built
    // (they are computed there, overlapping the rest of the build)
    cudaEvent_t ev_ops = nullptr;
    // the far-field chain of the stage-by-stage path (P2M, M2M, M2L, L2L) runs on
    // a high-priority stream, so that its short, latency-bound kernels get SMs
    // as soon as P2P blocks retire instead of queueing behind the whole P2P grid
    cudaStream_t hi_stream = nullptr;
    cudaEvent_t ev_join_hi = nullptr;
    // the tensor-core class operators are built on a stream of their own (they
    // overlap the rest of the build and the start of the evaluation)
    cudaStream_t ops_stream = nullptr;
    // fork and join of the CUDA-core M2L pairs on ops_stream during evaluation
    cudaEvent_t ev_rem_fork = nullptr, ev_rem_join = nullptr;
    int64_t* launch_ctr = nullptr;  // which counter launches currently go to
    int64_t n = 0;
    int ncell = 0, nlevel = 0, nleaf = 0;
    int64_t nm2l = 0, np2p = 0;
    // P2P work items: host bound of their number (the grid when the exact count
    // is not on the host), and pinned host words [items, split items] copied
    // from p2p_nitems during the build (valid once the build has synchronised);
    // without them no leaf is split
    int64_t p2p_items_bound = 0;
    int32_t* h_pin = nullptr;
    int level_start[FMM_MAX_LEVEL + 2] = {0};  // cells of level l: [level_start[l], level_start[l+1])
    double origin[3] = {0, 0, 0}, side = 1.0;
    int64_t device_bytes = 0;
    int nsys = 1;
    std::vector<int64_t> h_sys_off;   // host copy of the system offsets
    std::vector<double> h_geom;       // per system: origin x, y, z, side
    int num_sms = 148;
    int64_t tc_nclass = 0, tc_nitems = 0, tc_npairs = 0, tc_nrem = 0;
    int tc_nblocks = 0;
    int64_t dag_n_hi = 0, dag_n_tasks = 0, dag_nrem_tasks = 0, dag_m2l_total = 0;
    int64_t rem_nchunk = 0;
    // TMA map of d.tc_msplit (row gathers of the tensor-core M2L), encoded once
    // the table is allocated
    CUtensorMap tc_tmap;   // (the type is 64-byte aligned)
    bool tc_tmap_ok = false;
    int64_t q_n_hi = 0, q_n0 = 0, q_n_tasks = 0;
    fmm::TreeDev d;
};

// error reporting (capi.cu)
void fmm_set_error(const char* fmt, ...);

#define FMM_CUDA_TRY(call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            fmm_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? FMM_ERR_ALLOC : FMM_ERR_CUDA;       \
        }                                                                               \
    } while (0)

// internal entry points between translation units
namespace fmm {
// stage events: recorded only when the tree was built with FMM_TIMING
inline void stage_begin(fmm_tree* t, int s, cudaStream_t st) {
    if (t->timing) { cudaEventRecord(t->ev[2 * s], st); t->ev_used[s] = true; }
}
inline void stage_end(fmm_tree* t, int s, cudaStream_t st) {
    if (t->timing) cudaEventRecord(t->ev[2 * s + 1], st);
}
inline void count_launch(fmm_tree* t, int k = 1) {
    if (t && t->launch_ctr) *t->launch_ctr += k;
}
int build_tree_impl(fmm_tree* t, const void* pos, int pos_dtype, cudaStream_t st);
// a slot of PIN_WORDS pinned host words for one tree (nullptr when none is free)
constexpr int PIN_WORDS = 8;   // [0..3] P2P work items, [4] CUDA-core M2L chunks
int32_t* pinned_slot_acquire();
void pinned_slot_release(int32_t* p);
// defaults of the work-shape tunables (fmm_params): records per P2P work item
// of a split leaf (256: on a Plummer core, leaves of 64..256 records gain
// nothing from a split and lose the partial sums' combine; a clustered tree's
// leaves beside dense clusters hold thousands); the largest class left to the
// CUDA-core M2L (the
// tensor-core kernel assembles one operator per class, which does not pay for
// a handful of pairs: on a clustered 4M-particle tree 97 % of the classes hold
// under 1 % of the pairs)
constexpr int P2P_ITEM_RECORDS = 256;
constexpr int TC_MIN_PAIRS = 64;
int evaluate_impl(fmm_tree* t, const void* q, void* phi, void* force, int dtype, cudaStream_t st);
int alloc_eval_workspace(fmm_tree* t, cudaStream_t st);
int set_positions_impl(fmm_tree* t, const void* pos, int pos_dtype, cudaStream_t st);
int grad_combine(fmm_tree* t, const void* q, const void* w, const void* eq, const void* ew, void* dx, int dtype,
                 cudaStream_t st);
int build_m2l_classes(fmm_tree* t, const int2* pairs, cudaStream_t st);
// before_fold: an event the fold into L waits for (other M2L work adding into L)
int m2l_tensor_cores(fmm_tree* t, const float* M, float* L, cudaStream_t st, cudaEvent_t before_fold = nullptr);
int tc_kin(int p);
bool queue_supported(const fmm_tree* t);
int build_queue(fmm_tree* t, cudaStream_t st);
template <typename T, typename TP, typename O>
int evaluate_queue(fmm_tree* t, const double4_32a* xq64, const void* xqp, O* phi, O* force, cudaStream_t st,
                   const float4* xlo = nullptr);
bool tc_supported(int p);
// FMM_MUTUAL with an FP32 near field: cross-leaf pairs evaluated once for both
// leaves (p2p_mutual.cu); the evaluation then runs stage by stage
inline bool p2p_mutual(const fmm_tree* t) {
    return (t->prm.flags & FMM_MUTUAL) && t->prm.precision != FMM_PREC_FP64;
}
int build_p2p_modes(fmm_tree* t, const int32_t* tgt, cudaStream_t st);
// FMM_LISTS_UVWX: the M2L and P2P pairs from the parent-neighbour-child lists (uvwx.cu)
int uvwx_lists(fmm_tree* t, int2** m2l, int64_t* nm, int2** p2p, int64_t* np, cudaStream_t st);   // tgt: target of every record
int p2p_mutual_launch(fmm_tree* t, const float4* xq32, float4* acc, cudaStream_t st);
// the mixed form runs as one task-graph launch unless a stage-by-stage flag is set
inline bool tc_uses_dag(const fmm_tree* t) {
    return t->prm.precision == FMM_PREC_MIXED_TC && tc_supported(t->prm.p) && (t->prm.flags & FMM_TASK_GRAPH) &&
           !(t->prm.flags & (FMM_STAGED | FMM_NO_OVERLAP)) && !p2p_mutual(t);
}
int build_dag(fmm_tree* t, cudaStream_t st);
int tc_epilogue_warps();   // epilogue warps per tensor-core block: each counts an item once
struct DagArgs;
template <typename O>
int launch_m2l_dag(fmm_tree* t, const DagArgs& g, cudaStream_t st);
template <typename O>
int evaluate_dag(fmm_tree* t, const double4_32a* xq64, const float4* xq32, const float4* xlo32, O* phi, O* force,
                 cudaStream_t st);
void free_tree_device(fmm_tree* t);
template <typename T>
int dev_alloc(T** p, size_t count, fmm_tree* t, cudaStream_t st);
}  // namespace fmm
