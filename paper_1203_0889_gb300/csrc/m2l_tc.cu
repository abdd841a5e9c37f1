// m2l_tc.cu -- M2L on the tensor cores (tcgen05), grouped by translation class.
//
// Every M2L pair (t, s) whose cells are at most ten levels apart belongs to a
// translation class (dl = level_t - level_s, V = (2c_t - 2c_s) / min(side_t, side_s)),
// an integer vector.  With per-level scaled expansions the translation is one
// real matrix per class:
//   Lt(t) += T_c Mt(s),   T_c[(k,l), (n,m)] from (-1)^k rho^n conj(I_{n+k}^{m+l}(D/h_t)),
//   D/h_t = V / 2^(1 + max(0, -dl)),  rho = h_s / h_t = 2^dl,
// so all pairs of a class form one dense product.  This is the paper's M2L
// (Section 2.1) regrouped: classes replace the per-pair operator, and the
// tensor cores run the products.
//
// The product is taken transposed, C^T = T_c A^T (M = output coefficients,
// N = 128 pairs, K = input coefficients), in the real basis of (p+1)^2
// coefficients: the class operator is the MMA's A operand and lives in tensor
// memory, assembled there by the kernel from the class's irregular harmonics
// (no operator table in HBM); the pairs' source multipoles are the B operand,
// gathered row by row from HBM into shared memory by TMA (tile::gather4).
//
// Precision: operator and multipoles are split into bf16 hi + lo parts and the
// product is accumulated in FP32 in tensor memory as A_hi T_hi + A_hi T_lo +
// A_lo T_hi (about 16 significant bits per product).  Each result column (one
// pair) is added into the target's local expansion with coalesced FP32
// reductions; pairs of rarer classes (level gap above ten) go through the
// CUDA-core kernel first, which also initialises every local expansion.
#include <cub/cub.cuh>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "dag.cuh"
#include "fmm_internal.cuh"
#include "tc_sm100.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int TC_MAX_DL = 10;
constexpr int TC_ROWS = 128;                 // pairs per work item: the N of the transposed product
// Class keys use 53 bits: (level gap + 16) in bits 48..52, each offset component
// + 32768 in 16 bits.  A pair outside every class gets NOT_TC | target, so such
// pairs sort after all classes and by target.
constexpr uint64_t NOT_TC = 1ull << 53;
constexpr int CLASS_KEY_BITS = 54;

// Real coefficients of an expansion truncated at degree p, and the width of a
// gathered row: K = (p+1)^2 rounded up to whole 64-element swizzle atoms.
static inline int tc_kreal(int p) { return (p + 1) * (p + 1); }
int tc_kin(int p) { return (tc_kreal(p) + 63) & ~63; }
// the operator (K <= 128 rows) must fit the 128 lanes of tensor memory
bool tc_supported(int p) { return tc_kreal(p) <= 128; }

// ---------------------------------------------------------------------------
// build: class keys, grouping, operators, work items
// ---------------------------------------------------------------------------

// class key of an M2L pair (target, source); NOT_TC | target when the pair
// has no class
__device__ __forceinline__ uint64_t pair_class_key(const int2 pr, const int4* __restrict__ icentre) {
    const int4 a = icentre[pr.x], b = icentre[pr.y];
    const int dl = a.w - b.w;
    uint64_t key = NOT_TC | (uint64_t)(uint32_t)pr.x;
    if (dl <= TC_MAX_DL && dl >= -TC_MAX_DL) {
        // offset in units of the smaller cell's side 2^sh: twice-centre differences
        // are exact multiples of it, so the arithmetic shift divides exactly
        const int sh = FMM_MAX_LEVEL - max(a.w, b.w);
        const int64_t v[3] = {((int64_t)a.x - b.x) >> sh, ((int64_t)a.y - b.y) >> sh, ((int64_t)a.z - b.z) >> sh};
        bool fits = true;
        for (int d = 0; d < 3; d++) fits = fits && v[d] > -32768 && v[d] < 32768;
        if (fits)
            key = ((uint64_t)(dl + 16) << 48) | ((uint64_t)(v[0] + 32768) << 32) | ((uint64_t)(v[1] + 32768) << 16) |
                  (uint64_t)(v[2] + 32768);
    }
    return key;
}

__global__ void k_class_keys(int64_t np, const int2* __restrict__ pairs, const int4* __restrict__ icentre,
                             uint64_t* keys, int32_t* idx) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= np) return;
    keys[e] = pair_class_key(pairs[e], icentre);
    idx[e] = (int32_t)e;
}

// per segment: number of 128-row work items
__global__ void k_class_tiles(int nseg, const int32_t* counts, int32_t* tiles) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nseg) tiles[c] = (counts[c] + TC_ROWS - 1) / TC_ROWS;
}

// Spatial blocks of the tensor-core work: the octant at level TC_BLOCK_LEVEL
// of the target cell.  Work items are ordered by (spatial block, class), and
// every block of the kernel takes its share of each spatial block in turn, so
// that at any time the SMs gather sources and reduce into targets of one
// region of the tree.  Measured on 4M clustered particles at level 1 (8
// blocks): DRAM traffic of the kernel fell from 24 to 0.9 GB but its time did
// not (the gathers and reductions are bound per SM, not by DRAM), and the
// extra sort cost 2.3 ms of build, so one block (level 0, no re-sort) is used.
constexpr int TC_BLOCK_LEVEL = 0, TC_NSPATIAL = 1 << (3 * TC_BLOCK_LEVEL);
__device__ __forceinline__ int spatial_block(int level, uint64_t ckey) {
    return level >= TC_BLOCK_LEVEL ? (int)(ckey >> (3 * (level - TC_BLOCK_LEVEL)))
                                   : (int)(ckey << (3 * (TC_BLOCK_LEVEL - level)));
}

// sort key of position i of `order` (the kept classes' pairs in class order):
// spatial block of the target << cbits | class
// (by_level: FMM_MAX_LEVEL - level of the source instead, so that the task
// graph meets the deepest source levels first)
__global__ void k_segment_keys(int64_t ntc, int nclass, int cbits, int by_level, const int32_t* __restrict__ cfirst,
                               const int32_t* __restrict__ order, const int2* __restrict__ pairs,
                               const int32_t* __restrict__ level, const uint64_t* __restrict__ ckey, int32_t* key) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ntc) return;
    int lo = 0, hi = nclass;   // last class with cfirst <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cfirst[mid] <= i) lo = mid; else hi = mid;
    }
    const int2 pr = pairs[order[i]];
    const int grp = by_level ? FMM_MAX_LEVEL - level[pr.y] : spatial_block(level[pr.x], ckey[pr.x]);
    key[i] = (grp << cbits) | lo;
}

// work items of 128 pairs per segment (run of equal block and class):
// (class, first pair, rows, spatial block)
__global__ void k_emit_items(int nseg, int cbits, const int32_t* __restrict__ segkey, const int32_t* __restrict__ segc,
                             const int32_t* __restrict__ segf, const int32_t* __restrict__ tile_first, int4* items) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nseg) return;
    const int n = segc[g], f = segf[g], cls = segkey[g] & ((1 << cbits) - 1), blk = segkey[g] >> cbits;
    int w = tile_first[g];
    for (int r = 0; r < n; r += TC_ROWS) items[w++] = make_int4(cls, f + r, min(TC_ROWS, n - r), blk);
}

// Cost of each work item for splitting the work over the kernel's blocks: one
// unit, plus TC_RUN_COST when the item starts a class run (its block assembles
// the operator of that class).
constexpr int TC_RUN_COST = 2;
__global__ void k_item_cost(int64_t nitems, const int4* __restrict__ items, int32_t* cost) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nitems) return;
    cost[i] = 1 + ((i == 0 || items[i].x != items[i - 1].x) ? TC_RUN_COST : 0);
}

// One block of threads: kernel block k gets, from every spatial block b (items
// [bs_b, bs_{b+1})), the contiguous share whose inclusive cost prefix falls in
// (k / nb, (k + 1) / nb] of that spatial block's cost; list[first[k] ..
// first[k + 1]) holds those items, spatial block after spatial block.
__global__ void k_block_lists(int64_t nitems, const int4* __restrict__ items, const int32_t* __restrict__ pre, int nb,
                              int ngroup, int32_t* list, int32_t* first) {
    __shared__ int32_t bs[33];
    __shared__ int32_t off[257];
    const int k = threadIdx.x;
    if (k <= ngroup) {   // first item of group k
        int64_t lo = 0, hi = nitems;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (items[mid].w < k) lo = mid + 1; else hi = mid;
        }
        bs[k] = (int32_t)lo;
    }
    __syncthreads();
    auto bound = [&](int b, int kk) -> int32_t {   // first item of block kk's share of spatial block b
        const int32_t i0 = bs[b], i1 = bs[b + 1];
        if (kk <= 0 || i1 <= i0) return i0;
        if (kk >= nb) return i1;
        const int64_t base = i0 > 0 ? pre[i0 - 1] : 0, tot = (int64_t)pre[i1 - 1] - base;
        const int64_t target = base + tot * kk / nb;
        int32_t lo = i0, hi = i1;
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (pre[mid] > target) hi = mid; else lo = mid + 1;
        }
        return lo;
    };
    int32_t len = 0;
    if (k < nb)
        for (int b = 0; b < ngroup; b++) len += bound(b, k + 1) - bound(b, k);
    if (k < nb) off[k + 1] = len;
    __syncthreads();
    if (k == 0) {
        off[0] = 0;
        for (int j = 1; j <= nb; j++) off[j] += off[j - 1];
    }
    __syncthreads();
    if (k <= nb) first[k] = off[k];
    if (k < nb) {
        int32_t pos = off[k];
        for (int b = 0; b < ngroup; b++) {
            const int32_t e0 = bound(b, k), e1 = bound(b, k + 1);
            for (int32_t i = e0; i < e1; i++) list[pos++] = i;
        }
    }
}

__global__ void k_gather_pairs(int64_t np, const int32_t* __restrict__ order, const int2* __restrict__ pairs,
                               int32_t* otgt, int32_t* osrc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int2 pr = pairs[order[i]];
    otgt[i] = pr.x;
    osrc[i] = pr.y;
}

// number of sorted keys below NOT_TC (the pairs that belong to a class)
__global__ void k_count_classed(const uint64_t* keys, int64_t np, int64_t* out) {
    int64_t a = 0, b = np;
    while (a < b) {
        int64_t mid = (a + b) >> 1;
        if (keys[mid] < NOT_TC) a = mid + 1; else b = mid;
    }
    *out = a;
}

__global__ void k_csr_from_targets(const int32_t* tgt, int64_t np, int ncell, int64_t* start) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncell) return;
    int64_t a = 0, b = np;
    while (a < b) {
        int64_t mid = (a + b) >> 1;
        if (tgt[mid] < c) a = mid + 1; else b = mid;
    }
    start[c] = a;
}

// ---- grouping by hashing: class key -> slot of an open-addressing table;
// sorting the (few) occupied slots numbers the classes in key order, and a
// stable sort of the pairs on these short class ids groups them.
constexpr int CLASS_HASH_BITS = 17;
constexpr int CLASS_HASH_PROBES = 256;
constexpr uint64_t HASH_EMPTY = ~0ull;

__device__ __forceinline__ uint32_t class_hash(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}

// ctr[0]: pairs without a class, ctr[1]: probe limit reached
__global__ void k_class_hash(int64_t np, const int2* __restrict__ pairs, const int4* __restrict__ icentre,
                             uint64_t* table, uint32_t mask, int32_t* slot_of, unsigned long long* ctr) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int slot = -2;  // -2: no pair, -1: pair without a class
    if (e < np) {
        const uint64_t key = pair_class_key(pairs[e], icentre);
        slot = -1;
        if (!(key & NOT_TC)) {
            uint32_t h = class_hash(key) & mask;
            for (int probe = 0; probe < CLASS_HASH_PROBES; probe++) {
                uint64_t cur = table[h];
                if (cur == HASH_EMPTY) {
                    cur = atomicCAS(reinterpret_cast<unsigned long long*>(table + h), HASH_EMPTY, key);
                    if (cur == HASH_EMPTY) cur = key;
                }
                if (cur == key) { slot = (int)h; break; }
                h = (h + 1) & mask;
            }
            if (slot < 0) atomicExch(&ctr[1], 1ull);
        }
        slot_of[e] = slot;
    }
    const unsigned rem = __ballot_sync(0xffffffffu, slot == -1);
    if ((threadIdx.x & 31) == 0 && rem) atomicAdd(&ctr[0], (unsigned long long)__popc(rem));
}

// class c = rank of its key among the occupied slots
__global__ void k_number_classes(int nclass, const int32_t* __restrict__ sorted_slot, int32_t* class_of_slot) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nclass) class_of_slot[sorted_slot[c]] = c;
}

// sort keys of the pairs: their class, nclass for a pair without one
__global__ void k_class_ids(int64_t np, const int32_t* __restrict__ slot_of, const int32_t* __restrict__ class_of_slot,
                            int nclass, int32_t* cid, int32_t* idx) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int sl = slot_of[e];
    cid[e] = sl >= 0 ? class_of_slot[sl] : nclass;
    idx[e] = (int32_t)e;
}

// sizes of the classes from the sorted ids: counts[c] for c < nclass, and
// counts[nclass] = the first pair without a class
__global__ void k_class_bounds(int nclass, const int32_t* __restrict__ cid, int64_t np, int32_t* counts) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > nclass) return;
    auto lower = [&](int v) {
        int64_t a = 0, b = np;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (cid[m] < v) a = m + 1; else b = m;
        }
        return a;
    };
    const int64_t lo = lower(c);
    counts[c] = c < nclass ? (int32_t)(lower(c + 1) - lo) : (int32_t)lo;
}

__global__ void k_iota32(int n, int32_t* v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

// remainder pairs (no class) as (target << 32 | source) keys and back
__global__ void k_pack_rem(int64_t n, const int32_t* tg, const int32_t* sr, uint64_t* k) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) k[i] = ((uint64_t)(uint32_t)tg[i] << 32) | (uint32_t)sr[i];
}
__global__ void k_unpack_rem(int64_t n, const uint64_t* k, int32_t* tg, int32_t* sr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) { tg[i] = (int32_t)(k[i] >> 32); sr[i] = (int32_t)(k[i] & 0xffffffffu); }
}

// Offset of a class in units of the target cell: D / h_t, from the class key.
__device__ __forceinline__ void class_offset(uint64_t key, int& dl, double& dx, double& dy, double& dz) {
    dl = (int)((key >> 48) & 0x1f) - 16;
    const double scale = 1.0 / (double)(2 << max(0, -dl));
    dx = (double)((int)((key >> 32) & 0xffff) - 32768) * scale;
    dy = (double)((int)((key >> 16) & 0xffff) - 32768) * scale;
    dz = (double)((int)(key & 0xffff) - 32768) * scale;
}

// Irregular harmonics I_j^m(D / h_t), j <= 2p, of each class offset: computed
// in FP64, stored in FP32 (the operator is split to bf16 hi + lo anyway).  The
// tensor-core kernel assembles each class operator from these.  One warp per
// class, one column m per lane.
__global__ void k_class_harmonics(int p, int nclass, const uint64_t* __restrict__ ukeys,
                                  cplx<float>* __restrict__ harm) {
    extern __shared__ unsigned char smraw[];
    const int P = 2 * p, nh = ntri(P);
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + wib;
    if (c >= nclass) return;
    cplx<double>* I = reinterpret_cast<cplx<double>*>(smraw) + (size_t)wib * nh;
    int dl;
    double dx, dy, dz;
    class_offset(ukeys[c], dl, dx, dy, dz);
    for (int m = lane; m <= P; m += 32) irregular_column<double>(P, m, dx, dy, dz, I);
    __syncwarp();
    for (int e = lane; e < nh; e += 32) harm[(size_t)c * nh + e] = cmk<float>((float)I[e].re, (float)I[e].im);
}

// Work items and class harmonics of nclass classes with sizes counts[] and
// keys ukeys[] (both in class order); cfirst[c] receives the first pair of
// class c.
static int emit_classes(fmm_tree* t, int nclass, const uint64_t* ukeys, const int32_t* counts, int32_t* order,
                        int64_t ntc, const int2* pairs, int64_t* items_out, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    const int p = t->prm.p;
    *items_out = 0;
    if (nclass == 0) return FMM_OK;
    // the task graph takes items deepest source level first; every SM gets a
    // share of each level
    const bool by_level = tc_uses_dag(t);
    const int ngroup = by_level ? FMM_MAX_LEVEL + 1 : TC_NSPATIAL;
    int cbits = 1;
    while ((1 << cbits) < nclass) cbits++;
    const int kbits = cbits + (by_level ? 5 : 3 * TC_BLOCK_LEVEL);
    // segments: runs of equal (spatial block, class); with one spatial block the
    // pairs are in class order already and the segments are the classes
    int32_t *cfirst = nullptr, *k0 = nullptr, *k1 = nullptr, *o1 = nullptr, *segc = nullptr, *segf = nullptr;
    int32_t *tiles = nullptr, *tfirst = nullptr, *nseg_d = nullptr;
    size_t tb = 0, tb2 = 0;
    char* tmp = nullptr;
    int32_t nseg = 0;
    if (ngroup == 1) {
        nseg = nclass;
        if ((rc = dev_alloc(&k0, (size_t)nclass, nullptr, st))) return rc;
        if ((rc = dev_alloc(&segc, (size_t)nclass, nullptr, st))) return rc;
        k_iota32<<<nblk(nclass, 256), 256, 0, st>>>(nclass, k0);
        FMM_CUDA_TRY(cudaMemcpyAsync(segc, counts, sizeof(int32_t) * nclass, cudaMemcpyDeviceToDevice, st));
        cub::DeviceScan::ExclusiveSum(nullptr, tb, segc, segc, nclass, st);
        if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
        count_launch(t);
    } else {
        // the kept classes' pairs in (spatial block of the target, class) order,
        // stable, so each class keeps its target order within a block
        if ((rc = dev_alloc(&cfirst, (size_t)nclass, nullptr, st))) return rc;
        if ((rc = dev_alloc(&k0, (size_t)ntc, nullptr, st))) return rc;
        if ((rc = dev_alloc(&k1, (size_t)ntc, nullptr, st))) return rc;
        if ((rc = dev_alloc(&o1, (size_t)ntc, nullptr, st))) return rc;
        if ((rc = dev_alloc(&segc, (size_t)ntc, nullptr, st))) return rc;
        if ((rc = dev_alloc(&nseg_d, 1, nullptr, st))) return rc;
        cub::DeviceScan::ExclusiveSum(nullptr, tb, counts, cfirst, nclass, st);
        cub::DeviceRadixSort::SortPairs(nullptr, tb2, k0, k1, order, o1, ntc, 0, kbits, st);
        tb = std::max(tb, tb2);
        cub::DeviceRunLengthEncode::Encode(nullptr, tb2, k1, k0, segc, nseg_d, ntc, st);
        tb = std::max(tb, tb2);
        if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, counts, cfirst, nclass, st));
        k_segment_keys<<<nblk(ntc, 256), 256, 0, st>>>(ntc, nclass, cbits, by_level ? 1 : 0, cfirst, order, pairs,
                                                       d.level, d.ckey, k0);
        FMM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tb, k0, k1, order, o1, ntc, 0, kbits, st));
        FMM_CUDA_TRY(cudaMemcpyAsync(order, o1, sizeof(int32_t) * ntc, cudaMemcpyDeviceToDevice, st));
        FMM_CUDA_TRY(cub::DeviceRunLengthEncode::Encode(tmp, tb, k1, k0, segc, nseg_d, ntc, st));
        count_launch(t, 4);
        FMM_CUDA_TRY(cudaMemcpyAsync(&nseg, nseg_d, 4, cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    if ((rc = dev_alloc(&segf, (size_t)nseg, nullptr, st))) return rc;
    if ((rc = dev_alloc(&tiles, (size_t)nseg, nullptr, st))) return rc;
    if ((rc = dev_alloc(&tfirst, (size_t)nseg, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, segc, segf, nseg, st));
    k_class_tiles<<<nblk(nseg, 256), 256, 0, st>>>(nseg, segc, tiles);
    FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, tiles, tfirst, nseg, st));
    count_launch(t, 3);
    int32_t lt = 0, lf = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&lt, tiles + nseg - 1, 4, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(&lf, tfirst + nseg - 1, 4, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t h_items = (int64_t)lt + lf;
    if ((rc = dev_alloc(&d.tc_items, (size_t)h_items, t, st))) return rc;
    k_emit_items<<<nblk(nseg, 256), 256, 0, st>>>(nseg, cbits, k0, segc, segf, tfirst, d.tc_items);
    count_launch(t);
    // each kernel block's share of every spatial block, balanced by cost
    {
        const int nb = by_level ? std::min(t->num_sms, 255)
                                : (int)std::min<int64_t>(std::min<int64_t>(h_items, (int64_t)t->num_sms), 255);
        int32_t *cost = nullptr, *pre = nullptr;
        if ((rc = dev_alloc(&cost, (size_t)h_items, nullptr, st))) return rc;
        if ((rc = dev_alloc(&pre, (size_t)h_items, nullptr, st))) return rc;
        if ((rc = dev_alloc(&d.tc_block_first, (size_t)nb + 1, t, st))) return rc;
        if ((rc = dev_alloc(&d.tc_item_list, (size_t)h_items, t, st))) return rc;
        k_item_cost<<<nblk(h_items, 256), 256, 0, st>>>(h_items, d.tc_items, cost);
        size_t sb = 0;
        char* stmp = nullptr;
        cub::DeviceScan::InclusiveSum(nullptr, sb, cost, pre, h_items, st);
        if ((rc = dev_alloc(&stmp, sb, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceScan::InclusiveSum(stmp, sb, cost, pre, h_items, st));
        k_block_lists<<<1, 256, 0, st>>>(h_items, d.tc_items, pre, nb, ngroup, d.tc_item_list, d.tc_block_first);
        count_launch(t, 3);
        cudaFreeAsync(stmp, st);
        cudaFreeAsync(cost, st);
        cudaFreeAsync(pre, st);
        t->tc_nblocks = nb;
    }
    cudaFreeAsync(tmp, st); cudaFreeAsync(cfirst, st); cudaFreeAsync(k0, st); cudaFreeAsync(k1, st);
    cudaFreeAsync(o1, st); cudaFreeAsync(segc, st); cudaFreeAsync(segf, st); cudaFreeAsync(nseg_d, st);
    // harmonics: on the side stream, so that they overlap the rest of the
    // build and the upward pass; the tensor-core M2L waits for ev_ops
    const int nh = ntri(2 * p);
    cplx<float>* harm = nullptr;
    if ((rc = dev_alloc(&harm, (size_t)nclass * nh, t, st))) return rc;
    d.tc_harm = harm;
    if ((rc = dev_alloc(&d.tc_keys, (size_t)nclass, t, st))) return rc;
    FMM_CUDA_TRY(cudaMemcpyAsync(d.tc_keys, ukeys, sizeof(uint64_t) * nclass, cudaMemcpyDeviceToDevice, st));
    cudaStream_t so = st;
    if ((t->ops_stream || t->side_stream) && t->ev_ops) {
        so = t->ops_stream ? t->ops_stream : t->side_stream;
        FMM_CUDA_TRY(cudaEventRecord(t->ev_fork, st));
        FMM_CUDA_TRY(cudaStreamWaitEvent(so, t->ev_fork, 0));
    }
    constexpr int HW = 4;   // classes (warps) per block
    k_class_harmonics<<<nblk(nclass, HW), 32 * HW, HW * nh * sizeof(cplx<double>), so>>>(p, nclass, d.tc_keys,
                                                                                        harm);
    count_launch(t);
    FMM_CUDA_TRY(cudaGetLastError());
    if (so != st) FMM_CUDA_TRY(cudaEventRecord(t->ev_ops, so));
    cudaFreeAsync(tiles, st);
    cudaFreeAsync(tfirst, st);
    *items_out = h_items;
    return FMM_OK;
}

// A class with at most prm.tc_min_pairs pairs (default TC_MIN_PAIRS) is left
// to the CUDA-core kernel.

// flag[i] = pair i (of `order`, classes in class order first) belongs to a kept
// class: from its class id when the grouping gives one (cid, sorted like order),
// else by bisection over the classes' first pairs
__global__ void k_pair_keep_ids(int64_t np, int64_t ntc, int min_pairs, const int32_t* __restrict__ cid,
                                const int32_t* __restrict__ counts, char* __restrict__ flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    flag[i] = i < ntc && counts[cid[i]] > min_pairs;
}
__global__ void k_pair_keep(int64_t np, int64_t ntc, int nclass, int min_pairs, const int32_t* __restrict__ cfirst,
                            const int32_t* __restrict__ counts, char* __restrict__ flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    char f = 0;
    if (i < ntc) {
        int lo = 0, hi = nclass;   // last class with cfirst <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (cfirst[mid] <= i) lo = mid; else hi = mid;
        }
        f = counts[lo] > min_pairs;
    }
    flag[i] = f;
}
__global__ void k_class_keep(int nclass, int min_pairs, const int32_t* __restrict__ counts, char* __restrict__ keep) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nclass) keep[c] = counts[c] > min_pairs;
}

// Drops the classes of at most prm.tc_min_pairs pairs: order[np] (pair indices, the
// ntc classed ones in class order first) is partitioned stably into the kept
// classes' pairs followed by all others; ukeys and counts are compacted to the
// kept classes; nclass and ntc are updated.
static int drop_small_classes(fmm_tree* t, int64_t np, int32_t* order, int& nclass, uint64_t* ukeys, int32_t* counts,
                              int64_t& ntc, cudaStream_t st, const int32_t* cid = nullptr) {
    int rc;
    if (nclass == 0) return FMM_OK;
    int32_t *cfirst = nullptr, *order2 = nullptr, *counts2 = nullptr;
    uint64_t* ukeys2 = nullptr;
    char *flag = nullptr, *keep = nullptr;
    int64_t* nsel = nullptr;
    if ((rc = dev_alloc(&cfirst, (size_t)nclass, nullptr, st))) return rc;
    if ((rc = dev_alloc(&order2, (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&counts2, (size_t)nclass, nullptr, st))) return rc;
    if ((rc = dev_alloc(&ukeys2, (size_t)nclass, nullptr, st))) return rc;
    if ((rc = dev_alloc(&flag, (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&keep, (size_t)nclass, nullptr, st))) return rc;
    if ((rc = dev_alloc(&nsel, 3, nullptr, st))) return rc;
    size_t tb = 0, tb2 = 0;
    char* tmp = nullptr;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, counts, cfirst, nclass, st);
    cub::DevicePartition::Flagged(nullptr, tb2, order, flag, order2, nsel, np, st);
    tb = std::max(tb, tb2);
    cub::DeviceSelect::Flagged(nullptr, tb2, ukeys, keep, ukeys2, nsel + 1, nclass, st);
    tb = std::max(tb, tb2);
    cub::DeviceSelect::Flagged(nullptr, tb2, counts, keep, counts2, nsel + 2, nclass, st);
    tb = std::max(tb, tb2);
    if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, counts, cfirst, nclass, st));
    if (cid)
        k_pair_keep_ids<<<nblk(np, 256), 256, 0, st>>>(np, ntc, t->prm.tc_min_pairs, cid, counts, flag);
    else
        k_pair_keep<<<nblk(np, 256), 256, 0, st>>>(np, ntc, nclass, t->prm.tc_min_pairs, cfirst, counts, flag);
    k_class_keep<<<nblk(nclass, 256), 256, 0, st>>>(nclass, t->prm.tc_min_pairs, counts, keep);
    FMM_CUDA_TRY(cub::DevicePartition::Flagged(tmp, tb, order, flag, order2, nsel, np, st));
    FMM_CUDA_TRY(cub::DeviceSelect::Flagged(tmp, tb, ukeys, keep, ukeys2, nsel + 1, nclass, st));
    FMM_CUDA_TRY(cub::DeviceSelect::Flagged(tmp, tb, counts, keep, counts2, nsel + 2, nclass, st));
    count_launch(t, 6);
    int64_t h[3] = {0, 0, 0};
    FMM_CUDA_TRY(cudaMemcpyAsync(h, nsel, sizeof(h), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    FMM_CUDA_TRY(cudaMemcpyAsync(order, order2, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(ukeys, ukeys2, sizeof(uint64_t) * h[1], cudaMemcpyDeviceToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(counts, counts2, sizeof(int32_t) * h[2], cudaMemcpyDeviceToDevice, st));
    ntc = h[0];
    nclass = (int)h[1];
    cudaFreeAsync(tmp, st); cudaFreeAsync(cfirst, st); cudaFreeAsync(order2, st); cudaFreeAsync(counts2, st);
    cudaFreeAsync(ukeys2, st); cudaFreeAsync(flag, st); cudaFreeAsync(keep, st); cudaFreeAsync(nsel, st);
    return FMM_OK;
}

// chunks of at most M2L_CHUNK entries of each target's class-less list
__global__ void k_rem_nchunks(int ncell, const int64_t* __restrict__ start, int32_t* nch) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) nch[c] = (int32_t)((start[c + 1] - start[c] + M2L_CHUNK - 1) / M2L_CHUNK);
}
__global__ void k_rem_fill(int ncell, const int64_t* __restrict__ start, const int32_t* __restrict__ off, int2* chunks) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int k = off[c];
    for (int64_t e = start[c]; e < start[c + 1]; e += M2L_CHUNK) chunks[k++] = make_int2(c, (int)e);
}

__global__ void k_rem_count(int ncell, const int32_t* __restrict__ off, const int32_t* __restrict__ nch, int32_t* n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *n = off[ncell - 1] + nch[ncell - 1];
}

// The pairs without a class, tc_tgt/tc_src[ntc, np), sorted by (target,
// source), and their CSR by target for the CUDA-core kernel.  The number of
// chunks comes back through the tree's pinned words when it can wait for the
// build's last synchronisation (rem_nchunk = -1 until then); the task graph
// needs it now.
static int finish_remainder(fmm_tree* t, int64_t ntc, int64_t nrem, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    if (nrem > 0) {
        uint64_t *k0 = nullptr, *k1 = nullptr;
        if ((rc = dev_alloc(&k0, (size_t)nrem, nullptr, st))) return rc;
        if ((rc = dev_alloc(&k1, (size_t)nrem, nullptr, st))) return rc;
        k_pack_rem<<<nblk(nrem, 256), 256, 0, st>>>(nrem, d.tc_tgt + ntc, d.tc_src + ntc, k0);
        size_t tb = 0;
        char* tmp = nullptr;
        cub::DeviceRadixSort::SortKeys(nullptr, tb, k0, k1, nrem, 0, 64, st);
        if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp, tb, k0, k1, nrem, 0, 64, st));
        k_unpack_rem<<<nblk(nrem, 256), 256, 0, st>>>(nrem, k1, d.tc_tgt + ntc, d.tc_src + ntc);
        count_launch(t, 3);
        cudaFreeAsync(tmp, st);
        cudaFreeAsync(k0, st);
        cudaFreeAsync(k1, st);
    }
    if ((rc = dev_alloc(&d.rem_start, (size_t)t->ncell + 1, t, st))) return rc;
    k_csr_from_targets<<<nblk(t->ncell + 1, 256), 256, 0, st>>>(d.tc_tgt + ntc, nrem, t->ncell, d.rem_start);
    count_launch(t);
    // chunks of at most M2L_CHUNK pairs per target for the chunked CUDA-core M2L
    t->rem_nchunk = 0;
    if (nrem > 0) {
        const int nc = t->ncell;
        int32_t *nch = nullptr, *off = nullptr;
        if ((rc = dev_alloc(&nch, (size_t)nc, nullptr, st))) return rc;
        if ((rc = dev_alloc(&off, (size_t)nc, nullptr, st))) return rc;
        k_rem_nchunks<<<nblk(nc, 256), 256, 0, st>>>(nc, d.rem_start, nch);
        size_t tb = 0;
        char* tmp = nullptr;
        cub::DeviceScan::ExclusiveSum(nullptr, tb, nch, off, nc, st);
        if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, nch, off, nc, st));
        if (t->h_pin && !tc_uses_dag(t)) {
            // at most nrem / M2L_CHUNK full chunks plus one partial chunk per target
            const int64_t bound = nrem / M2L_CHUNK + std::min<int64_t>(nc, nrem) + 1;
            if ((rc = dev_alloc(&d.rem_chunks, (size_t)bound, t, st))) return rc;
            if ((rc = dev_alloc(&d.rem_count, 1, t, st))) return rc;
            k_rem_count<<<1, 32, 0, st>>>(nc, off, nch, d.rem_count);
            FMM_CUDA_TRY(cudaMemcpyAsync(t->h_pin + 4, d.rem_count, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            t->rem_nchunk = -1;
        } else {
            int32_t h[2] = {0, 0};
            FMM_CUDA_TRY(cudaMemcpyAsync(h, off + nc - 1, 4, cudaMemcpyDeviceToHost, st));
            FMM_CUDA_TRY(cudaMemcpyAsync(h + 1, nch + nc - 1, 4, cudaMemcpyDeviceToHost, st));
            FMM_CUDA_TRY(cudaStreamSynchronize(st));
            t->rem_nchunk = (int64_t)h[0] + h[1];
            if ((rc = dev_alloc(&d.rem_chunks, (size_t)std::max<int64_t>(1, t->rem_nchunk), t, st))) return rc;
        }
        k_rem_fill<<<nblk(nc, 256), 256, 0, st>>>(nc, d.rem_start, off, d.rem_chunks);
        count_launch(t, 3);
        cudaFreeAsync(tmp, st);
        cudaFreeAsync(nch, st);
        cudaFreeAsync(off, st);
    }
    return FMM_OK;
}

// Grouping by hashing (no sort of the pairs).  *done stays false when the
// table overflows; the caller then groups by sorting the class keys.
static int classes_by_hash(fmm_tree* t, const int2* pairs, bool* done, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    *done = false;
    const int64_t np = t->nm2l;
    const int H = 1 << CLASS_HASH_BITS;
    uint64_t *table = nullptr, *skeys = nullptr;
    int32_t *slot_of = nullptr, *iota = nullptr, *sslot = nullptr;
    unsigned long long* ctr = nullptr;
    int64_t* d_nclass = nullptr;
    if ((rc = dev_alloc(&table, H, nullptr, st))) return rc;
    if ((rc = dev_alloc(&skeys, H, nullptr, st))) return rc;
    if ((rc = dev_alloc(&iota, H, nullptr, st))) return rc;
    if ((rc = dev_alloc(&sslot, H, nullptr, st))) return rc;
    if ((rc = dev_alloc(&slot_of, (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&ctr, 2, nullptr, st))) return rc;
    if ((rc = dev_alloc(&d_nclass, 1, nullptr, st))) return rc;
    FMM_CUDA_TRY(cudaMemsetAsync(table, 0xff, sizeof(uint64_t) * H, st));
    FMM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * 2, st));
    k_class_hash<<<nblk(np, 256), 256, 0, st>>>(np, pairs, d.icentre, table, (uint32_t)(H - 1), slot_of, ctr);
    k_iota32<<<nblk(H, 256), 256, 0, st>>>(H, iota);
    size_t tb = 0;
    char* tmp = nullptr;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, table, skeys, iota, sslot, H, 0, CLASS_KEY_BITS, st);
    if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tb, table, skeys, iota, sslot, H, 0, CLASS_KEY_BITS, st));
    cudaFreeAsync(tmp, st);
    k_count_classed<<<1, 1, 0, st>>>(skeys, H, d_nclass);
    count_launch(t, 4);
    unsigned long long hc[2] = {0, 0};
    int64_t nclass64 = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(&nclass64, d_nclass, 8, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    auto release = [&]() {
        cudaFreeAsync(table, st); cudaFreeAsync(skeys, st); cudaFreeAsync(iota, st); cudaFreeAsync(sslot, st);
        cudaFreeAsync(slot_of, st); cudaFreeAsync(ctr, st); cudaFreeAsync(d_nclass, st);
    };
    if (hc[1] || nclass64 > H / 2) {  // probe limit hit, or a crowded table: sort the keys instead
        release();
        return FMM_OK;
    }
    int nclass = (int)nclass64;
    int64_t ntc = np - (int64_t)hc[0];
    // stable sort of the pairs by class id (a few bits: nclass + 1 ids)
    int32_t *class_of_slot = nullptr, *cid0 = nullptr, *cid1 = nullptr, *idx0 = nullptr, *idx1 = nullptr;
    int32_t *counts = nullptr, *cfirst = nullptr;
    if ((rc = dev_alloc(&class_of_slot, H, nullptr, st))) return rc;
    if ((rc = dev_alloc(&cid0, (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&cid1, (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&idx0, (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&idx1, (size_t)np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&counts, (size_t)nclass + 1, nullptr, st))) return rc;
    if ((rc = dev_alloc(&cfirst, (size_t)nclass + 1, nullptr, st))) return rc;
    if (nclass > 0) {
        k_number_classes<<<nblk(nclass, 256), 256, 0, st>>>(nclass, sslot, class_of_slot);
        count_launch(t);
    }
    k_class_ids<<<nblk(np, 256), 256, 0, st>>>(np, slot_of, class_of_slot, nclass, cid0, idx0);
    int bits = 1;
    while ((1ll << bits) <= nclass) bits++;
    tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, cid0, cid1, idx0, idx1, np, 0, bits, st);
    if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tb, cid0, cid1, idx0, idx1, np, 0, bits, st));
    cudaFreeAsync(tmp, st);
    k_class_bounds<<<nblk(nclass + 1, 256), 256, 0, st>>>(nclass, cid1, np, counts);
    count_launch(t, 3);
    if ((rc = drop_small_classes(t, np, idx1, nclass, skeys, counts, ntc, st, cid1))) return rc;
    const int64_t nrem = np - ntc;
    int64_t h_items = 0;
    if ((rc = emit_classes(t, nclass, skeys, counts, idx1, ntc, pairs, &h_items, st))) return rc;
    if ((rc = dev_alloc(&d.tc_tgt, (size_t)np, t, st))) return rc;
    if ((rc = dev_alloc(&d.tc_src, (size_t)np, t, st))) return rc;
    k_gather_pairs<<<nblk(np, 256), 256, 0, st>>>(np, idx1, pairs, d.tc_tgt, d.tc_src);
    count_launch(t);
    if ((rc = finish_remainder(t, ntc, nrem, st))) return rc;
    FMM_CUDA_TRY(cudaGetLastError());
    t->tc_nclass = nclass;
    t->tc_nitems = h_items;
    t->tc_npairs = ntc;
    t->tc_nrem = nrem;
    release();
    cudaFreeAsync(class_of_slot, st); cudaFreeAsync(cid0, st); cudaFreeAsync(cid1, st); cudaFreeAsync(idx0, st);
    cudaFreeAsync(idx1, st); cudaFreeAsync(counts, st); cudaFreeAsync(cfirst, st);
    *done = true;
    return FMM_OK;
}

int build_m2l_classes(fmm_tree* t, const int2* pairs, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    const int64_t np = t->nm2l;
    t->tc_nclass = 0; t->tc_nitems = 0; t->tc_npairs = 0;
    if (np == 0) {
        // no M2L pair at all: an empty class-less CSR keeps the M2L stage uniform
        if ((rc = dev_alloc(&d.tc_tgt, 1, t, st))) return rc;
        if ((rc = dev_alloc(&d.tc_src, 1, t, st))) return rc;
        if ((rc = dev_alloc(&d.rem_start, (size_t)t->ncell + 1, t, st))) return rc;
        FMM_CUDA_TRY(cudaMemsetAsync(d.rem_start, 0, sizeof(int64_t) * ((size_t)t->ncell + 1), st));
        return FMM_OK;
    }
    bool done = false;
    if (!(t->prm.flags & FMM_BUILD_FALLBACKS) && (rc = classes_by_hash(t, pairs, &done, st))) return rc;
    if (done) return FMM_OK;
    // grouping by sorting the class keys (tables too crowded for hashing)
    uint64_t *k0 = nullptr, *k1 = nullptr;
    int32_t *i0 = nullptr, *i1 = nullptr;
    if ((rc = dev_alloc(&k0, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&k1, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&i0, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&i1, np, nullptr, st))) return rc;
    k_class_keys<<<nblk(np, 256), 256, 0, st>>>(np, pairs, d.icentre, k0, i0);
    count_launch(t);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, k0, k1, i0, i1, (int64_t)np, 0, CLASS_KEY_BITS, st);
    char* tmp = nullptr;
    if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tb, k0, k1, i0, i1, (int64_t)np, 0, CLASS_KEY_BITS, st));
    count_launch(t);
    cudaFreeAsync(tmp, st);
    int64_t* d_ntc = nullptr;
    if ((rc = dev_alloc(&d_ntc, 1, nullptr, st))) return rc;
    k_count_classed<<<1, 1, 0, st>>>(k1, np, d_ntc);
    int64_t ntc = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&ntc, d_ntc, 8, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(d_ntc, st);
    const int64_t nrem = np - ntc;
    // run-length encode the sorted keys: classes and their sizes
    uint64_t* ukeys = nullptr;
    int32_t *counts = nullptr, *nruns = nullptr;
    if ((rc = dev_alloc(&ukeys, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&counts, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&nruns, 1, nullptr, st))) return rc;
    int32_t h_nruns = 0;
    if (ntc > 0) {
        tb = 0;
        cub::DeviceRunLengthEncode::Encode(nullptr, tb, k1, ukeys, counts, nruns, ntc, st);
        if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceRunLengthEncode::Encode(tmp, tb, k1, ukeys, counts, nruns, ntc, st));
        count_launch(t);
        cudaFreeAsync(tmp, st);
        FMM_CUDA_TRY(cudaMemcpyAsync(&h_nruns, nruns, 4, cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    int nclass = h_nruns;
    if ((rc = drop_small_classes(t, np, i1, nclass, ukeys, counts, ntc, st))) return rc;
    const int64_t nrem2 = np - ntc;
    int32_t* cfirst = nullptr;
    if ((rc = dev_alloc(&cfirst, (size_t)nclass + 1, nullptr, st))) return rc;
    int64_t h_items = 0;
    if ((rc = emit_classes(t, nclass, ukeys, counts, i1, ntc, pairs, &h_items, st))) return rc;
    // pairs in class order, then the rest (sorted by target below)
    if ((rc = dev_alloc(&d.tc_tgt, (size_t)np, t, st))) return rc;
    if ((rc = dev_alloc(&d.tc_src, (size_t)np, t, st))) return rc;
    k_gather_pairs<<<nblk(np, 256), 256, 0, st>>>(np, i1, pairs, d.tc_tgt, d.tc_src);
    count_launch(t);
    if ((rc = finish_remainder(t, ntc, nrem2, st))) return rc;
    FMM_CUDA_TRY(cudaGetLastError());
    t->tc_nclass = nclass;
    t->tc_nitems = h_items;
    t->tc_npairs = ntc;
    t->tc_nrem = nrem2;
    cudaFreeAsync(k0, st); cudaFreeAsync(k1, st); cudaFreeAsync(i0, st); cudaFreeAsync(i1, st);
    cudaFreeAsync(ukeys, st); cudaFreeAsync(counts, st); cudaFreeAsync(nruns, st);
    cudaFreeAsync(cfirst, st);
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// evaluate: real-basis split of the multipoles, transposed class product
// ---------------------------------------------------------------------------

// float offset of real coefficient c in a complex (m >= 0, triangular) row
__host__ __device__ inline int real_index_offset(int c) {
    const int d = real_index_decode(c);
    return 2 * tri(d & 0xff, (d >> 8) & 0xff) + (d >> 16);
}

// Mt (FP32 complex rows, ldM floats apart) -> [cell][hi: KI | lo: KI] bf16 in
// the real basis, zero beyond KR = (p+1)^2
__global__ void k_split_real(int ncell, int KR, int KI, int ldM, const float* __restrict__ M,
                             __nv_bfloat16* __restrict__ Ms) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)ncell * KI) return;
    const int c = (int)(e % KI);
    const int64_t cell = e / KI;
    const float v = c < KR ? M[cell * ldM + real_index_offset(c)] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Ms[cell * 2 * KI + c] = h;
    Ms[cell * 2 * KI + KI + c] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// One persistent block per SM runs its list of work items (128 pairs of one
// class each) as a warp-specialised pipeline:
//   producer (warp 16)      TMA row gather (tile::gather4) of the hi tile of the
//                           first 64-coefficient atom of each item; the source
//                           indices come through a cp.async ring;
//   gatherers (warps 8..15) cp.async 16-byte copies of the other tiles (the
//                           lo tile of that atom, both tiles of the others)
//                           into the same 128-byte swizzled layout: the TMA
//                           row gather alone delivers about 8 B/cycle per SM,
//                           cp.async from 8 warps about 18;
//   assemblers (warps 8..11, between their gathers) build the operator of each
//                           new class in one of two tensor-memory slots (lane
//                           = output coefficient, hi and lo bf16 parts) from
//                           the class harmonics;
//   MMA (warp 17)           one thread issues, per atom and K step of 16, the
//                           three products T_hi A_hi + T_lo A_hi + T_hi A_lo
//                           into one of `nacc` 128-column accumulators;
//   epilogue (warps 0..7)   reads an accumulator (lane = output coefficient,
//                           column = pair), transposes 4 x 4 blocks within
//                           lane quads, and adds 4 consecutive coefficients of
//                           a pair into the real-basis accumulator Lr with one
//                           16-byte vector reduction.
// Tensor memory: operator slot o in columns [o KI, (o+1) KI) (hi then lo,
// two bf16 per column), accumulators from column 2 KI on.  mbarriers: full /
// empty per stage (full: the producer's arrival with the TMA bytes, plus one
// arrival per gathering thread when its copies land), opfull / opempty per
// operator slot, accf / acce per accumulator, fin for the last MMAs.  Every
// wait is bounded; a wait that runs out raises a block-wide abort flag, every
// role leaves its loop, the copies in flight land before the block exits, and
// the kernel reports FMM_ERR_TIMEOUT through *status.
constexpr int TC_M = 128;                              // MMA M: output coefficients (K <= 128)
constexpr int TC_ATOM = 64;                            // coefficients per 128-byte swizzle atom
constexpr int TC_TILE_BYTES = TC_ROWS * TC_ATOM * 2;   // 128 rows x 128 B
constexpr int TC_STAGE_BYTES = 2 * TC_TILE_BYTES;      // hi and lo tiles of one atom
constexpr int TC_EPI_WARPS = 8, TC_ASM_WARPS = 4, TC_GATH_WARPS = 4;
constexpr int TC_GATHER_THREADS = 32 * (TC_ASM_WARPS + TC_GATH_WARPS);   // the assemblers gather too
constexpr int TC_PROD_WARP = TC_EPI_WARPS + TC_ASM_WARPS + TC_GATH_WARPS;
constexpr int TC_MMA_WARP = TC_PROD_WARP + 1;
constexpr int TC_THREADS = 32 * (TC_MMA_WARP + 1);
// Four stages (two items in flight) and 72 registers per thread leave room on
// each SM for blocks of the P2P kernel, which runs beside this one on another
// stream: measured on 4M clustered particles, the kernel alone 4.1 -> 4.5 ms,
// the whole overlapped evaluation 13.5 -> 12.8 ms.
constexpr int TC_MAX_STAGES = 4, TC_MAX_ACC = 3, TC_TMEM_COLS = 512, TC_MAX_REGS = 72;
constexpr int TC_SRC_AHEAD = 6, TC_SRC_RING = 8;   // producer: items of source indices in flight, ring slots
constexpr int TC_LR = 128;                         // floats per row of the real-basis accumulator

struct TcArgs {
    int p, KR, KI, nat, stages, nacc, nh;
    int wscratch;                // bytes of scratch per worker group (task-graph form)
    const int32_t* block_first;  // [gridDim.x + 1] range of each block in list
    const int32_t* list;         // work items of the blocks
    const int4* items;        // (class, first pair, rows, -)
    const int32_t* src;       // sources of the pairs in class order
    const int32_t* tgt;       // targets
    const uint64_t* keys;     // class keys
    const cplx<float>* harm;  // class harmonics
    const __nv_bfloat16* Ms;  // split multipoles, rows of [hi KI | lo KI]
    float* Lr;                // real-basis accumulator, rows of TC_LR floats
    int* status;
    long long budget_ns;
};

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, long long budget_ns, volatile int* abort_flag) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 0;; it++) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 15) {
            if (*abort_flag) return false;
            if (clock64() - t0 > 2 * budget_ns) {  // clock64 runs at about 2 GHz
                *abort_flag = 1;
                return false;
            }
        }
    }
}

// all threads of a named barrier (id, nthreads) leave together: true iff every
// one passed ok
__device__ __forceinline__ bool bar_all(int id, int nthreads, bool ok) {
    int all_ok;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\tselp.b32 %0, 1, 0, q;\n\t}\n"
        : "=r"(all_ok)
        : "r"((int)ok), "r"(id), "r"(nthreads)
        : "memory");
    return all_ok != 0;
}

// two FP32 values -> packed bf16 hi parts and packed bf16 lo parts
__device__ __forceinline__ void split_pack(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

// x0..x3 of lane 4g + r hold (row 4g + r, column k), k = 0..3; afterwards
// lane 4g + r holds (row 4g + k, column r): a 4 x 4 transpose within each lane
// quad, three shuffles.
__device__ __forceinline__ float sel4(float a0, float a1, float a2, float a3, int i) {
    const float lo = (i & 1) ? a1 : a0, hi = (i & 1) ? a3 : a2;
    return (i & 2) ? hi : lo;
}
__device__ __forceinline__ void quad_transpose(float& x0, float& x1, float& x2, float& x3, int r) {
    float o0 = x0, o1 = x1, o2 = x2, o3 = x3;
#pragma unroll
    for (int xm = 1; xm < 4; xm++) {
        const int k = r ^ xm;
        const float v = __shfl_xor_sync(0xffffffffu, sel4(x0, x1, x2, x3, k), xm);
        o0 = k == 0 ? v : o0;
        o1 = k == 1 ? v : o1;
        o2 = k == 2 ? v : o2;
        o3 = k == 3 ? v : o3;
    }
    x0 = o0; x1 = o1; x2 = o2; x3 = o3;
}
// p[0..3] += (a, b, c, d): one 16-byte vector reduction (p 16-byte aligned)
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// Entry of a class operator in the real basis: output (k, l, pa) (pa = 0 real
// part, 1 imaginary), input (n, m, pb).  From the complex M2L
//   L_k^l += (-1)^k sum_{n, |m| <= n} rho^n M_n^m conj(I_{n+k}^{m+l}),
// with M_n^{-m} = (-1)^m conj(M_n^m), the input pair (n, +-m) gives
//   I_{n+k}^{m+l} and I_{n+k}^{|l-m|} (the latter through X^{-m} = (-1)^m conj X^m),
// and the m = 0 term appears once (weight 1/2 on the symmetric form below).
// No branch: the kernel evaluates 32 entries of a row side by side.
//   colmeta  n | m << 4 | pb << 8 | tri(n, 0) << 9 | (input exists) << 15
//   Tk = tri(k, 0), ksgn = (-1)^k (0 for a padding row), H = the class harmonics
//   I_j^m as (re, im) at tri(j, 0) + m, rho^n = 2^(dl n).
__device__ __forceinline__ float class_operator_entry(uint32_t colmeta, int k, int l, int pa, int Tk, float ksgn,
                                                      int dl, const float2* __restrict__ H) {
    const int n = colmeta & 15, m = (colmeta >> 4) & 15, pb = (colmeta >> 8) & 1, trin = (colmeta >> 9) & 63;
    const int base = trin + Tk + n * k;   // tri(n + k, 0)
    const bool ge = l >= m;
    const float2 xa = H[base + m + l];
    const float2 xb = H[base + (ge ? l - m : m - l)];
    const float rp = ksgn * __int_as_float((127 + dl * n) << 23);   // (-1)^k 2^(dl n), exact
    const float sg = (((ge ? m : l) & 1) ? -1.f : 1.f);
    const float Ar = xa.x, Ai = -xa.y;
    const float Br = sg * xb.x, Bi = (ge ? -sg : sg) * xb.y;
    const float v = pa == 0 ? (pb == 0 ? Ar + Br : Bi - Ai) : (pb == 0 ? Ai + Bi : Ar - Br);
    const float w = ((colmeta >> 15) & 1) ? (m == 0 ? 0.5f : 1.f) : 0.f;
    return rp * w * v;
}

// bounded wait until every cell of level lev is final (task-graph form)
__device__ __forceinline__ bool dag_level_ready(const DagArgs& g, int lev, long long budget_ns, volatile int* abort_flag) {
    if (dag_vload(&g.lvl_done[lev]) >= g.lvl_count[lev]) return true;
    const long long t0 = clock64();
    for (;;) {
        __nanosleep(256);
        if (dag_vload(&g.lvl_done[lev]) >= g.lvl_count[lev]) return true;
        if (*abort_flag || dag_vload(g.status) != 0) { *abort_flag = 1; return false; }
        if (clock64() - t0 > 2 * budget_ns) { *abort_flag = 1; return false; }
    }
}

// DAG = false: the tensor-core M2L alone (stage-by-stage evaluation).
// DAG = true: the whole evaluation; DAG_GROUPS worker groups per block run the
// task graph of dag.cuh, items wait for their source level, and the epilogue
// counts its items towards the M2L gate.
template <bool DAG, typename O, int R>
__global__ void __maxnreg__(TC_MAX_REGS) k_m2l_tc(const __grid_constant__ CUtensorMap tmap, const TcArgs a,
                                                   const DagArgs g) {
    extern __shared__ unsigned char smraw[];
    // stages first (1024-byte aligned: the swizzle atoms), then the harmonics
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    cplx<float>* hbuf = reinterpret_cast<cplx<float>*>(sm + (size_t)a.stages * TC_STAGE_BYTES);
    __shared__ uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES], opfull[2], opempty[2], accf[TC_MAX_ACC],
        acce[TC_MAX_ACC], fin;
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    __shared__ int dec[TC_M];        // real index -> n | m << 8 | im << 16 (-1 beyond K)
    __shared__ uint32_t colmeta[TC_M];  // the same for the operator's columns (class_operator_entry)
    __shared__ int src_ring[TC_SRC_RING * TC_ROWS];
    __shared__ int wslot[DAG_GROUPS + 4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < a.stages; s++) {
            tc::mbar_init(&full[s], 1 + TC_GATHER_THREADS);
            tc::mbar_init(&empty[s], 1);
        }
        for (int o = 0; o < 2; o++) { tc::mbar_init(&opfull[o], TC_ASM_WARPS); tc::mbar_init(&opempty[o], 1); }
        for (int c = 0; c < a.nacc; c++) { tc::mbar_init(&accf[c], 1); tc::mbar_init(&acce[c], TC_EPI_WARPS); }
        tc::mbar_init(&fin, 1);
        abort_flag = 0;
    }
    if (tid < TC_M) {
        const int d = tid < a.KR ? real_index_decode(tid) : 0;
        const int n = d & 0xff, m = (d >> 8) & 0xff, pb = (d >> 16) & 1;
        dec[tid] = tid < a.KR ? d : -1;
        colmeta[tid] = (uint32_t)(n | (m << 4) | (pb << 8) | (tri(n, 0) << 9) | ((tid < a.KR ? 1 : 0) << 15));
    }
    if (warp == TC_MMA_WARP) { tc::tmem_alloc(&tslot, TC_TMEM_COLS); tc::tmem_relinquish(); }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tslot;
    const uint32_t acc_col0 = 2u * (uint32_t)a.KI;   // accumulators after the two operator slots
    const int i0 = a.block_first[blockIdx.x], nit = max(0, a.block_first[blockIdx.x + 1] - i0);
    volatile int* abort_p = &abort_flag;

    // the j-th work item of this block's list
    auto item = [&](int j) { return a.items[a.list[i0 + j]]; };
    const bool stage_scratch = (size_t)a.stages * TC_STAGE_BYTES >= (size_t)4 * a.wscratch;

    if (DAG && warp <= TC_MMA_WARP) {
        // until every multipole is final (every item then ready at once) and the
        // CUDA-core M2L tasks it releases are taken, the epilogue and gatherer
        // warps run as four more worker groups, with the stages as their
        // scratch; then every tensor-core role starts together
        if (warp < TC_PROD_WARP && stage_scratch) {
            const int grp = DAG_GROUPS + warp / 4;
            dag_worker<O, R>(g, grp, tid & (DAG_GROUP_THREADS - 1), sm + (size_t)(grp - DAG_GROUPS) * a.wscratch,
                             &wslot[grp], true);
        }
        asm volatile("bar.sync %0, %1;" ::"n"(DAG_BAR0 + DAG_GROUPS + 4), "n"(TC_THREADS) : "memory");
    }

    if (warp == TC_PROD_WARP) {
        // ---------------- producer: TMA row gather of the hi tile of each item's
        // first atom, lane l taking rows 4l .. 4l+3; plain arrivals for the
        // other stages.  The source indices of item j + TC_SRC_AHEAD are copied
        // into a ring in shared memory (cp.async) while item j is issued.
        int ctr = 0;
        bool ok = true;
        auto prefetch_rows = [&](int j) {
            if (j < nit) {
                const int4 it = item(j);
                int* ring = src_ring + (j % TC_SRC_RING) * TC_ROWS;
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int r = 4 * lane + u;
                    if (r < it.z)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_u32(ring + r)),
                                     "l"(a.src + it.y + r)
                                     : "memory");
                    else
                        ring[r] = -1;   // an empty row reads as zeros
                }
            }
            tc::cp_async_commit();   // one group per item (empty beyond the last)
        };
        for (int j = 0; j < TC_SRC_AHEAD; j++) prefetch_rows(j);
        for (int j = 0; j < nit && ok; j++) {
            if (DAG) ok = __all_sync(0xffffffffu, dag_level_ready(g, FMM_MAX_LEVEL - item(j).w, a.budget_ns, abort_p));
            if (!ok) break;
            asm volatile("cp.async.wait_group %0;" ::"n"(TC_SRC_AHEAD - 1) : "memory");
            const int* ring = src_ring + (j % TC_SRC_RING) * TC_ROWS;
            const int y[4] = {ring[4 * lane], ring[4 * lane + 1], ring[4 * lane + 2], ring[4 * lane + 3]};
            prefetch_rows(j + TC_SRC_AHEAD);
            for (int at = 0; at < a.nat; at++, ctr++) {
                const int s = ctr % a.stages, use = ctr / a.stages;
                if (use > 0) ok = tc_wait(&empty[s], (uint32_t)((use - 1) & 1), a.budget_ns, abort_p);
                if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                if (at == 0) {
                    if (lane == 0) tc::mbar_arrive_expect_tx(&full[s], TC_TILE_BYTES);
                    __syncwarp();
                    tc::tma_gather4(tc::smem_u32(sm + (size_t)s * TC_STAGE_BYTES) + 512u * lane, &tmap, 0, y[0], y[1],
                                    y[2], y[3], tc::smem_u32(&full[s]));
                } else if (lane == 0) {
                    tc::mbar_arrive(&full[s]);
                }
            }
        }
        // the copies of every stage still in flight land before the block exits
        tc::cp_async_wait_all();
        volatile int never = 0;
        for (int c = max(0, ctr - a.stages); c < ctr; c++)
            tc_wait(&full[c % a.stages], (uint32_t)((c / a.stages) & 1), a.budget_ns, &never);
    } else if (warp == TC_MMA_WARP) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_ROWS);
            int ctr = 0, cur_cls = -1, slot = 1, uses[2] = {0, 0};
            int cls_next = nit > 0 ? a.items[a.list[i0]].x : -1;
            for (int j = 0; j < nit; j++) {
                const int cls = cls_next;
                cls_next = j + 1 < nit ? a.items[a.list[i0 + j + 1]].x : -1;
                if (cls != cur_cls) {
                    slot ^= 1;
                    cur_cls = cls;
                    if (!tc_wait(&opfull[slot], (uint32_t)(uses[slot] & 1), a.budget_ns, abort_p)) break;
                    uses[slot]++;
                }
                const int acc = j % a.nacc;
                if (j >= a.nacc && !tc_wait(&acce[acc], (uint32_t)(((j / a.nacc) - 1) & 1), a.budget_ns, abort_p)) break;
                tc::fence_after_sync();
                const uint32_t dt = tbase + acc_col0 + (uint32_t)(acc * TC_ROWS);
                const uint32_t th = tbase + (uint32_t)(slot * a.KI), tl = th + (uint32_t)(a.KI / 2);
                bool ok = true;
                for (int at = 0; at < a.nat; at++, ctr++) {
                    const int s = ctr % a.stages;
                    if (!tc_wait(&full[s], (uint32_t)((ctr / a.stages) & 1), a.budget_ns, abort_p)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t bh = tc::smem_u32(sm + (size_t)s * TC_STAGE_BYTES), bl = bh + TC_TILE_BYTES;
#pragma unroll
                    for (int ks = 0; ks < TC_ATOM / 16; ks++) {
                        const uint32_t ca = (uint32_t)(8 * (4 * at + ks));
                        const uint64_t dbh = tc::make_desc_sw128(bh + 32 * ks), dbl = tc::make_desc_sw128(bl + 32 * ks);
                        tc::mma_bf16_ta(dt, th + ca, dbh, idesc, (at | ks) ? 1u : 0u);
                        tc::mma_bf16_ta(dt, tl + ca, dbh, idesc, 1u);
                        tc::mma_bf16_ta(dt, th + ca, dbl, idesc, 1u);
                    }
                    tc::commit(&empty[s]);
                }
                if (!ok) break;
                tc::commit(&accf[acc]);
                if (cls_next != cur_cls) tc::commit(&opempty[slot]);
            }
            // every MMA issued here has completed before tensor memory is released
            tc::commit(&fin);
            volatile int never = 0;
            tc_wait(&fin, 0u, a.budget_ns, &never);
        }
        __syncwarp();
    } else if (DAG && warp > TC_MMA_WARP) {
        // ---------------- worker groups of the task graph
        const int group = (warp - TC_MMA_WARP - 1) / 4;
        unsigned char* wbase = reinterpret_cast<unsigned char*>(hbuf) + ((size_t)a.nh * sizeof(cplx<float>) + 127) / 128 * 128;
        dag_worker<O, R>(g, group, tid - 32 * (TC_MMA_WARP + 1) - DAG_GROUP_THREADS * group,
                         wbase + (size_t)group * a.wscratch, &wslot[group]);
    } else if (warp >= TC_EPI_WARPS) {
        // ---------------- gatherers (warps 8..15): thread gi copies row
        // 16 (gi / 32) + (lane / 2), 16-byte chunks 4 (lane & 1) .. +3 of every
        // cp.async tile (one whole 32-byte sector per thread pair and row).
        // Warps 8..11 are also the assemblers: thread = output coefficient
        // (tensor-memory lane) of the operator of each new class.
        const int gi = tid - 32 * TC_EPI_WARPS;
        const int grow = 16 * (gi >> 5) + (lane >> 1), gc0 = 4 * (lane & 1);
        const uint32_t goff = (uint32_t)((grow >> 3) * 1024 + (grow & 7) * 128);
        const bool assembler = warp < TC_EPI_WARPS + TC_ASM_WARPS;
        const int q = (warp - TC_EPI_WARPS) & 3;
        const int co = 32 * q + lane;
        const int dco = dec[co];
        const int k = dco >= 0 ? (dco & 0xff) : 0, l = dco >= 0 ? ((dco >> 8) & 0xff) : 0, pa = (dco >> 16) & 1;
        const int Tk = tri(k, 0);
        const float ksgn = dco < 0 ? 0.f : ((k & 1) ? -1.f : 1.f);   // a padding row stays zero
        const float2* H = reinterpret_cast<const float2*>(hbuf);
        const uint32_t lane_base = tbase + ((uint32_t)(32 * q) << 16);
        int run = -1, cur_cls = -1;
        bool ok = true;
        int srcn = -1;
        if (nit > 0) { const int4 it = item(0); srcn = grow < it.z ? a.src[it.y + grow] : -1; }
        int ctr = 0;
        for (int j = 0; j < nit; j++) {
            const int4 it = item(j);
            const int src_j = srcn;
            if (j + 1 < nit) { const int4 in = item(j + 1); srcn = grow < in.z ? a.src[in.y + grow] : -1; }
            if (assembler && it.x != cur_cls) {
                // a new class run: its operator into slot run & 1 once the MMAs of
                // the run two back (the slot's last user) are done.  All 128
                // assemblers take part in every run, failed or not, and leave
                // together when one of them failed.
                cur_cls = it.x;
                run++;
                const int slot = run & 1, use = run >> 1;
                bool wok = ok;
                if (wok && use > 0) wok = tc_wait(&opempty[slot], (uint32_t)((use - 1) & 1), a.budget_ns, abort_p);
                if (!bar_all(1, 32 * TC_ASM_WARPS, wok)) {
                    ok = false;
                } else {
                    for (int e = lane + 32 * q; e < a.nh; e += 32 * TC_ASM_WARPS) hbuf[e] = a.harm[(size_t)cur_cls * a.nh + e];
                    int dl;
                    {
                        double dx, dy, dz;
                        class_offset(a.keys[cur_cls], dl, dx, dy, dz);
                    }
                    asm volatile("bar.sync 1, %0;" ::"n"(32 * TC_ASM_WARPS) : "memory");
                    const uint32_t ts = lane_base + (uint32_t)(slot * a.KI);
                    for (int ch = 0; ch < a.KI / 32; ch++) {
                        uint32_t hw[16], lw[16];
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            const float v0 = class_operator_entry(colmeta[32 * ch + 2 * i], k, l, pa, Tk, ksgn, dl, H);
                            const float v1 = class_operator_entry(colmeta[32 * ch + 2 * i + 1], k, l, pa, Tk, ksgn, dl, H);
                            split_pack(v0, v1, hw[i], lw[i]);
                        }
                        tc::tmem_st16(ts + (uint32_t)(16 * ch), hw);
                        tc::tmem_st16(ts + (uint32_t)(a.KI / 2 + 16 * ch), lw);
                    }
                    tc::tmem_wait_st();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&opfull[slot]);
                    // every assembler is past its last read of hbuf before the next run writes it
                    asm volatile("bar.sync 1, %0;" ::"n"(32 * TC_ASM_WARPS) : "memory");
                }
            }
            if (DAG && ok) ok = dag_level_ready(g, FMM_MAX_LEVEL - it.w, a.budget_ns, abort_p);
            if (!ok) {
                if (assembler) continue;   // stay in step with the other assemblers' runs
                break;
            }
            for (int at = 0; at < a.nat; at++, ctr++) {
                const int s = ctr % a.stages, use = ctr / a.stages;
                if (use > 0 && !tc_wait(&empty[s], (uint32_t)((use - 1) & 1), a.budget_ns, abort_p)) { ok = false; break; }
                const bool valid = src_j >= 0;
                const __nv_bfloat16* g = a.Ms + (size_t)(valid ? src_j : 0) * 2 * a.KI + TC_ATOM * at;
                unsigned char* base = sm + (size_t)s * TC_STAGE_BYTES + goff;
#pragma unroll
                for (int t2 = 0; t2 < 2; t2++) {
                    if (at == 0 && t2 == 0) continue;   // the producer's TMA tile
                    unsigned char* tile = base + t2 * TC_TILE_BYTES;
                    const __nv_bfloat16* gt = g + t2 * a.KI;
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const int ch = gc0 + c;
                        tc::cp_async16(tile + ((ch ^ (grow & 7)) << 4), gt + 8 * ch, valid ? 16u : 0u);
                    }
                }
                asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(&full[s]))
                             : "memory");
            }
        }
        tc::cp_async_wait_all();
    } else {
        // ---------------- epilogue: lane = output coefficient of quarter q,
        // columns (pairs) [64 part, 64 part + 64) of each accumulator.  Lane
        // quads swap 4 x 4 blocks, so lane 4g + r ends with coefficients
        // 32 q + 4g .. + 3 of one pair, added with one vector reduction.
        const int q = warp & 3, part = warp >> 2, r4 = lane & 3;
        const int cq = 32 * q + (lane & ~3);
        const bool quad_valid = cq < a.KR;
        const uint32_t lane_base = tbase + ((uint32_t)(32 * q) << 16) + acc_col0 + (uint32_t)(64 * part);
        auto load_targets = [&](int j, int& t0, int& t1) {
            const int4 it = item(j);
            const int r0 = 64 * part + lane, r1 = r0 + 32;
            t0 = r0 < it.z ? a.tgt[it.y + r0] : -1;
            t1 = r1 < it.z ? a.tgt[it.y + r1] : -1;
        };
        int tg0 = -1, tg1 = -1, ng0 = -1, ng1 = -1;
        if (nit > 0) load_targets(0, tg0, tg1);
        for (int j = 0; j < nit; j++) {
            const int acc = j % a.nacc;
            if (j + 1 < nit) load_targets(j + 1, ng0, ng1);
            const bool got = tc_wait(&accf[acc], (uint32_t)((j / a.nacc) & 1), a.budget_ns, abort_p);
            if (!__all_sync(0xffffffffu, got)) break;
            tc::fence_after_sync();
            uint32_t v[4][16];
            const uint32_t ta = lane_base + (uint32_t)(acc * TC_ROWS);
#pragma unroll
            for (int c = 0; c < 4; c++) tc::tmem_ld16_nowait(ta + 16 * c, v[c]);
            tc::tmem_wait_ld();
            // the accumulator is in registers: hand it back to the MMA thread
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[acc]);
#pragma unroll
            for (int c = 0; c < 4; c++)
#pragma unroll
                for (int b4 = 0; b4 < 4; b4++) {
                    float x0 = __uint_as_float(v[c][4 * b4]), x1 = __uint_as_float(v[c][4 * b4 + 1]);
                    float x2 = __uint_as_float(v[c][4 * b4 + 2]), x3 = __uint_as_float(v[c][4 * b4 + 3]);
                    quad_transpose(x0, x1, x2, x3, r4);
                    const int col = 16 * c + 4 * b4 + r4;   // the pair this lane now holds
                    const int t = __shfl_sync(0xffffffffu, c < 2 ? tg0 : tg1, col & 31);
                    if (t >= 0 && quad_valid) red_add_v4(a.Lr + (size_t)t * TC_LR + cq, x0, x1, x2, x3);
                }
            if (DAG) {   // this warp's share of the item has landed
                __threadfence();
                __syncwarp();
                if (lane == 0) dag_m2l_done(g, 1u);
            }
            tg0 = ng0;
            tg1 = ng1;
        }
    }
    if (DAG && warp <= TC_MMA_WARP) {
        // every tensor-core role of the block is done (its copies landed, its MMAs
        // completed, its results added): the epilogue and gatherer warps become
        // four more worker groups, with the stages as their scratch
        asm volatile("bar.sync %0, %1;" ::"n"(DAG_BAR0 + DAG_GROUPS + 4), "n"(TC_THREADS) : "memory");
        if (warp < TC_PROD_WARP && stage_scratch) {
            const int grp = DAG_GROUPS + warp / 4;
            dag_worker<O, R>(g, grp, tid & (DAG_GROUP_THREADS - 1), sm + (size_t)(grp - DAG_GROUPS) * a.wscratch,
                             &wslot[grp]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0 && abort_flag) atomicExch(a.status, 1);
    if (warp == TC_MMA_WARP) tc::tmem_dealloc(tbase, TC_TMEM_COLS);
}

// L (complex rows of ldL floats) += Lr (real-basis rows of TC_LR floats), the
// first KR coefficients of each cell
__global__ void k_fold_real(int ncell, int KR, int ldL, const float* __restrict__ Lr, float* __restrict__ L) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)ncell * KR) return;
    const int64_t cell = e / KR;
    const int c = (int)(e % KR);
    L[cell * ldL + real_index_offset(c)] += Lr[cell * TC_LR + c];
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library
// does not link the driver API)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// TMA map of the split multipole table: ncell rows of 2 KI bf16 (hi | lo),
// read in boxes of one row x 64 coefficients with the 128-byte swizzle
static int encode_split_map(fmm_tree* t) {
    const int KI = tc_kin(t->prm.p);
    auto enc = tensor_map_encoder();
    if (!enc) { fmm_set_error("tensor-core M2L: cuTensorMapEncodeTiled is unavailable"); return FMM_ERR_CUDA; }
    const cuuint64_t gdim[2] = {(cuuint64_t)(2 * KI), (cuuint64_t)t->ncell};
    const cuuint64_t gstride[1] = {(cuuint64_t)(4 * KI)};
    const cuuint32_t box[2] = {(cuuint32_t)TC_ATOM, 1u}, estride[2] = {1u, 1u};
    const CUresult r = enc(&t->tc_tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t->d.tc_msplit, gdim, gstride, box,
                           estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { fmm_set_error("tensor-core M2L: cuTensorMapEncodeTiled failed (%d)", (int)r); return FMM_ERR_CUDA; }
    t->tc_tmap_ok = true;
    return FMM_OK;
}

// Shape and arguments of the tensor-core kernel; wscratch: bytes per worker
// group (0 for the stage-by-stage form)
template <bool DAG, typename O, int R>
static int tc_setup(fmm_tree* t, size_t wscratch, TcArgs& a, size_t& smem, cudaStream_t st) {
    TreeDev& d = t->d;
    const int p = t->prm.p, KR = tc_kreal(p), KI = tc_kin(p), nh = ntri(2 * p);
    int rc;
    if (!t->tc_tmap_ok && (rc = encode_split_map(t))) return rc;
    int dev = 0, optin = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    FMM_CUDA_TRY(cudaFuncGetAttributes(&fa, k_m2l_tc<DAG, O, R>));
    const size_t hbytes = ((size_t)nh * sizeof(cplx<float>) + 127) / 128 * 128;
    const size_t other = 1024 + hbytes + (DAG ? DAG_GROUPS * wscratch : 0);   // 1024: alignment of the stages
    const size_t cap = (size_t)optin - fa.sharedSizeBytes - other;
    const int stages = (int)std::min<size_t>(TC_MAX_STAGES, cap / TC_STAGE_BYTES);
    const int nacc = std::min(TC_MAX_ACC, (TC_TMEM_COLS - 2 * KI) / TC_ROWS);
    if (stages < 2 || nacc < 1) {
        fmm_set_error("tensor-core M2L: p = %d does not fit shared or tensor memory", p);
        return FMM_ERR_ARG;
    }
    smem = (size_t)stages * TC_STAGE_BYTES + other;
    FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_tc<DAG, O, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (t->ev_ops) {
        // the class harmonics are built on a side stream; under stream capture
        // the wait enters the graph as an external event wait node
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        FMM_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        FMM_CUDA_TRY(cudaStreamWaitEvent(st, t->ev_ops,
                                         cs == cudaStreamCaptureStatusNone ? cudaEventWaitDefault : cudaEventWaitExternal));
    }
    FMM_CUDA_TRY(cudaMemsetAsync(d.tc_lr, 0, sizeof(float) * TC_LR * (size_t)t->ncell, st));
    a = TcArgs{};
    a.p = p; a.KR = KR; a.KI = KI; a.nat = KI / TC_ATOM; a.stages = stages; a.nacc = nacc;
    a.wscratch = (int)wscratch;
    a.Ms = (const __nv_bfloat16*)d.tc_msplit; a.Lr = (float*)d.tc_lr;
    a.nh = nh; a.block_first = d.tc_block_first; a.list = d.tc_item_list;
    a.items = d.tc_items; a.src = d.tc_src; a.tgt = d.tc_tgt; a.keys = d.tc_keys;
    a.harm = (const cplx<float>*)d.tc_harm; a.status = d.status; a.budget_ns = t->prm.timeout_ns;
    return FMM_OK;
}

int m2l_tensor_cores(fmm_tree* t, const float* M, float* L, cudaStream_t st, cudaEvent_t before_fold) {
    TreeDev& d = t->d;
    const int p = t->prm.p, KR = tc_kreal(p), KI = tc_kin(p), KS = kstride(p);
    if (t->tc_nitems == 0) return FMM_OK;
    int rc;
    const int64_t ne = (int64_t)t->ncell * KI;
    k_split_real<<<nblk(ne, 256), 256, 0, st>>>(t->ncell, KR, KI, 2 * KS, M, (__nv_bfloat16*)d.tc_msplit);
    count_launch(t);
    TcArgs a;
    size_t smem = 0;
    if ((rc = tc_setup<false, float, 3>(t, 0, a, smem, st))) return rc;
    stage_begin(t, FMM_STAGE_M2L_TC, st);
    k_m2l_tc<false, float, 3><<<t->tc_nblocks, TC_THREADS, smem, st>>>(t->tc_tmap, a, DagArgs{});
    count_launch(t);
    stage_end(t, FMM_STAGE_M2L_TC, st);
    if (before_fold) FMM_CUDA_TRY(cudaStreamWaitEvent(st, before_fold, 0));
    k_fold_real<<<nblk((int64_t)t->ncell * KR, 256), 256, 0, st>>>(t->ncell, KR, 2 * KS, (const float*)d.tc_lr, L);
    count_launch(t);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int tc_epilogue_warps() { return TC_EPI_WARPS; }

// The whole evaluation of the mixed form as one launch (task graph, dag.cuh):
// the tensor-core roles of every block take its item list, its worker groups
// the task queue.  One block per SM, all resident.
template <typename O>
int launch_m2l_dag(fmm_tree* t, const DagArgs& g, cudaStream_t st) {
    const size_t ws = dag_group_scratch(t->prm.p);
    TcArgs a;
    size_t smem = 0;
    int rc;
    // one block per SM, launched cooperatively: every block is resident (the
    // downward pass waits for the tensor-core items of all blocks)
    const int grid = std::min(t->num_sms, 255);
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(TC_THREADS + DAG_GROUPS * DAG_GROUP_THREADS);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (g.R <= 3) {
        if ((rc = tc_setup<true, O, 3>(t, ws, a, smem, st))) return rc;
        if (t->tc_nitems == 0) { a.block_first = t->d.dag_zero_first; a.list = t->d.dag_zero_first; }
        cfg.dynamicSmemBytes = smem;
        FMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_m2l_tc<true, O, 3>, t->tc_tmap, a, g));
    } else {
        if ((rc = tc_setup<true, O, 6>(t, ws, a, smem, st))) return rc;
        if (t->tc_nitems == 0) { a.block_first = t->d.dag_zero_first; a.list = t->d.dag_zero_first; }
        cfg.dynamicSmemBytes = smem;
        FMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_m2l_tc<true, O, 6>, t->tc_tmap, a, g));
    }
    count_launch(t);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}
template int launch_m2l_dag<float>(fmm_tree*, const DagArgs&, cudaStream_t);
template int launch_m2l_dag<double>(fmm_tree*, const DagArgs&, cudaStream_t);

}  // namespace fmm
