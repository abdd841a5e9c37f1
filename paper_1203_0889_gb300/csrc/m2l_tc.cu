// m2l_tc.cu -- M2L on the tensor cores (tcgen05), grouped by translation class.
//
// Every M2L pair (t, s) whose cells are at most ten levels apart belongs to a
// translation class (dl = level_t - level_s, V = (2c_t - 2c_s) / min(side_t, side_s)),
// an integer vector.  With per-level scaled expansions the translation is one
// real matrix per class:
//   Lt(t) += T_c Mt(s),   T_c[(k,l), (n,m)] from (-1)^k rho^n conj(I_{n+k}^{m+l}(D/h_t)),
//   D/h_t = V / 2^(1 + max(0, -dl)),  rho = h_s / h_t = 2^dl,
// so all pairs of a class form one dense product
//   C[pairs x K] = A[pairs x K] * T_c^T,  A rows = Mt of the sources (gathered).
// This is the paper's M2L (Section 2.1) regrouped: classes replace the
// per-pair operator, and the tensor cores run the products.
//
// Precision: A and T_c are split into bf16 hi + lo parts and the product is
// accumulated in FP32 in tensor memory as A_hi T_hi + A_hi T_lo + A_lo T_hi
// (about 16 significant bits per product).  Each result row is added into the
// target's local expansion with 16-byte vector atomics; pairs of rarer classes
// (level gap above ten) go through the CUDA-core kernel first, which also
// initialises every local expansion.
#include <cub/cub.cuh>
#include <cuda_bf16.h>

#include <algorithm>

#include "fmm_internal.cuh"
#include "tc_sm100.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

constexpr int TC_MAX_DL = 10;
constexpr int TC_ROWS = 128;                 // MMA M: pairs per work item
// Class keys use 53 bits: (level gap + 16) in bits 48..52, each offset component
// + 32768 in 16 bits.  A pair outside every class gets NOT_TC | target, so such
// pairs sort after all classes and by target.
constexpr uint64_t NOT_TC = 1ull << 53;
constexpr int CLASS_KEY_BITS = 54;

int tc_kpad(int p) { return ((2 * ntri(p)) + 15) & ~15; }
bool tc_supported(int p) { return tc_kpad(p) <= 144; }

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

// per class: number of 128-row work items
__global__ void k_class_tiles(int nclass, const int32_t* counts, int32_t* tiles) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nclass) tiles[c] = (counts[c] + TC_ROWS - 1) / TC_ROWS;
}

__global__ void k_emit_items(int nclass, const int32_t* counts, const int32_t* class_first,
                             const int32_t* tile_first, int4* items) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nclass) return;
    int n = counts[c], f = class_first[c], w = tile_first[c];
    for (int r = 0; r < n; r += TC_ROWS) items[w++] = make_int4(c, f + r, min(TC_ROWS, n - r), 0);
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

// The 2 x 2 real block of a class operator for output complex coefficient
// (k, l) and input (n, m): v[pa][pb], pa / pb = re|im of output / input;
// If holds the irregular harmonics of the class offset, rpow[n] = rho^n.
__device__ __forceinline__ void class_operator_block(int k, int l, int n, int m, const float* rpow,
                                                     const cplx<float>* If, float (&v)[2][2]) {
    const float s = (k & 1) ? -rpow[n] : rpow[n];
    const cplx<float>* Ij = If + tri(n + k, 0);
    if (m == 0) {
        const cplx<float> x = Ij[l];
        v[0][0] = s * x.re;
        v[1][0] = -s * x.im;
        v[0][1] = v[1][1] = 0.f;
        return;
    }
    const cplx<float> xa = Ij[m + l];
    const float Ar = xa.re, Ai = -xa.im;
    float Br, Bi;
    if (l >= m) {
        const cplx<float> xb = Ij[l - m];
        const float sg = (m & 1) ? -1.f : 1.f;
        Br = sg * xb.re;
        Bi = -sg * xb.im;
    } else {
        const cplx<float> xb = Ij[m - l];
        const float sg = (l & 1) ? -1.f : 1.f;
        Br = sg * xb.re;
        Bi = sg * xb.im;
    }
    v[0][0] = s * (Ar + Br);
    v[0][1] = s * (Bi - Ai);
    v[1][0] = s * (Ai + Bi);
    v[1][1] = s * (Ar - Br);
}

// two FP32 values split into bf16 hi and lo parts, packed in pairs
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

// Operator of one class, split into bf16 hi/lo, K-major core-matrix layout:
// rows = output coefficients (k, l, re|im), columns = input (n, m, re|im).
// A thread takes the two rows of one output complex coefficient against four
// input complex coefficients: two 16-byte core-matrix rows, adjacent in
// memory, for hi and for lo (consecutive threads, consecutive rows).
__global__ void k_class_operators(int p, int Kp, const uint64_t* __restrict__ ukeys,
                                  __nv_bfloat16* __restrict__ ops) {
    // harmonics in FP64 (one column per thread), entries assembled in FP32
    // (each entry is rounded to FP32 and split to bf16 anyway)
    extern __shared__ unsigned char smraw[];
    cplx<double>* I = reinterpret_cast<cplx<double>*>(smraw);
    cplx<float>* If = reinterpret_cast<cplx<float>*>(I + ntri(2 * p));
    float* rpow = reinterpret_cast<float*>(If + ntri(2 * p));   // rho^n, n <= p
    int8_t* tk = reinterpret_cast<int8_t*>(rpow + 32);            // tri index -> (n, m)
    int8_t* tm = tk + 256;
    const int c = blockIdx.x;
    const uint64_t key = ukeys[c];
    const int dl = (int)((key >> 48) & 0x1f) - 16;
    const double scale = 1.0 / (double)(2 << max(0, -dl));
    const double dx = (double)((int)((key >> 32) & 0xffff) - 32768) * scale;
    const double dy = (double)((int)((key >> 16) & 0xffff) - 32768) * scale;
    const double dz = (double)((int)(key & 0xffff) - 32768) * scale;
    for (int m = threadIdx.x; m <= 2 * p; m += blockDim.x) irregular_column<double>(2 * p, m, dx, dy, dz, I);
    for (int n = 0; n <= p; n++)
        for (int m = threadIdx.x; m <= n; m += blockDim.x) { tk[tri(n, m)] = (int8_t)n; tm[tri(n, m)] = (int8_t)m; }
    // rho = 2^dl exactly, so rho^n = 2^(dl n), rounded to FP32
    if (threadIdx.x <= p) rpow[threadIdx.x] = ldexpf(1.0f, dl * (int)threadIdx.x);
    __syncthreads();
    for (int e = threadIdx.x; e < ntri(2 * p); e += blockDim.x) If[e] = cmk<float>((float)I[e].re, (float)I[e].im);
    __syncthreads();
    const int K = ntri(p), kg = Kp >> 3, nchunk = Kp * kg;
    uint4* hi = reinterpret_cast<uint4*>(ops + (size_t)c * 2 * Kp * Kp);
    uint4* lo = hi + nchunk;
    for (int u = threadIdx.x; u < nchunk / 2; u += blockDim.x) {
        // 16-byte chunks 2u, 2u + 1 = rows o0, o0 + 1 of one core matrix, columns i0 .. i0 + 7
        const int core = u >> 2;
        const int o0 = (core / kg) * 8 + 2 * (u & 3), i0 = (core % kg) * 8;
        const int ko = o0 >> 1;
        float v[2][8];   // [re|im of the output][column - i0]
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int ki = (i0 >> 1) + q;
            float b[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
            if (ko < K && ki < K) class_operator_block(tk[ko], tm[ko], tk[ki], tm[ki], rpow, If, b);
            v[0][2 * q] = b[0][0];
            v[0][2 * q + 1] = b[0][1];
            v[1][2 * q] = b[1][0];
            v[1][2 * q + 1] = b[1][1];
        }
#pragma unroll
        for (int pa = 0; pa < 2; pa++) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int w = 0; w < 4; w++) split2(v[pa][2 * w], v[pa][2 * w + 1], h[w], l[w]);
            hi[2 * u + pa] = make_uint4(h[0], h[1], h[2], h[3]);
            lo[2 * u + pa] = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
}

// Work items and operators of nclass classes with sizes counts[] and keys
// ukeys[] (both in class order); cfirst[c] receives the first pair of class c.
static int emit_classes(fmm_tree* t, int nclass, const uint64_t* ukeys, const int32_t* counts, int32_t* cfirst,
                        int64_t* items_out, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    const int p = t->prm.p, Kp = tc_kpad(p);
    *items_out = 0;
    if (nclass == 0) return FMM_OK;
    int32_t *tiles = nullptr, *tfirst = nullptr;
    if ((rc = dev_alloc(&tiles, (size_t)nclass + 1, nullptr, st))) return rc;
    if ((rc = dev_alloc(&tfirst, (size_t)nclass + 1, nullptr, st))) return rc;
    size_t tb = 0;
    char* tmp = nullptr;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, counts, cfirst, nclass, st);
    if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, counts, cfirst, nclass, st));
    k_class_tiles<<<nblk(nclass, 256), 256, 0, st>>>(nclass, counts, tiles);
    FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, tb, tiles, tfirst, nclass, st));
    count_launch(t, 3);
    cudaFreeAsync(tmp, st);
    int32_t lt = 0, lf = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&lt, tiles + nclass - 1, 4, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(&lf, tfirst + nclass - 1, 4, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t h_items = (int64_t)lt + lf;
    if ((rc = dev_alloc(&d.tc_items, (size_t)h_items, t, st))) return rc;
    k_emit_items<<<nblk(nclass, 256), 256, 0, st>>>(nclass, counts, cfirst, tfirst, d.tc_items);
    count_launch(t);
    // operators: on the side stream, so that they overlap the rest of the
    // build and the upward pass; the tensor-core M2L waits for ev_ops
    size_t ob = (size_t)nclass * 2 * Kp * Kp;
    __nv_bfloat16* ops = nullptr;
    if ((rc = dev_alloc(&ops, ob, t, st))) return rc;
    d.tc_ops = ops;
    if ((rc = dev_alloc(&d.tc_keys, (size_t)nclass, t, st))) return rc;
    FMM_CUDA_TRY(cudaMemcpyAsync(d.tc_keys, ukeys, sizeof(uint64_t) * nclass, cudaMemcpyDeviceToDevice, st));
    cudaStream_t so = st;
    if ((t->ops_stream || t->side_stream) && t->ev_ops) {
        so = t->ops_stream ? t->ops_stream : t->side_stream;
        FMM_CUDA_TRY(cudaEventRecord(t->ev_fork, st));
        FMM_CUDA_TRY(cudaStreamWaitEvent(so, t->ev_fork, 0));
    }
    size_t smem = ntri(2 * p) * (sizeof(cplx<double>) + sizeof(cplx<float>)) + 32 * 4 + 512;
    k_class_operators<<<nclass, 256, smem, so>>>(p, Kp, d.tc_keys, ops);
    count_launch(t);
    FMM_CUDA_TRY(cudaGetLastError());
    if (so != st) FMM_CUDA_TRY(cudaEventRecord(t->ev_ops, so));
    cudaFreeAsync(tiles, st);
    cudaFreeAsync(tfirst, st);
    *items_out = h_items;
    return FMM_OK;
}

// The pairs without a class, tc_tgt/tc_src[ntc, np), sorted by (target,
// source), and their CSR by target for the CUDA-core kernel.
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
    const int nclass = (int)nclass64;
    const int64_t nrem = (int64_t)hc[0], ntc = np - nrem;
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
    int64_t h_items = 0;
    if ((rc = emit_classes(t, nclass, skeys, counts, cfirst, &h_items, st))) return rc;
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
    const int nclass = h_nruns;
    int32_t* cfirst = nullptr;
    if ((rc = dev_alloc(&cfirst, (size_t)nclass + 1, nullptr, st))) return rc;
    int64_t h_items = 0;
    if ((rc = emit_classes(t, nclass, ukeys, counts, cfirst, &h_items, st))) return rc;
    // pairs in class order; the tail (no class) is in target order already
    if ((rc = dev_alloc(&d.tc_tgt, (size_t)np, t, st))) return rc;
    if ((rc = dev_alloc(&d.tc_src, (size_t)np, t, st))) return rc;
    k_gather_pairs<<<nblk(np, 256), 256, 0, st>>>(np, i1, pairs, d.tc_tgt, d.tc_src);
    count_launch(t);
    if ((rc = finish_remainder(t, ntc, nrem, st))) return rc;
    FMM_CUDA_TRY(cudaGetLastError());
    t->tc_nclass = nclass;
    t->tc_nitems = h_items;
    t->tc_npairs = ntc;
    t->tc_nrem = nrem;
    cudaFreeAsync(k0, st); cudaFreeAsync(k1, st); cudaFreeAsync(i0, st); cudaFreeAsync(i1, st);
    cudaFreeAsync(ukeys, st); cudaFreeAsync(counts, st); cudaFreeAsync(nruns, st);
    cudaFreeAsync(cfirst, st);
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// evaluate: split multipoles, tensor-core product, vector-atomic accumulation
// ---------------------------------------------------------------------------

// Mt (FP32 complex, row stride KS) -> [cell][hi: Kp | lo: Kp] bf16, real layout (re, im)
__global__ void k_split_multipoles(int ncell, int K2, int KS, int Kp, const float* __restrict__ M,
                                   __nv_bfloat16* __restrict__ Ms) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)ncell * Kp) return;
    int c = (int)(e / Kp), j = (int)(e % Kp);
    float v = j < K2 ? M[(int64_t)c * 2 * KS + j] : 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    Ms[(int64_t)c * 2 * Kp + j] = h;
    Ms[(int64_t)c * 2 * Kp + Kp + j] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// One persistent block per SM runs its range of work items as a
// warp-specialised pipeline:
//   producer warps (4)  gather the 128 source rows of an item (hi and lo
//                       bf16 halves) into one of `stages` shared-memory stages
//                       with cp.async, plus the class operator into one of
//                       `nslots` operator slots when the class changes;
//   MMA warp (1)        one thread issues the 3 x Kp/16 tcgen05.mma of an item
//                       into one of `nacc` TMEM accumulators (Kp columns each)
//                       and commits them to mbarriers;
//   epilogue warps (8)  drain a finished accumulator into the targets' rows
//                       of L with float2 reductions, two warps per TMEM lane
//                       quarter, each taking half of the column blocks.
// mbarriers: full[s] (producers -> MMA), empty[s] (MMA completion ->
// producers), accf[a] (MMA completion -> epilogue), acce[a] (epilogue ->
// MMA), opfree[o] (MMA completion of a class run -> producers).  Every wait is
// bounded; a wait that runs out raises a block-wide abort flag, every role
// leaves its loop, and the kernel reports FMM_ERR_TIMEOUT through *status.
constexpr int TC_EPI_WARPS = 8, TC_PROD_WARPS = 4;
constexpr int TC_MMA_WARP = TC_EPI_WARPS + TC_PROD_WARPS;
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + TC_PROD_WARPS + 1);
constexpr int TC_PROD_THREADS = 32 * TC_PROD_WARPS;
constexpr int TC_MAX_STAGES = 4, TC_MAX_ACC = 4, TC_TMEM_COLS = 512;
// drain accumulators with TMA bulk reductions where the staging tiles fit
constexpr bool TC_BULK_DRAIN = true;

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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// producer thread pt (0..127): its share of the 128 x Kp source rows (hi,
// lo); src[r] is the source cell of row r, -1 for an empty row.  One warp
// instruction covers 8 rows x 4 consecutive 16-byte chunks: 64 contiguous
// bytes (two whole sectors) per source row, and four whole 128-byte core
// matrices in shared memory (no bank conflicts).
__device__ __forceinline__ void tc_gather(int pt, int Kp, int cpr, const int* src,
                                          const __nv_bfloat16* __restrict__ Ms, unsigned char* A_hi,
                                          unsigned char* A_lo) {
    const int lane = pt & 31, r_in = lane & 7, j_in = lane >> 3;
    const int ntile = (TC_ROWS / 8) * ((cpr + 3) / 4);
    for (int t = pt >> 5; t < ntile; t += TC_PROD_WARPS) {
        const int r = 8 * (t % (TC_ROWS / 8)) + r_in, j = 4 * (t / (TC_ROWS / 8)) + j_in;
        if (j >= cpr) continue;
        const int sc = src[r];
        const bool valid = sc >= 0;
        const __nv_bfloat16* g = Ms + (size_t)(valid ? sc : 0) * 2 * Kp + 8 * j;
        const uint32_t off = tc::core_offset(r, 8 * j, Kp);
        tc::cp_async16_ca(A_hi + off, g, valid ? 16u : 0u);
        tc::cp_async16_ca(A_lo + off, g + Kp, valid ? 16u : 0u);
    }
}

__device__ __forceinline__ void tc_load_operator(int pt, int Kp, int cls, const __nv_bfloat16* __restrict__ ops,
                                                 unsigned char* B) {
    const unsigned char* g = reinterpret_cast<const unsigned char*>(ops + (size_t)cls * 2 * Kp * Kp);
    const int nchunk = Kp * Kp * 2 * 2 / 16;  // hi then lo, contiguous in both places
    for (int q = pt; q < nchunk; q += TC_PROD_THREADS) tc::cp_async16(B + 16 * q, g + 16 * q, 16);
}

// Column blocks of 16 a drain warp reads per item: half of Kp / 16, at most
// 5 (Kp = 144).
constexpr int TC_MAX_CB = 5;

// Reads the warp's share of one accumulator: rows 32 quarter + 16 h + lane/4
// (v[h][c][0..1], v[h][c][4..5]) and that row + 8 (v[h][c][2..3],
// v[h][c][6..7]), column blocks cb0 + c for c < ncb, all loads issued before
// one wait.
__device__ __forceinline__ void tc_load_acc(uint32_t tacc, int quarter, int cb0, int ncb,
                                            uint32_t (&v)[2][TC_MAX_CB][8]) {
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int c = 0; c < TC_MAX_CB; c++)
            if (c < ncb) tc::tmem_ld16x256_nowait(tacc + ((uint32_t)(32 * quarter + 16 * h) << 16) + 16 * (cb0 + c), v[h][c]);
    tc::tmem_wait_ld();
}

// Adds one accumulator (TMEM columns from tacc on) into the targets' rows of
// L; tgt[h][0..1] are the targets of rows 32 quarter + 16 h + lane/4 (+ 8),
// -1 for an empty row.  The 16x256b TMEM load gives four consecutive threads
// eight consecutive columns of one row, so each warp-wide float2 reduction
// covers eight whole 32-byte sectors.
__device__ __forceinline__ void tc_drain(uint32_t tacc, int quarter, int cb0, int cb1, int ncols, int ldL,
                                         const int (&tgt)[2][2], float* __restrict__ L) {
    const int lane = threadIdx.x & 31;
    uint32_t v[2][TC_MAX_CB][8];
    tc_load_acc(tacc, quarter, cb0, cb1 - cb0, v);
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int ta = tgt[h][0], tb = tgt[h][1];
        float* La = L + (size_t)(ta < 0 ? 0 : ta) * ldL;
        float* Lb = L + (size_t)(tb < 0 ? 0 : tb) * ldL;
#pragma unroll
        for (int c = 0; c < TC_MAX_CB; c++) {
            if (c >= cb1 - cb0) break;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int col = 16 * (cb0 + c) + 8 * k + 2 * (lane & 3);
                if (col < ncols) {
                    if (ta >= 0)
                        atomicAdd(reinterpret_cast<float2*>(La + col),
                                  make_float2(__uint_as_float(v[h][c][4 * k]), __uint_as_float(v[h][c][4 * k + 1])));
                    if (tb >= 0)
                        atomicAdd(reinterpret_cast<float2*>(Lb + col), make_float2(__uint_as_float(v[h][c][4 * k + 2]),
                                                                                   __uint_as_float(v[h][c][4 * k + 3])));
                }
            }
        }
    }
}

// Bulk-reduction form of the drain: the warp's 32 rows x [c0, c1) columns go
// through a shared-memory tile (row stride `stride` floats), then lane r adds
// row r into its target's row of L with one TMA bulk reduction of
// 4 (c1 - c0) bytes.  tgt_row is the target of row 32 quarter + lane.
__device__ __forceinline__ void tc_drain_bulk(uint32_t tacc, int quarter, int cb0, int cb1, int c0, int c1,
                                              int stride, int ldL, int tgt_row, float* stg,
                                              float* __restrict__ L) {
    const int lane = threadIdx.x & 31;
    uint32_t v[2][TC_MAX_CB][8];
    tc_load_acc(tacc, quarter, cb0, cb1 - cb0, v);
    tc::bulk_wait_read();  // the previous item's reductions have read the tile
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int ra = 16 * h + (lane >> 2);
#pragma unroll
        for (int c = 0; c < TC_MAX_CB; c++) {
            if (c >= cb1 - cb0) break;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const int col = 16 * c + 8 * k + 2 * (lane & 3);
                *reinterpret_cast<uint2*>(stg + ra * stride + col) = make_uint2(v[h][c][4 * k], v[h][c][4 * k + 1]);
                *reinterpret_cast<uint2*>(stg + (ra + 8) * stride + col) =
                    make_uint2(v[h][c][4 * k + 2], v[h][c][4 * k + 3]);
            }
        }
    }
    tc::fence_proxy_async();
    __syncwarp();
    if (tgt_row >= 0 && c1 > c0) {
        tc::bulk_reduce_add_f32(L + (size_t)tgt_row * ldL + c0, stg + lane * stride, (uint32_t)(4 * (c1 - c0)));
        tc::bulk_commit();
    }
}

struct TcShape {
    int stages, nslots, nacc, stg_stride;  // stg_stride 0: float2 reductions, no staging tiles
    size_t smem;
};

// Stages and operator slots that fit `cap` bytes of shared memory, and TMEM
// accumulators that fit the 512 columns of one SM (one block per SM).  With
// `bulk`, each epilogue warp also gets a 32-row staging tile for the bulk
// reductions, if two stages and one operator slot still fit.  The tile's row
// stride is 8 mod 16 floats, so that the 8-byte stores of a half-warp (four
// rows of eight words) fall on distinct banks, unless that padding costs a
// pipeline stage (then 4 mod 16).
static TcShape tc_shape_stride(int Kp, size_t cap, int stride) {
    const size_t stage = (size_t)2 * TC_ROWS * Kp * 2 + TC_ROWS * sizeof(int), slot = (size_t)2 * Kp * Kp * 2;
    TcShape sh{};
    size_t stg = 0;
    if (stride > 0) {
        sh.stg_stride = stride;
        stg = (size_t)TC_EPI_WARPS * 32 * sh.stg_stride * 4;
        if (stg + 2 * stage + slot > cap) { sh.stg_stride = 0; stg = 0; }
    }
    sh.nslots = 2 * slot + 2 * stage + stg <= cap ? 2 : 1;
    sh.stages = (int)std::min<size_t>(TC_MAX_STAGES, (cap - stg - sh.nslots * slot) / stage);
    sh.nacc = std::min(TC_MAX_ACC, TC_TMEM_COLS / Kp);
    sh.smem = sh.stages * stage + sh.nslots * slot + stg;
    return sh;
}
static TcShape tc_shape(int Kp, size_t cap, bool bulk) {
    if (!bulk) return tc_shape_stride(Kp, cap, 0);
    const int w = 16 * ((Kp / 16 + 1) / 2);   // half a row (the columns of one epilogue warp)
    const TcShape a = tc_shape_stride(Kp, cap, w + 8), b = tc_shape_stride(Kp, cap, w + 4);
    return (a.stages >= b.stages && a.nslots >= b.nslots && a.stg_stride > 0) ? a : b;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_m2l_tc(int Kp, int stages, int nslots, int nacc, int stg_stride, int ncols, int ldL, int n_items, int per_cta,
             const int4* __restrict__ items, const int32_t* __restrict__ pc_src, const int32_t* __restrict__ pc_tgt,
             const __nv_bfloat16* __restrict__ ops, const __nv_bfloat16* __restrict__ Ms, float* __restrict__ L,
             int* status, long long budget_ns) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES], accf[TC_MAX_ACC], acce[TC_MAX_ACC], opfree[2];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    const size_t abytes = (size_t)TC_ROWS * Kp * 2, bbytes = (size_t)Kp * Kp * 2;
    // stage s: A hi at sm + 2 s abytes, A lo right after; operator slot o: hi at
    // sm + 2 stages abytes + 2 o bbytes, lo right after; then the row sources
    // of each stage (TC_ROWS ints per stage)
    auto A_of = [&](int s) { return sm + 2 * s * abytes; };
    auto B_of = [&](int o) { return sm + 2 * stages * abytes + 2 * o * bbytes; };
    int* src_idx = reinterpret_cast<int*>(sm + 2 * stages * abytes + 2 * nslots * bbytes);
    float* stg_all = reinterpret_cast<float*>(src_idx + stages * TC_ROWS);  // staging tiles (bulk drain)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < stages; s++) { tc::mbar_init(&full[s], TC_PROD_THREADS); tc::mbar_init(&empty[s], 1); }
        for (int a = 0; a < nacc; a++) { tc::mbar_init(&accf[a], 1); tc::mbar_init(&acce[a], TC_EPI_WARPS); }
        tc::mbar_init(&opfree[0], 1);
        tc::mbar_init(&opfree[1], 1);
        abort_flag = 0;
    }
    if (warp == TC_MMA_WARP) { tc::tmem_alloc(&tslot, TC_TMEM_COLS); tc::tmem_relinquish(); }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tslot;
    const int i0 = blockIdx.x * per_cta, i1 = min(n_items, i0 + per_cta), nit = max(0, i1 - i0);
    volatile int* abort_p = &abort_flag;

    if (warp >= TC_EPI_WARPS && warp < TC_MMA_WARP) {
        // ---------------- producers
        // Item j+1 and the source of row pt of item j+1 are loaded while item j
        // is gathered; the 128 sources of an item go through shared memory so
        // that no cp.async waits on a global load.  Each producer thread's
        // copies arrive on full[s] by themselves when they land
        // (cp.async.mbarrier.arrive.noinc), so the gather of item j+1 never
        // waits for item j.
        const int pt = tid - 32 * TC_EPI_WARPS, cpr = Kp / 8;
        int cur_cls = -1, cur_slot = 0, loads[2] = {0, 0};
        int4 item_n = nit > 0 ? items[i0] : make_int4(0, 0, 0, 0);
        int src_n = (nit > 0 && pt < item_n.z) ? pc_src[item_n.y + pt] : -1;
        for (int j = 0; j < nit; j++) {
            const int s = j % stages;
            const int4 item = item_n;
            const int src_j = src_n;
            if (j + 1 < nit) item_n = items[i0 + j + 1];
            bool ok = true;
            if (item.x != cur_cls) {
                const int o = (nslots == 2 && cur_cls >= 0) ? cur_slot ^ 1 : 0;
                const int n = o == 0 ? loads[0] : loads[1];
                // the slot is released once the MMAs of the last run that used it are done
                if (n > 0) ok = tc_wait(&opfree[o], (uint32_t)((n - 1) & 1), budget_ns, abort_p);
                if (ok) tc_load_operator(pt, Kp, item.x, ops, B_of(o));
                if (o == 0) loads[0]++; else loads[1]++;
                cur_cls = item.x;
                cur_slot = o;
            }
            if (ok && j >= stages) ok = tc_wait(&empty[s], (uint32_t)(((j / stages) - 1) & 1), budget_ns, abort_p);
            src_idx[s * TC_ROWS + pt] = src_j;
            // all producers leave together (a named barrier with an AND reduction)
            int all_ok;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %1, 0;\n\t"
                "bar.red.and.pred q, 1, %2, p;\n\tselp.b32 %0, 1, 0, q;\n\t}\n"
                : "=r"(all_ok)
                : "r"((int)ok), "n"(TC_PROD_THREADS)
                : "memory");
            if (!all_ok) break;
            if (j + 1 < nit) src_n = pt < item_n.z ? pc_src[item_n.y + pt] : -1;
            tc_gather(pt, Kp, cpr, src_idx + s * TC_ROWS, Ms, A_of(s), A_of(s) + abytes);
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(&full[s]))
                         : "memory");
        }
        cp_async_wait_group<0>();
    } else if (warp == TC_MMA_WARP) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(TC_ROWS, Kp);
            const uint32_t sbo = (Kp / 8) * 128;
            int cur_cls = -1, cur_slot = 0, last_a = -1;
            uint32_t last_parity = 0;
            int cls_n = nit > 0 ? items[i0].x : -1;
            for (int j = 0; j < nit; j++) {
                const int s = j % stages, a = j % nacc;
                const int4 item = make_int4(cls_n, 0, 0, 0);
                cls_n = j + 1 < nit ? items[i0 + j + 1].x : -1;   // used after this item's MMAs
                if (item.x != cur_cls) {
                    cur_slot = (nslots == 2 && cur_cls >= 0) ? cur_slot ^ 1 : 0;
                    cur_cls = item.x;
                }
                if (!tc_wait(&full[s], (uint32_t)((j / stages) & 1), budget_ns, abort_p)) break;
                if (j >= nacc && !tc_wait(&acce[a], (uint32_t)(((j / nacc) - 1) & 1), budget_ns, abort_p)) break;
                // the stage was written by the producers' cp.async (generic proxy)
                // and is read by the tensor core (async proxy)
                tc::fence_proxy_async();
                tc::fence_after_sync();
                const uint32_t ah = tc::smem_u32(A_of(s)), al = ah + (uint32_t)abytes;
                const uint32_t bh = tc::smem_u32(B_of(cur_slot)), bl = bh + (uint32_t)bbytes;
                const uint32_t dacc = tbase + (uint32_t)(a * Kp);
                for (int ks = 0; ks < Kp / 16; ks++) {
                    const uint32_t o = ks * 256;
                    const uint64_t dah = tc::make_desc(ah + o, 128, sbo), dal = tc::make_desc(al + o, 128, sbo);
                    const uint64_t dbh = tc::make_desc(bh + o, 128, sbo), dbl = tc::make_desc(bl + o, 128, sbo);
                    tc::mma_bf16(dacc, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                    tc::mma_bf16(dacc, dah, dbl, idesc, 1u);
                    tc::mma_bf16(dacc, dal, dbh, idesc, 1u);
                }
                tc::commit(&empty[s]);
                tc::commit(&accf[a]);
                last_a = a;
                last_parity = (uint32_t)((j / nacc) & 1);
                if (j + 1 < nit && cls_n != item.x) tc::commit(&opfree[cur_slot]);
            }
            // every MMA issued here has completed before TMEM is released
            if (last_a >= 0) {
                volatile int never = 0;
                tc_wait(&accf[last_a], last_parity, budget_ns, &never);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue
        // the targets of item j+1 are loaded while item j is drained
        const int quarter = warp & 3, part = warp >> 2, nblk = Kp / 16;
        const int cb0 = nblk * part / 2, cb1 = nblk * (part + 1) / 2;
        auto load_targets = [&](const int4 it, int (&tg)[2][2]) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int ra = 32 * quarter + 16 * h + (lane >> 2);
                tg[h][0] = ra < it.z ? pc_tgt[it.y + ra] : -1;
                tg[h][1] = ra + 8 < it.z ? pc_tgt[it.y + ra + 8] : -1;
            }
        };
        if (stg_stride > 0) {
            // bulk reductions: lane r owns row 32 quarter + r of the item
            const int c0 = 16 * cb0, c1 = min(16 * cb1, (ncols + 3) & ~3);
            float* stg = stg_all + (size_t)warp * 32 * stg_stride;
            const int row = 32 * quarter + lane;
            int4 item_n = nit > 1 ? items[i0 + 1] : make_int4(0, 0, 0, 0);
            int tg = -1, tg_n = -1;
            if (nit > 0) { const int4 it = items[i0]; tg = row < it.z ? pc_tgt[it.y + row] : -1; }
            for (int j = 0; j < nit; j++) {
                const int a = j % nacc;
                if (j + 1 < nit) tg_n = row < item_n.z ? pc_tgt[item_n.y + row] : -1;
                if (j + 2 < nit) item_n = items[i0 + j + 2];
                const bool got = tc_wait(&accf[a], (uint32_t)((j / nacc) & 1), budget_ns, abort_p);
                if (!__all_sync(0xffffffffu, got)) break;
                tc::fence_after_sync();
                tc_drain_bulk(tbase + (uint32_t)(a * Kp), quarter, cb0, cb1, c0, c1, stg_stride, ldL, tg, stg, L);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[a]);
                tg = tg_n;
            }
            tc::bulk_wait_all();
        } else {
            int tgt[2][2], tgt_n[2][2];
            int4 item_n = nit > 1 ? items[i0 + 1] : make_int4(0, 0, 0, 0);
            if (nit > 0) load_targets(items[i0], tgt);
            for (int j = 0; j < nit; j++) {
                const int a = j % nacc;
                if (j + 1 < nit) load_targets(item_n, tgt_n);
                if (j + 2 < nit) item_n = items[i0 + j + 2];
                const bool got = tc_wait(&accf[a], (uint32_t)((j / nacc) & 1), budget_ns, abort_p);
                if (!__all_sync(0xffffffffu, got)) break;
                tc::fence_after_sync();
                tc_drain(tbase + (uint32_t)(a * Kp), quarter, cb0, cb1, ncols, ldL, tgt, L);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[a]);
#pragma unroll
                for (int h = 0; h < 2; h++) { tgt[h][0] = tgt_n[h][0]; tgt[h][1] = tgt_n[h][1]; }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0 && abort_flag) atomicExch(status, 1);
    if (warp == TC_MMA_WARP) tc::tmem_dealloc(tbase, TC_TMEM_COLS);
}

int m2l_tensor_cores(fmm_tree* t, const float* M, float* L, cudaStream_t st) {
    TreeDev& d = t->d;
    const int p = t->prm.p, Kp = tc_kpad(p), K2 = 2 * ntri(p), KS = kstride(p);
    if (t->tc_nitems == 0) return FMM_OK;
    const int64_t ne = (int64_t)t->ncell * Kp;
    __nv_bfloat16* msplit = (__nv_bfloat16*)d.tc_msplit;
    const __nv_bfloat16* ops = (const __nv_bfloat16*)d.tc_ops;
    k_split_multipoles<<<nblk(ne, 256), 256, 0, st>>>(t->ncell, K2, KS, Kp, M, msplit);
    count_launch(t);
    int dev = 0, optin = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    FMM_CUDA_TRY(cudaFuncGetAttributes(&fa, k_m2l_tc));
    const size_t cap = (size_t)optin - fa.sharedSizeBytes - 128;  // slack for the 128-byte alignment
    const TcShape sh = tc_shape(Kp, cap, TC_BULK_DRAIN);
    if (sh.stages < 2 || sh.nacc < 2) {
        fmm_set_error("tensor-core M2L: Kp = %d does not fit shared memory", Kp);
        return FMM_ERR_ARG;
    }
    // at least half of the SM's shared memory, so that one block (and its 512
    // TMEM columns) runs per SM
    const size_t smem = std::max(sh.smem, (size_t)optin / 2 + 1024);
    FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = (int)std::min<int64_t>(t->tc_nitems, (int64_t)t->num_sms);
    int per_cta = (int)((t->tc_nitems + grid - 1) / grid);
    grid = (int)((t->tc_nitems + per_cta - 1) / per_cta);
    if (t->ev_ops) {
        // the class operators are built on the side stream; under stream capture
        // the wait enters the graph as an external event wait node
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        FMM_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
        FMM_CUDA_TRY(cudaStreamWaitEvent(st, t->ev_ops,
                                         cs == cudaStreamCaptureStatusNone ? cudaEventWaitDefault : cudaEventWaitExternal));
    }
    stage_begin(t, FMM_STAGE_M2L_TC, st);
    k_m2l_tc<<<grid, TC_THREADS, smem, st>>>(Kp, sh.stages, sh.nslots, sh.nacc, sh.stg_stride, K2, 2 * KS, (int)t->tc_nitems,
                                              per_cta, d.tc_items, d.tc_src, d.tc_tgt, ops, msplit, L, d.status,
                                              t->prm.timeout_ns);
    count_launch(t);
    stage_end(t, FMM_STAGE_M2L_TC, st);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmm
