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
constexpr uint64_t NOT_TC = ~0ull;

int tc_kpad(int p) { return ((2 * ntri(p)) + 15) & ~15; }
bool tc_supported(int p) { return tc_kpad(p) <= 144; }

// ---------------------------------------------------------------------------
// build: class keys, grouping, operators, work items
// ---------------------------------------------------------------------------

__global__ void k_class_keys(int64_t np, const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                             const int4* __restrict__ icentre, uint64_t* keys, int32_t* idx) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= np) return;
    int4 a = icentre[tgt[e]], b = icentre[src[e]];
    int dl = a.w - b.w;
    uint64_t key = NOT_TC;
    if (dl <= TC_MAX_DL && dl >= -TC_MAX_DL) {
        int64_t mn = (int64_t)1 << (FMM_MAX_LEVEL - max(a.w, b.w));  // side of the smaller cell, units u
        int64_t v[3] = {((int64_t)a.x - b.x) / mn, ((int64_t)a.y - b.y) / mn, ((int64_t)a.z - b.z) / mn};
        bool fits = true;
        for (int d = 0; d < 3; d++) fits = fits && v[d] > -32768 && v[d] < 32768;
        if (fits)
            key = ((uint64_t)(dl + 32) << 48) | ((uint64_t)(v[0] + 32768) << 32) | ((uint64_t)(v[1] + 32768) << 16) |
                  (uint64_t)(v[2] + 32768);
    }
    keys[e] = key;
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

__global__ void k_gather_pairs(int64_t np, const int32_t* __restrict__ order, const int32_t* __restrict__ tgt,
                               const int32_t* __restrict__ src, int32_t* otgt, int32_t* osrc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    int e = order[i];
    otgt[i] = tgt[e];
    osrc[i] = src[e];
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

// Operator of one class, split into bf16 hi/lo, K-major core-matrix layout:
// rows = output coefficients (k, l, re|im), columns = input (n, m, re|im).
__global__ void k_class_operators(int p, int Kp, const uint64_t* __restrict__ ukeys,
                                  __nv_bfloat16* __restrict__ ops) {
    // harmonics in FP64 (one column per thread), entries assembled in FP32
    // (each entry is rounded to FP32 and split to bf16 anyway)
    extern __shared__ unsigned char smraw[];
    cplx<double>* I = reinterpret_cast<cplx<double>*>(smraw);
    cplx<float>* If = reinterpret_cast<cplx<float>*>(I + ntri(2 * p));
    float* rpow = reinterpret_cast<float*>(If + ntri(2 * p));   // (-1)^k-free rho^n, n <= p
    int8_t* tk = reinterpret_cast<int8_t*>(rpow + 32);            // tri index -> (n, m)
    int8_t* tm = tk + 256;
    const int c = blockIdx.x;
    const uint64_t key = ukeys[c];
    const int dl = (int)((key >> 48) & 0xffff) - 32;
    const double scale = 1.0 / (double)(2 << max(0, -dl));
    const double dx = (double)((int)((key >> 32) & 0xffff) - 32768) * scale;
    const double dy = (double)((int)((key >> 16) & 0xffff) - 32768) * scale;
    const double dz = (double)((int)(key & 0xffff) - 32768) * scale;
    const double rho = dl >= 0 ? (double)(1 << dl) : 1.0 / (double)(1 << (-dl));
    for (int m = threadIdx.x; m <= 2 * p; m += blockDim.x) irregular_column<double>(2 * p, m, dx, dy, dz, I);
    for (int n = 0; n <= p; n++)
        for (int m = threadIdx.x; m <= n; m += blockDim.x) { tk[tri(n, m)] = (int8_t)n; tm[tri(n, m)] = (int8_t)m; }
    if (threadIdx.x <= p) rpow[threadIdx.x] = (float)pow(rho, (double)threadIdx.x);
    __syncthreads();
    for (int e = threadIdx.x; e < ntri(2 * p); e += blockDim.x) If[e] = cmk<float>((float)I[e].re, (float)I[e].im);
    __syncthreads();
    const int K2 = 2 * ntri(p);
    __nv_bfloat16* hi = ops + (size_t)c * 2 * Kp * Kp;
    __nv_bfloat16* lo = hi + (size_t)Kp * Kp;
    for (int e = threadIdx.x; e < Kp * Kp; e += blockDim.x) {
        int o = e / Kp, i = e % Kp;
        float v = 0.f;
        if (o < K2 && i < K2) {
            int k = tk[o >> 1], l = tm[o >> 1], pa = o & 1;
            int n = tk[i >> 1], m = tm[i >> 1], pb = i & 1;
            int j = n + k;
            float s = (k & 1) ? -rpow[n] : rpow[n];
            const cplx<float>* Ij = If + tri(j, 0);
            if (m == 0) {
                cplx<float> x = Ij[l];
                v = pb ? 0.f : (pa ? -s * x.im : s * x.re);
            } else {
                cplx<float> xa = Ij[m + l];
                float Ar = xa.re, Ai = -xa.im, Br, Bi;
                if (l >= m) {
                    cplx<float> xb = Ij[l - m];
                    float sg = (m & 1) ? -1.f : 1.f;
                    Br = sg * xb.re; Bi = -sg * xb.im;
                } else {
                    cplx<float> xb = Ij[m - l];
                    float sg = (l & 1) ? -1.f : 1.f;
                    Br = sg * xb.re; Bi = sg * xb.im;
                }
                if (!pa && !pb) v = s * (Ar + Br);
                else if (!pa && pb) v = s * (Bi - Ai);
                else if (pa && !pb) v = s * (Ai + Bi);
                else v = s * (Ar - Br);
            }
        }
        float f = v;
        __nv_bfloat16 h = __float2bfloat16_rn(f);
        __nv_bfloat16 r = __float2bfloat16_rn(f - __bfloat162float(h));
        uint32_t off = tc::core_offset(o, i, Kp) >> 1;
        hi[off] = h;
        lo[off] = r;
    }
}

int build_m2l_classes(fmm_tree* t, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    const int64_t np = t->nm2l;
    const int p = t->prm.p, Kp = tc_kpad(p);
    t->tc_nclass = 0; t->tc_nitems = 0; t->tc_npairs = 0;
    if (np == 0) return FMM_OK;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    int32_t *i0 = nullptr, *i1 = nullptr;
    if ((rc = dev_alloc(&k0, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&k1, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&i0, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&i1, np, nullptr, st))) return rc;
    k_class_keys<<<nblk(np, 256), 256, 0, st>>>(np, d.m2l_tgt, d.m2l_src, d.icentre, k0, i0);
    count_launch(t);
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, k0, k1, i0, i1, (int64_t)np, 0, 64, st);
    char* tmp = nullptr;
    if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tb, k0, k1, i0, i1, (int64_t)np, 0, 64, st));
    count_launch(t);
    cudaFreeAsync(tmp, st);
    // run-length encode the sorted keys: classes and their sizes
    uint64_t* ukeys = nullptr;
    int32_t *counts = nullptr, *nruns = nullptr;
    if ((rc = dev_alloc(&ukeys, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&counts, np, nullptr, st))) return rc;
    if ((rc = dev_alloc(&nruns, 1, nullptr, st))) return rc;
    tb = 0;
    cub::DeviceRunLengthEncode::Encode(nullptr, tb, k1, ukeys, counts, nruns, (int64_t)np, st);
    if ((rc = dev_alloc(&tmp, tb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceRunLengthEncode::Encode(tmp, tb, k1, ukeys, counts, nruns, (int64_t)np, st));
    count_launch(t);
    cudaFreeAsync(tmp, st);
    int32_t h_nruns = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&h_nruns, nruns, 4, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    uint64_t last_key = 0;
    int32_t last_count = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&last_key, ukeys + h_nruns - 1, 8, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(&last_count, counts + h_nruns - 1, 4, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    const int nclass = last_key == NOT_TC ? h_nruns - 1 : h_nruns;
    const int64_t nrem = last_key == NOT_TC ? last_count : 0;
    const int64_t ntc = np - nrem;
    // class offsets, items
    int32_t *cfirst = nullptr, *tiles = nullptr, *tfirst = nullptr;
    if ((rc = dev_alloc(&cfirst, (size_t)nclass + 1, nullptr, st))) return rc;
    if ((rc = dev_alloc(&tiles, (size_t)nclass + 1, nullptr, st))) return rc;
    if ((rc = dev_alloc(&tfirst, (size_t)nclass + 1, nullptr, st))) return rc;
    int32_t h_items = 0;
    if (nclass > 0) {
        tb = 0;
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
        h_items = lt + lf;
        if ((rc = dev_alloc(&d.tc_items, (size_t)h_items, t, st))) return rc;
        k_emit_items<<<nblk(nclass, 256), 256, 0, st>>>(nclass, counts, cfirst, tfirst, d.tc_items);
        count_launch(t);
        // operators
        size_t ob = (size_t)nclass * 2 * Kp * Kp;
        __nv_bfloat16* ops = nullptr;
        if ((rc = dev_alloc(&ops, ob, t, st))) return rc;
        d.tc_ops = ops;
        size_t smem = ntri(2 * p) * (sizeof(cplx<double>) + sizeof(cplx<float>)) + 32 * 4 + 512;
        k_class_operators<<<nclass, 256, smem, st>>>(p, Kp, ukeys, ops);
        count_launch(t);
    }
    // pairs in class order; the tail (no class) keeps target order for the CUDA-core kernel
    if ((rc = dev_alloc(&d.tc_tgt, (size_t)np, t, st))) return rc;
    if ((rc = dev_alloc(&d.tc_src, (size_t)np, t, st))) return rc;
    k_gather_pairs<<<nblk(np, 256), 256, 0, st>>>(np, i1, d.m2l_tgt, d.m2l_src, d.tc_tgt, d.tc_src);
    count_launch(t);
    if ((rc = dev_alloc(&d.rem_start, (size_t)t->ncell + 1, t, st))) return rc;
    k_csr_from_targets<<<nblk(t->ncell + 1, 256), 256, 0, st>>>(d.tc_tgt + ntc, nrem, t->ncell, d.rem_start);
    count_launch(t);
    FMM_CUDA_TRY(cudaGetLastError());
    t->tc_nclass = nclass;
    t->tc_nitems = h_items;
    t->tc_npairs = ntc;
    t->tc_nrem = nrem;
    cudaFreeAsync(k0, st); cudaFreeAsync(k1, st); cudaFreeAsync(i0, st); cudaFreeAsync(i1, st);
    cudaFreeAsync(ukeys, st); cudaFreeAsync(counts, st); cudaFreeAsync(nruns, st);
    cudaFreeAsync(cfirst, st); cudaFreeAsync(tiles, st); cudaFreeAsync(tfirst, st);
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

__global__ void __launch_bounds__(128) k_m2l_tc(int Kp, int ncol4, int ldL, int n_items, int per_cta,
                                                const int4* __restrict__ items, const int32_t* __restrict__ pc_src,
                                                const int32_t* __restrict__ pc_tgt,
                                                const __nv_bfloat16* __restrict__ ops,
                                                const __nv_bfloat16* __restrict__ Ms, float* __restrict__ L,
                                                int* status, long long budget_ns) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A_hi = sm;
    unsigned char* A_lo = A_hi + TC_ROWS * Kp * 2;
    unsigned char* B_hi = A_lo + TC_ROWS * Kp * 2;
    unsigned char* B_lo = B_hi + Kp * Kp * 2;
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tcols = Kp <= 128 ? 128u : 256u;
    if (warp == 0) { tc::tmem_alloc(&tslot, tcols); tc::tmem_relinquish(); }
    if (tid == 0) tc::mbar_init(&bar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    const uint32_t idesc = tc::idesc_bf16_f32(TC_ROWS, Kp);
    const uint32_t sbo_a = (Kp / 8) * 128, sbo_b = sbo_a;
    const int cpr = Kp / 8;  // 16-byte chunks per row
    const int i0 = blockIdx.x * per_cta, i1 = min(n_items, i0 + per_cta);
    int cur = -1;
    uint32_t phase = 0;
    bool ok = true;
    for (int it = i0; it < i1 && ok; it++) {
        const int4 item = items[it];
        if (item.x != cur) {
            const unsigned char* g = reinterpret_cast<const unsigned char*>(ops + (size_t)item.x * 2 * Kp * Kp);
            const int nchunk = Kp * Kp * 2 * 2 / 16;  // hi then lo, contiguous in both places
            for (int q = tid; q < nchunk; q += 128) tc::cp_async16(B_hi + 16 * q, g + 16 * q, 16);
            cur = item.x;
        }
        for (int q = tid; q < TC_ROWS * cpr; q += 128) {
            int r = q / cpr, j = q - r * cpr;
            bool valid = r < item.z;
            int s = valid ? pc_src[item.y + r] : 0;
            const __nv_bfloat16* g = Ms + (size_t)s * 2 * Kp + 8 * j;
            uint32_t off = tc::core_offset(r, 8 * j, Kp);
            tc::cp_async16(A_hi + off, g, valid ? 16u : 0u);
            tc::cp_async16(A_lo + off, g + Kp, valid ? 16u : 0u);
        }
        tc::cp_async_commit();
        tc::cp_async_wait_all();
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t ah = tc::smem_u32(A_hi), al = tc::smem_u32(A_lo);
            const uint32_t bh = tc::smem_u32(B_hi), bl = tc::smem_u32(B_lo);
            for (int ks = 0; ks < Kp / 16; ks++) {
                const uint32_t o = ks * 256;
                const uint64_t dah = tc::make_desc(ah + o, 128, sbo_a), dal = tc::make_desc(al + o, 128, sbo_a);
                const uint64_t dbh = tc::make_desc(bh + o, 128, sbo_b), dbl = tc::make_desc(bl + o, 128, sbo_b);
                tc::mma_bf16(taddr, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                tc::mma_bf16(taddr, dah, dbl, idesc, 1u);
                tc::mma_bf16(taddr, dal, dbh, idesc, 1u);
            }
            tc::commit(&bar);
        }
        bool done = tc::mbar_wait_bounded(&bar, phase, budget_ns);
        ok = __syncthreads_and(done) != 0;
        phase ^= 1u;
        tc::fence_after_sync();
        if (ok) {
            const int r = 32 * warp + lane;
            const int tg = r < item.z ? pc_tgt[item.y + r] : -1;
            float* Lrow = L + (size_t)(tg < 0 ? 0 : tg) * ldL;
            for (int cb = 0; cb < Kp / 16; cb++) {
                float v[16];
                tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + 16 * cb, v);
                if (tg >= 0) {
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        int c4 = 4 * cb + q;
                        if (c4 < ncol4)
                            atomicAdd(reinterpret_cast<float4*>(Lrow) + c4,
                                      make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(status, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, tcols);
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
    size_t smem = (size_t)2 * TC_ROWS * Kp * 2 + (size_t)2 * Kp * Kp * 2;
    FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = smem <= 100 * 1024 ? 2 : 1;
    int grid = std::min<int64_t>(t->tc_nitems, (int64_t)per_sm * t->num_sms);
    int per_cta = (int)((t->tc_nitems + grid - 1) / grid);
    grid = (int)((t->tc_nitems + per_cta - 1) / per_cta);
    const int ncol4 = (K2 + 3) / 4;
    stage_begin(t, FMM_STAGE_M2L_TC, st);
    k_m2l_tc<<<grid, 128, smem, st>>>(Kp, ncol4, 2 * KS, (int)t->tc_nitems, per_cta, d.tc_items, d.tc_src,
                                      d.tc_tgt, ops, msplit, L, d.status, t->prm.timeout_ns);
    count_launch(t);
    stage_end(t, FMM_STAGE_M2L_TC, st);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmm
