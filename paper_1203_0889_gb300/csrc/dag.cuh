// dag.cuh -- the worker side of the mixed-precision evaluation run as one
// persistent launch over a task graph (the paper's data-driven execution,
// Sections 3 and 4, with the M2L on the tensor cores).
//
// Every block of the launch holds the tensor-core M2L roles (m2l_tc.cu) and
// DAG_GROUPS worker groups of 128 threads.  A worker group takes a task from
// a device ready queue, runs it, and queues the tasks whose last dependency
// it completed:
//   P2M(4 leaves)   none                                  -> M final per leaf
//   M2M(c)          M final for each child of c            -> M final(c)
//   M final(c)      writes c's split row for the tensor cores (bf16 hi/lo,
//                   real basis) and counts c as final on its level; the last
//                   final cell of the tree queues the REM tasks
//   REM(4 chunks)   every multipole final                  (CUDA-core M2L of
//                   the pairs the tensor cores do not take, into L)
//   ROOT(r)         all M2L work landed (the tensor-core items, counted by
//                   their epilogue warps, and every REM chunk) -> L final(r)
//   L2L(c)          L final for c's parent (after the same gate)
//   L final(c)      queues L2L of each child, or counts towards L2P of a leaf
//   P2P(leaf)       none (a low-priority pool taken when the queue is empty)
//   L2P(leaf)       L final for the leaf and P2P(leaf) done
// The tensor-core items of a block are ordered by source level, deepest
// first; an item starts once every cell of its source level is final (a cell
// is final only after its children, so then every finer level is too).  The
// tensor cores add into the real-basis accumulator Lr; ROOT and L2L fold a
// cell's Lr row into its local expansion before translating it.  Interaction
// is non-mutual (Section 4): a task writes only its own cell or leaf, except
// the M2L contributions, which meet by FP32 atomics in L and Lr.
// Every wait is bounded by the tree's timeout; on expiry the status word gets
// FMM_ERR_TIMEOUT and every role returns.
#pragma once
#include <cuda_bf16.h>

#include "fmm_internal.cuh"
#include "stages.cuh"

namespace fmm {

enum DagKind { DK_P2M = 0, DK_M2M = 1, DK_REM = 2, DK_ROOT = 3, DK_L2L = 4, DK_L2P = 5, DK_P2P = 6 };
constexpr int DK_SHIFT = 28;
constexpr unsigned DK_MASK = (1u << DK_SHIFT) - 1u;
constexpr int DAG_GROUPS = 2;            // worker groups per block
constexpr int DAG_GROUP_THREADS = 128;
constexpr int DAG_GROUP_WARPS = DAG_GROUP_THREADS / 32;
constexpr int DAG_P2M_GROUP = 4;         // leaves per P2M task (one per warp)
constexpr int DAG_REM_GROUP = 4;         // CUDA-core M2L chunks per REM task (one per warp)
constexpr int DAG_BAR0 = 2;              // named barriers 2, 3: the worker groups

struct DagCounters {
    unsigned head_hi, tail_hi, head_lo, done;
    int avail;                // tasks pushed (slot written) and not yet claimed
    unsigned cells_final;     // cells whose multipole and split row are final
    unsigned m2l_done;        // tensor-core item completions (per epilogue warp) + REM chunks
    unsigned released;        // 1 once the last final cell has queued the REM tasks
};

struct DagArgs {
    int p, ncell, nleaf, nsys, field, KR, KI, R;
    unsigned n_hi, n_lo, n_tasks, m2l_total;
    int nrem_tasks;
    int64_t nrem_chunk;
    long long budget_cycles;
    const int32_t* leaves;
    const int32_t* first;
    const int32_t* count;
    const int32_t* parent;
    const int32_t* child_first;
    const int32_t* child_count;
    const int32_t* level;
    const uint64_t* ckey;
    const double4_32a* centre;
    const int4* icentre;
    const int32_t* perm;
    const float* shift_ops;
    const double4_32a* xq64;
    const float4* xq32;
    const float4* xlo32;       // residuals of the FP32 coordinates
    const int64_t* p2p_start;
    const int4* p2p_rec;
    const float* cu2f;
    const int2* rem_chunks;
    const int64_t* rem_start;
    const int32_t* rem_src;
    float* M;                  // [ncell][2 kstride] complex rows
    float* L;
    const float* Lr;           // [ncell][128] real-basis tensor-core results
    __nv_bfloat16* Ms;         // [ncell][hi KI | lo KI] split rows
    double* near;
    void* phi_out;
    void* force_out;
    int* q;                    // high-priority FIFO [n_hi]
    int* mcnt;                 // children not yet final
    int* pcnt;                 // L2P prerequisites (2 per leaf)
    int* lvl_done;             // final cells per level
    const int* lvl_count;      // cells per level
    DagCounters* ctr;
    int* status;
};

__device__ __forceinline__ unsigned dag_vload(const unsigned* p) { return *(volatile const unsigned*)p; }
__device__ __forceinline__ int dag_vload(const int* p) { return *(volatile const int*)p; }

// Push: reserve a slot, write it, then count it as available.
__device__ __forceinline__ void dag_push(const DagArgs& a, int kind, int idx) {
    const unsigned slot = atomicAdd(&a.ctr->tail_hi, 1u);
    if (slot >= a.n_hi) return;
    atomicExch(&a.q[slot], (kind << DK_SHIFT) | idx);
    __threadfence();
    atomicAdd(&a.ctr->avail, 1);
}
// One thread: push the n tasks kind:idx0 .. kind:idx0 + n - 1 with one
// reservation, one fence and one count.
__device__ __forceinline__ void dag_push_n(const DagArgs& a, int kind, int idx0, int n) {
    if (n <= 0) return;
    const unsigned base = atomicAdd(&a.ctr->tail_hi, (unsigned)n);
    if (base >= a.n_hi) return;
    const int m = (int)min((unsigned)n, a.n_hi - base);
    for (int k = 0; k < m; k++) *(volatile int*)&a.q[base + k] = (kind << DK_SHIFT) | (idx0 + k);
    __threadfence();
    atomicAdd(&a.ctr->avail, m);
}
// Warp (all lanes, n uniform): the same, the lanes writing the slots.
__device__ __forceinline__ void dag_push_n_warp(const DagArgs& a, int kind, int idx0, int n, int lane) {
    if (n <= 0) return;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(&a.ctr->tail_hi, (unsigned)n);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= a.n_hi) return;
    const int m = (int)min((unsigned)n, a.n_hi - base);
    for (int k = lane; k < m; k += 32) *(volatile int*)&a.q[base + k] = (kind << DK_SHIFT) | (idx0 + k);
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(&a.ctr->avail, m);
}

// One thread: the next task, or -1 when the graph is finished or failed (-2:
// until_upward is set, every multipole is final and no high-priority task is
// queued or being queued -- the CUDA-core M2L tasks the last final cell
// releases are taken first).  A claim that finds nothing available is undone
// and a P2P task is taken instead.
static __device__ int dag_pop(const DagArgs& a, bool until_upward) {
    const long long t0 = clock64();
    for (;;) {
        if (until_upward && dag_vload(&a.ctr->released) != 0u && dag_vload(&a.ctr->avail) <= 0 &&
            dag_vload(&a.ctr->head_hi) >= dag_vload(&a.ctr->tail_hi))
            return -2;
        if (dag_vload(&a.ctr->avail) > 0) {
            if (atomicSub(&a.ctr->avail, 1) > 0) {
                const unsigned h = atomicAdd(&a.ctr->head_hi, 1u);
                const long long t1 = clock64();
                int v;
                while ((v = dag_vload(&a.q[h])) < 0) {
                    if (clock64() - t1 > a.budget_cycles) { atomicExch(a.status, 1); return -1; }
                    __nanosleep(32);
                }
                __threadfence();
                return v;
            }
            atomicAdd(&a.ctr->avail, 1);
        }
        if (dag_vload(&a.ctr->head_lo) < a.n_lo) {
            const unsigned l = atomicAdd(&a.ctr->head_lo, 1u);
            if (l < a.n_lo) return (DK_P2P << DK_SHIFT) | (int)l;
        }
        if (dag_vload(&a.ctr->done) >= a.n_tasks || dag_vload(a.status) != 0) return -1;
        if (clock64() - t0 > a.budget_cycles) { atomicExch(a.status, 1); return -1; }
        __nanosleep(64);
    }
}

// the tasks released by the M2L gate: the roots' local expansions
__device__ __forceinline__ void dag_open_gate(const DagArgs& a) { dag_push_n(a, DK_ROOT, 0, a.nsys); }
// one unit of M2L work done (a tensor-core epilogue warp's item, or k REM chunks)
__device__ __forceinline__ void dag_m2l_done(const DagArgs& a, unsigned k) {
    __threadfence();
    const unsigned before = atomicAdd(&a.ctr->m2l_done, k);
    if (before + k == a.m2l_total) dag_open_gate(a);
}

// Warp: the multipole of cell c is final.  Writes c's split row (bf16 hi/lo
// in the real basis, tensor-core gather layout), then releases: the parent's
// M2M, c's level, and, for the last final cell, the REM tasks (or the gate when
// there is no M2L work at all).
static __device__ void dag_m_final(const DagArgs& a, int c, int lane) {
    const int KS = kstride(a.p);
    const float* Mc = a.M + (int64_t)c * 2 * KS;
    for (int j = lane; j < a.KI; j += 32) {
        float v = 0.f;
        if (j < a.KR) {
            const int d = real_index_decode(j);
            v = __ldcg(Mc + 2 * tri(d & 0xff, (d >> 8) & 0xff) + (d >> 16));
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        a.Ms[(int64_t)c * 2 * a.KI + j] = h;
        a.Ms[(int64_t)c * 2 * a.KI + a.KI + j] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) {
        const int par = a.parent[c];
        if (par >= 0 && atomicSub(&a.mcnt[par], 1) == 1) dag_push(a, DK_M2M, par);
        atomicAdd(&a.lvl_done[a.level[c]], 1);
        last = atomicAdd(&a.ctr->cells_final, 1u) + 1u == (unsigned)a.ncell;
    }
    if (__shfl_sync(0xffffffffu, last, 0)) {
        dag_push_n_warp(a, DK_REM, 0, a.nrem_tasks, lane);
        if (lane == 0) {
            if (a.m2l_total == 0) dag_open_gate(a);
            __threadfence();
            atomicExch(&a.ctr->released, 1u);
        }
    }
}

// Warp: the local expansion of cell c is final (L2L of the children, or the
// leaf's L2P once its P2P is done too).
static __device__ void dag_l_final(const DagArgs& a, int c, int lane) {
    const int nc = a.child_count[c];
    if (nc == 0) {
        if (lane == 0 && atomicSub(&a.pcnt[c], 1) == 1) dag_push(a, DK_L2P, c);
        return;
    }
    dag_push_n_warp(a, DK_L2L, a.child_first[c], nc, lane);
}

// Group: L(c) += the tensor-core results of c (real basis -> complex row)
static __device__ void dag_fold(const DagArgs& a, int c, int gtid) {
    const int KS = kstride(a.p);
    float* Lc = a.L + (int64_t)c * 2 * KS;
    const float* R = a.Lr + (int64_t)c * 128;
    for (int j = gtid; j < a.KR; j += DAG_GROUP_THREADS) {
        const int d = real_index_decode(j);
        float* dst = Lc + 2 * tri(d & 0xff, (d >> 8) & 0xff) + (d >> 16);
        *dst = __ldcg(dst) + __ldcg(R + j);
    }
}

// Scratch of one worker group, in bytes: the largest need of its tasks.
__host__ __device__ inline size_t dag_group_scratch(int p) {
    const int K = ntri(p), KI2 = ntri(2 * p);
    size_t s = (size_t)P2P_BUF * sizeof(float4) + (size_t)P2P_THREADS * 4 * sizeof(float);   // P2P
    const size_t rem = (size_t)4 * 2 * (K + KI2) * sizeof(cplx<float>);                         // REM
    const size_t p2m = (size_t)4 * K * sizeof(cplx<float>), l2p = (size_t)K * sizeof(cplx<float>);
    const size_t shift = (size_t)2 * DAG_GROUP_WARPS * 2 * K * sizeof(float);   // xin + red, NW * K2 each
    s = s > rem ? s : rem;
    s = s > p2m ? s : p2m;
    s = s > l2p ? s : l2p;
    s = s > shift ? s : shift;
    return (s + 127) & ~(size_t)127;
}

// One worker group (threads gtid = 0..127 of group `group`): takes tasks until
// the graph is finished or has failed, or, with until_upward, until every
// multipole is final and the high-priority queue is empty.  slot: the group's
// shared word.
template <typename O, int R>
__device__ void dag_worker(const DagArgs& a, int group, int gtid, unsigned char* scratch, int* slot,
                           bool until_upward = false) {
    const int warp = gtid >> 5, lane = gtid & 31, bar = DAG_BAR0 + group;
    const int p = a.p, K = ntri(p), KI2 = ntri(2 * p), KS = kstride(p);
    cplx<float>* M = reinterpret_cast<cplx<float>*>(a.M);
    cplx<float>* L = reinterpret_cast<cplx<float>*>(a.L);
    auto gsync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(DAG_GROUP_THREADS) : "memory"); };
    for (;;) {
        if (gtid == 0) *slot = dag_pop(a, until_upward);
        gsync();
        const int task = *slot;
        gsync();
        if (task < 0) return;
        const int kind = task >> DK_SHIFT, idx = task & (int)DK_MASK;
        if (kind == DK_P2M) {
            const int li = idx * DAG_P2M_GROUP + warp;
            if (li < a.nleaf) {
                const int c = a.leaves[li];
                cplx<float>* acc = reinterpret_cast<cplx<float>*>(scratch) + warp * K;
                p2m_leaf<float>(p, c, lane, a.first, a.count, a.centre, a.xq64, M, acc);
                __syncwarp();
                dag_m_final(a, c, lane);
            }
        } else if (kind == DK_M2M) {
            // warp w translates children w and w + 4; the partial sums meet in scratch
            float* xin = reinterpret_cast<float*>(scratch);
            shift_cell_block<float, R, DAG_GROUP_WARPS, true, GroupSync>(
                p, idx, 0, a.child_first, a.child_count, a.parent, a.ckey, a.shift_ops, M, xin,
                xin + DAG_GROUP_WARPS * 2 * K, warp, gtid, GroupSync{bar});
            gsync();
            if (warp == 0) dag_m_final(a, idx, lane);
        } else if (kind == DK_REM) {
            // warp w: chunk DAG_REM_GROUP idx + w, two half-warp source slots
            const int64_t k = (int64_t)idx * DAG_REM_GROUP + warp;
            if (k < a.nrem_chunk) {
                const int half = lane >> 4, hl = lane & 15;
                cplx<float>* Ms = reinterpret_cast<cplx<float>*>(scratch) + (warp * 2 + half) * (K + KI2);
                cplx<float>* Is = Ms + K;
                const int2 ch = a.rem_chunks[k];
                const int t = ch.x;
                const int64_t s0 = ch.y, s1 = min(a.rem_start[t + 1], s0 + (int64_t)M2L_CHUNK);
                int kk[R], ll[R];
                cplx<float> acc[R];
                m2l_output_index<R>(p, hl, kk, ll);
#pragma unroll
                for (int r = 0; r < R; r++) acc[r] = cmk<float>(0, 0);
                m2l_range<float, R, true>(p, t, s0, s1, half, 2, hl, a.rem_src, a.centre, M, Ms, Is, kk, ll, acc);
#pragma unroll
                for (int r = 0; r < R; r++) {
                    acc[r].re += __shfl_xor_sync(0xffffffffu, acc[r].re, 16);
                    acc[r].im += __shfl_xor_sync(0xffffffffu, acc[r].im, 16);
                }
                if (half == 0) {
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int j = hl + 16 * r;
                        if (j < K) {
                            const float sg = (kk[r] & 1) ? -1.f : 1.f;
                            atomicAdd(a.L + 2 * ((int64_t)t * KS + j), sg * acc[r].re);
                            atomicAdd(a.L + 2 * ((int64_t)t * KS + j) + 1, sg * acc[r].im);
                        }
                    }
                }
            }
        } else if (kind == DK_ROOT) {
            dag_fold(a, idx, gtid);
            __threadfence();
            gsync();
            if (warp == 0) dag_l_final(a, idx, lane);
        } else if (kind == DK_L2L) {
            // fold c's tensor-core results, then warp w shifts a quarter of the parent's coefficients
            dag_fold(a, idx, gtid);
            gsync();
            float* xin = reinterpret_cast<float*>(scratch);
            shift_cell_block<float, R, DAG_GROUP_WARPS, true, GroupSync>(
                p, idx, 1, a.child_first, a.child_count, a.parent, a.ckey, a.shift_ops, L, xin,
                xin + DAG_GROUP_WARPS * 2 * K, warp, gtid, GroupSync{bar});
            __threadfence();
            gsync();
            if (warp == 0) dag_l_final(a, idx, lane);
        } else if (kind == DK_L2P) {
            cplx<float>* Ls = reinterpret_cast<cplx<float>*>(scratch);
            for (int j = gtid; j < K; j += DAG_GROUP_THREADS) Ls[j] = ldc<true>(L + (int64_t)idx * KS + j);
            gsync();
            l2p_particles<float, O, true>(p, idx, gtid, DAG_GROUP_THREADS, Ls, a.first, a.count, a.centre, a.xq64,
                                          a.perm, a.near, (O*)a.phi_out, (O*)a.force_out, a.field);
        } else {   // DK_P2P: leaf rank idx
            float4* buf = reinterpret_cast<float4*>(scratch);
            float(*part)[4] = reinterpret_cast<float(*)[4]>(scratch + P2P_BUF * sizeof(float4));
            p2p_leaf<float, GroupSync>(a.leaves[idx], a.first, a.count, a.p2p_start, a.p2p_rec, a.xq32, a.xlo32, a.icentre,
                                       a.cu2f, a.near, buf, part, gtid, GroupSync{bar});
        }
        // publish the task's writes, then the releases that need the whole group
        __threadfence();
        gsync();
        if (gtid == 0) {
            if (kind == DK_P2P) {
                const int c = a.leaves[idx];
                if (atomicSub(&a.pcnt[c], 1) == 1) dag_push(a, DK_L2P, c);
            } else if (kind == DK_REM) {
                const int64_t k0 = (int64_t)idx * DAG_REM_GROUP;
                const int64_t nk = min((int64_t)DAG_REM_GROUP, a.nrem_chunk - k0);
                dag_m2l_done(a, (unsigned)nk);
            }
            atomicAdd(&a.ctr->done, 1u);
        }
    }
}

}  // namespace fmm
