// queue.cu -- the evaluation as one persistent kernel over a task graph.
//
// This replaces the paper's QUARK runtime (Sections 3 and 4): instead of
// worker threads taking tasks whose data dependencies (read-after-write on
// cells) have been resolved, resident thread blocks take tasks from a device
// ready queue, and a task is queued by whichever block completes its last
// dependency.  Interaction is non-mutual (Section 4): every task writes only
// its own target cell or leaf, so no two tasks write the same data and no
// floating-point atomics are needed.
//
// Tasks and their dependencies (one counter per task kind and cell):
//   P2M(group of 4 leaves)  none
//   M2M(c)                  M final for each child of c          (mcnt = #children)
//   M2L(c)                  M final for each source of c's list  (lcnt = #sources)
//   L2L(c), c != root       M2L(c) done, L final for c's parent  (dcnt = 2)
//   P2P(leaf)               none
//   L2P(leaf)               L final for the leaf, P2P(leaf) done (pcnt = 2)
// "M final" for c is the end of P2M(c) or M2M(c); "L final" for c is the end
// of L2L(c) (of M2L(root) for the root).  The successors of "M final(s)" for
// M2L are the targets whose list holds s (the transposed M2L list).
//
// Queues: P2P tasks have no dependencies and are the bulk of the work, so they
// sit in a static low-priority pool; every other task goes through a
// high-priority FIFO that a block drains first.  Each task is queued exactly
// once, so the FIFO never wraps.  Every wait (a reserved slot not yet
// written, an empty queue before the end) is bounded by the tree's timeout; on
// expiry the block records FMM_ERR_TIMEOUT in the status word and returns.
#include <cub/cub.cuh>

#include <algorithm>

#include "fmm_internal.cuh"
#include "stages.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

enum TaskKind { TK_P2M = 0, TK_M2M = 1, TK_M2L = 2, TK_L2L = 3, TK_L2P = 4, TK_P2P = 5 };
constexpr int TK_SHIFT = 28;
constexpr unsigned TK_MASK = (1u << TK_SHIFT) - 1u;
constexpr int QUEUE_THREADS = 128;
constexpr int P2M_GROUP = 4;
constexpr int M2L_SLOTS = 2 * QUEUE_THREADS / 32;

struct QueueCounters {
    unsigned head_hi, tail_hi, head_lo, done;
    int avail;   // tasks pushed (slot written) and not yet claimed
};

struct QueueArgs {
    int p, ncell, nleaf, field;
    unsigned n_hi, n_lo, n_tasks;
    long long budget_cycles;
    const float* cu2f;
    const int32_t* leaves;
    const int32_t* first;
    const int32_t* count;
    const int32_t* parent;
    const int32_t* child_first;
    const int32_t* child_count;
    const uint64_t* ckey;
    const double4_32a* centre;
    const int4* icentre;
    const int32_t* perm;
    const int64_t* m2l_start;
    const int32_t* m2l_src;
    const int64_t* p2p_start;
    const int4* p2p_rec;
    const int64_t* tr_start;
    const int32_t* tr_tgt;
    const void* shift_ops;
    const double4_32a* xq64;
    const void* xqp;        // P2P records (double4 or float4)
    const float4* xlo;      // FP32 P2P: residuals of the coordinates (null for FP64)
    void* M;
    void* L;
    double* near;
    void* phi_out;
    void* force_out;
    int* q;                 // high-priority FIFO [n_hi]
    int* mcnt;
    int* lcnt;
    int* dcnt;
    int* pcnt;
    QueueCounters* ctr;
    int* status;
};

__device__ __forceinline__ unsigned vload(const unsigned* p) { return *(volatile const unsigned*)p; }
__device__ __forceinline__ int vload(const int* p) { return *(volatile const int*)p; }

// Push: reserve a slot, write it, then count it as available.  Pop: claim one
// available task (a semaphore decrement that never retries), then take the next
// ticket; the ticket's slot has been reserved by a push that is at most a few
// instructions from writing it, so that wait is short.  A claim that finds
// nothing available is undone and the block takes a P2P task instead.
__device__ __forceinline__ void push(const QueueArgs& a, int kind, int idx) {
    unsigned slot = atomicAdd(&a.ctr->tail_hi, 1u);
    if (slot >= a.n_hi) return;
    atomicExch(&a.q[slot], (kind << TK_SHIFT) | idx);
    __threadfence();
    atomicAdd(&a.ctr->avail, 1);
}

// thread 0: next task, or -1 when the graph is finished (or on an error)
__device__ int pop(const QueueArgs& a) {
    long long t0 = clock64();
    for (;;) {
        if (vload(&a.ctr->avail) > 0) {
            if (atomicSub(&a.ctr->avail, 1) > 0) {
                const unsigned h = atomicAdd(&a.ctr->head_hi, 1u);
                long long t1 = clock64();
                int v;
                while ((v = vload(&a.q[h])) < 0) {
                    if (clock64() - t1 > a.budget_cycles) { atomicExch(a.status, 1); return -1; }
                    __nanosleep(32);
                }
                __threadfence();
                return v;
            }
            atomicAdd(&a.ctr->avail, 1);
        }
        if (vload(&a.ctr->head_lo) < a.n_lo) {
            unsigned l = atomicAdd(&a.ctr->head_lo, 1u);
            if (l < a.n_lo) return (TK_P2P << TK_SHIFT) | (int)l;
        }
        if (vload(&a.ctr->done) >= a.n_tasks || vload(a.status) != 0) return -1;
        if (clock64() - t0 > a.budget_cycles) { atomicExch(a.status, 1); return -1; }
        __nanosleep(64);
    }
}

// warp 0: successors of "M final" for cell c
__device__ void on_m_final(const QueueArgs& a, int c, int lane) {
    if (lane == 0) {
        int par = a.parent[c];
        if (par >= 0 && atomicSub(&a.mcnt[par], 1) == 1) push(a, TK_M2M, par);
    }
    for (int64_t k = a.tr_start[c] + lane; k < a.tr_start[c + 1]; k += 32) {
        int t = a.tr_tgt[k];
        if (atomicSub(&a.lcnt[t], 1) == 1) push(a, TK_M2L, t);
    }
}

// warp 0: successors of "L final" for cell c
__device__ void on_l_final(const QueueArgs& a, int c, int lane) {
    int nc = a.child_count[c];
    if (nc == 0) {
        if (lane == 0 && atomicSub(&a.pcnt[c], 1) == 1) push(a, TK_L2P, c);
        return;
    }
    int cf = a.child_first[c];
    for (int k = lane; k < nc; k += 32)
        if (atomicSub(&a.dcnt[cf + k], 1) == 1) push(a, TK_L2L, cf + k);
}

template <typename T, typename TP, typename O, int R>
__global__ void __launch_bounds__(QUEUE_THREADS) k_queue(QueueArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_task;
    typedef typename Vec4<TP>::type VP;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p = a.p, K = ntri(p), KI = ntri(2 * p), KS = kstride(p);
    cplx<T>* M = (cplx<T>*)a.M;
    cplx<T>* L = (cplx<T>*)a.L;
    for (;;) {
        if (tid == 0) s_task = pop(a);
        __syncthreads();
        const int task = s_task;
        if (task < 0) return;
        const int kind = task >> TK_SHIFT, idx = task & (int)TK_MASK;
        if (kind == TK_P2M) {
            const int li = idx * P2M_GROUP + warp;
            cplx<T>* acc = reinterpret_cast<cplx<T>*>(sm) + warp * K;
            if (warp < P2M_GROUP && li < a.nleaf)
                p2m_leaf<T>(p, a.leaves[li], lane, a.first, a.count, a.centre, a.xq64, M, acc);
        } else if (kind == TK_M2M || kind == TK_L2L) {
            if (warp == 0)
                shift_cell<T, R, true>(p, idx, kind == TK_M2M ? 0 : 1, lane, a.child_first, a.child_count, a.parent,
                                       a.ckey, (const T*)a.shift_ops, kind == TK_M2M ? M : L,
                                       reinterpret_cast<T*>(sm));
        } else if (kind == TK_M2L) {
            const int slot = warp * 2 + (lane >> 4), hl = lane & 15;
            cplx<T>* Ms = reinterpret_cast<cplx<T>*>(sm) + slot * (K + KI);
            int kk[R], ll[R];
            cplx<T> acc[R];
            m2l_output_index<R>(p, hl, kk, ll);
#pragma unroll
            for (int r = 0; r < R; r++) acc[r] = cmk<T>(0, 0);
            m2l_slot<T, R, true>(p, idx, slot, M2L_SLOTS, hl, a.m2l_start, a.m2l_src, a.centre, M, Ms, Ms + K, kk,
                                 ll, acc);
            __syncthreads();
            cplx<T>* red = reinterpret_cast<cplx<T>*>(sm);
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int j = hl + 16 * r;
                if (j < K) red[slot * K + j] = acc[r];
            }
            __syncthreads();
            for (int j = tid; j < K; j += QUEUE_THREADS) {
                cplx<T> s = cmk<T>(0, 0);
                for (int q = 0; q < M2L_SLOTS; q++) s = cadd(s, red[q * K + j]);
                int n = 0;
                while (tri(n + 1, 0) <= j) n++;
                L[(int64_t)idx * KS + j] = cscale(s, (n & 1) ? T(-1) : T(1));
            }
        } else if (kind == TK_L2P) {
            cplx<T>* Ls = reinterpret_cast<cplx<T>*>(sm);
            for (int j = tid; j < K; j += QUEUE_THREADS) Ls[j] = ldc<true>(L + (int64_t)idx * KS + j);
            __syncthreads();
            l2p_particles<T, O, true>(p, idx, tid, QUEUE_THREADS, Ls, a.first, a.count, a.centre, a.xq64, a.perm,
                                      a.near, (O*)a.phi_out, (O*)a.force_out, a.field);
        } else {  // TK_P2P
            VP* buf = reinterpret_cast<VP*>(sm);
            TP(*part)[4] = reinterpret_cast<TP(*)[4]>(sm + P2P_BUF * sizeof(VP));
            p2p_leaf<TP>(a.leaves[idx], a.first, a.count, a.p2p_start, a.p2p_rec, (const VP*)a.xqp,
                         sizeof(TP) == 4 ? a.xlo : nullptr, a.icentre, a.cu2f, a.near, buf, part, tid);
        }
        // publish this task's writes, then release its successors
        __threadfence();
        __syncthreads();
        if (warp == 0) {
            if (kind == TK_P2M) {
                for (int w = 0; w < P2M_GROUP; w++) {
                    const int li = idx * P2M_GROUP + w;
                    if (li < a.nleaf) on_m_final(a, a.leaves[li], lane);
                }
            } else if (kind == TK_M2M) {
                on_m_final(a, idx, lane);
            } else if (kind == TK_M2L) {
                if (a.parent[idx] < 0) on_l_final(a, idx, lane);   // a root: its local is final
                else if (lane == 0 && atomicSub(&a.dcnt[idx], 1) == 1) push(a, TK_L2L, idx);
            } else if (kind == TK_L2L) {
                on_l_final(a, idx, lane);
            } else if (kind == TK_P2P) {
                const int c = a.leaves[idx];
                if (lane == 0 && atomicSub(&a.pcnt[c], 1) == 1) push(a, TK_L2P, c);
            }
            __threadfence();
            if (lane == 0) atomicAdd(&a.ctr->done, 1u);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// build: transposed M2L list, initial counters, initial queue
// ---------------------------------------------------------------------------

__global__ void k_src_hist(int64_t np, const int32_t* src, int32_t* hist) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < np) atomicAdd(&hist[src[e]], 1);
}
__global__ void k_transpose_scatter(int ncell, const int64_t* start, const int32_t* src, const int64_t* tr_start,
                                    int32_t* fill, int32_t* tr_tgt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    for (int64_t e = start[t]; e < start[t + 1]; e++) {
        int s = src[e];
        int k = atomicAdd(&fill[s], 1);
        tr_tgt[tr_start[s] + k] = t;
    }
}
__global__ void k_queue_init_counters(int ncell, const int32_t* child_count, const int32_t* parent,
                                      const int64_t* m2l_start, int32_t* cnt, char* empty_m2l) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int nl = (int)(m2l_start[c + 1] - m2l_start[c]);
    cnt[c] = child_count[c];                     // mcnt
    cnt[ncell + c] = nl;                         // lcnt
    cnt[2 * ncell + c] = parent[c] < 0 ? 0 : 2;  // dcnt (roots have no L2L)
    cnt[3 * ncell + c] = child_count[c] == 0 ? 2 : 0;  // pcnt
    empty_m2l[c] = nl == 0;
}
__global__ void k_queue_seed(int ngroups, int nempty, const int32_t* empty_cells, int32_t* q) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ngroups) q[i] = (TK_P2M << TK_SHIFT) | i;
    else if (i < ngroups + nempty) q[i] = (TK_M2L << TK_SHIFT) | empty_cells[i - ngroups];
}
// queue heads and tails for a new evaluation (a kernel, so that an evaluation
// captured in a CUDA graph replays it)
__global__ void k_queue_reset(QueueCounters* c, unsigned n0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->head_hi = 0u; c->tail_hi = n0; c->head_lo = 0u; c->done = 0u; c->avail = (int)n0;
    }
}

__global__ void k_iota(int n, int32_t* v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

bool queue_supported(const fmm_tree* t) {
    return !(t->prm.flags & FMM_STAGED) && t->prm.precision != FMM_PREC_MIXED_TC && ntri(t->prm.p) <= 96 &&
           !p2p_mutual(t);
}

int build_queue(fmm_tree* t, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    const int nc = t->ncell;
    if (nc == 0) return FMM_OK;
    // transposed M2L list: source -> targets
    int32_t *hist = nullptr, *fill = nullptr;
    if ((rc = dev_alloc(&hist, (size_t)nc, nullptr, st))) return rc;
    if ((rc = dev_alloc(&fill, (size_t)nc, nullptr, st))) return rc;
    if ((rc = dev_alloc(&d.tr_start, (size_t)nc + 1, t, st))) return rc;
    if ((rc = dev_alloc(&d.tr_tgt, (size_t)std::max<int64_t>(1, t->nm2l), t, st))) return rc;
    FMM_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)nc * 4, st));
    FMM_CUDA_TRY(cudaMemsetAsync(fill, 0, (size_t)nc * 4, st));
    FMM_CUDA_TRY(cudaMemsetAsync(d.tr_start, 0, 8, st));
    if (t->nm2l) k_src_hist<<<nblk(t->nm2l, 256), 256, 0, st>>>(t->nm2l, d.m2l_src, hist);
    int64_t* hist64 = nullptr;
    if ((rc = dev_alloc(&hist64, (size_t)nc, nullptr, st))) return rc;
    // widen to int64 and scan into tr_start[1..]
    {
        size_t sb = 0;
        cub::DeviceScan::InclusiveSum(nullptr, sb, hist, d.tr_start + 1, nc, st);
        char* tmp = nullptr;
        if ((rc = dev_alloc(&tmp, sb, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceScan::InclusiveSum(tmp, sb, hist, d.tr_start + 1, nc, st));
        cudaFreeAsync(tmp, st);
    }
    k_transpose_scatter<<<nblk(nc, 128), 128, 0, st>>>(nc, d.m2l_start, d.m2l_src, d.tr_start, fill, d.tr_tgt);
    // initial counters and queue
    if ((rc = dev_alloc(&d.q_cnt_init, (size_t)4 * nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.q_cnt, (size_t)4 * nc, t, st))) return rc;
    char* empty = nullptr;
    int32_t *cells = nullptr, *empty_cells = nullptr, *nsel = nullptr;
    if ((rc = dev_alloc(&empty, (size_t)nc, nullptr, st))) return rc;
    if ((rc = dev_alloc(&cells, (size_t)nc, nullptr, st))) return rc;
    if ((rc = dev_alloc(&empty_cells, (size_t)nc, nullptr, st))) return rc;
    if ((rc = dev_alloc(&nsel, 1, nullptr, st))) return rc;
    k_queue_init_counters<<<nblk(nc, 256), 256, 0, st>>>(nc, d.child_count, d.parent, d.m2l_start, d.q_cnt_init,
                                                          empty);
    k_iota<<<nblk(nc, 256), 256, 0, st>>>(nc, cells);
    {
        size_t sb = 0;
        cub::DeviceSelect::Flagged(nullptr, sb, cells, empty, empty_cells, nsel, nc, st);
        char* tmp = nullptr;
        if ((rc = dev_alloc(&tmp, sb, nullptr, st))) return rc;
        FMM_CUDA_TRY(cub::DeviceSelect::Flagged(tmp, sb, cells, empty, empty_cells, nsel, nc, st));
        cudaFreeAsync(tmp, st);
    }
    int32_t nempty = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&nempty, nsel, 4, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    const int ngroups = (t->nleaf + P2M_GROUP - 1) / P2M_GROUP;
    const int ninternal = nc - t->nleaf;
    t->q_n_hi = (int64_t)ngroups + ninternal + nc + (nc - t->nsys) + t->nleaf;   // L2L for every non-root cell
    t->q_n0 = ngroups + nempty;
    t->q_n_tasks = t->q_n_hi + t->nleaf;
    if ((rc = dev_alloc(&d.q_init, (size_t)t->q_n_hi, t, st))) return rc;
    if ((rc = dev_alloc(&d.q_work, (size_t)t->q_n_hi, t, st))) return rc;
    FMM_CUDA_TRY(cudaMemsetAsync(d.q_init, 0xff, (size_t)t->q_n_hi * 4, st));
    k_queue_seed<<<nblk(t->q_n0, 256), 256, 0, st>>>(ngroups, nempty, empty_cells, d.q_init);
    if ((rc = dev_alloc(&d.q_ctr, sizeof(QueueCounters), t, st))) return rc;
    count_launch(t, 9);
    FMM_CUDA_TRY(cudaGetLastError());
    cudaFreeAsync(hist, st); cudaFreeAsync(fill, st); cudaFreeAsync(hist64, st); cudaFreeAsync(empty, st);
    cudaFreeAsync(cells, st); cudaFreeAsync(empty_cells, st); cudaFreeAsync(nsel, st);
    return FMM_OK;
}

template <typename T, typename TP, typename O, int R>
static int launch_queue(fmm_tree* t, QueueArgs& a, size_t smem, cudaStream_t st) {
    auto kern = k_queue<T, TP, O, R>;
    FMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, QUEUE_THREADS, smem));
    if (per_sm < 1) { fmm_set_error("task-queue kernel does not fit on an SM"); return FMM_ERR_ARG; }
    // every block resident: a block only ever waits for work queued by a running block
    int grid = per_sm * t->num_sms;
    kern<<<grid, QUEUE_THREADS, smem, st>>>(a);
    count_launch(t);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

template <typename T, typename TP, typename O>
int evaluate_queue(fmm_tree* t, const double4_32a* xq64, const void* xqp, O* phi, O* force, cudaStream_t st,
                   const float4* xlo) {
    TreeDev& d = t->d;
    const int p = t->prm.p, K = ntri(p), KI = ntri(2 * p);
    const int nc = t->ncell;
    FMM_CUDA_TRY(cudaMemcpyAsync(d.q_cnt, d.q_cnt_init, (size_t)4 * nc * 4, cudaMemcpyDeviceToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(d.q_work, d.q_init, (size_t)t->q_n_hi * 4, cudaMemcpyDeviceToDevice, st));
    k_queue_reset<<<1, 32, 0, st>>>((QueueCounters*)d.q_ctr, (unsigned)t->q_n0);
    count_launch(t);
    QueueArgs a;
    a.p = p; a.ncell = nc; a.nleaf = t->nleaf; a.field = (t->prm.flags & FMM_OUT_FIELD) ? 1 : 0;
    a.n_hi = (unsigned)t->q_n_hi; a.n_lo = (unsigned)t->nleaf; a.n_tasks = (unsigned)t->q_n_tasks;
    a.budget_cycles = (long long)(t->prm.timeout_ns * 2);  // clock64 runs near 2 GHz
    a.cu2f = d.cu2f;
    a.leaves = d.leaves; a.first = d.first; a.count = d.count; a.parent = d.parent;
    a.child_first = d.child_first; a.child_count = d.child_count; a.ckey = d.ckey; a.centre = d.centre;
    a.icentre = d.icentre; a.perm = d.perm; a.m2l_start = d.m2l_start; a.m2l_src = d.m2l_src;
    a.p2p_start = d.p2p_start; a.p2p_rec = d.p2p_rec; a.tr_start = d.tr_start; a.tr_tgt = d.tr_tgt;
    a.shift_ops = d.shift_ops; a.xq64 = xq64; a.xqp = xqp; a.xlo = xlo; a.M = d.M; a.L = d.L; a.near = d.near;
    a.phi_out = phi; a.force_out = force; a.q = d.q_work;
    a.mcnt = d.q_cnt; a.lcnt = d.q_cnt + nc; a.dcnt = d.q_cnt + 2 * nc; a.pcnt = d.q_cnt + 3 * nc;
    a.ctr = (QueueCounters*)d.q_ctr; a.status = d.status;
    size_t smem = 0;
    smem = std::max(smem, (size_t)P2M_GROUP * K * sizeof(cplx<T>));
    smem = std::max(smem, (size_t)2 * K * sizeof(T));
    smem = std::max(smem, (size_t)M2L_SLOTS * (K + KI) * sizeof(cplx<T>));
    smem = std::max(smem, (size_t)P2P_BUF * sizeof(typename Vec4<TP>::type) + (size_t)QUEUE_THREADS * 4 * sizeof(TP));
    const int r = (K + 15) / 16;
    stage_begin(t, FMM_STAGE_QUEUE, st);
    int rc;
    if (r <= 3) rc = launch_queue<T, TP, O, 3>(t, a, smem, st);
    else rc = launch_queue<T, TP, O, 6>(t, a, smem, st);
    stage_end(t, FMM_STAGE_QUEUE, st);
    return rc;
}

template int evaluate_queue<double, double, double>(fmm_tree*, const double4_32a*, const void*, double*, double*,
                                                    cudaStream_t, const float4*);
template int evaluate_queue<double, double, float>(fmm_tree*, const double4_32a*, const void*, float*, float*,
                                                   cudaStream_t, const float4*);
template int evaluate_queue<double, float, double>(fmm_tree*, const double4_32a*, const void*, double*, double*,
                                                   cudaStream_t, const float4*);
template int evaluate_queue<double, float, float>(fmm_tree*, const double4_32a*, const void*, float*, float*,
                                                  cudaStream_t, const float4*);
template int evaluate_queue<float, float, double>(fmm_tree*, const double4_32a*, const void*, double*, double*,
                                                  cudaStream_t, const float4*);
template int evaluate_queue<float, float, float>(fmm_tree*, const double4_32a*, const void*, float*, float*,
                                                 cudaStream_t, const float4*);

}  // namespace fmm
