// dag.cu -- build and launch of the mixed form's task-graph evaluation (the
// device side is dag.cuh and the tensor-core kernel in m2l_tc.cu).
//
// The paper schedules the FMM's stages as a graph of tasks whose data
// dependencies are resolved at run time (Sections 3 and 4).  Here the graph is
// materialised at tree build: a dependency counter per cell (children whose
// multipole is not final; the two prerequisites of a leaf's L2P), the count
// of cells per level (a tensor-core item waits for its source level), the
// initial ready queue (every P2M task), and the number of M2L completions
// that open the downward pass.  An evaluation resets these and runs one
// launch.
#include <algorithm>
#include <vector>

#include "dag.cuh"
#include "fmm_internal.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__global__ void k_dag_init_counters(int ncell, const int32_t* __restrict__ child_count, int32_t* cnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    cnt[c] = child_count[c];                         // children whose multipole is not final
    cnt[ncell + c] = child_count[c] == 0 ? 2 : 0;    // L2P: local final, P2P done
}
__global__ void k_dag_seed(int64_t n_hi, int ngroups, int32_t* q) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_hi) q[i] = i < ngroups ? (int32_t)((DK_P2M << DK_SHIFT) | (int)i) : -1;
}
// queue heads and counters for a new evaluation (a kernel, so that a captured
// evaluation replays it)
__global__ void k_dag_reset(DagCounters* c, unsigned n0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        c->head_hi = 0u; c->tail_hi = n0; c->head_lo = 0u; c->done = 0u; c->avail = (int)n0;
        c->cells_final = 0u; c->m2l_done = 0u; c->released = 0u;
    }
}

int build_dag(fmm_tree* t, cudaStream_t st) {
    TreeDev& d = t->d;
    int rc;
    const int nc = t->ncell;
    if (nc == 0) return FMM_OK;
    const int ngroups = (t->nleaf + DAG_P2M_GROUP - 1) / DAG_P2M_GROUP;
    const int64_t ninternal = nc - t->nleaf;
    t->dag_nrem_tasks = (t->rem_nchunk + DAG_REM_GROUP - 1) / DAG_REM_GROUP;
    // P2M groups, M2M, REM, ROOT (one per system), L2L (every other cell), L2P (leaves)
    t->dag_n_hi = ngroups + ninternal + t->dag_nrem_tasks + t->nsys + (nc - t->nsys) + t->nleaf;
    t->dag_n_tasks = t->dag_n_hi + t->nleaf;   // plus the P2P pool
    t->dag_m2l_total = (int64_t)tc_epilogue_warps() * t->tc_nitems + t->rem_nchunk;
    if ((rc = dev_alloc(&d.dag_cnt_init, (size_t)2 * nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.dag_cnt, (size_t)2 * nc, t, st))) return rc;
    if ((rc = dev_alloc(&d.dag_q_init, (size_t)t->dag_n_hi, t, st))) return rc;
    if ((rc = dev_alloc(&d.dag_q, (size_t)t->dag_n_hi, t, st))) return rc;
    if ((rc = dev_alloc(&d.dag_lvl, (size_t)2 * (FMM_MAX_LEVEL + 1), t, st))) return rc;
    if ((rc = dev_alloc(&d.dag_ctr, sizeof(DagCounters), t, st))) return rc;
    if ((rc = dev_alloc(&d.dag_zero_first, (size_t)t->num_sms + 1, t, st))) return rc;
    FMM_CUDA_TRY(cudaMemsetAsync(d.dag_zero_first, 0, sizeof(int32_t) * ((size_t)t->num_sms + 1), st));
    k_dag_init_counters<<<nblk(nc, 256), 256, 0, st>>>(nc, d.child_count, d.dag_cnt_init);
    k_dag_seed<<<nblk(t->dag_n_hi, 256), 256, 0, st>>>(t->dag_n_hi, ngroups, d.dag_q_init);
    count_launch(t, 2);
    // cells per level (host copy of the level ranges), then zeros for the final counts
    std::vector<int32_t> lv(2 * (FMM_MAX_LEVEL + 1), 0);
    for (int l = 0; l < t->nlevel && l <= FMM_MAX_LEVEL; l++) lv[l] = t->level_start[l + 1] - t->level_start[l];
    FMM_CUDA_TRY(cudaMemcpyAsync(d.dag_lvl, lv.data(), sizeof(int32_t) * lv.size(), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));   // lv leaves scope
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

template <typename O>
int evaluate_dag(fmm_tree* t, const double4_32a* xq64, const float4* xq32, const float4* xlo32, O* phi, O* force,
                 cudaStream_t st) {
    TreeDev& d = t->d;
    const int nc = t->ncell, p = t->prm.p;
    if (nc == 0) return FMM_OK;
    const int ngroups = (t->nleaf + DAG_P2M_GROUP - 1) / DAG_P2M_GROUP;
    FMM_CUDA_TRY(cudaMemcpyAsync(d.dag_cnt, d.dag_cnt_init, sizeof(int32_t) * 2 * (size_t)nc, cudaMemcpyDeviceToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(d.dag_q, d.dag_q_init, sizeof(int32_t) * (size_t)t->dag_n_hi, cudaMemcpyDeviceToDevice, st));
    FMM_CUDA_TRY(cudaMemsetAsync(d.dag_lvl + FMM_MAX_LEVEL + 1, 0, sizeof(int32_t) * (FMM_MAX_LEVEL + 1), st));
    FMM_CUDA_TRY(cudaMemsetAsync(d.L, 0, sizeof(cplx<float>) * (size_t)nc * kstride(p), st));
    k_dag_reset<<<1, 32, 0, st>>>((DagCounters*)d.dag_ctr, (unsigned)ngroups);
    count_launch(t);
    DagArgs g{};
    g.p = p; g.ncell = nc; g.nleaf = t->nleaf; g.nsys = t->nsys;
    g.field = (t->prm.flags & FMM_OUT_FIELD) ? 1 : 0;
    g.KR = (p + 1) * (p + 1); g.KI = tc_kin(p); g.R = ntri(p) <= 48 ? 3 : 6;
    g.n_hi = (unsigned)t->dag_n_hi; g.n_lo = (unsigned)t->nleaf; g.n_tasks = (unsigned)t->dag_n_tasks;
    g.m2l_total = (unsigned)t->dag_m2l_total;
    g.nrem_tasks = (int)t->dag_nrem_tasks; g.nrem_chunk = t->rem_nchunk;
    g.budget_cycles = (long long)(t->prm.timeout_ns * 2);   // clock64 runs near 2 GHz
    g.leaves = d.leaves; g.first = d.first; g.count = d.count; g.parent = d.parent;
    g.child_first = d.child_first; g.child_count = d.child_count; g.level = d.level; g.ckey = d.ckey;
    g.centre = d.centre; g.icentre = d.icentre; g.perm = d.perm; g.shift_ops = (const float*)d.shift_ops;
    g.xq64 = xq64; g.xq32 = xq32; g.xlo32 = xlo32; g.p2p_start = d.p2p_start; g.p2p_rec = d.p2p_rec; g.cu2f = d.cu2f;
    g.rem_chunks = d.rem_chunks; g.rem_start = d.rem_start; g.rem_src = d.tc_src + t->tc_npairs;
    g.M = (float*)d.M; g.L = (float*)d.L; g.Lr = (const float*)d.tc_lr; g.Ms = (__nv_bfloat16*)d.tc_msplit;
    g.near = d.near; g.phi_out = phi; g.force_out = force;
    g.q = d.dag_q; g.mcnt = d.dag_cnt; g.pcnt = d.dag_cnt + nc;
    g.lvl_count = d.dag_lvl; g.lvl_done = d.dag_lvl + FMM_MAX_LEVEL + 1;
    g.ctr = (DagCounters*)d.dag_ctr; g.status = d.status;
    stage_begin(t, FMM_STAGE_QUEUE, st);
    const int rc = launch_m2l_dag<O>(t, g, st);
    stage_end(t, FMM_STAGE_QUEUE, st);
    return rc;
}

template int evaluate_dag<float>(fmm_tree*, const double4_32a*, const float4*, const float4*, float*, float*,
                                  cudaStream_t);
template int evaluate_dag<double>(fmm_tree*, const double4_32a*, const float4*, const float4*, double*, double*,
                                   cudaStream_t);

}  // namespace fmm
