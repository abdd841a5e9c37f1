// capi.cu -- the extern "C" boundary: argument checks, tree lifetime, export.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "fmm_internal.cuh"

static thread_local char g_err[512] = "";

void fmm_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

namespace {

int check_params(const fmm_params* prm) {
    if (!prm) { fmm_set_error("params is NULL"); return FMM_ERR_ARG; }
    if (prm->p < 0 || prm->p > FMM_MAX_P) { fmm_set_error("p=%d outside [0, %d]", prm->p, FMM_MAX_P); return FMM_ERR_ARG; }
    if (prm->leaf_size < 1 || prm->leaf_size > 4096) {
        fmm_set_error("leaf_size=%d outside [1, 4096]", prm->leaf_size);
        return FMM_ERR_ARG;
    }
    if (!(prm->theta > 0.0 && prm->theta < 1.0)) { fmm_set_error("theta=%g outside (0, 1)", prm->theta); return FMM_ERR_ARG; }
    if (prm->precision < FMM_PREC_FP64 || prm->precision > FMM_PREC_MIXED_TC) {
        fmm_set_error("unknown precision %d", prm->precision);
        return FMM_ERR_ARG;
    }
    if (prm->flags & ~(FMM_OUT_FIELD | FMM_STAGED | FMM_TIMING | FMM_NO_OVERLAP | FMM_BUILD_FALLBACKS | FMM_TASK_GRAPH | FMM_MUTUAL | FMM_LISTS_UVWX)) { fmm_set_error("unknown flags 0x%x", prm->flags); return FMM_ERR_ARG; }
    if (prm->timeout_ns < 0) { fmm_set_error("timeout_ns < 0"); return FMM_ERR_ARG; }
    if (prm->p2p_item_records != 0 && (prm->p2p_item_records < 8 || prm->p2p_item_records > 65536)) {
        fmm_set_error("p2p_item_records=%d outside {0} and [8, 65536]", prm->p2p_item_records);
        return FMM_ERR_ARG;
    }
    if (prm->tc_min_pairs != 0 && (prm->tc_min_pairs < 1 || prm->tc_min_pairs > 4096)) {
        fmm_set_error("tc_min_pairs=%d outside {0} and [1, 4096]", prm->tc_min_pairs);
        return FMM_ERR_ARG;
    }
    return FMM_OK;
}

void setup_pool_once() {
    static bool done = false;
    if (done) return;
    done = true;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;  // keep freed blocks for reuse by this process
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

}  // namespace

namespace fmm {
// Pinned host words, PIN_WORDS per live tree, from one arena allocated on first
// use: the build copies a few device-computed sizes into its tree's slot
// asynchronously, so that the evaluation knows them without a host round trip.
namespace {
constexpr int PIN_SLOTS = 4096;
std::mutex g_pin_mu;
int32_t* g_pin = nullptr;
bool g_pin_failed = false;
std::vector<int> g_pin_free;
}  // namespace

int32_t* pinned_slot_acquire() {
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (!g_pin && !g_pin_failed) {
        if (cudaMallocHost(&g_pin, sizeof(int32_t) * PIN_WORDS * PIN_SLOTS) != cudaSuccess) {
            cudaGetLastError();
            g_pin = nullptr;
            g_pin_failed = true;
        } else {
            for (int i = PIN_SLOTS - 1; i >= 0; i--) g_pin_free.push_back(i);
        }
    }
    if (!g_pin || g_pin_free.empty()) return nullptr;
    const int i = g_pin_free.back();
    g_pin_free.pop_back();
    int32_t* w = g_pin + (size_t)i * PIN_WORDS;
    for (int k = 0; k < PIN_WORDS; k++) w[k] = -1;   // not written by a build yet
    return w;
}

void pinned_slot_release(int32_t* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pin_free.push_back((int)((p - g_pin) / PIN_WORDS));
}
}  // namespace fmm

extern "C" {

const char* fmm_last_error(void) { return g_err; }

const char* fmm_version(void) { return "paper_1203_0889_gb300 0.1 (sm_103a)"; }

static int build_common(const fmm_params* params, int64_t n, const void* pos, int pos_dtype, fmm_tree** out,
                        void* stream, const std::vector<int64_t>* offsets);

int fmm_build_tree(const fmm_params* params, int64_t n, const void* pos, int pos_dtype, fmm_tree** out,
                   void* stream) {
    return build_common(params, n, pos, pos_dtype, out, stream, nullptr);
}

static int build_common(const fmm_params* params, int64_t n, const void* pos, int pos_dtype, fmm_tree** out,
                        void* stream, const std::vector<int64_t>* offsets) {
    g_err[0] = 0;
    if (!out) { fmm_set_error("out is NULL"); return FMM_ERR_ARG; }
    *out = nullptr;
    int rc = check_params(params);
    if (rc) return rc;
    if (n < 0 || n >= ((int64_t)1 << 31)) { fmm_set_error("n=%lld outside [0, 2^31)", (long long)n); return FMM_ERR_ARG; }
    if (n > 0 && !pos) { fmm_set_error("pos is NULL"); return FMM_ERR_ARG; }
    if (pos_dtype != FMM_F64 && pos_dtype != FMM_F32) { fmm_set_error("pos_dtype must be FMM_F64 or FMM_F32"); return FMM_ERR_ARG; }
    setup_pool_once();
    fmm_tree* t = new (std::nothrow) fmm_tree();
    if (!t) { fmm_set_error("host allocation failed"); return FMM_ERR_ALLOC; }
    t->h_pin = fmm::pinned_slot_acquire();
    if (offsets) t->h_sys_off = *offsets;
    t->prm = *params;
    if (t->prm.timeout_ns == 0) t->prm.timeout_ns = 2000000000LL;
    if (t->prm.p2p_item_records == 0) t->prm.p2p_item_records = fmm::P2P_ITEM_RECORDS;
    if (t->prm.tc_min_pairs == 0) t->prm.tc_min_pairs = fmm::TC_MIN_PAIRS;
    t->n = n;
    if (t->h_sys_off.empty()) t->h_sys_off = {0, n};
    t->nsys = (int)t->h_sys_off.size() - 1;
    cudaStream_t st = (cudaStream_t)stream;
    if (t->prm.flags & FMM_TIMING) {
        t->timing = true;
        for (int i = 0; i < 2 * FMM_NUM_STAGES; i++) {
            cudaError_t e = cudaEventCreate(&t->ev[i]);
            if (e != cudaSuccess) {
                fmm_set_error("cudaEventCreate: %s", cudaGetErrorString(e));
                for (int k = 0; k < i; k++) cudaEventDestroy(t->ev[k]);
                fmm::pinned_slot_release(t->h_pin);
                delete t;
                return FMM_ERR_CUDA;
            }
        }
    }
    t->launch_ctr = &t->launches_build;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (t->n > 0 && (!fmm::queue_supported(t))) {
        // the stage-by-stage path runs P2P (and, at build time, the tensor-core
        // class operators) on a second stream, non-blocking with respect to the
        // legacy stream and joined by events
        if (cudaStreamCreateWithFlags(&t->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&t->ev_ops, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (t->side_stream) cudaStreamDestroy(t->side_stream);
            if (t->ev_fork) cudaEventDestroy(t->ev_fork);
            if (t->ev_join) cudaEventDestroy(t->ev_join);
            t->side_stream = nullptr; t->ev_fork = nullptr; t->ev_join = nullptr; t->ev_ops = nullptr;
        }
        int least = 0, greatest = 0;
        // the mixed form's third stream: the class operators at build time, the
        // CUDA-core M2L pairs beside the tensor-core kernel at evaluation time
        // (on the far field's critical path, hence the high priority)
        if (t->side_stream && t->prm.precision == FMM_PREC_MIXED_TC &&
            (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
             cudaStreamCreateWithPriority(&t->ops_stream, cudaStreamNonBlocking, greatest) != cudaSuccess ||
             cudaEventCreateWithFlags(&t->ev_rem_fork, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&t->ev_rem_join, cudaEventDisableTiming) != cudaSuccess)) {
            cudaGetLastError();
            if (t->ops_stream) cudaStreamDestroy(t->ops_stream);
            if (t->ev_rem_fork) cudaEventDestroy(t->ev_rem_fork);
            if (t->ev_rem_join) cudaEventDestroy(t->ev_rem_join);
            t->ops_stream = nullptr; t->ev_rem_fork = nullptr; t->ev_rem_join = nullptr;
        }
        if (t->side_stream && (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
                               cudaStreamCreateWithPriority(&t->hi_stream, cudaStreamNonBlocking, greatest) !=
                                   cudaSuccess ||
                               cudaEventCreateWithFlags(&t->ev_join_hi, cudaEventDisableTiming) != cudaSuccess)) {
            cudaGetLastError();
            if (t->hi_stream) cudaStreamDestroy(t->hi_stream);
            t->hi_stream = nullptr; t->ev_join_hi = nullptr;
        }
    }
    rc = fmm::build_tree_impl(t, pos, pos_dtype, st);
    if (!rc) rc = fmm::alloc_eval_workspace(t, st);
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { fmm_set_error("build: %s", cudaGetErrorString(e)); rc = FMM_ERR_CUDA; }
    }
    if (rc) {
        cudaStreamSynchronize(st);
        if (t->side_stream) cudaStreamSynchronize(t->side_stream);
        if (t->hi_stream) cudaStreamSynchronize(t->hi_stream);
        if (t->ops_stream) cudaStreamSynchronize(t->ops_stream);
        fmm::free_tree_device(t);
        if (t->timing) for (int i = 0; i < 2 * FMM_NUM_STAGES; i++) cudaEventDestroy(t->ev[i]);
        if (t->side_stream) cudaStreamDestroy(t->side_stream);
        if (t->hi_stream) cudaStreamDestroy(t->hi_stream);
        if (t->ops_stream) cudaStreamDestroy(t->ops_stream);
        if (t->ev_fork) cudaEventDestroy(t->ev_fork);
        if (t->ev_join) cudaEventDestroy(t->ev_join);
        if (t->ev_join_hi) cudaEventDestroy(t->ev_join_hi);
        if (t->ev_ops) cudaEventDestroy(t->ev_ops);
        if (t->ev_rem_fork) cudaEventDestroy(t->ev_rem_fork);
        if (t->ev_rem_join) cudaEventDestroy(t->ev_rem_join);
        fmm::pinned_slot_release(t->h_pin);
        delete t;
        return rc;
    }
    t->launch_ctr = nullptr;
    *out = t;
    return FMM_OK;
}

int fmm_evaluate(fmm_tree* tree, const void* q, void* phi, void* force, int dtype, void* stream) {
    g_err[0] = 0;
    if (!tree) { fmm_set_error("tree is NULL"); return FMM_ERR_ARG; }
    if (dtype != FMM_F64 && dtype != FMM_F32) { fmm_set_error("dtype must be FMM_F64 or FMM_F32"); return FMM_ERR_ARG; }
    if (tree->n > 0 && !q) { fmm_set_error("q is NULL"); return FMM_ERR_ARG; }
    tree->launches_eval = 0;
    tree->launch_ctr = &tree->launches_eval;
    if (tree->d.status) {
        cudaError_t e = cudaMemsetAsync(tree->d.status, 0, sizeof(int), (cudaStream_t)stream);
        if (e != cudaSuccess) { fmm_set_error("evaluate: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
    }
    for (int s = FMM_STAGE_PREPARE; s <= FMM_STAGE_M2L_TC; s++) tree->ev_used[s] = false;   // evaluation stages
    int rc = fmm::evaluate_impl(tree, q, phi, force, dtype, (cudaStream_t)stream);
    tree->launch_ctr = nullptr;
    return rc;
}

int fmm_tree_set_positions(fmm_tree* tree, const void* pos, int pos_dtype, void* stream) {
    g_err[0] = 0;
    if (!tree) { fmm_set_error("tree is NULL"); return FMM_ERR_ARG; }
    if (tree->n > 0 && !pos) { fmm_set_error("pos is NULL"); return FMM_ERR_ARG; }
    if (pos_dtype != FMM_F64 && pos_dtype != FMM_F32) { fmm_set_error("pos_dtype must be FMM_F64 or FMM_F32"); return FMM_ERR_ARG; }
    return fmm::set_positions_impl(tree, pos, pos_dtype, (cudaStream_t)stream);
}

int fmm_backward(fmm_tree* tree, const void* q, const void* w, const void* field_q, void* dq, void* dx, int dtype,
                 void* stream) {
    g_err[0] = 0;
    if (!tree) { fmm_set_error("tree is NULL"); return FMM_ERR_ARG; }
    if (!(tree->prm.flags & FMM_OUT_FIELD)) { fmm_set_error("fmm_backward needs a tree built with FMM_OUT_FIELD"); return FMM_ERR_STATE; }
    if (dtype != FMM_F64 && dtype != FMM_F32) { fmm_set_error("dtype must be FMM_F64 or FMM_F32"); return FMM_ERR_ARG; }
    if (tree->n == 0) return FMM_OK;
    if (!q || !w || (dx && !field_q)) { fmm_set_error("q, w (and field_q when dx is wanted) must not be NULL"); return FMM_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    if (!tree->d.grad_tmp) {
        cudaError_t e = cudaMallocAsync(&tree->d.grad_tmp, (size_t)tree->n * 3 * 8, st);
        if (e != cudaSuccess) { fmm_set_error("backward: %s", cudaGetErrorString(e)); return FMM_ERR_ALLOC; }
        tree->device_bytes += (int64_t)tree->n * 3 * 8;
    }
    int rc = fmm_evaluate(tree, w, dq, dx ? tree->d.grad_tmp : nullptr, dtype, stream);
    if (rc) return rc;
    return fmm::grad_combine(tree, q, w, field_q, tree->d.grad_tmp, dx, dtype, st);
}

int fmm_build_tree_batched(const fmm_params* params, int32_t nsys, const int64_t* offsets, const void* pos,
                           int pos_dtype, fmm_tree** out, void* stream) {
    g_err[0] = 0;
    if (out) *out = nullptr;
    if (nsys < 1 || !offsets) { fmm_set_error("fmm_build_tree_batched: nsys >= 1 and offsets are required"); return FMM_ERR_ARG; }
    if (offsets[0] != 0) { fmm_set_error("fmm_build_tree_batched: offsets[0] must be 0"); return FMM_ERR_ARG; }
    std::vector<int64_t> off(offsets, offsets + nsys + 1);
    for (int s = 0; s < nsys; s++)
        if (off[s + 1] <= off[s]) { fmm_set_error("fmm_build_tree_batched: system %d is empty or offsets descend", s); return FMM_ERR_ARG; }
    return build_common(params, off[nsys], pos, pos_dtype, out, stream, &off);
}

int fmm_evaluate_batched(fmm_tree* tree, const void* q, void* phi, void* force, int dtype, void* stream) {
    return fmm_evaluate(tree, q, phi, force, dtype, stream);
}

int fmm_tree_export_systems(const fmm_tree* t, double* origins, double* sides, int32_t* cell_system) {
    if (!t) { fmm_set_error("tree is NULL"); return FMM_ERR_ARG; }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { fmm_set_error("export: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
    for (int s = 0; s < t->nsys && !t->h_geom.empty(); s++) {
        if (origins) for (int k = 0; k < 3; k++) origins[3 * s + k] = t->h_geom[4 * s + k];
        if (sides) sides[s] = t->h_geom[4 * s + 3];
    }
    if (cell_system && t->ncell) {
        std::vector<int32_t> first(t->ncell);
        e = cudaMemcpy(first.data(), t->d.first, 4 * (size_t)t->ncell, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { fmm_set_error("export: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
        for (int c = 0; c < t->ncell; c++) {
            int s = (int)(std::upper_bound(t->h_sys_off.begin(), t->h_sys_off.end(), (int64_t)first[c]) -
                          t->h_sys_off.begin()) - 1;
            cell_system[c] = s;
        }
    }
    return FMM_OK;
}

int fmm_tree_get_info(const fmm_tree* t, fmm_tree_info* info) {
    if (!t || !info) { fmm_set_error("NULL argument"); return FMM_ERR_ARG; }
    memset(info, 0, sizeof(*info));
    info->n = t->n;
    info->ncell = t->ncell;
    info->nlevel = t->nlevel;
    info->nleaf = t->nleaf;
    info->p = t->prm.p;
    info->nm2l = t->nm2l;
    info->np2p = t->np2p;
    for (int k = 0; k < 3; k++) info->origin[k] = t->origin[k];
    info->side = t->side;
    info->device_bytes = t->device_bytes;
    info->tc_pairs = t->tc_npairs;
    info->tc_classes = t->tc_nclass;
    info->tc_items = t->tc_nitems;
    info->nsys = t->nsys;
    return FMM_OK;
}

int fmm_tree_export(const fmm_tree* t, uint64_t* keys, int64_t* perm, int32_t* level, uint64_t* cell_key,
                    int64_t* first, int64_t* count, int32_t* parent, int32_t* child_first,
                    int32_t* child_count, int32_t* m2l, int32_t* p2p) {
    if (!t) { fmm_set_error("tree is NULL"); return FMM_ERR_ARG; }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { fmm_set_error("export: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
    const size_t n = (size_t)t->n, nc = (size_t)t->ncell;
    const fmm::TreeDev& d = t->d;
#define CP(dst, srcp, cnt, sz)                                                                   \
    if ((dst) && (cnt)) {                                                                        \
        e = cudaMemcpy((dst), (srcp), (cnt) * (sz), cudaMemcpyDeviceToHost);                     \
        if (e != cudaSuccess) { fmm_set_error("export: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; } \
    }
    CP(keys, d.keys, n, 8);
    CP(level, d.level, nc, 4);
    CP(cell_key, d.ckey, nc, 8);
    CP(parent, d.parent, nc, 4);
    CP(child_first, d.child_first, nc, 4);
    CP(child_count, d.child_count, nc, 4);
    if (perm && n) {
        std::vector<int32_t> v(n);
        CP(v.data(), d.perm, n, 4);
        for (size_t i = 0; i < n; i++) perm[i] = v[i];
    }
    if ((first || count) && nc) {
        std::vector<int32_t> v(nc);
        if (first) { CP(v.data(), d.first, nc, 4); for (size_t i = 0; i < nc; i++) first[i] = v[i]; }
        if (count) { CP(v.data(), d.count, nc, 4); for (size_t i = 0; i < nc; i++) count[i] = v[i]; }
    }
    // lists: expand CSR back to (target, source) pairs
    if (m2l && t->nm2l && !d.m2l_start) {
        // tensor-core trees keep their M2L pairs in class order only: sort here
        std::vector<int32_t> tg((size_t)t->nm2l), sr((size_t)t->nm2l);
        CP(tg.data(), d.tc_tgt, (size_t)t->nm2l, 4);
        CP(sr.data(), d.tc_src, (size_t)t->nm2l, 4);
        std::vector<uint64_t> key((size_t)t->nm2l);
        for (size_t k = 0; k < key.size(); k++) key[k] = ((uint64_t)(uint32_t)tg[k] << 32) | (uint32_t)sr[k];
        std::sort(key.begin(), key.end());
        for (size_t k = 0; k < key.size(); k++) {
            m2l[2 * k] = (int32_t)(key[k] >> 32);
            m2l[2 * k + 1] = (int32_t)(key[k] & 0xffffffffu);
        }
    }
    for (int which = 0; which < 2; which++) {
        int32_t* out = which == 0 ? m2l : p2p;
        int64_t np = which == 0 ? t->nm2l : t->np2p;
        if (!out || np == 0) continue;
        if (which == 0 && !d.m2l_start) continue;
        std::vector<int64_t> st(nc + 1);
        std::vector<int32_t> src((size_t)np);
        CP(st.data(), which == 0 ? d.m2l_start : d.p2p_start, nc + 1, 8);
        CP(src.data(), which == 0 ? d.m2l_src : d.p2p_src, (size_t)np, 4);
        for (size_t c = 0; c < nc; c++)
            for (int64_t k = st[c]; k < st[c + 1]; k++) { out[2 * k] = (int32_t)c; out[2 * k + 1] = src[k]; }
    }
#undef CP
    return FMM_OK;
}

int fmm_inject_dependency(fmm_tree* t, int32_t counter, int32_t cell, int32_t delta) {
    if (!t) { fmm_set_error("tree is NULL"); return FMM_ERR_ARG; }
    if (!t->d.q_cnt_init && !t->d.dag_cnt_init) { fmm_set_error("tree does not use the task queue"); return FMM_ERR_STATE; }
    if (counter < 0 || counter > 3 || cell < 0 || cell >= t->ncell) { fmm_set_error("bad counter or cell"); return FMM_ERR_ARG; }
    int32_t* p = nullptr;
    if (t->d.q_cnt_init) {
        p = t->d.q_cnt_init + (size_t)counter * t->ncell + cell;
    } else {
        // the mixed form's task graph keeps counters 0 (children not final) and 3 (L2P)
        if (counter != 0 && counter != 3) { fmm_set_error("this tree's task graph has counters 0 and 3 only"); return FMM_ERR_ARG; }
        p = t->d.dag_cnt_init + (size_t)(counter == 0 ? 0 : 1) * t->ncell + cell;
    }
    int32_t v = 0;
    cudaError_t e = cudaMemcpy(&v, p, 4, cudaMemcpyDeviceToHost);
    v += delta;
    if (e == cudaSuccess) e = cudaMemcpy(p, &v, 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { fmm_set_error("inject: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
    return FMM_OK;
}

int fmm_status(fmm_tree* t) {
    if (!t) { fmm_set_error("tree is NULL"); return FMM_ERR_ARG; }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { fmm_set_error("status: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
    int s = 0;
    if (t->d.status) {
        e = cudaMemcpy(&s, t->d.status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { fmm_set_error("status: %s", cudaGetErrorString(e)); return FMM_ERR_CUDA; }
    }
    if (s) fmm_set_error("device status %d", s);
    return s ? FMM_ERR_TIMEOUT : FMM_OK;
}

void fmm_tree_destroy(fmm_tree* t) {
    if (!t) return;
    cudaDeviceSynchronize();
    if (t->side_stream) cudaStreamSynchronize(t->side_stream);
    if (t->hi_stream) cudaStreamSynchronize(t->hi_stream);
    if (t->ops_stream) cudaStreamSynchronize(t->ops_stream);
    fmm::free_tree_device(t);
    cudaStreamSynchronize(0);
    if (t->timing) for (int i = 0; i < 2 * FMM_NUM_STAGES; i++) cudaEventDestroy(t->ev[i]);
    if (t->side_stream) cudaStreamDestroy(t->side_stream);
    if (t->hi_stream) cudaStreamDestroy(t->hi_stream);
    if (t->ops_stream) cudaStreamDestroy(t->ops_stream);
    if (t->ev_join_hi) cudaEventDestroy(t->ev_join_hi);
    if (t->ev_fork) cudaEventDestroy(t->ev_fork);
    if (t->ev_join) cudaEventDestroy(t->ev_join);
    if (t->ev_ops) cudaEventDestroy(t->ev_ops);
    if (t->ev_rem_fork) cudaEventDestroy(t->ev_rem_fork);
    if (t->ev_rem_join) cudaEventDestroy(t->ev_rem_join);
    fmm::pinned_slot_release(t->h_pin);
    delete t;
}

static const char* k_stage_names[FMM_NUM_STAGES] = {"keys", "octree", "lists",    "setup",     "prepare", "p2p",
                                                     "p2m",  "m2m",    "m2l",      "l2l",       "l2p",     "queue",
                                                     "m2l_tc", "traversal", "classes", "p2p_list"};

const char* fmm_stage_name(int32_t i) { return (i >= 0 && i < FMM_NUM_STAGES) ? k_stage_names[i] : ""; }

int fmm_stage_times(const fmm_tree* t, double* ms, int32_t max_stages) {
    if (!t || !ms) { fmm_set_error("NULL argument"); return FMM_ERR_ARG; }
    if (!t->timing) { fmm_set_error("tree was built without FMM_TIMING"); return FMM_ERR_STATE; }
    for (int i = 0; i < max_stages; i++) {
        ms[i] = -1.0;
        if (i >= FMM_NUM_STAGES || !t->ev_used[i]) continue;
        cudaError_t e = cudaEventSynchronize(t->ev[2 * i + 1]);
        float f = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&f, t->ev[2 * i], t->ev[2 * i + 1]);
        if (e != cudaSuccess) { fmm_set_error("stage %d: %s", i, cudaGetErrorString(e)); return FMM_ERR_CUDA; }
        ms[i] = f;
    }
    return FMM_OK;
}

int64_t fmm_kernel_launches(const fmm_tree* t, int32_t build) {
    if (!t) return -1;
    return build ? t->launches_build : t->launches_eval;
}

}  // extern "C"
