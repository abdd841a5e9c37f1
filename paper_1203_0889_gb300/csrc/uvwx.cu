// uvwx.cu -- the parent-neighbour-child list builder (FMM_LISTS_UVWX): the
// M2L and P2P pair lists of a tree from the U, V, W and X lists of uvwx.cuh,
// in place of the dual traversal.  The pairs go through the same list
// finishing (sort, CSR, records, tensor-core classes) as the traversal's, so
// every evaluation path runs on them unchanged.
//
// Steps (one thread per cell or leaf; counts, an exclusive scan, then a fill
// that repeats the count's walk):
//   1. neighbours, level by level from the roots down;
//   2. V of every cell -> M2L pairs;
//   3. U and W of every leaf -> P2P pairs and W pairs;
//   4. the leaves inside every W cell -> P2P pairs in both directions.
#include <cub/cub.cuh>

#include <algorithm>

#include "fmm_internal.cuh"
#include "uvwx.cuh"

namespace fmm {

namespace {

template <typename T>
void uv_free(T*& p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
}

__global__ void k_uv_neighbours(int c0, int c1, UvTree T, int32_t* nb, int32_t* nbc, int* err) {
    const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= c1) return;
    const int cnt = uv_neighbours(T, c, nb + (int64_t)c * UV_NB);
    if (cnt > UV_NB) atomicOr(err, 1);
    nbc[c] = cnt < UV_NB ? cnt : UV_NB;
}

// fill = false: cnt[c] = |V(c)|; fill = true: pairs (c, v) from off[c]
__global__ void k_uv_v(int ncell, UvTree T, bool fill, int64_t* cnt, const int64_t* off, int2* pairs) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    if (!fill) {
        cnt[c] = uv_v_list(T, c, [](int) {});
        return;
    }
    int64_t o = off[c];
    const int64_t lim = o + cnt[c];
    uv_v_list(T, c, [&](int x) {
        if (o < lim) pairs[o] = make_int2(c, x);
        o++;
    });
}

// per leaf: U and W counts, then the pairs (U into the P2P list, W into wp)
__global__ void k_uv_uw(int nleaf, const int32_t* __restrict__ leaves, UvTree T, bool fill, int64_t* cu, int64_t* cw,
                        const int64_t* ou, const int64_t* ow, int2* up, int2* wp, int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaf) return;
    const int b = leaves[i];
    if (!fill) {
        int64_t nu = 0, nw = 0;
        if (!uv_uw_lists(T, b, [&](int) { nu++; }, [&](int) { nw++; })) atomicOr(err, 2);
        cu[i] = nu;
        cw[i] = nw;
        return;
    }
    int64_t u = ou[i], w = ow[i];
    const int64_t ulim = u + cu[i], wlim = w + cw[i];
    uv_uw_lists(T, b,
                [&](int a) {
                    if (u < ulim) up[u] = make_int2(b, a);
                    u++;
                },
                [&](int d) {
                    if (w < wlim) wp[w] = make_int2(b, d);
                    w++;
                });
}

// leaf of the first particle of every leaf run, and the runs' first particles
__global__ void k_uv_leaf_starts(int64_t n, const int32_t* __restrict__ pleaf, char* flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = i == 0 || pleaf[i] != pleaf[i - 1];
}
__global__ void k_uv_lfirst(int nleaf, const int32_t* __restrict__ lm, const int32_t* __restrict__ first,
                            int32_t* lfirst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nleaf) lfirst[k] = first[lm[k]];
}

// W pair j = (b, D): the leaves inside D, as pairs (b, L) and (L, b)
__global__ void k_uv_wexp(int64_t nw, const int2* __restrict__ wp, const int32_t* __restrict__ first,
                          const int32_t* __restrict__ count, const int32_t* __restrict__ lm,
                          const int32_t* __restrict__ lfirst, int nleaf, bool fill, int64_t* cnt, const int64_t* off,
                          int2* pairs) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nw) return;
    const int2 w = wp[j];
    int k0, k1;
    uv_leaf_run(lfirst, nleaf, first[w.y], count[w.y], k0, k1);
    if (!fill) {
        cnt[j] = 2 * (int64_t)(k1 - k0);
        return;
    }
    int64_t o = off[j];
    const int64_t lim = o + cnt[j];
    for (int k = k0; k < k1 && o + 2 <= lim; k++, o += 2) {
        pairs[o] = make_int2(w.x, lm[k]);
        pairs[o + 1] = make_int2(lm[k], w.x);
    }
}

inline unsigned uv_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// exclusive scan of cnt[0..n) into off, total to *total (host, synchronises)
int uv_scan(const int64_t* cnt, int64_t* off, int64_t n, int64_t* total, cudaStream_t st) {
    *total = 0;
    if (n == 0) return FMM_OK;
    size_t sb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, sb, cnt, off, n, st);
    char* tmp = nullptr;
    int rc;
    if ((rc = dev_alloc(&tmp, sb, nullptr, st))) return rc;
    FMM_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, sb, cnt, off, n, st));
    int64_t last[2] = {0, 0};
    FMM_CUDA_TRY(cudaMemcpyAsync(&last[0], off + n - 1, 8, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(&last[1], cnt + n - 1, 8, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    uv_free(tmp, st);
    *total = last[0] + last[1];
    return FMM_OK;
}

}  // namespace

int uvwx_lists(fmm_tree* t, int2** m2l_out, int64_t* nm_out, int2** p2p_out, int64_t* np_out, cudaStream_t st) {
    TreeDev& d = t->d;
    const int nc = t->ncell, nl = t->nleaf;
    int rc;
    *m2l_out = *p2p_out = nullptr;
    *nm_out = *np_out = 0;
    int32_t *nb = nullptr, *nbc = nullptr, *lm = nullptr, *lfirst = nullptr, *nsel = nullptr;
    int* err = nullptr;
    int64_t *c1 = nullptr, *o1 = nullptr, *c2 = nullptr, *o2 = nullptr;
    int2 *m2l = nullptr, *p2p = nullptr, *wp = nullptr;
    char *flag = nullptr, *tmp = nullptr;
    auto release = [&]() {
        uv_free(nb, st); uv_free(nbc, st); uv_free(lm, st); uv_free(lfirst, st); uv_free(nsel, st);
        uv_free(err, st); uv_free(c1, st); uv_free(o1, st); uv_free(c2, st); uv_free(o2, st);
        uv_free(wp, st); uv_free(flag, st); uv_free(tmp, st);
    };
    auto fail = [&](int code) {
        release();
        uv_free(m2l, st);
        uv_free(p2p, st);
        return code;
    };
    if (nc == 0) return FMM_OK;
    if ((rc = dev_alloc(&nb, (size_t)nc * UV_NB, nullptr, st)) || (rc = dev_alloc(&nbc, (size_t)nc, nullptr, st)) ||
        (rc = dev_alloc(&err, 1, nullptr, st)))
        return fail(rc);
    FMM_CUDA_TRY(cudaMemsetAsync(nbc, 0, sizeof(int32_t) * nc, st));
    FMM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    const UvTree T = {d.icentre, d.parent, d.child_first, d.child_count, nb, nbc};
    // 1. neighbours, top down (the roots have none)
    for (int l = 1; l < t->nlevel; l++) {
        const int a = t->level_start[l], b = t->level_start[l + 1];
        if (b > a) {
            k_uv_neighbours<<<uv_blocks(b - a, 128), 128, 0, st>>>(a, b, T, nb, nbc, err);
            count_launch(t);
        }
    }
    // 2. V -> M2L pairs
    if ((rc = dev_alloc(&c1, (size_t)nc, nullptr, st)) || (rc = dev_alloc(&o1, (size_t)nc, nullptr, st)))
        return fail(rc);
    k_uv_v<<<uv_blocks(nc, 128), 128, 0, st>>>(nc, T, false, c1, nullptr, nullptr);
    count_launch(t);
    int64_t nm = 0;
    if ((rc = uv_scan(c1, o1, nc, &nm, st))) return fail(rc);
    if ((rc = dev_alloc(&m2l, (size_t)std::max<int64_t>(nm, 1), nullptr, st))) return fail(rc);
    k_uv_v<<<uv_blocks(nc, 128), 128, 0, st>>>(nc, T, true, c1, o1, m2l);
    count_launch(t);
    uv_free(c1, st);
    uv_free(o1, st);
    // 3. U and W of the leaves
    if ((rc = dev_alloc(&c1, (size_t)std::max(nl, 1), nullptr, st)) ||
        (rc = dev_alloc(&o1, (size_t)std::max(nl, 1), nullptr, st)) ||
        (rc = dev_alloc(&c2, (size_t)std::max(nl, 1), nullptr, st)) ||
        (rc = dev_alloc(&o2, (size_t)std::max(nl, 1), nullptr, st)))
        return fail(rc);
    if (nl > 0) {
        k_uv_uw<<<uv_blocks(nl, 128), 128, 0, st>>>(nl, d.leaves, T, false, c1, c2, nullptr, nullptr, nullptr,
                                                     nullptr, err);
        count_launch(t);
    }
    int64_t nu = 0, nw = 0;
    if ((rc = uv_scan(c1, o1, nl, &nu, st)) || (rc = uv_scan(c2, o2, nl, &nw, st))) return fail(rc);
    int herr = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) {
        fmm_set_error("U/V/W/X lists: %s", (herr & 1) ? "more than 26 neighbours of a cell" : "tree too deep");
        return fail(FMM_ERR_STATE);
    }
    if ((rc = dev_alloc(&wp, (size_t)std::max<int64_t>(nw, 1), nullptr, st))) return fail(rc);
    // the P2P list: U first, then the expanded W (and X) pairs; its size needs step 4's count
    int2* up = nullptr;
    if ((rc = dev_alloc(&up, (size_t)std::max<int64_t>(nu, 1), nullptr, st))) return fail(rc);
    if (nl > 0) {
        k_uv_uw<<<uv_blocks(nl, 128), 128, 0, st>>>(nl, d.leaves, T, true, c1, c2, o1, o2, up, wp, err);
        count_launch(t);
    }
    uv_free(c1, st); uv_free(o1, st); uv_free(c2, st); uv_free(o2, st);
    // 4. leaves in particle order, then the leaves inside every W cell
    int64_t nx = 0;
    if (nw > 0) {
        size_t sb = 0;
        int32_t hsel = 0;
        if ((rc = dev_alloc(&flag, (size_t)t->n, nullptr, st)) || (rc = dev_alloc(&lm, (size_t)nl, nullptr, st)) ||
            (rc = dev_alloc(&lfirst, (size_t)nl, nullptr, st)) || (rc = dev_alloc(&nsel, 1, nullptr, st))) {
            uv_free(up, st);
            return fail(rc);
        }
        k_uv_leaf_starts<<<uv_blocks(t->n, 256), 256, 0, st>>>(t->n, d.pleaf, flag);
        count_launch(t);
        cub::DeviceSelect::Flagged(nullptr, sb, d.pleaf, flag, lm, nsel, t->n, st);
        if ((rc = dev_alloc(&tmp, sb, nullptr, st))) {
            uv_free(up, st);
            return fail(rc);
        }
        FMM_CUDA_TRY(cub::DeviceSelect::Flagged(tmp, sb, d.pleaf, flag, lm, nsel, t->n, st));
        count_launch(t);
        FMM_CUDA_TRY(cudaMemcpyAsync(&hsel, nsel, 4, cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
        if (hsel != nl) {
            fmm_set_error("U/V/W/X lists: %d leaf runs for %d leaves", hsel, nl);
            uv_free(up, st);
            return fail(FMM_ERR_STATE);
        }
        k_uv_lfirst<<<uv_blocks(nl, 256), 256, 0, st>>>(nl, lm, d.first, lfirst);
        count_launch(t);
        if ((rc = dev_alloc(&c1, (size_t)nw, nullptr, st)) || (rc = dev_alloc(&o1, (size_t)nw, nullptr, st))) {
            uv_free(up, st);
            return fail(rc);
        }
        k_uv_wexp<<<uv_blocks(nw, 256), 256, 0, st>>>(nw, wp, d.first, d.count, lm, lfirst, nl, false, c1, nullptr,
                                                       nullptr);
        count_launch(t);
        if ((rc = uv_scan(c1, o1, nw, &nx, st))) {
            uv_free(up, st);
            return fail(rc);
        }
    }
    if ((rc = dev_alloc(&p2p, (size_t)std::max<int64_t>(nu + nx, 1), nullptr, st))) {
        uv_free(up, st);
        return fail(rc);
    }
    if (nu > 0) FMM_CUDA_TRY(cudaMemcpyAsync(p2p, up, sizeof(int2) * nu, cudaMemcpyDeviceToDevice, st));
    uv_free(up, st);
    if (nx > 0) {
        k_uv_wexp<<<uv_blocks(nw, 256), 256, 0, st>>>(nw, wp, d.first, d.count, lm, lfirst, nl, true, c1, o1,
                                                       p2p + nu);
        count_launch(t);
    }
    FMM_CUDA_TRY(cudaGetLastError());
    release();
    *m2l_out = m2l;
    *p2p_out = p2p;
    *nm_out = nm;
    *np_out = nu + nx;
    return FMM_OK;
}

}  // namespace fmm
