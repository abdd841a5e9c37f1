// Host build of the U/V/W/X list functions (paper_1203_0889_gb300/csrc/uvwx.cuh)
// for tests/test_uvwx_host.py: reads a tree's arrays, runs the same per-cell
// and per-leaf functions the kernels of uvwx.cu run, in the kernels' order
// (neighbours level by level, then V, then U and W, then the leaves inside
// every W cell), and writes the M2L and P2P pairs.
//
// Input (binary, little-endian int32 unless stated): ncell, nleaf, n, nlevel;
// level_start[nlevel + 1]; icentre[ncell][4]; parent, child_first,
// child_count, first, count [ncell each]; leaves[nleaf]; pleaf[n].
// Output: int64 nm, int64 np, then nm and np (target, source) int32 pairs.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "uvwx.cuh"

using namespace fmm;

static void rd(FILE* f, void* p, size_t bytes) {
    if (bytes && fread(p, 1, bytes, f) != bytes) {
        fprintf(stderr, "short read\n");
        exit(2);
    }
}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t hdr[4];
    rd(f, hdr, sizeof(hdr));
    const int nc = hdr[0], nl = hdr[1], n = hdr[2], nlevel = hdr[3];
    std::vector<int32_t> ls(nlevel + 1), par(nc), cf(nc), cc(nc), first(nc), count(nc), leaves(nl), pleaf(n);
    std::vector<int4> ic(nc);
    rd(f, ls.data(), 4 * ls.size());
    rd(f, ic.data(), 16 * ic.size());
    rd(f, par.data(), 4 * nc); rd(f, cf.data(), 4 * nc); rd(f, cc.data(), 4 * nc);
    rd(f, first.data(), 4 * nc); rd(f, count.data(), 4 * nc);
    rd(f, leaves.data(), 4 * (size_t)nl); rd(f, pleaf.data(), 4 * (size_t)n);
    fclose(f);
    std::vector<int32_t> nb((size_t)nc * UV_NB, -1), nbc(nc, 0);
    const UvTree T = {ic.data(), par.data(), cf.data(), cc.data(), nb.data(), nbc.data()};
    for (int l = 1; l < nlevel; l++)
        for (int c = ls[l]; c < ls[l + 1]; c++) {
            const int k = uv_neighbours(T, c, nb.data() + (size_t)c * UV_NB);
            if (k > UV_NB) return 3;
            nbc[c] = k;
        }
    std::vector<int2> m2l, p2p, wp;
    for (int c = 0; c < nc; c++) uv_v_list(T, c, [&](int x) { m2l.push_back(make_int2(c, x)); });
    for (int i = 0; i < nl; i++) {
        const int b = leaves[i];
        if (!uv_uw_lists(T, b, [&](int a) { p2p.push_back(make_int2(b, a)); },
                         [&](int d) { wp.push_back(make_int2(b, d)); }))
            return 4;
    }
    std::vector<int32_t> lm, lfirst;
    for (int i = 0; i < n; i++)
        if (i == 0 || pleaf[i] != pleaf[i - 1]) lm.push_back(pleaf[i]);
    if ((int)lm.size() != nl) return 5;
    for (int k = 0; k < nl; k++) lfirst.push_back(first[lm[k]]);
    for (const int2& w : wp) {
        int k0, k1;
        uv_leaf_run(lfirst.data(), nl, first[w.y], count[w.y], k0, k1);
        for (int k = k0; k < k1; k++) {
            p2p.push_back(make_int2(w.x, lm[k]));
            p2p.push_back(make_int2(lm[k], w.x));
        }
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    const int64_t nm = (int64_t)m2l.size(), np = (int64_t)p2p.size();
    fwrite(&nm, 8, 1, o);
    fwrite(&np, 8, 1, o);
    fwrite(m2l.data(), sizeof(int2), m2l.size(), o);
    fwrite(p2p.data(), sizeof(int2), p2p.size(), o);
    fclose(o);
    return 0;
}
