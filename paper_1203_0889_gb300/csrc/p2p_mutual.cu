// p2p_mutual.cu -- mutual near-field interaction (paper Section 4: an
// interaction may update both cells, using the symmetry of the pair kernel).
//
// P2P between two different leaves a and b computes, for every particle pair,
// one separation d = x_i - x_j and one 1/r, and gives both particles their
// terms:  phi_i += q_j / r, grad_i -= q_j d / r^3  and  phi_j += q_i / r,
// grad_j += q_i d / r^3.  The non-mutual form (stages.cuh) evaluates every pair
// twice, once from each side.
//
// Which side does the work.  Every record (target a, source b) of the P2P list
// gets a mode at tree build, from one search: Y = "a is in b's list".
//   b == a            0  the leaf's own pairs (k_p2p_own, with the residuals)
//   b > a,  Y         2  a's item evaluates both directions
//   b > a, !Y         1  a's item evaluates a <- b only
//   b < a,  Y         0  b's item evaluates the pair (its record for a has mode 2)
//   b < a, !Y         1  a's item evaluates a <- b only
// so every directed pair is evaluated exactly once whether or not the lists are
// symmetric (the dual traversal's lists are symmetric on every workload
// measured, so mode 1 is a safeguard).
//
// Kernel layout (one warp per P2P work item, i.e. a run of a target leaf's
// records).  The target leaf's particles, 32 at a time, are held two per lane
// (in the halves of 64-bit registers, paired f32x2 arithmetic); W = ceil(nt/2)
// lanes form a ring and 32 / W rings share the warp.  The item's selected
// sources form one stream (records compacted per chunk of 32 records); each
// ring takes W sources at a time, one per lane, into shared memory, and runs W
// steps.  At step s the lane at ring position p pairs its two targets with
// source (p + s) mod W; the reaction accumulator of that source travels with it
// around the ring (one shuffle per component per step) and is back at the lane
// that loaded the source after W steps, which adds it to the source particle.
// Results of both sides go to a float4 accumulator per particle with vector
// atomic adds (red.global.add.v4.f32), so the summation order, and with it the
// last bits, vary from run to run; k_p2p_own then writes near = accumulator +
// the leaf's own pairs.
#include "stages.cuh"

namespace fmm {

// mode of every record (the rule above), one thread per record; the sources of
// a target are in ascending cell order (both list builders sort them so)
__global__ void k_p2p_modes(int64_t np, const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                            const int64_t* __restrict__ start, int8_t* __restrict__ mode) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int a = tgt[e], b = src[e];
    int8_t md = 0;
    if (b != a) {
        int64_t lo = start[b], hi = start[b + 1];   // search a among b's sources
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (src[mid] < a) lo = mid + 1; else hi = mid;
        }
        const bool y = lo < start[b + 1] && src[lo] == a;
        md = b > a ? (y ? 2 : 1) : (y ? 0 : 1);
    }
    mode[e] = md;
}

int build_p2p_modes(fmm_tree* t, const int32_t* tgt, cudaStream_t st) {
    TreeDev& d = t->d;
    if (t->np2p == 0) return FMM_OK;
    int rc;
    if ((rc = dev_alloc(&d.p2p_mode, (size_t)t->np2p, t, st))) return rc;
    k_p2p_modes<<<(unsigned)((t->np2p + 255) / 256), 256, 0, st>>>(t->np2p, tgt, d.p2p_src, d.p2p_start,
                                                                    d.p2p_mode);
    count_launch(t);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

__device__ __forceinline__ void red_add_v4(float4* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

constexpr int MU_WARPS = 4;
// targets per pass over an item's sources: two per lane, so rings of at most 16
// lanes and at least two rings per warp (64 left up to half the lanes idle on
// leaves of 33 .. 64 particles; a second pass costs one more reaction add per
// source)
constexpr int MU_TARGETS = 32;
// dummy particles (zero charge) of ragged rings: targets and sources far from
// every particle and from each other, so that every pair they enter is finite
// and contributes exactly zero to the real particles
constexpr float MU_FAR = 1e18f;

// the source of stream position k of the chunk (srec), in the target's frame,
// negated (-x, -y, -z, q); gi = the particle that takes its reaction, or -1
// (past the stream's end: a dummy at +MU_FAR)
__device__ __forceinline__ void mu_source(int k, int total, bool inring, const int4* srec, int& cur,
                                          const float4* __restrict__ xq, const int4* __restrict__ icentre, int4 ict,
                                          float u2f, float4& s, int& gi) {
    s = make_float4(-MU_FAR, -MU_FAR, -MU_FAR, 0.f);
    gi = -1;
    if (inring && k < total) {
        while (srec[cur].z + srec[cur].y <= k) cur++;
        const int4 q = srec[cur];
        const int src = q.w & 0x7fffffff;
        const int j = q.x + (k - q.z);
        const int4 ics = icentre[src];
        const float ox = (float)(ics.x - ict.x) * u2f, oy = (float)(ics.y - ict.y) * u2f,
                    oz = (float)(ics.z - ict.z) * u2f;
        const float4 v = xq[j];
        s = make_float4(-(v.x + ox), -(v.y + oy), -(v.z + oz), v.w);
        if (q.w < 0) gi = j;
    }
}

__global__ void __launch_bounds__(32 * MU_WARPS) k_p2p_mutual(const int4* __restrict__ items,
                                                              const int32_t* __restrict__ nitems,
                                                              const int32_t* __restrict__ first,
                                                              const int32_t* __restrict__ count,
                                                              const int64_t* __restrict__ start,
                                                              const int4* __restrict__ rec,
                                                              const int8_t* __restrict__ mode,
                                                              const float4* __restrict__ xq,
                                                              const int4* __restrict__ icentre,
                                                              const float* __restrict__ cu2f, float4* acc) {
    __shared__ float4 ssrc[MU_WARPS][32];   // the ring sources of the current round: -x, -y, -z, q
    __shared__ int4 srec[MU_WARPS][32];     // selected records of the chunk: first, count, stream offset, source
    const unsigned FULL = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wi = blockIdx.x * MU_WARPS + warp;
    if (wi >= nitems[0]) return;
    const int4 it = items[wi];
    const int c = it.x;
    const int64_t s0 = start[c] + it.y, s1 = s0 + it.z;
    const int tf = first[c], nt = count[c];
    const int4 ict = icentre[c];
    const float u2f = cu2f[c];
    const f2::u64 EPS2 = f2::pack(1e-30f, 1e-30f);
    for (int tb = 0; tb < nt; tb += MU_TARGETS) {
        const int ntc = min(MU_TARGETS, nt - tb);
        const int W = (ntc + 1) >> 1, R = 32 / W;
        const int g = lane / W, pos = lane - g * W;
        const bool inring = g < R;
        // lanes outside every ring read their own slot and pass to themselves
        const int rbase = inring ? g * W : lane, rw = inring ? W : 1;
        const int nxt = inring ? rbase + (pos + 1 == W ? 0 : pos + 1) : lane;
        // targets pos (low halves) and pos + W (high halves); dummy: far, no charge
        float4 t0 = make_float4(-MU_FAR, -MU_FAR, -MU_FAR, 0.f), t1 = t0;   // dummy sources sit at +MU_FAR
        if (inring) t0 = xq[tf + tb + pos];   // pos < W <= ntc
        if (inring && pos + W < ntc) t1 = xq[tf + tb + pos + W];
        const f2::u64 X = f2::pack(t0.x, t1.x), Y = f2::pack(t0.y, t1.y), Z = f2::pack(t0.z, t1.z),
                      Q = f2::pack(t0.w, t1.w);
        // potential and G = sum q_s d / r^3 of both targets (the gradient is -G)
        f2::u64 NP = 0, GX = 0, GY = 0, GZ = 0;
        for (int64_t cb = s0; cb < s1; cb += 32) {
            const int64_t e = cb + lane;
            int md = 0;
            int4 r = make_int4(0, 0, 0, 0);
            if (e < s1) {
                md = mode[e];
                r = rec[e];
            }
            const int cnt = md ? r.y : 0;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(FULL, incl, 31);
            const unsigned sel = __ballot_sync(FULL, md != 0);
            __syncwarp();   // the previous chunk's cursor reads of srec are done
            if (md) srec[warp][__popc(sel & ((1u << lane) - 1u))] =
                make_int4(r.x, r.y, incl - cnt, md == 2 ? (int)((uint32_t)r.w | 0x80000000u) : r.w);
            __syncwarp();
            const int nround = (total + W - 1) / W;
            int cur = 0;
            float4 s;
            int gi;
            mu_source(g * W + pos, total, inring, srec[warp], cur, xq, icentre, ict, u2f, s, gi);
            for (int rb = 0; rb < nround; rb += R) {
                __syncwarp();   // the previous round's reads of ssrc are done
                ssrc[warp][lane] = s;
                const int gcur = gi;
                __syncwarp();
                // the next round's source, loaded while this round runs
                if (rb + R < nround)
                    mu_source((rb + R + g) * W + pos, total, inring, srec[warp], cur, xq, icentre, ict, u2f, s, gi);
                float ap = 0.f, ax = 0.f, ay = 0.f, az = 0.f;   // reaction of the source in this lane's slot
                int idx = pos < rw ? pos : 0;
                for (int step = 0; step < W; step++) {
                    const float4 sj = ssrc[warp][rbase + idx];
                    const f2::u64 dx = f2::add(X, f2::pack(sj.x, sj.x)), dy = f2::add(Y, f2::pack(sj.y, sj.y)),
                                  dz = f2::add(Z, f2::pack(sj.z, sj.z));
                    // r^2 from 1e-30 like the non-mutual cross-leaf pairs: a
                    // near-duplicate across a leaf boundary stays finite
                    float ra, rb2;
                    f2::unpack(f2::fma(dz, dz, f2::fma(dy, dy, f2::fma(dx, dx, EPS2))), ra, rb2);
                    const f2::u64 ri = f2::pack(rsqrt_t(ra), rsqrt_t(rb2));
                    const f2::u64 ri2 = f2::mul(ri, ri);
                    const f2::u64 qs = f2::mul(f2::pack(sj.w, sj.w), ri);   // the source on the targets
                    NP = f2::add(NP, qs);
                    const f2::u64 gs = f2::mul(qs, ri2);
                    GX = f2::fma(gs, dx, GX); GY = f2::fma(gs, dy, GY); GZ = f2::fma(gs, dz, GZ);
                    const f2::u64 qt = f2::mul(Q, ri);   // the targets on the source
                    const f2::u64 gt = f2::mul(qt, ri2);
                    float qa, qb, ga, gb, da, db;
                    f2::unpack(qt, qa, qb);
                    f2::unpack(gt, ga, gb);
                    ap += qa + qb;
                    f2::unpack(dx, da, db); ax = fmaf(ga, da, fmaf(gb, db, ax));
                    f2::unpack(dy, da, db); ay = fmaf(ga, da, fmaf(gb, db, ay));
                    f2::unpack(dz, da, db); az = fmaf(ga, da, fmaf(gb, db, az));
                    ap = __shfl_sync(FULL, ap, nxt);
                    ax = __shfl_sync(FULL, ax, nxt);
                    ay = __shfl_sync(FULL, ay, nxt);
                    az = __shfl_sync(FULL, az, nxt);
                    idx = idx + 1 == rw ? 0 : idx + 1;
                }
                if (gcur >= 0) red_add_v4(acc + gcur, ap, ax, ay, az);
            }
        }
        if (inring) {
            float pa, pb, xa, xb, ya, yb, za, zb;
            f2::unpack(NP, pa, pb);
            f2::unpack(GX, xa, xb); f2::unpack(GY, ya, yb); f2::unpack(GZ, za, zb);
            red_add_v4(acc + tf + tb + pos, pa, -xa, -ya, -za);
            if (pos + W < ntc) red_add_v4(acc + tf + tb + pos + W, pb, -xb, -yb, -zb);
        }
    }
}

int p2p_mutual_launch(fmm_tree* t, const float4* xq32, float4* acc, cudaStream_t st) {
    const TreeDev& d = t->d;
    FMM_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(float4) * (size_t)t->n, st));
    const int64_t nitems = t->h_pin && t->h_pin[0] >= 0 ? t->h_pin[0] : t->p2p_items_bound;
    if (nitems > 0 && d.p2p_mode) {
        k_p2p_mutual<<<(unsigned)((nitems + MU_WARPS - 1) / MU_WARPS), 32 * MU_WARPS, 0, st>>>(
            d.p2p_items, d.p2p_nitems, d.first, d.count, d.p2p_start, d.p2p_rec, d.p2p_mode, xq32, d.icentre, d.cu2f,
            acc);
        count_launch(t);
    }
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

}  // namespace fmm
