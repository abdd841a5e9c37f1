// evaluate.cu -- the six FMM stages (paper Section 2.1) as CUDA kernels,
// launched stage by stage.
//
//   P2M  leaf multipoles          Mt_n^m = sum_j q_j R_n^m((x_j - c)/h)
//   M2M  child -> parent          Mt_n^m(P) += sum_{k,l} R_k^l(d/h_P) 2^{-(n-k)} Mt_{n-k}^{m-l}(C)
//   M2L  source -> target         Lt_k^l(t) += (-1)^k sum_{n,m} rho^n Mt_n^m(s) conj(I_{n+k}^{m+l}(D/h_t)),
//                                 rho = h_s/h_t, D = c_t - c_s
//   L2L  parent -> child          Lt_k^l(C) += 2^{-(k+1)} sum_{n>=k,m} Lt_n^m(P) R_{n-k}^{m-l}(d/h_P)
//   L2P  local -> particles       phi = (1/h) sum Lt_k^l R_k^l(u), grad phi = (1/h^2) sum Lt grad R(u)
//   P2P  near field               phi_i += q_j / r_ij,  grad phi_i -= q_j (x_i - x_j) / r_ij^3
//
// R and I are the regular and irregular solid harmonics with the
// normalisation R_n^m = r^n P_n^m e^{im phi}/(n+m)!, I_n^m = (n-m)! P_n^m e^{im phi}/r^{n+1}
// (P_n^m without the Condon-Shortley phase), for which the Laplace addition
// theorem takes the forms above.  Interaction is non-mutual (Section 4):
// every kernel writes only its target cell or target particles.
#include <algorithm>
#include <type_traits>

#include "fmm_internal.cuh"
#include "stages.cuh"

namespace fmm {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// prepare: sorted (x, y, z, q) for P2P and sorted charges for P2M
// ---------------------------------------------------------------------------

template <typename Q>
__global__ void k_prepare64(const double* __restrict__ spos, const int32_t* __restrict__ perm,
                            const Q* __restrict__ q, int64_t n, double4_32a* xq) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    xq[i] = make_double4_32a(spos[3 * i], spos[3 * i + 1], spos[3 * i + 2], (double)q[perm[i]]);
}

// FP32 copy relative to the centre of the particle's own leaf, so that the
// rounding of a coordinate scales with the leaf size, not with the position;
// xlo: what that rounding dropped (FP32 again), for very close pairs within a leaf.
template <typename Q>
__global__ void k_prepare32(const double* __restrict__ spos, const int32_t* __restrict__ perm,
                            const Q* __restrict__ q, int64_t n, const int32_t* __restrict__ pleaf,
                            const double4_32a* __restrict__ centre, double4_32a* xq64, float4* xq32, float4* xlo) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = spos[3 * i], y = spos[3 * i + 1], z = spos[3 * i + 2], qq = (double)q[perm[i]];
    xq64[i] = make_double4_32a(x, y, z, qq);
    double4_32a c = centre[pleaf[i]];
    const double dx = x - c.x, dy = y - c.y, dz = z - c.z;
    const float hx = (float)dx, hy = (float)dy, hz = (float)dz;
    xq32[i] = make_float4(hx, hy, hz, (float)qq);
    xlo[i] = make_float4((float)(dx - (double)hx), (float)(dy - (double)hy), (float)(dz - (double)hz), 0.f);
}

// Dense real forms of the child <-> parent shifts, one per octant (the shift
// d/h_P = (+-1/4, +-1/4, +-1/4) depends only on the octant).  For an input
// coefficient X = Xt_{n'}^{m'} (m' >= 0) the shift adds a X + b conj(X) to an
// output coefficient (b from the order -m' term), i.e. a real 2 x 2 block:
//   re += (a.re + b.re) X.re + (b.im - a.im) X.im,  im += (a.im + b.im) X.re + (a.re - b.re) X.im
//   M2M: out (n, m) <- in (n', m'):  a = R_{n-n'}^{m-m'} 2^-n',  b = (-1)^m' R_{n-n'}^{m+m'} 2^-n'
//   L2L: out (k, l) <- in (n, m):    a = R_{n-k}^{m-l} 2^-(k+1), b = (-1)^m R_{n-k}^{-m-l} 2^-(k+1)
// Stored input-major (row = input index) so that lanes reading consecutive
// outputs read consecutive words.  ops[kind][octant][in][out], kind 0 = M2M, 1 = L2L.
template <typename T>
__global__ void k_shift_operators(int p, T* ops) {
    extern __shared__ unsigned char smraw[];
    cplx<double>* R = reinterpret_cast<cplx<double>*>(smraw);
    const int kind = blockIdx.x >> 3, o = blockIdx.x & 7, K = ntri(p), K2 = 2 * K;
    if (threadIdx.x == 0)
        regular_harmonics<double>(p, (o & 1) ? 0.25 : -0.25, (o & 2) ? 0.25 : -0.25, (o & 4) ? 0.25 : -0.25, R);
    __syncthreads();
    T* out = ops + (size_t)blockIdx.x * K2 * K2;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        int jo = e / K, ji = e % K;   // output / input complex index
        int no = 0, ni = 0;
        while (tri(no + 1, 0) <= jo) no++;
        while (tri(ni + 1, 0) <= ji) ni++;
        int mo = jo - tri(no, 0), mi = ji - tri(ni, 0);
        cplx<double> a = {0, 0}, b = {0, 0};
        if (kind == 0 && ni <= no) {
            double sc = ldexp(1.0, -ni);
            a = get_sym(R, no - ni, mo - mi);
            if (mi > 0) b = get_sym(R, no - ni, mo + mi);
            if (mi & 1) { b.re = -b.re; b.im = -b.im; }
            a.re *= sc; a.im *= sc; b.re *= sc; b.im *= sc;
        } else if (kind == 1 && ni >= no) {
            double sc = ldexp(1.0, -(no + 1));
            a = get_sym(R, ni - no, mi - mo);
            if (mi > 0) b = get_sym(R, ni - no, -mi - mo);
            if (mi & 1) { b.re = -b.re; b.im = -b.im; }
            a.re *= sc; a.im *= sc; b.re *= sc; b.im *= sc;
        }
        // rows: inputs (2 ji + re|im), columns: outputs (2 jo + re|im)
        T* r0 = out + (size_t)(2 * ji) * K2 + 2 * jo;
        T* r1 = r0 + K2;
        r0[0] = (T)(a.re + b.re);
        r0[1] = (T)(a.im + b.im);
        r1[0] = mi > 0 ? (T)(b.im - a.im) : T(0);
        r1[1] = mi > 0 ? (T)(a.re - b.re) : T(0);
    }
}

// ---------------------------------------------------------------------------
// stage-by-stage kernels (bodies in stages.cuh)
// ---------------------------------------------------------------------------

// one warp per destination cell of one level
template <typename T, int RQ>
__global__ void __launch_bounds__(128) k_shift_dense(int p, int lb, int le, int kind,
                                                     const int32_t* __restrict__ child_first,
                                                     const int32_t* __restrict__ child_count,
                                                     const int32_t* __restrict__ parent,
                                                     const uint64_t* __restrict__ ckey, const T* __restrict__ ops,
                                                     cplx<T>* __restrict__ E) {
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* xin = reinterpret_cast<T*>(smem_raw) + warp * 2 * ntri(p);
    const int c = lb + blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= le) return;
    shift_cell<T, RQ, false>(p, c, kind, lane, child_first, child_count, parent, ckey, ops, E, xin);
}

// FP32, many destination cells (the fine levels): block (x, o) takes the
// (destination, input) pairs of octant o among destination cells
// lb + ndst x ... + ndst - 1 (M2M: a parent and its child in octant o; L2L: a
// child in octant o and its parent).  Pairs go through in chunks of 32 rows;
// thread (lane, warp g) computes outputs lane + 32 q of rows 4 g .. 4 g + 3
// with the octant's operator read through L1.  M2M results from the eight
// octants meet by FP32 atomics in parents zeroed beforehand; an L2L
// destination has one octant and is updated in place.
constexpr int SHO_THREADS = 256, SHO_CHUNK = 32;
static int shift_oct_ndst(int kind) { return kind == 0 ? 32 : 256; }

template <int RQ>
__global__ void __launch_bounds__(SHO_THREADS) k_shift_oct(int p, int lb, int le, int kind, int ndst,
                                                           const int32_t* __restrict__ child_first,
                                                           const int32_t* __restrict__ child_count,
                                                           const int32_t* __restrict__ parent,
                                                           const uint64_t* __restrict__ ckey,
                                                           const float* __restrict__ ops, cplx<float>* __restrict__ E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K2 = 2 * ntri(p), ld = 2 * kstride(p);
    float* xin = reinterpret_cast<float*>(smem_raw);
    int* pd = reinterpret_cast<int*>(xin + (size_t)SHO_CHUNK * K2);   // destination cell
    int* ps = pd + ndst;                                                 // input cell
    __shared__ int npair;
    float* Ef = reinterpret_cast<float*>(E);
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5, o = blockIdx.y;
    const int c0 = lb + blockIdx.x * ndst, nd = min(ndst, le - c0);
    if (tid == 0) npair = 0;
    __syncthreads();
    for (int d = tid; d < nd; d += SHO_THREADS) {
        const int c = c0 + d;
        int src = -1;
        if (kind == 0) {
            const int f = child_first[c], nc = child_count[c];
            for (int k = 0; k < nc; k++)
                if ((int)(ckey[f + k] & 7) == o) { src = f + k; break; }
        } else if ((int)(ckey[c] & 7) == o) {
            src = parent[c];
        }
        if (src >= 0) {
            const int slot = atomicAdd(&npair, 1);
            pd[slot] = c;
            ps[slot] = src;
        }
    }
    __syncthreads();
    const int np = npair;
    const float* op = ops + (size_t)(kind * 8 + o) * K2 * K2;
    for (int pc = 0; pc < np; pc += SHO_CHUNK) {
        const int npc = min(SHO_CHUNK, np - pc);
        for (int e = tid; e < npc * K2; e += SHO_THREADS) {
            const int r = e / K2, i = e - r * K2;
            xin[e] = Ef[(size_t)ps[pc + r] * ld + i];
        }
        __syncthreads();
        if (4 * g < npc) {
            float a[4][RQ];
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int q = 0; q < RQ; q++) a[u][q] = 0.f;
            for (int i = 0; i < K2; i++) {
                float w[RQ];
#pragma unroll
                for (int q = 0; q < RQ; q++) {
                    const int j = lane + 32 * q;
                    w[q] = j < K2 ? __ldg(op + (size_t)i * K2 + j) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const float x = xin[(4 * g + u) * K2 + i];
#pragma unroll
                    for (int q = 0; q < RQ; q++) a[u][q] = fmaf(w[q], x, a[u][q]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int r = 4 * g + u;
                if (r < npc) {
                    float* er = Ef + (size_t)pd[pc + r] * ld;
#pragma unroll
                    for (int q = 0; q < RQ; q++) {
                        const int j = lane + 32 * q;
                        if (j < K2) {
                            if (kind == 0) atomicAdd(er + j, a[u][q]);
                            else er[j] += a[u][q];
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// M of the cells with children set to zero (their M2M results are sums of
// atomics); leaves keep the multipoles P2M wrote
__global__ void k_zero_parents(int64_t ncell, int ld, const int32_t* __restrict__ child_count, float* __restrict__ M) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ncell * ld) return;
    if (child_count[e / ld] > 0) M[e] = 0.f;
}

// one block per destination cell of one level (NW warps)
template <typename T, int RQ, int NW>
__global__ void __launch_bounds__(32 * NW) k_shift_block(int p, int lb, int le, int kind,
                                                         const int32_t* __restrict__ child_first,
                                                         const int32_t* __restrict__ child_count,
                                                         const int32_t* __restrict__ parent,
                                                         const uint64_t* __restrict__ ckey, const T* __restrict__ ops,
                                                         cplx<T>* __restrict__ E) {
    extern __shared__ unsigned char smem_raw[];
    const int K2 = 2 * ntri(p);
    T* xin = reinterpret_cast<T*>(smem_raw);
    T* red = xin + NW * K2;
    const int c = lb + blockIdx.x;
    if (c >= le) return;
    if (kind == 0 && child_count[c] == 0) return;
    shift_cell_block<T, RQ, NW, false>(p, c, kind, child_first, child_count, parent, ckey, ops, E, xin, red,
                                       (int)(threadIdx.x >> 5), (int)threadIdx.x, BlockSync{});
}

// One warp per leaf, one particle per lane (32 at a time).  Each lane builds its
// particle's regular harmonics column by column (order m outer, degree n inner,
// the recurrence of p2m_leaf with the reciprocals from tables holding the values
// the divisions give, so every term is the same); a column goes to shared
// memory and the lane owning row r sums the column's entry n = m + r over the
// lanes with four independent partial sums.  No shuffle reduction per
// coefficient: the warp's dependent chains are 32 / 4 adds per column instead of
// five shuffle levels per coefficient.  Shared memory per warp: a column of
// p + 1 rows x 33 (padded) entries and the leaf's K accumulators.
constexpr int P2M_WARPS = 4;
template <typename T>
__host__ __device__ inline size_t p2m_warp_smem(int p) {
    return ((size_t)(p + 1) * 33 + ntri(p)) * sizeof(cplx<T>);
}
template <typename T>
__global__ void __launch_bounds__(32 * P2M_WARPS) k_p2m(int p, int nleaf, const int32_t* __restrict__ leaves,
                                                        const int32_t* __restrict__ first,
                                                        const int32_t* __restrict__ count,
                                                        const double4_32a* __restrict__ centre,
                                                        const double4_32a* __restrict__ xq, cplx<T>* __restrict__ M) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ T rm[FMM_MAX_P + 1], rt[(FMM_MAX_P + 1) * (FMM_MAX_P + 2) / 2];
    for (int m = threadIdx.x; m <= p; m += blockDim.x) rm[m] = m > 0 ? T(1) / T(2 * m) : T(0);
    for (int n = 0; n <= p; n++)
        for (int m = threadIdx.x; m <= n; m += blockDim.x) rt[tri(n, m)] = n >= m + 2 ? T(1) / T((n + m) * (n - m)) : T(0);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * (blockDim.x >> 5) + warp;
    if (li >= nleaf) return;
    const int K = ntri(p), KS = kstride(p);
    cplx<T>* col = reinterpret_cast<cplx<T>*>(smem_raw + (size_t)warp * p2m_warp_smem<T>(p));
    cplx<T>* acc = col + (size_t)(p + 1) * 33;
    for (int j = lane; j < K; j += 32) acc[j] = cmk<T>(0, 0);
    const int c = leaves[li];
    const double4_32a cc = centre[c];
    const double invh = 1.0 / cc.w;
    const int f = first[c], cnt = count[c];
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        T ux = 0, uy = 0, uz = 0, q = 0;
        if (i < cnt) {
            const double4_32a a = xq[f + i];
            ux = (T)((a.x - cc.x) * invh); uy = (T)((a.y - cc.y) * invh); uz = (T)((a.z - cc.z) * invh);
            q = (T)a.w;
        }
        const T r2 = ux * ux + uy * uy + uz * uz;
        cplx<T> rmm = cmk<T>(q, 0);
        for (int m = 0; m <= p; m++) {
            if (m > 0) rmm = cscale(cmul(rmm, cmk<T>(ux, uy)), rm[m]);
            cplx<T> a = rmm, b = cscale(rmm, uz);
            for (int n = m; n <= p; n++) {
                cplx<T> v;
                if (n == m) v = a;
                else if (n == m + 1) v = b;
                else {
                    const T inv = rt[tri(n, m)];
                    v = cmk<T>((T(2 * n - 1) * uz * b.re - r2 * a.re) * inv, (T(2 * n - 1) * uz * b.im - r2 * a.im) * inv);
                    a = b; b = v;
                }
                col[(n - m) * 33 + lane] = v;
            }
            __syncwarp();
            if (lane <= p - m) {
                const cplx<T>* row = col + lane * 33;
                cplx<T> s0 = row[0], s1 = row[1], s2 = row[2], s3 = row[3];
#pragma unroll
                for (int l = 4; l < 32; l += 4) {
                    s0 = cadd(s0, row[l]); s1 = cadd(s1, row[l + 1]);
                    s2 = cadd(s2, row[l + 2]); s3 = cadd(s3, row[l + 3]);
                }
                cplx<T>& o = acc[tri(m + lane, m)];
                o = cadd(o, cadd(cadd(s0, s1), cadd(s2, s3)));
            }
            __syncwarp();
        }
    }
    __syncwarp();
    for (int j = lane; j < K; j += 32) M[(int64_t)c * KS + j] = acc[j];
}

// M2L (any pair of cells): one warp per target, each half-warp one source
// at a time; lane (h, i) accumulates the outputs j = i, i + 16, ...
template <typename T, int RMAX>
__global__ void __launch_bounds__(128) k_m2l_generic(int p, int t0, int t1, const int64_t* __restrict__ start,
                                                     const int32_t* __restrict__ src,
                                                     const double4_32a* __restrict__ centre,
                                                     const cplx<T>* __restrict__ M, cplx<T>* __restrict__ L) {
    extern __shared__ unsigned char smem_raw[];
    const int K = ntri(p), KI = ntri(2 * p), KS = kstride(p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    cplx<T>* Ms = reinterpret_cast<cplx<T>*>(smem_raw) + (warp * 2 + half) * (K + KI);
    cplx<T>* Is = Ms + K;
    const int t = t0 + blockIdx.x * (blockDim.x >> 5) + warp;
    if (t >= t1) return;
    int kk[RMAX], ll[RMAX];
    cplx<T> acc[RMAX];
    m2l_output_index<RMAX>(p, hl, kk, ll);
#pragma unroll
    for (int r = 0; r < RMAX; r++) acc[r] = cmk<T>(0, 0);
    m2l_slot<T, RMAX, false>(p, t, half, 2, hl, start, src, centre, M, Ms, Is, kk, ll, acc);
#pragma unroll
    for (int r = 0; r < RMAX; r++) {
        acc[r].re += __shfl_xor_sync(0xffffffffu, acc[r].re, 16);
        acc[r].im += __shfl_xor_sync(0xffffffffu, acc[r].im, 16);
    }
    if (half == 0) {
#pragma unroll
        for (int r = 0; r < RMAX; r++) {
            const int j = hl + 16 * r;
            if (j < K) L[(int64_t)t * KS + j] = cscale(acc[r], (kk[r] & 1) ? T(-1) : T(1));
        }
    }
}

// CUDA-core M2L over chunks of at most M2L_CHUNK list entries of one target
// (chunks[c] = (target, first entry)), one warp per chunk, results added into
// L with FP32 atomics (L zeroed beforehand): a target with thousands of
// entries is spread over many warps.  Used for the pairs the tensor cores do
// not take in the mixed form, which concentrate on a few coarse targets.
template <int RMAX>
__global__ void __launch_bounds__(128) k_m2l_chunks(int p, int64_t nchunk, const int2* __restrict__ chunks,
                                                    const int64_t* __restrict__ start, const int32_t* __restrict__ src,
                                                    const double4_32a* __restrict__ centre,
                                                    const cplx<float>* __restrict__ M, float* __restrict__ L) {
    extern __shared__ unsigned char smem_raw[];
    const int K = ntri(p), KI = ntri(2 * p), KS = kstride(p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    cplx<float>* Ms = reinterpret_cast<cplx<float>*>(smem_raw) + (warp * 2 + half) * (K + KI);
    cplx<float>* Is = Ms + K;
    const int64_t c = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
    if (c >= nchunk) return;
    const int2 ch = chunks[c];
    const int t = ch.x;
    const int64_t s0 = ch.y, s1 = min(start[t + 1], s0 + (int64_t)M2L_CHUNK);
    int kk[RMAX], ll[RMAX];
    cplx<float> acc[RMAX];
    m2l_output_index<RMAX>(p, hl, kk, ll);
#pragma unroll
    for (int r = 0; r < RMAX; r++) acc[r] = cmk<float>(0, 0);
    m2l_range<float, RMAX, false>(p, t, s0, s1, half, 2, hl, src, centre, M, Ms, Is, kk, ll, acc);
#pragma unroll
    for (int r = 0; r < RMAX; r++) {
        acc[r].re += __shfl_xor_sync(0xffffffffu, acc[r].re, 16);
        acc[r].im += __shfl_xor_sync(0xffffffffu, acc[r].im, 16);
    }
    if (half == 0) {
#pragma unroll
        for (int r = 0; r < RMAX; r++) {
            const int j = hl + 16 * r;
            if (j < K) {
                const float sg = (kk[r] & 1) ? -1.f : 1.f;
                atomicAdd(L + 2 * ((int64_t)t * KS + j), sg * acc[r].re);
                atomicAdd(L + 2 * ((int64_t)t * KS + j) + 1, sg * acc[r].im);
            }
        }
    }
}

// One work item per block: a leaf's whole list, or a run of the records of a
// split leaf's list.  The k items of a split leaf write their sums to their
// own partial slots; the block that finishes last (a counter per leaf, reset
// by that block) adds the k slots in item order into near, so the result does
// not depend on the order the blocks ran in.  FP32: registers capped for 9
// resident blocks per SM, measured 2 % faster than the uncapped 62 registers.
template <typename T>
__global__ void __launch_bounds__(P2P_THREADS, sizeof(T) == 4 ? 9 : 1) k_p2p(const int4* __restrict__ items,
                                                     const int32_t* __restrict__ nitems,
                                                     const int4* __restrict__ split, int32_t* __restrict__ arrived,
                                                     double* __restrict__ partial,
                                                     const int32_t* __restrict__ first,
                                                     const int32_t* __restrict__ count,
                                                     const int64_t* __restrict__ start,
                                                     const int4* __restrict__ rec,
                                                     const typename Vec4<T>::type* __restrict__ xq,
                                                     const float4* __restrict__ xlo,
                                                     const int4* __restrict__ icentre, const float* __restrict__ cu2f,
                                                     double* __restrict__ near) {
    __shared__ typename Vec4<T>::type buf[P2P_BUF];
    __shared__ T part[P2P_THREADS][4];
    __shared__ int last;
    if ((int)blockIdx.x >= *nitems) return;   // the grid may be an upper bound
    const int4 it = items[blockIdx.x];
    const int64_t s0 = start[it.x] + it.y;
    if (!(it.w & 1)) {
        p2p_range<T>(it.x, s0, s0 + it.z, sizeof(T) == 8 && (it.w & 2) != 0, nullptr, first, count, rec, xq, xlo,
                     icentre, cu2f, near, buf, part, threadIdx.x);
        return;
    }
    // split leaf: si = (items k, this item's rank j, partial slot base lo / hi)
    const int4 si = split[blockIdx.x];
    const int nt = count[it.x];
    const int64_t pbase = (int64_t)(uint32_t)si.z | ((int64_t)si.w << 32);   // slot of (j = 0, target 0)
    p2p_range<T>(it.x, s0, s0 + it.z, sizeof(T) == 8 && (it.w & 2) != 0, partial + 4 * (pbase + (int64_t)si.y * nt),
                 first, count, rec, xq, xlo, icentre, cu2f, near, buf, part, threadIdx.x);
    __threadfence();
    __syncthreads();
    int32_t* ctr = arrived + (blockIdx.x - si.y);   // the leaf's first item
    if (threadIdx.x == 0) last = atomicAdd(ctr, 1) == si.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int tf = first[it.x];
    for (int t = threadIdx.x; t < nt; t += P2P_THREADS) {
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int j = 0; j < si.x; j++) {
            const double* q = partial + 4 * (pbase + (int64_t)j * nt + t);
            a0 += __ldcg(q); a1 += __ldcg(q + 1); a2 += __ldcg(q + 2); a3 += __ldcg(q + 3);
        }
        double* o = near + 4 * ((int64_t)tf + t);
        o[0] = a0; o[1] = a1; o[2] = a2; o[3] = a3;
    }
    if (threadIdx.x == 0) *ctr = 0;   // ready for the next evaluation
}

// FP32 P2P: the pairs within each leaf, after k_p2p (which stages a leaf's own
// particles at zero charge), added into near (acc given: the mutual form, near =
// acc + the leaf's own pairs).  One warp per leaf, a lane per
// target.  Separations come from the leaf-relative FP32 coordinates plus the
// difference of their residuals, so two particles much closer than the leaf's
// side keep their separation to FP32 precision; coincident pairs (separation
// at or below FLT_MIN) contribute nothing.
constexpr int P2P_OWN_WARPS = 4;
__global__ void __launch_bounds__(32 * P2P_OWN_WARPS) k_p2p_own(int nleaf, const int32_t* __restrict__ leaves,
                                                                const int32_t* __restrict__ first,
                                                                const int32_t* __restrict__ count,
                                                                const float4* __restrict__ xq,
                                                                const float4* __restrict__ xlo,
                                                                const float4* __restrict__ acc,
                                                                double* __restrict__ near) {
    __shared__ float4 sh[P2P_OWN_WARPS][32], sl[P2P_OWN_WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int li = blockIdx.x * P2P_OWN_WARPS + warp;
    if (li >= nleaf) return;
    const int c = leaves[li], tf = first[c], nt = count[c];
    for (int base = 0; base < nt; base += 32) {
        const int i = base + lane;
        const bool valid = i < nt;
        const float4 a = valid ? xq[tf + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 al = valid ? xlo[tf + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        for (int jb = 0; jb < nt; jb += 32) {
            __syncwarp();
            if (jb + lane < nt) { sh[warp][lane] = xq[tf + jb + lane]; sl[warp][lane] = xlo[tf + jb + lane]; }
            __syncwarp();
            const int nj = min(32, nt - jb);
            for (int j = 0; j < nj; j++) {
                const float4 s = sh[warp][j], l = sl[warp][j];
                const float dx = (a.x - s.x) + (al.x - l.x), dy = (a.y - s.y) + (al.y - l.y),
                            dz = (a.z - s.z) + (al.z - l.z);
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const float rinv = r2 > pair_floor(r2) ? rsqrt_t(r2) : 0.f;
                const float qr = s.w * rinv;
                ph += qr;
                const float qr3 = qr * rinv * rinv;
                gx = fmaf(-qr3, dx, gx); gy = fmaf(-qr3, dy, gy); gz = fmaf(-qr3, dz, gz);
            }
        }
        if (valid) {
            double* o = near + 4 * ((int64_t)tf + i);
            if (acc) {   // the mutual form's sums of the other leaves
                const float4 b = acc[tf + i];
                o[0] = (double)b.x + (double)ph; o[1] = (double)b.y + (double)gx;
                o[2] = (double)b.z + (double)gy; o[3] = (double)b.w + (double)gz;
            } else {
                o[0] += (double)ph; o[1] += (double)gx; o[2] += (double)gy; o[3] += (double)gz;
            }
        }
    }
}

// L2P + near field + output in input order, one thread per sorted particle
// (its leaf from pleaf; the leaf's local expansion read through L1, shared by
// the leaf's particles), with the recurrence's reciprocals from tables
constexpr int L2P_THREADS = 256;
template <typename T, typename O>
__global__ void __launch_bounds__(L2P_THREADS) k_l2p_points(int p, int64_t n, const int32_t* __restrict__ pleaf,
                                                            const double4_32a* __restrict__ centre,
                                                            const double4_32a* __restrict__ xq,
                                                            const int32_t* __restrict__ perm,
                                                            const cplx<T>* __restrict__ L,
                                                            const double* __restrict__ near, O* __restrict__ phi_out,
                                                            O* __restrict__ force_out, int field) {
    __shared__ T rm[FMM_MAX_P + 1], rt[(FMM_MAX_P + 1) * (FMM_MAX_P + 2) / 2];
    for (int m = threadIdx.x; m <= p; m += blockDim.x) rm[m] = m > 0 ? T(1) / T(2 * m) : T(0);
    for (int n = 0; n <= p; n++)
        for (int m = threadIdx.x; m <= n; m += blockDim.x) rt[tri(n, m)] = n >= m + 2 ? T(1) / T((n + m) * (n - m)) : T(0);
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = pleaf[i];
    const double4_32a cc = centre[c];
    const double invh = 1.0 / cc.w;
    const double4_32a a = xq[i];
    const T ux = (T)((a.x - cc.x) * invh), uy = (T)((a.y - cc.y) * invh), uz = (T)((a.z - cc.z) * invh);
    T fp, gx, gy, gz;
    l2p_point<T, true>(p, ux, uy, uz, L + (int64_t)c * kstride(p), rm, rt, fp, gx, gy, gz);
    l2p_store<T, O, false>(i, invh, a.w, fp, gx, gy, gz, perm, near, phi_out, force_out, field);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static bool exp_fp64(const fmm_tree* t) {
    return t->prm.precision == FMM_PREC_FP64 || t->prm.precision == FMM_PREC_FP32_P2P;
}
static bool p2p_fp64(const fmm_tree* t) { return t->prm.precision == FMM_PREC_FP64; }

int alloc_eval_workspace(fmm_tree* t, cudaStream_t st) {
    int rc;
    TreeDev& d = t->d;
    if (t->n == 0) return FMM_OK;
    size_t K = (size_t)kstride(t->prm.p);
    size_t csz = exp_fp64(t) ? sizeof(cplx<double>) : sizeof(cplx<float>);
    char *M = nullptr, *L = nullptr, *xq = nullptr;
    if ((rc = dev_alloc(&M, (size_t)t->ncell * K * csz, t, st))) return rc;
    if ((rc = dev_alloc(&L, (size_t)t->ncell * K * csz, t, st))) return rc;
    // double4_32a copy always (P2M/L2P positions), plus float4 for FP32 P2P
    // (and, for the mutual near field, a float4 accumulator per particle)
    size_t xb = (size_t)t->n * sizeof(double4_32a) +
                (p2p_fp64(t) ? 0 : (size_t)(p2p_mutual(t) ? 3 : 2) * t->n * sizeof(float4));
    if ((rc = dev_alloc(&xq, xb, t, st))) return rc;
    if ((rc = dev_alloc(&d.near, (size_t)t->n * 4, t, st))) return rc;
    d.M = M; d.L = L; d.xq = xq;
    // partial slots of the split P2P leaves: their number comes back from the
    // build through the pinned words (the build's work has to finish before it
    // returns anyway, so waiting for it here costs next to nothing)
    if (t->h_pin && (d.p2p_items || t->rem_nchunk < 0)) {
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
        if (d.p2p_items) {
            const int64_t nslot = (int64_t)(uint32_t)t->h_pin[2] | ((int64_t)t->h_pin[3] << 32);
            if (nslot > 0 && (rc = dev_alloc(&d.p2p_part, (size_t)nslot * 4, t, st))) return rc;
        }
        if (t->rem_nchunk < 0) t->rem_nchunk = t->h_pin[4];
    }
    {
        const int K2 = 2 * ntri(t->prm.p);
        size_t tsz = exp_fp64(t) ? sizeof(double) : sizeof(float);
        char* ops = nullptr;
        if ((rc = dev_alloc(&ops, (size_t)16 * K2 * K2 * tsz, t, st))) return rc;
        d.shift_ops = ops;
        size_t smem = (size_t)ntri(t->prm.p) * sizeof(cplx<double>);
        if (exp_fp64(t))
            k_shift_operators<double><<<16, 256, smem, st>>>(t->prm.p, (double*)ops);
        else
            k_shift_operators<float><<<16, 256, smem, st>>>(t->prm.p, (float*)ops);
        count_launch(t);
    }
    if (t->prm.precision == FMM_PREC_MIXED_TC && tc_supported(t->prm.p) && (t->tc_nitems > 0 || tc_uses_dag(t))) {
        char* ms = nullptr;
        if ((rc = dev_alloc(&ms, (size_t)t->ncell * 2 * tc_kin(t->prm.p) * 2, t, st))) return rc;
        d.tc_msplit = ms;
        char* lr = nullptr;
        if ((rc = dev_alloc(&lr, (size_t)t->ncell * 128 * sizeof(float), t, st))) return rc;
        d.tc_lr = lr;
    }
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

template <typename T>
static int launch_shift(fmm_tree* t, int kind, int lb, int le, cplx<T>* E, cudaStream_t st) {
    const int p = t->prm.p, K2 = 2 * ntri(p), W = 4;
    if (le <= lb) return FMM_OK;
    const TreeDev& d = t->d;
    const T* ops = (const T*)d.shift_ops;
    int rq = (K2 + 31) / 32;
    // few cells (the top levels): a block of warps per cell splits the inputs;
    // many cells: one warp per cell
    const bool block_mode = (le - lb) < 8 * t->num_sms;
    const int NWB = kind == 0 ? 8 : 4;
    size_t smem = block_mode ? (size_t)2 * NWB * K2 * sizeof(T) : (size_t)W * K2 * sizeof(T);
    unsigned grid = block_mode ? (unsigned)(le - lb) : nblk(le - lb, W);
    // many cells, FP32: one block per (run of destination cells, octant)
    const int ndst = shift_oct_ndst(kind);
    const size_t osmem = sizeof(float) * (size_t)SHO_CHUNK * K2 + 2 * sizeof(int) * ndst;
#define SHIFT_CASE(R)                                                                                         \
    if (rq <= R) {                                                                                            \
        if (block_mode && kind == 0) {                                                                        \
            if (smem > 48 * 1024)                                                                             \
                FMM_CUDA_TRY(cudaFuncSetAttribute(k_shift_block<T, R, 8>,                                     \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));    \
            k_shift_block<T, R, 8><<<grid, 256, smem, st>>>(p, lb, le, kind, d.child_first, d.child_count,     \
                                                            d.parent, d.ckey, ops, E);                        \
        } else if (block_mode) {                                                                              \
            if (smem > 48 * 1024)                                                                             \
                FMM_CUDA_TRY(cudaFuncSetAttribute(k_shift_block<T, R, 4>,                                     \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));    \
            k_shift_block<T, R, 4><<<grid, 128, smem, st>>>(p, lb, le, kind, d.child_first, d.child_count,     \
                                                            d.parent, d.ckey, ops, E);                        \
        } else if constexpr (sizeof(T) == 4) {                                                                \
            k_shift_oct<R><<<dim3(nblk(le - lb, ndst), 8), SHO_THREADS, osmem, st>>>(                         \
                p, lb, le, kind, ndst, d.child_first, d.child_count, d.parent, d.ckey, (const float*)ops,     \
                (cplx<float>*)E);                                                                             \
        } else {                                                                                              \
            k_shift_dense<T, R><<<grid, 32 * W, smem, st>>>(p, lb, le, kind, d.child_first, d.child_count,     \
                                                            d.parent, d.ckey, ops, E);                        \
        }                                                                                                     \
        count_launch(t);                                                                                      \
        FMM_CUDA_TRY(cudaGetLastError());                                                                     \
        return FMM_OK;                                                                                        \
    }
    SHIFT_CASE(1) SHIFT_CASE(2) SHIFT_CASE(3) SHIFT_CASE(5) SHIFT_CASE(8) SHIFT_CASE(12) SHIFT_CASE(15)
#undef SHIFT_CASE
    fmm_set_error("order too high for the shift kernel");
    return FMM_ERR_ARG;
}

template <typename T>
static int launch_m2l_generic(fmm_tree* t, int p, int t0, int t1, const int64_t* start, const int32_t* src,
                              const TreeDev& d, const cplx<T>* M, cplx<T>* L, cudaStream_t st) {
    if (t1 <= t0) return FMM_OK;
    const int K = ntri(p), KI = ntri(2 * p), KS = kstride(p);
    size_t smem = (size_t)4 * 2 * (K + KI) * sizeof(cplx<T>);
    int rmax = (K + 15) / 16;
    unsigned grid = nblk(t1 - t0, 4);
#define M2L_CASE(R)                                                                                   \
    if (rmax <= R) {                                                                                  \
        if (smem > 48 * 1024)                                                                         \
            FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_generic<T, R>,                                    \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_m2l_generic<T, R><<<grid, 128, smem, st>>>(p, t0, t1, start, src, d.centre, M, L);               \
        count_launch(t);                                                                              \
        return FMM_OK;                                                                                \
    }
    M2L_CASE(2) M2L_CASE(4) M2L_CASE(6) M2L_CASE(8) M2L_CASE(12) M2L_CASE(16)
#undef M2L_CASE
    fmm_set_error("order too high for the M2L kernel");
    return FMM_ERR_ARG;
}

static int launch_m2l_chunks(fmm_tree* t, int p, const TreeDev& d, const cplx<float>* M, float* L, cudaStream_t st) {
    const int K = ntri(p), KI = ntri(2 * p);
    const size_t smem = (size_t)4 * 2 * (K + KI) * sizeof(cplx<float>);
    const int rmax = (K + 15) / 16;
    const unsigned grid = nblk(t->rem_nchunk, 4);
    const int32_t* src = d.tc_src + t->tc_npairs;
#define M2LC_CASE(R)                                                                                       \
    if (rmax <= R) {                                                                                       \
        if (smem > 48 * 1024)                                                                              \
            FMM_CUDA_TRY(cudaFuncSetAttribute(k_m2l_chunks<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_m2l_chunks<R><<<grid, 128, smem, st>>>(p, t->rem_nchunk, d.rem_chunks, d.rem_start, src, d.centre, M, L); \
        count_launch(t);                                                                                   \
        FMM_CUDA_TRY(cudaGetLastError());                                                                  \
        return FMM_OK;                                                                                     \
    }
    M2LC_CASE(2) M2LC_CASE(4) M2LC_CASE(6) M2LC_CASE(8) M2LC_CASE(12) M2LC_CASE(16)
#undef M2LC_CASE
    fmm_set_error("order too high for the M2L kernel");
    return FMM_ERR_ARG;
}

template <typename T>
static int far_field(fmm_tree* t, cplx<T>* M, cplx<T>* L, const double4_32a* xq64, cudaStream_t st);

template <typename T, typename Q, typename O>
static int evaluate_typed(fmm_tree* t, const Q* q, O* phi, O* force, cudaStream_t st) {
    const int p = t->prm.p, K = ntri(p);
    TreeDev& d = t->d;
    const int64_t n = t->n;
    double4_32a* xq64 = (double4_32a*)d.xq;
    float4* xq32 = (float4*)((char*)d.xq + (size_t)n * sizeof(double4_32a));
    float4* xlo32 = xq32 + n;   // residuals of the FP32 coordinates (FP32 P2P only)
    float4* acc32 = xq32 + 2 * n;   // mutual near field: sums of both leaves of every pair
    cplx<T>* M = (cplx<T>*)d.M;
    cplx<T>* L = (cplx<T>*)d.L;
    // particles in sorted order
    stage_begin(t, FMM_STAGE_PREPARE, st);
    if (p2p_fp64(t))
        k_prepare64<Q><<<nblk(n, 256), 256, 0, st>>>(d.spos, d.perm, q, n, xq64);
    else
        k_prepare32<Q><<<nblk(n, 256), 256, 0, st>>>(d.spos, d.perm, q, n, d.pleaf, d.centre, xq64, xq32, xlo32);
    count_launch(t);
    stage_end(t, FMM_STAGE_PREPARE, st);
    if constexpr (sizeof(T) == 4) {
        if (tc_uses_dag(t)) return evaluate_dag<O>(t, xq64, xq32, xlo32, phi, force, st);
    }
    if (queue_supported(t)) {
        // one persistent launch runs the whole task graph
        if constexpr (std::is_same<T, double>::value) {
            if (p2p_fp64(t)) return evaluate_queue<T, double, O>(t, xq64, xq64, phi, force, st);
        }
        return evaluate_queue<T, float, O>(t, xq64, xq32, phi, force, st, xlo32);
    }
    // P2P (near field) depends on nothing but the particles: it runs on the
    // tree's second stream, concurrently with the upward pass, M2L and L2L,
    // and joins before L2P (the far field and the near field meet there)
    const bool overlap = !(t->prm.flags & FMM_NO_OVERLAP);
    cudaStream_t sp = (overlap && t->side_stream) ? t->side_stream : st;
    if (sp != st) {
        FMM_CUDA_TRY(cudaEventRecord(t->ev_fork, st));
        FMM_CUDA_TRY(cudaStreamWaitEvent(sp, t->ev_fork, 0));
    }
    stage_begin(t, FMM_STAGE_P2P, sp);
    // the item count from the build (pinned host words), else the bound with the
    // surplus blocks returning at once; split leaves add into a zeroed near
    const unsigned nitems = (unsigned)(t->h_pin && t->h_pin[0] >= 0 ? t->h_pin[0] : t->p2p_items_bound);
    // mutual form: the cross-leaf pairs once for both leaves into acc32, then
    // near = acc32 + each leaf's own pairs
    const bool mutual = p2p_mutual(t);
    if (nitems == 0)
        ;
    else if (p2p_fp64(t))
        k_p2p<double><<<nitems, P2P_THREADS, 0, sp>>>(d.p2p_items, d.p2p_nitems, d.p2p_split, d.p2p_arrived,
                                                        d.p2p_part, d.first, d.count, d.p2p_start,
                                                        d.p2p_rec, xq64, nullptr, d.icentre, d.cu2f, d.near);
    else if (mutual) {
        const int rcm = p2p_mutual_launch(t, xq32, acc32, sp);
        if (rcm) return rcm;
    } else
        k_p2p<float><<<nitems, P2P_THREADS, 0, sp>>>(d.p2p_items, d.p2p_nitems, d.p2p_split, d.p2p_arrived,
                                                       d.p2p_part, d.first, d.count, d.p2p_start,
                                                       d.p2p_rec, xq32, xlo32, d.icentre, d.cu2f, d.near);
    if (!mutual) count_launch(t);
    if (nitems > 0 && !p2p_fp64(t)) {
        k_p2p_own<<<nblk(t->nleaf, P2P_OWN_WARPS), 32 * P2P_OWN_WARPS, 0, sp>>>(
            t->nleaf, d.leaves, d.first, d.count, xq32, xlo32, mutual ? acc32 : nullptr, d.near);
        count_launch(t);
    }
    stage_end(t, FMM_STAGE_P2P, sp);
    if (sp != st) FMM_CUDA_TRY(cudaEventRecord(t->ev_join, sp));
    // the far-field chain on the high-priority stream (joined before L2P)
    cudaStream_t sf = st;
    if (overlap && sp != st && t->hi_stream && t->ev_join_hi) {
        sf = t->hi_stream;
        FMM_CUDA_TRY(cudaStreamWaitEvent(sf, t->ev_fork, 0));
    }
    {
        const int rcf = far_field<T>(t, M, L, xq64, sf);
        if (rcf) return rcf;
    }
    if (sf != st) {
        FMM_CUDA_TRY(cudaEventRecord(t->ev_join_hi, sf));
        FMM_CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join_hi, 0));
    }
    if (sp != st) FMM_CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join, 0));
    const int W = 4;
    stage_begin(t, FMM_STAGE_L2P, st);
    k_l2p_points<T, O><<<nblk(n, L2P_THREADS), L2P_THREADS, 0, st>>>(p, n, d.pleaf, d.centre, xq64, d.perm, L, d.near,
                                                                   phi, force, (t->prm.flags & FMM_OUT_FIELD) ? 1 : 0);
    count_launch(t);
    stage_end(t, FMM_STAGE_L2P, st);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

// P2M, M2M, M2L and L2L of the stage-by-stage path, all on stream st
template <typename T>
static int far_field(fmm_tree* t, cplx<T>* M, cplx<T>* L, const double4_32a* xq64, cudaStream_t st) {
    const TreeDev& d = t->d;
    const int p = t->prm.p, K = ntri(p);
    // upward pass
    stage_begin(t, FMM_STAGE_P2M, st);
    {
        const size_t smem = P2M_WARPS * p2m_warp_smem<T>(p);   // 59 KB at most (p = 20, FP64)
        if (smem > 48 * 1024)
            FMM_CUDA_TRY(cudaFuncSetAttribute(k_p2m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_p2m<T><<<nblk(t->nleaf, P2M_WARPS), 32 * P2M_WARPS, smem, st>>>(p, t->nleaf, d.leaves, d.first, d.count,
                                                                          d.centre, xq64, M);
    }
    count_launch(t);
    stage_end(t, FMM_STAGE_P2M, st);
    stage_begin(t, FMM_STAGE_M2M, st);
    if constexpr (sizeof(T) == 4) {
        const int64_t ldf = 2 * kstride(p);
        k_zero_parents<<<nblk((int64_t)t->ncell * ldf, 256), 256, 0, st>>>(t->ncell, (int)ldf, d.child_count,
                                                                          (float*)M);
        count_launch(t);
    }
    for (int l = t->nlevel - 2; l >= 0; l--) {
        int rc0 = launch_shift<T>(t, 0, t->level_start[l], t->level_start[l + 1], M, st);
        if (rc0) return rc0;
    }
    stage_end(t, FMM_STAGE_M2M, st);
    // M2L over every target's list (writes L of every cell)
    stage_begin(t, FMM_STAGE_M2L, st);
    int rc;
    if (d.rem_start) {
        // every L from zero, then the pairs the tensor cores do not take on the
        // CUDA cores in chunks (atomics into L), and the classes on the tensor
        // cores (into the real-basis accumulator, folded into L at the end).
        // With a third stream the chunks run beside the tensor-core kernel and
        // join before the fold, which reads and writes L.
        FMM_CUDA_TRY(cudaMemsetAsync(L, 0, sizeof(cplx<T>) * (size_t)t->ncell * kstride(p), st));
        rc = FMM_OK;
        cudaEvent_t rem_done = nullptr;
        if constexpr (sizeof(T) == 4) {
            if (t->rem_nchunk > 0) {
                cudaStream_t sr = st;
                if (t->ops_stream && t->ev_rem_fork && t->ev_rem_join && t->tc_nitems > 0 &&
                    !(t->prm.flags & FMM_NO_OVERLAP)) {
                    sr = t->ops_stream;
                    FMM_CUDA_TRY(cudaEventRecord(t->ev_rem_fork, st));
                    FMM_CUDA_TRY(cudaStreamWaitEvent(sr, t->ev_rem_fork, 0));
                }
                rc = launch_m2l_chunks(t, p, d, (const cplx<float>*)M, (float*)L, sr);
                if (!rc && sr != st) {
                    FMM_CUDA_TRY(cudaEventRecord(t->ev_rem_join, sr));
                    rem_done = t->ev_rem_join;
                }
            }
        }
        if (rc) return rc;
        rc = m2l_tensor_cores(t, (const float*)M, (float*)L, st, rem_done);
    } else {
        rc = launch_m2l_generic<T>(t, p, 0, t->ncell, d.m2l_start, d.m2l_src, d, M, L, st);
    }
    if (rc) return rc;
    stage_end(t, FMM_STAGE_M2L, st);
    // downward pass
    stage_begin(t, FMM_STAGE_L2L, st);
    for (int l = 1; l < t->nlevel; l++) {
        rc = launch_shift<T>(t, 1, t->level_start[l], t->level_start[l + 1], L, st);
        if (rc) return rc;
    }
    stage_end(t, FMM_STAGE_L2L, st);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
}

int evaluate_impl(fmm_tree* t, const void* q, void* phi, void* force, int dtype, cudaStream_t st) {
    if (t->n == 0) return FMM_OK;
    bool e64 = exp_fp64(t);
    if (dtype == FMM_F64) {
        return e64 ? evaluate_typed<double, double, double>(t, (const double*)q, (double*)phi, (double*)force, st)
                   : evaluate_typed<float, double, double>(t, (const double*)q, (double*)phi, (double*)force, st);
    }
    return e64 ? evaluate_typed<double, float, float>(t, (const float*)q, (float*)phi, (float*)force, st)
               : evaluate_typed<float, float, float>(t, (const float*)q, (float*)phi, (float*)force, st);
}

}  // namespace fmm
