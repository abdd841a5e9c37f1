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

#include "fmm_internal.cuh"

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
// rounding of a coordinate scales with the leaf size, not with the position.
template <typename Q>
__global__ void k_prepare32(const double* __restrict__ spos, const int32_t* __restrict__ perm,
                            const Q* __restrict__ q, int64_t n, const int32_t* __restrict__ pleaf,
                            const double4_32a* __restrict__ centre, double4_32a* xq64, float4* xq32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = spos[3 * i], y = spos[3 * i + 1], z = spos[3 * i + 2], qq = (double)q[perm[i]];
    xq64[i] = make_double4_32a(x, y, z, qq);
    double4_32a c = centre[pleaf[i]];
    xq32[i] = make_float4((float)(x - c.x), (float)(y - c.y), (float)(z - c.z), (float)qq);
}

// R_k^l(d/h_P) for the eight child octants, d/h_P = (+-1/4, +-1/4, +-1/4);
// bit 0 of the octant is x, bit 1 y, bit 2 z.
template <typename T>
__global__ void k_octant_table(int p, cplx<T>* Roct) {
    int o = threadIdx.x;
    if (o >= 8) return;
    T x = (o & 1) ? T(0.25) : T(-0.25), y = (o & 2) ? T(0.25) : T(-0.25), z = (o & 4) ? T(0.25) : T(-0.25);
    regular_harmonics<T>(p, x, y, z, Roct + o * ntri(p));
}

// ---------------------------------------------------------------------------
// P2M: one warp per leaf; each coefficient is reduced over the warp
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void k_p2m(int p, int nleaf, const int32_t* __restrict__ leaves, const int32_t* __restrict__ first,
                      const int32_t* __restrict__ count, const double4_32a* __restrict__ centre,
                      const double4_32a* __restrict__ xq, cplx<T>* __restrict__ M) {
    extern __shared__ unsigned char smem_raw[];
    const int K = ntri(p), KS = kstride(p);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cplx<T>* acc = reinterpret_cast<cplx<T>*>(smem_raw) + warp * K;
    int li = blockIdx.x * (blockDim.x >> 5) + warp;
    if (li >= nleaf) return;
    int c = leaves[li];
    for (int j = lane; j < K; j += 32) acc[j] = cmk<T>(0, 0);
    __syncwarp();
    double4_32a cc = centre[c];
    double invh = 1.0 / cc.w;
    int f = first[c], cnt = count[c];
    for (int base = 0; base < cnt; base += 32) {
        int i = base + lane;
        T ux = 0, uy = 0, uz = 0, q = 0;
        if (i < cnt) {
            double4_32a a = xq[f + i];
            ux = (T)((a.x - cc.x) * invh); uy = (T)((a.y - cc.y) * invh); uz = (T)((a.z - cc.z) * invh);
            q = (T)a.w;
        }
        T r2 = ux * ux + uy * uy + uz * uz;
        cplx<T> rmm = cmk<T>(q, 0);
        for (int m = 0; m <= p; m++) {
            if (m > 0) rmm = cscale(cmul(rmm, cmk<T>(ux, uy)), T(1) / T(2 * m));
            cplx<T> a = rmm, b = cscale(rmm, uz);
            for (int n = m; n <= p; n++) {
                cplx<T> v;
                if (n == m) v = a;
                else if (n == m + 1) v = b;
                else {
                    T inv = T(1) / T((n + m) * (n - m));
                    v = cmk<T>((T(2 * n - 1) * uz * b.re - r2 * a.re) * inv,
                               (T(2 * n - 1) * uz * b.im - r2 * a.im) * inv);
                    a = b; b = v;
                }
                T sr = warp_sum(v.re), si = warp_sum(v.im);
                if (lane == 0) { acc[tri(n, m)].re += sr; acc[tri(n, m)].im += si; }
            }
        }
    }
    __syncwarp();
    for (int j = lane; j < K; j += 32) M[(int64_t)c * KS + j] = acc[j];
}

// ---------------------------------------------------------------------------
// M2M: one warp per parent cell of one level
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_m2m(int p, int lb, int le, const int32_t* __restrict__ child_first,
                      const int32_t* __restrict__ child_count, const uint64_t* __restrict__ ckey,
                      const cplx<T>* __restrict__ Roct, cplx<T>* __restrict__ M) {
    extern __shared__ unsigned char smem_raw[];
    const int K = ntri(p), KS = kstride(p);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cplx<T>* Mc = reinterpret_cast<cplx<T>*>(smem_raw) + warp * 2 * K;
    cplx<T>* acc = Mc + K;
    int c = lb + blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= le) return;
    int nc = child_count[c];
    if (nc == 0) return;
    for (int j = lane; j < K; j += 32) acc[j] = cmk<T>(0, 0);
    int cf = child_first[c];
    for (int ch = 0; ch < nc; ch++) {
        int cidx = cf + ch;
        __syncwarp();
        for (int j = lane; j < K; j += 32) Mc[j] = M[(int64_t)cidx * KS + j];
        __syncwarp();
        const cplx<T>* R = Roct + (int)(ckey[cidx] & 7) * K;
        for (int j = lane; j < K; j += 32) {
            int n = 0;
            while (tri(n + 1, 0) <= j) n++;
            int m = j - tri(n, 0);
            cplx<T> s = cmk<T>(0, 0);
            T scale = T(1);
            for (int k = n; k >= 0; k--) {      // source degree n-k, scale 2^{-(n-k)}
                int js = n - k;
                for (int l = -k; l <= k; l++) {
                    int ms = m - l;
                    if (ms > js || -ms > js) continue;
                    cplx<T> r = get_sym(R, k, l), mv = get_sym(Mc, js, ms);
                    cplx<T> t = cmul(r, mv);
                    s.re += scale * t.re; s.im += scale * t.im;
                }
                scale *= T(0.5);
            }
            acc[j] = cadd(acc[j], s);
        }
    }
    __syncwarp();
    for (int j = lane; j < K; j += 32) M[(int64_t)c * KS + j] = acc[j];
}

// ---------------------------------------------------------------------------
// M2L (any pair of cells): one warp per target, each half-warp one source.
// Lane (h, i) accumulates the outputs j = i, i+16, ... < ntri(p).
// ---------------------------------------------------------------------------

template <typename T, int RMAX>
__global__ void __launch_bounds__(128) k_m2l_generic(int p, int t0, int t1, const int64_t* __restrict__ start,
                                                     const int32_t* __restrict__ src,
                                                     const double4_32a* __restrict__ centre,
                                                     const cplx<T>* __restrict__ M, cplx<T>* __restrict__ L) {
    extern __shared__ unsigned char smem_raw[];
    const int K = ntri(p), KI = ntri(2 * p), KS = kstride(p);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    cplx<T>* base = reinterpret_cast<cplx<T>*>(smem_raw) + warp * 2 * (K + KI);
    cplx<T>* Ms = base + half * (K + KI);
    cplx<T>* Is = Ms + K;
    int t = t0 + blockIdx.x * (blockDim.x >> 5) + warp;
    if (t >= t1) return;
    int kk[RMAX], ll[RMAX];
    cplx<T> acc[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; r++) {
        int j = hl + 16 * r, n = 0;
        if (j < K) { while (tri(n + 1, 0) <= j) n++; }
        kk[r] = n;
        ll[r] = j < K ? j - tri(n, 0) : 0;
        acc[r] = cmk<T>(0, 0);
    }
    int64_t s0 = start[t], s1 = start[t + 1];
    double4_32a ct = centre[t];
    double invht = 1.0 / ct.w;
    for (int64_t e = s0; e < s1; e += 2) {
        int64_t my = e + half;
        bool valid = my < s1;
        if (valid) {
            int s = src[my];
            double4_32a cs = centre[s];
            T rho = (T)(cs.w * invht);
            // stage rho^n Mt_n^m(s)
            for (int j = hl; j < K; j += 16) {
                int n = 0;
                while (tri(n + 1, 0) <= j) n++;
                T sc = T(1);
                for (int i = 0; i < n; i++) sc *= rho;
                Ms[j] = cscale(M[(int64_t)s * KS + j], sc);
            }
            T dx = (T)((ct.x - cs.x) * invht), dy = (T)((ct.y - cs.y) * invht), dz = (T)((ct.z - cs.z) * invht);
            for (int m = hl; m <= 2 * p; m += 16) irregular_column<T>(2 * p, m, dx, dy, dz, Is);
        }
        __syncwarp();
        if (valid) {
#pragma unroll
            for (int r = 0; r < RMAX; r++) {
                if (hl + 16 * r >= K) break;
                int k = kk[r], l = ll[r];
                cplx<T> a = acc[r];
                for (int n = 0; n <= p; n++) {
                    const cplx<T>* Ij = Is + tri(n + k, 0);
                    const cplx<T>* Mn = Ms + tri(n, 0);
                    // m = 0: Mt_n^0 real
                    {
                        T mr = Mn[0].re;
                        cplx<T> x = Ij[l];
                        a.re += mr * x.re;
                        a.im -= mr * x.im;
                    }
                    for (int m = 1; m <= n; m++) {
                        cplx<T> mv = Mn[m];
                        cfma_cj(a, mv, Ij[m + l]);                       // M conj(I^{m+l})
                        // negative order -m:  (-1)^m conj(M) conj(I^{l-m})
                        bool ge = l >= m;
                        cplx<T> x = Ij[ge ? l - m : m - l];
                        T sgn = ((ge ? m : l) & 1) ? T(-1) : T(1);
                        // conj(M) * (ge ? conj(x) : x) * sgn
                        T xi = ge ? -x.im : x.im;
                        a.re += sgn * (mv.re * x.re + mv.im * xi);
                        a.im += sgn * (mv.re * xi - mv.im * x.re);
                    }
                }
                acc[r] = a;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < RMAX; r++) {
        acc[r].re += __shfl_xor_sync(0xffffffffu, acc[r].re, 16);
        acc[r].im += __shfl_xor_sync(0xffffffffu, acc[r].im, 16);
    }
    if (half == 0) {
#pragma unroll
        for (int r = 0; r < RMAX; r++) {
            int j = hl + 16 * r;
            if (j < K) {
                T sg = (kk[r] & 1) ? T(-1) : T(1);
                L[(int64_t)t * KS + j] = cscale(acc[r], sg);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// L2L: one warp per child cell of one level
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_l2l(int p, int lb, int le, const int32_t* __restrict__ parent, const uint64_t* __restrict__ ckey,
                      const cplx<T>* __restrict__ Roct, cplx<T>* __restrict__ L) {
    extern __shared__ unsigned char smem_raw[];
    const int K = ntri(p), KS = kstride(p);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cplx<T>* Lp = reinterpret_cast<cplx<T>*>(smem_raw) + warp * K;
    int c = lb + blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= le) return;
    int pc = parent[c];
    for (int j = lane; j < K; j += 32) Lp[j] = L[(int64_t)pc * KS + j];
    __syncwarp();
    const cplx<T>* R = Roct + (int)(ckey[c] & 7) * K;
    for (int j = lane; j < K; j += 32) {
        int k = 0;
        while (tri(k + 1, 0) <= j) k++;
        int l = j - tri(k, 0);
        cplx<T> s = cmk<T>(0, 0);
        for (int n = k; n <= p; n++)
            for (int m = -n; m <= n; m++) {
                int mr = m - l;
                if (mr > n - k || -mr > n - k) continue;
                cfma(s, get_sym(Lp, n, m), get_sym(R, n - k, mr));
            }
        T sc = T(1);
        for (int i = 0; i <= k; i++) sc *= T(0.5);
        cplx<T> o = L[(int64_t)c * KS + j];
        L[(int64_t)c * KS + j] = cadd(o, cscale(s, sc));
    }
}

// ---------------------------------------------------------------------------
// P2P: one block per target leaf; sources staged in shared memory.
// Thread t works on target (t mod nt) and source stream (t / nt).
// ---------------------------------------------------------------------------

template <typename T> struct Vec4;
template <> struct Vec4<double> { typedef double4_32a type; };
template <> struct Vec4<float> { typedef float4 type; };

// FP64 records hold absolute positions; FP32 records hold positions relative
// to their own leaf centre, so a source is shifted by (c_s - c_t) when staged.
// The offset c_s - c_t comes from the exact integer centres times side/2^22 in
// FP32: no FP64 instruction per source (the FP64 pipe is narrow on this GPU).
template <typename T> struct Offset3 { T x, y, z; };
__device__ __forceinline__ double4_32a shift_src(double4_32a v, Offset3<double>) { return v; }
__device__ __forceinline__ float4 shift_src(float4 v, Offset3<float> o) {
    return make_float4(v.x + o.x, v.y + o.y, v.z + o.z, v.w);
}

__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

constexpr int P2P_THREADS = 128;
constexpr int P2P_BUF = 512;

template <typename T>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p(int nleaf, const int32_t* __restrict__ leaves,
                                                     const int32_t* __restrict__ first,
                                                     const int32_t* __restrict__ count,
                                                     const int64_t* __restrict__ start,
                                                     const int32_t* __restrict__ src,
                                                     const typename Vec4<T>::type* __restrict__ xq,
                                                     const int4* __restrict__ icentre, float u2f,
                                                     double* __restrict__ near) {
    typedef typename Vec4<T>::type V;
    __shared__ V buf[P2P_BUF];
    __shared__ T part[P2P_THREADS][4];
    int li = blockIdx.x;
    if (li >= nleaf) return;
    int c = leaves[li];
    int tf = first[c], nt = count[c];
    int64_t s0 = start[c], s1 = start[c + 1];
    const int4 ict = icentre[c];
    for (int tb = 0; tb < nt; tb += P2P_THREADS) {
        int ntc = min(P2P_THREADS, nt - tb);
        int G = P2P_THREADS / ntc;
        int ti = threadIdx.x % ntc, sub = threadIdx.x / ntc;
        bool active = sub < G;
        V me = xq[tf + tb + ti];
        T phi = 0, gx = 0, gy = 0, gz = 0;
        int fill = 0;
        auto compute = [&](int nfill) {
            if (!active) return;
            for (int j = sub; j < nfill; j += G) {
                V s = buf[j];
                T dx = me.x - s.x, dy = me.y - s.y, dz = me.z - s.z;
                T r2 = dx * dx + dy * dy + dz * dz;
                T rinv = r2 > T(0) ? rsqrt_t(r2) : T(0);
                T qr = s.w * rinv;
                phi += qr;
                T qr3 = qr * rinv * rinv;
                gx -= qr3 * dx; gy -= qr3 * dy; gz -= qr3 * dz;
            }
        };
        for (int64_t e = s0; e < s1; e++) {
            int sc = src[e];
            int rf = first[sc], rc = count[sc], off = 0;
            const int4 ics = icentre[sc];
            Offset3<T> o;
            o.x = (T)((float)(ics.x - ict.x) * u2f);
            o.y = (T)((float)(ics.y - ict.y) * u2f);
            o.z = (T)((float)(ics.z - ict.z) * u2f);
            while (off < rc) {
                int take = min(rc - off, P2P_BUF - fill);
                for (int k = threadIdx.x; k < take; k += P2P_THREADS)
                    buf[fill + k] = shift_src(xq[rf + off + k], o);
                fill += take;
                off += take;
                if (fill == P2P_BUF) {
                    __syncthreads();
                    compute(fill);
                    __syncthreads();
                    fill = 0;
                }
            }
        }
        if (fill) {
            __syncthreads();
            compute(fill);
            __syncthreads();
        }
        part[threadIdx.x][0] = phi; part[threadIdx.x][1] = gx; part[threadIdx.x][2] = gy; part[threadIdx.x][3] = gz;
        __syncthreads();
        if (threadIdx.x < ntc) {
            double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            for (int s = 0; s < G; s++) {
                int k = s * ntc + threadIdx.x;
                a0 += part[k][0]; a1 += part[k][1]; a2 += part[k][2]; a3 += part[k][3];
            }
            int64_t i = tf + tb + threadIdx.x;
            near[4 * i] = a0; near[4 * i + 1] = a1; near[4 * i + 2] = a2; near[4 * i + 3] = a3;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// L2P + near field + output in input order: one warp per leaf, one particle per lane
// ---------------------------------------------------------------------------

template <typename T, typename O>
__global__ void k_l2p_finalize(int p, int nleaf, const int32_t* __restrict__ leaves,
                               const int32_t* __restrict__ first, const int32_t* __restrict__ count,
                               const double4_32a* __restrict__ centre, const double4_32a* __restrict__ xq,
                               const int32_t* __restrict__ perm, const cplx<T>* __restrict__ L,
                               const double* __restrict__ near, O* __restrict__ phi_out, O* __restrict__ force_out,
                               int field) {
    extern __shared__ unsigned char smem_raw[];
    const int K = ntri(p), KS = kstride(p);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cplx<T>* Ls = reinterpret_cast<cplx<T>*>(smem_raw) + warp * K;
    int li = blockIdx.x * (blockDim.x >> 5) + warp;
    if (li >= nleaf) return;
    int c = leaves[li];
    for (int j = lane; j < K; j += 32) Ls[j] = L[(int64_t)c * KS + j];
    __syncwarp();
    double4_32a cc = centre[c];
    double invh = 1.0 / cc.w;
    int f = first[c], cnt = count[c];
    for (int i = lane; i < cnt; i += 32) {
        double4_32a a = xq[f + i];
        T ux = (T)((a.x - cc.x) * invh), uy = (T)((a.y - cc.y) * invh), uz = (T)((a.z - cc.z) * invh);
        T r2 = ux * ux + uy * uy + uz * uz;
        T fp = 0, gx = 0, gy = 0, gz = 0;
        cplx<T> rmm = cmk<T>(1, 0);
        for (int m = 0; m <= p; m++) {
            if (m > 0) rmm = cscale(cmul(rmm, cmk<T>(ux, uy)), T(1) / T(2 * m));
            cplx<T> a0 = rmm, b0 = cscale(rmm, uz);
            T w = m == 0 ? T(1) : T(2);
            for (int n = m; n <= p; n++) {
                cplx<T> S;
                if (n == m) S = a0;
                else if (n == m + 1) S = b0;
                else {
                    T inv = T(1) / T((n + m) * (n - m));
                    S = cmk<T>((T(2 * n - 1) * uz * b0.re - r2 * a0.re) * inv,
                               (T(2 * n - 1) * uz * b0.im - r2 * a0.im) * inv);
                    a0 = b0; b0 = S;
                }
                cplx<T> Lnm = Ls[tri(n, m)];
                fp += w * (Lnm.re * S.re - Lnm.im * S.im);
                if (n + 1 <= p) {
                    const cplx<T>* L1 = Ls + tri(n + 1, 0);
                    cplx<T> lz = L1[m];
                    gz += w * (lz.re * S.re - lz.im * S.im);
                    if (m == 0) {
                        gx += L1[1].re * S.re;
                        gy -= L1[1].im * S.re;
                    } else {
                        cplx<T> up = L1[m + 1], dn = L1[m - 1];
                        cplx<T> A = csub(up, dn), B = cadd(up, dn);
                        gx += A.re * S.re - A.im * S.im;
                        gy += -(B.im * S.re + B.re * S.im);  // Re(i B S)
                    }
                }
            }
        }
        int64_t gi = f + i;
        double ph = (double)fp * invh + near[4 * gi];
        double ih2 = invh * invh;
        double ex = -((double)gx * ih2 + near[4 * gi + 1]);
        double ey = -((double)gy * ih2 + near[4 * gi + 2]);
        double ez = -((double)gz * ih2 + near[4 * gi + 3]);
        int64_t o = perm[gi];
        if (phi_out) phi_out[o] = (O)ph;
        if (force_out) {
            double s = field ? 1.0 : a.w;
            force_out[3 * o] = (O)(s * ex);
            force_out[3 * o + 1] = (O)(s * ey);
            force_out[3 * o + 2] = (O)(s * ez);
        }
    }
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
    if ((rc = dev_alloc(&M, (size_t)t->ncell * K * csz + 8 * K * csz, t, st))) return rc;
    if ((rc = dev_alloc(&L, (size_t)t->ncell * K * csz, t, st))) return rc;
    // double4_32a copy always (P2M/L2P positions), plus float4 for FP32 P2P
    size_t xb = (size_t)t->n * sizeof(double4_32a) + (p2p_fp64(t) ? 0 : (size_t)t->n * sizeof(float4));
    if ((rc = dev_alloc(&xq, xb, t, st))) return rc;
    if ((rc = dev_alloc(&d.near, (size_t)t->n * 4, t, st))) return rc;
    d.M = M; d.L = L; d.xq = xq;
    if (t->prm.precision == FMM_PREC_MIXED_TC && t->tc_nitems > 0) {
        char* ms = nullptr;
        if ((rc = dev_alloc(&ms, (size_t)t->ncell * 2 * tc_kpad(t->prm.p) * 2, t, st))) return rc;
        d.tc_msplit = ms;
    }
    // octant table after the multipoles
    if (exp_fp64(t))
        k_octant_table<double><<<1, 32, 0, st>>>(t->prm.p, (cplx<double>*)(M + (size_t)t->ncell * K * csz));
    else
        k_octant_table<float><<<1, 32, 0, st>>>(t->prm.p, (cplx<float>*)(M + (size_t)t->ncell * K * csz));
    count_launch(t);
    FMM_CUDA_TRY(cudaGetLastError());
    return FMM_OK;
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

template <typename T, typename Q, typename O>
static int evaluate_typed(fmm_tree* t, const Q* q, O* phi, O* force, cudaStream_t st) {
    const int p = t->prm.p, K = ntri(p);
    TreeDev& d = t->d;
    const int64_t n = t->n;
    double4_32a* xq64 = (double4_32a*)d.xq;
    float4* xq32 = (float4*)((char*)d.xq + (size_t)n * sizeof(double4_32a));
    cplx<T>* M = (cplx<T>*)d.M;
    cplx<T>* L = (cplx<T>*)d.L;
    const cplx<T>* Roct = M + (size_t)t->ncell * kstride(p);
    // particles in sorted order
    stage_begin(t, FMM_STAGE_PREPARE, st);
    if (p2p_fp64(t))
        k_prepare64<Q><<<nblk(n, 256), 256, 0, st>>>(d.spos, d.perm, q, n, xq64);
    else
        k_prepare32<Q><<<nblk(n, 256), 256, 0, st>>>(d.spos, d.perm, q, n, d.pleaf, d.centre, xq64, xq32);
    count_launch(t);
    stage_end(t, FMM_STAGE_PREPARE, st);
    // P2P (near field)
    stage_begin(t, FMM_STAGE_P2P, st);
    if (p2p_fp64(t))
        k_p2p<double><<<t->nleaf, P2P_THREADS, 0, st>>>(t->nleaf, d.leaves, d.first, d.count, d.p2p_start,
                                                          d.p2p_src, xq64, d.icentre, 0.f, d.near);
    else
        k_p2p<float><<<t->nleaf, P2P_THREADS, 0, st>>>(t->nleaf, d.leaves, d.first, d.count, d.p2p_start,
                                                         d.p2p_src, xq32, d.icentre,
                                                         (float)(t->side / 4194304.0), d.near);
    count_launch(t);
    stage_end(t, FMM_STAGE_P2P, st);
    // upward pass
    const int W = 4;
    stage_begin(t, FMM_STAGE_P2M, st);
    k_p2m<T><<<nblk(t->nleaf, W), 32 * W, W * K * sizeof(cplx<T>), st>>>(p, t->nleaf, d.leaves, d.first, d.count,
                                                                          d.centre, xq64, M);
    count_launch(t);
    stage_end(t, FMM_STAGE_P2M, st);
    stage_begin(t, FMM_STAGE_M2M, st);
    for (int l = t->nlevel - 2; l >= 0; l--) {
        int lb = t->level_start[l], le = t->level_start[l + 1];
        k_m2m<T><<<nblk(le - lb, W), 32 * W, W * 2 * K * sizeof(cplx<T>), st>>>(p, lb, le, d.child_first,
                                                                                 d.child_count, d.ckey, Roct, M);
        count_launch(t);
    }
    stage_end(t, FMM_STAGE_M2M, st);
    // M2L over every target's list (writes L of every cell)
    stage_begin(t, FMM_STAGE_M2L, st);
    int rc;
    if (t->prm.precision == FMM_PREC_MIXED_TC && t->tc_nitems > 0) {
        // class-less pairs on the CUDA cores (this also initialises every L), then
        // the classes on the tensor cores, accumulated into L
        rc = launch_m2l_generic<T>(t, p, 0, t->ncell, d.rem_start, d.tc_src + t->tc_npairs, d, M, L, st);
        if (rc) return rc;
        rc = m2l_tensor_cores(t, (const float*)M, (float*)L, st);
    } else {
        rc = launch_m2l_generic<T>(t, p, 0, t->ncell, d.m2l_start, d.m2l_src, d, M, L, st);
    }
    if (rc) return rc;
    stage_end(t, FMM_STAGE_M2L, st);
    // downward pass
    stage_begin(t, FMM_STAGE_L2L, st);
    for (int l = 1; l < t->nlevel; l++) {
        int lb = t->level_start[l], le = t->level_start[l + 1];
        k_l2l<T><<<nblk(le - lb, W), 32 * W, W * K * sizeof(cplx<T>), st>>>(p, lb, le, d.parent, d.ckey, Roct, L);
        count_launch(t);
    }
    stage_end(t, FMM_STAGE_L2L, st);
    stage_begin(t, FMM_STAGE_L2P, st);
    k_l2p_finalize<T, O><<<nblk(t->nleaf, W), 32 * W, W * K * sizeof(cplx<T>), st>>>(
        p, t->nleaf, d.leaves, d.first, d.count, d.centre, xq64, d.perm, L, d.near, phi, force,
        (t->prm.flags & FMM_OUT_FIELD) ? 1 : 0);
    count_launch(t);
    stage_end(t, FMM_STAGE_L2P, st);
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
