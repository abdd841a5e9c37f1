// stages.cuh -- the FMM stages (paper Section 2.1) as device functions, shared
// by the stage-by-stage kernels (evaluate.cu) and the persistent task-queue
// kernel (queue.cu).
//
// Expansions are per-level scaled (see fmm_internal.cuh):
//   P2M  Mt_n^m = sum_j q_j R_n^m((x_j - c)/h)
//   M2M  Mt(P) = sum_children S_o Mt(C)         (dense real operator per octant o)
//   M2L  Lt_k^l(t) += (-1)^k sum_{n,m} rho^n Mt_n^m(s) conj(I_{n+k}^{m+l}(D/h_t)), rho = h_s/h_t, D = c_t - c_s
//   L2L  Lt(C) += S'_o Lt(P)                      (dense real operator per octant o)
//   L2P  phi = (1/h) sum Lt_k^l R_k^l(u), grad phi = (1/h^2) sum Lt grad R(u), u = (x - c)/h
//   P2P  phi_i += q_j / r_ij,  grad phi_i -= q_j (x_i - x_j) / r_ij^3  (r_ij > 0)
// Interaction is non-mutual (Section 4): each function writes only its target.
//
// Load policy: the persistent kernel reads expansions that other blocks wrote
// during the same launch, so it reads them through L2 (COH = true, __ldcg);
// the staged kernels use the ordinary cached path.
#pragma once
#include "fmm_internal.cuh"

namespace fmm {

template <bool COH, typename X>
__device__ __forceinline__ X ldx(const X* p) {
    if (COH) return __ldcg(p);
    return *p;
}
template <bool COH, typename T>
__device__ __forceinline__ cplx<T> ldc(const cplx<T>* p) {
    if (COH) {
        const T* f = reinterpret_cast<const T*>(p);
        return cmk<T>(__ldcg(f), __ldcg(f + 1));
    }
    return *p;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- P2M
// One warp, one leaf c; acc: the warp's shared scratch of ntri(p) entries.
template <typename T>
__device__ void p2m_leaf(int p, int c, int lane, const int32_t* __restrict__ first, const int32_t* __restrict__ count,
                         const double4_32a* __restrict__ centre, const double4_32a* __restrict__ xq,
                         cplx<T>* __restrict__ M, cplx<T>* acc, const T* rm = nullptr, const T* rt = nullptr) {
    const int K = ntri(p), KS = kstride(p);
    for (int j = lane; j < K; j += 32) acc[j] = cmk<T>(0, 0);
    __syncwarp();
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
            if (m > 0) rmm = cscale(cmul(rmm, cmk<T>(ux, uy)), rm ? rm[m] : T(1) / T(2 * m));
            cplx<T> a = rmm, b = cscale(rmm, uz);
            for (int n = m; n <= p; n++) {
                cplx<T> v;
                if (n == m) v = a;
                else if (n == m + 1) v = b;
                else {
                    const T inv = rt ? rt[tri(n, m)] : T(1) / T((n + m) * (n - m));
                    v = cmk<T>((T(2 * n - 1) * uz * b.re - r2 * a.re) * inv, (T(2 * n - 1) * uz * b.im - r2 * a.im) * inv);
                    a = b; b = v;
                }
                const T sr = warp_sum(v.re), si = warp_sum(v.im);
                if (lane == 0) { acc[tri(n, m)].re += sr; acc[tri(n, m)].im += si; }
            }
        }
    }
    __syncwarp();
    for (int j = lane; j < K; j += 32) M[(int64_t)c * KS + j] = acc[j];
}

// ---------------------------------------------------------------- M2M / L2L
// One warp, destination cell c.  kind 0 (M2M): inputs are c's children, the
// result is stored in E[c]; kind 1 (L2L): input is c's parent, the result is
// added to E[c].  ops[kind][octant] is stored input-major (row = input).
template <typename T, int RQ, bool COH>
__device__ void shift_cell(int p, int c, int kind, int lane, const int32_t* __restrict__ child_first,
                           const int32_t* __restrict__ child_count, const int32_t* __restrict__ parent,
                           const uint64_t* __restrict__ ckey, const T* __restrict__ ops, cplx<T>* E, T* xin) {
    const int K2 = 2 * ntri(p), ld = 2 * kstride(p);
    T* Ef = reinterpret_cast<T*>(E);
    T acc[RQ];
#pragma unroll
    for (int q = 0; q < RQ; q++) acc[q] = T(0);
    int nin = 1, src0 = 0;
    if (kind == 0) {
        nin = child_count[c];
        src0 = child_first[c];
        if (nin == 0) return;
    } else {
        src0 = parent[c];
#pragma unroll
        for (int q = 0; q < RQ; q++) {
            const int j = lane + 32 * q;
            if (j < K2) acc[q] = ldx<COH>(Ef + (size_t)c * ld + j);
        }
    }
    for (int k = 0; k < nin; k++) {
        const int s = src0 + k;
        const int oct = (int)(ckey[kind == 0 ? s : c] & 7);
        const T* op = ops + (size_t)(kind * 8 + oct) * K2 * K2;
        __syncwarp();
        for (int j = lane; j < K2; j += 32) xin[j] = ldx<COH>(Ef + (size_t)s * ld + j);
        __syncwarp();
        // eight operator rows in flight per step (the top levels have few cells)
        for (int i0 = 0; i0 < K2; i0 += 8) {
            T w[8][RQ];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const T* row = op + (size_t)min(i0 + u, K2 - 1) * K2;
#pragma unroll
                for (int q = 0; q < RQ; q++) {
                    const int j = lane + 32 * q;
                    w[u][q] = j < K2 ? __ldg(row + j) : T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const T x = (i0 + u < K2) ? xin[i0 + u] : T(0);
#pragma unroll
                for (int q = 0; q < RQ; q++) acc[q] = fma(w[u][q], x, acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RQ; q++) {
        const int j = lane + 32 * q;
        if (j < K2) Ef[(size_t)c * ld + j] = acc[q];
    }
}

constexpr int P2P_THREADS = 128;   // threads of a P2P block or worker group

struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct GroupSync {
    int id;   // named barrier id, P2P_THREADS threads
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(P2P_THREADS) : "memory");
    }
};

// Group version: NW warps share one destination cell and split its inputs
// (M2M: warp w takes children w, w + NW, ...; L2L: warp w takes a slice of the
// parent's coefficients), so the chain of dependent operator-row loads per
// warp is NW times shorter; partial sums meet in shared memory.  warp / tix:
// the caller's warp and thread index within the NW warps; sync: their barrier.
// COH: read E through L2 (E is written by other blocks of the same launch).
// red: NW * K2 entries; xin: NW * K2 entries.
template <typename T, int RQ, int NW, bool COH, typename Sync>
__device__ void shift_cell_block(int p, int c, int kind, const int32_t* __restrict__ child_first,
                                 const int32_t* __restrict__ child_count, const int32_t* __restrict__ parent,
                                 const uint64_t* __restrict__ ckey, const T* __restrict__ ops, cplx<T>* E, T* xin,
                                 T* red, int warp, int tix, Sync sync) {
    const int K2 = 2 * ntri(p), ld = 2 * kstride(p);
    const int lane = tix & 31;
    T* Ef = reinterpret_cast<T*>(E);
    T* xw = xin + warp * K2;
    T acc[RQ];
#pragma unroll
    for (int q = 0; q < RQ; q++) acc[q] = T(0);
    int s_first = 0, s_step = 1, s_end = 0, i_lo = 0, i_hi = K2;
    if (kind == 0) {
        s_first = child_first[c] + warp;
        s_step = NW;
        s_end = child_first[c] + child_count[c];
    } else {
        s_first = parent[c];
        s_end = s_first + 1;
        const int per = (K2 + NW - 1) / NW;
        i_lo = min(K2, warp * per);
        i_hi = min(K2, i_lo + per);
    }
    for (int s = s_first; s < s_end && i_hi > i_lo; s += s_step) {
        const int oct = (int)(ckey[kind == 0 ? s : c] & 7);
        const T* op = ops + (size_t)(kind * 8 + oct) * K2 * K2;
        __syncwarp();
        for (int j = lane; j < K2; j += 32) xw[j] = ldx<COH>(Ef + (size_t)s * ld + j);
        __syncwarp();
        for (int i0 = i_lo; i0 < i_hi; i0 += 8) {
            T w[8][RQ];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const T* row = op + (size_t)min(i0 + u, K2 - 1) * K2;
#pragma unroll
                for (int q = 0; q < RQ; q++) {
                    const int j = lane + 32 * q;
                    w[u][q] = j < K2 ? __ldg(row + j) : T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const T x = (i0 + u < i_hi) ? xw[i0 + u] : T(0);
#pragma unroll
                for (int q = 0; q < RQ; q++) acc[q] = fma(w[u][q], x, acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RQ; q++) {
        const int j = lane + 32 * q;
        if (j < K2) red[warp * K2 + j] = acc[q];
    }
    sync();
    for (int j = tix; j < K2; j += 32 * NW) {
        T v = kind == 0 ? T(0) : ldx<COH>(Ef + (size_t)c * ld + j);
        for (int w = 0; w < NW; w++) v += red[w * K2 + j];
        Ef[(size_t)c * ld + j] = v;
    }
}

// ---------------------------------------------------------------- M2L
// One source slot (a half-warp) accumulates, into acc[r], the outputs
// j = hl + 16 r of target t over the list entries e = s0 + slot, s0 + slot + nslot, ... < s1
// Ms / Is: the slot's shared scratch (ntri(p) and ntri(2p) entries).
// The caller combines the slots and applies the (-1)^k sign.
template <typename T, int RMAX, bool COH>
__device__ void m2l_range(int p, int t, int64_t s0, int64_t s1, int slot, int nslot, int hl,
                          const int32_t* __restrict__ src, const double4_32a* __restrict__ centre,
                          const cplx<T>* __restrict__ M, cplx<T>* Ms, cplx<T>* Is, const int* kk, const int* ll,
                          cplx<T>* acc) {
    const int K = ntri(p), KS = kstride(p);
    const double4_32a ct = centre[t];
    const double invht = 1.0 / ct.w;
    // every slot of the warp runs the same number of rounds (warp-synchronous scratch)
    const int64_t rounds = (s1 - s0 + nslot - 1) / nslot;
    for (int64_t rr = 0; rr < rounds; rr++) {
        const int64_t my = s0 + rr * nslot + slot;
        const bool valid = my < s1;
        if (valid) {
            const int s = src[my];
            const double4_32a cs = centre[s];
            const T rho = (T)(cs.w * invht);
            for (int j = hl; j < K; j += 16) {
                int n = 0;
                while (tri(n + 1, 0) <= j) n++;
                T sc = T(1);
                for (int i = 0; i < n; i++) sc *= rho;
                Ms[j] = cscale(ldc<COH>(M + (int64_t)s * KS + j), sc);
            }
            const T dx = (T)((ct.x - cs.x) * invht), dy = (T)((ct.y - cs.y) * invht), dz = (T)((ct.z - cs.z) * invht);
            for (int m = hl; m <= 2 * p; m += 16) irregular_column<T>(2 * p, m, dx, dy, dz, Is);
        }
        __syncwarp();
        if (valid) {
#pragma unroll
            for (int r = 0; r < RMAX; r++) {
                if (hl + 16 * r >= K) break;
                const int k = kk[r], l = ll[r];
                cplx<T> a = acc[r];
                for (int n = 0; n <= p; n++) {
                    const cplx<T>* Ij = Is + tri(n + k, 0);
                    const cplx<T>* Mn = Ms + tri(n, 0);
                    {   // m = 0: Mt_n^0 is real
                        const T mr = Mn[0].re;
                        const cplx<T> x = Ij[l];
                        a.re += mr * x.re;
                        a.im -= mr * x.im;
                    }
                    for (int m = 1; m <= n; m++) {
                        const cplx<T> mv = Mn[m];
                        cfma_cj(a, mv, Ij[m + l]);  // M conj(I^{m+l})
                        // order -m: (-1)^m conj(M) conj(I^{l-m}), I^{l-m} by symmetry when l < m
                        const bool ge = l >= m;
                        const cplx<T> x = Ij[ge ? l - m : m - l];
                        const T sgn = ((ge ? m : l) & 1) ? T(-1) : T(1);
                        const T xi = ge ? -x.im : x.im;
                        a.re += sgn * (mv.re * x.re + mv.im * xi);
                        a.im += sgn * (mv.re * xi - mv.im * x.re);
                    }
                }
                acc[r] = a;
            }
        }
        __syncwarp();
    }
}

// the whole list of target t: sources start[t] .. start[t + 1]
template <typename T, int RMAX, bool COH>
__device__ __forceinline__ void m2l_slot(int p, int t, int slot, int nslot, int hl, const int64_t* __restrict__ start,
                                         const int32_t* __restrict__ src, const double4_32a* __restrict__ centre,
                                         const cplx<T>* __restrict__ M, cplx<T>* Ms, cplx<T>* Is, const int* kk,
                                         const int* ll, cplx<T>* acc) {
    m2l_range<T, RMAX, COH>(p, t, start[t], start[t + 1], slot, nslot, hl, src, centre, M, Ms, Is, kk, ll, acc);
}

template <int RMAX>
__device__ __forceinline__ void m2l_output_index(int p, int hl, int* kk, int* ll) {
    const int K = ntri(p);
#pragma unroll
    for (int r = 0; r < RMAX; r++) {
        const int j = hl + 16 * r;
        int n = 0;
        if (j < K) { while (tri(n + 1, 0) <= j) n++; }
        kk[r] = n;
        ll[r] = j < K ? j - tri(n, 0) : 0;
    }
}

// ---------------------------------------------------------------- P2P
template <typename T> struct Vec4;
template <> struct Vec4<double> { typedef double4_32a type; };
template <> struct Vec4<float> { typedef float4 type; };

// FP32 records are relative to their own leaf centre; a source is shifted by
// c_s - c_t when staged.  The offset comes from the exact integer centres
// times side/2^22 in FP32 (no FP64 instruction per source: the FP64 pipe is
// narrow on this GPU).
template <typename T> struct Offset3 { T x, y, z; };
__device__ __forceinline__ double4_32a shift_src(double4_32a v, Offset3<double>) { return v; }
__device__ __forceinline__ float4 shift_src(float4 v, Offset3<float> o) {
    return make_float4(v.x + o.x, v.y + o.y, v.z + o.z, v.w);
}
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
// FP32: the hardware reciprocal square root (PTX rsqrt.approx.ftz.f32, relative
// error below 2^-22.9), one MUFU instruction per pair interaction
__device__ __forceinline__ float rsqrt_t(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// a pair closer than this is treated as coincident (the FP32 reciprocal square
// root flushes subnormal inputs)
__device__ __forceinline__ double pair_floor(double) { return 0.0; }
__device__ __forceinline__ float pair_floor(float) { return 1.17549435e-38f; }

constexpr int P2P_BUF = 1024;

template <typename T>
__device__ __forceinline__ void p2p_pair(const typename Vec4<T>::type& me, const typename Vec4<T>::type& s, T& phi,
                                         T& gx, T& gy, T& gz) {
    const T dx = me.x - s.x, dy = me.y - s.y, dz = me.z - s.z;
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T rinv = r2 > pair_floor(r2) ? rsqrt_t(r2) : T(0);
    const T qr = s.w * rinv;
    phi += qr;
    const T qr3 = qr * rinv * rinv;
    gx -= qr3 * dx; gy -= qr3 * dy; gz -= qr3 * dz;
}

// Paired FP32 arithmetic (PTX add/mul/fma .f32x2, sm_100 and later): one
// instruction applies the operation to both 32-bit halves of a 64-bit
// register pair.  The FP32 pair kernel keeps its two targets in the two
// halves, which halves the issue slots of the pair arithmetic.
namespace f2 {
typedef unsigned long long u64;
__device__ __forceinline__ u64 pack(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack(u64 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 add(u64 a, u64 b) {
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 mul(u64 a, u64 b) {
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 fma(u64 a, u64 b, u64 c) {
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
}  // namespace f2

// One staged source against the two targets held in the halves of X, Y, Z.
// The source is staged negated and duplicated: s01 = (-x, -x | -y, -y),
// s23 = (-z, -z | -q, -q), so that d = X + (-x) and the negated potential
// and field accumulate with adds and fmas only (NP = -phi, G = the field
// term, both per half).  GUARD: a distance at or below FLT_MIN counts as
// coincident and contributes nothing (the target leaf's own particles).
// Without it (every other leaf, staged with the target leaf's own particles
// at zero charge) r^2 starts from 1e-30 instead of 0: a zero-charge copy of
// the target itself then contributes exactly 0, a near-duplicate across a
// leaf boundary stays finite, and no other pair changes (its r^2 is many
// orders larger).
template <bool GUARD>
__device__ __forceinline__ void p2p_pair_x2(f2::u64 X, f2::u64 Y, f2::u64 Z, const ulonglong2 s01,
                                            const ulonglong2 s23, f2::u64& NP, f2::u64& GX, f2::u64& GY,
                                            f2::u64& GZ) {
    const f2::u64 dx = f2::add(X, s01.x), dy = f2::add(Y, s01.y), dz = f2::add(Z, s23.x);
    const f2::u64 r0 = GUARD ? 0ull : f2::pack(1e-30f, 1e-30f);
    const f2::u64 r2 = f2::fma(dz, dz, f2::fma(dy, dy, f2::fma(dx, dx, r0)));
    float ra, rb;
    f2::unpack(r2, ra, rb);
    if (GUARD) {
        ra = ra > pair_floor(ra) ? rsqrt_t(ra) : 0.f;
        rb = rb > pair_floor(rb) ? rsqrt_t(rb) : 0.f;
    } else {
        ra = rsqrt_t(ra);
        rb = rsqrt_t(rb);
    }
    const f2::u64 rinv = f2::pack(ra, rb);
    const f2::u64 nqr = f2::mul(s23.y, rinv);
    NP = f2::add(NP, nqr);
    const f2::u64 nqr3 = f2::mul(f2::mul(nqr, rinv), rinv);
    GX = f2::fma(nqr3, dx, GX);
    GY = f2::fma(nqr3, dy, GY);
    GZ = f2::fma(nqr3, dz, GZ);
}

// A source of the target leaf itself (guarded like p2p_pair_x2<true>).  Two
// particles of one leaf much closer than its side lose their separation to the
// rounding of their leaf-relative FP32 coordinates (about 2^-24 of the side):
// a pair closer than sqrt(close2) gets the difference of the coordinates'
// residuals added, fix(dx, dy, dz) doing so, which is rare enough to stay out
// of the common path.
template <typename Fix>
__device__ __forceinline__ void p2p_pair_x2_own(f2::u64 X, f2::u64 Y, f2::u64 Z, const ulonglong2 s01,
                                                const ulonglong2 s23, float close2, Fix fix, f2::u64& NP,
                                                f2::u64& GX, f2::u64& GY, f2::u64& GZ) {
    f2::u64 dx = f2::add(X, s01.x), dy = f2::add(Y, s01.y), dz = f2::add(Z, s23.x);
    f2::u64 r2 = f2::fma(dz, dz, f2::fma(dy, dy, f2::mul(dx, dx)));
    float ra, rb;
    f2::unpack(r2, ra, rb);
    if (ra < close2 || rb < close2) {
        fix(dx, dy, dz);
        r2 = f2::fma(dz, dz, f2::fma(dy, dy, f2::mul(dx, dx)));
        f2::unpack(r2, ra, rb);
    }
    ra = ra > pair_floor(ra) ? rsqrt_t(ra) : 0.f;
    rb = rb > pair_floor(rb) ? rsqrt_t(rb) : 0.f;
    const f2::u64 rinv = f2::pack(ra, rb);
    const f2::u64 nqr = f2::mul(s23.y, rinv);
    NP = f2::add(NP, nqr);
    const f2::u64 nqr3 = f2::mul(f2::mul(nqr, rinv), rinv);
    GX = f2::fma(nqr3, dx, GX);
    GY = f2::fma(nqr3, dy, GY);
    GZ = f2::fma(nqr3, dz, GZ);
}

// Targets held by one thread: each staged source feeds this many pair
// interactions (four was measured slower than two in FP32: fewer source
// streams per target and more registers).
template <typename T>
struct P2PBlocking { static constexpr int TPT = 2; };

// One block of P2P_THREADS threads, target leaf c.  The target's sources are
// one concatenated particle stream (each P2P record gives a source leaf's
// offset in it), staged P2P_BUF at a time, the four warps copying different
// source leaves.  Each thread holds TPT targets, so one staged source feeds TPT
// pair interactions: thread t works on targets TPT u + i (u = t mod nu,
// nu = ceil(nt / TPT)) over the staged sources j = (t / nu) (mod G),
// G = P2P_THREADS / nu.
// Barrier of the P2P_THREADS threads running p2p_leaf: the whole block, or a
// named barrier of one 128-thread group inside a larger block.

// p2p_range: records s0 .. s1 - 1 of the leaf's list only (a contiguous run of
// its source stream); own: add the leaf's own particles (FP32: they are staged
// at zero charge and added by a guarded loop, very close pairs with the
// coordinates' residuals xlo, which every FP32 caller passes); partial: when not null, the
// sums go to partial[4 t + 0..3] (t = target within the leaf) instead of near
// (the leaf's list is split over several blocks, combined afterwards).
template <typename T, typename Sync = BlockSync>
__device__ void p2p_range(int c, int64_t s0, int64_t s1, bool own, double* partial, const int32_t* __restrict__ first,
                          const int32_t* __restrict__ count, const int4* __restrict__ rec,
                          const typename Vec4<T>::type* __restrict__ xq, const float4* __restrict__ xlo,
                          const int4* __restrict__ icentre,
                          const float* __restrict__ cu2f, double* __restrict__ near, typename Vec4<T>::type* buf,
                          T (*part)[4], int tix, Sync sync = Sync()) {
    typedef typename Vec4<T>::type V;
    constexpr int TPT = P2PBlocking<T>::TPT;
    static_assert(sizeof(T) == 8 || TPT == 2, "the paired FP32 loop holds two targets");
    // sources per staging round: FP32 stages each source as two float4 (negated,
    // duplicated for the paired arithmetic), so half as many fit the buffer
    constexpr int NB = sizeof(T) == 4 ? P2P_BUF / 2 : P2P_BUF;
    const int warp = tix >> 5, lane = tix & 31;
    const int tf = first[c], nt = count[c];
    int sb = 0, se = 0;   // the records' run of the source stream
    if (s1 > s0) { sb = rec[s0].z; const int4 r = rec[s1 - 1]; se = r.z + r.y; }
    const int4 ict = icentre[c];
    const float u2f = cu2f[c];   // side/2^22 of the target's system (sources share it)
    for (int tb = 0; tb < nt; tb += TPT * P2P_THREADS) {
        const int ntc = min(TPT * P2P_THREADS, nt - tb);
        const int nu = (ntc + TPT - 1) / TPT;
        const int G = P2P_THREADS / nu;
        const int u = tix % nu, sub = tix / nu;
        const bool active = sub < G;
        V me[TPT];
        T ph[TPT], gx[TPT], gy[TPT], gz[TPT];
#pragma unroll
        for (int i = 0; i < TPT; i++) {
            const int ti = TPT * u + i;
            me[i] = xq[tf + tb + (ti < ntc ? ti : TPT * u)];
            ph[i] = gx[i] = gy[i] = gz[i] = T(0);
        }
        // FP32: paired accumulators, targets TPT u (low half) and TPT u + 1 (high)
        f2::u64 X = 0, Y = 0, Z = 0, NP = 0, GX = 0, GY = 0, GZ = 0;
        if constexpr (sizeof(T) == 4) {
            X = f2::pack(me[0].x, me[1].x);
            Y = f2::pack(me[0].y, me[1].y);
            Z = f2::pack(me[0].z, me[1].z);
        }
        int64_t e_lo = s0;
        for (int base = sb; base < se; base += NB) {
            const int lim = min(NB, se - base);
            for (int64_t e = e_lo + warp; e < s1; e += P2P_THREADS / 32) {
                const int4 r = rec[e];
                if (r.z >= base + NB) break;
                const int k0 = max(0, base - r.z), k1 = min(r.y, base + NB - r.z);
                if (k1 <= k0) continue;
                Offset3<T> o = {T(0), T(0), T(0)};
                if (sizeof(T) == 4) {
                    const int4 ics = icentre[r.w];
                    o.x = (T)((float)(ics.x - ict.x) * u2f);
                    o.y = (T)((float)(ics.y - ict.y) * u2f);
                    o.z = (T)((float)(ics.z - ict.z) * u2f);
                }
                for (int k = k0 + lane; k < k1; k += 32) {
                    const V v = shift_src(xq[r.x + k], o);
                    if constexpr (sizeof(T) == 4) {
                        float4* b2 = reinterpret_cast<float4*>(buf) + 2 * (r.z + k - base);
                        const float nq = r.w == c ? 0.f : -v.w;   // own leaf: added below, guarded
                        b2[0] = make_float4(-v.x, -v.x, -v.y, -v.y);
                        b2[1] = make_float4(-v.z, -v.z, nq, nq);
                    } else {
                        buf[r.z + k - base] = v;
                    }
                }
            }
            sync();
            if (active) {
                if constexpr (sizeof(T) == 4) {
                    const ulonglong2* b2 = reinterpret_cast<const ulonglong2*>(buf);
#pragma unroll 8
                    for (int j = sub; j < lim; j += G)
                        p2p_pair_x2<false>(X, Y, Z, b2[2 * j], b2[2 * j + 1], NP, GX, GY, GZ);
                } else {
                    int j = sub;
                    for (; j + G < lim; j += 2 * G) {
                        const V a = buf[j], bb = buf[j + G];
#pragma unroll
                        for (int i = 0; i < TPT; i++) p2p_pair<T>(me[i], a, ph[i], gx[i], gy[i], gz[i]);
#pragma unroll
                        for (int i = 0; i < TPT; i++) p2p_pair<T>(me[i], bb, ph[i], gx[i], gy[i], gz[i]);
                    }
                    if (j < lim) {
                        const V a = buf[j];
#pragma unroll
                        for (int i = 0; i < TPT; i++) p2p_pair<T>(me[i], a, ph[i], gx[i], gy[i], gz[i]);
                    }
                }
            }
            sync();
            while (e_lo < s1) {
                const int4 r = rec[e_lo];
                if (r.z + r.y > base + NB) break;
                e_lo++;
            }
        }
        if constexpr (sizeof(T) == 4) {
            // the target leaf's own particles (same leaf frame, no shift), guarded
            if (active && own) {
                // pairs closer than 1 % of the leaf's side: separation from the residuals too
                const float side = ldexpf(u2f, 22 - ict.w), close2 = 1e-4f * side * side;
                const int t0 = tf + tb + TPT * u, t1 = tf + tb + (TPT * u + 1 < ntc ? TPT * u + 1 : TPT * u);
                for (int j = sub; j < nt; j += G) {
                    const V s = xq[tf + j];
                    const ulonglong2 s01 = make_ulonglong2(f2::pack(-s.x, -s.x), f2::pack(-s.y, -s.y));
                    const ulonglong2 s23 = make_ulonglong2(f2::pack(-s.z, -s.z), f2::pack(-s.w, -s.w));
                    p2p_pair_x2_own(X, Y, Z, s01, s23, close2, [&](f2::u64& dx, f2::u64& dy, f2::u64& dz) {
                        const float4 a = xlo[t0], b = xlo[t1], l = xlo[tf + j];
                        dx = f2::add(dx, f2::pack(a.x - l.x, b.x - l.x));
                        dy = f2::add(dy, f2::pack(a.y - l.y, b.y - l.y));
                        dz = f2::add(dz, f2::pack(a.z - l.z, b.z - l.z));
                    }, NP, GX, GY, GZ);
                }
            }
            float a, b;
            f2::unpack(NP, a, b); ph[0] = -a; ph[1] = -b;
            f2::unpack(GX, a, b); gx[0] = a; gx[1] = b;
            f2::unpack(GY, a, b); gy[0] = a; gy[1] = b;
            f2::unpack(GZ, a, b); gz[0] = a; gz[1] = b;
        }
        // partial sums of the TPT targets, reduced over the G source streams
#pragma unroll
        for (int h = 0; h < TPT; h++) {
            part[tix][0] = ph[h]; part[tix][1] = gx[h];
            part[tix][2] = gy[h]; part[tix][3] = gz[h];
            sync();
            if (tix < nu && TPT * tix + h < ntc) {
                T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                for (int q = 0; q < G; q++) {
                    const int k = q * nu + tix;
                    a0 += part[k][0]; a1 += part[k][1]; a2 += part[k][2]; a3 += part[k][3];
                }
                const int64_t i = tf + tb + TPT * tix + h;
                if (partial) {
                    double* o = partial + 4 * (i - tf);
                    o[0] = (double)a0; o[1] = (double)a1; o[2] = (double)a2; o[3] = (double)a3;
                } else {
                    near[4 * i] = (double)a0; near[4 * i + 1] = (double)a1; near[4 * i + 2] = (double)a2;
                    near[4 * i + 3] = (double)a3;
                }
            }
            sync();
        }
    }
}

// the whole list of target leaf c (xlo: residuals of the FP32 coordinates, null for FP64)
template <typename T, typename Sync = BlockSync>
__device__ __forceinline__ void p2p_leaf(int c, const int32_t* __restrict__ first, const int32_t* __restrict__ count,
                                         const int64_t* __restrict__ start, const int4* __restrict__ rec,
                                         const typename Vec4<T>::type* __restrict__ xq,
                                         const float4* __restrict__ xlo, const int4* __restrict__ icentre,
                                         const float* __restrict__ cu2f, double* __restrict__ near,
                                         typename Vec4<T>::type* buf, T (*part)[4], int tix, Sync sync = Sync()) {
    p2p_range<T, Sync>(c, start[c], start[c + 1], true, nullptr, first, count, rec, xq, xlo, icentre, cu2f, near, buf,
                       part, tix, sync);
}

// ---------------------------------------------------------------- L2P
// Lt(c) and its gradient at u = (x - centre) / h: the regular harmonics of u
// by the recurrence in n for each m, accumulated against Ls.  TAB: the
// reciprocals 1/(2m) and 1/((n+m)(n-m)) come from tables (rm[m],
// rt[tri(n, m)]) holding the values the divisions give, so both forms agree
// bit for bit.
template <typename T, bool TAB>
__device__ __forceinline__ void l2p_point(int p, T ux, T uy, T uz, const cplx<T>* Ls, const T* rm, const T* rt,
                                          T& fp, T& gx, T& gy, T& gz) {
    const T r2 = ux * ux + uy * uy + uz * uz;
    fp = 0; gx = 0; gy = 0; gz = 0;
    cplx<T> rmm = cmk<T>(1, 0);
    for (int m = 0; m <= p; m++) {
        if (m > 0) rmm = cscale(cmul(rmm, cmk<T>(ux, uy)), TAB ? rm[m] : T(1) / T(2 * m));
        cplx<T> a0 = rmm, b0 = cscale(rmm, uz);
        const T w = m == 0 ? T(1) : T(2);
        for (int n = m; n <= p; n++) {
            cplx<T> S;
            if (n == m) S = a0;
            else if (n == m + 1) S = b0;
            else {
                const T inv = TAB ? rt[tri(n, m)] : T(1) / T((n + m) * (n - m));
                S = cmk<T>((T(2 * n - 1) * uz * b0.re - r2 * a0.re) * inv, (T(2 * n - 1) * uz * b0.im - r2 * a0.im) * inv);
                a0 = b0; b0 = S;
            }
            const cplx<T> Lnm = Ls[tri(n, m)];
            fp += w * (Lnm.re * S.re - Lnm.im * S.im);
            if (n + 1 <= p) {
                const cplx<T>* L1 = Ls + tri(n + 1, 0);
                const cplx<T> lz = L1[m];
                gz += w * (lz.re * S.re - lz.im * S.im);
                if (m == 0) {
                    gx += L1[1].re * S.re;
                    gy -= L1[1].im * S.re;
                } else {
                    const cplx<T> up = L1[m + 1], dn = L1[m - 1];
                    const cplx<T> A = csub(up, dn), B = cadd(up, dn);
                    gx += A.re * S.re - A.im * S.im;
                    gy += -(B.im * S.re + B.re * S.im);  // Re(i B S)
                }
            }
        }
    }
}

// sorted particle gi: far field (scaled by the leaf's 1/h) plus near field,
// written in input order
template <typename T, typename O, bool COH>
__device__ __forceinline__ void l2p_store(int64_t gi, double invh, double qi, T fp, T gx, T gy, T gz,
                                          const int32_t* __restrict__ perm, const double* __restrict__ near,
                                          O* __restrict__ phi_out, O* __restrict__ force_out, int field) {
    const double ph = (double)fp * invh + ldx<COH>(near + 4 * gi);
    const double ih2 = invh * invh;
    const double ex = -((double)gx * ih2 + ldx<COH>(near + 4 * gi + 1));
    const double ey = -((double)gy * ih2 + ldx<COH>(near + 4 * gi + 2));
    const double ez = -((double)gz * ih2 + ldx<COH>(near + 4 * gi + 3));
    const int64_t o = perm[gi];
    if (phi_out) phi_out[o] = (O)ph;
    if (force_out) {
        const double s = field ? 1.0 : qi;
        force_out[3 * o] = (O)(s * ex);
        force_out[3 * o + 1] = (O)(s * ey);
        force_out[3 * o + 2] = (O)(s * ez);
    }
}

// Particles tid, tid + nthr, ... of leaf c, with Lt(c) already in Ls; adds the
// near field and writes the outputs in input order.
template <typename T, typename O, bool COH>
__device__ void l2p_particles(int p, int c, int tid, int nthr, const cplx<T>* Ls, const int32_t* __restrict__ first,
                              const int32_t* __restrict__ count, const double4_32a* __restrict__ centre,
                              const double4_32a* __restrict__ xq, const int32_t* __restrict__ perm,
                              const double* __restrict__ near, O* __restrict__ phi_out, O* __restrict__ force_out,
                              int field) {
    const double4_32a cc = centre[c];
    const double invh = 1.0 / cc.w;
    const int f = first[c], cnt = count[c];
    for (int i = tid; i < cnt; i += nthr) {
        const double4_32a a = xq[f + i];
        const T ux = (T)((a.x - cc.x) * invh), uy = (T)((a.y - cc.y) * invh), uz = (T)((a.z - cc.z) * invh);
        T fp, gx, gy, gz;
        l2p_point<T, false>(p, ux, uy, uz, Ls, nullptr, nullptr, fp, gx, gy, gz);
        l2p_store<T, O, COH>(f + i, invh, a.w, fp, gx, gy, gz, perm, near, phi_out, force_out, field);
    }
}

}  // namespace fmm
