/*
 * fmm_oracle.c -- CPU FP64 oracle for the adaptive 3-D Laplace FMM.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or helper with the CUDA path.  It is written to be read against the
 * method, not to be fast: plain loops, complex arithmetic with the full range
 * of orders m = -n..n, no blocking, no symmetry tricks.
 *
 * What the paper fixes and what is read into it:
 *  - Six stages P2M, M2M, M2L, P2P, L2L, L2P on a cubic adaptive octree whose
 *    depth keeps particles per leaf bounded (Section 2.1, "Overview").
 *  - Morton keys give cell location (Section 2.2).
 *  - Pairs come from a breadth-first (queue) dual tree traversal; a pair is
 *    well separated by the ratio of cell size to distance (Sections 2.1, 4, 5).
 *  - Non-mutual interaction: every pair is (target, source) and only the
 *    target is written (Section 4).
 *  The paper defers the operator formulas to Cheng et al. 1999 and Epton &
 *  Dembart 1995.  They are restated here from the Laplace addition theorem:
 *
 *  Associated Legendre P_n^m (m >= 0) WITHOUT the Condon-Shortley phase.
 *  Regular solid harmonic   R_n^m(x) = r^n P_n^m(cos t) e^{i m f} / (n+m)!
 *  Irregular solid harmonic I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m f} / r^{n+1}
 *  and for negative orders  R_n^{-m} = (-1)^m conj(R_n^m),  same for I.
 *  With these,
 *    1/|x-y| = sum_{n,m} conj(R_n^m(y)) I_n^m(x)                 (|y| < |x|)
 *    R_n^m(a+b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b)
 *    I_n^m(a+b) = sum_{k,l} (-1)^k conj(R_k^l(b)) I_{n+k}^{m+l}(a) (|b| < |a|)
 *  Multipole about c:  M_n^m = sum_j q_j R_n^m(x_j - c)
 *      phi(x) = sum_{n,m} conj(M_n^m) I_n^m(x - c)
 *  Local about c:      phi(x) = sum_{n,m} L_n^m R_n^m(x - c)
 *  M2M (child c' -> parent c, d = c' - c):
 *      M_n^m(c) += sum_{k,l} R_k^l(d) M_{n-k}^{m-l}(c')
 *  M2L (multipole at s -> local at t, D = t - s):
 *      L_k^l(t) += (-1)^k sum_{n,m} M_n^m conj(I_{n+k}^{m+l}(D))
 *  L2L (parent c -> child c', d = c' - c):
 *      L_k^l(c') += sum_{n>=k,m} L_n^m R_{n-k}^{m-l}(d)
 *  L2P gradient from the derivatives of R:
 *      d/dz R_n^m = R_{n-1}^m
 *      d/dx R_n^m = (R_{n-1}^{m-1} - R_{n-1}^{m+1}) / 2
 *      d/dy R_n^m = i (R_{n-1}^{m-1} + R_{n-1}^{m+1}) / 2
 *  "Order p" keeps degrees n = 0..p, so an expansion has (p+1)^2 coefficients;
 *  M2L maps the whole truncated multipole (n <= p) to the truncated local
 *  (k <= p).
 *
 *  Readings where the paper is silent (the same readings bind the CUDA path):
 *  root cube, 21-bit quantisation, leaf rule, MAC in integer units, split
 *  rule, canonical cell order, list order -- see the functions below.
 *
 *  Coefficient layout in this file: complex, index n*n + n + m, m = -n..n.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define MAXLEVEL 21

static int hidx(int n, int m) { return n * n + n + m; }

/* ------------------------------------------------------------------ */
/* Associated Legendre functions and solid harmonics (definitions)     */
/* ------------------------------------------------------------------ */

/* P_n^m(t), 0 <= m <= n <= nmax, no Condon-Shortley phase, by the standard
 * three-term recurrences:  P_m^m = (2m-1)!! (1-t^2)^{m/2},
 * P_{m+1}^m = (2m+1) t P_m^m,
 * (n-m) P_n^m = (2n-1) t P_{n-1}^m - (n+m-1) P_{n-2}^m.
 * Output P[n*(nmax+1) + m]. */
static void legendre(int nmax, double t, double *P) {
    int w = nmax + 1;
    double s = sqrt(fmax(0.0, 1.0 - t * t));
    double pmm = 1.0;
    for (int m = 0; m <= nmax; m++) {
        if (m > 0) pmm *= (2.0 * m - 1.0) * s;
        P[m * w + m] = pmm;
        if (m + 1 <= nmax) P[(m + 1) * w + m] = (2.0 * m + 1.0) * t * pmm;
        for (int n = m + 2; n <= nmax; n++)
            P[n * w + m] = ((2.0 * n - 1.0) * t * P[(n - 1) * w + m]
                            - (n + m - 1.0) * P[(n - 2) * w + m]) / (double)(n - m);
    }
}

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; i++) f *= i;
    return f;
}

static void spherical(double x, double y, double z, double *r, double *ct, double *ph) {
    *r = sqrt(x * x + y * y + z * z);
    *ct = (*r > 0.0) ? z / *r : 1.0;
    *ph = atan2(y, x);
}

/* R_n^m(x) for all n <= nmax, m = -n..n. */
static void regular_harmonics(int nmax, double x, double y, double z, cplx *R) {
    double r, ct, ph;
    spherical(x, y, z, &r, &ct, &ph);
    double *P = malloc(sizeof(double) * (nmax + 1) * (nmax + 1));
    legendre(nmax, ct, P);
    for (int n = 0; n <= nmax; n++) {
        double rn = pow(r, n);
        for (int m = 0; m <= n; m++) {
            cplx v = rn * P[n * (nmax + 1) + m] / factorial(n + m) * cexp(I * (double)m * ph);
            R[hidx(n, m)] = v;
            R[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(v);
        }
    }
    free(P);
}

/* I_n^m(x) for all n <= nmax, m = -n..n (x != 0). */
static void irregular_harmonics(int nmax, double x, double y, double z, cplx *Ih) {
    double r, ct, ph;
    spherical(x, y, z, &r, &ct, &ph);
    double *P = malloc(sizeof(double) * (nmax + 1) * (nmax + 1));
    legendre(nmax, ct, P);
    for (int n = 0; n <= nmax; n++) {
        double rn1 = pow(r, n + 1);
        for (int m = 0; m <= n; m++) {
            cplx v = factorial(n - m) * P[n * (nmax + 1) + m] / rn1 * cexp(I * (double)m * ph);
            Ih[hidx(n, m)] = v;
            Ih[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(v);
        }
    }
    free(P);
}

/* ------------------------------------------------------------------ */
/* The six operators                                                   */
/* ------------------------------------------------------------------ */

/* P2M: M_n^m(c) += sum_j q_j R_n^m(x_j - c). */
void oracle_p2m(int p, const double *c, int64_t n, const double *pos, const double *q, cplx *M) {
    int K = (p + 1) * (p + 1);
    cplx *R = malloc(sizeof(cplx) * K);
    for (int64_t j = 0; j < n; j++) {
        regular_harmonics(p, pos[3 * j] - c[0], pos[3 * j + 1] - c[1], pos[3 * j + 2] - c[2], R);
        for (int i = 0; i < K; i++) M[i] += q[j] * R[i];
    }
    free(R);
}

/* M2M: child expansion about c + d ... parent about c:  d = c_child - c_parent. */
void oracle_m2m(int p, const cplx *Mc, const double *d, cplx *Mp) {
    int K = (p + 1) * (p + 1);
    cplx *R = malloc(sizeof(cplx) * K);
    regular_harmonics(p, d[0], d[1], d[2], R);
    for (int n = 0; n <= p; n++)
        for (int m = -n; m <= n; m++) {
            cplx acc = 0.0;
            for (int k = 0; k <= n; k++)
                for (int l = -k; l <= k; l++) {
                    int j = n - k, mm = m - l;
                    if (mm < -j || mm > j) continue;
                    acc += R[hidx(k, l)] * Mc[hidx(j, mm)];
                }
            Mp[hidx(n, m)] += acc;
        }
    free(R);
}

/* M2L: multipole about s -> local about t, D = t - s. */
void oracle_m2l(int p, const cplx *M, const double *D, cplx *L) {
    int K2 = (2 * p + 1) * (2 * p + 1);
    cplx *Ih = malloc(sizeof(cplx) * K2);
    irregular_harmonics(2 * p, D[0], D[1], D[2], Ih);
    for (int k = 0; k <= p; k++)
        for (int l = -k; l <= k; l++) {
            cplx acc = 0.0;
            for (int n = 0; n <= p; n++)
                for (int m = -n; m <= n; m++)
                    acc += M[hidx(n, m)] * conj(Ih[hidx(n + k, m + l)]);
            L[hidx(k, l)] += ((k & 1) ? -1.0 : 1.0) * acc;
        }
    free(Ih);
}

/* L2L: parent local about c -> child local about c + d. */
void oracle_l2l(int p, const cplx *Lp, const double *d, cplx *Lc) {
    int K = (p + 1) * (p + 1);
    cplx *R = malloc(sizeof(cplx) * K);
    regular_harmonics(p, d[0], d[1], d[2], R);
    for (int k = 0; k <= p; k++)
        for (int l = -k; l <= k; l++) {
            cplx acc = 0.0;
            for (int n = k; n <= p; n++)
                for (int m = -n; m <= n; m++) {
                    int j = n - k, mm = m - l;
                    if (mm < -j || mm > j) continue;
                    acc += Lp[hidx(n, m)] * R[hidx(j, mm)];
                }
            Lc[hidx(k, l)] += acc;
        }
    free(R);
}

/* L2P: phi(x) and grad phi(x) from a local expansion about c, y = x - c. */
void oracle_l2p(int p, const cplx *L, const double *y, double *phi, double *grad) {
    int K = (p + 1) * (p + 1);
    cplx *R = malloc(sizeof(cplx) * K);
    regular_harmonics(p, y[0], y[1], y[2], R);
#define RR(n, m) (((m) < -(n) || (m) > (n)) ? (cplx)0.0 : R[hidx((n), (m))])
    cplx f = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int n = 0; n <= p; n++)
        for (int m = -n; m <= n; m++) {
            cplx Lnm = L[hidx(n, m)];
            f += Lnm * R[hidx(n, m)];
            if (n == 0) continue;
            gz += Lnm * RR(n - 1, m);
            gx += Lnm * 0.5 * (RR(n - 1, m - 1) - RR(n - 1, m + 1));
            gy += Lnm * 0.5 * I * (RR(n - 1, m - 1) + RR(n - 1, m + 1));
        }
#undef RR
    *phi = creal(f);
    if (grad) { grad[0] = creal(gx); grad[1] = creal(gy); grad[2] = creal(gz); }
    free(R);
}

/* M2P: phi(x) from a multipole about c, y = x - c (|y| outside the sources). */
void oracle_m2p(int p, const cplx *M, const double *y, double *phi) {
    int K = (p + 1) * (p + 1);
    cplx *Ih = malloc(sizeof(cplx) * K);
    irregular_harmonics(p, y[0], y[1], y[2], Ih);
    cplx f = 0.0;
    for (int i = 0; i < K; i++) f += conj(M[i]) * Ih[i];
    *phi = creal(f);
    free(Ih);
}

/* ------------------------------------------------------------------ */
/* Direct sum (the exact result the FMM approximates)                  */
/* ------------------------------------------------------------------ */

/* phi_i = sum_{j != i, r_ij > 0} q_j / r_ij ;  grad phi_i = -sum q_j (x_i - x_j)/r^3.
 * Sources in ascending index order.  Targets listed in tidx (ntarget of them). */
void oracle_direct_targets(int64_t n, const double *pos, const double *q, int64_t ntarget,
                           const int64_t *tidx, double *phi, double *grad) {
    for (int64_t t = 0; t < ntarget; t++) {
        int64_t i = tidx[t];
        double f = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                   dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            f += q[j] / r;
            double s = q[j] / (r2 * r);
            g[0] -= s * dx; g[1] -= s * dy; g[2] -= s * dz;
        }
        phi[t] = f;
        if (grad) { grad[3 * t] = g[0]; grad[3 * t + 1] = g[1]; grad[3 * t + 2] = g[2]; }
    }
}

void oracle_direct(int64_t n, const double *pos, const double *q, double *phi, double *grad) {
    int64_t *idx = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) idx[i] = i;
    oracle_direct_targets(n, pos, q, n, idx, phi, grad);
    free(idx);
}

/* ------------------------------------------------------------------ */
/* Tree: root cube, Morton keys, octree, dual traversal                */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int32_t p_unused;
    int32_t ncell;
    int64_t nm2l, np2p;
    int32_t nlevel;         /* deepest level + 1 */
    int32_t leaf_size;
    double theta;
    double origin[3];
    double side;
    uint64_t *keys;         /* [n] full 63-bit keys, sorted */
    int64_t *perm;          /* [n] sorted slot -> input index */
    int32_t *level;         /* [ncell] */
    uint64_t *cell_key;     /* [ncell] key prefix (level*3 bits) */
    int64_t *first;         /* [ncell] first sorted particle */
    int64_t *count;         /* [ncell] particles */
    int32_t *parent;        /* [ncell] -1 for the root */
    int32_t *child_first;   /* [ncell] */
    int32_t *child_count;   /* [ncell] 0 for a leaf */
    int32_t *m2l;           /* [2*nm2l] (target, source) sorted */
    int32_t *p2p;           /* [2*np2p] (target, source) sorted */
} oracle_tree;

/* Root cube: lo/hi per axis, side = longest extent (1 if all coincide),
 * origin = midpoint - side/2.  Quantise k = clamp(floor((x - o) * 2^21/side)).
 * Every step is one IEEE round-to-nearest operation; this file is compiled
 * without FMA contraction so the CUDA path can reproduce the keys bit for bit. */
static void root_cube(int64_t n, const double *pos, double *origin, double *side) {
    double lo[3], hi[3];
    for (int d = 0; d < 3; d++) { lo[d] = pos[d]; hi[d] = pos[d]; }
    for (int64_t i = 1; i < n; i++)
        for (int d = 0; d < 3; d++) {
            double v = pos[3 * i + d];
            if (v < lo[d]) lo[d] = v;
            if (v > hi[d]) hi[d] = v;
        }
    double s = 0.0;
    for (int d = 0; d < 3; d++) { double e = hi[d] - lo[d]; if (e > s) s = e; }
    if (s == 0.0) s = 1.0;
    for (int d = 0; d < 3; d++) origin[d] = (lo[d] + hi[d]) * 0.5 - s * 0.5;
    *side = s;
}

static uint64_t quantise(double x, double o, double inv) {
    double v = floor((x - o) * inv);
    if (v < 0.0) v = 0.0;
    if (v > 2097151.0) v = 2097151.0;
    return (uint64_t)v;
}

/* Morton interleave: bit b of kx -> 3b, of ky -> 3b+1, of kz -> 3b+2. */
static uint64_t morton(uint64_t kx, uint64_t ky, uint64_t kz) {
    uint64_t key = 0;
    for (int b = 0; b < MAXLEVEL; b++) {
        key |= ((kx >> b) & 1ull) << (3 * b);
        key |= ((ky >> b) & 1ull) << (3 * b + 1);
        key |= ((kz >> b) & 1ull) << (3 * b + 2);
    }
    return key;
}

static void demorton(uint64_t key, int64_t *k) {
    k[0] = k[1] = k[2] = 0;
    for (int b = 0; b < MAXLEVEL; b++) {
        k[0] |= (int64_t)((key >> (3 * b)) & 1ull) << b;
        k[1] |= (int64_t)((key >> (3 * b + 1)) & 1ull) << b;
        k[2] |= (int64_t)((key >> (3 * b + 2)) & 1ull) << b;
    }
}

typedef struct { uint64_t key; int64_t idx; } keyidx;

static int cmp_keyidx(const void *a, const void *b) {
    const keyidx *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

typedef struct { int32_t t, s; } pair32;

static int cmp_pair(const void *a, const void *b) {
    const pair32 *x = a, *y = b;
    if (x->t != y->t) return x->t < y->t ? -1 : 1;
    return (x->s > y->s) - (x->s < y->s);
}

/* growable arrays */
typedef struct { void *data; int64_t n, cap; size_t elem; } vec;
static void vpush(vec *v, const void *e) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->data = realloc(v->data, v->cap * v->elem);
    }
    memcpy((char *)v->data + v->n * v->elem, e, v->elem);
    v->n++;
}

/* Cell geometry in integer units u = side / 2^21: size s = 2^(21-l) and twice
 * the centre, 2c = 2*kc*s + s per axis (kc = cell coordinate at its level). */
static void cell_geom(const oracle_tree *t, int c, int64_t *s, int64_t *twoc) {
    int l = t->level[c];
    *s = (int64_t)1 << (MAXLEVEL - l);
    int64_t kc[3];
    demorton(t->cell_key[c], kc);  /* prefix of 3l bits -> l-bit coordinates */
    for (int d = 0; d < 3; d++) twoc[d] = 2 * kc[d] * (*s) + (*s);
}

/* Expansion centre of cell c in input coordinates (the geometric centre). */
static void cell_centre(const oracle_tree *t, int c, double *x) {
    int64_t s, twoc[3];
    cell_geom(t, c, &s, twoc);
    double u2 = t->side / 4194304.0; /* side / 2^22 : the unit of 2c */
    for (int d = 0; d < 3; d++) x[d] = t->origin[d] + (double)twoc[d] * u2;
}

static int is_leaf(const oracle_tree *t, int c) { return t->child_count[c] == 0; }

/* Multipole acceptance: (s_i + s_j)^2 < theta^2 |D|^2, D = 2c_i - 2c_j, all in
 * units u.  The cell radius is taken as half the side, so the test reads
 * R_i + R_j < theta * distance of centres.  The left side is an exact integer,
 * the right side is (theta*theta) * |D|^2 in two rounded FP64 products. */
static int mac_accept(const oracle_tree *t, int ci, int cj) {
    int64_t si, sj, ci2[3], cj2[3];
    cell_geom(t, ci, &si, ci2);
    cell_geom(t, cj, &sj, cj2);
    int64_t D2 = 0;
    for (int d = 0; d < 3; d++) { int64_t e = ci2[d] - cj2[d]; D2 += e * e; }
    int64_t S = si + sj;
    double lhs = (double)(S * S);
    double th2 = t->theta * t->theta;
    double rhs = th2 * (double)D2;
    return lhs < rhs;
}

oracle_tree *oracle_build_tree(int64_t n, const double *pos, int32_t leaf_size, double theta) {
    oracle_tree *t = calloc(1, sizeof(oracle_tree));
    t->n = n; t->leaf_size = leaf_size; t->theta = theta;
    t->keys = malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    t->perm = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (n == 0) {
        t->side = 1.0;
        return t;
    }
    /* O2: root cube and quantisation; O3: keys */
    root_cube(n, pos, t->origin, &t->side);
    double inv = 2097152.0 / t->side;
    keyidx *ki = malloc(sizeof(keyidx) * n);
    for (int64_t i = 0; i < n; i++) {
        uint64_t kx = quantise(pos[3 * i], t->origin[0], inv);
        uint64_t ky = quantise(pos[3 * i + 1], t->origin[1], inv);
        uint64_t kz = quantise(pos[3 * i + 2], t->origin[2], inv);
        ki[i].key = morton(kx, ky, kz);
        ki[i].idx = i;
    }
    /* O4: stable sort (ties by input index) */
    qsort(ki, n, sizeof(keyidx), cmp_keyidx);
    for (int64_t i = 0; i < n; i++) { t->keys[i] = ki[i].key; t->perm[i] = ki[i].idx; }
    free(ki);

    /* O4: octree, built level by level so cells come out ordered by (level, key).
     * A cell at level l holds the particles that share its 3l top key bits; it
     * splits iff count > leaf_size and l < 21; empty children are not made. */
    vec lev = {0, 0, 0, sizeof(int32_t)}, ck = {0, 0, 0, sizeof(uint64_t)},
        fi = {0, 0, 0, sizeof(int64_t)}, co = {0, 0, 0, sizeof(int64_t)},
        pa = {0, 0, 0, sizeof(int32_t)};
    int32_t l0 = 0, m1 = -1; uint64_t k0 = 0; int64_t f0 = 0;
    vpush(&lev, &l0); vpush(&ck, &k0); vpush(&fi, &f0); vpush(&co, &n); vpush(&pa, &m1);
    int64_t begin = 0, end = 1;
    int level = 0;
    while (begin < end) {
        for (int64_t c = begin; c < end; c++) {
            int64_t cf = ((int64_t *)fi.data)[c], cc = ((int64_t *)co.data)[c];
            if (!(cc > leaf_size && level < MAXLEVEL)) continue;
            int shift = 3 * (MAXLEVEL - (level + 1));
            int64_t i = cf;
            while (i < cf + cc) {
                uint64_t pre = t->keys[i] >> shift;
                int64_t j = i;
                while (j < cf + cc && (t->keys[j] >> shift) == pre) j++;
                int32_t lv = level + 1, par = (int32_t)c;
                int64_t cnt = j - i;
                vpush(&lev, &lv); vpush(&ck, &pre); vpush(&fi, &i); vpush(&co, &cnt); vpush(&pa, &par);
                i = j;
            }
        }
        begin = end;
        end = lev.n;
        level++;
    }
    t->ncell = (int32_t)lev.n;
    t->level = lev.data; t->cell_key = ck.data; t->first = fi.data; t->count = co.data;
    t->parent = pa.data;
    t->child_first = malloc(sizeof(int32_t) * t->ncell);
    t->child_count = calloc(t->ncell, sizeof(int32_t));
    for (int c = 0; c < t->ncell; c++) t->child_first[c] = -1;
    int maxl = 0;
    for (int c = 1; c < t->ncell; c++) {
        int par = t->parent[c];
        if (t->child_first[par] < 0) t->child_first[par] = c;
        t->child_count[par]++;
    }
    for (int c = 0; c < t->ncell; c++) {
        if (t->child_first[c] < 0) t->child_first[c] = 0;
        if (t->level[c] > maxl) maxl = t->level[c];
    }
    t->nlevel = maxl + 1;

    /* O6: breadth-first dual traversal from (root, root) with a FIFO queue. */
    vec q = {0, 0, 0, sizeof(pair32)}, vm = {0, 0, 0, sizeof(pair32)}, vp = {0, 0, 0, sizeof(pair32)};
    pair32 root = {0, 0};
    vpush(&q, &root);
    for (int64_t h = 0; h < q.n; h++) {
        pair32 pr = ((pair32 *)q.data)[h];
        int ci = pr.t, cj = pr.s;
        if (mac_accept(t, ci, cj)) { vpush(&vm, &pr); continue; }
        int li = is_leaf(t, ci), lj = is_leaf(t, cj);
        if (li && lj) { vpush(&vp, &pr); continue; }
        /* split the larger cell; on equal size (or a leaf source) split the target */
        if (lj || (!li && t->level[ci] <= t->level[cj])) {
            for (int k = 0; k < t->child_count[ci]; k++) {
                pair32 np = {t->child_first[ci] + k, cj};
                vpush(&q, &np);
            }
        } else {
            for (int k = 0; k < t->child_count[cj]; k++) {
                pair32 np = {ci, t->child_first[cj] + k};
                vpush(&q, &np);
            }
        }
    }
    free(q.data);
    qsort(vm.data, vm.n, sizeof(pair32), cmp_pair);
    qsort(vp.data, vp.n, sizeof(pair32), cmp_pair);
    t->nm2l = vm.n; t->np2p = vp.n;
    t->m2l = vm.data ? vm.data : malloc(8);
    t->p2p = vp.data ? vp.data : malloc(8);
    return t;
}

void oracle_free_tree(oracle_tree *t) {
    if (!t) return;
    free(t->keys); free(t->perm); free(t->level); free(t->cell_key); free(t->first);
    free(t->count); free(t->parent); free(t->child_first); free(t->child_count);
    free(t->m2l); free(t->p2p); free(t);
}

/* ------------------------------------------------------------------ */
/* FMM evaluation (O8)                                                 */
/* ------------------------------------------------------------------ */

typedef struct {
    const oracle_tree *t;
    int p, K;
    const double *spos;   /* sorted positions [n*3] */
    const double *sq;     /* sorted charges [n] */
    cplx *M, *L;
    double *centre;       /* [ncell*3] */
    int64_t *m2l_start;   /* CSR over targets [ncell+1] */
    int64_t *p2p_start;
    double *phi, *grad;   /* sorted outputs */
    /* work split */
    const int32_t *items;
    int64_t nitems;
    int stage;
    int nthreads;
} eval_ctx;

typedef struct { eval_ctx *e; int tid; } worker_arg;

static void near_field(eval_ctx *e, int c) {
    const oracle_tree *t = e->t;
    for (int64_t i = t->first[c]; i < t->first[c] + t->count[c]; i++) {
        double f = 0.0, g[3] = {0, 0, 0};
        for (int64_t k = e->p2p_start[c]; k < e->p2p_start[c + 1]; k++) {
            int s = t->p2p[2 * k + 1];
            for (int64_t j = t->first[s]; j < t->first[s] + t->count[s]; j++) {
                if (j == i) continue;
                double dx = e->spos[3 * i] - e->spos[3 * j], dy = e->spos[3 * i + 1] - e->spos[3 * j + 1],
                       dz = e->spos[3 * i + 2] - e->spos[3 * j + 2];
                double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 == 0.0) continue;
                double r = sqrt(r2);
                f += e->sq[j] / r;
                double w = e->sq[j] / (r2 * r);
                g[0] -= w * dx; g[1] -= w * dy; g[2] -= w * dz;
            }
        }
        e->phi[i] += f;
        e->grad[3 * i] += g[0]; e->grad[3 * i + 1] += g[1]; e->grad[3 * i + 2] += g[2];
    }
}

static void far_field_eval(eval_ctx *e, int c) {
    const oracle_tree *t = e->t;
    for (int64_t i = t->first[c]; i < t->first[c] + t->count[c]; i++) {
        double y[3], f, g[3];
        for (int d = 0; d < 3; d++) y[d] = e->spos[3 * i + d] - e->centre[3 * c + d];
        oracle_l2p(e->p, e->L + (int64_t)c * e->K, y, &f, g);
        e->phi[i] += f;
        for (int d = 0; d < 3; d++) e->grad[3 * i + d] += g[d];
    }
}

static void m2l_target(eval_ctx *e, int c) {
    const oracle_tree *t = e->t;
    for (int64_t k = e->m2l_start[c]; k < e->m2l_start[c + 1]; k++) {
        int s = t->m2l[2 * k + 1];
        double D[3];
        for (int d = 0; d < 3; d++) D[d] = e->centre[3 * c + d] - e->centre[3 * s + d];
        oracle_m2l(e->p, e->M + (int64_t)s * e->K, D, e->L + (int64_t)c * e->K);
    }
}

static void p2m_leaf(eval_ctx *e, int c) {
    const oracle_tree *t = e->t;
    oracle_p2m(e->p, e->centre + 3 * c, t->count[c], e->spos + 3 * t->first[c], e->sq + t->first[c],
               e->M + (int64_t)c * e->K);
}

static void *worker(void *arg) {
    worker_arg *wa = arg;
    eval_ctx *e = wa->e;
    for (int64_t k = wa->tid; k < e->nitems; k += e->nthreads) {
        int c = e->items[k];
        if (e->stage == 0) p2m_leaf(e, c);
        else if (e->stage == 2) m2l_target(e, c);
        else if (e->stage == 4) { far_field_eval(e, c); near_field(e, c); }
    }
    return NULL;
}

static void run_stage(eval_ctx *e, int stage, const int32_t *items, int64_t nitems) {
    e->stage = stage; e->items = items; e->nitems = nitems;
    if (e->nthreads <= 1) {
        worker_arg wa = {e, 0};
        int keep = e->nthreads; e->nthreads = 1;
        worker(&wa);
        e->nthreads = keep;
        return;
    }
    pthread_t *th = malloc(sizeof(pthread_t) * e->nthreads);
    worker_arg *wa = malloc(sizeof(worker_arg) * e->nthreads);
    for (int i = 0; i < e->nthreads; i++) { wa[i].e = e; wa[i].tid = i; pthread_create(&th[i], NULL, worker, &wa[i]); }
    for (int i = 0; i < e->nthreads; i++) pthread_join(th[i], NULL);
    free(th); free(wa);
}

static int64_t *csr_of(const int32_t *pairs, int64_t npair, int ncell) {
    int64_t *st = calloc(ncell + 1, sizeof(int64_t));
    for (int64_t k = 0; k < npair; k++) st[pairs[2 * k] + 1]++;
    for (int c = 0; c < ncell; c++) st[c + 1] += st[c];
    return st;
}

/* Set up sorted inputs, centres, and the upward pass (P2M, then M2M by
 * descending level).  Returns an initialised context. */
static void eval_setup(eval_ctx *e, const oracle_tree *t, const double *pos, int p, const double *q, int nthreads) {
    int64_t n = t->n;
    memset(e, 0, sizeof(*e));
    e->t = t; e->p = p; e->K = (p + 1) * (p + 1); e->nthreads = nthreads;
    double *spos = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    double *sq = malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        for (int d = 0; d < 3; d++) spos[3 * i + d] = pos[3 * t->perm[i] + d];
        sq[i] = q[t->perm[i]];
    }
    e->spos = spos; e->sq = sq;
    int nc = t->ncell;
    e->M = calloc((size_t)nc * e->K + 1, sizeof(cplx));
    e->L = calloc((size_t)nc * e->K + 1, sizeof(cplx));
    e->centre = malloc(sizeof(double) * 3 * (nc + 1));
    for (int c = 0; c < nc; c++) cell_centre(t, c, e->centre + 3 * c);
    e->m2l_start = csr_of(t->m2l, t->nm2l, nc);
    e->p2p_start = csr_of(t->p2p, t->np2p, nc);
    /* P2M on every leaf */
    int32_t *leaves = malloc(sizeof(int32_t) * (nc + 1));
    int64_t nl = 0;
    for (int c = 0; c < nc; c++) if (is_leaf(t, c)) leaves[nl++] = c;
    run_stage(e, 0, leaves, nl);
    free(leaves);
    /* M2M, children before parents: cells are ordered by level, so walk backwards */
    for (int c = nc - 1; c >= 1; c--) {
        int par = t->parent[c];
        double d[3];
        for (int k = 0; k < 3; k++) d[k] = e->centre[3 * c + k] - e->centre[3 * par + k];
        oracle_m2m(p, e->M + (int64_t)c * e->K, d, e->M + (int64_t)par * e->K);
    }
}

static void eval_free(eval_ctx *e) {
    free((void *)e->spos); free((void *)e->sq); free(e->M); free(e->L); free(e->centre);
    free(e->m2l_start); free(e->p2p_start);
}

/* Full FMM: phi and grad phi for every particle, in INPUT order.
 * nthreads > 1 splits M2L and the leaf evaluation over target cells; each
 * target's arithmetic is the same for any thread count. */
void oracle_fmm_evaluate(const oracle_tree *t, const double *pos, int p, const double *q,
                         double *phi, double *grad, int nthreads) {
    int64_t n = t->n;
    if (n == 0) return;
    eval_ctx e;
    eval_setup(&e, t, pos, p, q, nthreads);
    int nc = t->ncell;
    int32_t *all = malloc(sizeof(int32_t) * nc);
    for (int c = 0; c < nc; c++) all[c] = c;
    run_stage(&e, 2, all, nc);                 /* M2L over each target's list */
    for (int c = 1; c < nc; c++) {             /* L2L, parents before children */
        int par = t->parent[c];
        double d[3];
        for (int k = 0; k < 3; k++) d[k] = e.centre[3 * c + k] - e.centre[3 * par + k];
        oracle_l2l(p, e.L + (int64_t)par * e.K, d, e.L + (int64_t)c * e.K);
    }
    double *sphi = calloc(n, sizeof(double)), *sgrad = calloc(3 * n, sizeof(double));
    e.phi = sphi; e.grad = sgrad;
    int64_t nl = 0;
    for (int c = 0; c < nc; c++) if (is_leaf(t, c)) all[nl++] = c;
    run_stage(&e, 4, all, nl);                 /* L2P + P2P per leaf */
    for (int64_t i = 0; i < n; i++) {
        int64_t o = t->perm[i];
        phi[o] = sphi[i];
        if (grad) for (int d = 0; d < 3; d++) grad[3 * o + d] = sgrad[3 * i + d];
    }
    free(sphi); free(sgrad); free(all);
    eval_free(&e);
}

/* Sampled FMM: the same result as oracle_fmm_evaluate, but only for the
 * particles of the listed leaves.  The upward pass runs on every cell; the
 * local expansion is built only along each sampled leaf's ancestor chain.
 * Outputs are in SORTED order of the sampled leaves' particles, concatenated
 * in the order of `leaves`. */
void oracle_fmm_evaluate_leaves(const oracle_tree *t, const double *pos, int p, const double *q,
                                int64_t nleaves, const int32_t *leaves, double *phi, double *grad) {
    if (t->n == 0) return;
    eval_ctx e;
    eval_setup(&e, t, pos, p, q, 1);
    int64_t out = 0;
    int chain[MAXLEVEL + 2];
    double *lphi = calloc(t->n, sizeof(double)), *lgrad = calloc(3 * t->n, sizeof(double));
    e.phi = lphi; e.grad = lgrad;
    for (int64_t s = 0; s < nleaves; s++) {
        int c = leaves[s], depth = 0;
        for (int a = c; a >= 0; a = t->parent[a]) chain[depth++] = a;
        for (int k = depth - 1; k >= 0; k--) {
            int a = chain[k];
            memset(e.L + (int64_t)a * e.K, 0, sizeof(cplx) * e.K);
            m2l_target(&e, a);
            if (k < depth - 1) {
                int par = chain[k + 1];
                double d[3];
                for (int x = 0; x < 3; x++) d[x] = e.centre[3 * a + x] - e.centre[3 * par + x];
                oracle_l2l(p, e.L + (int64_t)par * e.K, d, e.L + (int64_t)a * e.K);
            }
        }
        far_field_eval(&e, c);
        near_field(&e, c);
        for (int64_t i = t->first[c]; i < t->first[c] + t->count[c]; i++, out++) {
            phi[out] = lphi[i];
            if (grad) for (int d = 0; d < 3; d++) grad[3 * out + d] = lgrad[3 * i + d];
            lphi[i] = 0.0; lgrad[3 * i] = lgrad[3 * i + 1] = lgrad[3 * i + 2] = 0.0;
        }
    }
    free(lphi); free(lgrad);
    eval_free(&e);
}
