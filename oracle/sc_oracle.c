/*
 * CPU oracle for coupled-configuration generation, de-duplication and the
 * variational energy.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the benchmark's CPU-baseline leg call it; the library never does.  It shares
 * no code with the CUDA path.
 *
 * Plain FP64, no blocking, no tables, no fused multiply-add (build with
 * -ffp-contract=off).  Every matrix element is the Slater-Condon closed form
 * written out, with the fermionic phase taken by applying the creation and
 * annihilation operators one at a time.
 *
 * Conventions (the paper leaves them open, Sec. 2.1 / Sec. 4.2.1):
 *  - norb spatial orbitals; spin orbital s = 2p + sigma (sigma 0 = alpha,
 *    1 = beta); bit s of a determinant is bit (s & 63) of word (s >> 6).
 *  - H = Ecore + sum_{pq,sigma} h_pq a+_{p sigma} a_{q sigma}
 *        + 1/2 sum_{pqrs,sigma tau} (pq|rs) a+_{p sigma} a+_{r tau} a_{s tau} a_{q sigma}
 *    with real chemists'-notation integrals, h2[((p*n+q)*n+r)*n+s] = (pq|rs).
 *  - a_s or a+_s acting on D gives the phase (-1)^(number of occupied spin
 *    orbitals below s) and toggles bit s.
 *
 * Coupled set C_i (Sec. 2.1: every j with H_ij != 0, reached by moving one or
 * two electrons; j = i included), emitted in the canonical order:
 *   1. the diagonal (always kept);
 *   2. singles, occupied i ascending, then same-spin virtual a ascending;
 *   3. doubles, occupied pairs (i<j) lexicographic, then (a,b) lexicographic
 *      with a<b for a same-spin pair and a of i's spin, b of j's spin otherwise.
 * Off-diagonal entries are kept iff |H| > eps (the screening test of
 * Algorithm 1; eps < 0 keeps every structural excitation).
 *
 * Summation orders (fixed here, matched by any implementation that claims
 * bit-exact elements):
 *   diagonal: e1 = sum_{i in O} h_ii (i ascending), e2 = sum over pairs i<j of O
 *             (lexicographic) of  +(ii|jj)  then, same spin only,  -(ij|ji);
 *             H = (Ecore + e1) + e2.
 *   single i->a: acc = h_ai; for k in O ascending, k != i:
 *             acc += (ai|kk); if spin(k) == spin(a): acc -= (ak|ki).
 *             H = phase * acc.
 *   double: same spin  H = phase * ((ai|bj) - (aj|bi)),
 *           opposite   H = phase * (ai|bj)      (integrals on spatial indices).
 *
 * De-duplication (Sec. 4.1, "local unique"): sorted unique list of W-word keys
 * in numeric order (word W-1 most significant) and, per key, its position in
 * that list.
 *
 * Energy (Sec. 2.1, the Rayleigh quotient restricted to the selected set S):
 * (H psi)_i = sum over j in C_i that are members of S of H_ij psi_j, in
 * canonical order; E = sum psi_i (H psi)_i / sum psi_i^2 (both sums Neumaier
 * compensated in index order); dE/dpsi_i = 2 ((H psi)_i - E psi_i) / sum psi^2.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXW 4
#define ORC_MAXSO 256

typedef struct {
    int norb, n_alpha, n_beta, W;
    const double *h1, *h2;
    double ecore;
} orc_sys;

static double I1(const orc_sys *s, int p, int q) { return s->h1[p * s->norb + q]; }
static double I2(const orc_sys *s, int p, int q, int r, int t) {
    int n = s->norb;
    return s->h2[(((size_t)p * n + q) * n + r) * n + t];
}

static int bit_of(const uint64_t *d, int s) { return (int)((d[s >> 6] >> (s & 63)) & 1u); }
static void toggle(uint64_t *d, int s) { d[s >> 6] ^= (uint64_t)1 << (s & 63); }

/* number of occupied spin orbitals with index below s, one bit at a time */
static int occupied_below(const uint64_t *d, int s) {
    int c = 0;
    for (int t = 0; t < s; t++) c += bit_of(d, t);
    return c;
}

/* apply a+_s (create = 1) or a_s (create = 0) to d; returns 0 if the result
 * vanishes, else the phase +1 / -1, and d becomes the new determinant. */
static int apply_op(uint64_t *d, int s, int create) {
    int occ = bit_of(d, s);
    if (create ? occ : !occ) return 0;
    int phase = (occupied_below(d, s) & 1) ? -1 : 1;
    toggle(d, s);
    return phase;
}

int orc_apply_op(uint64_t *d, int s, int create) { return apply_op(d, s, create); }

typedef struct {
    uint64_t *dets; /* nullable */
    double *h;      /* nullable */
    int64_t n;
    int W;
} sink;

static void emit(sink *k, const uint64_t *det, double h) {
    if (k->dets) memcpy(k->dets + (size_t)k->n * k->W, det, sizeof(uint64_t) * k->W);
    if (k->h) k->h[k->n] = h;
    k->n++;
}

/* the coupled set of one determinant, in canonical order */
static void coupled_one(const orc_sys *s, const uint64_t *det, double eps, sink *out) {
    const int W = s->W, M = 2 * s->norb;
    int occ[ORC_MAXSO], nocc = 0;
    int vir[2][ORC_MAXSO], nvir[2] = {0, 0};
    for (int t = 0; t < M; t++) {
        if (bit_of(det, t)) occ[nocc++] = t;
        else { vir[t & 1][nvir[t & 1]++] = t; }
    }
    uint64_t work[ORC_MAXW];

    /* 1. diagonal */
    double e1 = 0.0, e2 = 0.0;
    for (int x = 0; x < nocc; x++) e1 += I1(s, occ[x] >> 1, occ[x] >> 1);
    for (int x = 0; x < nocc; x++)
        for (int y = x + 1; y < nocc; y++) {
            int i = occ[x], j = occ[y], pi = i >> 1, pj = j >> 1;
            e2 += I2(s, pi, pi, pj, pj);
            if ((i & 1) == (j & 1)) e2 -= I2(s, pi, pj, pj, pi);
        }
    emit(out, det, (s->ecore + e1) + e2);

    /* 2. singles */
    for (int x = 0; x < nocc; x++) {
        int i = occ[x], sg = i & 1, pi = i >> 1;
        for (int y = 0; y < nvir[sg]; y++) {
            int a = vir[sg][y], pa = a >> 1;
            memcpy(work, det, sizeof(uint64_t) * W);
            int ph = apply_op(work, i, 0);
            ph *= apply_op(work, a, 1);
            double acc = I1(s, pa, pi);
            for (int z = 0; z < nocc; z++) {
                int k = occ[z], pk = k >> 1;
                if (k == i) continue;
                acc += I2(s, pa, pi, pk, pk);
                if ((k & 1) == (a & 1)) acc -= I2(s, pa, pk, pk, pi);
            }
            double h = (double)ph * acc;
            if (fabs(h) > eps) emit(out, work, h);
        }
    }

    /* 3. doubles */
    for (int x = 0; x < nocc; x++)
        for (int y = x + 1; y < nocc; y++) {
            int i = occ[x], j = occ[y], si = i & 1, sj = j & 1;
            int pi = i >> 1, pj = j >> 1;
            for (int u = 0; u < nvir[si]; u++) {
                int a = vir[si][u], pa = a >> 1;
                for (int v = 0; v < nvir[sj]; v++) {
                    int b = vir[sj][v], pb = b >> 1;
                    if (si == sj && b <= a) continue;
                    double val = I2(s, pa, pi, pb, pj);
                    if (si == sj) val = val - I2(s, pa, pj, pb, pi);
                    memcpy(work, det, sizeof(uint64_t) * W);
                    int ph = apply_op(work, i, 0);
                    ph *= apply_op(work, j, 0);
                    ph *= apply_op(work, b, 1);
                    ph *= apply_op(work, a, 1);
                    double h = (double)ph * val;
                    if (fabs(h) > eps) emit(out, work, h);
                }
            }
        }
}

static orc_sys make_sys(int norb, int na, int nb, const double *h1, const double *h2, double ecore) {
    orc_sys s;
    s.norb = norb; s.n_alpha = na; s.n_beta = nb; s.W = (2 * norb + 63) / 64;
    s.h1 = h1; s.h2 = h2; s.ecore = ecore;
    return s;
}

/* counts[k] = |C_k| after screening; returns the total */
int64_t orc_count(int norb, int na, int nb, const double *h1, const double *h2, double ecore,
                  const uint64_t *dets, int64_t n, double eps, int64_t *counts) {
    orc_sys s = make_sys(norb, na, nb, h1, h2, ecore);
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (int64_t k = 0; k < n; k++) {
        sink z = {NULL, NULL, 0, s.W};
        coupled_one(&s, dets + (size_t)k * s.W, eps, &z);
        counts[k] = z.n;
        total += z.n;
    }
    return total;
}

/* writes C_k to rows [offsets[k], offsets[k+1]) of out_dets / out_h */
void orc_gen(int norb, int na, int nb, const double *h1, const double *h2, double ecore,
             const uint64_t *dets, int64_t n, double eps, const int64_t *offsets,
             uint64_t *out_dets, double *out_h) {
    orc_sys s = make_sys(norb, na, nb, h1, h2, ecore);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; k++) {
        sink z = {out_dets + (size_t)offsets[k] * s.W, out_h + offsets[k], 0, s.W};
        coupled_one(&s, dets + (size_t)k * s.W, eps, &z);
    }
}

/* ---------------- de-duplication ---------------- */

static int cmp_words(const uint64_t *x, const uint64_t *y, int W) {
    for (int w = W - 1; w >= 0; w--) {
        if (x[w] < y[w]) return -1;
        if (x[w] > y[w]) return 1;
    }
    return 0;
}

static int cmp_qsort(const void *x, const void *y, void *arg) {
    return cmp_words((const uint64_t *)x, (const uint64_t *)y, *(const int *)arg);
}

/* first position of key in sorted[0..n) (n if absent) */
static int64_t lower_bound_words(const uint64_t *sorted, int64_t n, const uint64_t *key, int W) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cmp_words(sorted + (size_t)mid * W, key, W) < 0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* unique: capacity total*W; inverse: total entries; returns the unique count */
int64_t orc_dedup(const uint64_t *keys, int64_t total, int W, uint64_t *unique, int64_t *inverse) {
    if (total == 0) return 0;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * W * (size_t)total);
    if (!tmp) return -1;
    memcpy(tmp, keys, sizeof(uint64_t) * W * (size_t)total);
    qsort_r(tmp, (size_t)total, sizeof(uint64_t) * W, cmp_qsort, &W);
    int64_t nu = 0;
    for (int64_t k = 0; k < total; k++) {
        const uint64_t *x = tmp + (size_t)k * W;
        if (nu == 0 || cmp_words(unique + (size_t)(nu - 1) * W, x, W) != 0) {
            memcpy(unique + (size_t)nu * W, x, sizeof(uint64_t) * W);
            nu++;
        }
    }
    free(tmp);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < total; k++)
        inverse[k] = lower_bound_words(unique, nu, keys + (size_t)k * W, W);
    return nu;
}

/* ---------------- energy ---------------- */

typedef struct { double sum, comp; } neumaier;
static void nm_add(neumaier *a, double x) {
    double t = a->sum + x;
    if (fabs(a->sum) >= fabs(x)) a->comp += (a->sum - t) + x;
    else a->comp += (x - t) + a->sum;
    a->sum = t;
}
static double nm_value(const neumaier *a) { return a->sum + a->comp; }

/* (H psi)_i restricted to S (Eq. 1 with j running over S only) for one row i
 * of the sorted unique set S: every entry of C_i, in canonical order, whose
 * target is found in S by binary search contributes H_ij psi_j.  dbuf / hbuf
 * (capacity *cap entries) are grown as needed. */
static double hpsi_row(const orc_sys *s, const uint64_t *S, int64_t nS, const double *psi,
                       double eps, int64_t i, uint64_t **dbuf, double **hbuf, int64_t *cap) {
    const int W = s->W;
    sink c = {NULL, NULL, 0, W};
    coupled_one(s, S + (size_t)i * W, eps, &c);
    if (c.n > *cap) {
        *cap = c.n;
        *dbuf = (uint64_t *)realloc(*dbuf, sizeof(uint64_t) * W * *cap);
        *hbuf = (double *)realloc(*hbuf, sizeof(double) * *cap);
    }
    sink z = {*dbuf, *hbuf, 0, W};
    coupled_one(s, S + (size_t)i * W, eps, &z);
    double acc = 0.0;
    for (int64_t e = 0; e < z.n; e++) {
        const uint64_t *jd = *dbuf + (size_t)e * W;
        int64_t j = lower_bound_words(S, nS, jd, W);
        if (j < nS && cmp_words(S + (size_t)j * W, jd, W) == 0) acc += (*hbuf)[e] * psi[j];
    }
    return acc;
}

/* (H psi)_i restricted to S, for every i of the sorted unique set S */
void orc_hpsi(int norb, int na, int nb, const double *h1, const double *h2, double ecore,
              const uint64_t *S, int64_t nS, const double *psi, double eps, double *hpsi) {
    orc_sys s = make_sys(norb, na, nb, h1, h2, ecore);
#pragma omp parallel
    {
        int64_t cap = 1 << 16;
        uint64_t *dbuf = (uint64_t *)malloc(sizeof(uint64_t) * s.W * cap);
        double *hbuf = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < nS; i++)
            hpsi[i] = hpsi_row(&s, S, nS, psi, eps, i, &dbuf, &hbuf, &cap);
        free(dbuf);
        free(hbuf);
    }
}

/* the same (H psi)_i for the chosen rows only: out[r] = (H psi)_{rows[r]} */
void orc_hpsi_rows(int norb, int na, int nb, const double *h1, const double *h2, double ecore,
                   const uint64_t *S, int64_t nS, const double *psi, double eps,
                   const int64_t *rows, int64_t nrows, double *out) {
    orc_sys s = make_sys(norb, na, nb, h1, h2, ecore);
#pragma omp parallel
    {
        int64_t cap = 1 << 16;
        uint64_t *dbuf = (uint64_t *)malloc(sizeof(uint64_t) * s.W * cap);
        double *hbuf = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < nrows; r++)
            out[r] = hpsi_row(&s, S, nS, psi, eps, rows[r], &dbuf, &hbuf, &cap);
        free(dbuf);
        free(hbuf);
    }
}

/* E and sum psi^2 from psi and H psi */
void orc_energy_reduce(const double *psi, const double *hpsi, int64_t nS, double *E, double *norm2) {
    neumaier num = {0.0, 0.0}, den = {0.0, 0.0};
    for (int64_t i = 0; i < nS; i++) {
        nm_add(&num, psi[i] * hpsi[i]);
        nm_add(&den, psi[i] * psi[i]);
    }
    *norm2 = nm_value(&den);
    *E = nm_value(&num) / *norm2;
}

/* grad_i = g * 2 ((H psi)_i - E psi_i) / norm2 */
void orc_energy_grad(const double *psi, const double *hpsi, int64_t nS, double E, double norm2,
                     double g, double *grad) {
    for (int64_t i = 0; i < nS; i++) grad[i] = g * (2.0 * (hpsi[i] - E * psi[i]) / norm2);
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------- local energy (Eq. 5 form) ----------------
 * Coupled lists of the sources S in CSR form (offsets[n+1], H per entry) and,
 * per entry, the index of its target in the distinct set U (inverse); psi_u
 * are the amplitudes on U.  The source i is its own first entry (the diagonal),
 * so psi_i = psi_u[inverse[offsets[i]]].
 *   y_i = sum_{e in row i} H_e psi_u[inverse[e]]   (entries in order)
 *   E   = sum_i psi_i y_i / sum_i psi_i^2           (Neumaier, index order)
 *   dE/dpsi_u[u] = ( sum_{e: inverse[e] = u} psi_{i(e)} H_e
 *                    + sum_{i: s(i) = u} (y_i - 2 E psi_i) ) / sum psi_i^2
 * (times the incoming gradient g). */
void orc_local_energy(const int64_t *offsets, int64_t n, const double *h, const int64_t *inverse,
                      const double *psi_u, int64_t n_unique, double g, double *y, double *E,
                      double *norm2, double *grad_u) {
    neumaier num = {0.0, 0.0}, den = {0.0, 0.0};
    for (int64_t i = 0; i < n; i++) {
        double acc = 0.0;
        for (int64_t e = offsets[i]; e < offsets[i + 1]; e++) acc += h[e] * psi_u[inverse[e]];
        y[i] = acc;
        const double p = psi_u[inverse[offsets[i]]];
        nm_add(&num, p * acc);
        nm_add(&den, p * p);
    }
    *norm2 = nm_value(&den);
    *E = nm_value(&num) / *norm2;
    for (int64_t u = 0; u < n_unique; u++) grad_u[u] = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double p = psi_u[inverse[offsets[i]]];
        for (int64_t e = offsets[i]; e < offsets[i + 1]; e++) grad_u[inverse[e]] += p * h[e];
        grad_u[inverse[offsets[i]]] += y[i] - 2.0 * (*E) * p;
    }
    for (int64_t u = 0; u < n_unique; u++) grad_u[u] = g * (grad_u[u] / *norm2);
}
