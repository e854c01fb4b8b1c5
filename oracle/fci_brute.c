/*
 * Brute-force Hamiltonian matrix by term-by-term second quantization.
 * TEST INFRASTRUCTURE ONLY (it pins the Slater-Condon oracle; nothing in the
 * library calls it).  It shares no code with the oracle or the CUDA path.
 *
 * For every basis determinant |D> and every term of
 *   H = Ecore + sum_{pq,sigma} h_pq a+_{p sigma} a_{q sigma}
 *       + 1/2 sum_{pqrs,sigma tau} (pq|rs) a+_{p sigma} a+_{r tau} a_{s tau} a_{q sigma}
 * the operators are applied right to left; a non-vanishing result c|D'> adds
 * c * coefficient to H[D', D].  The phase of a_s / a+_s is (-1)^(occupied spin
 * orbitals below s), spin orbital s = 2p + sigma.  The basis must be sorted
 * ascending as W-word unsigned integers (word W-1 most significant).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FB_MAXW 4

static int fb_bit(const uint64_t *d, int s) { return (int)((d[s >> 6] >> (s & 63)) & 1u); }

/* returns 0 if the operator kills d, else the phase; updates d */
static int fb_op(uint64_t *d, int s, int create) {
    if (fb_bit(d, s) == create) return 0;
    int below = 0;
    for (int t = 0; t < s; t++) below += fb_bit(d, t);
    d[s >> 6] ^= (uint64_t)1 << (s & 63);
    return (below & 1) ? -1 : 1;
}

static int64_t fb_find(const uint64_t *basis, int64_t n, int W, const uint64_t *d) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        const uint64_t *x = basis + (size_t)mid * W;
        int c = 0;
        for (int w = W - 1; w >= 0 && c == 0; w--) c = (x[w] < d[w]) ? -1 : (x[w] > d[w]) ? 1 : 0;
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Column c of H: out[r] = <basis_r| H |D> for the single determinant D.
 * Returns the number of operator strings that left the basis. */
int64_t fci_brute_column(int norb, const double *h1, const double *h2, double ecore,
                         const uint64_t *basis, int64_t n, int W, const uint64_t *D,
                         double *out) {
    int64_t outside = 0;
    uint64_t d[FB_MAXW];
    memset(out, 0, sizeof(double) * (size_t)n);
    int64_t self = fb_find(basis, n, W, D);
    if (self >= 0) out[self] += ecore;
    else outside++;
    /* one-body terms */
    for (int sg = 0; sg < 2; sg++)
        for (int p = 0; p < norb; p++)
            for (int q = 0; q < norb; q++) {
                double coef = h1[p * norb + q];
                if (coef == 0.0) continue;
                memcpy(d, D, sizeof(uint64_t) * W);
                int ph = fb_op(d, 2 * q + sg, 0);
                if (!ph) continue;
                int ph2 = fb_op(d, 2 * p + sg, 1);
                if (!ph2) continue;
                int64_t r = fb_find(basis, n, W, d);
                if (r < 0) { outside++; continue; }
                out[r] += coef * (double)(ph * ph2);
            }
    /* two-body terms */
    for (int sg = 0; sg < 2; sg++)
        for (int ta = 0; ta < 2; ta++)
            for (int p = 0; p < norb; p++)
                for (int q = 0; q < norb; q++)
                    for (int r = 0; r < norb; r++)
                        for (int s = 0; s < norb; s++) {
                            double coef = h2[(((size_t)p * norb + q) * norb + r) * norb + s];
                            if (coef == 0.0) continue;
                            memcpy(d, D, sizeof(uint64_t) * W);
                            int ph = fb_op(d, 2 * q + sg, 0);
                            if (!ph) continue;
                            int t = fb_op(d, 2 * s + ta, 0);
                            if (!t) continue;
                            ph *= t;
                            t = fb_op(d, 2 * r + ta, 1);
                            if (!t) continue;
                            ph *= t;
                            t = fb_op(d, 2 * p + sg, 1);
                            if (!t) continue;
                            ph *= t;
                            int64_t row = fb_find(basis, n, W, d);
                            if (row < 0) { outside++; continue; }
                            out[row] += 0.5 * coef * (double)ph;
                        }
    return outside;
}

/* H is n*n row-major, H[r*n + c] = <basis_r| H |basis_c>; returns the number of
 * operator strings that mapped a basis state outside the basis (0 when the basis
 * is a full particle-number / spin sector). */
int64_t fci_brute_H(int norb, const double *h1, const double *h2, double ecore,
                    const uint64_t *basis, int64_t n, int W, double *H) {
    int64_t outside = 0;
    double *col = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!col) return -1;
    for (int64_t c = 0; c < n; c++) {
        outside += fci_brute_column(norb, h1, h2, ecore, basis, n, W, basis + (size_t)c * W, col);
        for (int64_t r = 0; r < n; r++) H[(size_t)r * n + c] = col[r];
    }
    free(col);
    return outside;
}
