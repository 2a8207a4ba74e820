/*
 * A fast CPU program for FSI -- TIMED CPU BASELINE, TEST INFRASTRUCTURE.
 *
 * Not the oracle: the oracle (fsi_oracle.c) evaluates the closed form with
 * explicit superset sums, which is slow by design.  This file computes the
 * same scores the way a careful CPU implementation would, so that the GPU's
 * speed can be set against a fair CPU figure as well as against the oracle:
 *
 *   1. a = Moebius(v) in place, one butterfly level per player
 *      (a[S u i] -= a[S], Section 3.2's per-player Kronecker factors),
 *      the low 14 levels inside cache-sized blocks;
 *   2. for each s = 1..l: x_s(T) = w(s, |T|) a(T) for |T| > l, else 0
 *      (Eq. weight), then the superset sums x_s(S) = sum_{T >= S} x_s(T),
 *      one level per player, blocked the same way, skipping the sets whose
 *      processed part already has more than s players (they are never read);
 *   3. phi(S) = a(S) + x_{|S|}(S) for the scored S (Eq. fsi_closed with
 *      Eq. correction).
 *
 * float64 throughout, OpenMP over games.  Only bench.py's CPU-baseline leg
 * and the tests (which check it against the oracle) use it.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int pc64(uint64_t x) { return __builtin_popcountll(x); }

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* w(s,t) of Eq. weight (0 for t <= l) */
static double wgt(int ell, int s, int t)
{
    if (s < 1 || s > ell || t <= ell) return 0.0;
    double r = (double)s / (double)(ell + s) * binom(ell, s) * binom(t - 1, ell) / binom(t + ell - 1, ell + s);
    return ((ell - s) & 1) ? -r : r;
}

#define BLOCK_BITS 14

static void mobius_inplace(double *a, int d)
{
    const uint64_t n = (uint64_t)1 << d;
    const int kb = d < BLOCK_BITS ? d : BLOCK_BITS;
    const uint64_t nb = (uint64_t)1 << kb;
    for (uint64_t base = 0; base < n; base += nb)
        for (int i = 0; i < kb; ++i) {
            const uint64_t h = (uint64_t)1 << i;
            for (uint64_t j = base; j < base + nb; j += 2 * h)
                for (uint64_t k = 0; k < h; ++k) a[j + h + k] -= a[j + k];
        }
    for (int i = kb; i < d; ++i) {
        const uint64_t h = (uint64_t)1 << i;
        for (uint64_t j = 0; j < n; j += 2 * h)
            for (uint64_t k = 0; k < h; ++k) a[j + h + k] -= a[j + k];
    }
}

/* superset sums over every player, keeping only what |S| <= s can read:
 * after level i an entry S with more than s players among bits 0..i is
 * never used again, so it is not updated */
static void zeta_up_pruned(double *x, int d, int s)
{
    const uint64_t n = (uint64_t)1 << d;
    const int kb = d < BLOCK_BITS ? d : BLOCK_BITS;
    const uint64_t nb = (uint64_t)1 << kb;
    for (uint64_t base = 0; base < n; base += nb)
        for (int i = 0; i < kb; ++i) {
            const uint64_t h = (uint64_t)1 << i, low = (h << 1) - 1;
            for (uint64_t j = base; j < base + nb; j += 2 * h)
                for (uint64_t k = 0; k < h; ++k)
                    if (pc64((j + k) & low) <= s) x[j + k] += x[j + h + k];
        }
    for (int i = kb; i < d; ++i) {
        const uint64_t h = (uint64_t)1 << i, low = (h << 1) - 1;
        for (uint64_t j = 0; j < n; j += 2 * h)
            for (uint64_t k = 0; k < h; ++k)
                if (pc64((j + k) & low) <= s) x[j + k] += x[j + h + k];
    }
}

/* phi [B, n_masks] of games v [B, 2^d]; masks in the score order.
 * Returns 0, or -1 on a bad argument or allocation failure. */
int cpu_fast_fsi(int d, int ell, int64_t B, const double *v, int64_t n_masks, const uint64_t *masks, double *phi)
{
    if (d < 1 || d > 30 || ell < 1 || B < 0) return -1;
    const uint64_t n = (uint64_t)1 << d;
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int64_t b = 0; b < B; ++b) {
        double *a = (double *)malloc(n * sizeof(double));
        double *x = (double *)malloc(n * sizeof(double));
        if (!a || !x) {
            free(a);
            free(x);
            fail |= 1;
            continue;
        }
        memcpy(a, v + (size_t)b * n, n * sizeof(double));
        mobius_inplace(a, d);
        double *out = phi + (size_t)b * n_masks;
        for (int64_t k = 0; k < n_masks; ++k) out[k] = a[masks[k]];
        const int smax = ell < d ? ell : d;
        if (ell < d) {
            double wt[64];
            for (int s = 1; s <= smax; ++s) {
                for (int t = 0; t <= d; ++t) wt[t] = wgt(ell, s, t);
                for (uint64_t T = 0; T < n; ++T) x[T] = wt[pc64(T)] * a[T];
                zeta_up_pruned(x, d, s);
                for (int64_t k = 0; k < n_masks; ++k)
                    if (pc64(masks[k]) == s) out[k] += x[masks[k]];
            }
        }
        free(a);
        free(x);
    }
    return fail ? -1 : 0;
}
