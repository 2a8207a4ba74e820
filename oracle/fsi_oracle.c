/*
 * CPU oracle for Faithful Shapley Interactions (FSI) -- TEST INFRASTRUCTURE.
 *
 * This file is the plain, slow reference that the CUDA path is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the library never links or calls it.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Conventions: a game on d players is a float64 vector of length 2^d indexed
 * by coalition bitmask (bit i = player i).  Scores are returned for every S
 * with |S| <= min(l, d), graded by |S| and lexicographic over the sorted
 * player tuple within a grade (empty set first).
 *
 * Every routine states the passage of the paper (Kim & Lee, "TT-FSI:
 * Scalable Faithful Shapley Interactions via Tensor-Train") it writes out.
 * Arithmetic is IEEE float64 in a fixed order; build with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* Binomial coefficient C(n, k) as an exact integer (0 when k < 0 or k > n). */
static u128 binom_exact(int n, int k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    u128 r = 1;
    for (int i = 1; i <= k; ++i) {
        r = r * (u128)(n - k + i) / (u128)i; /* exact at every step */
    }
    return r;
}

static int popcount64(uint64_t x)
{
    int c = 0;
    while (x) { x &= x - 1; ++c; }
    return c;
}

/*
 * Correction weight w(s, t) of Eq. (weight) (Section 3.3, restated in the
 * proof of Lemma "weight function correctness"):
 *   w(s,t) = (-1)^(l-s) * s/(l+s) * C(l,s) * C(t-1,l) / C(t+l-1, l+s).
 * Numerator and denominator are formed as exact integers; the quotient is
 * rounded to float64 once the two have been converted.
 */
double oracle_weight(int ell, int s, int t)
{
    if (s < 0 || t < 1 || ell < 1) return 0.0;
    u128 num = (u128)s * binom_exact(ell, s) * binom_exact(t - 1, ell);
    u128 den = (u128)(ell + s) * binom_exact(t + ell - 1, ell + s);
    if (num == 0 || den == 0) return 0.0;
    double w = (double)num / (double)den;
    return ((ell - s) % 2 == 0) ? w : -w;
}

/* Number of scores: sum_{k <= min(l, d)} C(d, k). */
int64_t oracle_num_scores(int d, int ell)
{
    int64_t n = 0;
    int top = ell < d ? ell : d;
    for (int k = 0; k <= top; ++k) n += (int64_t)binom_exact(d, k);
    return n;
}

/*
 * Output order: grade k = 0..min(l,d); within a grade the sorted index tuples
 * (i_1 < ... < i_k) in lexicographic order.  Writes the coalition masks.
 */
int64_t oracle_score_masks(int d, int ell, uint64_t *masks)
{
    int64_t n = 0;
    int top = ell < d ? ell : d;
    int idx[64];
    for (int k = 0; k <= top; ++k) {
        for (int i = 0; i < k; ++i) idx[i] = i;
        for (;;) {
            uint64_t m = 0;
            for (int i = 0; i < k; ++i) m |= (uint64_t)1 << idx[i];
            masks[n++] = m;
            /* next combination in lexicographic order */
            int p = k - 1;
            while (p >= 0 && idx[p] == d - k + p) --p;
            if (p < 0) break;
            ++idx[p];
            for (int i = p + 1; i < k; ++i) idx[i] = idx[i - 1] + 1;
        }
    }
    return n;
}

/*
 * Moebius transform of Eq. (fsi_closed):
 *   a(S) = sum_{T subset of S} (-1)^(|S|-|T|) v(T),
 * written out by enumerating every submask T of S in ascending order
 * (3^d terms in all).
 */
void oracle_mobius_submask(int d, const double *v, double *a)
{
    uint64_t n = (uint64_t)1 << d;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t S = 0; S < (int64_t)n; ++S) {
        int s = popcount64((uint64_t)S);
        double acc = 0.0;
        uint64_t T = 0;
        for (;;) {
            int t = popcount64(T);
            double term = v[T];
            acc += ((s - t) % 2 == 0) ? term : -term;
            if (T == (uint64_t)S) break;
            T = (T - (uint64_t)S) & (uint64_t)S; /* next submask, ascending */
        }
        a[S] = acc;
    }
}

/*
 * The same transform through its Kronecker form (Section 3.2, and Appendix B:
 * the Moebius operator is the d-fold Kronecker product of [[1,0],[-1,1]]):
 * one factor per player, applied as x[S u {i}] -= x[S] for every S without i.
 * This is Yates' method for a Kronecker product; it is used where 3^d terms
 * are too many and is checked against the submask form in the tests.
 */
void oracle_mobius_yates(int d, const double *v, double *a)
{
    uint64_t n = (uint64_t)1 << d;
    if (a != v) memcpy(a, v, n * sizeof(double));
    for (int i = 0; i < d; ++i) {
        uint64_t bit = (uint64_t)1 << i;
        for (uint64_t S = 0; S < n; ++S) {
            if (S & bit) a[S] -= a[S ^ bit];
        }
    }
}

/*
 * FSI scores from the Moebius coefficients, Eq. (fsi_closed) with the
 * correction of Eq. (correction):
 *   phi(S) = a(S) + sum_{T strict superset of S, |T| > l} w(|S|, |T|) a(T)
 * for each requested S (|S| <= l; the correction vanishes for S empty since
 * w(0, t) = 0).  Supersets T = S u U are enumerated over the submasks U of the
 * complement in ascending order.
 */
void oracle_fsi_from_mobius(int d, int ell, const double *a, int64_t n_masks,
                            const uint64_t *masks, double *phi)
{
    uint64_t full = (d == 64) ? ~(uint64_t)0 : (((uint64_t)1 << d) - 1);
    double wtab[65][65];
    for (int s = 0; s <= 64; ++s)
        for (int t = 0; t <= 64; ++t)
            wtab[s][t] = (s <= d && t <= d) ? oracle_weight(ell, s, t) : 0.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_masks; ++k) {
        uint64_t S = masks[k];
        int s = popcount64(S);
        double corr = 0.0;
        if (s >= 1 && s <= ell) {
            uint64_t comp = full & ~S;
            uint64_t U = 0;
            for (;;) {
                U = (U - comp) & comp; /* next non-empty submask, ascending */
                if (U == 0) break;
                uint64_t T = S | U;
                int t = popcount64(T);
                if (t > ell) corr += wtab[s][t] * a[T];
            }
        }
        phi[k] = a[S] + corr;
    }
}

/*
 * For each listed coalition S (|S| <= l): the sums of v(R) over the bins
 * (r, q) = (|R|, |R n S|), bins[k][r * (l + 1) + q], each accumulated with
 * Neumaier's compensated summation (Neumaier 1974) so that the bin sums are
 * accurate to a few units in the last place whatever d.  With these, a score
 * is a short weighted sum (the direct route of the oracle, no Moebius
 * transform).  OpenMP over the listed coalitions.
 */
void oracle_bin_sums(int d, int ell, const double *v, int64_t n_masks, const uint64_t *masks, double *bins)
{
    const uint64_t n = (uint64_t)1 << d;
    const int nb = (d + 1) * (ell + 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n_masks; ++k) {
        const uint64_t S = masks[k];
        double *sum = (double *)calloc((size_t)nb * 2, sizeof(double));
        if (!sum) continue;
        double *cmp = sum + nb;
        for (uint64_t R = 0; R < n; ++R) {
            const int b = popcount64(R) * (ell + 1) + popcount64(R & S);
            const double x = v[R], t = sum[b] + x;
            if (fabs(sum[b]) >= fabs(x))
                cmp[b] += (sum[b] - t) + x;
            else
                cmp[b] += (x - t) + sum[b];
            sum[b] = t;
        }
        for (int b = 0; b < nb; ++b) bins[k * nb + b] = sum[b] + cmp[b];
        free(sum);
    }
}

/*
 * FSI of B games of d players (v is [B, 2^d] row-major, phi is
 * [B, n_scores]): Moebius by the per-player factors, then the explicit
 * superset sums above.  Returns 0, or -1 on bad arguments / no memory.
 */
int oracle_fsi(int d, int ell, int64_t B, const double *v, double *phi)
{
    if (d < 1 || d > 30 || ell < 1 || B < 0) return -1;
    uint64_t n = (uint64_t)1 << d;
    int64_t n_out = oracle_num_scores(d, ell);
    uint64_t *masks = (uint64_t *)malloc((size_t)n_out * sizeof(uint64_t));
    double *a = (double *)malloc((size_t)n * sizeof(double));
    if (!masks || !a) { free(masks); free(a); return -1; }
    oracle_score_masks(d, ell, masks);
    for (int64_t b = 0; b < B; ++b) {
        oracle_mobius_yates(d, v + (size_t)b * n, a);
        oracle_fsi_from_mobius(d, ell, a, n_out, masks, phi + (size_t)b * n_out);
    }
    free(masks);
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Other interaction indices (Appendix A), by their definitions               */
/* ------------------------------------------------------------------------ */

/*
 * Discrete derivative of Appendix A: Delta_S v(T) = sum over R subset of S of
 * (-1)^(|S|-|R|) v(T u R), for T disjoint from S.
 */
static double discrete_derivative(const double *v, uint64_t S, int s, uint64_t T)
{
    double acc = 0.0;
    uint64_t R = S;
    for (;;) {
        double x = v[T | R];
        acc += ((s - popcount64(R)) % 2 == 0) ? x : -x;
        if (R == 0) break;
        R = (R - 1) & S;
    }
    return acc;
}

/*
 * Scores of B games by the definitions over discrete derivatives, summing
 * over every T in the complement of S (ascending submasks, T = {} first):
 *   index 1, SII (Appendix A, Shapley interaction index):
 *     sum_T |T|! (d-|S|-|T|)! / (d-|S|+1)! Delta_S v(T)
 *       = sum_T Delta_S v(T) / ((d-|S|+1) C(d-|S|, |T|));
 *   index 2, BII (Appendix A, Banzhaf: the uniform weight over the 2^(d-|S|)
 *     sets T): sum_T 2^-(d-|S|) Delta_S v(T);
 *   index 3, STII of order l (Appendix A; Sundararajan et al.'s definition):
 *     Delta_S v({}) for |S| < l, and (l/d) sum_T Delta_S v(T) / C(d-1, |T|)
 *     for |S| = l.
 * Work O(n_scores 2^d); meant for d <= 16.  Returns 0, or -1 on bad input.
 */
int oracle_index_definition(int d, int ell, int index, int64_t B, const double *v, double *phi)
{
    if (d < 1 || d > 24 || ell < 1 || B < 0 || index < 1 || index > 3) return -1;
    uint64_t n = (uint64_t)1 << d;
    uint64_t full = n - 1;
    int64_t n_out = oracle_num_scores(d, ell);
    uint64_t *masks = (uint64_t *)malloc((size_t)n_out * sizeof(uint64_t));
    if (!masks) return -1;
    oracle_score_masks(d, ell, masks);
    for (int64_t b = 0; b < B; ++b) {
        const double *vb = v + (size_t)b * n;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t k = 0; k < n_out; ++k) {
            uint64_t S = masks[k];
            int s = popcount64(S);
            double out = 0.0;
            if (index == 3 && s < ell) {
                out = discrete_derivative(vb, S, s, 0);
            } else {
                uint64_t comp = full & ~S;
                uint64_t T = 0;
                for (;;) {
                    int t = popcount64(T);
                    double w;
                    if (index == 1)
                        w = 1.0 / ((double)(d - s + 1) * (double)binom_exact(d - s, t));
                    else if (index == 2)
                        w = ldexp(1.0, -(d - s));
                    else
                        w = ((double)ell / (double)d) / (double)binom_exact(d - 1, t);
                    out += w * discrete_derivative(vb, S, s, T);
                    T = (T - comp) & comp; /* next submask of the complement, ascending */
                    if (T == 0) break;
                }
            }
            phi[(size_t)b * n_out + k] = out;
        }
    }
    free(masks);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Masked-model value function                                              */
/* ------------------------------------------------------------------------ */

/* GELU in its exact form, 0.5 z (1 + erf(z / sqrt 2)). */
static double gelu(double z) { return 0.5 * z * (1.0 + erf(z * 0.70710678118654752440)); }

/*
 * Value function of Section 2.1 ("v(S) is the model's prediction when only
 * the features in S are present"), with absent features set to a baseline:
 *   v_x(S) = f(z),  z_i = x_i if i in S else baseline_i,
 *   f(z) = W3 gelu(W2 gelu(W1 z + b1) + b2) + b3.
 * Weights are row-major: W1 [h1, d], W2 [h2, h1], W3 [h2].  Evaluates the
 * coalitions listed in `coal` (n_coal of them) straight from the definition,
 * one full forward pass each.
 */
void oracle_masked_game(int d, int h1, int h2, const double *W1, const double *b1,
                        const double *W2, const double *b2, const double *W3, double b3,
                        const double *x, const double *baseline, int64_t n_coal,
                        const uint64_t *coal, double *out)
{
#pragma omp parallel
    {
        double *z = (double *)malloc((size_t)d * sizeof(double));
        double *y1 = (double *)malloc((size_t)h1 * sizeof(double));
        double *y2 = (double *)malloc((size_t)h2 * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t k = 0; k < n_coal; ++k) {
            uint64_t S = coal[k];
            for (int i = 0; i < d; ++i) z[i] = ((S >> i) & 1) ? x[i] : baseline[i];
            for (int j = 0; j < h1; ++j) {
                double acc = b1[j];
                for (int i = 0; i < d; ++i) acc += W1[(size_t)j * d + i] * z[i];
                y1[j] = gelu(acc);
            }
            for (int j = 0; j < h2; ++j) {
                double acc = b2[j];
                for (int i = 0; i < h1; ++i) acc += W2[(size_t)j * h1 + i] * y1[i];
                y2[j] = gelu(acc);
            }
            double acc = b3;
            for (int i = 0; i < h2; ++i) acc += W3[i] * y2[i];
            out[k] = acc;
        }
        free(z);
        free(y1);
        free(y2);
    }
}

/* Number of threads an OpenMP region of this library uses. */
int oracle_num_threads(void)
{
    int n = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
#endif
    return n;
}
