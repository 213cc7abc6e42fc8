/*
 * FP64 CPU oracle for the local contractions of Deinsum (arXiv 2206.08301).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA library: it has its own (trivial) argument conventions and no
 * tiling, splitting, blocking or reordering beyond the definitions it cites.
 *
 * Conventions (paper Sec. III-A: 0-based indices, dense tensors; row-major
 * layout as in the NumPy listings of Sec. II-A):
 *   - X is an order-N tensor with extents dims[0..N-1], last index fastest.
 *   - Factor U^m is dims[m] x R (MTTKRP) or dims[m] x ranks[m] (TTMc),
 *     row-major, contracted on its first index (the einsum "i_m r", Sec. III-B).
 *   - All arithmetic is IEEE binary64; inputs given in binary32 are widened
 *     exactly by the caller.
 *   - Outputs are overwritten (Listing 1 accumulates into a zeroed output).
 *
 * Every function cites the passage it follows.  Compile with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_ORDER 8

/* ---------------------------------------------------------------------------
 * MTTKRP, definition (Sec. III-B, the mode-n MTTKRP einsum
 *   i_0..i_{N-1}, i_0 r, ..., i_{n-1} r, i_{n+1} r, ..., i_{N-1} r -> i_n r):
 *
 *   M[i_n, r] = sum over all i_m (m != n) of  X[i_0..i_{N-1}] * prod_{m != n} U^m[i_m, r]
 *
 * Written out directly: for every output row i_n, an odometer walks all the
 * other indices; for every r the product over the factors is formed and the
 * term added.  OpenMP splits the output rows only.
 * ------------------------------------------------------------------------- */
int oracle_mttkrp(int order, const int64_t *dims, int mode, int64_t R,
                  const double *X, const double *const *U, double *M)
{
    if (order < 2 || order > ORACLE_MAX_ORDER || mode < 0 || mode >= order || R < 1)
        return 1;
    int64_t strides[ORACLE_MAX_ORDER];
    int64_t total = 1;
    for (int m = order - 1; m >= 0; --m) { strides[m] = total; total *= dims[m]; }
    const int64_t In = dims[mode];

    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t in = 0; in < In; ++in) {
        int64_t idx[ORACLE_MAX_ORDER];
        for (int m = 0; m < order; ++m) idx[m] = 0;
        idx[mode] = in;
        double *out = M + in * R;
        for (int64_t r = 0; r < R; ++r) out[r] = 0.0;
        int64_t rest = total / In;
        for (int64_t t = 0; t < rest; ++t) {
            int64_t off = 0;
            for (int m = 0; m < order; ++m) off += idx[m] * strides[m];
            const double x = X[off];
            for (int64_t r = 0; r < R; ++r) {
                double term = x;
                for (int m = 0; m < order; ++m)
                    if (m != mode) term = term * U[m][idx[m] * R + r];
                out[r] = out[r] + term;
            }
            /* odometer over every mode except `mode`, last mode fastest */
            for (int m = order - 1; m >= 0; --m) {
                if (m == mode) continue;
                if (++idx[m] < dims[m]) break;
                idx[m] = 0;
            }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * MTTKRP on sampled output rows.  Same definition as oracle_mttkrp, but the
 * caller passes, for each requested row i_n = rows[s], the slab
 * X[i_0..i_{n-1}, rows[s], i_{n+1}..i_{N-1}] as a contiguous row-major block
 * of prod_{m != n} dims[m] values (slabs[s * rest + ...]).  Output:
 * Mrows[s * R + r] = M[rows[s], r].
 * ------------------------------------------------------------------------- */
int oracle_mttkrp_rows(int order, const int64_t *dims, int mode, int64_t R,
                       int64_t n_rows, const double *slabs,
                       const double *const *U, double *Mrows)
{
    if (order < 2 || order > ORACLE_MAX_ORDER || mode < 0 || mode >= order || R < 1)
        return 1;
    int64_t rest = 1;
    for (int m = 0; m < order; ++m) if (m != mode) rest *= dims[m];

    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < n_rows; ++s) {
        int64_t idx[ORACLE_MAX_ORDER];
        for (int m = 0; m < order; ++m) idx[m] = 0;
        const double *slab = slabs + s * rest;
        double *out = Mrows + s * R;
        for (int64_t r = 0; r < R; ++r) out[r] = 0.0;
        for (int64_t t = 0; t < rest; ++t) {
            const double x = slab[t];
            for (int64_t r = 0; r < R; ++r) {
                double term = x;
                for (int m = 0; m < order; ++m)
                    if (m != mode) term = term * U[m][idx[m] * R + r];
                out[r] = out[r] + term;
            }
            for (int m = order - 1; m >= 0; --m) {
                if (m == mode) continue;
                if (++idx[m] < dims[m]) break;
                idx[m] = 0;
            }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * MTTKRP in the factored form of Sec. II-A (the FLOP-reducing decomposition
 * of the running example): first the Khatri-Rao product of all factors except
 * U^n is materialised,
 *     K[(i_m, m != n), r] = prod_{m != n} U^m[i_m, r]          (KRP, Sec. III-B)
 * then the tensor dot product over all modes except n,
 *     M[i_n, r] = sum_{(i_m, m != n)} X[...] * K[(...), r]      (TDOT).
 * K is stored with the non-n modes in their original order, last fastest.
 * Memory grows as prod_{m != n} dims[m] * R: small inputs only.
 * ------------------------------------------------------------------------- */
int oracle_mttkrp_krp(int order, const int64_t *dims, int mode, int64_t R,
                      const double *X, const double *const *U, double *M)
{
    if (order < 2 || order > ORACLE_MAX_ORDER || mode < 0 || mode >= order || R < 1)
        return 1;
    int64_t rest = 1, total = 1;
    for (int m = 0; m < order; ++m) { total *= dims[m]; if (m != mode) rest *= dims[m]; }
    double *K = (double *)malloc(sizeof(double) * (size_t)(rest * R));
    if (!K) return 2;
    /* KRP */
    {
        int64_t idx[ORACLE_MAX_ORDER] = {0};
        for (int64_t t = 0; t < rest; ++t) {
            for (int64_t r = 0; r < R; ++r) {
                double v = 1.0;
                for (int m = 0; m < order; ++m)
                    if (m != mode) v = v * U[m][idx[m] * R + r];
                K[t * R + r] = v;
            }
            for (int m = order - 1; m >= 0; --m) {
                if (m == mode) continue;
                if (++idx[m] < dims[m]) break;
                idx[m] = 0;
            }
        }
    }
    /* TDOT: walk X once in memory order, split its flat index into (i_n, t) */
    const int64_t In = dims[mode];
    int64_t inner = 1;  /* prod of dims after `mode` */
    for (int m = mode + 1; m < order; ++m) inner *= dims[m];
    for (int64_t i = 0; i < In * R; ++i) M[i] = 0.0;
    for (int64_t f = 0; f < total; ++f) {
        const int64_t q = f % inner;
        const int64_t in = (f / inner) % In;
        const int64_t p = f / (inner * In);
        const int64_t t = p * inner + q;
        for (int64_t r = 0; r < R; ++r)
            M[in * R + r] = M[in * R + r] + X[f] * K[t * R + r];
    }
    free(K);
    return 0;
}

/* ---------------------------------------------------------------------------
 * TTM, the mode-m tensor product (Sec. III-B, einsum
 *   i_0..i_{N-1}, i_m r -> i_0..i_{m-1} r i_{m+1}..i_{N-1}):
 *   Y[.., r, ..] = sum_{i_m} X[.., i_m, ..] * U[i_m, r]
 * X is viewed as (A, dims[m], B) with A = prod of earlier extents and
 * B = prod of later ones; Y is (A, Rm, B).
 * ------------------------------------------------------------------------- */
static void ttm_mode(int64_t A, int64_t Im, int64_t B, int64_t Rm,
                     const double *X, const double *U, double *Y)
{
    #pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < A; ++a) {
        for (int64_t r = 0; r < Rm; ++r) {
            double *y = Y + (a * Rm + r) * B;
            for (int64_t b = 0; b < B; ++b) y[b] = 0.0;
            for (int64_t i = 0; i < Im; ++i) {
                const double u = U[i * Rm + r];
                const double *x = X + (a * Im + i) * B;
                for (int64_t b = 0; b < B; ++b) y[b] = y[b] + x[b] * u;
            }
        }
    }
}

/* ---------------------------------------------------------------------------
 * TTMc, keep-mode n (Sec. III-B): the chain
 *   Y = X x_0 U^0 ... x_{n-1} U^{n-1} x_{n+1} U^{n+1} ... x_{N-1} U^{N-1}
 * computed one TTM at a time, from the last mode down to the first (every
 * order gives the same value up to rounding: the modes are independent).
 * ranks[m] is the column count of U^m (ranks[n] is ignored).  The output has
 * extents ranks[m] in every mode except n, which keeps dims[n].
 * ------------------------------------------------------------------------- */
int oracle_ttmc(int order, const int64_t *dims, int keep, const int64_t *ranks,
                const double *X, const double *const *U, double *Y)
{
    if (order < 2 || order > ORACLE_MAX_ORDER || keep < 0 || keep >= order) return 1;
    int64_t cur[ORACLE_MAX_ORDER];
    int64_t size = 1;
    for (int m = 0; m < order; ++m) { cur[m] = dims[m]; size *= dims[m]; }
    double *buf = (double *)malloc(sizeof(double) * (size_t)size);
    if (!buf) return 2;
    memcpy(buf, X, sizeof(double) * (size_t)size);
    for (int m = order - 1; m >= 0; --m) {
        if (m == keep) continue;
        int64_t A = 1, B = 1;
        for (int k = 0; k < m; ++k) A *= cur[k];
        for (int k = m + 1; k < order; ++k) B *= cur[k];
        const int64_t nsize = A * ranks[m] * B;
        double *nb = (double *)malloc(sizeof(double) * (size_t)nsize);
        if (!nb) { free(buf); return 2; }
        ttm_mode(A, cur[m], B, ranks[m], buf, U[m], nb);
        free(buf);
        buf = nb;
        cur[m] = ranks[m];
        size = nsize;
    }
    memcpy(Y, buf, sizeof(double) * (size_t)size);
    free(buf);
    return 0;
}

/* ---------------------------------------------------------------------------
 * TTMc on sampled keep-mode slices.  For each requested i_n = rows[s] the
 * caller passes the slab X[.., rows[s], ..] (contiguous, other modes in order);
 * the chain of TTMs over the other modes of that slab gives
 * Yrows[s] = Y[.., rows[s], ..] with the rank extents in mode order.
 * ------------------------------------------------------------------------- */
int oracle_ttmc_rows(int order, const int64_t *dims, int keep, const int64_t *ranks,
                     int64_t n_rows, const double *slabs, const double *const *U,
                     double *Yrows)
{
    if (order < 2 || order > ORACLE_MAX_ORDER || keep < 0 || keep >= order) return 1;
    int64_t sdims[ORACLE_MAX_ORDER], sranks[ORACLE_MAX_ORDER];
    const double *sU[ORACLE_MAX_ORDER];
    int so = 0;
    int64_t rest = 1, orest = 1;
    for (int m = 0; m < order; ++m) {
        if (m == keep) continue;
        sdims[so] = dims[m]; sranks[so] = ranks[m]; sU[so] = U[m];
        rest *= dims[m]; orest *= ranks[m];
        ++so;
    }
    /* a slab with the keep mode removed is an order-(N-1) tensor; chaining a TTM
       over each of its modes is the TTMc of the full tensor restricted to i_n.
       A dummy leading mode of extent 1 is kept so that order >= 2. */
    int64_t d2[ORACLE_MAX_ORDER + 1], r2[ORACLE_MAX_ORDER + 1];
    const double *u2[ORACLE_MAX_ORDER + 1];
    d2[0] = 1; r2[0] = 1; u2[0] = NULL;
    for (int k = 0; k < so; ++k) { d2[k + 1] = sdims[k]; r2[k + 1] = sranks[k]; u2[k + 1] = sU[k]; }
    for (int64_t s = 0; s < n_rows; ++s) {
        int rc = oracle_ttmc(so + 1, d2, 0, r2, slabs + s * rest, u2, Yrows + s * orest);
        if (rc) return rc;
    }
    return 0;
}

/* Frobenius norms used by the tests: returns sqrt(sum a^2) in long double
 * accumulation to keep the reference error far below any tolerance. */
double oracle_frobenius(const double *a, int64_t n)
{
    long double s = 0.0L;
    for (int64_t i = 0; i < n; ++i) s += (long double)a[i] * (long double)a[i];
    return (double)__builtin_sqrtl(s);
}

/* Threads of the OpenMP loops above (for timing the oracle on a given number of
 * host cores); returns the number now in force (1 without OpenMP). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
