/*
 * Timed CPU baseline (tier b) of the generalized RBT + GENP solver
 * (arXiv 2312.09376): the same method as the plain oracle in rbt_oracle.c --
 * the same butterfly coefficients (orc_generate), the same transform order
 * (Eq. rbt-depth-d, innermost layer first), Gaussian elimination with no
 * pivoting, the same substitutions and the same stationary refinement on the
 * original A (Sec. 5) -- written to use every host core: OpenMP threads, a
 * right-looking blocked GENP whose trailing update is a packed, register-
 * blocked matrix product, and parallel transform, residual and substitution
 * loops.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the oracle: only the tests and
 * the benchmark's CPU-baseline leg load it.  It shares no code with the CUDA
 * path.  Plain C with OpenMP; no intrinsics, so it builds on x86-64 and on
 * Arm alike.  Results differ from the oracle's by rounding order only (the
 * blocked product sums in another order, and the compiler may contract
 * multiply-adds); the tests bound that difference.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "rbt_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#else
/* built without OpenMP: one thread, wall time from the C library */
#include <time.h>
static int omp_get_max_threads(void) { return 1; }
static double omp_get_wtime(void)
{
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}
#endif

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

static const double INV_SQRT2 = 0.70710678118654752440084436210485;

int cpu_threads(void) { return omp_get_max_threads(); }

/* Threads for the following calls (n <= 0: leave as is); returns the count in effect. */
int cpu_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
    return omp_get_max_threads();
}

/* ------------------------------------------------------------ transforms */

/* X <- B_k X on n x ncols (column-parallel), the pairing of orc_layer_rows. */
static void layer_rows(int64_t n, int d, int k, double *X, int64_t ldx, int64_t ncols)
{
    if (k > orc_depth_eff(n, d))
        return;
    const int64_t h = orc_ref_size(n, d) >> k;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < ncols; c++) {
        double *x = X + (size_t)c * (size_t)ldx;
        for (int64_t start = 0; start < n; start += 2 * h) {
            const int64_t end = start + h < n ? start + h : n;
            for (int64_t i = start; i < end; i++) {
                const int64_t p = i + h;
                if (p >= n)
                    break;
                const double a = x[i], b = x[p];
                x[i] = (a + b) * INV_SQRT2;
                x[p] = (a - b) * INV_SQRT2;
            }
        }
    }
}

/* X <- X B_k (pairs of columns, parallel over the pairs). */
static void layer_cols(int64_t n, int d, int k, double *X, int64_t ldx, int64_t nrows)
{
    if (k > orc_depth_eff(n, d))
        return;
    const int64_t h = orc_ref_size(n, d) >> k;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        if ((j / h) % 2 != 0)
            continue; /* bottom half of a butterfly: handled by its top row */
        const int64_t p = j + h;
        if (p >= n)
            continue;
        double *a = X + (size_t)j * (size_t)ldx, *b = X + (size_t)p * (size_t)ldx;
        for (int64_t r = 0; r < nrows; r++) {
            const double x = a[r], y = b[r];
            a[r] = (x + y) * INV_SQRT2;
            b[r] = (x - y) * INV_SQRT2;
        }
    }
}

/* A <- U^T A V: for k = d .. 1, B_k on both sides, then R_k and R'_k. */
static void transform_2sided(int64_t n, int d, const double *U, const double *V, double *A, int64_t lda)
{
    for (int k = d; k >= 1; k--) {
        layer_rows(n, d, k, A, lda, n);
        layer_cols(n, d, k, A, lda, n);
        const double *u = U + (size_t)(k - 1) * (size_t)n, *v = V + (size_t)(k - 1) * (size_t)n;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) {
            double *a = A + (size_t)j * (size_t)lda;
            const double vj = v[j];
            for (int64_t i = 0; i < n; i++)
                a[i] = a[i] * u[i] * vj;
        }
    }
}

/* W^T B (trans) or W B on n x nrhs, as orc_transform_vec. */
static void transform_vec(int64_t n, int d, const double *W, int trans, double *B, int64_t ldb, int64_t nrhs)
{
    if (trans) {
        for (int k = d; k >= 1; k--) {
            layer_rows(n, d, k, B, ldb, nrhs);
            const double *w = W + (size_t)(k - 1) * (size_t)n;
            for (int64_t c = 0; c < nrhs; c++)
                for (int64_t i = 0; i < n; i++)
                    B[IDX(i, c, ldb)] *= w[i];
        }
    } else {
        for (int k = 1; k <= d; k++) {
            const double *w = W + (size_t)(k - 1) * (size_t)n;
            for (int64_t c = 0; c < nrhs; c++)
                for (int64_t i = 0; i < n; i++)
                    B[IDX(i, c, ldb)] *= w[i];
            layer_rows(n, d, k, B, ldb, nrhs);
        }
    }
}

/* ------------------------------------------------- packed matrix product */

enum { MR = 8, NR = 4, MC = 128, NC = 256, KC = 256 };

/* C (mr x nr, ldc) -= a-panel (k x MR, row index fastest) * b-panel (k x NR) */
static void micro(int kc, const double *restrict a, const double *restrict b, double *restrict c, int64_t ldc,
                  int mr, int nr)
{
    double acc[NR][MR];
    for (int j = 0; j < NR; j++)
        for (int i = 0; i < MR; i++)
            acc[j][i] = 0.0;
    for (int k = 0; k < kc; k++) {
        const double *ak = a + (size_t)MR * k, *bk = b + (size_t)NR * k;
        for (int j = 0; j < NR; j++) {
            const double bj = bk[j];
            for (int i = 0; i < MR; i++)
                acc[j][i] += ak[i] * bj;
        }
    }
    for (int j = 0; j < nr; j++)
        for (int i = 0; i < mr; i++)
            c[IDX(i, j, ldc)] -= acc[j][i];
}

/* C (M x N) -= A (M x K) B (K x N), column-major.  Tiles of MC x NC are dealt
 * to the threads; each packs its A block into MR-row panels and its B block
 * into NR-column panels (zero padded) and runs the register-blocked kernel. */
static void gemm_sub(int64_t M, int64_t N, int64_t K, const double *A, int64_t lda, const double *B, int64_t ldb,
                     double *C, int64_t ldc)
{
    if (M <= 0 || N <= 0 || K <= 0)
        return;
    const int64_t tm = (M + MC - 1) / MC, tn = (N + NC - 1) / NC;
#pragma omp parallel
    {
        double *pa = (double *)malloc(sizeof(double) * (size_t)MC * KC);
        double *pb = (double *)malloc(sizeof(double) * (size_t)NC * KC);
#pragma omp for schedule(dynamic, 1) collapse(2)
        for (int64_t bj = 0; bj < tn; bj++)
            for (int64_t bi = 0; bi < tm; bi++) {
                const int64_t i0 = bi * MC, j0 = bj * NC;
                const int64_t mc = M - i0 < MC ? M - i0 : MC, nc = N - j0 < NC ? N - j0 : NC;
                for (int64_t k0 = 0; k0 < K; k0 += KC) {
                    const int kc = (int)(K - k0 < KC ? K - k0 : KC);
                    for (int64_t ip = 0; ip < mc; ip += MR)
                        for (int k = 0; k < kc; k++)
                            for (int i = 0; i < MR; i++)
                                pa[(size_t)ip * kc + (size_t)MR * k + i] =
                                    ip + i < mc ? A[IDX(i0 + ip + i, k0 + k, lda)] : 0.0;
                    for (int64_t jp = 0; jp < nc; jp += NR)
                        for (int k = 0; k < kc; k++)
                            for (int j = 0; j < NR; j++)
                                pb[(size_t)jp * kc + (size_t)NR * k + j] =
                                    jp + j < nc ? B[IDX(k0 + k, j0 + jp + j, ldb)] : 0.0;
                    for (int64_t jp = 0; jp < nc; jp += NR)
                        for (int64_t ip = 0; ip < mc; ip += MR)
                            micro(kc, pa + (size_t)ip * kc, pb + (size_t)jp * kc, C + IDX(i0 + ip, j0 + jp, ldc), ldc,
                                  (int)(mc - ip < MR ? mc - ip : MR), (int)(nc - jp < NR ? nc - jp : NR));
                }
            }
        free(pa);
        free(pb);
    }
}

/* ------------------------------------------------------------------ GENP */

/* Right-looking blocked elimination without row exchanges, block size nb:
 * factor the diagonal block, L21 = A21 U11^{-1} (rows in parallel),
 * U12 = L11^{-1} A12 (columns in parallel), A22 -= L21 U12.  Returns -1, or
 * the first pivot that is exactly zero or not finite (as orc_genp). */
int64_t cpu_genp(int64_t n, double *A, int64_t lda, int nb)
{
    if (nb <= 0)
        nb = 128;
    for (int64_t k = 0; k < n; k += nb) {
        const int64_t kb = n - k < nb ? n - k : nb;
        /* diagonal block: textbook kij elimination */
        for (int64_t j = k; j < k + kb; j++) {
            const double p = A[IDX(j, j, lda)];
            if (p == 0.0 || !isfinite(p))
                return j;
            for (int64_t i = j + 1; i < k + kb; i++)
                A[IDX(i, j, lda)] /= p;
            for (int64_t c = j + 1; c < k + kb; c++) {
                const double u = A[IDX(j, c, lda)];
                for (int64_t i = j + 1; i < k + kb; i++)
                    A[IDX(i, c, lda)] -= A[IDX(i, j, lda)] * u;
            }
        }
        const int64_t r0 = k + kb, rest = n - r0;
        if (rest <= 0)
            break;
        /* L21 = A21 U11^{-1}: blocks of 64 rows, column by column */
#pragma omp parallel for schedule(static)
        for (int64_t i0 = r0; i0 < n; i0 += 64) {
            const int64_t i1 = i0 + 64 < n ? i0 + 64 : n;
            for (int64_t j = k; j < k + kb; j++) {
                const double p = A[IDX(j, j, lda)];
                double *l = A + IDX(0, j, lda);
                for (int64_t i = i0; i < i1; i++)
                    l[i] /= p;
                for (int64_t c = j + 1; c < k + kb; c++) {
                    const double u = A[IDX(j, c, lda)];
                    double *a = A + IDX(0, c, lda);
                    for (int64_t i = i0; i < i1; i++)
                        a[i] -= l[i] * u;
                }
            }
        }
        /* U12 = L11^{-1} A12: each column by forward substitution */
#pragma omp parallel for schedule(static)
        for (int64_t c = r0; c < n; c++) {
            double *a = A + IDX(0, c, lda);
            for (int64_t j = k; j < k + kb; j++) {
                const double u = a[j];
                const double *l = A + IDX(0, j, lda);
                for (int64_t i = j + 1; i < k + kb; i++)
                    a[i] -= l[i] * u;
            }
        }
        gemm_sub(rest, rest, kb, A + IDX(r0, k, lda), lda, A + IDX(k, r0, lda), lda, A + IDX(r0, r0, lda), lda);
    }
    return -1;
}

/* (L U)^{-1} B, column by column: forward with unit L, back with U, each
 * triangle in blocks of 256 rows (the block's own substitution, then a
 * parallel update of the rows still to solve). */
static void genp_solve(int64_t n, int64_t nrhs, const double *LU, int64_t lda, double *B, int64_t ldb)
{
    const int64_t bs = 256;
    for (int64_t c = 0; c < nrhs; c++) {
        double *b = B + (size_t)c * (size_t)ldb;
        for (int64_t j0 = 0; j0 < n; j0 += bs) {
            const int64_t j1 = j0 + bs < n ? j0 + bs : n;
            for (int64_t j = j0; j < j1; j++)
                for (int64_t i = j + 1; i < j1; i++)
                    b[i] -= LU[IDX(i, j, lda)] * b[j];
#pragma omp parallel for schedule(static)
            for (int64_t i0 = j1; i0 < n; i0 += 512) {
                const int64_t i1 = i0 + 512 < n ? i0 + 512 : n;
                for (int64_t j = j0; j < j1; j++) {
                    const double x = b[j];
                    const double *l = LU + IDX(0, j, lda);
                    for (int64_t i = i0; i < i1; i++)
                        b[i] -= l[i] * x;
                }
            }
        }
        for (int64_t j1 = n; j1 > 0; j1 -= bs) {
            const int64_t j0 = j1 - bs > 0 ? j1 - bs : 0;
            for (int64_t j = j1 - 1; j >= j0; j--) {
                b[j] /= LU[IDX(j, j, lda)];
                for (int64_t i = j0; i < j; i++)
                    b[i] -= LU[IDX(i, j, lda)] * b[j];
            }
#pragma omp parallel for schedule(static)
            for (int64_t i0 = 0; i0 < j0; i0 += 512) {
                const int64_t i1 = i0 + 512 < j0 ? i0 + 512 : j0;
                for (int64_t j = j0; j < j1; j++) {
                    const double x = b[j];
                    const double *u = LU + IDX(0, j, lda);
                    for (int64_t i = i0; i < i1; i++)
                        b[i] -= u[i] * x;
                }
            }
        }
    }
}

/* ------------------------------------------------------ residual, berr */

/* R = B - A X and Eq. (inf-norm-backerr) with ||A||_inf given. */
static double residual_berr(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X, int64_t ldx,
                            const double *B, int64_t ldb, double *R, double anorm)
{
    double worst = 0.0;
    for (int64_t c = 0; c < nrhs; c++) {
        const double *x = X + (size_t)c * (size_t)ldx, *b = B + (size_t)c * (size_t)ldb;
        double *r = R + (size_t)c * (size_t)n;
        double rmax = 0.0, xmax = 0.0, bmax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : rmax)
        for (int64_t i0 = 0; i0 < n; i0 += 256) {
            const int64_t i1 = i0 + 256 < n ? i0 + 256 : n;
            double acc[256];
            for (int64_t i = i0; i < i1; i++)
                acc[i - i0] = b[i];
            for (int64_t j = 0; j < n; j++) {
                const double xj = x[j];
                const double *a = A + IDX(0, j, lda);
                for (int64_t i = i0; i < i1; i++)
                    acc[i - i0] -= a[i] * xj;
            }
            for (int64_t i = i0; i < i1; i++) {
                r[i] = acc[i - i0];
                const double v = fabs(acc[i - i0]);
                if (v > rmax || isnan(v))
                    rmax = v;
            }
        }
        for (int64_t i = 0; i < n; i++) {
            if (fabs(x[i]) > xmax || isnan(x[i]))
                xmax = fabs(x[i]);
            if (fabs(b[i]) > bmax)
                bmax = fabs(b[i]);
        }
        const double den = anorm * xmax + bmax;
        const double e = den > 0.0 ? rmax / den : (rmax > 0.0 ? INFINITY : 0.0);
        if (e > worst || isnan(e))
            worst = e;
    }
    return worst;
}

static double norm_inf(int64_t n, const double *A, int64_t lda)
{
    double best = 0.0;
#pragma omp parallel for schedule(static) reduction(max : best)
    for (int64_t i0 = 0; i0 < n; i0 += 256) {
        const int64_t i1 = i0 + 256 < n ? i0 + 256 : n;
        double s[256] = {0};
        for (int64_t j = 0; j < n; j++)
            for (int64_t i = i0; i < i1; i++)
                s[i - i0] += fabs(A[IDX(i, j, lda)]);
        for (int64_t i = i0; i < i1; i++)
            if (s[i - i0] > best || isnan(s[i - i0]))
                best = s[i - i0];
    }
    return best;
}

/* ------------------------------------------------------------ full solve */

/* Eq. (precond) with stationary refinement (Sec. 5), as orc_rbt_solve with
 * the non-tiled reference size.  out: [0] first backward error, [1] final
 * backward error, [2] refinement steps, [3] seconds of the factorization
 * (transform + GENP), [4] seconds of the whole call.  Returns -1 or the
 * first bad pivot. */
int64_t cpu_rbt_solve(int64_t n, int64_t nrhs, int d, uint64_t seed, const double *A, int64_t lda, const double *B,
                      int64_t ldb, double *X, int64_t ldx, int refine_max, double tol, int nb, double *out)
{
    const double t0 = omp_get_wtime();
    const size_t nn = (size_t)n * (size_t)n;
    double *U = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(d > 0 ? d : 1));
    double *V = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(d > 0 ? d : 1));
    double *At = (double *)malloc(sizeof(double) * (nn > 0 ? nn : 1));
    double *R = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(nrhs > 0 ? nrhs : 1));
    int64_t status = -1;
    out[0] = out[1] = NAN;
    out[2] = 0.0;
    orc_generate(n, d, seed, U, V, n);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        memcpy(At + (size_t)j * (size_t)n, A + (size_t)j * (size_t)lda, sizeof(double) * (size_t)n);
    transform_2sided(n, d, U, V, At, n);
    status = cpu_genp(n, At, n, nb);
    out[3] = omp_get_wtime() - t0;
    if (status >= 0)
        goto done;
    for (int64_t c = 0; c < nrhs; c++)
        memcpy(X + (size_t)c * (size_t)ldx, B + (size_t)c * (size_t)ldb, sizeof(double) * (size_t)n);
    transform_vec(n, d, U, 1, X, ldx, nrhs);
    genp_solve(n, nrhs, At, n, X, ldx);
    transform_vec(n, d, V, 0, X, ldx, nrhs);
    {
        const double anorm = norm_inf(n, A, lda);
        double berr = residual_berr(n, nrhs, A, lda, X, ldx, B, ldb, R, anorm);
        out[0] = berr;
        int it = 0;
        while (it < refine_max && !(berr <= tol)) {
            transform_vec(n, d, U, 1, R, n, nrhs);
            genp_solve(n, nrhs, At, n, R, n);
            transform_vec(n, d, V, 0, R, n, nrhs);
            for (int64_t c = 0; c < nrhs; c++)
                for (int64_t i = 0; i < n; i++)
                    X[IDX(i, c, ldx)] += R[IDX(i, c, n)];
            berr = residual_berr(n, nrhs, A, lda, X, ldx, B, ldb, R, anorm);
            it++;
        }
        out[1] = berr;
        out[2] = (double)it;
    }
done:
    out[4] = omp_get_wtime() - t0;
    free(U);
    free(V);
    free(At);
    free(R);
    return status;
}
