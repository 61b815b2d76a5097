/*
 * Plain FP64 CPU oracle for the generalized RBT + GENP solver
 * (arXiv 2312.09376).  TEST INFRASTRUCTURE ONLY: only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg use it.  It shares no code
 * with the CUDA path.  See rbt_oracle.h for the conventions adopted.
 *
 * Everything here is deliberately the slow literal form: one butterfly layer
 * at a time, one elimination step at a time, naive summation order.
 */
#include "rbt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* 1/sqrt(2), the nonzero magnitude of the butterfly blocks of Eq. (O-matrix-definition) */
static const double INV_SQRT2 = 0.70710678118654752440084436210485;

/* ------------------------------------------------------------------ sizes */

int orc_ceil_log2(int64_t n)
{
    int c = 0;
    int64_t p = 1;
    while (p < n) {
        p *= 2;
        c++;
    }
    return c;
}

/* Layers beyond ceil(log2 n) can hold no butterfly of size >= 2 once the
 * recursion of Lemma 2 has reached blocks of size one; they are diagonal only. */
int orc_depth_eff(int64_t n, int d)
{
    int l = orc_ceil_log2(n);
    return d < l ? d : l;
}

/* Sec. 3 (Algorithm 1's reference size): the smallest multiple of
 * 2^d_s * align that is >= n.  align = 1 is the non-tiled rule; align = n_b,
 * the tile size, is the tiled rule, which puts every butterfly boundary on a
 * tile boundary. */
int64_t orc_ref_size_tiled(int64_t n, int d, int64_t align)
{
    int ds = orc_depth_eff(n, d);
    int64_t p = ((int64_t)1 << ds) * (align > 1 ? align : 1);
    return p * ((n + p - 1) / p);
}

int64_t orc_ref_size(int64_t n, int d) { return orc_ref_size_tiled(n, d, 1); }

/* Least common multiple of two positive integers (Euclid's gcd). */
int64_t orc_lcm(int64_t p, int64_t q)
{
    int64_t a = p, b = q;
    while (b != 0) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return p / a * q;
}

/* Sec. 6 (Performance), Eq. (comm-free-rbt-size): on a p x q process grid
 * holding n_b x n_b tiles block-cyclically, the top half of the first layer
 * (the layer of one butterfly) spans
 *     lcm(p, q) 2^(d-1) ceil(n_t 2^-d / lcm(p, q))  tiles,   n_t = ceil(n / n_b),
 * the number of tile rows of A.  The reference size m is twice that many
 * rows.  d is the effective depth d_s here (layers past it hold no pair);
 * with d_s = 0 there is no butterfly, and the tiled rule with the same
 * alignment is returned. */
int64_t orc_ref_size_comm_free(int64_t n, int d, int64_t nb, int64_t p, int64_t q)
{
    int ds = orc_depth_eff(n, d);
    int64_t l = orc_lcm(p, q);
    if (ds == 0) return orc_ref_size_tiled(n, d, nb * l);
    int64_t nt = (n + nb - 1) / nb;
    int64_t two_d = (int64_t)1 << ds;
    int64_t per = two_d * l;                    /* ceil(n_t 2^-d / lcm) = ceil(n_t / (2^d lcm)) */
    int64_t top_tiles = l * (two_d / 2) * ((nt + per - 1) / per);
    return 2 * top_tiles * nb;
}

/* -------------------------------------------------------------- generator */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the first output of a
 * generator whose state is `key`: advance by the golden gamma, then mix. */
uint64_t orc_splitmix64(uint64_t key)
{
    uint64_t z = key + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Sec. 6: each random diagonal entry is exp(r/20) with r uniform on [-1,1].
 * Counter-based key: seed, side (0 = U, 1 = V), layer k (1-based), row i. */
double orc_coef(uint64_t seed, int side, int layer, int64_t i)
{
    uint64_t key = seed ^ ((uint64_t)side << 62) ^ ((uint64_t)layer << 48) ^ (uint64_t)i;
    uint64_t x = orc_splitmix64(key);
    double u = (double)(x >> 11) * (1.0 / 9007199254740992.0); /* [0,1), 53 bits */
    double r = 2.0 * u - 1.0;                                   /* [-1,1) */
    return exp(r / 20.0);
}

/* Packed storage (Sec. 3, Algorithm 1): column k-1 of U holds diag(R_k). */
void orc_generate(int64_t n, int d, uint64_t seed, double *U, double *V, int64_t ld)
{
    for (int k = 1; k <= d; k++)
        for (int64_t i = 0; i < n; i++) {
            U[IDX(i, k - 1, ld)] = orc_coef(seed, 0, k, i);
            V[IDX(i, k - 1, ld)] = orc_coef(seed, 1, k, i);
        }
}

/* ------------------------------------------------------- butterfly layers */

/* Layer k of Eq. (rbt-depth-d) is block diagonal with 2^(k-1) butterflies
 * O^<l>_{mu,nu} (Eq. O-matrix-definition).  With the alignment rule
 * (Eq. butterfly-alignment) and the semi-Parker choice, butterfly b of layer
 * k covers rows [2 b h, 2 b h + 2 h) clipped to n, where h = m / 2^k.  Its
 * top part is the first h of those rows; top row i pairs with bottom row
 * i + h when that row exists (the mu rows), and otherwise passes through
 * unscaled (the nu rows of the identity block). */
void orc_layer_rows_tiled(int64_t n, int d, int64_t align, int k, double *X, int64_t ldx, int64_t ncols)
{
    if (k > orc_depth_eff(n, d))
        return; /* diagonal-only layer */
    int64_t m = orc_ref_size_tiled(n, d, align);
    int64_t h = m >> k;
    for (int64_t c = 0; c < ncols; c++) {
        for (int64_t start = 0; start < n; start += 2 * h) {
            for (int64_t i = start; i < start + h && i < n; i++) {
                int64_t p = i + h;
                if (p >= n)
                    continue; /* nu row: identity */
                double a = X[IDX(i, c, ldx)];
                double b = X[IDX(p, c, ldx)];
                X[IDX(i, c, ldx)] = (a + b) * INV_SQRT2;
                X[IDX(p, c, ldx)] = (a - b) * INV_SQRT2;
            }
        }
    }
}

/* X <- X B_k.  B_k is symmetric, so its action on the columns of X is the
 * same pairing applied along each row. */
void orc_layer_cols_tiled(int64_t n, int d, int64_t align, int k, double *X, int64_t ldx, int64_t nrows)
{
    if (k > orc_depth_eff(n, d))
        return;
    int64_t m = orc_ref_size_tiled(n, d, align);
    int64_t h = m >> k;
    for (int64_t start = 0; start < n; start += 2 * h) {
        for (int64_t j = start; j < start + h && j < n; j++) {
            int64_t p = j + h;
            if (p >= n)
                continue;
            for (int64_t r = 0; r < nrows; r++) {
                double a = X[IDX(r, j, ldx)];
                double b = X[IDX(r, p, ldx)];
                X[IDX(r, j, ldx)] = (a + b) * INV_SQRT2;
                X[IDX(r, p, ldx)] = (a - b) * INV_SQRT2;
            }
        }
    }
}

void orc_layer_rows(int64_t n, int d, int k, double *X, int64_t ldx, int64_t ncols)
{
    orc_layer_rows_tiled(n, d, 1, k, X, ldx, ncols);
}

void orc_layer_cols(int64_t n, int d, int k, double *X, int64_t ldx, int64_t nrows)
{
    orc_layer_cols_tiled(n, d, 1, k, X, ldx, nrows);
}

/* ---------------------------------------------------------- transforms */

/* A <- U^T A V with U = B_d R_d ... B_1 R_1 and V likewise (Eq. rbt-depth-d).
 * U^T = R_1 B_1 ... R_d B_d, so the innermost factor acts first: for
 * k = d down to 1 apply B_k on both sides, then R_k (rows) and R'_k
 * (columns). */
void orc_transform_2sided_tiled(int64_t n, int d, int64_t align, const double *U, int64_t ldu,
                                const double *V, int64_t ldv, double *A, int64_t lda)
{
    for (int k = d; k >= 1; k--) {
        orc_layer_rows_tiled(n, d, align, k, A, lda, n);
        orc_layer_cols_tiled(n, d, align, k, A, lda, n);
        for (int64_t j = 0; j < n; j++)
            for (int64_t i = 0; i < n; i++)
                A[IDX(i, j, lda)] *= U[IDX(i, k - 1, ldu)];
        for (int64_t j = 0; j < n; j++) {
            double v = V[IDX(j, k - 1, ldv)];
            for (int64_t i = 0; i < n; i++)
                A[IDX(i, j, lda)] *= v;
        }
    }
}

void orc_transform_2sided(int64_t n, int d, const double *U, int64_t ldu,
                          const double *V, int64_t ldv, double *A, int64_t lda)
{
    orc_transform_2sided_tiled(n, d, 1, U, ldu, V, ldv, A, lda);
}

/* W^T B: for k = d..1, B <- B_k B then R_k B.
 * W B  : for k = 1..d, B <- R_k B then B_k B. */
void orc_transform_vec_tiled(int64_t n, int d, int64_t align, const double *W, int64_t ldw, int trans,
                             double *B, int64_t ldb, int64_t nrhs)
{
    if (trans) {
        for (int k = d; k >= 1; k--) {
            orc_layer_rows_tiled(n, d, align, k, B, ldb, nrhs);
            for (int64_t c = 0; c < nrhs; c++)
                for (int64_t i = 0; i < n; i++)
                    B[IDX(i, c, ldb)] *= W[IDX(i, k - 1, ldw)];
        }
    } else {
        for (int k = 1; k <= d; k++) {
            for (int64_t c = 0; c < nrhs; c++)
                for (int64_t i = 0; i < n; i++)
                    B[IDX(i, c, ldb)] *= W[IDX(i, k - 1, ldw)];
            orc_layer_rows_tiled(n, d, align, k, B, ldb, nrhs);
        }
    }
}

void orc_transform_vec(int64_t n, int d, const double *W, int64_t ldw, int trans,
                       double *B, int64_t ldb, int64_t nrhs)
{
    orc_transform_vec_tiled(n, d, 1, W, ldw, trans, B, ldb, nrhs);
}

/* ------------------------------------------------- rotation butterflies */

/* Sec. 3, the block-rotation variant after Eq. (rbt-depth-d): every
 * butterfly is [[C, 0, S], [0, I_nu, 0], [S, 0, -C]] with C, S diagonal and
 * C^2 + S^2 = I (the truncated rows take the angle 0, i.e. the identity),
 * and the layers are composed as in Eq. (rbt-depth-d) with R_k = I, so the
 * transform is orthogonal.  The angle of the pair whose top row is i in
 * layer k is theta = 2 pi u, u uniform on [0, 1) from the same counter as
 * the diagonal entries (seed, side, layer, i).
 * Packed storage (n x d, like the scaled form): in column k-1, cos(theta)
 * at the top row of each pair, sin(theta) at its bottom row, and 1 at the
 * nu rows and in every layer k > d_s. */
static const double TWO_PI = 6.283185307179586476925286766559;

double orc_rot_u(uint64_t seed, int side, int layer, int64_t i)
{
    uint64_t key = seed ^ ((uint64_t)side << 62) ^ ((uint64_t)layer << 48) ^ (uint64_t)i;
    return (double)(orc_splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
}

void orc_generate_rot(int64_t n, int d, int64_t align, uint64_t seed, double *U, double *V, int64_t ld)
{
    int ds = orc_depth_eff(n, d);
    int64_t m = orc_ref_size_tiled(n, d, align);
    for (int side = 0; side < 2; side++) {
        double *W = side ? V : U;
        for (int k = 1; k <= d; k++) {
            for (int64_t i = 0; i < n; i++)
                W[IDX(i, k - 1, ld)] = 1.0;
            if (k > ds)
                continue;
            int64_t h = m >> k;
            for (int64_t start = 0; start < n; start += 2 * h)
                for (int64_t i = start; i < start + h && i + h < n; i++) {
                    double th = TWO_PI * orc_rot_u(seed, side, k, i);
                    W[IDX(i, k - 1, ld)] = cos(th);
                    W[IDX(i + h, k - 1, ld)] = sin(th);
                }
        }
    }
}

/* X <- B_k X for layer k of the rotation form, coefficients in column k-1
 * of W: each pair (i, i + h) becomes (c x_i + s x_p, s x_i - c x_p). */
void orc_layer_rows_rot(int64_t n, int d, int64_t align, int k, const double *W, int64_t ldw, double *X,
                        int64_t ldx, int64_t ncols)
{
    if (k > orc_depth_eff(n, d))
        return;
    int64_t m = orc_ref_size_tiled(n, d, align);
    int64_t h = m >> k;
    for (int64_t col = 0; col < ncols; col++)
        for (int64_t start = 0; start < n; start += 2 * h)
            for (int64_t i = start; i < start + h && i + h < n; i++) {
                int64_t p = i + h;
                double c = W[IDX(i, k - 1, ldw)], sn = W[IDX(p, k - 1, ldw)];
                double a = X[IDX(i, col, ldx)], b = X[IDX(p, col, ldx)];
                X[IDX(i, col, ldx)] = c * a + sn * b;
                X[IDX(p, col, ldx)] = sn * a - c * b;
            }
}

/* X <- X B_k: B_k is symmetric, so the same pair operation runs along each row. */
void orc_layer_cols_rot(int64_t n, int d, int64_t align, int k, const double *W, int64_t ldw, double *X,
                        int64_t ldx, int64_t nrows)
{
    if (k > orc_depth_eff(n, d))
        return;
    int64_t m = orc_ref_size_tiled(n, d, align);
    int64_t h = m >> k;
    for (int64_t start = 0; start < n; start += 2 * h)
        for (int64_t j = start; j < start + h && j + h < n; j++) {
            int64_t p = j + h;
            double c = W[IDX(j, k - 1, ldw)], sn = W[IDX(p, k - 1, ldw)];
            for (int64_t r = 0; r < nrows; r++) {
                double a = X[IDX(r, j, ldx)], b = X[IDX(r, p, ldx)];
                X[IDX(r, j, ldx)] = c * a + sn * b;
                X[IDX(r, p, ldx)] = sn * a - c * b;
            }
        }
}

/* U^T A V with U = B^U_d ... B^U_1, V = B^V_d ... B^V_1 (each B symmetric):
 * U^T A V = B^U_1 ... B^U_d A B^V_d ... B^V_1, so layer d acts first. */
void orc_transform_2sided_rot(int64_t n, int d, int64_t align, const double *U, int64_t ldu, const double *V,
                              int64_t ldv, double *A, int64_t lda)
{
    for (int k = d; k >= 1; k--) {
        orc_layer_rows_rot(n, d, align, k, U, ldu, A, lda, n);
        orc_layer_cols_rot(n, d, align, k, V, ldv, A, lda, n);
    }
}

/* W^T B = B_1 ... B_d B (layer d first); W B = B_d ... B_1 B (layer 1 first). */
void orc_transform_vec_rot(int64_t n, int d, int64_t align, const double *W, int64_t ldw, int trans, double *B,
                           int64_t ldb, int64_t nrhs)
{
    if (trans)
        for (int k = d; k >= 1; k--)
            orc_layer_rows_rot(n, d, align, k, W, ldw, B, ldb, nrhs);
    else
        for (int k = 1; k <= d; k++)
            orc_layer_rows_rot(n, d, align, k, W, ldw, B, ldb, nrhs);
}

/* ------------------------------------------------------------------ GENP */

/* Textbook right-looking Gaussian elimination without row exchanges.
 * Stops at the first pivot that is exactly zero or not finite. */
int64_t orc_genp(int64_t n, double *A, int64_t lda)
{
    for (int64_t k = 0; k < n; k++) {
        double p = A[IDX(k, k, lda)];
        if (p == 0.0 || !isfinite(p))
            return k;
        for (int64_t i = k + 1; i < n; i++)
            A[IDX(i, k, lda)] /= p;
        for (int64_t j = k + 1; j < n; j++) {
            double u = A[IDX(k, j, lda)];
            for (int64_t i = k + 1; i < n; i++)
                A[IDX(i, j, lda)] -= A[IDX(i, k, lda)] * u;
        }
    }
    return -1;
}

void orc_genp_solve(int64_t n, int64_t nrhs, const double *LU, int64_t lda, int trans,
                    double *B, int64_t ldb)
{
    for (int64_t c = 0; c < nrhs; c++) {
        double *b = B + (size_t)c * (size_t)ldb;
        if (!trans) {
            /* L y = b (unit lower), then U x = y */
            for (int64_t i = 0; i < n; i++) {
                double s = b[i];
                for (int64_t j = 0; j < i; j++)
                    s -= LU[IDX(i, j, lda)] * b[j];
                b[i] = s;
            }
            for (int64_t i = n - 1; i >= 0; i--) {
                double s = b[i];
                for (int64_t j = i + 1; j < n; j++)
                    s -= LU[IDX(i, j, lda)] * b[j];
                b[i] = s / LU[IDX(i, i, lda)];
            }
        } else {
            /* U^T y = b (lower, non-unit), then L^T x = y (upper, unit) */
            for (int64_t i = 0; i < n; i++) {
                double s = b[i];
                for (int64_t j = 0; j < i; j++)
                    s -= LU[IDX(j, i, lda)] * b[j];
                b[i] = s / LU[IDX(i, i, lda)];
            }
            for (int64_t i = n - 1; i >= 0; i--) {
                double s = b[i];
                for (int64_t j = i + 1; j < n; j++)
                    s -= LU[IDX(j, i, lda)] * b[j];
                b[i] = s;
            }
        }
    }
}

/* ----------------------------------------------------- backward error */

void orc_residual(int64_t n, int64_t nrhs, const double *A, int64_t lda,
                  const double *X, int64_t ldx, const double *B, int64_t ldb,
                  double *R, int64_t ldr)
{
    for (int64_t c = 0; c < nrhs; c++)
        for (int64_t i = 0; i < n; i++) {
            double s = B[IDX(i, c, ldb)];
            for (int64_t j = 0; j < n; j++)
                s -= A[IDX(i, j, lda)] * X[IDX(j, c, ldx)];
            R[IDX(i, c, ldr)] = s;
        }
}

/* infinity norm: largest absolute row sum */
double orc_norm_inf_mat(int64_t n, const double *A, int64_t lda)
{
    double best = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = 0; j < n; j++)
            s += fabs(A[IDX(i, j, lda)]);
        if (s > best || isnan(s))
            best = s;
    }
    return best;
}

static double norm_inf_vec(int64_t n, const double *x)
{
    double best = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double a = fabs(x[i]);
        if (a > best || isnan(a))
            best = a;
    }
    return best;
}

/* Eq. (inf-norm-backerr): ||b - A x|| / (||A|| ||x|| + ||b||), infinity norms,
 * with the norm of the original A.  Several right-hand sides: the largest. */
double orc_backward_error(int64_t n, int64_t nrhs, const double *A, int64_t lda,
                          const double *X, int64_t ldx, const double *B, int64_t ldb)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double anorm = orc_norm_inf_mat(n, A, lda);
    double worst = 0.0;
    for (int64_t c = 0; c < nrhs; c++) {
        orc_residual(n, 1, A, lda, X + (size_t)c * (size_t)ldx, ldx,
                     B + (size_t)c * (size_t)ldb, ldb, r, n);
        double num = norm_inf_vec(n, r);
        double den = anorm * norm_inf_vec(n, X + (size_t)c * (size_t)ldx) +
                     norm_inf_vec(n, B + (size_t)c * (size_t)ldb);
        double e = den > 0.0 ? num / den : (num > 0.0 ? INFINITY : 0.0);
        if (e > worst || isnan(e))
            worst = e;
    }
    free(r);
    return worst;
}

/* ------------------------------------------------------------ full solve */

/* Eq. (precond) recipe: A~ = U^T A V, b~ = U^T b, GENP solve of A~ x~ = b~,
 * x = V x~; then stationary iterative refinement on the original system
 * (Sec. 5): r = b - A x, dx = V A~^{-1} U^T r, x += dx, until the backward
 * error reaches tol or refine_max steps were taken. */
static void xform_2sided(int kind, int64_t n, int d, int64_t align, const double *U, const double *V, double *A)
{
    if (kind == 1)
        orc_transform_2sided_rot(n, d, align, U, n, V, n, A, n);
    else
        orc_transform_2sided_tiled(n, d, align, U, n, V, n, A, n);
}

static void xform_vec(int kind, int64_t n, int d, int64_t align, const double *W, int trans, double *B, int64_t ldb,
                      int64_t nrhs)
{
    if (kind == 1)
        orc_transform_vec_rot(n, d, align, W, n, trans, B, ldb, nrhs);
    else
        orc_transform_vec_tiled(n, d, align, W, n, trans, B, ldb, nrhs);
}

/* kind 0: the scaled butterflies of Eq. (rbt-depth-d); kind 1: the rotation form. */
int64_t orc_rbt_solve_kind(int64_t n, int64_t nrhs, int d, int64_t align, int kind, uint64_t seed,
                           const double *A, int64_t lda, const double *B, int64_t ldb,
                           double *X, int64_t ldx, int refine_max, double tol, double *out)
{
    size_t nn = (size_t)n * (size_t)n;
    double *U = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(d > 0 ? d : 1));
    double *V = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(d > 0 ? d : 1));
    double *At = (double *)malloc(sizeof(double) * (nn > 0 ? nn : 1));
    double *R = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(nrhs > 0 ? nrhs : 1));
    int64_t status = -1;

    if (kind == 1)
        orc_generate_rot(n, d, align, seed, U, V, n);
    else
        orc_generate(n, d, seed, U, V, n);
    for (int64_t j = 0; j < n; j++)
        memcpy(At + (size_t)j * (size_t)n, A + (size_t)j * (size_t)lda, sizeof(double) * (size_t)n);
    xform_2sided(kind, n, d, align, U, V, At);
    status = orc_genp(n, At, n);
    if (status >= 0)
        goto done;

    for (int64_t c = 0; c < nrhs; c++)
        memcpy(X + (size_t)c * (size_t)ldx, B + (size_t)c * (size_t)ldb, sizeof(double) * (size_t)n);
    xform_vec(kind, n, d, align, U, 1, X, ldx, nrhs);
    orc_genp_solve(n, nrhs, At, n, 0, X, ldx);
    xform_vec(kind, n, d, align, V, 0, X, ldx, nrhs);

    double berr = orc_backward_error(n, nrhs, A, lda, X, ldx, B, ldb);
    out[0] = berr;
    int it = 0;
    while (it < refine_max && !(berr <= tol)) {
        orc_residual(n, nrhs, A, lda, X, ldx, B, ldb, R, n);
        xform_vec(kind, n, d, align, U, 1, R, n, nrhs);
        orc_genp_solve(n, nrhs, At, n, 0, R, n);
        xform_vec(kind, n, d, align, V, 0, R, n, nrhs);
        for (int64_t c = 0; c < nrhs; c++)
            for (int64_t i = 0; i < n; i++)
                X[IDX(i, c, ldx)] += R[IDX(i, c, n)];
        berr = orc_backward_error(n, nrhs, A, lda, X, ldx, B, ldb);
        it++;
    }
    out[1] = berr;
    out[2] = (double)it;

done:
    free(U);
    free(V);
    free(At);
    free(R);
    return status;
}

int64_t orc_rbt_solve_tiled(int64_t n, int64_t nrhs, int d, int64_t align, uint64_t seed,
                            const double *A, int64_t lda, const double *B, int64_t ldb,
                            double *X, int64_t ldx, int refine_max, double tol, double *out)
{
    return orc_rbt_solve_kind(n, nrhs, d, align, 0, seed, A, lda, B, ldb, X, ldx, refine_max, tol, out);
}

int64_t orc_rbt_solve(int64_t n, int64_t nrhs, int d, uint64_t seed,
                      const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *X, int64_t ldx, int refine_max, double tol, double *out)
{
    return orc_rbt_solve_tiled(n, nrhs, d, 1, seed, A, lda, B, ldb, X, ldx, refine_max, tol, out);
}

/* ------------------------------------------------------------- GMRES-IR */

static double dot_vec(int64_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s += x[i] * y[i];
    return s;
}

/* Refinement by restarted GMRES (the GMRES-based refinement the paper lists
 * as the stronger alternative to stationary refinement, Sec. 5), right
 * preconditioned by the transformed factorization M^{-1} = V (L U)^{-1} U^T:
 * each cycle solves A M^{-1} u = r, r = b - A x, by GMRES(restart) with
 * modified Gram-Schmidt Arnoldi and Givens rotations, then x += M^{-1} Q y.
 * LU holds factors of U^T A V of whatever accuracy (they only precondition).
 * One right-hand side.  Cycles repeat while the backward error exceeds tol,
 * up to max_iter preconditioned products in all.
 * out[0] = backward error on entry, out[1] = final backward error,
 * out[2] = preconditioned products used, out[3] = cycles;
 * hist (max_iter + 1 entries, may be NULL) receives the Arnoldi residual
 * estimate |g_{j+1}| after each inner step, cycle after cycle. */
void orc_gmres_ir(int64_t n, int d, int64_t align, const double *U, const double *V, const double *LU,
                  const double *A, int64_t lda, const double *b, double *x, int restart, int max_iter,
                  double tol, double *out, double *hist)
{
    int m = restart > 0 ? restart : 1;
    double *Q = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double berr = orc_backward_error(n, 1, A, lda, x, n, b, n);
    out[0] = berr;
    int used = 0, cycles = 0;
#define HH(i, j) H[(size_t)(i) + (size_t)(j) * (size_t)(m + 1)]
    while (used < max_iter && !(berr <= tol)) {
        cycles++;
        orc_residual(n, 1, A, lda, x, n, b, n, w, n); /* r = b - A x */
        double beta = sqrt(dot_vec(n, w, w));
        if (!(beta > 0.0))
            break;
        for (int64_t i = 0; i < n; i++)
            Q[i] = w[i] / beta;
        for (int i = 0; i <= m; i++)
            g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m && used < max_iter; j++) {
            /* w = A M^{-1} q_j */
            memcpy(z, Q + (size_t)j * (size_t)n, sizeof(double) * (size_t)n);
            orc_transform_vec_tiled(n, d, align, U, n, 1, z, n, 1);
            orc_genp_solve(n, 1, LU, n, 0, z, n);
            orc_transform_vec_tiled(n, d, align, V, n, 0, z, n, 1);
            used++;
            for (int64_t i = 0; i < n; i++) {
                double s = 0.0;
                for (int64_t c = 0; c < n; c++)
                    s += A[IDX(i, c, lda)] * z[c];
                w[i] = s;
            }
            for (int i = 0; i <= j; i++) { /* modified Gram-Schmidt */
                const double *qi = Q + (size_t)i * (size_t)n;
                double h = dot_vec(n, qi, w);
                HH(i, j) = h;
                for (int64_t r = 0; r < n; r++)
                    w[r] -= h * qi[r];
            }
            double hn = sqrt(dot_vec(n, w, w));
            HH(j + 1, j) = hn;
            if (hn > 0.0)
                for (int64_t r = 0; r < n; r++)
                    Q[(size_t)(j + 1) * (size_t)n + r] = w[r] / hn;
            for (int i = 0; i < j; i++) { /* earlier rotations on the new column */
                double a = HH(i, j), c2 = HH(i + 1, j);
                HH(i, j) = cs[i] * a + sn[i] * c2;
                HH(i + 1, j) = -sn[i] * a + cs[i] * c2;
            }
            double a = HH(j, j), c2 = HH(j + 1, j);
            double rr = sqrt(a * a + c2 * c2);
            cs[j] = rr > 0.0 ? a / rr : 1.0;
            sn[j] = rr > 0.0 ? c2 / rr : 0.0;
            HH(j, j) = rr;
            HH(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (hist)
                hist[used - 1] = fabs(g[j + 1]);
            k = j + 1;
            if (!(hn > 0.0) || fabs(g[j + 1]) <= 1e-14 * beta)
                break;
        }
        /* y = R^{-1} g, then x += M^{-1} (Q y) */
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int c = i + 1; c < k; c++)
                s -= HH(i, c) * y[c];
            y[i] = s / HH(i, i);
        }
        for (int64_t r = 0; r < n; r++) {
            double s = 0.0;
            for (int i = 0; i < k; i++)
                s += Q[(size_t)i * (size_t)n + r] * y[i];
            z[r] = s;
        }
        orc_transform_vec_tiled(n, d, align, U, n, 1, z, n, 1);
        orc_genp_solve(n, 1, LU, n, 0, z, n);
        orc_transform_vec_tiled(n, d, align, V, n, 0, z, n, 1);
        for (int64_t r = 0; r < n; r++)
            x[r] += z[r];
        berr = orc_backward_error(n, 1, A, lda, x, n, b, n);
    }
#undef HH
    out[1] = berr;
    out[2] = (double)used;
    out[3] = (double)cycles;
    free(Q);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    free(z);
    free(w);
}
