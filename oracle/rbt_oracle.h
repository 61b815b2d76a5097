/*
 * Plain FP64 CPU oracle for the generalized random butterfly transform (RBT)
 * solver of Lindquist, Luszczek and Dongarra, "Generalizing Random Butterfly
 * Transforms to Arbitrary Matrix Sizes" (arXiv 2312.09376).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this code; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no source with the CUDA path.
 *
 * Every routine is the slow, literal form of the definition it cites:
 * explicit loops, one layer or one elimination step at a time, double
 * precision throughout.  Matrices are column-major with a leading dimension.
 *
 * Conventions (readings of the paper where it is silent or inconsistent):
 *  - U = B_d R_d ... B_1 R_1 exactly as in Eq. (rbt-depth-d): each butterfly
 *    layer B_k sits to the LEFT of its random diagonal R_k.  The worked
 *    depth-1 example of Sec. 4 (Eq. example-for-small-d) fixes this order.
 *  - Effective depth d_s = min(d, ceil(log2 n)); reference size
 *    m = 2^d_s * ceil(n / 2^d_s) (the non-tiled rule of Sec. 3);
 *    layer k <= d_s has half-butterfly size h_k = m / 2^k; layers k > d_s are
 *    diagonal only (butterflies of size one, the leaves of the recursion in
 *    the proof of Lemma 2).
 *  - Packed storage (Sec. 3, Algorithm 1): column k-1 of the n x d array U
 *    holds the diagonal of R_k.
 *  - Random values exp(r/20), r uniform on [-1, 1) (Sec. 6), drawn with the
 *    counter-based SplitMix64 generator (Steele, Lea, Flood 2014).
 */
#ifndef RBT_ORACLE_H
#define RBT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- sizes (Sec. 3, Algorithm 1 reference size) ---- */
int     orc_ceil_log2(int64_t n);
int     orc_depth_eff(int64_t n, int d);
int64_t orc_ref_size(int64_t n, int d);
int64_t orc_ref_size_tiled(int64_t n, int d, int64_t align);
int64_t orc_lcm(int64_t p, int64_t q);
int64_t orc_ref_size_comm_free(int64_t n, int d, int64_t nb, int64_t p, int64_t q);

/* ---- generator (Sec. 6 distribution; SplitMix64 published definition) ---- */
uint64_t orc_splitmix64(uint64_t key);
/* one random coefficient: side 0 = U, 1 = V; layer k in 1..d; row i */
double   orc_coef(uint64_t seed, int side, int layer, int64_t i);
/* U, V: n x d column-major, leading dimension ld >= n */
void     orc_generate(int64_t n, int d, uint64_t seed, double *U, double *V, int64_t ld);

/* ---- one butterfly layer B_k (Eq. O-matrix-definition, alignment rule) ----
 * X <- B_k X on the rows of an n x ncols block.  rbt_depth d is needed for
 * the reference size only. */
void orc_layer_rows(int64_t n, int d, int k, double *X, int64_t ldx, int64_t ncols);
void orc_layer_rows_tiled(int64_t n, int d, int64_t align, int k, double *X, int64_t ldx, int64_t ncols);
/* X <- X B_k on the columns of an nrows x n block */
void orc_layer_cols(int64_t n, int d, int k, double *X, int64_t ldx, int64_t nrows);
void orc_layer_cols_tiled(int64_t n, int d, int64_t align, int k, double *X, int64_t ldx, int64_t nrows);

/* ---- two-sided transform A <- U^T A V (Eq. rbt-depth-d, Eq. precond) ---- */
void orc_transform_2sided(int64_t n, int d, const double *U, int64_t ldu,
                          const double *V, int64_t ldv, double *A, int64_t lda);
/* the same with the tiled reference size (align = tile size n_b, Sec. 3) */
void orc_transform_2sided_tiled(int64_t n, int d, int64_t align, const double *U, int64_t ldu,
                                const double *V, int64_t ldv, double *A, int64_t lda);

/* ---- one-sided transforms on an n x nrhs block (Eq. precond steps 1, 3) ----
 * trans = 1: B <- W^T B ;  trans = 0: B <- W B */
void orc_transform_vec(int64_t n, int d, const double *W, int64_t ldw, int trans,
                       double *B, int64_t ldb, int64_t nrhs);
void orc_transform_vec_tiled(int64_t n, int d, int64_t align, const double *W, int64_t ldw, int trans,
                             double *B, int64_t ldb, int64_t nrhs);

/* ---- Gaussian elimination with no pivoting (Sec. 1, Sec. 4) ----
 * In-place Doolittle LU: unit lower L below the diagonal, U on and above.
 * Returns -1 on success, else the 0-based index of the first pivot that is
 * exactly zero or not finite (elimination stops there). */
int64_t orc_genp(int64_t n, double *A, int64_t lda);

/* ---- triangular solves with the GENP factors ----
 * trans = 0: B <- (L U)^{-1} B ; trans = 1: B <- (L U)^{-T} B */
void orc_genp_solve(int64_t n, int64_t nrhs, const double *LU, int64_t lda, int trans,
                    double *B, int64_t ldb);

/* ---- residual and infinity-norm backward error (Eq. inf-norm-backerr) ---- */
/* R <- B - A X */
void   orc_residual(int64_t n, int64_t nrhs, const double *A, int64_t lda,
                    const double *X, int64_t ldx, const double *B, int64_t ldb,
                    double *R, int64_t ldr);
double orc_norm_inf_mat(int64_t n, const double *A, int64_t lda);
/* largest over the right-hand sides of ||b-Ax||/(||A|| ||x|| + ||b||) */
double orc_backward_error(int64_t n, int64_t nrhs, const double *A, int64_t lda,
                          const double *X, int64_t ldx, const double *B, int64_t ldb);

/* ---- full RBT solve (Eq. precond recipe + Sec. 5 iterative refinement) ----
 * Does not modify A or B.  Returns -1 on success, else the zero-pivot index.
 * out[0] = backward error before refinement, out[1] = final backward error,
 * out[2] = refinement steps taken. */
int64_t orc_rbt_solve(int64_t n, int64_t nrhs, int d, uint64_t seed,
                      const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *X, int64_t ldx, int refine_max, double tol, double *out);
/* Rotation butterflies (Sec. 3, block-rotation variant; R_k = I, orthogonal). */
double orc_rot_u(uint64_t seed, int side, int layer, int64_t i);
void orc_generate_rot(int64_t n, int d, int64_t align, uint64_t seed, double *U, double *V, int64_t ld);
void orc_layer_rows_rot(int64_t n, int d, int64_t align, int k, const double *W, int64_t ldw, double *X,
                        int64_t ldx, int64_t ncols);
void orc_layer_cols_rot(int64_t n, int d, int64_t align, int k, const double *W, int64_t ldw, double *X,
                        int64_t ldx, int64_t nrows);
void orc_transform_2sided_rot(int64_t n, int d, int64_t align, const double *U, int64_t ldu, const double *V,
                              int64_t ldv, double *A, int64_t lda);
void orc_transform_vec_rot(int64_t n, int d, int64_t align, const double *W, int64_t ldw, int trans, double *B,
                           int64_t ldb, int64_t nrhs);
int64_t orc_rbt_solve_kind(int64_t n, int64_t nrhs, int d, int64_t align, int kind, uint64_t seed,
                           const double *A, int64_t lda, const double *B, int64_t ldb,
                           double *X, int64_t ldx, int refine_max, double tol, double *out);
int64_t orc_rbt_solve_tiled(int64_t n, int64_t nrhs, int d, int64_t align, uint64_t seed,
                            const double *A, int64_t lda, const double *B, int64_t ldb,
                            double *X, int64_t ldx, int refine_max, double tol, double *out);

/* ---- refinement by restarted GMRES, right preconditioned by V (LU)^{-1} U^T ----
 * LU: factors of U^T A V (any accuracy), n x n with ld n; one right-hand
 * side; x in/out.  out[0..3] = backward error on entry, final backward
 * error, preconditioned products, cycles; hist (max_iter entries or NULL)
 * = Arnoldi residual estimates after each inner step. */
void orc_gmres_ir(int64_t n, int d, int64_t align, const double *U, const double *V, const double *LU,
                  const double *A, int64_t lda, const double *b, double *x, int restart, int max_iter,
                  double tol, double *out, double *hist);

#ifdef __cplusplus
}
#endif
#endif
