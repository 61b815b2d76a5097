// Internal interfaces between the GENP kernels, the tensor-core GEMM and the
// solve driver.
#pragma once

#include "common.cuh"

namespace rbt {

constexpr int kMaxNB = 128;       // largest GENP block size (shared-memory bound)
constexpr int kDefaultNB64 = 64;  // default block size, double
constexpr int kDefaultNB32 = 128; // default block size, float storage
constexpr int kSolveNB = 128;     // block size of the triangular solves

// C (M x N) -= A (M x K) B (K x N), SIMT, column-major.
template <typename T>
rbt_status gemm_sub_simt(int64_t M, int64_t N, int K, const T *Am, int64_t lda_a, const T *Bm, int64_t ldb_b,
                         T *C, int64_t ldc, const int64_t *info, cudaStream_t stream);

// Block steps k0, k0+nb, ... < k_end: diagonal factor + both TRSMs, and the
// trailing update too when trailing_simt is set.
template <typename T>
rbt_status genp_panel_steps(int64_t n, T *A, int64_t lda, int64_t *info, int nb, int64_t k0, int64_t k_end,
                            bool trailing_simt, cudaStream_t stream);

rbt_status genp_configure(int prec, int nb);

template <typename T>
rbt_status lu_solve(int64_t n, int64_t nrhs, const T *LU, int64_t lda, int trans, T *B, int64_t ldb,
                    cudaStream_t stream);

rbt_status narrow_block(int64_t n, int64_t nrhs, const double *B, int64_t ldb, float *F, int64_t ldf,
                        cudaStream_t stream);
rbt_status widen_block(int64_t n, int64_t nrhs, const float *F, int64_t ldf, double *B, int64_t ldb,
                       cudaStream_t stream);

size_t residual_ws(int64_t n, int64_t nrhs);
// bytes of the partial sums residual_impl / norm_inf_impl write into `part`
// (n x nrhs x ceil(n / chunk) doubles; at most residual_ws(n, nrhs) - 272)
size_t residual_part_bytes(int64_t n, int64_t nrhs);
rbt_status norm_inf_impl(int64_t n, const double *A, int64_t lda, double *d_out, double *part,
                         cudaStream_t stream);
rbt_status residual_impl(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X, int64_t ldx,
                         const double *B, int64_t ldb, double *R, int64_t ldr, const double *d_anorm,
                         double *d_berr, double *part, cudaStream_t stream);
rbt_status add_block(int64_t n, int64_t nrhs, const double *D, int64_t ldd, double *X, int64_t ldx,
                     cudaStream_t stream);

// Byte offsets of rbt_solve's workspace (the adjoint reuses the factors).
struct SolveLayout {
    size_t at, at64, u, v, r, info, scal, res, fac, sol, gm, total;
    int64_t ldt;
};
void solve_layout(const rbt_opts *o, int64_t n, int64_t nrhs, SolveLayout *out);

// The working-copy and one-sided transforms with the reference size's tile
// alignment (align = n_b of Sec. 3's tiled rule; 0 or 1 = non-tiled) and the
// butterfly kind (RBT_KIND_SCALED or RBT_KIND_ROTATION).
rbt_status apply_2sided_wp(int64_t n, int32_t d, int64_t align, const double *U, const double *V, int64_t ldw,
                           const double *A_in, int64_t lda_in, void *A_out, int64_t lda_out, int32_t prec,
                           cudaStream_t stream, int32_t kind = RBT_KIND_SCALED);
rbt_status apply_vec(int64_t n, int32_t d, int64_t align, const double *W, int64_t ldw, int32_t trans,
                     double *B, int64_t ldb, int64_t nrhs, cudaStream_t stream, int32_t kind = RBT_KIND_SCALED);

// GMRES-based refinement: vector kernels (gmres.cu)
constexpr int kGmresDefaultRestart = 30;
constexpr int kGmresMaxRestart = 64;
int64_t gm_part_len(int64_t n);
rbt_status gm_dots(int64_t n, const double *Q, int64_t ldq, int k, const double *w, double *part, double *out,
                   cudaStream_t s);
rbt_status gm_sub(int64_t n, const double *Q, int64_t ldq, int k, const double *h, double *w, cudaStream_t s);
rbt_status gm_gemv(int64_t n, const double *Q, int64_t ldq, int k, const double *y, double *z, cudaStream_t s);
rbt_status gm_scale(int64_t n, double alpha, const double *src, double *dst, cudaStream_t s);
rbt_status gm_add(int64_t n, const double *z, double *x, cudaStream_t s);

// genp_solve / genp_solve_wp on validated arguments (work of their size
// queries), leaving the timeout flag at the front of work as it is: set by a
// chained solve that gave up, cleared only by whoever owns the call.
rbt_status genp_solve_run(int64_t n, int64_t nrhs, int32_t prec, const void *LU, int64_t lda, int32_t trans,
                          double *B, int64_t ldb, void *work, cudaStream_t stream);
rbt_status genp_solve_wp_run(int64_t n, int64_t nrhs, int32_t prec, const void *LU, int64_t lda, int32_t trans,
                             double *B, int64_t ldb, void *work, cudaStream_t stream);

size_t genp_factor_workspace_impl(int64_t n, int prec, int nb);
rbt_status genp_factor_impl(int64_t n, int prec, void *A, int64_t lda, int64_t *info, void *work,
                            size_t work_bytes, int nb, cudaStream_t stream);

}  // namespace rbt
