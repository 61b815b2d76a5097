/*
 * gb300-rbt: generalized random butterfly transform (RBT) + Gaussian
 * elimination with no pivoting (GENP) on one NVIDIA GB300 (sm_103a).
 *
 * Method: Lindquist, Luszczek, Dongarra, "Generalizing Random Butterfly
 * Transforms to Arbitrary Matrix Sizes", arXiv 2312.09376.  The linear system
 * A x = b is rewritten (Eq. precond) as (U^T A V)(V^{-1} x) = U^T b, where U
 * and V are depth-d generalized RBTs (Eq. rbt-depth-d) whose butterfly layers
 * are truncated to the order n, so n need not be a multiple of 2^d.
 *
 * Conventions shared by every entry point
 *  - Matrices are column-major.  A leading dimension (lda, ldb, ...) is the
 *    distance in elements between consecutive columns and must be >= the
 *    number of rows (and >= 1).
 *  - Every pointer argument named A, B, X, U, V, W, LU, R, work or d_* is a
 *    DEVICE pointer on the current CUDA device; host pointers are called out
 *    explicitly (opts, info, sizes of batched calls).  The caller owns every
 *    buffer; the library never allocates device memory on its own (scratch
 *    comes from the caller's `work`) and never frees.
 *  - Every call is asynchronous and ordered on `stream` (0 = legacy default
 *    stream) unless documented otherwise; device results are valid after the
 *    stream is synchronized.  rbt_solve synchronizes `stream` once per
 *    refinement step because it decides on the host whether to continue.
 *  - Return value: RBT_OK, a negative rbt_status for an argument or CUDA
 *    error (nothing further is enqueued), or a positive numerical outcome.
 *  - Packed butterfly storage (Sec. 3, Algorithm 1): U and V are n x d arrays
 *    (leading dimension ldw); column k-1 holds the random diagonal R_k of
 *    layer k, layer 1 being the rightmost factor (one butterfly of order n).
 *  - Butterfly order (Eq. rbt-depth-d): U = B_d R_d ... B_1 R_1, each
 *    butterfly layer B_k LEFT of its diagonal R_k.  Layer k <= d_s =
 *    min(d, ceil(log2 n)) has half-butterfly size h_k = m / 2^k with
 *    m = 2^d_s ceil(n / 2^d_s) (non-tiled reference size of Sec. 3); layers
 *    k > d_s are diagonal only.  The rotation form (rbt_generate_rot,
 *    RBT_KIND_ROTATION) has the same layer structure with R_k = I and its
 *    own per-pair coefficients in the same n x d storage.
 */
#ifndef GB300_RBT_H
#define GB300_RBT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cudaStream_t;

typedef enum {
    RBT_OK = 0,
    RBT_ERR_ARG = -1,          /* invalid argument (size, depth, pointer, ld) */
    RBT_ERR_CUDA = -2,         /* a CUDA runtime call or kernel launch failed */
    RBT_ERR_WORKSPACE = -3,    /* work_bytes smaller than the size query */
    RBT_ERR_TIMEOUT = -4,      /* a bounded device wait gave up */
    RBT_ERR_UNSUPPORTED = -5,  /* valid request the library does not implement */
    RBT_ZERO_PIVOT = 1,        /* GENP met a pivot that is exactly zero */
    RBT_NONFINITE = 2,         /* GENP met a pivot that is Inf or NaN */
    RBT_NOT_CONVERGED = 3      /* refinement (and any fallback) missed tol */
} rbt_status;

/* Working precision of the factorization. */
typedef enum {
    RBT_F64 = 0,   /* double storage and arithmetic */
    RBT_F32 = 1,   /* float storage, float SIMT trailing updates */
    RBT_TF32 = 2,  /* float storage, TF32 tensor-core trailing updates (fp32 accumulate) */
    RBT_BF16 = 3,  /* float storage, BF16 tensor-core operands (fp32 accumulate) */
    RBT_DF64 = 4,  /* double-float storage (pair of floats hi + lo, about 48 bits) and
                      double-float arithmetic on the FP32 pipes */
    RBT_DF64TC = 5, /* double-float storage; the GENP updates run on the BF16 tensor
                       cores by exact integer digit slicing (eight 7-bit digits per
                       entry, about 53 bits relative to each row's / column's
                       largest entry; 36 digit products), panels in double-float */
    RBT_DF64TC7 = 6 /* as RBT_DF64TC with seven digits per entry (about 47 bits
                       relative to the row / column maxima; 28 digit products, the
                       update about 14% faster); refinement takes more steps, and
                       with rbt_opts.fallback a stalled attempt refactors with
                       eight digits (RBT_DF64TC) before double */
} rbt_prec;

/* Options of rbt_solve (host struct). */
typedef struct {
    int32_t depth;       /* RBT depth d >= 0 (0 = plain GENP) */
    uint64_t seed;       /* seed of the butterfly coefficients */
    int32_t prec;        /* rbt_prec of the factorization */
    int32_t refine_max;  /* most refinement steps (Sec. 5); 0 = none */
    double tol;          /* stop once the backward error is <= tol */
    int32_t fallback;    /* nonzero: on stalled refinement refactor in FP64 */
    int32_t nb;          /* block size of GENP; 0 = library default */
    int64_t align;       /* reference size m (Sec. 3, Algorithm 1): 0 or 1 = the
                            non-tiled rule m = 2^d_s ceil(n / 2^d_s); n_b > 1 =
                            the tiled rule m = 2^d_s n_b ceil(n / (2^d_s n_b)),
                            which aligns every butterfly to n_b-row tiles */
    int32_t refine_mode; /* RBT_REFINE_STATIONARY (0): x += V A~^{-1} U^T r per
                            step (Sec. 5); RBT_REFINE_GMRES (1): restarted GMRES
                            on A M^{-1} u = r with M^{-1} = V A~^{-1} U^T (right
                            preconditioning by the factors), x += M^{-1} Q y per
                            cycle; refine_max then counts cycles and
                            rbt_info.iters preconditioned products */
    int32_t restart;     /* GMRES basis size per cycle, 0 = 30, at most 64 */
    int32_t kind;        /* butterflies: RBT_KIND_SCALED (0) = Eq. rbt-depth-d with
                            random diagonals; RBT_KIND_ROTATION (1) = the
                            block-rotation variant of Sec. 3 (orthogonal, R_k = I;
                            coefficients of rbt_generate_rot) */
    int32_t grid_p;      /* process grid p x q of the communication-free size of
                            Sec. 6, Eq. (comm-free-rbt-size): the top half of the
                            first layer spans lcm(p, q) 2^(d-1) ceil(n_t 2^-d /
                            lcm(p, q)) tiles of align rows (n_t = ceil(n / align)),
                            i.e. the tiled rule with tiles of lcm(p, q) align rows,
                            so that on a p x q block-cyclic distribution no
                            butterfly pairs rows (columns) of different process
                            rows (columns).  0 or 1 each = no grid (the rule of
                            align alone); at most 4096 each.  See
                            rbt_reference_size. */
    int32_t grid_q;      /* (the q of grid_p's p x q grid) */
} rbt_opts;

enum { RBT_REFINE_STATIONARY = 0, RBT_REFINE_GMRES = 1 };
enum { RBT_KIND_SCALED = 0, RBT_KIND_ROTATION = 1 };

/* Outcome of rbt_solve (host struct, written before return). */
typedef struct {
    int32_t status;          /* rbt_status of the solve */
    int64_t zero_pivot;      /* -1, or the 0-based index of the first bad pivot */
    int32_t iters;           /* refinement steps taken (all attempts) */
    int32_t fell_back;       /* 0: X comes from the factors of opts->prec;
                                1: the FP64 refactorization ran (X from it);
                                2: RBT_DF64TC7 only: the eight-digit (RBT_DF64TC)
                                   refactorization ran and X comes from it */
    double berr_unrefined;   /* Eq. inf-norm-backerr before refinement */
    double berr;             /* Eq. inf-norm-backerr of the returned X */
} rbt_info;

/* Human-readable name of a status code (static string). */
const char *rbt_status_string(int status);

/* rbt_reference_size -- the reference size m every butterfly layer is built
 * on (host function, no GPU): m = 2^d_s a ceil(n / (2^d_s a)) with
 * d_s = min(d, ceil(log2 n)) and a = max(align, 1) lcm(max(grid_p, 1),
 * max(grid_q, 1)).  align <= 1 and no grid: the non-tiled rule of Sec. 3;
 * align = n_b: the tiled rule of Sec. 3 (Algorithm 1); a p x q grid: the
 * communication-free size of Sec. 6, Eq. (comm-free-rbt-size), twice
 * lcm(p, q) 2^(d_s - 1) ceil(n_t 2^-d_s / lcm(p, q)) tiles of n_b rows.
 * Returns -1 for n < 0, d < 0 or > 62, align < 0, a grid side outside
 * [0, 4096], or an m that would not fit in int64. */
int64_t rbt_reference_size(int64_t n, int32_t d, int64_t align, int32_t grid_p, int32_t grid_q);

/* ---------------------------------------------------------------------------
 * rbt_generate -- random butterfly coefficients (Sec. 6: exp(r/20), r uniform
 * on [-1, 1); packed storage of Sec. 3).  Writes U and V, each n x d with
 * leading dimension ldw >= n.  Entry (i, k-1) of side s (0 = U, 1 = V) is
 * exp(r/20) with r = 2 u - 1, u = (x >> 11) 2^-53 and
 * x = SplitMix64(seed ^ (s << 62) ^ (k << 48) ^ i), SplitMix64 being the
 * first output of the generator of Steele, Lea and Flood (2014) started at
 * that state.  Errors: RBT_ERR_ARG for n < 0, d < 0, ldw < max(1, n).
 */
rbt_status rbt_generate(int64_t n, int32_t d, uint64_t seed, double *U, double *V,
                        int64_t ldw, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * rbt_generate_rot -- coefficients of the rotation form of the butterflies
 * (Sec. 3, the block-rotation variant after Eq. rbt-depth-d: every butterfly
 * is [[C, 0, S], [0, I_nu, 0], [S, 0, -C]] with C, S diagonal, C^2 + S^2 = I,
 * the truncated rows rotated by angle 0; the layers composed with R_k = I,
 * so U and V are orthogonal).  The pair of layer k with top row i (bottom
 * row i + m / 2^k, m the reference size for n, d and align as in
 * rbt_apply_2sided_tiled) turns by theta = 2 pi u, u = (x >> 11) 2^-53 and x
 * the SplitMix64 output of rbt_generate for (side, k, i).  Packed storage,
 * U and V n x d with leading dimension ldw: column k-1 holds cos(theta) at
 * each pair's top row, sin(theta) at its bottom row, and 1 at the unpaired
 * rows and in every layer k > min(d, ceil(log2 n)).  Transform with
 * rbt_transform_2sided / rbt_transform_vec, kind RBT_KIND_ROTATION, and the
 * same align.  Errors: RBT_ERR_ARG for n < 0, d < 0 or > 62, align < 0,
 * ldw < max(1, n).
 */
rbt_status rbt_generate_rot(int64_t n, int32_t d, int64_t align, uint64_t seed, double *U, double *V,
                            int64_t ldw, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * rbt_apply_2sided -- A_out <- U^T A_in V (Eq. rbt-depth-d, Algorithm 1),
 * all d layers fused into one pass over the matrix when d <= 3 (the
 * single-pass reorganization suggested at the end of Sec. 3); deeper
 * transforms take ceil(d_s / 3) passes.
 * A_in (n x n, lda_in) is read; A_out (n x n, lda_out) is written.  They may
 * be the same buffer with the same leading dimension (in place); otherwise
 * they must not overlap.  U, V: packed coefficients, leading dimension ldw.
 * Errors: RBT_ERR_ARG for n < 0, d < 0, bad leading dimensions or a partial
 * overlap of A_in and A_out.
 */
rbt_status rbt_apply_2sided(int64_t n, int32_t d, const double *U, const double *V, int64_t ldw,
                            const double *A_in, int64_t lda_in, double *A_out, int64_t lda_out,
                            cudaStream_t stream);

/* rbt_apply_2sided with the tiled reference size of Sec. 3 (Algorithm 1,
 * the tiled choice of m): align = the tile size n_b (0 or 1: the non-tiled
 * rule, the same as rbt_apply_2sided), m = 2^d_s n_b ceil(n / (2^d_s n_b)),
 * so the half size m / 2^k of every layer's butterflies is a multiple of
 * n_b.  Other arguments and errors as rbt_apply_2sided; RBT_ERR_ARG also for
 * align < 0. */
rbt_status rbt_apply_2sided_tiled(int64_t n, int32_t d, int64_t align, const double *U, const double *V,
                                  int64_t ldw, const double *A_in, int64_t lda_in, double *A_out, int64_t lda_out,
                                  cudaStream_t stream);

/* Same transform written as the working copy of a factorization in
 * precision prec (A_out: n x n, lda_out, element type double for RBT_F64,
 * float for RBT_F32 / RBT_TF32 / RBT_BF16, a pair of floats {hi, lo} for
 * RBT_DF64, RBT_DF64TC and RBT_DF64TC7), in the same single pass; A_in is not modified and must not
 * overlap A_out.  Requires min(d, ceil(log2 n)) <= 3 for the narrower types
 * (one pass must hold every layer); RBT_ERR_UNSUPPORTED otherwise.  The
 * float copy is computed in float arithmetic from the double input (it only
 * needs float accuracy: refinement measures against A in double), so it
 * differs from the double transform rounded to float by a few float ulps of
 * (|U|^T |A| |V|)_ij.  Likewise the float-pair copy is computed in
 * double-float arithmetic on the FP32 pipes: within about 2^-44
 * (|U|^T |A| |V|)_ij of the double transform (for d_s = 0 it is the double
 * result rounded to the pair). */
rbt_status rbt_apply_2sided_wp(int64_t n, int32_t d, const double *U, const double *V, int64_t ldw,
                               const double *A_in, int64_t lda_in, void *A_out, int64_t lda_out,
                               int32_t prec, cudaStream_t stream);

/* The general two-sided transform: A_out <- U^T A_in V with the tiled or
 * non-tiled reference size (align as rbt_apply_2sided_tiled), the butterfly
 * kind (RBT_KIND_SCALED: coefficients of rbt_generate, the transform of
 * rbt_apply_2sided; RBT_KIND_ROTATION: coefficients of rbt_generate_rot,
 * each pair (a, b) with packed (c, s) becoming (c a + s b, s a - c b) on the
 * rows with U and on the columns with V, layer d first), written in
 * precision prec as rbt_apply_2sided_wp describes (prec = RBT_F64: double
 * output, in place allowed as for rbt_apply_2sided).  Errors: those of
 * rbt_apply_2sided_tiled and rbt_apply_2sided_wp; RBT_ERR_ARG for an
 * unknown kind. */
rbt_status rbt_transform_2sided(int64_t n, int32_t d, int64_t align, int32_t kind, int32_t prec,
                                const double *U, const double *V, int64_t ldw, const double *A_in,
                                int64_t lda_in, void *A_out, int64_t lda_out, cudaStream_t stream);

/* The layer-by-layer form of Algorithm 1 on the GPU: one pass over the
 * matrix per butterfly layer (d passes), in place.  Same result as
 * rbt_apply_2sided up to rounding; kept as the comparison point for the
 * fused kernel's d-fold saving in data movement (Sec. 3). */
rbt_status rbt_apply_2sided_layered(int64_t n, int32_t d, const double *U, const double *V,
                                    int64_t ldw, double *A, int64_t lda, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * rbt_apply_vec -- one-sided transform of an n x nrhs block B (ldb), in
 * place (Eq. precond steps 1 and 3; the adjoint uses the other two):
 *   trans = 1: B <- W^T B   (b~ = U^T b, and V^T g in the adjoint)
 *   trans = 0: B <- W B     (x = V x~,   and U g in the adjoint)
 * W: packed coefficients (n x d, ldw) of U or V.
 */
rbt_status rbt_apply_vec(int64_t n, int32_t d, const double *W, int64_t ldw, int32_t trans,
                         double *B, int64_t ldb, int64_t nrhs, cudaStream_t stream);

/* rbt_apply_vec with the tiled reference size (align as in
 * rbt_apply_2sided_tiled). */
rbt_status rbt_apply_vec_tiled(int64_t n, int32_t d, int64_t align, const double *W, int64_t ldw, int32_t trans,
                               double *B, int64_t ldb, int64_t nrhs, cudaStream_t stream);

/* The general one-sided transform: rbt_apply_vec_tiled for the butterfly
 * kind (RBT_KIND_SCALED or RBT_KIND_ROTATION, coefficients of rbt_generate or
 * rbt_generate_rot).  The rotation layers are symmetric, so W^T applies
 * layers d .. 1 and W layers 1 .. d.  Errors: those of rbt_apply_vec_tiled;
 * RBT_ERR_ARG for an unknown kind. */
rbt_status rbt_transform_vec(int64_t n, int32_t d, int64_t align, int32_t kind, const double *W, int64_t ldw,
                             int32_t trans, double *B, int64_t ldb, int64_t nrhs, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * genp_factor -- in-place LU without pivoting (Sec. 1; the "solve without
 * pivoting" of Eq. precond step 2): A = L U with L unit lower triangular
 * (strictly below the diagonal) and U upper triangular (on and above).
 * A: n x n, lda; element type double for RBT_F64, a float pair for RBT_DF64,
 * RBT_DF64TC and RBT_DF64TC7, float otherwise.
 * d_info: one device int64, set to -1 on success or to the 0-based index of
 * the first pivot that is exactly zero or not finite (elimination stops
 * there; the factor past that column is undefined), or -2 when a bounded
 * device wait of the tensor-core update gave up (TF32 / BF16 / DF64TC /
 * DF64TC7).  Read it after the
 * stream is synchronized: the call itself returns RBT_OK once enqueued.
 * work: device scratch of genp_factor_workspace(n, prec, nb) bytes (may be
 * NULL when that is 0).  nb: block size, 0 = default.
 */
size_t genp_factor_workspace(int64_t n, int32_t prec, int32_t nb);
rbt_status genp_factor(int64_t n, int32_t prec, void *A, int64_t lda, int64_t *d_info,
                       void *work, size_t work_bytes, int32_t nb, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * genp_update -- C <- C - A B, the trailing update of the blocked
 * factorization (all of its flops but O(n^2 nb)), on its own.
 * A: M x K (lda), B: K x N (ldb), C: M x N (ldc), all float, column-major.
 * prec RBT_TF32 / RBT_BF16: operands rounded to TF32 / BF16 and multiplied on
 * the tensor cores (tcgen05.mma, FP32 accumulation in tensor memory, operands
 * staged K-major in `work` and loaded by TMA); RBT_F32: float SIMT kernel;
 * RBT_DF64: A, B, C hold double-float pairs (two floats per element, the
 * leading dimensions count elements), products and sums in double-float
 * arithmetic on the FP32 pipes; RBT_DF64TC (RBT_DF64TC7): double-float
 * pairs as for RBT_DF64, K <= 512, products by exact digit slicing on the
 * BF16 tensor cores with eight (seven) digits per entry.
 * d_status (one device int64) becomes -1, or -2 if a bounded device wait of
 * the tensor-core kernel gave up (then C is undefined).
 * work: genp_update_workspace(M, N, K, prec) bytes (0 for RBT_F32 and RBT_DF64).
 * For the TF32 / BF16 factorizations genp_factor reports the same timeout
 * as d_info = -2.
 */
size_t genp_update_workspace(int64_t M, int64_t N, int64_t K, int32_t prec);
rbt_status genp_update(int32_t prec, int64_t M, int64_t N, int64_t K, const float *A, int64_t lda,
                       const float *B, int64_t ldb, float *C, int64_t ldc, int64_t *d_status,
                       void *work, size_t work_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * genp_solve -- B <- (L U)^{-1} B (trans = 0) or B <- (L U)^{-T} B
 * (trans = 1) with the factors of genp_factor (LU: n x n, lda, element type
 * per prec).  B: double, n x nrhs, ldb.  For float factors the solve runs in
 * float on a float copy of B held in `work` (genp_solve_workspace bytes) and
 * the result is widened back into B; for double-float factors (RBT_DF64,
 * RBT_DF64TC, RBT_DF64TC7) likewise in double-float arithmetic.  The first int of `work` is cleared on
 * entry and is nonzero after a call whose chained triangular solve gave up
 * waiting (B is then undefined; see rbt_debug_wait_limit).
 */
size_t genp_solve_workspace(int64_t n, int64_t nrhs, int32_t prec);
rbt_status genp_solve(int64_t n, int64_t nrhs, int32_t prec, const void *LU, int64_t lda,
                      int32_t trans, double *B, int64_t ldb, void *work, size_t work_bytes,
                      cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * genp_solve_wp -- the same solve, always in double arithmetic: B <- (L U)^{-1}
 * B or (L U)^{-T} B with the factors of genp_factor held in precision prec
 * (float or double-float entries are widened to double as they are read; B
 * stays double throughout).  This is the preconditioner application of
 * GMRES-based refinement (Sec. 5 cites restarted GMRES as the more robust
 * recovery; its preconditioned products are taken in the working precision
 * with the low-precision factors).  LU: n x n, lda, device, not modified.
 * B: device double, n x nrhs, ldb, overwritten.  work: device,
 * genp_solve_wp_workspace(n, nrhs) bytes; its first int is nonzero after a
 * call whose chained triangular solve gave up waiting (B is then undefined).
 * Errors: RBT_ERR_ARG for a bad size, leading dimension or prec;
 * RBT_ERR_WORKSPACE if work is short.
 */
size_t genp_solve_wp_workspace(int64_t n, int64_t nrhs);
rbt_status genp_solve_wp(int64_t n, int64_t nrhs, int32_t prec, const void *LU, int64_t lda,
                         int32_t trans, double *B, int64_t ldb, void *work, size_t work_bytes,
                         cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * rbt_residual -- R <- B - A X in double (the residual of Sec. 5's
 * refinement) and, if d_berr is not NULL, d_berr[0] <- the largest over the
 * columns of Eq. (inf-norm-backerr) ||b - A x|| / (||A|| ||x|| + ||b||).
 * d_anorm: device double holding ||A||_inf, or NULL to have it computed into
 * work.  work: rbt_residual_workspace(n, nrhs) bytes.
 */
size_t rbt_residual_workspace(int64_t n, int64_t nrhs);
rbt_status rbt_residual(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X,
                        int64_t ldx, const double *B, int64_t ldb, double *R, int64_t ldr,
                        const double *d_anorm, double *d_berr, void *work, size_t work_bytes,
                        cudaStream_t stream);

/* rbt_residual_noalloc -- rbt_residual for callers that cannot allocate
 * device memory (no counterpart in the paper: this is an interface need, not
 * part of the method).  Code that runs while someone else captures a CUDA
 * graph, plugins whose host framework owns every allocation, and C callers
 * with no device allocator cannot obtain the workspace rbt_residual asks for;
 * this call takes its scratch from a fixed device array inside the library
 * (rbt_residual_noalloc_max_bytes() bytes, held on every GPU that loads the
 * library until the process exits) and calls no allocator.
 * Arguments and results are those of rbt_residual without work/work_bytes.
 * Limit: rbt_residual_workspace(n, nrhs) must not exceed
 * rbt_residual_noalloc_max_bytes() (about n * ceil(n/1024) * nrhs doubles;
 * n = 40000 with one right-hand side fits); larger requests return
 * RBT_ERR_WORKSPACE before anything is enqueued.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call on a device shares the one array:
 * calls whose executions overlap on the GPU (other streams, or graph replays
 * running concurrently) race and give wrong results; serialize them. */
size_t rbt_residual_noalloc_max_bytes(void);
rbt_status rbt_residual_noalloc(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X,
                                int64_t ldx, const double *B, int64_t ldb, double *R, int64_t ldr,
                                const double *d_anorm, double *d_berr, cudaStream_t stream);

/* d_out[0] <- ||A||_inf (largest absolute row sum) of an n x n A. */
rbt_status rbt_norm_inf(int64_t n, const double *A, int64_t lda, double *d_out, void *work,
                        size_t work_bytes, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * rbt_solve -- the whole method: A~ = U^T A V, GENP of A~ in opts->prec,
 * b~ = U^T B, triangular solves, X = V x~ (Eq. precond), then iterative
 * refinement on the original A in double (Sec. 5) until the backward error
 * (Eq. inf-norm-backerr) is <= opts->tol or opts->refine_max steps were
 * taken.  With opts->fallback set, a low-precision refinement that stalls
 * (a step that lowers the backward error by less than 10%) refactors the
 * same A~ in double and refines again ("responsibly reckless" fallback of
 * Sec. 5); for RBT_DF64TC7 the first refactorization uses eight digits
 * (RBT_DF64TC) and only a stall of that one goes on to double.
 * A (n x n, lda) and B (n x nrhs, ldb) are not modified; X (n x nrhs, ldx)
 * receives the solution.  work: rbt_solve_workspace(opts, n, nrhs) bytes.
 * info (host) is written before return.  Returns RBT_OK, RBT_ZERO_PIVOT,
 * RBT_NONFINITE, RBT_NOT_CONVERGED or an error (RBT_ERR_TIMEOUT when any
 * bounded device wait of the call gave up).
 */
size_t rbt_solve_workspace(const rbt_opts *opts, int64_t n, int64_t nrhs);
rbt_status rbt_solve(const rbt_opts *opts, int64_t n, int64_t nrhs, const double *A, int64_t lda,
                     const double *B, int64_t ldb, double *X, int64_t ldx, void *work,
                     size_t work_bytes, rbt_info *info, cudaStream_t stream);

/* rbt_solve_host -- rbt_solve (Eq. precond with the refinement of Sec. 5)
 * with A, B and X in host memory (the end-to-end form: no device copy of the
 * inputs needed).  A (n x n, lda) and B
 * (n x nrhs, ldb) are read into device scratch at the front of `work`, the
 * solve runs as rbt_solve, and X (n x nrhs, ldx) is written back; the call
 * synchronizes `stream` before it returns.  Pinned or registered host memory
 * is read by SM loads of its device mapping (on GB300 these held the host
 * link's rate where the copy engines varied several-fold from call to call);
 * other host memory goes through cudaMemcpy2DAsync.  work (device):
 * rbt_solve_host_workspace(opts, n, nrhs) bytes, 0 for invalid options.
 * Returns what rbt_solve returns; X is not written after a negative status
 * and is undefined after RBT_ZERO_PIVOT / RBT_NONFINITE. */
size_t rbt_solve_host_workspace(const rbt_opts *opts, int64_t n, int64_t nrhs);
rbt_status rbt_solve_host(const rbt_opts *opts, int64_t n, int64_t nrhs, const double *A, int64_t lda,
                          const double *B, int64_t ldb, double *X, int64_t ldx, void *work, size_t work_bytes,
                          rbt_info *info, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Adjoint of X = A^{-1} B (reverse-mode differentiation).  With
 * A^{-1} = V A~^{-1} U^T (Eq. precond):
 *   grad_B = A^{-T} grad_X = U A~^{-T} V^T grad_X,   grad_A = -grad_B X^T.
 * rbt_solve_adjoint solves A^T Y = G (n x nrhs, ldg) into Y (ldy) with the
 * factors, U and V that a successful rbt_solve with the same opts, n and
 * A left in `work` (its contents after rbt_solve returned must be intact);
 * fwd is that call's info (its fell_back flag selects the fallback's factors).
 * Transposed triangular solves, then refinement in double against A^T until
 * opts->tol or opts->refine_max steps.  Same status conventions as rbt_solve.
 * nrhs may differ from the forward call's; work_bytes must cover
 * rbt_solve_workspace(opts, n, nrhs) (the factors sit before everything that
 * depends on nrhs).
 * rbt_outer: C (n x m, ldc) <- alpha * Y (n x k, ldy) * X^T (X: m x k, ldx),
 * in double (the rank-nrhs grad_A).
 */
rbt_status rbt_solve_adjoint(const rbt_opts *opts, const rbt_info *fwd, int64_t n, int64_t nrhs,
                             const double *A, int64_t lda, const double *G, int64_t ldg, double *Y,
                             int64_t ldy, void *work, size_t work_bytes, rbt_info *info,
                             cudaStream_t stream);
rbt_status rbt_outer(int64_t n, int64_t m, int64_t k, double alpha, const double *Y, int64_t ldy,
                     const double *X, int64_t ldx, double *C, int64_t ldc, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Batched solves: thousands of independent systems of uneven order, each with
 * its own butterflies (seed seeds[i], or opts->seed + i when seeds is NULL),
 * in ONE persistent kernel: each CTA takes the next system from a device work
 * queue (largest first) and runs Eq. precond with refinement (Sec. 5) on it:
 * coefficients, fused transform, blocked GENP, solves, double residual and
 * backward error, refinement until opts->tol, opts->refine_max steps, or a
 * step that gains less than 10% (stationary steps only: refine_mode must be
 * RBT_REFINE_STATIONARY).  opts->prec: RBT_F64 or RBT_F32 (float
 * factors refined in double); with opts->fallback a float system whose
 * refinement misses tol (or whose float GENP meets a bad pivot) is redone
 * inside the same launch, on the same A~ (Sec. 5's fallback): in
 * double-float (pairs of floats, about 48 bits, on the FP32 pipes) and, if
 * that misses too, in double;
 * min(d, ceil(log2 n_i)) <= 3.
 *
 *  rbt_solve_batched_workspace  bytes of `work` for this batch.
 *  rbt_solve_batched_plan       host call: validates, lays out per-system
 *                               scratch, copies the descriptor table into
 *                               `work` and synchronizes `stream`.  Host
 *                               arrays: n, nrhs (NULL = all 1), A, lda, B, ldb,
 *                               X, ldx (device pointers in host arrays), seeds.
 *  rbt_solve_batched_run        device-only: a memset of the queue counter and
 *                               one kernel on `stream` (float with fallback: a
 *                               second memset and kernel, the double redo of
 *                               the systems still unsolved); may be captured in a
 *                               CUDA graph and replayed (plan first).
 *  rbt_solve_batched_autotune   times every compiled variant (threads per CTA
 *                               x GENP block size) on the planned batch (runs
 *                               the batch 8 times) and keeps the fastest for
 *                               batches with the same size histogram on this
 *                               device; later runs use it.
 *  rbt_solve_batched_variant    the variant runs will use (-1 if not planned).
 * d_infos: device array of `batch` rbt_batched_info, written by the run.
 * A and B are not modified; X (n_i x nrhs_i) receives the solution.
 */
typedef struct {
    int32_t status;          /* rbt_status of this system */
    int32_t iters;           /* refinement steps (all attempts) */
    int32_t fell_back;       /* float systems: 1 if refactored in double-float,
                                2 if then also in double (X from the last) */
    int32_t reserved;
    int64_t zero_pivot;      /* -1 or the first bad pivot */
    double berr_unrefined;   /* of the last attempt */
    double berr;
} rbt_batched_info;

size_t rbt_solve_batched_workspace(const rbt_opts *opts, int64_t batch, const int64_t *n,
                                   const int64_t *nrhs);
rbt_status rbt_solve_batched_plan(const rbt_opts *opts, int64_t batch, const int64_t *n,
                                  const int64_t *nrhs, const double *const *A, const int64_t *lda,
                                  const double *const *B, const int64_t *ldb, double *const *X,
                                  const int64_t *ldx, const uint64_t *seeds, void *work,
                                  size_t work_bytes, cudaStream_t stream);
rbt_status rbt_solve_batched_run(const rbt_opts *opts, void *work, rbt_batched_info *d_infos,
                                 cudaStream_t stream);
rbt_status rbt_solve_batched_autotune(const rbt_opts *opts, void *work, rbt_batched_info *d_infos,
                                      cudaStream_t stream, int32_t *chosen, double *best_ms);
int32_t rbt_solve_batched_variant(void *work, int32_t *threads, int32_t *nb);

/* Batched adjoint after a batched run on the same plan (`work` untouched
 * since): per system, Y_i = A_i^{-T} G_i (G_i, Y_i: n_i x nrhs_i; refined in
 * double against A_i^T) and, when GA and GA[i] are not NULL,
 * GA_i = -Y_i X_i^T (n_i x n_i).  One persistent launch; d_infos receives the
 * adjoint solves' outcomes (read by the kernel first: systems whose forward
 * status was a pivot failure are skipped).  Synchronizes `stream`. */
rbt_status rbt_solve_batched_adjoint(const rbt_opts *opts, void *work, int64_t batch, const double *const *G,
                                     const int64_t *ldg, double *const *Y, const int64_t *ldy,
                                     double *const *GA, const int64_t *ldga, rbt_batched_info *d_infos,
                                     cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper).
 * rbt_kernel_launches: number of CUDA kernels this library has launched in
 * this process so far (host counter; monotone).
 */
uint64_t rbt_kernel_launches(void);

/* Per-phase device time.  While enabled, the library records a pair of CUDA
 * events around every launch of a phase class on the launching stream:
 *   0 = GENP trailing update, 1 = two-sided transform, 2 = GENP diagonal
 *   factor and TRSMs, 3 = triangular solves, 4 = residual and norms,
 *   5 = digit slicing and balancing exponents of the sliced update (RBT_DF64TC
 *   and RBT_DF64TC7; class 0 then holds the tensor-core kernel alone).
 * rbt_prof_read synchronizes on the recorded events and returns the summed
 * milliseconds and the number of timed launches of class cls since the last
 * reset.  Off by default; the events add a few microseconds per launch. */
void rbt_prof_enable(int32_t on);
void rbt_prof_reset(void);
rbt_status rbt_prof_read(int32_t cls, double *ms, int64_t *launches);

/* ---------------------------------------------------------------------------
 * Bounded device waits and their test hooks (no counterpart in the paper).
 * Every spin-wait in the library's kernels (the chained triangular solves
 * waiting for earlier row blocks; the sliced tensor-core update waiting for
 * its TMA copies and tensor-core operations) gives up after a time limit,
 * records a timeout and lets the kernel end, so that a lost dependency never
 * hangs the GPU.  A timeout is reported as RBT_ERR_TIMEOUT by rbt_solve and
 * rbt_solve_adjoint (sticky over the whole call), as d_info = -2 by
 * genp_factor, as d_status = -2 by genp_update, and as a nonzero first int
 * of the work buffer after genp_solve / genp_solve_wp; results are then
 * undefined.
 * rbt_debug_wait_limit: the limit in nanoseconds for kernels launched from
 * now on (ns <= 0 restores the default, one second); returns the previous
 * limit.  Process-wide.
 * rbt_debug_stall: make one kind of wait run out on purpose, to test the
 * timeout paths without any fault: RBT_STALL_CHAIN starts the chained
 * solves' block queue at block 1, so that block 0 is never solved and the
 * first wait for it runs out (the other waits then stop at once);
 * RBT_STALL_OZ_COPY keeps the sliced update's copy warp from issuing any
 * copy, so that the tensor-core warp's first wait runs out (no copy is ever
 * in flight, and the tensor memory is freed as usual).  Returns the previous
 * setting.  Process-wide; RBT_STALL_NONE (the default) for normal use.
 */
enum { RBT_STALL_NONE = 0, RBT_STALL_CHAIN = 1, RBT_STALL_OZ_COPY = 2 };
int64_t rbt_debug_wait_limit(int64_t ns);
int32_t rbt_debug_stall(int32_t which);

/* rbt_debug_oz_products -- the raw accumulators of the sliced tensor-core
 * update (RBT_DF64TC) for caller-given digits (testing; no counterpart in the
 * paper).  The slicing of the update is exact only if the FP32 tensor-core
 * accumulation of integer digit products is exact while the sums stay within
 * 2^24; this call runs the update kernel's own copy and tensor-core pipeline
 * on given digits so that a test can check exactly that.
 * da: device int8, the 8 digit matrices of an M x K operand A, digit p
 * (0-based) of A(m, k) at da[(p M + m) K + k]; db: the same for the N x K
 * transposed operand (digit q of B(k, n) at db[(q N + n) K + k]).  K <= 512.
 * acc: device float, 8 x M x N: acc[(t M + m) N + n] = sum over p + q = t
 * (t = 0 .. 7) and k of a_p(m, k) b_q(n, k), as the kernel accumulated it
 * (products with p + q > 7 are dropped, as in the update).  work:
 * rbt_debug_oz_products_workspace(M, N, K) bytes.  Errors: RBT_ERR_ARG,
 * RBT_ERR_UNSUPPORTED for K > 512, RBT_ERR_WORKSPACE.
 */
size_t rbt_debug_oz_products_workspace(int64_t M, int64_t N, int64_t K);
rbt_status rbt_debug_oz_products(int64_t M, int64_t N, int64_t K, const int8_t *da, const int8_t *db, float *acc,
                                 void *work, size_t work_bytes, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif
