// Residual r = b - A x in double and the infinity-norm backward error of
// Eq. (inf-norm-backerr) (sm_103a).
//
// The matrix-vector product is split over column chunks so that a 40000 x
// 40000 matrix gives tens of thousands of CTAs; each chunk writes a partial
// sum per row into the workspace and a second kernel adds the partials in a
// fixed order (deterministic result).  Consecutive threads take consecutive
// rows, so every column of A is read coalesced, once per group of eight
// right-hand sides.
#include "common.cuh"
#include "genp_internal.cuh"

namespace rbt {

constexpr int kResRows = 128;
constexpr int kResChunk = 1024;
constexpr int kResRhs = 8;

static inline int64_t res_chunks(int64_t n) { return cdiv(n, kResChunk); }

__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || isnan(b)) ? b : a; }

// Non-negative doubles order like their bit patterns (NaN above +Inf).
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v)
{
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// partial[ch][c][r] = sum over the columns of chunk ch of A[r, j] X[j, c]
// (abs_mode: sum of |A[r, j]|, one column).
__global__ void __launch_bounds__(kResRows)
matvec_partial_kernel(int64_t n, int64_t nrhs, const double *__restrict__ A, int64_t lda,
                      const double *__restrict__ X, int64_t ldx, double *__restrict__ part, int abs_mode)
{
    __shared__ double xs[kResChunk * kResRhs];
    const int64_t r = (int64_t)blockIdx.x * kResRows + threadIdx.x;
    const int64_t ch = blockIdx.y;
    const int64_t j0 = ch * kResChunk;
    const int jn = (int)(n - j0 < kResChunk ? n - j0 : kResChunk);
    const int64_t ncol = abs_mode ? 1 : nrhs;
    for (int64_t c0 = 0; c0 < ncol; c0 += kResRhs) {
        const int nc = (int)(ncol - c0 < kResRhs ? ncol - c0 : kResRhs);
        if (!abs_mode) {
            __syncthreads();
            for (int e = threadIdx.x; e < jn * nc; e += kResRows) {
                int j = e % jn, c = e / jn;
                xs[c * kResChunk + j] = X[(j0 + j) + (c0 + c) * ldx];
            }
            __syncthreads();
        }
        if (r >= n) continue;
        double acc[kResRhs];
#pragma unroll
        for (int c = 0; c < kResRhs; c++) acc[c] = 0.0;
        const double *a = A + r + j0 * lda;
        if (abs_mode) {
            for (int j = 0; j < jn; j++) acc[0] += fabs(a[j * lda]);
        } else if (nc == 1) {
            for (int j = 0; j < jn; j++) acc[0] = fma(a[j * lda], xs[j], acc[0]);
        } else {
            for (int j = 0; j < jn; j++) {
                double v = a[j * lda];
#pragma unroll
                for (int c = 0; c < kResRhs; c++)
                    if (c < nc) acc[c] = fma(v, xs[c * kResChunk + j], acc[c]);
            }
        }
        for (int c = 0; c < nc; c++) part[(ch * ncol + c0 + c) * n + r] = acc[c];
    }
}

// R[r, c] = B[r, c] - sum_ch partial[ch][c][r]
__global__ void residual_reduce_kernel(int64_t n, int64_t nrhs, int64_t nch, const double *__restrict__ part,
                                       const double *__restrict__ B, int64_t ldb, double *R, int64_t ldr)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t r = idx % n, c = idx / n;
    double s = 0.0;
    for (int64_t ch = 0; ch < nch; ch++) s += part[(ch * nrhs + c) * n + r];
    R[r + c * ldr] = B[r + c * ldb] - s;
}

// out = max_r sum_ch partial[ch][0][r]  (out zeroed beforehand)
__global__ void rowsum_max_kernel(int64_t n, int64_t nch, const double *__restrict__ part, double *out)
{
    __shared__ double red[256];
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double s = 0.0;
    if (r < n)
        for (int64_t ch = 0; ch < nch; ch++) s += part[ch * n + r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = nan_max(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomic_max_nonneg(out, red[0]);
}

// berr = max_c ||r_c|| / (||A|| ||x_c|| + ||b_c||); one CTA per column.
__global__ void berr_kernel(int64_t n, const double *R, int64_t ldr, const double *X, int64_t ldx,
                            const double *B, int64_t ldb, const double *anorm, double *berr)
{
    __shared__ double sr[256], sx[256], sb[256];
    const int64_t c = blockIdx.x;
    double mr = 0.0, mx = 0.0, mb = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        mr = nan_max(mr, fabs(R[i + c * ldr]));
        mx = nan_max(mx, fabs(X[i + c * ldx]));
        mb = nan_max(mb, fabs(B[i + c * ldb]));
    }
    sr[threadIdx.x] = mr;
    sx[threadIdx.x] = mx;
    sb[threadIdx.x] = mb;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sr[threadIdx.x] = nan_max(sr[threadIdx.x], sr[threadIdx.x + o]);
            sx[threadIdx.x] = nan_max(sx[threadIdx.x], sx[threadIdx.x + o]);
            sb[threadIdx.x] = nan_max(sb[threadIdx.x], sb[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double den = (*anorm) * sx[0] + sb[0];
        double e = den > 0.0 ? sr[0] / den : (sr[0] > 0.0 ? INFINITY : 0.0);
        if (isnan(sr[0]) || isnan(den)) e = NAN;
        atomic_max_nonneg(berr, e);
    }
}

__global__ void axpy_kernel(int64_t n, int64_t nrhs, const double *D, int64_t ldd, double *X, int64_t ldx)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t i = idx % n, c = idx / n;
    X[i + c * ldx] += D[i + c * ldd];
}

rbt_status add_block(int64_t n, int64_t nrhs, const double *D, int64_t ldd, double *X, int64_t ldx,
                     cudaStream_t stream)
{
    if (n * nrhs == 0) return RBT_OK;
    axpy_kernel<<<(unsigned)cdiv(n * nrhs, 256), 256, 0, stream>>>(n, nrhs, D, ldd, X, ldx);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

size_t residual_part_bytes(int64_t n, int64_t nrhs)
{
    if (n <= 0) return 0;
    int64_t cols = nrhs > 1 ? nrhs : 1;
    return (size_t)res_chunks(n) * (size_t)n * (size_t)cols * sizeof(double);
}

size_t residual_ws(int64_t n, int64_t nrhs)
{
    if (n <= 0) return 0;
    int64_t cols = nrhs > 1 ? nrhs : 1;
    return (size_t)res_chunks(n) * (size_t)n * (size_t)cols * sizeof(double) + 2 * sizeof(double) + 256;
}

rbt_status norm_inf_impl(int64_t n, const double *A, int64_t lda, double *d_out, double *part,
                         cudaStream_t stream)
{
    ProfScope ps(kProfResidual, stream);
    RBT_CUDA_TRY(cudaMemsetAsync(d_out, 0, sizeof(double), stream));
    if (n == 0) return RBT_OK;
    int64_t nch = res_chunks(n);
    dim3 grid((unsigned)cdiv(n, kResRows), (unsigned)nch);
    matvec_partial_kernel<<<grid, kResRows, 0, stream>>>(n, 1, A, lda, nullptr, 1, part, 1);
    RBT_LAUNCH_CHECK();
    rowsum_max_kernel<<<(unsigned)cdiv(n, 256), 256, 0, stream>>>(n, nch, part, d_out);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

rbt_status residual_impl(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X, int64_t ldx,
                         const double *B, int64_t ldb, double *R, int64_t ldr, const double *d_anorm,
                         double *d_berr, double *part, cudaStream_t stream)
{
    ProfScope ps(kProfResidual, stream);
    if (n == 0 || nrhs == 0) {
        if (d_berr) RBT_CUDA_TRY(cudaMemsetAsync(d_berr, 0, sizeof(double), stream));
        return RBT_OK;
    }
    int64_t nch = res_chunks(n);
    dim3 grid((unsigned)cdiv(n, kResRows), (unsigned)nch);
    matvec_partial_kernel<<<grid, kResRows, 0, stream>>>(n, nrhs, A, lda, X, ldx, part, 0);
    RBT_LAUNCH_CHECK();
    residual_reduce_kernel<<<(unsigned)cdiv(n * nrhs, 256), 256, 0, stream>>>(n, nrhs, nch, part, B, ldb, R, ldr);
    RBT_LAUNCH_CHECK();
    if (d_berr) {
        RBT_CUDA_TRY(cudaMemsetAsync(d_berr, 0, sizeof(double), stream));
        berr_kernel<<<(unsigned)nrhs, 256, 0, stream>>>(n, R, ldr, X, ldx, B, ldb, d_anorm, d_berr);
        RBT_LAUNCH_CHECK();
    }
    return RBT_OK;
}

}  // namespace rbt

using namespace rbt;

extern "C" {

size_t rbt_residual_workspace(int64_t n, int64_t nrhs) { return residual_ws(n, nrhs); }

rbt_status rbt_residual(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X, int64_t ldx,
                        const double *B, int64_t ldb, double *R, int64_t ldr, const double *d_anorm,
                        double *d_berr, void *work, size_t work_bytes, cudaStream_t stream)
{
    int64_t mn = n > 1 ? n : 1;
    if (n < 0 || nrhs < 0 || lda < mn || ldx < mn || ldb < mn || ldr < mn) return RBT_ERR_ARG;
    if (n > 0 && nrhs > 0 && (!A || !X || !B || !R)) return RBT_ERR_ARG;
    if (work_bytes < residual_ws(n, nrhs)) return RBT_ERR_WORKSPACE;
    if (n > 0 && !work) return RBT_ERR_WORKSPACE;
    double *part = (double *)work;
    double *own_norm = (double *)((char *)work + (work_bytes - 2 * sizeof(double)) / 8 * 8);
    if (n > 0 && nrhs > 0 && d_berr && !d_anorm) {
        rbt_status st = norm_inf_impl(n, A, lda, own_norm, part, stream);
        if (st != RBT_OK) return st;
        d_anorm = own_norm;
    }
    return residual_impl(n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, d_anorm, d_berr, part, stream);
}

rbt_status rbt_norm_inf(int64_t n, const double *A, int64_t lda, double *d_out, void *work, size_t work_bytes,
                        cudaStream_t stream)
{
    if (n < 0 || lda < (n > 1 ? n : 1) || !d_out) return RBT_ERR_ARG;
    if (n > 0 && !A) return RBT_ERR_ARG;
    if (work_bytes < residual_ws(n, 1) || (n > 0 && !work)) return RBT_ERR_WORKSPACE;
    return norm_inf_impl(n, A, lda, d_out, (double *)work, stream);
}

}  // extern "C"
