// Vector kernels of the GMRES-based refinement (classical Gram-Schmidt
// applied twice, in double): dot products of a vector against the columns of
// a basis, the basis-vector products Q h, scaling and accumulation.  The
// Arnoldi recurrence, the Givens rotations and the small triangular solve
// run on the host in the refinement driver.
#include "common.cuh"
#include "genp_internal.cuh"

namespace rbt {

constexpr int kGmRows = 1024;  // rows per CTA of the dot products (256 threads x 4)

// part[i * nblk + blockIdx.x] = sum over this CTA's rows of Q[:, i] . w, i < k
__global__ void __launch_bounds__(256) gm_dots_partial_kernel(int64_t n, const double *__restrict__ Q, int64_t ldq,
                                                              int k, const double *__restrict__ w,
                                                              double *__restrict__ part, int64_t nblk)
{
    __shared__ double red[256];
    const int64_t r0 = (int64_t)blockIdx.x * kGmRows;
    for (int i = 0; i < k; i++) {
        double s = 0.0;
        for (int64_t r = r0 + threadIdx.x; r < n && r < r0 + kGmRows; r += 256) s = fma(Q[r + i * ldq], w[r], s);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[i * nblk + blockIdx.x] = red[0];
        __syncthreads();
    }
}

// out[i] = sum_b part[i * nblk + b]; one CTA per i
__global__ void __launch_bounds__(256) gm_dots_reduce_kernel(const double *__restrict__ part, int64_t nblk,
                                                             double *__restrict__ out)
{
    __shared__ double red[256];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nblk; b += 256) s += part[i * nblk + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = red[0];
}

// w -= Q h (k columns)
__global__ void gm_sub_kernel(int64_t n, const double *__restrict__ Q, int64_t ldq, int k, const double *__restrict__ h,
                              double *__restrict__ w)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double s = w[r];
    for (int i = 0; i < k; i++) s = fma(-Q[r + i * ldq], h[i], s);
    w[r] = s;
}

// z = Q y (k columns)
__global__ void gm_gemv_kernel(int64_t n, const double *__restrict__ Q, int64_t ldq, int k,
                               const double *__restrict__ y, double *__restrict__ z)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double s = 0.0;
    for (int i = 0; i < k; i++) s = fma(Q[r + i * ldq], y[i], s);
    z[r] = s;
}

__global__ void gm_scale_kernel(int64_t n, double alpha, const double *__restrict__ src, double *__restrict__ dst)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) dst[r] = alpha * src[r];
}

__global__ void gm_add_kernel(int64_t n, const double *__restrict__ z, double *__restrict__ x)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) x[r] += z[r];
}

int64_t gm_part_len(int64_t n) { return cdiv(n > 0 ? n : 1, kGmRows); }

rbt_status gm_dots(int64_t n, const double *Q, int64_t ldq, int k, const double *w, double *part, double *out,
                   cudaStream_t s)
{
    const int64_t nblk = gm_part_len(n);
    gm_dots_partial_kernel<<<(unsigned)nblk, 256, 0, s>>>(n, Q, ldq, k, w, part, nblk);
    RBT_LAUNCH_CHECK();
    gm_dots_reduce_kernel<<<(unsigned)k, 256, 0, s>>>(part, nblk, out);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

rbt_status gm_sub(int64_t n, const double *Q, int64_t ldq, int k, const double *h, double *w, cudaStream_t s)
{
    gm_sub_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(n, Q, ldq, k, h, w);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

rbt_status gm_gemv(int64_t n, const double *Q, int64_t ldq, int k, const double *y, double *z, cudaStream_t s)
{
    gm_gemv_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(n, Q, ldq, k, y, z);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

rbt_status gm_scale(int64_t n, double alpha, const double *src, double *dst, cudaStream_t s)
{
    gm_scale_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(n, alpha, src, dst);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

rbt_status gm_add(int64_t n, const double *z, double *x, cudaStream_t s)
{
    gm_add_kernel<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(n, z, x);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

}  // namespace rbt
