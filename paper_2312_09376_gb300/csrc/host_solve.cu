// rbt_solve with host buffers (sm_103a): A and B are read from host memory
// into device scratch, the solve runs as rbt_solve, and X is written back.
//
// The host-to-device copies of pinned (or registered) host memory are done by
// SM loads of the memory's device mapping over the host link, not by the copy
// engines: on GB300 hosts the copy engine's 12.8 GB transfer of an n = 40003
// matrix was measured anywhere between 61 and 730 ms from one call to the
// next, while SM loads of the same buffer held about 210 GB/s (61 ms), the
// link's rate.  Host memory without a device mapping (pageable memory) goes
// through cudaMemcpy2DAsync instead.
#include "common.cuh"

namespace rbt {

// dst (m x k, ldd) <- src (m x k, lds), doubles, column-major; consecutive
// threads take consecutive rows of a column (coalesced on both sides).
__global__ void copy2d_kernel(const double *__restrict__ src, int64_t lds, double *__restrict__ dst, int64_t ldd,
                              int64_t m, int64_t k)
{
    const int64_t total = m * k;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t i = e % m, j = e / m;
        dst[i + j * ldd] = src[i + j * lds];
    }
}

// A contiguous run of 16-byte words (both ends 16-byte aligned).
__global__ void copy16_kernel(const uint4 *__restrict__ src, uint4 *__restrict__ dst, int64_t n16)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n16; e += stride) dst[e] = src[e];
}

// The device address of a host pointer, or nullptr when it has none (pageable
// memory).
static const double *device_view(const double *host)
{
    void *p = nullptr;
    if (cudaHostGetDevicePointer(&p, const_cast<double *>(host), 0) != cudaSuccess) {
        (void)cudaGetLastError();  // not mapped: not an error of the call
        return nullptr;
    }
    return (const double *)p;
}

// Device dst (m x k, ldd) <- host src (m x k, lds).
static rbt_status host_to_device(const double *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int64_t k,
                                 cudaStream_t stream)
{
    if (m <= 0 || k <= 0) return RBT_OK;
    const double *mapped = device_view(src);
    if (!mapped) {
        RBT_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)ldd * 8, src, (size_t)lds * 8, (size_t)m * 8, (size_t)k,
                                       cudaMemcpyHostToDevice, stream));
        return RBT_OK;
    }
    const unsigned grid = (unsigned)device_sm_count() * 4;
    const int64_t bytes = m * k * 8;
    if (lds == m && ldd == m && (uintptr_t)mapped % 16 == 0 && (uintptr_t)dst % 16 == 0 && bytes % 16 == 0) {
        copy16_kernel<<<grid, 512, 0, stream>>>((const uint4 *)mapped, (uint4 *)dst, bytes / 16);
    } else {
        copy2d_kernel<<<grid, 512, 0, stream>>>(mapped, lds, dst, ldd, m, k);
    }
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

static inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace rbt

using namespace rbt;

extern "C" {

size_t rbt_solve_host_workspace(const rbt_opts *opts, int64_t n, int64_t nrhs)
{
    if (n < 0 || nrhs < 0) return 0;
    const size_t ws = rbt_solve_workspace(opts, n, nrhs);
    if (ws == 0 && n > 0) return 0;  // invalid options
    const size_t nn = (size_t)(n > 0 ? n : 1), nr = (size_t)(nrhs > 0 ? nrhs : 1);
    return up256(nn * nn * 8) + 2 * up256(nn * nr * 8) + ws;
}

rbt_status rbt_solve_host(const rbt_opts *opts, int64_t n, int64_t nrhs, const double *A, int64_t lda,
                          const double *B, int64_t ldb, double *X, int64_t ldx, void *work, size_t work_bytes,
                          rbt_info *info, cudaStream_t stream)
{
    if (info) {
        info->status = RBT_ERR_ARG;
        info->zero_pivot = -1;
        info->iters = 0;
        info->fell_back = 0;
        info->berr_unrefined = NAN;
        info->berr = NAN;
    }
    const int64_t mn = n > 1 ? n : 1;
    if (!opts || !info || n < 0 || nrhs < 0 || lda < mn || ldb < mn || ldx < mn) return RBT_ERR_ARG;
    if (n == 0 || nrhs == 0) return rbt_solve(opts, n, nrhs, A, lda, B, ldb, X, ldx, work, work_bytes, info, stream);
    if (!A || !B || !X || !work) return RBT_ERR_ARG;
    const size_t need = rbt_solve_host_workspace(opts, n, nrhs);
    if (need == 0) return RBT_ERR_ARG;
    if (work_bytes < need) return RBT_ERR_WORKSPACE;
    char *w = (char *)work;
    double *Ad = (double *)w;
    w += up256((size_t)n * n * 8);
    double *Bd = (double *)w;
    w += up256((size_t)n * nrhs * 8);
    double *Xd = (double *)w;
    w += up256((size_t)n * nrhs * 8);
    const size_t rest = work_bytes - (size_t)(w - (char *)work);
    // once a copy of the caller's host memory is enqueued, every return waits
    // for the stream: the caller may release that memory when the call ends
    auto finish = [&](rbt_status st) -> rbt_status {
        const cudaError_t e = cudaStreamSynchronize(stream);
        return (st == RBT_OK && e != cudaSuccess) ? RBT_ERR_CUDA : st;
    };
    rbt_status st = host_to_device(A, lda, Ad, n, n, n, stream);
    if (st == RBT_OK) st = host_to_device(B, ldb, Bd, n, n, nrhs, stream);
    if (st != RBT_OK) return finish(st);
    st = rbt_solve(opts, n, nrhs, Ad, n, Bd, n, Xd, n, w, rest, info, stream);
    if (st < 0) return finish(st);  // argument or CUDA error: X is not written
    if (cudaMemcpy2DAsync(X, (size_t)ldx * 8, Xd, (size_t)n * 8, (size_t)n * 8, (size_t)nrhs,
                          cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return finish(RBT_ERR_CUDA);
    const rbt_status done = finish(RBT_OK);
    return done != RBT_OK ? done : st;
}

}  // extern "C"
