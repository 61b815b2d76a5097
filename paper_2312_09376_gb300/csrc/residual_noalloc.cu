// rbt_residual_noalloc: the residual and backward-error check of
// rbt_residual, for callers that cannot allocate device memory.
//
// Some callers have no way to hand this library a workspace: code running
// while a CUDA graph is being captured by someone else, callbacks and plugins
// of host frameworks that own the allocator, or C callers built without any
// device allocator at all.  cudaMalloc there is either forbidden (it is not a
// stream-ordered call and breaks capture) or unavailable.  This entry point
// takes its scratch from a fixed array in device memory instead, so it
// allocates nothing.
//
// The array below is a file-scope __device__ variable: every GPU on which the
// library is loaded holds it (kNoallocScratchBytes) until the process exits.
// In host code its name is only a host-side stand-in, so the device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device.
#include <mutex>

#include "common.cuh"
#include "genp_internal.cuh"

namespace rbt {

constexpr size_t kNoallocScratchBytes = ((size_t)16 << 20) + 4096;  // 16 MiB of partial sums + slack
// Layout: the norm accumulator in the first 256 bytes, the partial sums after
// them.  Both are checked against the array's size on every call.
constexpr size_t kNoallocNormBytes = 256;
static_assert(kNoallocScratchBytes % 256 == 0 && kNoallocScratchBytes > 2 * kNoallocNormBytes,
              "the norm slot and the partial sums must both fit, 256-byte aligned");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kMaxDevices];

// Device address of g_noalloc_scratch on the current device (set-up on first use).
static rbt_status noalloc_scratch(void **out)
{
    int dev = 0;
    RBT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return RBT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return RBT_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return RBT_OK;
}

}  // namespace rbt

using namespace rbt;

extern "C" {

size_t rbt_residual_noalloc_max_bytes(void) { return kNoallocScratchBytes; }

rbt_status rbt_residual_noalloc(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X, int64_t ldx,
                                const double *B, int64_t ldb, double *R, int64_t ldr, const double *d_anorm,
                                double *d_berr, cudaStream_t stream)
{
    int64_t mn = n > 1 ? n : 1;
    if (n < 0 || nrhs < 0 || lda < mn || ldx < mn || ldb < mn || ldr < mn) return RBT_ERR_ARG;
    if (n > 0 && nrhs > 0 && (!A || !X || !B || !R)) return RBT_ERR_ARG;
    // partial sums (as in rbt_residual's workspace) plus one double for ||A||
    const size_t need = residual_ws(n, nrhs);
    if (need > kNoallocScratchBytes) return RBT_ERR_WORKSPACE;  // beyond the fixed scratch array
    // the partial sums start after the norm slot; they must end inside the array
    if (kNoallocNormBytes + residual_part_bytes(n, nrhs) > kNoallocScratchBytes) return RBT_ERR_WORKSPACE;
    if (n == 0 || nrhs == 0) {
        if (d_berr) RBT_CUDA_TRY(cudaMemsetAsync(d_berr, 0, sizeof(double), stream));
        return RBT_OK;
    }
    void *scratch = nullptr;
    rbt_status st = noalloc_scratch(&scratch);
    if (st != RBT_OK) return st;
    // the norm accumulator first (norm_inf_impl zeroes it), the partial sums after it
    double *own_norm = (double *)scratch;
    double *part = (double *)((char *)scratch + kNoallocNormBytes);
    if (d_berr && !d_anorm) {
        st = norm_inf_impl(n, A, lda, own_norm, part, stream);
        if (st != RBT_OK) return st;
        d_anorm = own_norm;
    }
    return residual_impl(n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, d_anorm, d_berr, part, stream);
}

}  // extern "C"
