// Adjoint of X = A^{-1} B for reverse-mode differentiation (sm_103a).
//
// With A^{-1} = V A~^{-1} U^T (Eq. precond), the cotangent of B is
//     grad_B = A^{-T} grad_X = U A~^{-T} V^T grad_X,
// solved with the factors of A~ that the forward rbt_solve left in its
// workspace (transposed triangular solves, no refactorization), refined in
// double against A^T, and the cotangent of A is the rank-nrhs product
//     grad_A = -grad_B X^T.
#include <cmath>

#include "common.cuh"
#include "genp_internal.cuh"

namespace rbt {

constexpr int kAdjWarps = 8;
constexpr int kAdjRhs = 8;

// R[:, c] = G[:, c] - A^T Y[:, c]; one warp per row of the result (a column
// of A, read contiguously); also the largest absolute column sum of A
// (= ||A^T||_inf) into colmax when want_norm.
__global__ void __launch_bounds__(32 * kAdjWarps)
resid_t_kernel(int64_t n, int64_t nrhs, const double *__restrict__ A, int64_t lda, const double *__restrict__ Y,
               int64_t ldy, const double *__restrict__ G, int64_t ldg, double *R, int64_t ldr, double *colmax,
               int want_norm)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * kAdjWarps + threadIdx.x / 32;
    if (j >= n) return;
    const double *a = A + j * lda;
    double asum = 0.0;
    for (int64_t c0 = 0; c0 < nrhs; c0 += kAdjRhs) {
        const int nc = (int)(nrhs - c0 < kAdjRhs ? nrhs - c0 : kAdjRhs);
        double acc[kAdjRhs];
#pragma unroll
        for (int c = 0; c < kAdjRhs; c++) acc[c] = 0.0;
        for (int64_t i = lane; i < n; i += 32) {
            const double v = a[i];
            if (want_norm && c0 == 0) asum += fabs(v);
#pragma unroll
            for (int c = 0; c < kAdjRhs; c++)
                if (c < nc) acc[c] = fma(v, Y[i + (c0 + c) * ldy], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < kAdjRhs; c++)
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane == 0)
            for (int c = 0; c < nc; c++) R[j + (c0 + c) * ldr] = G[j + (c0 + c) * ldg] - acc[c];
    }
    if (want_norm) {
        for (int o = 16; o > 0; o >>= 1) asum += __shfl_xor_sync(0xffffffffu, asum, o);
        if (lane == 0)
            atomicMax(reinterpret_cast<unsigned long long *>(colmax), (unsigned long long)__double_as_longlong(asum));
    }
}

// C (n x m) = alpha * Y (n x k) X^T (X: m x k), double, 64 x 64 tiles.
__global__ void __launch_bounds__(256) outer_kernel(int64_t n, int64_t m, int64_t k, double alpha,
                                                    const double *__restrict__ Y, int64_t ldy,
                                                    const double *__restrict__ X, int64_t ldx, double *C, int64_t ldc)
{
    __shared__ double sy[16][64 + 1], sx[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t i0 = (int64_t)blockIdx.x * 64, j0 = (int64_t)blockIdx.y * 64;
    double acc[4][4] = {};
    for (int64_t p0 = 0; p0 < k; p0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            int r = e % 64, p = e / 64;
            sy[p][r] = (i0 + r < n && p0 + p < k) ? Y[(i0 + r) + (p0 + p) * ldy] : 0.0;
            sx[p][r] = (j0 + r < m && p0 + p < k) ? X[(j0 + r) + (p0 + p) * ldx] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < 16; p++) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                a[u] = sy[p][tx + 16 * u];
                b[u] = sx[p][ty + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < 4; v++) {
        int64_t j = j0 + ty + 16 * v;
        if (j >= m) continue;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            int64_t i = i0 + tx + 16 * u;
            if (i < n) C[i + j * ldc] = alpha * acc[u][v];
        }
    }
}

__global__ void berr_t_kernel(int64_t n, const double *R, int64_t ldr, const double *Y, int64_t ldy,
                              const double *G, int64_t ldg, const double *anorm, double *berr)
{
    __shared__ double sr[256], sy[256], sg[256];
    const int64_t c = blockIdx.x;
    double mr = 0.0, my = 0.0, mg = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double v = fabs(R[i + c * ldr]);
        if (v > mr || isnan(v)) mr = v;
        v = fabs(Y[i + c * ldy]);
        if (v > my || isnan(v)) my = v;
        v = fabs(G[i + c * ldg]);
        if (v > mg || isnan(v)) mg = v;
    }
    sr[threadIdx.x] = mr;
    sy[threadIdx.x] = my;
    sg[threadIdx.x] = mg;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            if (sr[threadIdx.x + o] > sr[threadIdx.x] || isnan(sr[threadIdx.x + o])) sr[threadIdx.x] = sr[threadIdx.x + o];
            if (sy[threadIdx.x + o] > sy[threadIdx.x] || isnan(sy[threadIdx.x + o])) sy[threadIdx.x] = sy[threadIdx.x + o];
            if (sg[threadIdx.x + o] > sg[threadIdx.x] || isnan(sg[threadIdx.x + o])) sg[threadIdx.x] = sg[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double den = (*anorm) * sy[0] + sg[0];
        double e = den > 0.0 ? sr[0] / den : (sr[0] > 0.0 ? INFINITY : 0.0);
        if (isnan(sr[0]) || isnan(den)) e = NAN;
        atomicMax(reinterpret_cast<unsigned long long *>(berr), (unsigned long long)__double_as_longlong(e));
    }
}

static rbt_status resid_t(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *Y, int64_t ldy,
                          const double *G, int64_t ldg, double *R, int64_t ldr, double *anorm, bool want_norm,
                          double *berr, cudaStream_t s)
{
    ProfScope ps(kProfResidual, s);
    if (want_norm) RBT_CUDA_TRY(cudaMemsetAsync(anorm, 0, 8, s));
    resid_t_kernel<<<(unsigned)cdiv(n, kAdjWarps), 32 * kAdjWarps, 0, s>>>(n, nrhs, A, lda, Y, ldy, G, ldg, R, ldr,
                                                                            anorm, want_norm ? 1 : 0);
    RBT_LAUNCH_CHECK();
    RBT_CUDA_TRY(cudaMemsetAsync(berr, 0, 8, s));
    berr_t_kernel<<<(unsigned)nrhs, 256, 0, s>>>(n, R, ldr, Y, ldy, G, ldg, anorm, berr);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

}  // namespace rbt

using namespace rbt;

extern "C" {

rbt_status rbt_outer(int64_t n, int64_t m, int64_t k, double alpha, const double *Y, int64_t ldy, const double *X,
                     int64_t ldx, double *C, int64_t ldc, cudaStream_t stream)
{
    if (n < 0 || m < 0 || k < 0 || ldy < (n > 1 ? n : 1) || ldx < (m > 1 ? m : 1) || ldc < (n > 1 ? n : 1))
        return RBT_ERR_ARG;
    if (n == 0 || m == 0) return RBT_OK;
    if (!C || (k > 0 && (!Y || !X))) return RBT_ERR_ARG;
    dim3 grid((unsigned)cdiv(n, 64), (unsigned)cdiv(m, 64));
    outer_kernel<<<grid, 256, 0, stream>>>(n, m, k, alpha, Y, ldy, X, ldx, C, ldc);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

rbt_status rbt_solve_adjoint(const rbt_opts *opts, const rbt_info *fwd, int64_t n, int64_t nrhs, const double *A,
                             int64_t lda, const double *G, int64_t ldg, double *Y, int64_t ldy, void *work,
                             size_t work_bytes, rbt_info *info, cudaStream_t s)
{
    if (!opts || !fwd || !info || n < 0 || nrhs < 0) return RBT_ERR_ARG;
    int64_t mn = n > 1 ? n : 1;
    if (lda < mn || ldg < mn || ldy < mn) return RBT_ERR_ARG;
    info->status = RBT_ERR_ARG;
    info->zero_pivot = -1;
    info->iters = 0;
    info->fell_back = fwd->fell_back;
    info->berr_unrefined = NAN;
    info->berr = NAN;
    if (fwd->status != RBT_OK && fwd->status != RBT_NOT_CONVERGED) return RBT_ERR_ARG;  // no usable factors
    if (n == 0 || nrhs == 0) {
        info->status = RBT_OK;
        info->berr = info->berr_unrefined = 0.0;
        return RBT_OK;
    }
    if (!A || !G || !Y || !work) return RBT_ERR_ARG;
    size_t need = rbt_solve_workspace(opts, n, nrhs);
    if (work_bytes < need) return RBT_ERR_WORKSPACE;
    SolveLayout L;
    solve_layout(opts, n, nrhs, &L);
    char *w = (char *)work;
    // the factors of the forward solution: its own precision, or those of its
    // fallback (double, or eight digits after a seven-digit attempt)
    const int prec = opts->prec == RBT_F64 ? RBT_F64
                     : fwd->fell_back == 1 ? RBT_F64
                     : fwd->fell_back == 2 ? RBT_DF64TC
                                           : opts->prec;
    const void *At = (fwd->fell_back && opts->prec != RBT_F64) ? (const void *)(w + L.at64) : (const void *)(w + L.at);
    const double *U = (const double *)(w + L.u), *V = (const double *)(w + L.v);
    double *R = (double *)(w + L.r);
    double *scal = (double *)(w + L.scal);  // [2] ||A^T||, [3] berr
    void *sol = w + L.sol;
    size_t sol_bytes = L.total - L.sol;
    const int d = opts->depth;
    if (rbt_reference_size(n, d, opts->align, opts->grid_p, opts->grid_q) < 0) return RBT_ERR_ARG;
    const int64_t align = effective_align(opts->align, opts->grid_p, opts->grid_q);
    auto corr = [&](double *Z, int64_t ldz) -> rbt_status {
        // Z <- U A~^{-T} V^T Z
        rbt_status st = apply_vec(n, d, align, V, n, 1, Z, ldz, nrhs, s, opts->kind);
        if (st != RBT_OK) return st;
        st = genp_solve_run(n, nrhs, prec, At, L.ldt, 1, Z, ldz, sol, s);
        if (st != RBT_OK) return st;
        return apply_vec(n, d, align, U, n, 0, Z, ldz, nrhs, s, opts->kind);
    };
    (void)sol_bytes;  // sized by the solve layout
    // the chained solves' timeout flag: cleared once, read before returning
    RBT_CUDA_TRY(cudaMemsetAsync(sol, 0, sizeof(int), s));
    auto timed_out = [&](bool *out) -> rbt_status {
        int h = 0;
        RBT_CUDA_TRY(cudaMemcpyAsync(&h, sol, 4, cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaStreamSynchronize(s));
        *out = h != 0;
        return RBT_OK;
    };
    RBT_CUDA_TRY(cudaMemcpy2DAsync(Y, ldy * 8, G, ldg * 8, n * 8, nrhs, cudaMemcpyDeviceToDevice, s));
    rbt_status st = corr(Y, ldy);
    if (st != RBT_OK) return st;
    st = resid_t(n, nrhs, A, lda, Y, ldy, G, ldg, R, n, scal + 2, true, scal + 3, s);
    if (st != RBT_OK) return st;
    double berr = 0.0;
    RBT_CUDA_TRY(cudaMemcpyAsync(&berr, scal + 3, 8, cudaMemcpyDeviceToHost, s));
    RBT_CUDA_TRY(cudaStreamSynchronize(s));
    info->berr_unrefined = berr;
    int it = 0;
    while (!(berr <= opts->tol) && it < opts->refine_max) {
        st = corr(R, n);
        if (st != RBT_OK) return st;
        st = add_block(n, nrhs, R, n, Y, ldy, s);
        if (st != RBT_OK) return st;
        st = resid_t(n, nrhs, A, lda, Y, ldy, G, ldg, R, n, scal + 2, false, scal + 3, s);
        if (st != RBT_OK) return st;
        double prev = berr;
        RBT_CUDA_TRY(cudaMemcpyAsync(&berr, scal + 3, 8, cudaMemcpyDeviceToHost, s));
        RBT_CUDA_TRY(cudaStreamSynchronize(s));
        it++;
        if (!(berr < 0.9 * prev)) break;
    }
    bool to = false;
    st = timed_out(&to);
    if (st != RBT_OK) return st;
    if (to) return RBT_ERR_TIMEOUT;
    info->iters = it;
    info->berr = berr;
    info->status = berr <= opts->tol ? RBT_OK : RBT_NOT_CONVERGED;
    return (rbt_status)info->status;
}

}  // extern "C"
