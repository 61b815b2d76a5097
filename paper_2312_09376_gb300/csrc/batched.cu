// Batched RBT solves in one persistent launch (sm_103a).
//
// Thousands of independent systems of uneven order, each with its own seeded
// butterflies, are solved by one kernel: each CTA takes the next system from
// a device work queue (largest first) and runs the whole method on it with
// its threads -- coefficients (Sec. 6), the fused two-sided transform
// (Eq. rbt-depth-d, all layers in one pass), blocked GENP, the transformed
// solve (Eq. precond) and double-precision iterative refinement (Sec. 5) --
// without returning to the host.  The launch is a memset of the queue counter
// plus one kernel, so it can be captured in a CUDA graph.  The working
// precision is double or float (then refined to double).
//
// Per-system scratch lives in the caller's workspace at offsets fixed by the
// plan; the descriptor table and the queue order are copied there by
// rbt_solve_batched_plan.  The variant (threads per CTA, GENP block size) is
// chosen by rbt_solve_batched_autotune, which times every compiled variant on
// the planned batch and keeps the fastest for that batch's size histogram.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "genp_internal.cuh"
#include "rbt_dev.cuh"

namespace rbt {
namespace bat {

struct SysDesc {
    int64_t n, nrhs;
    const double *A;
    int64_t lda;
    const double *B;
    int64_t ldb;
    double *X;
    int64_t ldx;
    uint64_t seed;
    int64_t off;  // byte offset of the system's scratch inside the workspace
};

constexpr int kMaxRhsChunk = 8;
constexpr int kTile = 64;  // trailing-update tile

// ------------------------------------------------------------- CTA routines

template <int NT>
__device__ double block_max(double v, double *red)
{
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (tid < o) {
            double b = red[tid + o];
            if (b > red[tid] || isnan(b)) red[tid] = b;
        }
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

// One system's scratch layout (bytes), shared by host and device.
struct Layout {
    int64_t u, v, at, xt, r, total;
};

__host__ __device__ inline int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

template <typename T>
__host__ __device__ inline Layout sys_layout(int64_t n, int64_t nrhs, int d)
{
    Layout L;
    int64_t o = 0;
    int64_t dd = d > 0 ? d : 1;
    L.u = o;
    o = align256(o + n * dd * 8);
    L.v = o;
    o = align256(o + n * dd * 8);
    L.at = o;
    o = align256(o + n * n * (int64_t)sizeof(T));
    L.xt = o;
    o = align256(o + n * nrhs * (int64_t)sizeof(T));
    L.r = o;
    o = align256(o + n * nrhs * 8);
    L.total = o;
    return L;
}

// Blocked right-looking GENP of an n x n matrix (ld n) held in global memory
// (L2-resident for the sizes of a batch) by one CTA.  Returns -1 or the first
// zero / non-finite pivot.
template <typename T, int NT, int NB>
__device__ int64_t cta_genp(int64_t n, T *A, T *s_diag, T *s_a, T *s_b, int *s_flag)
{
    const int tid = threadIdx.x;
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        // diagonal block in shared memory
        for (int e = tid; e < kb * kb; e += NT) s_diag[e] = A[(k0 + e % kb) + (k0 + e / kb) * n];
        if (tid == 0) *s_flag = -1;
        __syncthreads();
        for (int j = 0; j < kb; j++) {
            T p = s_diag[j + j * kb];
            if (p == T(0) || !isfinite(p)) {
                if (tid == 0) *s_flag = j;
                break;  // uniform: every thread reads the same pivot
            }
            for (int i = j + 1 + tid; i < kb; i += NT) s_diag[i + j * kb] /= p;
            __syncthreads();
            const int rem = kb - j - 1;
            for (int e = tid; e < rem * rem; e += NT) {
                int i = j + 1 + e % rem, c = j + 1 + e / rem;
                s_diag[i + c * kb] -= s_diag[i + j * kb] * s_diag[j + c * kb];
            }
            __syncthreads();
        }
        __syncthreads();
        if (*s_flag >= 0) return k0 + *s_flag;
        for (int e = tid; e < kb * kb; e += NT) A[(k0 + e % kb) + (k0 + e / kb) * n] = s_diag[e];
        const int64_t r0 = k0 + kb;
        // U12 <- L11^{-1} A12 (one thread per column) and L21 <- A21 U11^{-1}
        // (one per row).  The substitutions run over all NB positions with
        // compile-time triangular bounds (straight-line code); for a short
        // last block (kb < NB) the positions past kb read other entries of
        // s_diag (still inside its NB x NB allocation) and are never stored.
        for (int64_t c = r0 + tid; c < n; c += NT) {
            T x[NB];
#pragma unroll
            for (int i = 0; i < NB; i++) x[i] = (i < kb) ? A[(k0 + i) + c * n] : T(0);
#pragma unroll
            for (int i = 1; i < NB; i++) {
                T s = x[i];
#pragma unroll
                for (int p = 0; p < i; p++) s -= s_diag[i + p * kb] * x[p];
                x[i] = s;
            }
#pragma unroll
            for (int i = 0; i < NB; i++)
                if (i < kb) A[(k0 + i) + c * n] = x[i];
        }
        for (int64_t r = r0 + tid; r < n; r += NT) {
            T x[NB];
#pragma unroll
            for (int j = 0; j < NB; j++) x[j] = (j < kb) ? A[r + (k0 + j) * n] : T(0);
#pragma unroll
            for (int j = 0; j < NB; j++) {
                T s = x[j];
#pragma unroll
                for (int p = 0; p < j; p++) s -= x[p] * s_diag[p + j * kb];
                x[j] = (j < kb) ? s / s_diag[j + j * kb] : T(0);
            }
#pragma unroll
            for (int j = 0; j < NB; j++)
                if (j < kb) A[r + (k0 + j) * n] = x[j];
        }
        __syncthreads();
        // A22 -= L21 U12, 64 x 64 tiles, each thread a (64*64/NT) register tile
        const int64_t rest = n - r0;
        const int64_t nt = (rest + kTile - 1) / kTile;
        constexpr int TPR = kTile * kTile / NT;  // outputs per thread
        constexpr int TW = (TPR >= 16) ? 4 : 2;  // register tile TW x (TPR / TW)
        constexpr int TH = TPR / TW;
        constexpr int GX = kTile / TW;           // threads along rows
        const int tx = tid % GX, ty = tid / GX;
        for (int64_t t = 0; t < nt * nt; t++) {
            const int64_t ti = t % nt, tj = t / nt;
            const int64_t i0 = r0 + ti * kTile, j0 = r0 + tj * kTile;
            for (int e = tid; e < kTile * kb; e += NT) {
                int i = e % kTile, p = e / kTile;
                s_a[i + p * kTile] = (i0 + i < n) ? A[(i0 + i) + (k0 + p) * n] : T(0);
            }
            for (int e = tid; e < kTile * kb; e += NT) {
                int p = e % kb, j = e / kb;
                s_b[p + j * NB] = (j0 + j < n) ? A[(k0 + p) + (j0 + j) * n] : T(0);
            }
            __syncthreads();
            T acc[TW][TH];
#pragma unroll
            for (int a = 0; a < TW; a++)
#pragma unroll
                for (int b = 0; b < TH; b++) acc[a][b] = T(0);
            for (int p = 0; p < kb; p++) {
                T ra[TW], rb[TH];
#pragma unroll
                for (int a = 0; a < TW; a++) ra[a] = s_a[(tx + a * GX) + p * kTile];
#pragma unroll
                for (int b = 0; b < TH; b++) rb[b] = s_b[p + (ty + b * (NT / GX)) * NB];
#pragma unroll
                for (int a = 0; a < TW; a++)
#pragma unroll
                    for (int b = 0; b < TH; b++) acc[a][b] = fma(ra[a], rb[b], acc[a][b]);
            }
#pragma unroll
            for (int b = 0; b < TH; b++) {
                int64_t j = j0 + ty + b * (NT / GX);
                if (j >= n) continue;
#pragma unroll
                for (int a = 0; a < TW; a++) {
                    int64_t i = i0 + tx + a * GX;
                    if (i < n) A[i + j * n] -= acc[a][b];
                }
            }
            __syncthreads();
        }
    }
    return -1;
}

// The diagonal-block substitutions of the CTA solves: the kb x kb block
// (kb <= NB <= 32) sits in shared memory (s_blk, column-major), and one warp
// per right-hand side solves it right-looking: lane i holds x_i; at step j,
// x_j is final and reaches every lane by a shuffle, and the lanes of the rows
// still to solve subtract their multiple of it.  M(i, j) is the entry the
// triangle uses (taken from s_blk directly or transposed).
template <typename T, int NT, bool LOWER, bool UNIT, bool TRANS>
__device__ __forceinline__ void cta_block_subst(int kb, int64_t nrhs, const T *s_blk, T *X, int64_t n, int64_t k0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    auto M = [&](int i, int j) { return TRANS ? s_blk[j + i * kb] : s_blk[i + j * kb]; };
    for (int64_t c = warp; c < nrhs; c += NW) {
        T *x = X + c * n + k0;
        T xi = lane < kb ? x[lane] : T(0);
        if (LOWER) {
            for (int j = 0; j < kb; j++) {
                if (!UNIT && lane == j) xi = xi / M(j, j);
                const T xj = shfl_idx(xi, j);
                if (lane > j && lane < kb) xi -= M(lane, j) * xj;
            }
        } else {
            for (int j = kb - 1; j >= 0; j--) {
                if (!UNIT && lane == j) xi = xi / M(j, j);
                const T xj = shfl_idx(xi, j);
                if (lane < j) xi -= M(lane, j) * xj;
            }
        }
        if (lane < kb) x[lane] = xi;
    }
}

template <typename T, int NT>
__device__ __forceinline__ void cta_load_block(int kb, const T *LU, int64_t n, int64_t k0, T *s_blk)
{
    for (int e = threadIdx.x; e < kb * kb; e += NT) s_blk[e] = LU[(k0 + e % kb) + (k0 + e / kb) * n];
}

// Xt (n x nrhs, ld n) <- (L U)^{-1} Xt, one CTA, blocked by NB rows: each
// diagonal block by cta_block_subst, then the rows still to solve take the
// block's contribution (all threads).  s_blk: NB x NB of shared memory.
template <typename T, int NT, int NB>
__device__ void cta_lu_solve(int64_t n, int64_t nrhs, const T *LU, T *X, T *s_blk)
{
    static_assert(NB <= 32, "one lane per row of a diagonal block");
    const int tid = threadIdx.x;
    // forward, unit lower
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        cta_load_block<T, NT>(kb, LU, n, k0, s_blk);
        __syncthreads();
        cta_block_subst<T, NT, true, true, false>(kb, nrhs, s_blk, X, n, k0);
        __syncthreads();
        for (int64_t e = tid; e < (n - k0 - kb) * nrhs; e += NT) {
            int64_t r = k0 + kb + e % (n - k0 - kb), c = e / (n - k0 - kb);
            T s = T(0);
            for (int p = 0; p < kb; p++) s = fma(LU[r + (k0 + p) * n], X[(k0 + p) + c * n], s);
            X[r + c * n] -= s;
        }
        __syncthreads();
    }
    // backward, upper
    const int64_t nblk = (n + NB - 1) / NB;
    for (int64_t b = nblk - 1; b >= 0; b--) {
        const int64_t k0 = b * NB;
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        cta_load_block<T, NT>(kb, LU, n, k0, s_blk);
        __syncthreads();
        cta_block_subst<T, NT, false, false, false>(kb, nrhs, s_blk, X, n, k0);
        __syncthreads();
        for (int64_t e = tid; e < k0 * nrhs; e += NT) {
            int64_t r = e % k0, c = e / k0;
            T s = T(0);
            for (int p = 0; p < kb; p++) s = fma(LU[r + (k0 + p) * n], X[(k0 + p) + c * n], s);
            X[r + c * n] -= s;
        }
        __syncthreads();
    }
}

// R = B - A X in double; returns the largest backward error over the columns
// (Eq. inf-norm-backerr).  anorm: ||A||_inf, computed when *anorm < 0.
// Rows tid, tid + NT, ... of R(:, c0 .. c0 + NC) = B - A X for exactly NC
// right-hand sides (a compile-time count: every multiply-add issued is one
// the residual needs; the FP64 pipe is this routine's bound), and the
// largest absolute row sum of A when norm is set.
template <int NT, int NC>
__device__ __forceinline__ void residual_rows(int64_t n, int64_t c0, const double *A, int64_t lda, const double *X,
                                              int64_t ldx, const double *B, int64_t ldb, double *R, bool norm,
                                              double &rowmax)
{
    for (int64_t r = threadIdx.x; r < n; r += NT) {
        double acc[NC];
#pragma unroll
        for (int c = 0; c < NC; c++) acc[c] = 0.0;
        double asum = 0.0;
        for (int64_t j = 0; j < n; j++) {
            const double a = A[r + j * lda];
            if (norm) asum += fabs(a);
#pragma unroll
            for (int c = 0; c < NC; c++) acc[c] = fma(a, X[j + (c0 + c) * ldx], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < NC; c++) R[r + (c0 + c) * n] = B[r + (c0 + c) * ldb] - acc[c];
        if (norm && (asum > rowmax || isnan(asum))) rowmax = asum;
    }
}

template <int NT>
__device__ double cta_residual(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X, int64_t ldx,
                               const double *B, int64_t ldb, double *R, double *anorm, double *red)
{
    const int tid = threadIdx.x;
    const bool want_norm = *anorm < 0.0;
    double rowmax = 0.0;
    // the right-hand sides in chunks of 8, the rest by 4, 2 and 1
    for (int64_t c0 = 0; c0 < nrhs;) {
        const int64_t left = nrhs - c0;
        const bool norm = want_norm && c0 == 0;
        if (left >= 8) {
            residual_rows<NT, 8>(n, c0, A, lda, X, ldx, B, ldb, R, norm, rowmax);
            c0 += 8;
        } else if (left >= 4) {
            residual_rows<NT, 4>(n, c0, A, lda, X, ldx, B, ldb, R, norm, rowmax);
            c0 += 4;
        } else if (left >= 2) {
            residual_rows<NT, 2>(n, c0, A, lda, X, ldx, B, ldb, R, norm, rowmax);
            c0 += 2;
        } else {
            residual_rows<NT, 1>(n, c0, A, lda, X, ldx, B, ldb, R, norm, rowmax);
            c0 += 1;
        }
    }
    if (want_norm) {
        double m = block_max<NT>(rowmax, red);
        if (tid == 0) *anorm = m;
        __syncthreads();
    }
    __syncthreads();
    const double an = *anorm;
    double worst = 0.0;
    for (int64_t c = 0; c < nrhs; c++) {
        double mr = 0.0, mx = 0.0, mb = 0.0;
        for (int64_t r = tid; r < n; r += NT) {
            double v = fabs(R[r + c * n]);
            if (v > mr || isnan(v)) mr = v;
            v = fabs(X[r + c * ldx]);
            if (v > mx || isnan(v)) mx = v;
            v = fabs(B[r + c * ldb]);
            if (v > mb || isnan(v)) mb = v;
        }
        mr = block_max<NT>(mr, red);
        mx = block_max<NT>(mx, red);
        mb = block_max<NT>(mb, red);
        double den = an * mx + mb;
        double e = den > 0.0 ? mr / den : (mr > 0.0 ? INFINITY : 0.0);
        if (isnan(mr) || isnan(den)) e = NAN;
        if (e > worst || isnan(e)) worst = e;
    }
    return worst;
}

// x <- W^T x (trans) or W x, one CTA, every right-hand side; d_s <= 3.
template <int NT>
__device__ void cta_vec(int64_t n, int d, const double *W, int trans, double *X, int64_t ldx, int64_t nrhs)
{
    const int ds = eff_depth(n, d);
    const int64_t m = ref_size(n, d);
    if (ds == 0) {
        for (int64_t e = threadIdx.x; e < n * nrhs; e += NT) {
            int64_t i = e % n, c = e / n;
            double p = X[i + c * ldx];
            for (int k = 1; k <= d; k++) p *= W[i + (k - 1) * n];
            X[i + c * ldx] = p;
        }
        __syncthreads();
        return;
    }
    const int64_t h = m >> ds;
    for (int64_t e = threadIdx.x; e < h * nrhs; e += NT) {
        const int64_t gr = e % h, c = e / h;
        switch (ds) {
        case 1: vec_group<1>(n, h, ds, trans, ds + 1, d, W, n, X + c * ldx, gr); break;
        case 2: vec_group<2>(n, h, ds, trans, ds + 1, d, W, n, X + c * ldx, gr); break;
        default: vec_group<3>(n, h, ds, trans, ds + 1, d, W, n, X + c * ldx, gr); break;
        }
    }
    __syncthreads();
}

// Transform, factor, solve and refine one system in working precision T with
// this CTA (coefficients U, V already generated).  Writes X; fills info.
template <typename T, int NT, int NB>
__device__ void solve_sys(const SysDesc &S, char *w, int d, int refine_max, double tol, unsigned char *smem_raw,
                          int *s_flag, double *red, double *s_anorm, rbt_batched_info &info)
{
    const int tid = threadIdx.x;
    const int64_t n = S.n, nrhs = S.nrhs;
    const Layout L = sys_layout<T>(n, nrhs, d);
    const double *U = (const double *)(w + L.u), *V = (const double *)(w + L.v);
    double *R = (double *)(w + L.r);
    T *At = (T *)(w + L.at), *Xt = (T *)(w + L.xt);
    T *s_diag = (T *)smem_raw;
    T *s_a = s_diag + NB * NB;
    T *s_b = s_a + kTile * NB;
    info.status = RBT_OK;
    info.iters = 0;
    info.zero_pivot = -1;
    info.berr_unrefined = NAN;
    info.berr = NAN;
    {
        const int ds = eff_depth(n, d);
        const int64_t h = ds > 0 ? (ref_size(n, d) >> ds) : 0;
        if (ds == 0) {
            for (int64_t e = tid; e < n * n; e += NT) {
                int64_t i = e % n, j = e / n;
                double p = S.A[i + j * S.lda];
                for (int k = 1; k <= d; k++) p *= U[i + (k - 1) * n] * V[j + (k - 1) * n];
                At[i + j * n] = (T)p;
            }
        } else {
            for (int64_t e = tid; e < h * h; e += NT) {
                const int64_t gr = e % h, gc = e / h;
                switch (ds) {
                case 1: transform_group<1, T>(n, h, ds, ds + 1, d, U, V, n, S.A, S.lda, At, n, gr, gc); break;
                case 2: transform_group<2, T>(n, h, ds, ds + 1, d, U, V, n, S.A, S.lda, At, n, gr, gc); break;
                default: transform_group<3, T>(n, h, ds, ds + 1, d, U, V, n, S.A, S.lda, At, n, gr, gc); break;
                }
            }
        }
    }
    __syncthreads();
    const int64_t piv = cta_genp<T, NT, NB>(n, At, s_diag, s_a, s_b, s_flag);
    if (piv >= 0) {
        T p = At[piv + piv * n];
        info.status = (p == T(0)) ? RBT_ZERO_PIVOT : RBT_NONFINITE;
        info.zero_pivot = piv;
        __syncthreads();
        return;
    }
    // x = V A~^{-1} U^T b (Eq. precond)
    for (int64_t e = tid; e < n * nrhs; e += NT) S.X[e % n + (e / n) * S.ldx] = S.B[e % n + (e / n) * S.ldb];
    __syncthreads();
    cta_vec<NT>(n, d, U, 1, S.X, S.ldx, nrhs);
    for (int64_t e = tid; e < n * nrhs; e += NT) Xt[e] = (T)S.X[e % n + (e / n) * S.ldx];
    __syncthreads();
    cta_lu_solve<T, NT, NB>(n, nrhs, At, Xt, s_diag);
    for (int64_t e = tid; e < n * nrhs; e += NT) S.X[e % n + (e / n) * S.ldx] = (double)Xt[e];
    __syncthreads();
    cta_vec<NT>(n, d, V, 0, S.X, S.ldx, nrhs);
    if (tid == 0) *s_anorm = -1.0;
    __syncthreads();
    double berr = cta_residual<NT>(n, nrhs, S.A, S.lda, S.X, S.ldx, S.B, S.ldb, R, s_anorm, red);
    info.berr_unrefined = berr;
    // refinement in double (Sec. 5): dx = V A~^{-1} U^T r, while it still gains
    int it = 0;
    while (!(berr <= tol) && it < refine_max) {
        cta_vec<NT>(n, d, U, 1, R, n, nrhs);
        for (int64_t e = tid; e < n * nrhs; e += NT) Xt[e] = (T)R[e];
        __syncthreads();
        cta_lu_solve<T, NT, NB>(n, nrhs, At, Xt, s_diag);
        for (int64_t e = tid; e < n * nrhs; e += NT) R[e] = (double)Xt[e];
        __syncthreads();
        cta_vec<NT>(n, d, V, 0, R, n, nrhs);
        for (int64_t e = tid; e < n * nrhs; e += NT) S.X[e % n + (e / n) * S.ldx] += R[e];
        __syncthreads();
        const double prev = berr;
        berr = cta_residual<NT>(n, nrhs, S.A, S.lda, S.X, S.ldx, S.B, S.ldb, R, s_anorm, red);
        it++;
        if (!(berr < 0.9 * prev)) break;  // stalled: less than 10% gained
    }
    info.iters = it;
    info.berr = berr;
    info.status = berr <= tol ? RBT_OK : RBT_NOT_CONVERGED;
}

template <typename T, int NT, int NB>
__global__ void __launch_bounds__(NT)
batched_kernel(const SysDesc *__restrict__ sys, const int *__restrict__ order, int batch, int *counter,
               rbt_batched_info *infos, char *work, int d, int refine_max, double tol, int fallback)
{
    __shared__ int s_idx, s_flag;
    __shared__ __align__(16) unsigned char smem_raw[sizeof(double) * (NB * NB + 2 * kTile * NB)];
    __shared__ double red[NT];
    __shared__ double s_anorm;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_idx = atomicAdd(counter, 1);
        __syncthreads();
        const int q = s_idx;
        __syncthreads();
        if (q >= batch) return;
        const int id = order[q];
        const SysDesc S = sys[id];
        const int64_t n = S.n;
        char *w = work + S.off;
        const Layout L = sys_layout<T>(n, S.nrhs, d);
        double *U = (double *)(w + L.u), *V = (double *)(w + L.v);
        // coefficients (Sec. 6), shared by the working-precision and fallback attempts
        for (int64_t e = tid; e < 2 * n * d; e += NT) {
            int side = e >= n * d ? 1 : 0;
            int64_t rem = e - side * n * d;
            int layer = (int)(rem / n) + 1;
            int64_t i = rem - (int64_t)(layer - 1) * n;
            (side ? V : U)[i + (int64_t)(layer - 1) * n] = coef_value(S.seed, side, layer, i);
        }
        __syncthreads();
        rbt_batched_info info;
        info.fell_back = 0;
        info.reserved = 0;
        solve_sys<T, NT, NB>(S, w, d, refine_max, tol, smem_raw, &s_flag, red, &s_anorm, info);
        if (sizeof(T) < sizeof(double) && fallback && info.status != RBT_OK) {
            // "responsibly reckless" fallback (Sec. 5): the same A~ in double
            const int prior = info.iters;
            solve_sys<double, NT, NB>(S, w, d, refine_max, tol, smem_raw, &s_flag, red, &s_anorm, info);
            info.fell_back = 1;
            info.iters += prior;
        }
        if (tid == 0) infos[id] = info;
        __syncthreads();
    }
}

// Xt <- (L U)^{-T} Xt: U^T z = g (forward, non-unit, U's columns), then
// L^T y = z (backward, unit, L's columns); one CTA, blocked by NB, the
// diagonal blocks by cta_block_subst on the transposed block.
template <typename T, int NT, int NB>
__device__ void cta_lu_solve_t(int64_t n, int64_t nrhs, const T *LU, T *X, T *s_blk)
{
    static_assert(NB <= 32, "one lane per row of a diagonal block");
    const int tid = threadIdx.x;
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        cta_load_block<T, NT>(kb, LU, n, k0, s_blk);
        __syncthreads();
        cta_block_subst<T, NT, true, false, true>(kb, nrhs, s_blk, X, n, k0);
        __syncthreads();
        for (int64_t e = tid; e < (n - k0 - kb) * nrhs; e += NT) {
            int64_t r = k0 + kb + e % (n - k0 - kb), c = e / (n - k0 - kb);
            T s = T(0);
            for (int p = 0; p < kb; p++) s = fma(LU[(k0 + p) + r * n], X[(k0 + p) + c * n], s);
            X[r + c * n] -= s;
        }
        __syncthreads();
    }
    const int64_t nblk = (n + NB - 1) / NB;
    for (int64_t b = nblk - 1; b >= 0; b--) {
        const int64_t k0 = b * NB;
        const int kb = (int)(n - k0 < NB ? n - k0 : NB);
        cta_load_block<T, NT>(kb, LU, n, k0, s_blk);
        __syncthreads();
        cta_block_subst<T, NT, false, true, true>(kb, nrhs, s_blk, X, n, k0);
        __syncthreads();
        for (int64_t e = tid; e < k0 * nrhs; e += NT) {
            int64_t r = e % k0, c = e / k0;
            T s = T(0);
            for (int p = 0; p < kb; p++) s = fma(LU[(k0 + p) + r * n], X[(k0 + p) + c * n], s);
            X[r + c * n] -= s;
        }
        __syncthreads();
    }
}

// R = G - A^T Y in double; largest backward error of A^T y = g over the
// columns, with ||A^T||_inf = largest column sum of |A| (computed when *anorm < 0).
template <int NT>
__device__ double cta_residual_t(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *Y, int64_t ldy,
                                 const double *G, int64_t ldg, double *R, double *anorm, double *red)
{
    const int tid = threadIdx.x;
    const bool want_norm = *anorm < 0.0;
    double colmax = 0.0;
    for (int64_t j = tid; j < n; j += NT) {
        const double *a = A + j * lda;
        double asum = 0.0;
        for (int64_t c0 = 0; c0 < nrhs; c0 += kMaxRhsChunk) {
            const int nc = (int)(nrhs - c0 < kMaxRhsChunk ? nrhs - c0 : kMaxRhsChunk);
            double acc[kMaxRhsChunk];
#pragma unroll
            for (int c = 0; c < kMaxRhsChunk; c++) acc[c] = 0.0;
            for (int64_t i = 0; i < n; i++) {
                const double v = a[i];
                if (want_norm && c0 == 0) asum += fabs(v);
#pragma unroll
                for (int c = 0; c < kMaxRhsChunk; c++)
                    if (c < nc) acc[c] = fma(v, Y[i + (c0 + c) * ldy], acc[c]);
            }
            for (int c = 0; c < nc; c++) R[j + (c0 + c) * n] = G[j + (c0 + c) * ldg] - acc[c];
        }
        if (want_norm && (asum > colmax || isnan(asum))) colmax = asum;
    }
    if (want_norm) {
        double m = block_max<NT>(colmax, red);
        if (tid == 0) *anorm = m;
    }
    __syncthreads();
    const double an = *anorm;
    double worst = 0.0;
    for (int64_t c = 0; c < nrhs; c++) {
        double mr = 0.0, my = 0.0, mg = 0.0;
        for (int64_t r = tid; r < n; r += NT) {
            double v = fabs(R[r + c * n]);
            if (v > mr || isnan(v)) mr = v;
            v = fabs(Y[r + c * ldy]);
            if (v > my || isnan(v)) my = v;
            v = fabs(G[r + c * ldg]);
            if (v > mg || isnan(v)) mg = v;
        }
        mr = block_max<NT>(mr, red);
        my = block_max<NT>(my, red);
        mg = block_max<NT>(mg, red);
        double den = an * my + mg;
        double e = den > 0.0 ? mr / den : (mr > 0.0 ? INFINITY : 0.0);
        if (isnan(mr) || isnan(den)) e = NAN;
        if (e > worst || isnan(e)) worst = e;
    }
    return worst;
}

struct AdjDesc {
    const double *G;
    int64_t ldg;
    double *Y;
    int64_t ldy;
    double *GA;  // grad_A (n x n) or null
    int64_t ldga;
};

// grad_B = U A~^{-T} V^T grad_X (refined in double against A^T) and
// grad_A = -grad_B X^T, per system, with the factors the forward run left.
// A^T y = g for one system with the factors of precision T left by the
// forward run; refined in double against A^T.
template <typename T, int NT, int NB>
__device__ void adjoint_sys(const SysDesc &S, const AdjDesc &D, char *w, int d, int refine_max, double tol,
                            double *red, double *s_anorm, T *s_blk, rbt_batched_info &info)
{
    const int tid = threadIdx.x;
    const int64_t n = S.n, nrhs = S.nrhs;
    const Layout L = sys_layout<T>(n, nrhs, d);
    const double *U = (const double *)(w + L.u), *V = (const double *)(w + L.v);
    double *R = (double *)(w + L.r);
    const T *At = (const T *)(w + L.at);
    T *Xt = (T *)(w + L.xt);
    for (int64_t e = tid; e < n * nrhs; e += NT) D.Y[e % n + (e / n) * D.ldy] = D.G[e % n + (e / n) * D.ldg];
    __syncthreads();
    cta_vec<NT>(n, d, V, 1, D.Y, D.ldy, nrhs);
    for (int64_t e = tid; e < n * nrhs; e += NT) Xt[e] = (T)D.Y[e % n + (e / n) * D.ldy];
    __syncthreads();
    cta_lu_solve_t<T, NT, NB>(n, nrhs, At, Xt, s_blk);
    for (int64_t e = tid; e < n * nrhs; e += NT) D.Y[e % n + (e / n) * D.ldy] = (double)Xt[e];
    __syncthreads();
    cta_vec<NT>(n, d, U, 0, D.Y, D.ldy, nrhs);
    if (tid == 0) *s_anorm = -1.0;
    __syncthreads();
    double berr = cta_residual_t<NT>(n, nrhs, S.A, S.lda, D.Y, D.ldy, D.G, D.ldg, R, s_anorm, red);
    info.berr_unrefined = berr;
    int it = 0;
    while (!(berr <= tol) && it < refine_max) {
        cta_vec<NT>(n, d, V, 1, R, n, nrhs);
        for (int64_t e = tid; e < n * nrhs; e += NT) Xt[e] = (T)R[e];
        __syncthreads();
        cta_lu_solve_t<T, NT, NB>(n, nrhs, At, Xt, s_blk);
        for (int64_t e = tid; e < n * nrhs; e += NT) R[e] = (double)Xt[e];
        __syncthreads();
        cta_vec<NT>(n, d, U, 0, R, n, nrhs);
        for (int64_t e = tid; e < n * nrhs; e += NT) D.Y[e % n + (e / n) * D.ldy] += R[e];
        __syncthreads();
        const double prev = berr;
        berr = cta_residual_t<NT>(n, nrhs, S.A, S.lda, D.Y, D.ldy, D.G, D.ldg, R, s_anorm, red);
        it++;
        if (!(berr < 0.9 * prev)) break;
    }
    info.iters = it;
    info.berr = berr;
    info.status = berr <= tol ? RBT_OK : RBT_NOT_CONVERGED;
}

// grad_B = U A~^{-T} V^T grad_X (refined in double against A^T) and
// grad_A = -grad_B X^T, per system, with the factors the forward run left
// (the double ones when that system fell back).
template <typename T, int NT, int NB>
__global__ void __launch_bounds__(NT)
batched_adjoint_kernel(const SysDesc *__restrict__ sys, const AdjDesc *__restrict__ adj,
                       const int *__restrict__ order, int batch, int *counter, rbt_batched_info *infos, char *work,
                       int d, int refine_max, double tol)
{
    __shared__ int s_idx;
    __shared__ double red[NT];
    __shared__ double s_anorm;
    __shared__ __align__(16) double s_blk[NB * NB];  // diagonal block of the solves
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_idx = atomicAdd(counter, 1);
        __syncthreads();
        const int q = s_idx;
        __syncthreads();
        if (q >= batch) return;
        const int id = order[q];
        const SysDesc S = sys[id];
        const AdjDesc D = adj[id];
        const rbt_batched_info fwd = infos[id];
        __syncthreads();
        if (fwd.status != RBT_OK && fwd.status != RBT_NOT_CONVERGED) continue;  // no usable factors
        char *w = work + S.off;
        rbt_batched_info info;
        info.zero_pivot = -1;
        info.fell_back = fwd.fell_back;
        info.reserved = 0;
        if (fwd.fell_back)
            adjoint_sys<double, NT, NB>(S, D, w, d, refine_max, tol, red, &s_anorm, s_blk, info);
        else
            adjoint_sys<T, NT, NB>(S, D, w, d, refine_max, tol, red, &s_anorm, (T *)s_blk, info);
        const int64_t n = S.n, nrhs = S.nrhs;
        if (D.GA) {
            // grad_A = -Y X^T (rank nrhs)
            for (int64_t e = tid; e < n * n; e += NT) {
                const int64_t i = e % n, j = e / n;
                double s = 0.0;
                for (int64_t c = 0; c < nrhs; c++) s = fma(D.Y[i + c * D.ldy], S.X[j + c * S.ldx], s);
                D.GA[i + j * D.ldga] = -s;
            }
        }
        if (tid == 0) infos[id] = info;
        __syncthreads();
    }
}

// ------------------------------------------------------------- host side

struct Variant {
    int nt, nb;
};
static const Variant kVariants[] = {{128, 16}, {128, 32}, {256, 16}, {256, 32}};
constexpr int kNumVariants = 4;

struct PlanInfo {
    int64_t batch;
    int32_t prec, depth, fallback;
    size_t desc_off, order_off, counter_off, adj_off, sys_off;
    std::string signature;
};

static std::mutex g_mu;
static std::map<const void *, PlanInfo> g_plans;             // by workspace pointer
static std::map<std::string, int> g_tuned;                   // signature -> variant

template <typename T>
static rbt_status launch_variant(int v, const PlanInfo &P, char *w, rbt_batched_info *d_infos, int refine_max,
                                 double tol, cudaStream_t stream)
{
    const SysDesc *descs = (const SysDesc *)(w + P.desc_off);
    const int *order = (const int *)(w + P.order_off);
    int *counter = (int *)(w + P.counter_off);
    char *sys_base = w + P.sys_off;
    RBT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), stream));
    int sms = device_sm_count();
    int per_sm = 1;
    int grid;
#define RBT_BATCHED_LAUNCH(NT_, NB_)                                                                         \
    {                                                                                                        \
        RBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<T, NT_, NB_>, NT_, 0)); \
        grid = sms * (per_sm > 0 ? per_sm : 1);                                                              \
        if (grid > P.batch) grid = (int)P.batch;                                                             \
        batched_kernel<T, NT_, NB_><<<grid, NT_, 0, stream>>>(descs, order, (int)P.batch, counter, d_infos,  \
                                                              sys_base, P.depth, refine_max, tol, P.fallback); \
    }
    switch (v) {
    case 0: RBT_BATCHED_LAUNCH(128, 16) break;
    case 1: RBT_BATCHED_LAUNCH(128, 32) break;
    case 2: RBT_BATCHED_LAUNCH(256, 16) break;
    default: RBT_BATCHED_LAUNCH(256, 32) break;
    }
#undef RBT_BATCHED_LAUNCH
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

static std::string make_signature(int64_t batch, const int64_t *n, const int64_t *nrhs, int prec, int d)
{
    // histogram of orders in buckets of 64 and of right-hand sides, plus the device
    int hist[64] = {0};
    int64_t maxn = 0, sumr = 0;
    for (int64_t i = 0; i < batch; i++) {
        int b = (int)std::min<int64_t>(n[i] / 64, 63);
        hist[b]++;
        maxn = std::max(maxn, n[i]);
        sumr += nrhs ? nrhs[i] : 1;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    std::string name = cudaGetDeviceProperties(&p, dev) == cudaSuccess ? p.name : "gpu";
    std::string s = name + "|p" + std::to_string(prec) + "|d" + std::to_string(d) + "|b" + std::to_string(batch) +
                    "|r" + std::to_string(sumr) + "|";
    for (int i = 0; i < 64; i++)
        if (hist[i]) s += std::to_string(i) + ":" + std::to_string(hist[i] * 16 / std::max<int64_t>(batch, 1)) + ",";
    return s;
}

}  // namespace bat
}  // namespace rbt

using namespace rbt;
using namespace rbt::bat;

static size_t plan_bytes(const rbt_opts *o, int64_t batch, const int64_t *n, const int64_t *nrhs, size_t *desc_off,
                         size_t *order_off, size_t *counter_off, size_t *adj_off, size_t *sys_off)
{
    size_t off = 0;
    *desc_off = off;
    off = (size_t)align256((int64_t)(off + batch * sizeof(SysDesc)));
    *order_off = off;
    off = (size_t)align256((int64_t)(off + batch * sizeof(int)));
    *counter_off = off;
    off = (size_t)align256((int64_t)(off + 256));
    *adj_off = off;
    off = (size_t)align256((int64_t)(off + batch * sizeof(AdjDesc)));
    *sys_off = off;
    for (int64_t i = 0; i < batch; i++) {
        int64_t r = nrhs ? nrhs[i] : 1;
        // float systems that may fall back keep room for the double factors
        Layout L = (o->prec == RBT_F64 || o->fallback) ? sys_layout<double>(n[i], r, o->depth)
                                                        : sys_layout<float>(n[i], r, o->depth);
        off += (size_t)L.total;
    }
    return off;
}

extern "C" {

size_t rbt_solve_batched_workspace(const rbt_opts *opts, int64_t batch, const int64_t *n, const int64_t *nrhs)
{
    if (!opts || batch < 0 || (batch > 0 && !n)) return 0;
    size_t a, b, c, d, e;
    return plan_bytes(opts, batch, n, nrhs, &a, &b, &c, &d, &e);
}

rbt_status rbt_solve_batched_plan(const rbt_opts *opts, int64_t batch, const int64_t *n, const int64_t *nrhs,
                                  const double *const *A, const int64_t *lda, const double *const *B,
                                  const int64_t *ldb, double *const *X, const int64_t *ldx, const uint64_t *seeds,
                                  void *work, size_t work_bytes, cudaStream_t stream)
{
    if (!opts || batch < 0 || batch > INT32_MAX) return RBT_ERR_ARG;
    if (opts->prec != RBT_F64 && opts->prec != RBT_F32) return RBT_ERR_UNSUPPORTED;
    if (opts->depth < 0 || opts->depth > 62 || opts->refine_max < 0 || opts->align < 0 || opts->grid_p < 0 ||
        opts->grid_q < 0)
        return RBT_ERR_ARG;
    // batched systems use the non-tiled reference size (no tiles, no process grid)
    if (opts->align > 1 || opts->grid_p > 1 || opts->grid_q > 1) return RBT_ERR_UNSUPPORTED;
    if (opts->kind != RBT_KIND_SCALED && opts->kind != RBT_KIND_ROTATION) return RBT_ERR_ARG;
    if (opts->kind != RBT_KIND_SCALED) return RBT_ERR_UNSUPPORTED;  // batched systems use the scaled butterflies
    if (batch == 0) return RBT_OK;
    if (!n || !A || !lda || !B || !ldb || !X || !ldx || !work) return RBT_ERR_ARG;
    for (int64_t i = 0; i < batch; i++) {
        int64_t r = nrhs ? nrhs[i] : 1;
        if (n[i] < 1 || r < 1 || lda[i] < n[i] || ldb[i] < n[i] || ldx[i] < n[i] || !A[i] || !B[i] || !X[i])
            return RBT_ERR_ARG;
        if (eff_depth(n[i], opts->depth) > 3 || n[i] > (1 << 20)) return RBT_ERR_UNSUPPORTED;
    }
    PlanInfo P;
    size_t need = plan_bytes(opts, batch, n, nrhs, &P.desc_off, &P.order_off, &P.counter_off, &P.adj_off, &P.sys_off);
    if (work_bytes < need) return RBT_ERR_WORKSPACE;
    P.batch = batch;
    P.prec = opts->prec;
    P.depth = opts->depth;
    P.fallback = opts->fallback ? 1 : 0;
    P.signature = make_signature(batch, n, nrhs, opts->prec, opts->depth);
    std::vector<SysDesc> descs((size_t)batch);
    int64_t off = 0;
    for (int64_t i = 0; i < batch; i++) {
        SysDesc &s = descs[(size_t)i];
        s.n = n[i];
        s.nrhs = nrhs ? nrhs[i] : 1;
        s.A = A[i];
        s.lda = lda[i];
        s.B = B[i];
        s.ldb = ldb[i];
        s.X = X[i];
        s.ldx = ldx[i];
        s.seed = seeds ? seeds[i] : opts->seed + (uint64_t)i;
        s.off = off;
        Layout L = (opts->prec == RBT_F64 || opts->fallback) ? sys_layout<double>(s.n, s.nrhs, opts->depth)
                                                             : sys_layout<float>(s.n, s.nrhs, opts->depth);
        off += L.total;
    }
    // largest systems first: the persistent CTAs then finish together
    std::vector<int> order((size_t)batch);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    char *w = (char *)work;
    RBT_CUDA_TRY(cudaMemcpyAsync(w + P.desc_off, descs.data(), descs.size() * sizeof(SysDesc), cudaMemcpyHostToDevice,
                                 stream));
    RBT_CUDA_TRY(cudaMemcpyAsync(w + P.order_off, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 stream));
    RBT_CUDA_TRY(cudaStreamSynchronize(stream));  // the host vectors die with this call
    std::lock_guard<std::mutex> lk(g_mu);
    g_plans[work] = P;
    return RBT_OK;
}

rbt_status rbt_solve_batched_run(const rbt_opts *opts, void *work, rbt_batched_info *d_infos, cudaStream_t stream)
{
    if (!opts || !work) return RBT_ERR_ARG;
    PlanInfo P;
    int v = 3;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(work);
        if (it == g_plans.end()) return RBT_ERR_ARG;  // not planned
        P = it->second;
        auto t = g_tuned.find(P.signature);
        if (t != g_tuned.end()) v = t->second;
    }
    if (P.batch == 0) return RBT_OK;
    if (!d_infos) return RBT_ERR_ARG;
    if (opts->prec != P.prec || opts->depth != P.depth || (opts->fallback ? 1 : 0) != P.fallback) return RBT_ERR_ARG;
    if (P.prec == RBT_F64)
        return launch_variant<double>(v, P, (char *)work, d_infos, opts->refine_max, opts->tol, stream);
    return launch_variant<float>(v, P, (char *)work, d_infos, opts->refine_max, opts->tol, stream);
}

rbt_status rbt_solve_batched_autotune(const rbt_opts *opts, void *work, rbt_batched_info *d_infos,
                                      cudaStream_t stream, int32_t *chosen, double *best_ms)
{
    if (!opts || !work || !d_infos) return RBT_ERR_ARG;
    PlanInfo P;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(work);
        if (it == g_plans.end()) return RBT_ERR_ARG;
        P = it->second;
    }
    if (P.batch == 0) return RBT_OK;
    cudaEvent_t e0, e1;
    RBT_CUDA_TRY(cudaEventCreate(&e0));
    RBT_CUDA_TRY(cudaEventCreate(&e1));
    int best = 3;
    float best_t = 1e30f;
    for (int v = 0; v < kNumVariants; v++) {
        for (int rep = 0; rep < 2; rep++) {  // first run warms up
            RBT_CUDA_TRY(cudaEventRecord(e0, stream));
            rbt_status s = P.prec == RBT_F64
                               ? launch_variant<double>(v, P, (char *)work, d_infos, opts->refine_max, opts->tol, stream)
                               : launch_variant<float>(v, P, (char *)work, d_infos, opts->refine_max, opts->tol, stream);
            if (s != RBT_OK) return s;
            RBT_CUDA_TRY(cudaEventRecord(e1, stream));
            RBT_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            RBT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 1 && ms < best_t) {
                best_t = ms;
                best = v;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_tuned[P.signature] = best;
    }
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return RBT_OK;
}

rbt_status rbt_solve_batched_adjoint(const rbt_opts *opts, void *work, int64_t batch, const double *const *G,
                                     const int64_t *ldg, double *const *Y, const int64_t *ldy, double *const *GA,
                                     const int64_t *ldga, rbt_batched_info *d_infos, cudaStream_t stream)
{
    if (!opts || !work) return RBT_ERR_ARG;
    PlanInfo P;
    int v = 3;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_plans.find(work);
        if (it == g_plans.end()) return RBT_ERR_ARG;
        P = it->second;
        auto t = g_tuned.find(P.signature);
        if (t != g_tuned.end()) v = t->second;
    }
    if (batch != P.batch || opts->prec != P.prec || opts->depth != P.depth) return RBT_ERR_ARG;
    if (batch == 0) return RBT_OK;
    if (!G || !ldg || !Y || !ldy || !d_infos || (GA && !ldga)) return RBT_ERR_ARG;
    std::vector<SysDesc> descs((size_t)batch);
    char *w = (char *)work;
    RBT_CUDA_TRY(cudaMemcpyAsync(descs.data(), w + P.desc_off, descs.size() * sizeof(SysDesc), cudaMemcpyDeviceToHost,
                                 stream));
    RBT_CUDA_TRY(cudaStreamSynchronize(stream));
    std::vector<AdjDesc> adj((size_t)batch);
    for (int64_t i = 0; i < batch; i++) {
        const int64_t n = descs[(size_t)i].n;
        if (!G[i] || !Y[i] || ldg[i] < n || ldy[i] < n || (GA && GA[i] && ldga[i] < n)) return RBT_ERR_ARG;
        adj[(size_t)i] = AdjDesc{G[i], ldg[i], Y[i], ldy[i], GA ? GA[i] : nullptr, GA ? ldga[i] : 0};
    }
    RBT_CUDA_TRY(cudaMemcpyAsync(w + P.adj_off, adj.data(), adj.size() * sizeof(AdjDesc), cudaMemcpyHostToDevice,
                                 stream));
    int *counter = (int *)(w + P.counter_off);
    RBT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), stream));
    int sms = device_sm_count(), per_sm = 1, grid = 1;
    const SysDesc *dd = (const SysDesc *)(w + P.desc_off);
    const AdjDesc *da = (const AdjDesc *)(w + P.adj_off);
    const int *order = (const int *)(w + P.order_off);
    char *sys_base = w + P.sys_off;
#define RBT_ADJ_LAUNCH(T_, NT_, NB_)                                                                           \
    {                                                                                                          \
        RBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_adjoint_kernel<T_, NT_, NB_>, \
                                                                   NT_, 0));                                    \
        grid = sms * (per_sm > 0 ? per_sm : 1);                                                                \
        if (grid > batch) grid = (int)batch;                                                                   \
        batched_adjoint_kernel<T_, NT_, NB_><<<grid, NT_, 0, stream>>>(dd, da, order, (int)batch, counter,     \
                                                                       d_infos, sys_base, P.depth,             \
                                                                       opts->refine_max, opts->tol);           \
    }
    if (P.prec == RBT_F64) {
        switch (v) {
        case 0: RBT_ADJ_LAUNCH(double, 128, 16) break;
        case 1: RBT_ADJ_LAUNCH(double, 128, 32) break;
        case 2: RBT_ADJ_LAUNCH(double, 256, 16) break;
        default: RBT_ADJ_LAUNCH(double, 256, 32) break;
        }
    } else {
        switch (v) {
        case 0: RBT_ADJ_LAUNCH(float, 128, 16) break;
        case 1: RBT_ADJ_LAUNCH(float, 128, 32) break;
        case 2: RBT_ADJ_LAUNCH(float, 256, 16) break;
        default: RBT_ADJ_LAUNCH(float, 256, 32) break;
        }
    }
#undef RBT_ADJ_LAUNCH
    RBT_LAUNCH_CHECK();
    RBT_CUDA_TRY(cudaStreamSynchronize(stream));  // the host descriptor vector dies with this call
    return RBT_OK;
}

int32_t rbt_solve_batched_variant(void *work, int32_t *threads, int32_t *nb)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(work);
    if (it == g_plans.end()) return -1;
    int v = 3;
    auto t = g_tuned.find(it->second.signature);
    if (t != g_tuned.end()) v = t->second;
    if (threads) *threads = kVariants[v].nt;
    if (nb) *nb = kVariants[v].nb;
    return v;
}

}  // extern "C"
