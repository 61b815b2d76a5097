// Device code of the batched RBT solver (one CTA per system, persistent
// kernels); included by the kernel objects (batched_kernels.cu, one
// precision and variant each) and by the host planner (batched.cu), which
// uses the descriptors and the scratch layout only.
#pragma once

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
// Threads per SM the kernels' launch bounds ask room for: 512, i.e. at most
// 128 registers a thread, two CTAs of 256 threads (or four of 128) per SM.
// Uncapped, the compiler gives the whole solver 255 registers (one CTA per
// SM) for the sake of its rarely used depth-3 transform, and the solver is
// latency-bound: two CTAs per SM are faster despite some spills there.
constexpr int kMinCtaThreads = 512;

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

// The working-precision value of a double (rounded; the exact leading 48
// bits for double-float) and back.
__device__ __forceinline__ double widen_of(double v) { return v; }
__device__ __forceinline__ double widen_of(float v) { return (double)v; }
__device__ __forceinline__ double widen_of(df64 v) { return df_to_double(v); }

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
                At[i + j * n] = narrow_to<T>(p);
            }
        } else if (ds < 3) {
            for (int64_t e = tid; e < h * h; e += NT) {
                const int64_t gr = e % h, gc = e / h;
                if (ds == 1)
                    transform_group<1, T>(n, h, ds, ds + 1, d, U, V, n, S.A, S.lda, At, n, gr, gc);
                else
                    transform_group<2, T>(n, h, ds, ds + 1, d, U, V, n, S.A, S.lda, At, n, gr, gc);
            }
        } else {
            // depth 3: eight lanes per 8 x 8 group, one row each (NT is a
            // multiple of 8, so the eight lanes of a group share every trip)
            const int s = tid & 7;
            const unsigned mask = 0xFFu << (tid & 24);
            for (int64_t e = tid >> 3; e < h * h; e += NT / 8) {
                const int64_t gr = e % h, gc = e / h;
                transform_group_rows<3, T>(n, h, ds, ds + 1, d, U, V, n, S.A, S.lda, At, n, gr, gc, s, mask);
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
    for (int64_t e = tid; e < n * nrhs; e += NT) Xt[e] = narrow_to<T>(S.X[e % n + (e / n) * S.ldx]);
    __syncthreads();
    cta_lu_solve<T, NT, NB>(n, nrhs, At, Xt, s_diag);
    for (int64_t e = tid; e < n * nrhs; e += NT) S.X[e % n + (e / n) * S.ldx] = widen_of(Xt[e]);
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
        for (int64_t e = tid; e < n * nrhs; e += NT) Xt[e] = narrow_to<T>(R[e]);
        __syncthreads();
        cta_lu_solve<T, NT, NB>(n, nrhs, At, Xt, s_diag);
        for (int64_t e = tid; e < n * nrhs; e += NT) R[e] = widen_of(Xt[e]);
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

// One persistent launch over the queue.  Float kernels with fallback redo a
// system that misses tol in double-float on the same A~ (fell_back = 1);
// a system that misses it there too is left for a second launch of the
// double kernel with redo set, which solves only the systems whose info is
// not RBT_OK, in double (fell_back = 2).
template <typename T, int NT, int NB>
__global__ void __launch_bounds__(NT, kMinCtaThreads / NT)
batched_kernel(const SysDesc *__restrict__ sys, const int *__restrict__ order, int batch, int *counter,
               rbt_batched_info *infos, char *work, int d, int refine_max, double tol, int fallback, int redo)
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
        int prior = 0;
        if (redo) {
            const rbt_batched_info first = infos[id];  // the same value in every thread
            if (first.status == RBT_OK) continue;
            prior = first.iters;
        }
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
        if (redo) {
            info.fell_back = 2;
            info.iters += prior;
        }
        if constexpr (sizeof(T) < sizeof(double)) {
            if (fallback && info.status != RBT_OK) {
                // "responsibly reckless" fallback (Sec. 5) on the same A~, in
                // double-float: about 48 bits on the FP32 pipes, several times
                // faster than double on this GPU
                prior = info.iters;
                solve_sys<df64, NT, NB>(S, w, d, refine_max, tol, smem_raw, &s_flag, red, &s_anorm, info);
                info.fell_back = 1;
                info.iters += prior;
            }
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
    for (int64_t e = tid; e < n * nrhs; e += NT) Xt[e] = narrow_to<T>(D.Y[e % n + (e / n) * D.ldy]);
    __syncthreads();
    cta_lu_solve_t<T, NT, NB>(n, nrhs, At, Xt, s_blk);
    for (int64_t e = tid; e < n * nrhs; e += NT) D.Y[e % n + (e / n) * D.ldy] = widen_of(Xt[e]);
    __syncthreads();
    cta_vec<NT>(n, d, U, 0, D.Y, D.ldy, nrhs);
    if (tid == 0) *s_anorm = -1.0;
    __syncthreads();
    double berr = cta_residual_t<NT>(n, nrhs, S.A, S.lda, D.Y, D.ldy, D.G, D.ldg, R, s_anorm, red);
    info.berr_unrefined = berr;
    int it = 0;
    while (!(berr <= tol) && it < refine_max) {
        cta_vec<NT>(n, d, V, 1, R, n, nrhs);
        for (int64_t e = tid; e < n * nrhs; e += NT) Xt[e] = narrow_to<T>(R[e]);
        __syncthreads();
        cta_lu_solve_t<T, NT, NB>(n, nrhs, At, Xt, s_blk);
        for (int64_t e = tid; e < n * nrhs; e += NT) R[e] = widen_of(Xt[e]);
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
// (the double-float or double ones when that system fell back).
template <typename T, int NT, int NB>
__global__ void __launch_bounds__(NT, kMinCtaThreads / NT)
batched_adjoint_kernel(const SysDesc *__restrict__ sys, const AdjDesc *__restrict__ adj,
                       const int *__restrict__ order, int batch, int *counter, rbt_batched_info *infos, char *work,
                       int d, int refine_max, double tol, int redo)
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
        // systems whose factors are double (fell_back = 2) belong to the
        // double kernel's redo launch; a redo launch takes only those
        if (redo ? fwd.fell_back != 2 : (sizeof(T) < sizeof(double) && fwd.fell_back == 2)) continue;
        char *w = work + S.off;
        rbt_batched_info info;
        info.zero_pivot = -1;
        info.fell_back = fwd.fell_back;
        info.reserved = 0;
        if constexpr (sizeof(T) < sizeof(double)) {
            if (fwd.fell_back == 1)
                adjoint_sys<df64, NT, NB>(S, D, w, d, refine_max, tol, red, &s_anorm, (df64 *)s_blk, info);
            else
                adjoint_sys<T, NT, NB>(S, D, w, d, refine_max, tol, red, &s_anorm, (T *)s_blk, info);
        } else {
            adjoint_sys<T, NT, NB>(S, D, w, d, refine_max, tol, red, &s_anorm, (T *)s_blk, info);
        }
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

struct Variant {
    int nt, nb;
};
// threads per CTA and GENP block size of the compiled variants
constexpr Variant kVariants[] = {{128, 16}, {128, 32}, {256, 16}, {256, 32}};
constexpr int kNumVariants = 4;

// Arguments of one launch of the solver or of its adjoint.
struct BatchedLaunch {
    const SysDesc *descs;
    const AdjDesc *adj;  // adjoint only
    const int *order;
    int batch;
    int *counter;
    rbt_batched_info *infos;
    char *sys_base;
    int depth, refine_max;
    double tol;
    int fallback;
    int redo;  // double kernels: only the systems a float launch left unsolved
};

// Launch the solver / its adjoint for working precision T and variant
// (NT, NB); each instantiation is compiled in an object of its own.
template <typename T, int NT, int NB> rbt_status run_batched(const BatchedLaunch &a, cudaStream_t stream);
template <typename T, int NT, int NB> rbt_status run_adjoint(const BatchedLaunch &a, cudaStream_t stream);

}  // namespace bat
}  // namespace rbt
