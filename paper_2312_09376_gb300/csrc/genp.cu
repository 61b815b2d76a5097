// Gaussian elimination with no pivoting and its triangular solves (sm_103a).
//
// Blocked right-looking LU without row exchanges (Sec. 1; the GENP step of
// Eq. precond).  Without pivoting the diagonal block needs nothing from the
// rows below it, so each block step is
//   1. factor the kb x kb diagonal block in shared memory (one CTA),
//   2. U12 <- L11^{-1} A12 and L21 <- A21 U11^{-1} (independent columns /
//      rows, both at once),
//   3. A22 <- A22 - L21 U12 (the dense contraction: all but O(n^2 kb) of the
//      2n^3/3 flops).
// Step 3 runs on the tensor cores for the TF32 / BF16 precisions (gemm_tc.cu)
// and as a register-tiled SIMT kernel for double and float.
//
// Pivot status: d_info starts at -1.  The diagonal kernel writes the global
// index of the first pivot that is zero or not finite and stops; every later
// kernel of the factorization reads d_info first and returns at once when it
// is set, so the enqueued remainder costs almost nothing.
#include "common.cuh"
#include "genp_internal.cuh"
#include "df64.cuh"

#include <type_traits>

namespace rbt {

__device__ __forceinline__ bool info_set(const int64_t *info)
{
    return *((volatile const int64_t *)info) >= 0;
}

template <typename T> __device__ __forceinline__ bool bad_pivot(T p)
{
    return p == T(0) || !isfinite(p);
}

// ---------------------------------------------------------------- diagonal

// Unblocked Doolittle on the kb x kb block at (k0, k0); kb <= kMaxNB.  256
// threads: thread (i0, q) = (tid % 64, tid / 64) updates rows i0 + 64 r in
// the columns c = q (mod 4), so each elimination step is one barrier and a
// quarter row of independent multiply-adds per row of the thread.  The
// multipliers l_ij are kept in registers and stored into column j during the
// next step, when no thread reads column j any more.
template <typename T>
__global__ void __launch_bounds__(256) diag_factor_kernel(int64_t k0, int kb, T *A, int64_t lda, int64_t *info)
{
    constexpr int RPT = kMaxNB / 64;  // rows per thread
    extern __shared__ unsigned char smem_raw[];
    T *a = reinterpret_cast<T *>(smem_raw);  // kb x kb, column-major, ld = kb
    if (info_set(info)) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < kb * kb; e += nt) {
        int i = e % kb, j = e / kb;
        a[e] = A[(k0 + i) + (k0 + j) * lda];
    }
    __syncthreads();
    const int i0 = tid % 64, q = tid / 64;
    T pend[RPT];
    int pend_j = -1;
    for (int j = 0; j < kb; j++) {
        const T p = a[j + j * kb];
        if (bad_pivot(p)) {  // every thread reads the same pivot: a uniform exit
            if (tid == 0) *info = k0 + j;
            break;
        }
        if (pend_j >= 0) {
#pragma unroll
            for (int r = 0; r < RPT; r++) {
                const int i = i0 + 64 * r;
                if (i > pend_j && i < kb) a[i + pend_j * kb] = pend[r];
            }
            pend_j = -1;
        }
        const int c0 = j + 1 + ((q - (j + 1)) & 3);
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            const int i = i0 + 64 * r;
            if (i > j && i < kb) {
                const T l = a[i + j * kb] / p;
                for (int c = c0; c < kb; c += 4) a[i + c * kb] -= l * a[j + c * kb];
                pend[r] = l;
            }
        }
        if (q == 0) pend_j = j;
        __syncthreads();
    }
    if (pend_j >= 0) {
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            const int i = i0 + 64 * r;
            if (i > pend_j && i < kb) a[i + pend_j * kb] = pend[r];
        }
    }
    __syncthreads();
    // write back (the partial factor too when stopped: the caller ignores it)
    for (int e = tid; e < kb * kb; e += nt) {
        int ii = e % kb, jj = e / kb;
        A[(k0 + ii) + (k0 + jj) * lda] = a[e];
    }
}

// ------------------------------------------------------------------ TRSMs

// Both TRSMs of a panel step in one launch, four lanes per vector:
//   blocks [0, nbu):        U12 <- L11^{-1} A12, a vector is a column of A12
//                           (unit forward substitution, x_i = a_i - sum_{p<i} L_ip x_p);
//   blocks [nbu, nbu+nbl):  L21 <- A21 U11^{-1}, a vector is a row of A21
//                           (x_j = (a_j - sum_{p<j} x_p U_pj) / U_jj).
// 64 vectors per CTA, vector v on lanes 4 v' .. 4 v' + 3 of one warp; lane q
// owns the entries i = q (mod 4) of its vector.  The substitution is
// right-looking in blocks of four entries: the four lanes finish entries
// j0 .. j0 + 3 (lane q the entry j0 + q: scale by the reciprocal of the
// pivot, broadcast by shuffle, the later lanes subtract it), then every lane
// subtracts the four new values from each entry it owns past the block.
// The serial part of a block is four scalings and shuffles; the rest are
// independent multiply-adds (the panel has only (n - k) / 64 CTAs of work).
constexpr int kTrsmVec = 64, kTrsmLanes = 4, kTrsmThreads = kTrsmVec * kTrsmLanes;
// padded shared-memory strides: the four lanes of a vector read the diagonal
// block at i, i+1, i+2, i+3 and the vector's entries at the same offsets;
// ld kb + 1 for the block and 68 for the vectors keep them off one bank
constexpr int kTrsmXS = kTrsmVec + 4;
template <typename T> constexpr size_t trsm_smem_bytes(int kb)
{
    return ((size_t)kb * (kb + 1) + (size_t)kb * kTrsmXS + (size_t)kb) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(kTrsmThreads) trsm_panel_kernel(int64_t k0, int kb, int64_t n, T *A, int64_t lda,
                                                                  int nbu, const int64_t *info)
{
    extern __shared__ unsigned char smem_raw[];
    const int ldm = kb + 1;
    T *Mt = reinterpret_cast<T *>(smem_raw);  // kb x kb diagonal block (ld kb + 1)
    T *X = Mt + kb * ldm;                      // kb x 64, X[e * kTrsmXS + v]
    T *rd = X + kb * kTrsmXS;                  // 1 / U_jj (the L21 part)
    if (info_set(info)) return;
    const int tid = threadIdx.x;
    const int q = tid % kTrsmLanes, v = tid / kTrsmLanes;
    const bool upper = (int)blockIdx.x < nbu;  // the U12 part
    const int64_t v0 = k0 + kb + (int64_t)(upper ? blockIdx.x : blockIdx.x - nbu) * kTrsmVec;
    for (int e = tid; e < kb * kb; e += kTrsmThreads) {
        const int i = e % kb, j = e / kb;
        Mt[i + j * ldm] = A[(k0 + i) + (k0 + j) * lda];
    }
    // coalesced tile load: consecutive threads walk down a column of A
    for (int e = tid; e < kb * kTrsmVec; e += kTrsmThreads) {
        if (upper) {
            const int i = e % kb, c = e / kb;
            const int64_t col = v0 + c;
            X[i * kTrsmXS + c] = col < n ? A[(k0 + i) + col * lda] : T(0);
        } else {
            const int r = e % kTrsmVec, j = e / kTrsmVec;
            const int64_t row = v0 + r;
            X[j * kTrsmXS + r] = row < n ? A[row + (k0 + j) * lda] : T(0);
        }
    }
    __syncthreads();
    if (!upper) {
        for (int j = tid; j < kb; j += kTrsmThreads) rd[j] = T(1) / Mt[j + j * ldm];
        __syncthreads();
    }
    // m(i, j): the factor entry that couples entry j into entry i
    auto coef = [&](int i, int j) { return upper ? Mt[i + j * ldm] : Mt[j + i * ldm]; };
    const int gbase = (tid & 31) & ~(kTrsmLanes - 1);  // first lane of this vector's group
    for (int j0 = 0; j0 < kb; j0 += kTrsmLanes) {
        const int jn = kb - j0 < kTrsmLanes ? kb - j0 : kTrsmLanes;  // the same on every lane
        T own = q < jn ? X[(j0 + q) * kTrsmXS + v] : T(0);
        T xs[kTrsmLanes];
#pragma unroll
        for (int jj = 0; jj < kTrsmLanes; jj++) {
            xs[jj] = T(0);
            if (jj < jn) {
                T x = own;
                if (!upper && q == jj) x = x * rd[j0 + jj];
                if (q == jj) own = x;
                x = shfl_idx(x, gbase | jj);
                xs[jj] = x;
                if (q > jj && q < jn) own = own - coef(j0 + q, j0 + jj) * x;
            }
        }
        if (q < jn) X[(j0 + q) * kTrsmXS + v] = own;
        if (jn == kTrsmLanes) {
            for (int i = j0 + kTrsmLanes + q; i < kb; i += kTrsmLanes) {
                T a = X[i * kTrsmXS + v];
#pragma unroll
                for (int jj = 0; jj < kTrsmLanes; jj++) a = a - coef(i, j0 + jj) * xs[jj];
                X[i * kTrsmXS + v] = a;
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < kb * kTrsmVec; e += kTrsmThreads) {
        if (upper) {
            const int i = e % kb, c = e / kb;
            const int64_t col = v0 + c;
            if (col < n) A[(k0 + i) + col * lda] = X[i * kTrsmXS + c];
        } else {
            const int r = e % kTrsmVec, j = e / kTrsmVec;
            const int64_t row = v0 + r;
            if (row < n) A[row + (k0 + j) * lda] = X[j * kTrsmXS + r];
        }
    }
}

// ------------------------------------------------------------- SIMT GEMM

// C (M x N) -= Am (M x K) * Bm (K x N); column-major; register tiles TM x TN.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_sub_kernel(int64_t M, int64_t N, int K, const T *__restrict__ Am, int64_t lda_a,
                const T *__restrict__ Bm, int64_t ldb_b, T *C, int64_t ldc, const int64_t *info)
{
    constexpr int NT = (BM / TM) * (BN / TN);
    __shared__ T sa[BK][BM + 1];
    __shared__ T sb[BK][BN + 1];
    if (info && info_set(info)) return;
    const int tid = threadIdx.x;
    const int tx = tid % (BM / TM), ty = tid / (BM / TM);
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = T(0);

    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NT) {
            int i = e % BM, k = e / BM;
            int64_t gi = m0 + i;
            sa[k][i] = (gi < M && k0 + k < K) ? Am[gi + (int64_t)(k0 + k) * lda_a] : T(0);
        }
        for (int e = tid; e < BN * BK; e += NT) {
            int k = e % BK, j = e / BK;
            int64_t gj = n0 + j;
            sb[k][j] = (gj < N && k0 + k < K) ? Bm[(k0 + k) + gj * ldb_b] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; k++) {
            T ra[TM], rb[TN];
#pragma unroll
            for (int i = 0; i < TM; i++) ra[i] = sa[k][tx + i * (BM / TM)];
#pragma unroll
            for (int j = 0; j < TN; j++) rb[j] = sb[k][ty + j * (BN / TN)];
#pragma unroll
            for (int i = 0; i < TM; i++)
#pragma unroll
                for (int j = 0; j < TN; j++) acc[i][j] = fma(ra[i], rb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TN; j++) {
        int64_t gj = n0 + ty + j * (BN / TN);
        if (gj >= N) continue;
#pragma unroll
        for (int i = 0; i < TM; i++) {
            int64_t gi = m0 + tx + i * (BM / TM);
            if (gi < M) C[gi + gj * ldc] -= acc[i][j];
        }
    }
}

// Double-float C -= A B.  The product of two pairs keeps the exact error of
// the leading product (one FMA) and the two cross terms; the running sum keeps
// its leading part exact with TwoSum and gathers every error term in a float
// accumulator that is folded in once at the end (about 12 FP32 operations per
// multiply-add instead of about 18 with a renormalized sum each step).
constexpr int kDfBM = 64, kDfBN = 64, kDfBK = 16, kDfTM = 4, kDfTN = 4;

__global__ void __launch_bounds__(256)
gemm_sub_df64_kernel(int64_t M, int64_t N, int K, const df64 *__restrict__ Am, int64_t lda_a,
                     const df64 *__restrict__ Bm, int64_t ldb_b, df64 *C, int64_t ldc, const int64_t *info)
{
    __shared__ float sah[kDfBK][kDfBM + 4], sal[kDfBK][kDfBM + 4];
    __shared__ float sbh[kDfBK][kDfBN + 4], sbl[kDfBK][kDfBN + 4];
    if (info && info_set(info)) return;
    const int tid = threadIdx.x;
    const int tx = tid % (kDfBM / kDfTM), ty = tid / (kDfBM / kDfTM);
    const int64_t m0 = (int64_t)blockIdx.x * kDfBM, n0 = (int64_t)blockIdx.y * kDfBN;
    float ah[kDfTM][kDfTN], al[kDfTM][kDfTN];
#pragma unroll
    for (int i = 0; i < kDfTM; i++)
#pragma unroll
        for (int j = 0; j < kDfTN; j++) ah[i][j] = al[i][j] = 0.f;

    for (int k0 = 0; k0 < K; k0 += kDfBK) {
        for (int e = tid; e < kDfBM * kDfBK; e += 256) {
            int i = e % kDfBM, k = e / kDfBM;
            int64_t gi = m0 + i;
            df64 v = (gi < M && k0 + k < K) ? Am[gi + (int64_t)(k0 + k) * lda_a] : df64(0);
            sah[k][i] = v.hi;
            sal[k][i] = v.lo;
        }
        for (int e = tid; e < kDfBN * kDfBK; e += 256) {
            int k = e % kDfBK, j = e / kDfBK;
            int64_t gj = n0 + j;
            df64 v = (gj < N && k0 + k < K) ? Bm[(k0 + k) + gj * ldb_b] : df64(0);
            sbh[k][j] = v.hi;
            sbl[k][j] = v.lo;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kDfBK; k++) {
            float xh[kDfTM], xl[kDfTM], yh[kDfTN], yl[kDfTN];
#pragma unroll
            for (int i = 0; i < kDfTM; i++) {
                xh[i] = sah[k][tx + i * (kDfBM / kDfTM)];
                xl[i] = sal[k][tx + i * (kDfBM / kDfTM)];
            }
#pragma unroll
            for (int j = 0; j < kDfTN; j++) {
                yh[j] = sbh[k][ty + j * (kDfBN / kDfTN)];
                yl[j] = sbl[k][ty + j * (kDfBN / kDfTN)];
            }
#pragma unroll
            for (int i = 0; i < kDfTM; i++)
#pragma unroll
                for (int j = 0; j < kDfTN; j++) {
                    float p = __fmul_rn(xh[i], yh[j]);
                    float pe = __fmaf_rn(xh[i], yh[j], -p);
                    float s, se;
                    two_sum(ah[i][j], p, s, se);
                    ah[i][j] = s;
                    float l = __fadd_rn(al[i][j], __fadd_rn(se, pe));
                    l = __fmaf_rn(xh[i], yl[j], l);
                    al[i][j] = __fmaf_rn(xl[i], yh[j], l);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kDfTN; j++) {
        int64_t gj = n0 + ty + j * (kDfBN / kDfTN);
        if (gj >= N) continue;
#pragma unroll
        for (int i = 0; i < kDfTM; i++) {
            int64_t gi = m0 + tx + i * (kDfBM / kDfTM);
            if (gi < M) {
                df64 acc = df_norm(ah[i][j], al[i][j]);
                C[gi + gj * ldc] = C[gi + gj * ldc] - acc;
            }
        }
    }
}

// Large double-float updates: a persistent kernel, one 256-thread CTA per SM,
// 128 x 128 output tiles dealt round-robin, each thread an 8 x 8 register
// tile (two 4-row and two 4-column strips).  Operand k-slices of 16 travel
// by cp.async (8-byte copies: a leading dimension may be odd) into a
// 3-stage shared-memory ring that runs on across tile boundaries, so the
// next tile's first slices and, through an L2 prefetch, its block of C
// arrive while the current tile still computes.
constexpr int kDf2BM = 128, kDf2BN = 128, kDf2BK = 16, kDf2Stages = 3;
constexpr int kDf2StageElems = kDf2BK * kDf2BM + kDf2BN * kDf2BK;   // df64 elements per stage
constexpr size_t kDf2Smem = (size_t)kDf2Stages * kDf2StageElems * sizeof(df64);

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    // src-size 0 fills the 8 bytes with zeros and reads nothing
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(256, 1)
gemm_sub_df64_pipe_kernel(int64_t M, int64_t N, int K, const df64 *__restrict__ Am, int64_t lda_a,
                          const df64 *__restrict__ Bm, int64_t ldb_b, df64 *__restrict__ C, int64_t ldc,
                          const int64_t *info)
{
    extern __shared__ __align__(16) unsigned char df2_smem[];
    df64 *ring = reinterpret_cast<df64 *>(df2_smem);
    if (info && info_set(info)) return;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t tiles_m = (M + kDf2BM - 1) / kDf2BM;
    const int64_t ntiles = tiles_m * ((N + kDf2BN - 1) / kDf2BN);
    if ((int64_t)blockIdx.x >= ntiles) return;
    const int ksteps = (K + kDf2BK - 1) / kDf2BK;
    const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const int64_t total = my_tiles * ksteps;

    // stage s of this CTA's sequence: tile blockIdx.x + (s / ksteps) * gridDim.x, k-slice s % ksteps
    auto issue = [&](int64_t s) {
        const int64_t t = blockIdx.x + (s / ksteps) * gridDim.x;
        const int k0 = (int)(s % ksteps) * kDf2BK;
        const int64_t m0 = (t % tiles_m) * kDf2BM, n0 = (t / tiles_m) * kDf2BN;
        df64 *sa = ring + (s % kDf2Stages) * kDf2StageElems;
        df64 *sb = sa + kDf2BK * kDf2BM;
#pragma unroll
        for (int q = 0; q < (kDf2BM * kDf2BK) / 256; q++) {
            const int e = tid + q * 256;
            const int i = e % kDf2BM, k = e / kDf2BM;
            const bool ok = m0 + i < M && k0 + k < K;
            cp_async8(sa + k * kDf2BM + i, ok ? Am + (m0 + i) + (int64_t)(k0 + k) * lda_a : Am, ok);
        }
#pragma unroll
        for (int q = 0; q < (kDf2BN * kDf2BK) / 256; q++) {
            const int e = tid + q * 256;
            const int k = e % kDf2BK, j = e / kDf2BK;
            const bool ok = n0 + j < N && k0 + k < K;
            cp_async8(sb + j * kDf2BK + k, ok ? Bm + (k0 + k) + (n0 + j) * ldb_b : Bm, ok);
        }
    };

#pragma unroll
    for (int s = 0; s < kDf2Stages - 1; s++) {
        if (s < total) issue(s);
        cp_async_commit();
    }
    float ah[8][8], al[8][8];
    for (int64_t s = 0; s < total; s++) {
        cp_async_wait<kDf2Stages - 2>();
        // every thread's copies of stage s have landed, and every thread is
        // done with stage s - 1, whose buffer the next issue refills
        __syncthreads();
        if (s + kDf2Stages - 1 < total) issue(s + kDf2Stages - 1);
        cp_async_commit();
        const int kstep = (int)(s % ksteps);
        const int64_t t = blockIdx.x + (s / ksteps) * gridDim.x;
        const int64_t m0 = (t % tiles_m) * kDf2BM, n0 = (t / tiles_m) * kDf2BN;
        if (kstep == 0) {
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) ah[i][j] = al[i][j] = 0.f;
            // pull this CTA's next block of C towards L2: 128 columns, nine
            // addresses each (one per 16 rows, plus the last row)
            const int64_t tn = t + gridDim.x;
            if (tn < ntiles) {
                const int64_t pm = (tn % tiles_m) * kDf2BM, pn = (tn / tiles_m) * kDf2BN;
                for (int q = tid; q < kDf2BN * 9; q += 256) {
                    const int c = q / 9, r = q % 9;
                    const int64_t gi = pm + (r < 8 ? r * 16 : kDf2BM - 1), gj = pn + c;
                    if (gi < M && gj < N)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(C + gi + gj * ldc));
                }
            }
        }
        const df64 *sa = ring + (s % kDf2Stages) * kDf2StageElems;
        const df64 *sb = sa + kDf2BK * kDf2BM;
#pragma unroll 2
        for (int k = 0; k < kDf2BK; k++) {
            float xh[8], xl[8], yh[8], yl[8];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const float4 u0 = *reinterpret_cast<const float4 *>(sa + k * kDf2BM + h * 64 + tx * 4);
                const float4 u1 = *reinterpret_cast<const float4 *>(sa + k * kDf2BM + h * 64 + tx * 4 + 2);
                xh[h * 4 + 0] = u0.x; xl[h * 4 + 0] = u0.y;
                xh[h * 4 + 1] = u0.z; xl[h * 4 + 1] = u0.w;
                xh[h * 4 + 2] = u1.x; xl[h * 4 + 2] = u1.y;
                xh[h * 4 + 3] = u1.z; xl[h * 4 + 3] = u1.w;
#pragma unroll
                for (int jj = 0; jj < 4; jj++) {
                    const float2 v = *reinterpret_cast<const float2 *>(sb + (h * 64 + ty * 4 + jj) * kDf2BK + k);
                    yh[h * 4 + jj] = v.x;
                    yl[h * 4 + jj] = v.y;
                }
            }
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    float p = __fmul_rn(xh[i], yh[j]);
                    float pe = __fmaf_rn(xh[i], yh[j], -p);
                    float s2, se;
                    two_sum(ah[i][j], p, s2, se);
                    ah[i][j] = s2;
                    float l = __fadd_rn(al[i][j], __fadd_rn(se, pe));
                    l = __fmaf_rn(xh[i], yl[j], l);
                    al[i][j] = __fmaf_rn(xl[i], yh[j], l);
                }
        }
        if (kstep == ksteps - 1) {
            // C -= acc, two columns (16 entries) per batch so that their loads overlap
#pragma unroll
            for (int jb = 0; jb < 8; jb += 2) {
                df64 cv[2][8];
#pragma unroll
                for (int jj = 0; jj < 2; jj++) {
                    const int j = jb + jj;
                    const int64_t gj = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int64_t gi = m0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
                        cv[jj][i] = (gi < M && gj < N) ? C[gi + gj * ldc] : df64(0);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 2; jj++) {
                    const int j = jb + jj;
                    const int64_t gj = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int64_t gi = m0 + (i < 4 ? tx * 4 + i : 64 + tx * 4 + (i - 4));
                        if (gi < M && gj < N) C[gi + gj * ldc] = cv[jj][i] - df_norm(ah[i][j], al[i][j]);
                    }
                }
            }
        }
    }
    cp_async_wait<0>();
}

template <typename T>
rbt_status gemm_sub_simt(int64_t M, int64_t N, int K, const T *Am, int64_t lda_a, const T *Bm, int64_t ldb_b,
                         T *C, int64_t ldc, const int64_t *info, cudaStream_t stream)
{
    if (M <= 0 || N <= 0 || K <= 0) return RBT_OK;
    if (std::is_same<T, df64>::value) {
        if (M >= 2048 && N >= 2048) {
            // large updates: the persistent pipelined 128 x 128 kernel, one CTA per SM
            static PerDeviceOnce once;
            rbt_status cst = smem_opt_in(once, gemm_sub_df64_pipe_kernel, (int)kDf2Smem);
            if (cst != RBT_OK) return cst;
            const int64_t ntiles = cdiv(M, kDf2BM) * cdiv(N, kDf2BN);
            const int64_t grid = std::min<int64_t>(ntiles, device_sm_count());
            gemm_sub_df64_pipe_kernel<<<(unsigned)grid, 256, kDf2Smem, stream>>>(
                M, N, K, (const df64 *)Am, lda_a, (const df64 *)Bm, ldb_b, (df64 *)C, ldc, info);
        } else {
            dim3 grid((unsigned)cdiv(M, kDfBM), (unsigned)cdiv(N, kDfBN));
            gemm_sub_df64_kernel<<<grid, 256, 0, stream>>>(M, N, K, (const df64 *)Am, lda_a, (const df64 *)Bm, ldb_b,
                                                           (df64 *)C, ldc, info);
        }
    } else if (sizeof(T) == 8) {
        dim3 grid((unsigned)cdiv(M, 64), (unsigned)cdiv(N, 64));
        gemm_sub_kernel<T, 64, 64, 16, 4, 4><<<grid, 256, 0, stream>>>(M, N, K, Am, lda_a, Bm, ldb_b, C, ldc, info);
    } else {
        dim3 grid((unsigned)cdiv(M, 128), (unsigned)cdiv(N, 128));
        gemm_sub_kernel<T, 128, 128, 16, 8, 8><<<grid, 256, 0, stream>>>(M, N, K, Am, lda_a, Bm, ldb_b, C, ldc, info);
    }
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

template rbt_status gemm_sub_simt<double>(int64_t, int64_t, int, const double *, int64_t, const double *, int64_t,
                                          double *, int64_t, const int64_t *, cudaStream_t);
template rbt_status gemm_sub_simt<float>(int64_t, int64_t, int, const float *, int64_t, const float *, int64_t,
                                         float *, int64_t, const int64_t *, cudaStream_t);
template rbt_status gemm_sub_simt<df64>(int64_t, int64_t, int, const df64 *, int64_t, const df64 *, int64_t,
                                        df64 *, int64_t, const int64_t *, cudaStream_t);

// ------------------------------------------------------------ factor driver

template <typename T>
rbt_status genp_panel_steps(int64_t n, T *A, int64_t lda, int64_t *info, int nb, int64_t k0, int64_t k_end,
                            bool trailing_simt, cudaStream_t stream)
{
    for (int64_t k = k0; k < k_end; k += nb) {
        int kb = (int)(n - k < nb ? n - k : nb);
        int64_t rest = n - k - kb;
        {
            ProfScope ps(kProfPanel, stream);
            size_t sm = (size_t)kb * kb * sizeof(T);
            diag_factor_kernel<T><<<1, 256, sm, stream>>>(k, kb, A, lda, info);
            RBT_LAUNCH_CHECK();
            if (rest <= 0) continue;
            size_t sm_t = trsm_smem_bytes<T>(kb);
            const int nbv = (int)cdiv(rest, kTrsmVec);
            trsm_panel_kernel<T><<<(unsigned)(2 * nbv), kTrsmThreads, sm_t, stream>>>(k, kb, n, A, lda, nbv, info);
            RBT_LAUNCH_CHECK();
        }
        if (trailing_simt) {
            ProfScope ps(kProfUpdate, stream);
            T *a21 = A + (k + kb) + k * lda;
            T *a12 = A + k + (k + kb) * lda;
            T *a22 = A + (k + kb) + (k + kb) * lda;
            rbt_status st = gemm_sub_simt<T>(rest, rest, kb, a21, lda, a12, lda, a22, lda, info, stream);
            if (st != RBT_OK) return st;
        }
    }
    return RBT_OK;
}

template rbt_status genp_panel_steps<double>(int64_t, double *, int64_t, int64_t *, int, int64_t, int64_t, bool,
                                             cudaStream_t);
template rbt_status genp_panel_steps<float>(int64_t, float *, int64_t, int64_t *, int, int64_t, int64_t, bool,
                                            cudaStream_t);
template rbt_status genp_panel_steps<df64>(int64_t, df64 *, int64_t, int64_t *, int, int64_t, int64_t, bool,
                                           cudaStream_t);

template <typename T> static rbt_status configure_smem(int nb)
{
    static PerDeviceOnce once;
    return once_per_device(once, [nb]() -> rbt_status {
        size_t sm = (size_t)nb * nb * sizeof(T);
        int tri = (int)trsm_smem_bytes<T>(nb);
        RBT_CUDA_TRY(cudaFuncSetAttribute(diag_factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        RBT_CUDA_TRY(cudaFuncSetAttribute(trsm_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, tri));
        return RBT_OK;
    });
}

rbt_status genp_configure(int prec, int nb)
{
    (void)nb;
    if (is_df64_storage(prec)) return configure_smem<df64>(kMaxNB);
    if (prec == RBT_F64) return configure_smem<double>(kMaxNB);
    return configure_smem<float>(kMaxNB);
}

// ------------------------------------------------------- triangular solves

// Diagonal block solve for every right-hand side: one CTA per column.
// lower: unit lower L11 (trans 0) or U11^T (trans 1, non-unit);
// upper: U11 (trans 0) or L11^T (trans 1, unit).
template <typename T>
__global__ void __launch_bounds__(128) trsv_diag_kernel(int64_t k0, int kb, const T *LU, int64_t lda, T *B,
                                                        int64_t ldb, int lower, int trans)
{
    __shared__ T x[kMaxNB];
    extern __shared__ unsigned char smem_raw[];
    T *M = reinterpret_cast<T *>(smem_raw);  // kb x kb block of LU
    const int tid = threadIdx.x;
    const int64_t c = blockIdx.x;
    for (int e = tid; e < kb * kb; e += blockDim.x) {
        int i = e % kb, j = e / kb;
        M[e] = LU[(k0 + i) + (k0 + j) * lda];
    }
    for (int i = tid; i < kb; i += blockDim.x) x[i] = B[(k0 + i) + c * ldb];
    __syncthreads();
    // op(M)(i, p): entry of the triangular matrix actually solved with
    const bool unit = (lower && !trans) || (!lower && trans);
    if (lower) {
        for (int i = 0; i < kb; i++) {
            if (tid == 0) {
                T xi = x[i];
                if (!unit) xi /= M[i + i * kb];
                x[i] = xi;
            }
            __syncthreads();
            T xi = x[i];
            for (int r = i + 1 + tid; r < kb; r += blockDim.x) {
                T m = trans ? M[i + r * kb] : M[r + i * kb];
                x[r] -= m * xi;
            }
            __syncthreads();
        }
    } else {
        for (int i = kb - 1; i >= 0; i--) {
            if (tid == 0) {
                T xi = x[i];
                if (!unit) xi /= M[i + i * kb];
                x[i] = xi;
            }
            __syncthreads();
            T xi = x[i];
            for (int r = tid; r < i; r += blockDim.x) {
                T m = trans ? M[i + r * kb] : M[r + i * kb];
                x[r] -= m * xi;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < kb; i += blockDim.x) B[(k0 + i) + c * ldb] = x[i];
}

// y[rows] -= op(M)[rows, blk] * x[blk] for all rhs, notrans: M(r, p) = LU[r + p lda].
// One thread per row; coalesced over rows.
template <typename T>
__global__ void __launch_bounds__(128) trsv_update_n_kernel(int64_t r0, int64_t r1, int64_t p0, int kb,
                                                            const T *LU, int64_t lda, T *B, int64_t ldb,
                                                            int64_t nrhs)
{
    __shared__ T xs[kMaxNB * 8];
    const int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t c0 = 0; c0 < nrhs; c0 += 8) {
        int nc = (int)(nrhs - c0 < 8 ? nrhs - c0 : 8);
        __syncthreads();
        for (int e = threadIdx.x; e < kb * nc; e += blockDim.x) {
            int p = e % kb, c = e / kb;
            xs[c * kMaxNB + p] = B[(p0 + p) + (c0 + c) * ldb];
        }
        __syncthreads();
        if (r < r1) {
            T acc[8];
#pragma unroll
            for (int c = 0; c < 8; c++) acc[c] = T(0);
            for (int p = 0; p < kb; p++) {
                T m = LU[r + (p0 + p) * lda];
#pragma unroll
                for (int c = 0; c < 8; c++)
                    if (c < nc) acc[c] = fma(m, xs[c * kMaxNB + p], acc[c]);
            }
            for (int c = 0; c < nc; c++) B[r + (c0 + c) * ldb] -= acc[c];
        }
    }
}

// transposed: M(r, p) = LU[p + r lda]; one warp per row, lanes over p.
template <typename T>
__global__ void __launch_bounds__(128) trsv_update_t_kernel(int64_t r0, int64_t r1, int64_t p0, int kb,
                                                            const T *LU, int64_t lda, T *B, int64_t ldb,
                                                            int64_t nrhs)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = r0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (r >= r1) return;
    for (int64_t c = 0; c < nrhs; c++) {
        T acc = T(0);
        for (int p = lane; p < kb; p += 32) acc = fma(LU[(p0 + p) + r * lda], B[(p0 + p) + c * ldb], acc);
        for (int o = 16; o > 0; o >>= 1) acc += shfl_xor(acc, o);
        if (lane == 0) B[r + c * ldb] -= acc;
    }
}

template <typename T>
static rbt_status tri_solve(int64_t n, int64_t nrhs, const T *LU, int64_t lda, int lower, int trans, T *B,
                            int64_t ldb, int nb, cudaStream_t stream)
{
    const int64_t nblk = cdiv(n, nb);
    for (int64_t bi = 0; bi < nblk; bi++) {
        int64_t blk = lower ? bi : (nblk - 1 - bi);
        int64_t k0 = blk * nb;
        int kb = (int)(n - k0 < nb ? n - k0 : nb);
        for (int64_t c0 = 0; c0 < nrhs; c0 += 65535) {
            int64_t nc = nrhs - c0 < 65535 ? nrhs - c0 : 65535;
            trsv_diag_kernel<T><<<(unsigned)nc, 128, (size_t)kb * kb * sizeof(T), stream>>>(
                k0, kb, LU, lda, B + c0 * ldb, ldb, lower, trans);
            RBT_LAUNCH_CHECK();
        }
        int64_t r0 = lower ? k0 + kb : 0, r1 = lower ? n : k0;
        if (r1 <= r0) continue;
        if (!trans) {
            trsv_update_n_kernel<T><<<(unsigned)cdiv(r1 - r0, 128), 128, 0, stream>>>(r0, r1, k0, kb, LU, lda, B,
                                                                                       ldb, nrhs);
        } else {
            trsv_update_t_kernel<T><<<(unsigned)cdiv((r1 - r0) * 32, 128), 128, 0, stream>>>(r0, r1, k0, kb, LU,
                                                                                              lda, B, ldb, nrhs);
        }
        RBT_LAUNCH_CHECK();
    }
    return RBT_OK;
}

// ------------------------------------------- chained triangular solve

// One persistent launch per triangle.  Row blocks of kChainNB rows are taken
// in solve order from a device counter; the CTA holding block b streams the
// columns of all earlier blocks that are already finished (four column lanes
// per row, many loads in flight; warp 0 finds the finished prefix 32 flags at
// a time), and when it has caught up it fetches its entries of the next
// block's columns before waiting for that block's solution.  It then finishes
// its diagonal block with the precomputed inverse plus one correction step
// (x0 = D^-1 r, x = x0 + D^-1 (r - D x0), each product split over the four
// lanes) and publishes it.  A CTA only waits on blocks taken before its own, which belong
// to running CTAs, so the chain always advances; every wait is bounded and
// records a timeout in err instead of hanging.
//
// The time per block on the chain is what the solve costs (the streaming
// keeps up easily): the wait for the previous block's flag, then its columns,
// the lane reduction and the three block products.  So the kernel is compiled
// for the number R of right-hand sides it carries per pass (one, the common
// case, or kChainRhs), its block's right-hand side is read before the wait,
// and every per-lane sum runs as two interleaved chains (even and odd column
// groups, fixed by the column index so the rounding does not depend on how
// the finished columns were grouped).
constexpr int kChainNB = 64;
constexpr int kChainLanes = 4;                          // column lanes per row when streaming
constexpr int kChainThreads = kChainNB * kChainLanes;  // 256
constexpr int kChainRhs = 8;                            // right-hand sides per pass beyond one

// An entry of the stored factor in the solve's arithmetic type T: the same
// type, a float widened to double, or a double-float pair rounded to double.
template <typename T, typename TF> __device__ __forceinline__ T elem_as(TF v) { return T(v); }
template <> __device__ __forceinline__ double elem_as<double, df64>(df64 v) { return df_to_double(v); }

// Inverse of every diagonal block of the triangle op(M) solves with (lower or
// upper part of LU or of LU^T, unit diagonal where the factor has one): one
// CTA per block, thread c computes column c of the inverse by substitution.
// The chained solve then finishes a block with a parallel product instead of
// a serial substitution on its critical path.
template <typename T, typename TF = T>
__global__ void __launch_bounds__(kChainNB) diag_inv_kernel(int64_t n, const TF *__restrict__ LU, int64_t lda,
                                                            int lower, int trans, T *inv)
{
    __shared__ T D[kChainNB][kChainNB + 1];
    __shared__ T X[kChainNB][kChainNB + 1];
    const int c = threadIdx.x;
    const int64_t pb = blockIdx.x;
    const int64_t r0 = pb * kChainNB;
    const int kb = (int)(n - r0 < kChainNB ? n - r0 : kChainNB);
    const bool unit = (lower && !trans) || (!lower && trans);
    for (int e = c; e < kChainNB * kChainNB; e += kChainNB) {
        int r = trans ? e / kChainNB : e % kChainNB, p = trans ? e % kChainNB : e / kChainNB;
        D[r][p] = (r < kb && p < kb) ? elem_as<T>(trans ? LU[(r0 + p) + (r0 + r) * lda] : LU[(r0 + r) + (r0 + p) * lda])
                                     : T(0);
    }
    __syncthreads();
    if (c < kb) {
        if (lower) {
            for (int i = 0; i < kb; i++) {
                if (i < c) {
                    X[i][c] = T(0);
                    continue;
                }
                T s = (i == c) ? T(1) : T(0);
                for (int p = c; p < i; p++) s -= D[i][p] * X[p][c];
                X[i][c] = unit ? s : s / D[i][i];
            }
        } else {
            for (int i = kb - 1; i >= 0; i--) {
                if (i > c) {
                    X[i][c] = T(0);
                    continue;
                }
                T s = (i == c) ? T(1) : T(0);
                for (int p = i + 1; p <= c; p++) s -= D[i][p] * X[p][c];
                X[i][c] = unit ? s : s / D[i][i];
            }
        }
    }
    __syncthreads();
    T *out = inv + pb * kChainNB * kChainNB;  // column-major 64 x 64, zero outside kb x kb
    for (int e = c; e < kChainNB * kChainNB; e += kChainNB) {
        int r = e % kChainNB, q = e / kChainNB;
        out[e] = (r < kb && q < kb) ? X[r][q] : T(0);
    }
}

template <typename T, typename TF, int R>
__global__ void __launch_bounds__(kChainThreads, R == 1 ? 2 : 1)
trsv_chain_kernel(int64_t n, int64_t nrhs, const TF *__restrict__ LU, int64_t lda, int lower, int trans, T *X,
                  int64_t ldx, int *flags, int *counter, int *err, const T *__restrict__ inv, int first_blk,
                  long long wait_ns)
{
    // dynamic shared memory (T):
    //   D[64][65]      diagonal block of op(M)
    //   Di[64][65]     its inverse (from diag_inv_kernel)
    //   xs[64][R+1]    right-hand sides of the block, R columns per pass
    //   red[4][64][R]  partial sums of the four column lanes
    extern __shared__ __align__(16) unsigned char chain_smem[];
    typedef T Row[kChainNB + 1];
    typedef T RowS[R + 1];
    Row *D = reinterpret_cast<Row *>(chain_smem);
    Row *Di = D + kChainNB;
    RowS *xs = reinterpret_cast<RowS *>(Di + kChainNB);
    T *red = reinterpret_cast<T *>(xs + kChainNB);
    __shared__ int s_blk, s_hi;
    constexpr int U = kChainNB / kChainLanes;  // columns of one block per lane
    const int tid = threadIdx.x;
    const int rr = tid % kChainNB, pl = tid / kChainNB;  // row of the block, column lane
    const int64_t nblk = (n + kChainNB - 1) / kChainNB;
    // physical block of solve step j, and the columns [cb, ce) of steps j0 .. j1-1
    auto phys = [&](int64_t j) { return lower ? j : nblk - 1 - j; };
    auto col_range = [&](int64_t j0, int64_t j1, int64_t &cb, int64_t &ce) {
        cb = lower ? j0 * kChainNB : (nblk - j1) * kChainNB;
        ce = lower ? j1 * kChainNB : (nblk - j0) * kChainNB;
        if (ce > n) ce = n;
    };
    for (;;) {
        if (tid == 0) s_blk = first_blk + atomicAdd(counter, 1);
        __syncthreads();
        const int64_t b = s_blk;
        __syncthreads();
        if (b >= nblk) return;
        const int64_t pb = phys(b);
        const int64_t r0 = pb * kChainNB;
        const int kb = (int)(n - r0 < kChainNB ? n - r0 : kChainNB);
        const bool unit = (lower && !trans) || (!lower && trans);
        for (int e = tid; e < kChainNB * kChainNB; e += kChainThreads) {
            // only the triangle being solved with, unit diagonal where the factor has one
            const int r = trans ? e / kChainNB : e % kChainNB, p = trans ? e % kChainNB : e / kChainNB;
            const bool in_tri = r < kb && p < kb && (lower ? p <= r : p >= r);
            T v = T(0);
            if (in_tri)
                v = (p == r && unit) ? T(1)
                                     : elem_as<T>(trans ? LU[(r0 + p) + (r0 + r) * lda] : LU[(r0 + r) + (r0 + p) * lda]);
            D[r][p] = v;
            Di[e % kChainNB][e / kChainNB] = inv[pb * kChainNB * kChainNB + e];
        }
        const int64_t grow = r0 + rr;
        auto entry = [&](int64_t p) { return elem_as<T>(trans ? LU[p + grow * lda] : LU[grow + p * lda]); };
        for (int64_t c0 = 0; c0 < nrhs; c0 += R) {
            const int nc = R == 1 ? 1 : (int)(nrhs - c0 < R ? nrhs - c0 : R);
            // the block's own right-hand sides stay as they are until it is solved
            T rhs[R];
#pragma unroll
            for (int c = 0; c < R; c++) rhs[c] = (pl == 0 && rr < kb && c < nc) ? X[grow + (c0 + c) * ldx] : T(0);
            T acc0[R], acc1[R];
#pragma unroll
            for (int c = 0; c < R; c++) acc0[c] = acc1[c] = T(0);
            // column p = cb + pl + 4 q of this lane: q's parity picks the chain
            // (cb is a multiple of 64, so the parity is that of p / 4)
            auto mac = [&](T(&acc)[R], T m, int64_t p) {
#pragma unroll
                for (int c = 0; c < R; c++)
                    if (c < nc) acc[c] = fma(m, ld_cg(X + p + (c0 + c) * ldx), acc[c]);
            };
            for (int64_t jl = 0; jl < b;) {
                // finished prefix [jl, hi) of the earlier steps: warp 0 reads 32 flags per round
                if (tid < 32) {
                    int64_t hi = jl;
                    for (;;) {
                        const int64_t q = hi + tid;
                        const bool rdy = q < b && *((volatile int *)(flags + phys(q))) != 0;
                        const unsigned m = __ballot_sync(0xffffffffu, rdy);
                        if (m == 0xffffffffu) {
                            hi += 32;
                            if (hi < b) continue;
                            hi = b;
                        } else {
                            hi += __ffs(~m) - 1;
                        }
                        break;
                    }
                    __threadfence();
                    if (tid == 0) s_hi = (int)hi;
                }
                __syncthreads();
                const int64_t hi = s_hi;
                int64_t cb, ce;
                if (hi > jl) {
                    col_range(jl, hi, cb, ce);
                    // A lower solve meets its finished steps in ascending column
                    // order and an upper one in descending order, whatever the
                    // grouping of the steps into chunks, when each chunk is walked
                    // the same way: so each chain's summation order (and the
                    // rounding) is the same on every run.
                    const int64_t span = ce - cb - pl;
                    if (rr < kb && span > 0) {
                        const int64_t qn = (span - 1) / kChainLanes + 1;
                        auto col = [&](int64_t q) { return cb + pl + kChainLanes * q; };
                        if (lower) {
                            int64_t q = 0;
#pragma unroll 2
                            for (; q + 1 < qn; q += 2) {
                                const T m0 = entry(col(q)), m1 = entry(col(q + 1));
                                mac(acc0, m0, col(q));
                                mac(acc1, m1, col(q + 1));
                            }
                            if (q < qn) mac(acc0, entry(col(q)), col(q));
                        } else {
                            int64_t q = qn - 1;
                            if (q & 1) {
                                mac(acc1, entry(col(q)), col(q));
                                q--;
                            }
#pragma unroll 2
                            for (; q >= 1; q -= 2) {
                                const T m0 = entry(col(q)), m1 = entry(col(q - 1));
                                mac(acc0, m0, col(q));
                                mac(acc1, m1, col(q - 1));
                            }
                            if (q == 0) mac(acc0, entry(col(0)), col(0));
                        }
                    }
                    jl = hi;
                } else {
                    // step jl is the front and not finished: its entries in this row
                    // block are final already, so fetch them before waiting
                    col_range(jl, jl + 1, cb, ce);
                    T mp[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int64_t p = cb + pl + kChainLanes * u;
                        mp[u] = (rr < kb && p < ce) ? entry(p) : T(0);
                    }
                    if (tid == 0) {
                        // bounded by wait_ns of %globaltimer; a timeout (or one
                        // seen from another CTA) ends every later wait at once
                        const int64_t pj = phys(jl);
                        unsigned long long t0 = 0;
                        bool timing = false;
                        while (*((volatile int *)(flags + pj)) == 0 && *((volatile int *)err) == 0) {
                            if (!timing) {
                                t0 = global_ns();
                                timing = true;
                            } else if ((long long)(global_ns() - t0) > wait_ns) {
                                atomicExch(err, 1);
                                break;
                            }
                            __nanosleep(32);
                        }
                        __threadfence();
                    }
                    __syncthreads();
                    if (rr < kb) {
                        // the same per-lane column order and chains as the chunked form
                        auto step_u = [&](int u) {
                            const int64_t p = cb + pl + kChainLanes * u;
                            if (p < ce) {
                                if (u & 1)
                                    mac(acc1, mp[u], p);
                                else
                                    mac(acc0, mp[u], p);
                            }
                        };
                        if (lower) {
#pragma unroll
                            for (int u = 0; u < U; u++) step_u(u);
                        } else {
#pragma unroll
                            for (int u = U - 1; u >= 0; u--) step_u(u);
                        }
                    }
                    jl += 1;
                }
                __syncthreads();
            }
            // reduce the column lanes; residual right-hand side of the block
#pragma unroll
            for (int c = 0; c < R; c++) red[(pl * kChainNB + rr) * R + c] = acc0[c] + acc1[c];
            __syncthreads();
            auto lane_sum = [&](int c) {
                T s = red[rr * R + c];
                for (int l = 1; l < kChainLanes; l++) s += red[(l * kChainNB + rr) * R + c];
                return s;
            };
            if (pl == 0 && rr < kb) {
#pragma unroll
                for (int c = 0; c < R; c++)
                    if (c < nc) {
                        rhs[c] -= lane_sum(c);
                        xs[rr][c] = rhs[c];
                    }
            }
            __syncthreads();
            // block solve D x = r: x0 = Di r, then one correction x = x0 + Di (r - D x0).
            // Each product is split over the four column lanes (16 terms each,
            // two chains) and summed through shared memory; row rr's lane 0
            // keeps r and x0 in registers.  Each row's lane 0 only rewrites its
            // own row of xs, after the barrier that ends the product reading it.
            auto lane_products = [&](const Row *Mx) {
                T q0[R], q1[R];
#pragma unroll
                for (int c = 0; c < R; c++) q0[c] = q1[c] = T(0);
                if (rr < kb) {
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int p = pl + kChainLanes * u;
                        if (p < kb) {
                            const T m = Mx[rr][p];
#pragma unroll
                            for (int c = 0; c < R; c++)
                                if (c < nc) {
                                    if (u & 1)
                                        q1[c] = fma(m, xs[p][c], q1[c]);
                                    else
                                        q0[c] = fma(m, xs[p][c], q0[c]);
                                }
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < R; c++) red[(pl * kChainNB + rr) * R + c] = q0[c] + q1[c];
            };
            T x0[R];
            lane_products(Di);  // x0 = Di r
            __syncthreads();
            if (pl == 0 && rr < kb) {
#pragma unroll
                for (int c = 0; c < R; c++)
                    if (c < nc) {
                        x0[c] = lane_sum(c);
                        xs[rr][c] = x0[c];
                    }
            }
            __syncthreads();
            lane_products(D);  // D x0
            __syncthreads();
            if (pl == 0 && rr < kb) {
#pragma unroll
                for (int c = 0; c < R; c++)
                    if (c < nc) xs[rr][c] = rhs[c] - lane_sum(c);
            }
            __syncthreads();
            lane_products(Di);  // Di (r - D x0)
            __syncthreads();
            if (pl == 0 && rr < kb) {
#pragma unroll
                for (int c = 0; c < R; c++)
                    if (c < nc) X[grow + (c0 + c) * ldx] = x0[c] + lane_sum(c);
            }
            if (R > 1) __syncthreads();  // xs and red are reused by the next pass
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicExch(flags + pb, 1);
    }
}

template <typename T, int R> constexpr size_t chain_smem_bytes()
{
    return (2 * kChainNB * (kChainNB + 1) + kChainNB * (R + 1) + kChainLanes * kChainNB * R) * sizeof(T);
}

template <typename T, typename TF, int R>
static rbt_status launch_chain(int64_t n, int64_t nrhs, const TF *LU, int64_t lda, int lower, int trans, T *B,
                               int64_t ldb, int *scratch, const T *inv, cudaStream_t stream)
{
    static PerDeviceOnce once;
    rbt_status cst = smem_opt_in(once, trsv_chain_kernel<T, TF, R>, (int)chain_smem_bytes<T, R>());
    if (cst != RBT_OK) return cst;
    const int64_t nblk = cdiv(n, kChainNB);
    int *err = scratch, *counter = scratch + 1, *flags = scratch + 2;
    RBT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int) * (size_t)(nblk + 1), stream));
    int per_sm = 1;
    RBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trsv_chain_kernel<T, TF, R>, kChainThreads,
                                                               chain_smem_bytes<T, R>()));
    int64_t grid = (int64_t)device_sm_count() * (per_sm > 0 ? per_sm : 1);
    if (grid > nblk) grid = nblk;
    // the test stall starts the queue at block 1: block 0 is never solved
    const int first_blk = debug_stall() == RBT_STALL_CHAIN ? 1 : 0;
    trsv_chain_kernel<T, TF, R><<<(unsigned)grid, kChainThreads, chain_smem_bytes<T, R>(), stream>>>(
        n, nrhs, LU, lda, lower, trans, B, ldb, flags, counter, err, inv, first_blk, wait_limit_ns());
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

// scratch: [0] timeout flag (cleared by the public entry point or the solve
// driver, once per call: it stays set across the triangles and refinement
// steps of one call), [1] block counter, [2..] block flags, then (256-byte
// aligned) the inverses of the diagonal blocks.
template <typename T, typename TF = T>
static rbt_status tri_chain(int64_t n, int64_t nrhs, const TF *LU, int64_t lda, int lower, int trans, T *B,
                            int64_t ldb, int *scratch, cudaStream_t stream)
{
    const int64_t nblk = cdiv(n, kChainNB);
    T *inv = (T *)((char *)scratch + ((size_t)(nblk + 2) * sizeof(int) + 255) / 256 * 256);
    diag_inv_kernel<T, TF><<<(unsigned)nblk, kChainNB, 0, stream>>>(n, LU, lda, lower, trans, inv);
    RBT_LAUNCH_CHECK();
    if (nrhs == 1) return launch_chain<T, TF, 1>(n, nrhs, LU, lda, lower, trans, B, ldb, scratch, inv, stream);
    return launch_chain<T, TF, kChainRhs>(n, nrhs, LU, lda, lower, trans, B, ldb, scratch, inv, stream);
}

size_t chain_scratch_bytes(int64_t n, size_t es)
{
    const int64_t nblk = cdiv(n > 0 ? n : 1, kChainNB);
    return ((size_t)(nblk + 2) * sizeof(int) + 255) / 256 * 256 + (size_t)nblk * kChainNB * kChainNB * es + 256;
}

// ------------------------------------- blocked solves for many right-hand sides
//
// With many right-hand sides the chain's per-block critical path grows with
// them (a block is published only after all its right-hand sides); a
// right-looking blocked solve is then faster: for each 64-row block in solve
// order, finish the block with its precomputed inverse plus one correction
// step, then subtract its contribution from all the rows still to solve with
// one wide update kernel.
constexpr int kBlkRhs = 32;       // right-hand sides per pass of the block kernels
constexpr int kBlkRhsMin = 4;     // fewer right-hand sides take the chained solve

// X_b <- op(M)_bb^{-1} X_b for step block pb: x0 = Di r, x = x0 + Di (r - D x0).
template <typename T>
__global__ void __launch_bounds__(256) blk_diag_kernel(int64_t n, int64_t nrhs, const T *__restrict__ LU,
                                                       int64_t lda, int lower, int trans, int64_t pb,
                                                       const T *__restrict__ inv, T *X, int64_t ldx)
{
    extern __shared__ __align__(16) unsigned char blk_smem[];
    typedef T Row[kChainNB + 1];
    typedef T RowR[kBlkRhs + 1];
    Row *D = reinterpret_cast<Row *>(blk_smem);
    Row *Di = D + kChainNB;
    RowR *r = reinterpret_cast<RowR *>(Di + kChainNB);
    RowR *x0 = r + kChainNB;
    const int tid = threadIdx.x;
    const int64_t r0 = pb * kChainNB;
    const int kb = (int)(n - r0 < kChainNB ? n - r0 : kChainNB);
    const bool unit = (lower && !trans) || (!lower && trans);
    for (int e = tid; e < kChainNB * kChainNB; e += 256) {
        const int i = trans ? e / kChainNB : e % kChainNB, p = trans ? e % kChainNB : e / kChainNB;
        const bool in_tri = i < kb && p < kb && (lower ? p <= i : p >= i);
        T v = T(0);
        if (in_tri) v = (p == i && unit) ? T(1) : (trans ? LU[(r0 + p) + (r0 + i) * lda] : LU[(r0 + i) + (r0 + p) * lda]);
        D[i][p] = v;
        Di[e % kChainNB][e / kChainNB] = inv[pb * kChainNB * kChainNB + e];
    }
    for (int64_t c0 = 0; c0 < nrhs; c0 += kBlkRhs) {
        const int nc = (int)(nrhs - c0 < kBlkRhs ? nrhs - c0 : kBlkRhs);
        for (int e = tid; e < kChainNB * kBlkRhs; e += 256) {
            const int i = e % kChainNB, c = e / kChainNB;
            r[i][c] = (i < kb && c < nc) ? X[(r0 + i) + (c0 + c) * ldx] : T(0);
        }
        __syncthreads();
        // x0 = Di r
        for (int e = tid; e < kChainNB * kBlkRhs; e += 256) {
            const int i = e % kChainNB, c = e / kChainNB;
            T s = T(0);
            for (int p = 0; p < kb; p++) s = fma(Di[i][p], r[p][c], s);
            x0[i][c] = s;
        }
        __syncthreads();
        // r <- r - D x0 (each entry read and written by its own thread)
        for (int e = tid; e < kChainNB * kBlkRhs; e += 256) {
            const int i = e % kChainNB, c = e / kChainNB;
            T s = r[i][c];
            for (int p = 0; p < kb; p++) s -= D[i][p] * x0[p][c];
            r[i][c] = s;
        }
        __syncthreads();
        // x = x0 + Di r
        for (int e = tid; e < kChainNB * kBlkRhs; e += 256) {
            const int i = e % kChainNB, c = e / kChainNB;
            if (i < kb && c < nc) {
                T s = x0[i][c];
                for (int p = 0; p < kb; p++) s = fma(Di[i][p], r[p][c], s);
                X[(r0 + i) + (c0 + c) * ldx] = s;
            }
        }
        __syncthreads();
    }
}

// C (M x N) -= A (M x K) Xb (K x N), K <= 64, for the rows still to solve:
// A column-major (lda), or its transpose when TA (A(i, k) at A[k + i lda]).
// One row per thread, Xb staged in shared memory kBlkRhs columns at a time.
template <typename T, bool TA>
__global__ void __launch_bounds__(128) blk_update_kernel(int64_t M, int64_t N, int K, const T *__restrict__ A,
                                                         int64_t lda, const T *Xb, int64_t ldx, T *C, int64_t ldc)
{
    __shared__ T xs[kChainNB][kBlkRhs + 1];
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    for (int64_t c0 = 0; c0 < N; c0 += kBlkRhs) {
        const int nc = (int)(N - c0 < kBlkRhs ? N - c0 : kBlkRhs);
        for (int e = threadIdx.x; e < kChainNB * kBlkRhs; e += 128) {
            const int k = e % kChainNB, c = e / kChainNB;
            xs[k][c] = (k < K && c < nc) ? Xb[k + (c0 + c) * ldx] : T(0);
        }
        __syncthreads();
        if (i < M) {
            T acc[kBlkRhs];
#pragma unroll
            for (int c = 0; c < kBlkRhs; c++) acc[c] = T(0);
            for (int k = 0; k < K; k++) {
                const T a = TA ? A[k + i * lda] : A[i + (int64_t)k * lda];
#pragma unroll
                for (int c = 0; c < kBlkRhs; c++) acc[c] = fma(a, xs[k][c], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < kBlkRhs; c++)
                if (c < nc) C[i + (c0 + c) * ldc] -= acc[c];
        }
        __syncthreads();
    }
}

template <typename T> constexpr size_t blk_diag_smem_bytes()
{
    return (2 * kChainNB * (kChainNB + 1) + 2 * kChainNB * (kBlkRhs + 1)) * sizeof(T);
}

// One triangle of op(M) (as tri_chain) by blocks; the inverses of the
// diagonal blocks go to the chain scratch's inverse area.
template <typename T>
static rbt_status tri_blocked(int64_t n, int64_t nrhs, const T *LU, int64_t lda, int lower, int trans, T *B,
                              int64_t ldb, int *scratch, cudaStream_t stream)
{
    const int64_t nblk = cdiv(n, kChainNB);
    T *inv = (T *)((char *)scratch + ((size_t)(nblk + 2) * sizeof(int) + 255) / 256 * 256);
    diag_inv_kernel<T><<<(unsigned)nblk, kChainNB, 0, stream>>>(n, LU, lda, lower, trans, inv);
    RBT_LAUNCH_CHECK();
    static PerDeviceOnce once;
    rbt_status cst = smem_opt_in(once, blk_diag_kernel<T>, (int)blk_diag_smem_bytes<T>());
    if (cst != RBT_OK) return cst;
    for (int64_t j = 0; j < nblk; j++) {
        const int64_t pb = lower ? j : nblk - 1 - j;
        const int64_t r0 = pb * kChainNB;
        const int kb = (int)(n - r0 < kChainNB ? n - r0 : kChainNB);
        blk_diag_kernel<T><<<1, 256, blk_diag_smem_bytes<T>(), stream>>>(n, nrhs, LU, lda, lower, trans, pb, inv, B,
                                                                         ldb);
        RBT_LAUNCH_CHECK();
        // rows still to solve: below the block (lower) or above it (upper)
        const int64_t m0 = lower ? r0 + kb : 0, M = lower ? n - r0 - kb : r0;
        if (M <= 0) continue;
        // op(M)(m0 + i, r0 + k): the lower part is L (trans = 0) or U^T (trans = 1),
        // the upper part U (trans = 0) or L^T (trans = 1)
        const unsigned grid = (unsigned)cdiv(M, 128);
        if (!trans) {
            blk_update_kernel<T, false><<<grid, 128, 0, stream>>>(M, nrhs, kb, LU + m0 + r0 * lda, lda, B + r0, ldb,
                                                                  B + m0, ldb);
        } else {
            blk_update_kernel<T, true><<<grid, 128, 0, stream>>>(M, nrhs, kb, LU + r0 + m0 * lda, lda, B + r0, ldb,
                                                                 B + m0, ldb);
        }
        RBT_LAUNCH_CHECK();
    }
    return RBT_OK;
}

// (L U)^{-1} B or (L U)^{-T} B: two chained launches, or two blocked sweeps
// for many right-hand sides; scratch[0] (device) becomes nonzero when a wait
// of the chained form gave up, and is never cleared here.
template <typename T>
rbt_status lu_solve_chain(int64_t n, int64_t nrhs, const T *LU, int64_t lda, int trans, T *B, int64_t ldb,
                          int *scratch, cudaStream_t stream)
{
    ProfScope ps(kProfSolve, stream);
    if (nrhs >= kBlkRhsMin) {
        rbt_status st = tri_blocked<T>(n, nrhs, LU, lda, 1, trans, B, ldb, scratch, stream);
        if (st != RBT_OK) return st;
        return tri_blocked<T>(n, nrhs, LU, lda, 0, trans, B, ldb, scratch, stream);
    }
    rbt_status st = tri_chain<T>(n, nrhs, LU, lda, 1, trans, B, ldb, scratch, stream);  // L y = b or U^T y = b
    if (st != RBT_OK) return st;
    return tri_chain<T>(n, nrhs, LU, lda, 0, trans, B, ldb, scratch, stream);           // U x = y or L^T x = y
}

// (L U)^{-1} B or (L U)^{-T} B in double arithmetic with factors stored in a
// lower precision TF (float, or double-float pairs): the chained form, any
// number of right-hand sides.  Each entry is widened as it is read, so the
// solve reads the factors' own bytes and the only error beyond the factors'
// is that of a double substitution.
template <typename TF>
static rbt_status lu_solve_wp(int64_t n, int64_t nrhs, const TF *LU, int64_t lda, int trans, double *B, int64_t ldb,
                              int *scratch, cudaStream_t stream)
{
    ProfScope ps(kProfSolve, stream);
    rbt_status st = tri_chain<double, TF>(n, nrhs, LU, lda, 1, trans, B, ldb, scratch, stream);
    if (st != RBT_OK) return st;
    return tri_chain<double, TF>(n, nrhs, LU, lda, 0, trans, B, ldb, scratch, stream);
}

template <typename T>
rbt_status lu_solve(int64_t n, int64_t nrhs, const T *LU, int64_t lda, int trans, T *B, int64_t ldb,
                    cudaStream_t stream)
{
    ProfScope ps(kProfSolve, stream);
    static PerDeviceOnce once;
    rbt_status cst = smem_opt_in(once, trsv_diag_kernel<T>, (int)(kSolveNB * kSolveNB * sizeof(T)));
    if (cst != RBT_OK) return cst;
    rbt_status st;
    if (!trans) {
        st = tri_solve<T>(n, nrhs, LU, lda, 1, 0, B, ldb, kSolveNB, stream);  // L y = b
        if (st != RBT_OK) return st;
        return tri_solve<T>(n, nrhs, LU, lda, 0, 0, B, ldb, kSolveNB, stream);  // U x = y
    }
    st = tri_solve<T>(n, nrhs, LU, lda, 1, 1, B, ldb, kSolveNB, stream);  // U^T y = b
    if (st != RBT_OK) return st;
    return tri_solve<T>(n, nrhs, LU, lda, 0, 1, B, ldb, kSolveNB, stream);  // L^T x = y
}

template rbt_status lu_solve<double>(int64_t, int64_t, const double *, int64_t, int, double *, int64_t,
                                     cudaStream_t);
template rbt_status lu_solve<float>(int64_t, int64_t, const float *, int64_t, int, float *, int64_t, cudaStream_t);
template rbt_status lu_solve<df64>(int64_t, int64_t, const df64 *, int64_t, int, df64 *, int64_t, cudaStream_t);

// -------------------------------------------------------- conversions

__global__ void narrow_kernel(int64_t n, int64_t nrhs, const double *B, int64_t ldb, float *F, int64_t ldf)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t i = idx % n, c = idx / n;
    F[i + c * ldf] = (float)B[i + c * ldb];
}

__global__ void widen_kernel(int64_t n, int64_t nrhs, const float *F, int64_t ldf, double *B, int64_t ldb)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t i = idx % n, c = idx / n;
    B[i + c * ldb] = (double)F[i + c * ldf];
}

__global__ void narrow_df_kernel(int64_t n, int64_t nrhs, const double *B, int64_t ldb, df64 *F, int64_t ldf)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t i = idx % n, c = idx / n;
    F[i + c * ldf] = df_from_double(B[i + c * ldb]);
}

__global__ void widen_df_kernel(int64_t n, int64_t nrhs, const df64 *F, int64_t ldf, double *B, int64_t ldb)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * nrhs) return;
    int64_t i = idx % n, c = idx / n;
    B[i + c * ldb] = df_to_double(F[i + c * ldf]);
}

rbt_status narrow_block(int64_t n, int64_t nrhs, const double *B, int64_t ldb, float *F, int64_t ldf,
                        cudaStream_t stream)
{
    if (n * nrhs == 0) return RBT_OK;
    narrow_kernel<<<(unsigned)cdiv(n * nrhs, 256), 256, 0, stream>>>(n, nrhs, B, ldb, F, ldf);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

rbt_status widen_block(int64_t n, int64_t nrhs, const float *F, int64_t ldf, double *B, int64_t ldb,
                       cudaStream_t stream)
{
    if (n * nrhs == 0) return RBT_OK;
    widen_kernel<<<(unsigned)cdiv(n * nrhs, 256), 256, 0, stream>>>(n, nrhs, F, ldf, B, ldb);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

static rbt_status narrow_block_df(int64_t n, int64_t nrhs, const double *B, int64_t ldb, df64 *F, int64_t ldf,
                                  cudaStream_t stream)
{
    if (n * nrhs == 0) return RBT_OK;
    narrow_df_kernel<<<(unsigned)cdiv(n * nrhs, 256), 256, 0, stream>>>(n, nrhs, B, ldb, F, ldf);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

static rbt_status widen_block_df(int64_t n, int64_t nrhs, const df64 *F, int64_t ldf, double *B, int64_t ldb,
                                 cudaStream_t stream)
{
    if (n * nrhs == 0) return RBT_OK;
    widen_df_kernel<<<(unsigned)cdiv(n * nrhs, 256), 256, 0, stream>>>(n, nrhs, F, ldf, B, ldb);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

// genp_solve / genp_solve_wp after validation, without clearing the timeout
// flag at the front of work (the caller owns its lifetime).
rbt_status genp_solve_run(int64_t n, int64_t nrhs, int32_t prec, const void *LU, int64_t lda, int32_t trans,
                          double *B, int64_t ldb, void *work, cudaStream_t stream)
{
    if (n == 0 || nrhs == 0) return RBT_OK;
    int *scratch = (int *)work;
    const size_t wes = prec == RBT_F64 ? sizeof(double) : ((is_df64_storage(prec)) ? sizeof(df64) : sizeof(float));
    char *rest = (char *)work + ((chain_scratch_bytes(n, wes) + 255) / 256 * 256);
    if (prec == RBT_F64)
        return lu_solve_chain<double>(n, nrhs, (const double *)LU, lda, trans ? 1 : 0, B, ldb, scratch, stream);
    if (is_df64_storage(prec)) {
        df64 *F = (df64 *)rest;
        rbt_status st = narrow_block_df(n, nrhs, B, ldb, F, n, stream);
        if (st != RBT_OK) return st;
        st = lu_solve_chain<df64>(n, nrhs, (const df64 *)LU, lda, trans ? 1 : 0, F, n, scratch, stream);
        if (st != RBT_OK) return st;
        return widen_block_df(n, nrhs, F, n, B, ldb, stream);
    }
    float *F = (float *)rest;
    rbt_status st = narrow_block(n, nrhs, B, ldb, F, n, stream);
    if (st != RBT_OK) return st;
    st = lu_solve_chain<float>(n, nrhs, (const float *)LU, lda, trans ? 1 : 0, F, n, scratch, stream);
    if (st != RBT_OK) return st;
    return widen_block(n, nrhs, F, n, B, ldb, stream);
}

rbt_status genp_solve_wp_run(int64_t n, int64_t nrhs, int32_t prec, const void *LU, int64_t lda, int32_t trans,
                             double *B, int64_t ldb, void *work, cudaStream_t stream)
{
    if (n == 0 || nrhs == 0) return RBT_OK;
    int *scratch = (int *)work;
    const int t = trans ? 1 : 0;
    if (prec == RBT_F64) return lu_solve_chain<double>(n, nrhs, (const double *)LU, lda, t, B, ldb, scratch, stream);
    if (is_df64_storage(prec))
        return lu_solve_wp<df64>(n, nrhs, (const df64 *)LU, lda, t, B, ldb, scratch, stream);
    return lu_solve_wp<float>(n, nrhs, (const float *)LU, lda, t, B, ldb, scratch, stream);
}

}  // namespace rbt

using namespace rbt;

extern "C" {

size_t genp_factor_workspace(int64_t n, int32_t prec, int32_t nb)
{
    return genp_factor_workspace_impl(n, prec, nb);
}

rbt_status genp_factor(int64_t n, int32_t prec, void *A, int64_t lda, int64_t *d_info, void *work,
                       size_t work_bytes, int32_t nb, cudaStream_t stream)
{
    if (n < 0 || lda < (n > 1 ? n : 1) || !d_info || prec < RBT_F64 || prec > kLastPrec) return RBT_ERR_ARG;
    if (nb < 0 || nb > kMaxNB) return RBT_ERR_ARG;
    RBT_CUDA_TRY(cudaMemsetAsync(d_info, 0xff, sizeof(int64_t), stream));  // -1
    if (n == 0) return RBT_OK;
    if (!A) return RBT_ERR_ARG;
    if (work_bytes < genp_factor_workspace_impl(n, prec, nb)) return RBT_ERR_WORKSPACE;
    return genp_factor_impl(n, prec, A, lda, d_info, work, work_bytes, nb, stream);
}

size_t genp_solve_workspace(int64_t n, int64_t nrhs, int32_t prec)
{
    if (n <= 0 || nrhs <= 0) return 0;
    size_t es = prec == RBT_F64 ? 0 : ((is_df64_storage(prec)) ? sizeof(df64) : sizeof(float));
    size_t ws = prec == RBT_F64 ? sizeof(double) : (es ? es : sizeof(float));
    return (size_t)n * (size_t)nrhs * es + chain_scratch_bytes(n, ws) + 256;
}

// Solve flag at the front of the workspace: nonzero after a call whose chained
// triangular solve gave up waiting (the result is then undefined).  The public
// calls clear it on entry; the *_run forms (the solve driver's) never clear it,
// so that one timeout stays visible for the rest of the driver's call.
rbt_status genp_solve(int64_t n, int64_t nrhs, int32_t prec, const void *LU, int64_t lda, int32_t trans,
                      double *B, int64_t ldb, void *work, size_t work_bytes, cudaStream_t stream)
{
    if (n < 0 || nrhs < 0 || prec < RBT_F64 || prec > kLastPrec) return RBT_ERR_ARG;
    if (lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1)) return RBT_ERR_ARG;
    if (n == 0 || nrhs == 0) return RBT_OK;
    if (!LU || !B) return RBT_ERR_ARG;
    if (work_bytes < genp_solve_workspace(n, nrhs, prec) || !work) return RBT_ERR_WORKSPACE;
    RBT_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(int), stream));
    return genp_solve_run(n, nrhs, prec, LU, lda, trans, B, ldb, work, stream);
}

size_t genp_solve_wp_workspace(int64_t n, int64_t nrhs)
{
    if (n <= 0 || nrhs <= 0) return 0;
    return chain_scratch_bytes(n, sizeof(double)) + 256;
}

rbt_status genp_solve_wp(int64_t n, int64_t nrhs, int32_t prec, const void *LU, int64_t lda, int32_t trans,
                         double *B, int64_t ldb, void *work, size_t work_bytes, cudaStream_t stream)
{
    if (n < 0 || nrhs < 0 || prec < RBT_F64 || prec > kLastPrec) return RBT_ERR_ARG;
    if (lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1)) return RBT_ERR_ARG;
    if (n == 0 || nrhs == 0) return RBT_OK;
    if (!LU || !B) return RBT_ERR_ARG;
    if (work_bytes < genp_solve_wp_workspace(n, nrhs) || !work) return RBT_ERR_WORKSPACE;
    RBT_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(int), stream));
    return genp_solve_wp_run(n, nrhs, prec, LU, lda, trans, B, ldb, work, stream);
}

}  // extern "C"
