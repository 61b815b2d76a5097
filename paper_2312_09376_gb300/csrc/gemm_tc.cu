// Tensor-core GENP update on sm_103a: C (float, M x N) -= A (M x K) B (K x N)
// with tcgen05.mma (TF32 or BF16 operands, FP32 accumulation in tensor
// memory), operands staged to shared memory by TMA, and a two-level blocked
// GENP that feeds it long K (the trailing update of Eq. precond step 2's
// factorization is the method's only dense contraction).
//
// Kernel structure (one 128 x 256 output tile per CTA, 4 warps):
//   warp 0      allocates 256 TMEM columns; lane 0 is the TMA producer;
//   warp 1      lane 0 issues tcgen05.mma (one thread per CTA) and commits;
//   warps 0..3  epilogue: tcgen05.ld of their 32 TMEM lanes, C -= acc.
// Operands are K-major (each row of the tile holds 128 contiguous bytes of
// K), 128-byte swizzled by TMA; a stage holds one 128-byte slab of K
// (64 bf16 or 32 tf32) for A and B, consumed by four MMAs (K = 16 / 8).
// Every mbarrier wait gives up after about a second of SM clocks and
// records RBT_ERR_TIMEOUT in a device status word.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cuda_bf16.h>

#include <mutex>

#include "gemm_tc.cuh"
#include "genp_internal.cuh"

namespace rbt {
namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int STAGES = 2;
constexpr int ROW_BYTES = 128;
constexpr int A_STAGE_BYTES = BM * ROW_BYTES;  // 16 KB
constexpr int B_STAGE_BYTES = BN * ROW_BYTES;  // 32 KB
constexpr int STAGE_BYTES = A_STAGE_BYTES + B_STAGE_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*alignment slack*/ + 256 /*barriers*/;
constexpr int TMEM_COLS = 256;

struct Status {
    int err;  // 0 or an rbt_status (RBT_ERR_TIMEOUT)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and the status word set) when the phase does not
// complete within wait_ns of %globaltimer.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, Status *st, long long wait_ns)
{
    if (mbar_test(bar, parity)) return true;  // the common case: no timer read
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if ((long long)(global_ns() - t0) > wait_ns) {
            atomicExch(&st->err, (int)RBT_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // version
    d |= (uint64_t)2 << 61;              // SWIZZLE_128B
    return d;
}

// Instruction descriptor: FP32 accumulate, K-major A and B, M = 128, N = BN.
template <int KIND>  // 0 = bf16 (kind::f16), 1 = tf32
__host__ __device__ constexpr uint32_t instr_desc()
{
    return (1u << 4)                                   // D format F32
           | ((KIND == 0 ? 1u : 2u) << 7)              // A format BF16 / TF32
           | ((KIND == 0 ? 1u : 2u) << 10)             // B format BF16 / TF32
           | ((uint32_t)(BN >> 3) << 17)               // N >> 3
           | ((uint32_t)(BM >> 4) << 24);              // M >> 4
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    constexpr uint32_t idesc = instr_desc<KIND>();
    if (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// C (M x N, ldc, float) -= A_k (M x K, K-major, from tmap_a) * B_k (N x K, K-major, from tmap_b)
template <int KIND>
__global__ void __launch_bounds__(128, 1)
tc_update_kernel(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b,
                 int M, int N, int K, float *C, int64_t ldc, const int64_t *info, Status *st, long long wait_ns)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);

    if (*((volatile const int64_t *)info) >= 0) return;  // an earlier pivot failed
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    constexpr int KSTEP = KIND == 0 ? 64 : 32;   // elements of K per 128-byte row
    const int nk = (K + KSTEP - 1) / KSTEP;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int i = 0; i < nk; i++) {
            const int s = i % STAGES, r = i / STAGES;
            if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1, st, wait_ns)) break;
            unsigned char *sa = smem + s * STAGE_BYTES;
            unsigned char *sb = sa + A_STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(sa, &tmap_a, i * KSTEP, m0, &full[s]);
            tma_load_2d(sb, &tmap_b, i * KSTEP, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer (single thread)
        for (int i = 0; i < nk; i++) {
            const int s = i % STAGES, r = i / STAGES;
            if (!mbar_wait(&full[s], r & 1, st, wait_ns)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
            const uint32_t sb = sa + A_STAGE_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
                // advance 32 bytes of K inside the 128-byte swizzled row
                mma<KIND>(tmem, smem_desc(sa + kk * 32), smem_desc(sb + kk * 32), (i > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(done);
    }
    __syncwarp();

    // epilogue: all four warps, warp w owns TMEM lanes [32w, 32w + 32)
    bool ok = mbar_wait(done, 0, st, wait_ns);
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 32) {
            if (n0 + c0 >= N) break;  // warp-uniform
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < M) {
                float *c = C + row + (int64_t)(n0 + c0) * ldc;
#pragma unroll
                for (int j = 0; j < 32; j++)
                    if (n0 + c0 + j < N) c[(int64_t)j * ldc] -= __uint_as_float(r[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------- staging

__device__ __forceinline__ void cvt_store(float *dst, float v) { *dst = v; }
__device__ __forceinline__ void cvt_store(__nv_bfloat16 *dst, float v) { *dst = __float2bfloat16_rn(v); }

// A (M x K, column-major, lda, float) -> Ak (M rows x Kp, K contiguous, zero padded), via a 32 x 32 tile transpose.
template <typename TO>
__global__ void stage_a_kernel(int M, int K, int Kp, const float *A, int64_t lda, TO *Ak)
{
    __shared__ float tile[32][33];
    const int m0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int m = m0 + threadIdx.x, k = k0 + j;
        tile[j][threadIdx.x] = (m < M && k < K) ? A[m + (int64_t)k * lda] : 0.f;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        int m = m0 + j, k = k0 + threadIdx.x;
        if (m < M && k < Kp) cvt_store(Ak + (int64_t)m * Kp + k, tile[threadIdx.x][j]);
    }
}

// B (K x N, column-major, ldb, float) -> Bk (N rows x Kp, K contiguous): a copy per column.
template <typename TO>
__global__ void stage_b_kernel(int K, int N, int Kp, const float *B, int64_t ldb, TO *Bk)
{
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)N * Kp) return;
    int k = (int)(idx % Kp), n = (int)(idx / Kp);
    cvt_store(Bk + idx, k < K ? B[k + (int64_t)n * ldb] : 0.f);
}

// d_info <- -2 when a device wait of the factorization timed out
__global__ void status_to_info_kernel(const Status *st, int64_t *info)
{
    if (st->err != 0 && *info < 0) *info = -2;
}

// ----------------------------------------------------------- host helpers

static PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 2-D K-major operand: rows x Kp elements, box (128 bytes of K) x box_rows.
static bool make_map(CUtensorMap *map, const void *base, int rows, int Kp, int esize, int box_rows)
{
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * esize};
    cuuint32_t box[2] = {(cuuint32_t)(ROW_BYTES / esize), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace tc

// ------------------------------------------------------------------ API

// Workspace of one tensor-core update of at most n x n x kmax: staged A and B
// operands plus the status word.
static size_t stage_bytes(int64_t n, int prec, int kmax)
{
    size_t es = prec == RBT_BF16 ? 2 : 4;
    size_t kp = (size_t)((kmax + 63) / 64 * 64);
    return 2 * (size_t)n * kp * es + 1024;
}

constexpr int kOuterNB = 1024;  // K of the trailing update (two-level blocking)
constexpr int kInnerNB = 128;   // panel block (shared-memory diagonal factor)

size_t tc_update_workspace(int64_t n, int prec, int nb)
{
    (void)nb;
    if (n <= 0) return 0;
    return stage_bytes(n, prec, kOuterNB) + 256;
}

// C (M x N) -= A (M x K) B (K x N), all float column-major slices of the
// working matrix; one call stages the operands and launches the kernel.
static rbt_status tc_update(int prec, int M, int N, int K, const float *A, int64_t lda, const float *B, int64_t ldb,
                            float *C, int64_t ldc, const int64_t *info, void *work, tc::Status *st,
                            cudaStream_t stream)
{
    if (M <= 0 || N <= 0 || K <= 0) return RBT_OK;
    ProfScope ps(kProfUpdate, stream);
    const int es = prec == RBT_BF16 ? 2 : 4;
    const int kstep = tc::ROW_BYTES / es;
    const int Kp = (K + kstep - 1) / kstep * kstep;
    char *wa = (char *)work;
    char *wb = wa + (((size_t)M * Kp * es + 1023) / 1024 * 1024);
    dim3 tb(32, 8);
    dim3 ga((unsigned)cdiv(M, 32), (unsigned)cdiv(Kp, 32));
    int64_t nbk = (int64_t)N * Kp;
    if (prec == RBT_BF16) {
        tc::stage_a_kernel<__nv_bfloat16><<<ga, tb, 0, stream>>>(M, K, Kp, A, lda, (__nv_bfloat16 *)wa);
        RBT_LAUNCH_CHECK();
        tc::stage_b_kernel<__nv_bfloat16><<<(unsigned)cdiv(nbk, 256), 256, 0, stream>>>(K, N, Kp, B, ldb,
                                                                                         (__nv_bfloat16 *)wb);
        RBT_LAUNCH_CHECK();
    } else {
        tc::stage_a_kernel<float><<<ga, tb, 0, stream>>>(M, K, Kp, A, lda, (float *)wa);
        RBT_LAUNCH_CHECK();
        tc::stage_b_kernel<float><<<(unsigned)cdiv(nbk, 256), 256, 0, stream>>>(K, N, Kp, B, ldb, (float *)wb);
        RBT_LAUNCH_CHECK();
    }
    CUtensorMap ma, mb;
    if (!tc::make_map(&ma, wa, M, Kp, es, tc::BM) || !tc::make_map(&mb, wb, N, Kp, es, tc::BN))
        return RBT_ERR_CUDA;
    dim3 grid((unsigned)cdiv(M, tc::BM), (unsigned)cdiv(N, tc::BN));
    if (prec == RBT_BF16)
        tc::tc_update_kernel<0><<<grid, 128, tc::SMEM_BYTES, stream>>>(ma, mb, M, N, Kp, C, ldc, info, st,
                                                                        wait_limit_ns());
    else
        tc::tc_update_kernel<1><<<grid, 128, tc::SMEM_BYTES, stream>>>(ma, mb, M, N, Kp, C, ldc, info, st,
                                                                        wait_limit_ns());
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

static rbt_status tc_configure()
{
    static PerDeviceOnce once;
    return once_per_device(once, []() -> rbt_status {
        RBT_CUDA_TRY(cudaFuncSetAttribute(tc::tc_update_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tc::SMEM_BYTES));
        RBT_CUDA_TRY(cudaFuncSetAttribute(tc::tc_update_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tc::SMEM_BYTES));
        return RBT_OK;
    });
}

// Two-level blocked GENP: panels of kOuterNB columns are factored with
// kInnerNB inner steps (shared-memory diagonal factor, both TRSMs, tensor-core
// updates of the panel and of the row block to its right); then the trailing
// matrix takes one rank-kOuterNB tensor-core update.
rbt_status genp_factor_tc(int64_t n, int prec, float *A, int64_t lda, int64_t *info, void *work,
                          size_t work_bytes, int nb, cudaStream_t stream)
{
    (void)nb;
    if (n > (int64_t)1 << 30) return RBT_ERR_UNSUPPORTED;
    if (work_bytes < tc_update_workspace(n, prec, nb) || !work) return RBT_ERR_WORKSPACE;
    rbt_status s = tc_configure();
    if (s != RBT_OK) return s;
    tc::Status *st = (tc::Status *)((char *)work + stage_bytes(n, prec, kOuterNB));
    RBT_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(tc::Status), stream));
    for (int64_t k = 0; k < n; k += kOuterNB) {
        const int64_t kb = n - k < kOuterNB ? n - k : kOuterNB;
        for (int64_t j = k; j < k + kb; j += kInnerNB) {
            const int jb = (int)(k + kb - j < kInnerNB ? k + kb - j : kInnerNB);
            s = genp_panel_steps<float>(n, A, lda, info, jb, j, j + jb, false, stream);  // diag + both TRSMs
            if (s != RBT_OK) return s;
            const int64_t r0 = j + jb;
            // panel columns [j+jb, k+kb), all rows below
            s = tc_update(prec, (int)(n - r0), (int)(k + kb - r0), jb, A + r0 + j * lda, lda, A + j + r0 * lda, lda,
                          A + r0 + r0 * lda, lda, info, work, st, stream);
            if (s != RBT_OK) return s;
            // row block right of the panel: rows [j+jb, k+kb), columns [k+kb, n)
            s = tc_update(prec, (int)(k + kb - r0), (int)(n - k - kb), jb, A + r0 + j * lda, lda,
                          A + j + (k + kb) * lda, lda, A + r0 + (k + kb) * lda, lda, info, work, st, stream);
            if (s != RBT_OK) return s;
        }
        const int64_t t0 = k + kb;
        s = tc_update(prec, (int)(n - t0), (int)(n - t0), (int)kb, A + t0 + k * lda, lda, A + k + t0 * lda, lda,
                      A + t0 + t0 * lda, lda, info, work, st, stream);
        if (s != RBT_OK) return s;
    }
    tc::status_to_info_kernel<<<1, 1, 0, stream>>>(st, info);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

size_t tc_gemm_workspace(int64_t M, int64_t N, int64_t K, int prec)
{
    size_t es = prec == RBT_BF16 ? 2 : 4;
    size_t kp = (size_t)((K + 63) / 64 * 64);
    return ((size_t)M * kp * es + 1023) / 1024 * 1024 + (size_t)N * kp * es + 1024 + 256;
}

// One standalone update C -= A B (tensor cores); the status word sits after the operands.
rbt_status tc_gemm(int prec, int64_t M, int64_t N, int64_t K, const float *A, int64_t lda, const float *B, int64_t ldb,
                   float *C, int64_t ldc, int64_t *d_info, void *work, size_t work_bytes, cudaStream_t stream)
{
    if (work_bytes < tc_gemm_workspace(M, N, K, prec)) return RBT_ERR_WORKSPACE;
    if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return RBT_ERR_UNSUPPORTED;
    rbt_status s = tc_configure();
    if (s != RBT_OK) return s;
    tc::Status *st = (tc::Status *)((char *)work + tc_gemm_workspace(M, N, K, prec) - 256);
    RBT_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(tc::Status), stream));
    RBT_CUDA_TRY(cudaMemsetAsync(d_info, 0xff, sizeof(int64_t), stream));
    s = tc_update(prec, (int)M, (int)N, (int)K, A, lda, B, ldb, C, ldc, d_info, work, st, stream);
    if (s != RBT_OK) return s;
    tc::status_to_info_kernel<<<1, 1, 0, stream>>>(st, d_info);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}


}  // namespace rbt

using namespace rbt;

extern "C" {

size_t genp_update_workspace(int64_t M, int64_t N, int64_t K, int32_t prec)
{
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    if (prec == RBT_TF32 || prec == RBT_BF16) return tc_gemm_workspace(M, N, K, prec);
    if (is_sliced(prec)) return oz_update_workspace(M, N, K, sliced_digits(prec)) + 256;
    return 0;
}

rbt_status genp_update(int32_t prec, int64_t M, int64_t N, int64_t K, const float *A, int64_t lda, const float *B,
                       int64_t ldb, float *C, int64_t ldc, int64_t *d_status, void *work, size_t work_bytes,
                       cudaStream_t stream)
{
    if (M < 0 || N < 0 || K < 0 || !d_status) return RBT_ERR_ARG;
    if (prec != RBT_F32 && prec != RBT_TF32 && prec != RBT_BF16 && prec != RBT_DF64 && !is_sliced(prec))
        return RBT_ERR_ARG;
    if (lda < (M > 1 ? M : 1) || ldb < (K > 1 ? K : 1) || ldc < (M > 1 ? M : 1)) return RBT_ERR_ARG;
    if (M == 0 || N == 0 || K == 0) {
        RBT_CUDA_TRY(cudaMemsetAsync(d_status, 0xff, sizeof(int64_t), stream));
        return RBT_OK;
    }
    if (!A || !B || !C) return RBT_ERR_ARG;
    if (prec == RBT_F32) {
        RBT_CUDA_TRY(cudaMemsetAsync(d_status, 0xff, sizeof(int64_t), stream));
        if (K > INT32_MAX) return RBT_ERR_UNSUPPORTED;
        return gemm_sub_simt<float>(M, N, (int)K, A, lda, B, ldb, C, ldc, nullptr, stream);
    }
    if (prec == RBT_DF64) {
        RBT_CUDA_TRY(cudaMemsetAsync(d_status, 0xff, sizeof(int64_t), stream));
        if (K > INT32_MAX) return RBT_ERR_UNSUPPORTED;
        return gemm_sub_simt<df64>(M, N, (int)K, (const df64 *)A, lda, (const df64 *)B, ldb, (df64 *)C, ldc, nullptr,
                                   stream);
    }
    if (!work) return RBT_ERR_WORKSPACE;
    if (is_sliced(prec)) {
        if (work_bytes < genp_update_workspace(M, N, K, prec)) return RBT_ERR_WORKSPACE;
        const int digits = sliced_digits(prec);
        void *status = (char *)work + oz_update_workspace(M, N, K, digits);
        RBT_CUDA_TRY(cudaMemsetAsync(status, 0, 256, stream));
        RBT_CUDA_TRY(cudaMemsetAsync(d_status, 0xff, sizeof(int64_t), stream));
        rbt_status st = oz_update(M, N, K, (const df64 *)A, lda, (const df64 *)B, ldb, (df64 *)C, ldc, d_status, work,
                                  oz_update_workspace(M, N, K, digits), status, digits, stream);
        if (st != RBT_OK) return st;
        return oz_status_to_info(status, d_status, stream);
    }
    return tc_gemm(prec, M, N, K, A, lda, B, ldb, C, ldc, d_status, work, work_bytes, stream);
}

}  // extern "C"
