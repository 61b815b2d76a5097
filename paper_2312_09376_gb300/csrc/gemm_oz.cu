// Double-float GENP update on BF16 tensor cores by exact integer slicing
// (sm_103a): C -= A B with A, B, C stored as double-float pairs.
//
// The product is split so that every tensor-core operation is exact, in the
// manner of the Ozaki scheme (Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012):
//   * each row i of A is scaled by 2^-e_i (|A_i.| < 2^(e_i - 1)) and each
//     column j of B by 2^-f_j, then written as S = 8 (or 7) balanced
//     base-128 digits,
//         A_ik = 2^e_i sum_p a_ik^(p) 2^(-7p),  a^(p) integers, |a^(p)| <= 64,
//     which BF16 (8 significant bits) holds exactly;
//   * the digit matrices are multiplied on the tensor cores with FP32
//     accumulation; a digit product is at most 2^12, and the at most S K
//     products of one weight sum exactly below 2^24 for K <= 512;
//   * products of equal weight t = p + q (t <= S + 1: 36 products for S = 8,
//     28 for S = 7) share a TMEM accumulator, and the epilogue folds the S
//     accumulators back into double-float: C_ij -= 2^(e_i + f_j) sum_t acc_t 2^(-7 t).
// The representation keeps 7S bits relative to each row's and column's
// largest entry; the dropped digit products (t >= S + 2) weigh about
// 2^-(7S - 3) of those per k.  The error is relative to those maxima, not to
// each entry, so it is larger than a double-float product's where rows or
// columns mix large and small entries.  GENP's panels do: column k of L21 carries 1/u_kk and row
// k of U12 carries u_kk, so a row of L21 spans many binades across k.  Before
// slicing, each k is therefore balanced by an exact power of two,
//     A_ik B_kj = (A_ik 2^t_k) (B_kj 2^-t_k),
//     t_k = floor((E(B_k.) - E(A_.k)) / 2),  E = binary exponent of the max,
// which brings the largest entries of column k of A and row k of B to the
// same binade (on RBT-transformed GENP panels the bound relative to the
// entrywise one drops from about 2^12 to 2^4 in the median).
//
// Kernel: persistent, one CTA per SM, 128 x 64 output tiles (S accumulators
// x 64 columns in the 512 TMEM columns) dealt round-robin in an L2-friendly
// grouped order; a TMA producer warp streams 32-element K slabs of all S
// digit slices of A and of B (64-byte rows, 64-byte swizzle) through a
// 2-stage ring across tile boundaries; one thread issues the MMAs of a slab
// (24 for S = 8, 20 for S = 7: each digit of A against up to four adjacent
// digit slices of B, N <= 256); eight epilogue warps fold the accumulators
// and update C while the next tile's first slabs load.  Bounded waits as in the TF32 / BF16
// kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "df64.cuh"
#include "gemm_tc.cuh"
#include "genp_internal.cuh"

namespace rbt {
namespace oz {

constexpr int BETA = 7;     // bits per digit
constexpr int BM = 128;
// TMEM holds one 128 x BN FP32 accumulator per digit weight t = 2 .. S + 1
// (S accumulators, S <= 8) in 512 columns.
constexpr int BN = 64;
constexpr int KSLAB = 32;   // bf16 elements per 64-byte row
constexpr int A_SLICE_BYTES = BM * 64;
constexpr int B_SLICE_BYTES = BN * 64;
// S digits per operand (7 or 8): the stage ring is sized per digit count
template <int S> constexpr int kStageBytes = S * (A_SLICE_BYTES + B_SLICE_BYTES);  // S = 8: 96 KB
template <int S> constexpr int kStages = (227 * 1024 - 2048) / kStageBytes<S>;     // S = 7, 8: 2
template <int S> constexpr int kSmemBytes = kStages<S> * kStageBytes<S> + 1024 + 256;
constexpr int kOzEpiWarps = 8;                    // epilogue warps (two per TMEM lane quarter)
constexpr int kProdWarp = kOzEpiWarps;            // TMA producer
constexpr int kMmaWarp = kOzEpiWarps + 1;         // MMA issuer, TMEM owner
constexpr int kOzThreads = (kOzEpiWarps + 2) * 32;
constexpr int TMEM_COLS = 512;
// a digit product is at most 64 * 64 = 2^12 and a weight holds at most S of
// them per k: S * K * 2^12 <= 2^24 keeps every accumulation exact
constexpr int KMAX = 512;
constexpr int kMaxDigits = 8;
static_assert(kMaxDigits * KMAX * 4096 <= (1 << 24), "digit accumulation must stay exact");
static_assert(kMaxDigits * BN <= TMEM_COLS, "one accumulator per digit weight in TMEM");
static_assert(kStages<8> >= 2 && kStages<7> >= 2, "at least double buffering");
constexpr int kGroupM = 16;  // row tiles per group of the tile order (L2 reuse of the digit slices)

struct Status {
    int err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

// Wait for phase `parity` of bar, for at most wait_ns of %globaltimer.
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

// K-major, 64-byte swizzle: 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc64(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;  // SWIZZLE_64B
    return d;
}

// instruction descriptor for an M = 128, N = n BF16 x BF16 -> FP32 MMA (n a multiple of 16, <= 256)
__host__ __device__ constexpr uint32_t idesc_n(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_n(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}

// Wait for this thread's TMEM loads; the loaded registers are operands, so
// that no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ __forceinline__ float pow2f(int e)
{
    // 2^e for the normal range of float
    e = e < -126 ? -126 : (e > 127 ? 127 : e);
    return __int_as_float((e + 127) << 23);
}

// Bounded wait that also gives up when another role of the CTA has given up
// (*abort set); a timeout records RBT_ERR_TIMEOUT and raises *abort.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t *bar, uint32_t parity, Status *st, volatile int *abort,
                                             long long wait_ns)
{
    if (mbar_test(bar, parity)) return true;  // the common case: no timer read
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (*abort) return false;
        if ((long long)(global_ns() - t0) > wait_ns) {
            atomicExch(&st->err, (int)RBT_ERR_TIMEOUT);
            *abort = 1;
            return false;
        }
    }
    return true;
}

// Output tile i of this CTA (tiles dealt round-robin over the grid, in the
// grouped order below).  Groups of kGroupM row tiles, columns outer and rows
// inner within a group: the tiles in flight at one time share a band of
// kGroupM x 128 rows of A's digit slices and a few column tiles of B's, both
// L2-resident, instead of every wave streaming A's slices from DRAM.
__device__ __forceinline__ void tile_origin(int64_t i, int tiles_m, int tiles_n, int &m0, int &n0)
{
    const int64_t t = blockIdx.x + i * gridDim.x;
    const int64_t per_group = (int64_t)kGroupM * tiles_n;
    const int grp = (int)(t / per_group), in_grp = (int)(t % per_group);
    const int first_m = grp * kGroupM;
    const int gm = tiles_m - first_m < kGroupM ? tiles_m - first_m : kGroupM;
    m0 = (first_m + in_grp % gm) * BM;
    n0 = (in_grp / gm) * BN;
}

// C (df64, M x N, ldc) -= A B from the digit slices; ea[m] / fb[n] are the
// row / column exponents.  Every wait gives up after wait_ns (then st->err
// records the timeout, the other roles stop, and TMEM is freed as usual);
// with no_copy set (a test stall) the producer issues no copy at all, so the
// MMA warp's first wait runs out.  A slices: rows p*Mp + a0 + m of the A map,
// B slices: rows q*Np + b0 + n of the B map (p, q = 0 .. S-1 for digits
// 1 .. S; Mp, Np the padded row counts of one digit slice, a0 and b0 the
// first slice row of this block: C may be a sub-block of the sliced product,
// with ea and fb offset to match).
//
// Persistent, one CTA per SM, warp-specialized:
//   warp kProdWarp   (one lane) TMA producer, running ahead over the slabs of
//                    this CTA's whole tile sequence through the STAGES ring;
//   warp kMmaWarp    (one lane) MMA issuer; owns the TMEM allocation;
//   warps 0 .. 7     epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and
//                    columns 32 (w / 4) .. + 31 of each accumulator.
// The accumulators fill all 512 TMEM columns, so the next tile's MMAs wait
// for the epilogue to release them (tmem_empty, signalled as soon as the
// last accumulator has been read, before its arithmetic and the update of
// C); the next tile's first slabs are loaded meanwhile, and each tile's
// block of C is prefetched into L2 while that tile's MMAs run.
// RAW (testing only): the epilogue writes the S accumulators themselves to
// raw[(t M + m) N + n] instead of folding them into C (ea, fb, C unused).
template <bool RAW, int S>
__global__ void __launch_bounds__(kOzThreads, 1)
oz_update_kernel(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_b, int M,
                 int N, int K, int Mp, int Np, int a0, int b0, const int *__restrict__ ea, const int *__restrict__ fb,
                 df64 *__restrict__ C, int64_t ldc, const int64_t *info, Status *st, long long wait_ns,
                 int no_copy, float *__restrict__ raw)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + kStages<S> * kStageBytes<S>);
    uint64_t *empty = full + kStages<S>;
    uint64_t *tmem_full = empty + kStages<S>;
    uint64_t *tmem_empty = tmem_full + 1;
    uint64_t *drain = tmem_empty + 1;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort = (volatile int *)(tmem_slot + 1);

    static_assert(S >= 5 && S <= kMaxDigits, "digit count");
    if (*((volatile const int64_t *)info) >= 0) return;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
    const int64_t ntiles = (int64_t)tiles_m * tiles_n;
    if ((int64_t)blockIdx.x >= ntiles) return;
    const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const int nk = (K + KSLAB - 1) / KSLAB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages<S>; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(tmem_full)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(tmem_empty)), "r"(kOzEpiWarps)
                     : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(drain)) : "memory");
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == kProdWarp) {
        if (lane == 0) {
            int64_t g = 0;
            for (int64_t i = 0; i < my_tiles && !*abort && !no_copy; i++) {
                int m0, n0;
                tile_origin(i, tiles_m, tiles_n, m0, n0);
                for (int kt = 0; kt < nk; kt++, g++) {
                    const int s = (int)(g % kStages<S>);
                    const int64_t r = g / kStages<S>;
                    if (r > 0 && !mbar_wait_ab(&empty[s], (uint32_t)((r - 1) & 1), st, abort, wait_ns)) break;
                    unsigned char *sa = smem + s * kStageBytes<S>;
                    unsigned char *sb = sa + S * A_SLICE_BYTES;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[s])),
                                 "r"(kStageBytes<S>)
                                 : "memory");
                    for (int p = 0; p < S; p++) {
                        tma_load_2d(sa + p * A_SLICE_BYTES, &tmap_a, kt * KSLAB, p * Mp + a0 + m0, &full[s]);
                        tma_load_2d(sb + p * B_SLICE_BYTES, &tmap_b, kt * KSLAB, p * Np + b0 + n0, &full[s]);
                    }
                }
            }
            // before the CTA may end: every load issued into a stage has landed
            for (int s = 0; s < kStages<S> && s < g; s++) {
                const int64_t last = g - 1 - ((g - 1 - s) % kStages<S>);  // last load issued into stage s
                mbar_wait(&full[s], (uint32_t)((last / kStages<S>) & 1), st, wait_ns);
            }
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            int64_t g = 0;
            for (int64_t i = 0; i < my_tiles && !*abort; i++) {
                if (i > 0 && !mbar_wait_ab(tmem_empty, (uint32_t)((i - 1) & 1), st, abort, wait_ns)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                bool ok = true;
                for (int kt = 0; kt < nk; kt++, g++) {
                    const int s = (int)(g % kStages<S>);
                    if (!mbar_wait_ab(&full[s], (uint32_t)((g / kStages<S>) & 1), st, abort, wait_ns)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_u32(smem + s * kStageBytes<S>);
                    const uint32_t sb = sa + S * A_SLICE_BYTES;
                    // Digit p of A meets digits q = 1 .. S + 1 - p of B, whose
                    // accumulators (weights p + q) are adjacent in TMEM and whose
                    // slices are adjacent in shared memory: one MMA covers up to
                    // four of them (N = 256).  p = 1 writes every accumulator first.
#pragma unroll
                    for (int p = 1; p <= S; p++) {
#pragma unroll
                        for (int q0 = 1; q0 <= S + 1 - p; q0 += 4) {
                            const int nq = (S + 1 - p - q0 + 1) < 4 ? (S + 1 - p - q0 + 1) : 4;
                            const uint32_t dcol = tmem + (uint32_t)((p + q0 - 2) * BN);
#pragma unroll
                            for (int kk = 0; kk < 2; kk++) {
                                const uint32_t acc = (kt > 0 || p > 1 || kk > 0) ? 1u : 0u;
                                mma_bf16_n(dcol, smem_desc64(sa + (p - 1) * A_SLICE_BYTES + kk * 32),
                                           smem_desc64(sb + (q0 - 1) * B_SLICE_BYTES + kk * 32), idesc_n(nq * BN),
                                           acc);
                            }
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(tmem_full);
            }
            // every MMA issued has completed before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, st, wait_ns);
        }
        __syncwarp();
    } else {
        // epilogue warps
        constexpr int EC = BN / 2;  // columns per warp
        const int q = warp % 4, ch = warp / 4;  // TMEM lane quarter, half of the tile's columns
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        for (int64_t i = 0; i < my_tiles; i++) {
            int m0, n0;
            tile_origin(i, tiles_m, tiles_n, m0, n0);
            const int row = m0 + q * 32 + lane;
            const bool rok = row < M;
            const int cbase = ch * EC;
            // this tile's block of C towards L2 while its MMAs run: 64
            // columns, nine addresses each (one per 16 rows and the last row)
            if (!RAW)
                for (int e = threadIdx.x; e < BN * 9; e += kOzEpiWarps * 32) {
                    const int c = e / 9, r = e % 9;
                    const int gi = m0 + (r < 8 ? r * 16 : BM - 1), gj = n0 + c;
                    if (gi < M && gj < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(C + gi + (int64_t)gj * ldc));
                }
            const int er = (!RAW && rok) ? ea[row] : 0;
            bool ok = mbar_wait_ab(tmem_full, (uint32_t)(i & 1), st, abort, wait_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = tmem + lane_base + (uint32_t)cbase;
            if constexpr (RAW) {
#pragma unroll 1
                for (int t = 0; t < S; t++) {
                    uint32_t a[EC];
                    tmem_ld32(base + (uint32_t)(t * BN), a);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (rok)
                        for (int j = 0; j < EC; j++) {
                            const int col = n0 + cbase + j;
                            if (col < N) raw[((int64_t)t * M + row) * N + col] = __uint_as_float(a[j]);
                        }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tmem_empty)) : "memory");
                continue;
            }
            // fold sum_t acc_t 2^(-7 t) into pairs (h, l), exactly term by
            // term, one accumulator (EC columns) at a time.  Two register
            // buffers: the next accumulator's TMEM load is issued before the
            // current one is folded; the accumulators go back to the MMA warp
            // as soon as the last of them has landed, before its fold.
            float h[EC], l[EC];
            uint32_t r0[EC], r1[EC];
            tmem_ld32(base, r0);
            tmem_wait32(r0);
            tmem_ld32(base + (uint32_t)BN, r1);
#pragma unroll
            for (int j = 0; j < EC; j++) {
                h[j] = __uint_as_float(r0[j]) * pow2f(-2 * BETA);
                l[j] = 0.f;
            }
#pragma unroll
            for (int t = 1; t < S; t++) {
                uint32_t(&cur)[EC] = (t & 1) ? r1 : r0;
                uint32_t(&nxt)[EC] = (t & 1) ? r0 : r1;
                tmem_wait32(cur);
                if (t + 1 < S) tmem_ld32(base + (uint32_t)((t + 1) * BN), nxt);
                if (t == S - 1) {
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tmem_empty)) : "memory");
                }
                const float w = pow2f(-(t + 2) * BETA);
#pragma unroll
                for (int j = 0; j < EC; j++) {
                    float s, e;
                    two_sum(h[j], __uint_as_float(cur[j]) * w, s, e);
                    h[j] = s;
                    l[j] = __fadd_rn(l[j], e);
                }
            }
            // C -= the folded product, eight columns per round of loads (outside
            // the accumulators' hold: the next tile's MMAs are running)
            if (rok) {
#pragma unroll
                for (int j0 = 0; j0 < EC; j0 += 8) {
                    df64 cv[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const int col = n0 + cbase + j0 + j;
                        cv[j] = col < N ? C[row + (int64_t)col * ldc] : df64(0);
                    }
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const int col = n0 + cbase + j0 + j;
                        if (col < N) {
                            const float sc = pow2f(er + fb[col]);
                            C[row + (int64_t)col * ldc] = cv[j] - df_norm(h[j0 + j] * sc, l[j0 + j] * sc);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------- slicing

// Balanced base-128 digits of round(v 2^(7 S - e)), v = hi + lo, |v| < 2^(e-1):
// the scaled value has at most 7 S - 1 bits and the leading digit stays within
// [-64, 64].  ldexpf scales exactly for any e (the scaled hi is below 2^55; a
// scaled lo that underflows rounds to 0).
template <int S> __device__ __forceinline__ void digits(df64 v, int e, int (&d)[S])
{
    // Y = rint(hi 2^(S BETA - e)) + rint(lo 2^(S BETA - e)) (|Y| < 2^(7 S - 1)),
    // written as S balanced base-2^BETA digits, most significant first.  Each
    // scaled part is an integer-valued float; it is split exactly at
    // 2^(4 BETA) into two 32-bit integers, so the digits come from 32-bit masks
    // and shifts: the low four from the low halves (carry into the high half),
    // the other S - 4 from the high halves.
    static_assert(S >= 5 && S <= 8 && BETA == 7, "the split at 2^28 leaves at most four digits above it");
    const float hs = rintf(ldexpf(v.hi, S * BETA - e));
    const float ls = rintf(ldexpf(v.lo, S * BETA - e));
    const float hh = rintf(hs * 0x1p-28f), lh = rintf(ls * 0x1p-28f);
    int low = __float2int_rn(fmaf(-hh, 0x1p28f, hs)) + __float2int_rn(fmaf(-lh, 0x1p28f, ls));  // |low| <= 2^28
    int high = __float2int_rn(hh) + __float2int_rn(lh);
#pragma unroll
    for (int p = S - 1; p >= S - 4; p--) {
        const int r = ((low & 127) ^ 64) - 64;  // low mod 128, in -64 .. 63
        d[p] = r;
        low = (low - r) >> BETA;
    }
    high += low;
#pragma unroll
    for (int p = S - 5; p >= 1; p--) {
        const int r = ((high & 127) ^ 64) - 64;
        d[p] = r;
        high = (high - r) >> BETA;
    }
    d[0] = high;
}

// A digit (an integer of at most 8 significant bits) as a bf16: it is exact in
// float (2^23 + 2^22 + r - (2^23 + 2^22) in float arithmetic), and its float's
// upper half is then the exact bf16.
__device__ __forceinline__ __nv_bfloat16 bf16_of_digit(int r)
{
    const float f = __int_as_float(0x4B400000 + r) - 12582912.0f;
    return __ushort_as_bfloat16((unsigned short)(__float_as_uint(f) >> 16));
}

// Binary exponent e of a nonzero float (|x| < 2^e <= 2 |x|); kNoExp for zero.
// kNoExp is the int whose four bytes are 0x80, so that one memset initializes
// the atomicMax targets below.
constexpr int kNoExp = (int)0x80808080u;
__device__ __forceinline__ int exp_of(float x)
{
    if (x == 0.f) return kNoExp;
    int e;
    frexpf(x, &e);
    return e;
}

// k-balancing exponents, stored as atomicMax targets (initialized to kNoExp):
// ka[k] = max over rows of E(A_ik), kb[k] = max over columns of E(B_kj).
// One launch for both: blocks [0, na) take A (block b: column k = b / ca,
// rows of chunk b % ca, 4096 rows each), the rest take B (64 columns each;
// threads over k, K <= 512: two per thread at most).
__global__ void __launch_bounds__(256) kexp_kernel(int M, int K, int N, int ca, int na, const df64 *__restrict__ A,
                                                   int64_t lda, const df64 *__restrict__ B, int64_t ldb, int *ka,
                                                   int *kb)
{
    const int b = blockIdx.x;
    if (b < na) {
        const int k = b / ca, chunk = b % ca;
        int e = kNoExp;
        const int r1 = min(M, (chunk + 1) * 4096);
        for (int r = chunk * 4096 + threadIdx.x; r < r1; r += 256) e = max(e, exp_of(A[r + (int64_t)k * lda].hi));
        for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        if (threadIdx.x % 32 == 0 && e > kNoExp) atomicMax(ka + k, e);
        return;
    }
    const int c0 = (b - na) * 64, c1 = min(N, c0 + 64);
    for (int k = threadIdx.x; k < K; k += 256) {
        int e = kNoExp;
        for (int c = c0; c < c1; c++) e = max(e, exp_of(B[k + (int64_t)c * ldb].hi));
        if (e > kNoExp) atomicMax(kb + k, e);
    }
}

// t_k of the balancing (0 where column k of A or row k of B is all zero)
__device__ __forceinline__ int kshift(const int *ka, const int *kb, int k)
{
    const int a = ka[k], b = kb[k];
    if (a == kNoExp || b == kNoExp) return 0;
    const int d = b - a;
    return d >= 0 ? d / 2 : -((1 - d) / 2);  // floor(d / 2)
}

// A (M x K df64, column-major lda) -> S digit slices, slice p at rows p*Mp.. of
// a K-major [S*Mp][Kp] bf16 array (rows >= M and columns >= K zero), and the
// row exponents.  32 rows per CTA, 256 threads.  The digit pass goes through
// a 32 x 32 shared tile: loaded with consecutive threads down a column of A,
// written with consecutive threads along k of one output row.
template <int S>
__device__ __forceinline__ void slice_rows_block(int blk, int M, int K, int Kp, int Mp, const df64 *__restrict__ A,
                                                 int64_t lda, const int *__restrict__ ka, const int *__restrict__ kb,
                                                 __nv_bfloat16 *out, int *ea)
{
    __shared__ int smax[32][9];
    __shared__ int sexp[32];
    __shared__ df64 tile[32][33];
    const int r = threadIdx.x % 32, kl = threadIdx.x / 32;  // 32 rows x 8 lanes of K
    const int m = blk * 32 + r;
    int emax = kNoExp;  // max over k of E(A_mk 2^t_k)
    if (m < M)
        for (int k = kl; k < K; k += 8) {
            const int e = exp_of(A[m + (int64_t)k * lda].hi);
            if (e != kNoExp) emax = max(emax, e + kshift(ka, kb, k));
        }
    smax[r][kl] = emax;
    __syncthreads();
    if (threadIdx.x < 32) {
        int mx = kNoExp;
        for (int j = 0; j < 8; j++) mx = max(mx, smax[threadIdx.x][j]);
        // the pair's low part can push |hi + lo| just past a power of two: one more bit of headroom
        int e = mx == kNoExp ? 0 : mx + 1;
        sexp[threadIdx.x] = e;
        int mm = blk * 32 + threadIdx.x;
        if (mm < M) ea[mm] = e;
    }
    const int kk = threadIdx.x % 32, rw = threadIdx.x / 32;  // digit pass: lane = k, warp = row (+ 8 j)
    for (int k0 = 0; k0 < Kp; k0 += 32) {
        __syncthreads();  // sexp ready; the previous tile consumed
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int k = k0 + kl + 8 * j;
            tile[r][kl + 8 * j] = (m < M && k < K) ? A[m + (int64_t)k * lda] : df64(0.f, 0.f);
        }
        __syncthreads();
        const int k = k0 + kk;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int rr = rw + 8 * j;
            const int mm = blk * 32 + rr;
            if (mm >= Mp) continue;
            int d[S];
            if (mm < M && k < K) {
                digits(tile[rr][kk], sexp[rr] - kshift(ka, kb, k), d);
            } else {
#pragma unroll
                for (int p = 0; p < S; p++) d[p] = 0;
            }
#pragma unroll
            for (int p = 0; p < S; p++) out[((int64_t)p * Mp + mm) * Kp + k] = bf16_of_digit(d[p]);
        }
    }
}

// B (K x N df64, column-major ldb) -> digit slices of B^T (rows n, K-major), column exponents.
// One warp per column.
template <int S>
__device__ __forceinline__ void slice_cols_warp(int n, int K, int N, int Kp, int Np, const df64 *__restrict__ B,
                                                int64_t ldb, const int *__restrict__ ka, const int *__restrict__ kb,
                                                __nv_bfloat16 *out, int *fb)
{
    const int lane = threadIdx.x % 32;
    if (n >= Np) return;
    int emax = kNoExp;  // max over k of E(B_kn 2^-t_k)
    if (n < N)
        for (int k = lane; k < K; k += 32) {
            const int e = exp_of(B[k + (int64_t)n * ldb].hi);
            if (e != kNoExp) emax = max(emax, e - kshift(ka, kb, k));
        }
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    const int e = emax == kNoExp ? 0 : emax + 1;
    if (lane == 0 && n < N) fb[n] = e;
    for (int k = lane; k < Kp; k += 32) {
        int d[S];
        if (n < N && k < K) {
            digits(B[k + (int64_t)n * ldb], e + kshift(ka, kb, k), d);
        } else {
#pragma unroll
            for (int p = 0; p < S; p++) d[p] = 0;
        }
#pragma unroll
        for (int p = 0; p < S; p++) out[((int64_t)p * Np + n) * Kp + k] = bf16_of_digit(d[p]);
    }
}

// Both slicings in one launch: blocks [0, nra) slice 32 rows of A each, the
// rest slice 8 columns of B each (one warp per column).
template <int S>
__global__ void __launch_bounds__(256, 4) slice_kernel(int M, int N, int K, int Kp, int Mp, int Np, int nra,
                                                    const df64 *__restrict__ A, int64_t lda,
                                                    const df64 *__restrict__ B, int64_t ldb,
                                                    const int *__restrict__ ka, const int *__restrict__ kb,
                                                    __nv_bfloat16 *sa, int *ea, __nv_bfloat16 *sb, int *fb)
{
    if ((int)blockIdx.x < nra) {
        slice_rows_block<S>(blockIdx.x, M, K, Kp, Mp, A, lda, ka, kb, sa, ea);
    } else {
        const int n = ((int)blockIdx.x - nra) * 8 + (int)threadIdx.x / 32;
        slice_cols_warp<S>(n, K, N, Kp, Np, B, ldb, ka, kb, sb, fb);
    }
}

__global__ void status_to_info_kernel(const Status *st, int64_t *info)
{
    if (st->err != 0 && *info < 0) *info = -2;
}

// ---------------------------------------------------------------- host side

static PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

static bool make_map(CUtensorMap *map, const void *base, int rows, int Kp, int box_rows)
{
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)KSLAB, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace oz

size_t oz_update_workspace(int64_t M, int64_t N, int64_t K, int digits)
{
    using namespace oz;
    const int64_t S = digits;
    const int64_t Mp = rup(M, BM), Np = rup(N, BN), Kp = rup(K, KSLAB);
    return (size_t)rup(S * Mp * Kp * 2, 1024) + (size_t)rup(S * Np * Kp * 2, 1024) + (size_t)rup(Mp * 4, 256) +
           (size_t)rup(Np * 4, 256) + 2 * (size_t)rup(Kp * 4, 256) + 256;
}

namespace oz {

template <int S> static rbt_status configure()
{
    static PerDeviceOnce once;
    static PerDeviceOnce once_raw;
    rbt_status st = smem_opt_in(once, oz_update_kernel<false, S>, kSmemBytes<S>);
    if (st != RBT_OK || S != 8) return st;
    return smem_opt_in(once_raw, oz_update_kernel<true, 8>, kSmemBytes<8>);
}

// One update's digit slices and exponents, carved from a workspace of
// oz_update_workspace(M, N, K, S) bytes (the layout that function sizes).
struct Slices {
    __nv_bfloat16 *sa, *sb;
    int *ea, *fb, *ka, *kb;
    int64_t M, N, K, Mp, Np, Kp;
};

static Slices carve(int64_t M, int64_t N, int64_t K, int S, void *work)
{
    Slices sl;
    sl.M = M;
    sl.N = N;
    sl.K = K;
    sl.Mp = rup(M, BM);
    sl.Np = rup(N, BN);
    sl.Kp = rup(K, KSLAB);
    char *w = (char *)work;
    sl.sa = (__nv_bfloat16 *)w;
    w += rup(S * sl.Mp * sl.Kp * 2, 1024);
    sl.sb = (__nv_bfloat16 *)w;
    w += rup(S * sl.Np * sl.Kp * 2, 1024);
    sl.ea = (int *)w;
    w += rup(sl.Mp * 4, 256);
    sl.fb = (int *)w;
    w += rup(sl.Np * 4, 256);
    sl.ka = (int *)w;
    w += rup(sl.Kp * 4, 256);
    sl.kb = (int *)w;
    return sl;
}

// The balancing exponents and digit slices of A (M x K) and B (K x N).
template <int S>
static rbt_status slice(const Slices &sl, const df64 *A, int64_t lda, const df64 *B, int64_t ldb, cudaStream_t stream)
{
    const int64_t M = sl.M, N = sl.N, K = sl.K;
    if (M <= 0 || N <= 0 || K <= 0) return RBT_OK;
    ProfScope pslice(kProfSlice, stream);
    // both exponent arrays start at kNoExp (every byte 0x80)
    RBT_CUDA_TRY(cudaMemsetAsync(sl.ka, 0x80, (size_t)rup(sl.Kp * 4, 256) * 2, stream));
    const int ca = (int)cdiv(M, 4096), na = ca * (int)K;
    kexp_kernel<<<(unsigned)(na + cdiv(N, 64)), 256, 0, stream>>>((int)M, (int)K, (int)N, ca, na, A, lda, B, ldb,
                                                                    sl.ka, sl.kb);
    RBT_LAUNCH_CHECK();
    const int nra = (int)cdiv(sl.Mp, 32);
    slice_kernel<S><<<(unsigned)(nra + cdiv(sl.Np, 8)), 256, 0, stream>>>(
        (int)M, (int)N, (int)K, (int)sl.Kp, (int)sl.Mp, (int)sl.Np, nra, A, lda, B, ldb, sl.ka, sl.kb, sl.sa, sl.ea,
        sl.sb, sl.fb);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

// C (Ms x Ns, ldc) -= rows [a0, a0 + Ms) of A times columns [b0, b0 + Ns) of
// B from the slices (a0 a multiple of BM, b0 of BN, both blocks inside the
// sliced product), on at most max_ctas CTAs.
template <int S>
static rbt_status multiply(const Slices &sl, int64_t a0, int64_t b0, int64_t Ms, int64_t Ns, df64 *C, int64_t ldc,
                           const int64_t *info, void *status, unsigned max_ctas, cudaStream_t stream)
{
    if (Ms <= 0 || Ns <= 0) return RBT_OK;
    if (a0 % BM || b0 % BN || a0 < 0 || b0 < 0 || a0 + Ms > sl.M || b0 + Ns > sl.N) return RBT_ERR_ARG;
    ProfScope ps(kProfUpdate, stream);
    CUtensorMap ma, mb;
    if (!make_map(&ma, sl.sa, (int)(S * sl.Mp), (int)sl.Kp, BM) || !make_map(&mb, sl.sb, (int)(S * sl.Np), (int)sl.Kp, BN))
        return RBT_ERR_CUDA;
    const int64_t ntiles = cdiv(Ms, BM) * cdiv(Ns, BN);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, max_ctas));
    oz_update_kernel<false, S><<<grid, kOzThreads, kSmemBytes<S>, stream>>>(
        ma, mb, (int)Ms, (int)Ns, (int)sl.Kp, (int)sl.Mp, (int)sl.Np, (int)a0, (int)b0, sl.ea + a0, sl.fb + b0, C,
        ldc, info, (Status *)status, wait_limit_ns(), debug_stall() == RBT_STALL_OZ_COPY ? 1 : 0, nullptr);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

template <int S>
static rbt_status update(int64_t M, int64_t N, int64_t K, const df64 *A, int64_t lda, const df64 *B, int64_t ldb,
                         df64 *C, int64_t ldc, const int64_t *info, void *work, void *status, unsigned max_ctas,
                         cudaStream_t stream)
{
    if (M <= 0 || N <= 0 || K <= 0) return RBT_OK;
    rbt_status s = configure<S>();
    if (s != RBT_OK) return s;
    const Slices sl = carve(M, N, K, S, work);
    s = slice<S>(sl, A, lda, B, ldb, stream);
    if (s != RBT_OK) return s;
    return multiply<S>(sl, 0, 0, M, N, C, ldc, info, status, max_ctas, stream);
}

}  // namespace oz

// C -= A B, all double-float column-major; K <= 512; digits = 7 or 8 per
// entry; at most max_ctas CTAs (0 = one per SM).
rbt_status oz_update(int64_t M, int64_t N, int64_t K, const df64 *A, int64_t lda, const df64 *B, int64_t ldb, df64 *C,
                     int64_t ldc, const int64_t *info, void *work, size_t work_bytes, void *status, int digits,
                     cudaStream_t stream, unsigned max_ctas)
{
    using namespace oz;
    if (M <= 0 || N <= 0 || K <= 0) return RBT_OK;
    if (digits != 7 && digits != 8) return RBT_ERR_ARG;
    if (K > KMAX || M > INT32_MAX / digits || N > INT32_MAX / digits) return RBT_ERR_UNSUPPORTED;
    if (work_bytes < oz_update_workspace(M, N, K, digits)) return RBT_ERR_WORKSPACE;
    const unsigned ctas = max_ctas ? max_ctas : (unsigned)device_sm_count();
    return digits == 7 ? update<7>(M, N, K, A, lda, B, ldb, C, ldc, info, work, status, ctas, stream)
                       : update<8>(M, N, K, A, lda, B, ldb, C, ldc, info, work, status, ctas, stream);
}

rbt_status oz_status_to_info(void *status, int64_t *info, cudaStream_t stream)
{
    oz::status_to_info_kernel<<<1, 1, 0, stream>>>((const oz::Status *)status, info);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

namespace oz {

// The test entry point takes eight digits per entry.
constexpr int kRawDigits = 8;

// Caller digits (int8, [kRawDigits][rows][K] row-major) -> the K-major bf16 slices the
// update kernel reads ([kRawDigits][rows_p][Kp], zero padding).
__global__ void digits_to_slices_kernel(int rows, int rows_p, int K, int Kp, const int8_t *__restrict__ d,
                                        __nv_bfloat16 *__restrict__ out)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)kRawDigits * rows_p * Kp;
    if (idx >= total) return;
    const int k = (int)(idx % Kp);
    const int64_t pr = idx / Kp;
    const int r = (int)(pr % rows_p), p = (int)(pr / rows_p);
    const int v = (r < rows && k < K) ? (int)d[((int64_t)p * rows + r) * K + k] : 0;
    out[idx] = bf16_of_digit(v);
}

}  // namespace oz

size_t oz_products_workspace(int64_t M, int64_t N, int64_t K)
{
    using namespace oz;
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    const int64_t Mp = rup(M, BM), Np = rup(N, BN), Kp = rup(K, KSLAB);
    return (size_t)rup(kRawDigits * Mp * Kp * 2, 1024) + (size_t)rup(kRawDigits * Np * Kp * 2, 1024) + 256;
}

// The update kernel's copy and tensor-core pipeline on caller digits, with the
// raw-accumulator epilogue.
rbt_status oz_products(int64_t M, int64_t N, int64_t K, const int8_t *da, const int8_t *db, float *acc, void *work,
                       size_t work_bytes, cudaStream_t stream)
{
    using namespace oz;
    if (M < 0 || N < 0 || K < 0) return RBT_ERR_ARG;
    if (M == 0 || N == 0 || K == 0) return RBT_OK;
    if (!da || !db || !acc) return RBT_ERR_ARG;
    if (K > KMAX || M > INT32_MAX / kRawDigits || N > INT32_MAX / kRawDigits) return RBT_ERR_UNSUPPORTED;
    if (!work || work_bytes < oz_products_workspace(M, N, K)) return RBT_ERR_WORKSPACE;
    rbt_status s = configure<kRawDigits>();
    if (s != RBT_OK) return s;
    const int64_t Mp = rup(M, BM), Np = rup(N, BN), Kp = rup(K, KSLAB);
    char *w = (char *)work;
    __nv_bfloat16 *sa = (__nv_bfloat16 *)w;
    w += rup(kRawDigits * Mp * Kp * 2, 1024);
    __nv_bfloat16 *sb = (__nv_bfloat16 *)w;
    w += rup(kRawDigits * Np * Kp * 2, 1024);
    Status *status = (Status *)w;             // [0, 8): status word, [8, 16): "no failed pivot" (-1)
    int64_t *info = (int64_t *)(w + 8);
    RBT_CUDA_TRY(cudaMemsetAsync(w, 0, 8, stream));
    RBT_CUDA_TRY(cudaMemsetAsync(info, 0xff, 8, stream));
    const int64_t ta = (int64_t)kRawDigits * Mp * Kp, tb = (int64_t)kRawDigits * Np * Kp;
    digits_to_slices_kernel<<<(unsigned)cdiv(ta, 256), 256, 0, stream>>>((int)M, (int)Mp, (int)K, (int)Kp, da, sa);
    RBT_LAUNCH_CHECK();
    digits_to_slices_kernel<<<(unsigned)cdiv(tb, 256), 256, 0, stream>>>((int)N, (int)Np, (int)K, (int)Kp, db, sb);
    RBT_LAUNCH_CHECK();
    CUtensorMap ma, mb;
    if (!make_map(&ma, sa, (int)(kRawDigits * Mp), (int)Kp, BM) || !make_map(&mb, sb, (int)(kRawDigits * Np), (int)Kp, BN))
        return RBT_ERR_CUDA;
    const int64_t ntiles = (Mp / BM) * (Np / BN);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, device_sm_count());
    oz_update_kernel<true, kRawDigits><<<grid, kOzThreads, kSmemBytes<kRawDigits>, stream>>>(ma, mb, (int)M, (int)N, (int)Kp, (int)Mp,
                                                                     (int)Np, 0, 0, nullptr, nullptr, nullptr, 0, info,
                                                                     status, wait_limit_ns(), 0, acc);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

}  // namespace rbt

extern "C" {

size_t rbt_debug_oz_products_workspace(int64_t M, int64_t N, int64_t K)
{
    return rbt::oz_products_workspace(M, N, K);
}

rbt_status rbt_debug_oz_products(int64_t M, int64_t N, int64_t K, const int8_t *da, const int8_t *db, float *acc,
                                 void *work, size_t work_bytes, cudaStream_t stream)
{
    return rbt::oz_products(M, N, K, da, db, acc, work, work_bytes, stream);
}

}  // extern "C"

namespace rbt {

constexpr int kOzOuterNB = 512;  // K of the trailing update (digit-product exactness bound)
constexpr int kOzInnerNB = 64;   // panel step (double-float diagonal factor and TRSMs)

size_t oz_factor_workspace(int64_t n)
{
    if (n <= 0) return 0;
    return oz_update_workspace(n, n, kOzOuterNB, oz::kMaxDigits) + 256;  // any digit count
}

namespace {

// Two-level blocked GENP in double-float: panels of 512 columns factored with
// 64-column steps (shared-memory diagonal factor and both TRSMs in
// double-float, sliced tensor-core updates of the panel and of the row block
// to its right), then one rank-512 sliced tensor-core update of the trailing
// matrix per panel.
template <int S>
rbt_status factor_oz(int64_t n, df64 *A, int64_t lda, int64_t *info, void *work, cudaStream_t stream)
{
    const size_t ws = oz_update_workspace(n, n, kOzOuterNB, oz::kMaxDigits);
    void *status = (char *)work + ws;
    RBT_CUDA_TRY(cudaMemsetAsync(status, 0, 256, stream));
    const unsigned sms = (unsigned)device_sm_count();
    rbt_status s;
    for (int64_t k = 0; k < n; k += kOzOuterNB) {
        const int64_t kb = n - k < kOzOuterNB ? n - k : kOzOuterNB;
        for (int64_t j = k; j < k + kb; j += kOzInnerNB) {
            const int jb = (int)(k + kb - j < kOzInnerNB ? k + kb - j : kOzInnerNB);
            s = genp_panel_steps<df64>(n, A, lda, info, jb, j, j + jb, false, stream);
            if (s != RBT_OK) return s;
            const int64_t r0 = j + jb;
            s = oz::update<S>(n - r0, k + kb - r0, jb, A + r0 + j * lda, lda, A + j + r0 * lda, lda,
                              A + r0 + r0 * lda, lda, info, work, status, sms, stream);
            if (s != RBT_OK) return s;
            s = oz::update<S>(k + kb - r0, n - k - kb, jb, A + r0 + j * lda, lda, A + j + (k + kb) * lda, lda,
                              A + r0 + (k + kb) * lda, lda, info, work, status, sms, stream);
            if (s != RBT_OK) return s;
        }
        const int64_t t0 = k + kb;
        s = oz::update<S>(n - t0, n - t0, kb, A + t0 + k * lda, lda, A + k + t0 * lda, lda, A + t0 + t0 * lda, lda,
                          info, work, status, sms, stream);
        if (s != RBT_OK) return s;
    }
    return oz_status_to_info(status, info, stream);
}

}  // namespace

// digits = 7 or 8 per entry of the sliced operands
rbt_status genp_factor_oz(int64_t n, df64 *A, int64_t lda, int64_t *info, void *work, size_t work_bytes, int digits,
                          cudaStream_t stream)
{
    if (work_bytes < oz_factor_workspace(n) || !work) return RBT_ERR_WORKSPACE;
    if (digits != 7 && digits != 8) return RBT_ERR_ARG;
    if (n > INT32_MAX / oz::kMaxDigits) return RBT_ERR_UNSUPPORTED;
    return digits == 7 ? factor_oz<7>(n, A, lda, info, work, stream) : factor_oz<8>(n, A, lda, info, work, stream);
}

}  // namespace rbt
