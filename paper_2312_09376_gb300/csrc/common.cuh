// Shared helpers of the CUDA path (sm_103a).  Nothing here is shared with the
// CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/rbt.h"

#define RBT_CUDA_TRY(call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return RBT_ERR_CUDA;          \
    } while (0)

// Every kernel launch of the library is followed by this check, which also
// counts the launch (rbt_kernel_launches()).
#define RBT_LAUNCH_CHECK()                                   \
    do {                                                     \
        rbt::count_launch();                                 \
        if (cudaPeekAtLastError() != cudaSuccess) {          \
            (void)cudaGetLastError();                        \
            return RBT_ERR_CUDA;                             \
        }                                                    \
    } while (0)

namespace rbt {

void count_launch();

// Optional per-class device timing (rbt_prof_*): events around launches.
enum ProfClass { kProfUpdate = 0, kProfTransform = 1, kProfPanel = 2, kProfSolve = 3, kProfResidual = 4,
                 kProfSlice = 5, kProfClasses = 6 };
bool prof_on();
void prof_record(int cls, cudaStream_t s, bool begin);

struct ProfScope {
    int cls;
    cudaStream_t s;
    bool on;
    ProfScope(int c, cudaStream_t st) : cls(c), s(st), on(prof_on())
    {
        if (on) prof_record(cls, s, true);
    }
    ~ProfScope()
    {
        if (on) prof_record(cls, s, false);
    }
};

// Working precisions stored as double-float pairs (8 bytes an entry), and
// the sliced tensor-core ones with their digit counts.
__host__ __device__ inline bool is_sliced(int prec) { return prec == RBT_DF64TC || prec == RBT_DF64TC7; }
__host__ __device__ inline bool is_df64_storage(int prec) { return prec == RBT_DF64 || is_sliced(prec); }
__host__ __device__ inline int sliced_digits(int prec) { return prec == RBT_DF64TC7 ? 7 : 8; }
constexpr int kLastPrec = 6;  // RBT_DF64TC7, the largest rbt_prec

constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (queried at run time where it matters)

__host__ __device__ inline int ceil_log2_i64(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n) c++;
    return c;
}

// Effective depth: layers past ceil(log2 n) are diagonal only.
__host__ __device__ inline int eff_depth(int64_t n, int d)
{
    int l = ceil_log2_i64(n);
    return d < l ? d : l;
}

// Non-tiled reference size of Sec. 3 at the effective depth.
__host__ __device__ inline int64_t ref_size(int64_t n, int d)
{
    int ds = eff_depth(n, d);
    int64_t p = (int64_t)1 << ds;
    return p * ((n + p - 1) / p);
}

// Tiled reference size of Sec. 3: the smallest multiple of 2^d_s * align that
// is >= n (align = the tile size n_b; 1 gives the non-tiled rule).
__host__ __device__ inline int64_t ref_size(int64_t n, int d, int64_t align)
{
    int ds = eff_depth(n, d);
    int64_t p = ((int64_t)1 << ds) * (align > 1 ? align : 1);
    return p * ((n + p - 1) / p);
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Least common multiple of two positive integers.
inline int64_t lcm_i64(int64_t p, int64_t q)
{
    int64_t a = p, b = q;
    while (b != 0) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return p / a * q;
}

constexpr int32_t kMaxGridSide = 4096;

// Alignment of the reference size for a tile size and an optional p x q
// process grid: Eq. (comm-free-rbt-size) of Sec. 6 is the tiled rule with
// tiles of lcm(p, q) n_b rows (ceil(ceil(n / n_b) / c) = ceil(n / (n_b c))).
inline int64_t effective_align(int64_t align, int32_t grid_p, int32_t grid_q)
{
    const int64_t a = align > 1 ? align : 1;
    return a * lcm_i64(grid_p > 1 ? grid_p : 1, grid_q > 1 ? grid_q : 1);
}

int device_sm_count();

// A one-shot set-up per device: once_per_device(o, fn) runs fn the first time
// it is called with a given device current and skips it afterwards on that
// device.  Kernel attributes (the opt-in to large dynamic shared memory) are
// per device context, so a process that drives several GPUs needs each of
// them set.  Thread-safe: two threads racing on a device's first call may
// both run fn, which every use here tolerates (the set-ups are idempotent).
struct PerDeviceOnce {
    std::atomic<unsigned long long> done{0ull};
};

template <typename F> rbt_status once_per_device(PerDeviceOnce &o, F fn)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RBT_ERR_CUDA;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (o.done.load(std::memory_order_acquire) & bit)) return RBT_OK;
    rbt_status st = fn();
    if (st == RBT_OK && bit) o.done.fetch_or(bit, std::memory_order_acq_rel);
    return st;
}

// Opt kernel k in to `bytes` of dynamic shared memory, once per device.
template <typename K> rbt_status smem_opt_in(PerDeviceOnce &o, K k, int bytes)
{
    return once_per_device(o, [&]() -> rbt_status {
        RBT_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        return RBT_OK;
    });
}

// Bounded device waits.  Every spin-wait of the library on another CTA or on
// an asynchronous copy gives up after wait_limit_ns() nanoseconds of
// %globaltimer, records a timeout and returns (rbt_debug_wait_limit).
constexpr long long kDefaultWaitNs = 1000000000LL;  // one second
long long wait_limit_ns();
// Test stall in effect (rbt_debug_stall): RBT_STALL_NONE in normal use.
int debug_stall();

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace rbt
