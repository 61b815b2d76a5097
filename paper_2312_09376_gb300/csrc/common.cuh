// Shared helpers of the CUDA path (sm_103a).  Nothing here is shared with the
// CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

int device_sm_count();

}  // namespace rbt
