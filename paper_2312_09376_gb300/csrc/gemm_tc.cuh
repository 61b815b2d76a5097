// Tensor-core (tcgen05 / TMEM) trailing update of the mixed-precision GENP.
#pragma once

#include "common.cuh"

namespace rbt {

size_t tc_update_workspace(int64_t n, int prec, int nb);

// GENP of a float matrix whose trailing updates run on the tensor cores
// (prec = RBT_TF32 or RBT_BF16).
rbt_status genp_factor_tc(int64_t n, int prec, float *A, int64_t lda, int64_t *info, void *work,
                          size_t work_bytes, int nb, cudaStream_t stream);

size_t tc_gemm_workspace(int64_t M, int64_t N, int64_t K, int prec);
rbt_status tc_gemm(int prec, int64_t M, int64_t N, int64_t K, const float *A, int64_t lda, const float *B, int64_t ldb,
                   float *C, int64_t ldc, int64_t *d_info, void *work, size_t work_bytes, cudaStream_t stream);

struct df64;
// digits = 7 or 8 balanced 7-bit digits per sliced entry
size_t oz_update_workspace(int64_t M, int64_t N, int64_t K, int digits);
rbt_status oz_update(int64_t M, int64_t N, int64_t K, const df64 *A, int64_t lda, const df64 *B, int64_t ldb, df64 *C,
                     int64_t ldc, const int64_t *info, void *work, size_t work_bytes, void *status, int digits,
                     cudaStream_t stream, unsigned max_ctas = 0);
rbt_status oz_status_to_info(void *status, int64_t *info, cudaStream_t stream);
size_t oz_factor_workspace(int64_t n);
rbt_status genp_factor_oz(int64_t n, df64 *A, int64_t lda, int64_t *info, void *work, size_t work_bytes, int digits,
                          cudaStream_t stream);

}  // namespace rbt
