// Tensor-core trailing update for the TF32 / BF16 GENP (sm_103a).
#include "gemm_tc.cuh"
#include "genp_internal.cuh"

namespace rbt {

size_t tc_update_workspace(int64_t n, int prec, int nb)
{
    (void)n;
    (void)prec;
    (void)nb;
    return 0;
}

rbt_status genp_factor_tc(int64_t n, int prec, float *A, int64_t lda, int64_t *info, void *work,
                          size_t work_bytes, int nb, cudaStream_t stream)
{
    (void)n; (void)prec; (void)A; (void)lda; (void)info; (void)work; (void)work_bytes; (void)nb; (void)stream;
    return RBT_ERR_UNSUPPORTED;
}

}  // namespace rbt
