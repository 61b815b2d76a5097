// Kernels of the batched RBT solver and of its adjoint, with their launchers.
//
// Each working precision and variant (threads per CTA, GENP block size) is a
// whole solver inlined into one persistent kernel.  The build compiles this
// file once per (precision, variant) with RBT_BAT_PREC (0 = double, 1 =
// float), RBT_BAT_NT and RBT_BAT_NB defined, so that NVVM optimises every
// instantiation at its full level in objects built in parallel; without those
// macros the file holds all eight (one long compilation).
#include "batched_dev.cuh"

namespace rbt {
namespace bat {

template <typename T, int NT, int NB> rbt_status run_batched(const BatchedLaunch &a, cudaStream_t stream)
{
    int per_sm = 1;
    RBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<T, NT, NB>, NT, 0));
    int grid = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    if (grid > a.batch) grid = a.batch;
    batched_kernel<T, NT, NB><<<grid, NT, 0, stream>>>(a.descs, a.order, a.batch, a.counter, a.infos, a.sys_base,
                                                       a.depth, a.refine_max, a.tol, a.fallback, a.redo);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

template <typename T, int NT, int NB> rbt_status run_adjoint(const BatchedLaunch &a, cudaStream_t stream)
{
    int per_sm = 1;
    RBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_adjoint_kernel<T, NT, NB>, NT, 0));
    int grid = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    if (grid > a.batch) grid = a.batch;
    batched_adjoint_kernel<T, NT, NB><<<grid, NT, 0, stream>>>(a.descs, a.adj, a.order, a.batch, a.counter,
                                                               a.infos, a.sys_base, a.depth, a.refine_max, a.tol,
                                                               a.redo);
    RBT_LAUNCH_CHECK();
    return RBT_OK;
}

#define RBT_BAT_INSTANTIATE(T, NT, NB)                                                     \
    template rbt_status run_batched<T, NT, NB>(const BatchedLaunch &, cudaStream_t);       \
    template rbt_status run_adjoint<T, NT, NB>(const BatchedLaunch &, cudaStream_t);

#if defined(RBT_BAT_PREC) && defined(RBT_BAT_NT) && defined(RBT_BAT_NB)
#if RBT_BAT_PREC == 0
RBT_BAT_INSTANTIATE(double, RBT_BAT_NT, RBT_BAT_NB)
#else
RBT_BAT_INSTANTIATE(float, RBT_BAT_NT, RBT_BAT_NB)
#endif
#else
RBT_BAT_INSTANTIATE(double, 128, 16)
RBT_BAT_INSTANTIATE(double, 128, 32)
RBT_BAT_INSTANTIATE(double, 256, 16)
RBT_BAT_INSTANTIATE(double, 256, 32)
RBT_BAT_INSTANTIATE(float, 128, 16)
RBT_BAT_INSTANTIATE(float, 128, 32)
RBT_BAT_INSTANTIATE(float, 256, 16)
RBT_BAT_INSTANTIATE(float, 256, 32)
#endif

}  // namespace bat
}  // namespace rbt
