// TMA-staged fused step kernels for __half population storage (a translation
// unit of its own so that they compile in parallel with the other kernels).
#include "lbm_fused_tma.cuh"

namespace lbm {
template cudaError_t launch_fused_tma_storage<__half>(const void*, void*, const StepArgs&,
                                                   const CUtensorMap*, int, int, int,
                                                   int*, cudaStream_t);
template cudaError_t launch_fused_tma_batch_storage<__half>(
    const void*, void*, const BatchCase*, int, int, bool, const CUtensorMap*, int, int, int, int*,
    int, cudaStream_t);
template bool tma_config_fits_storage<__half>(int, int);
template cudaError_t tma_set_wait_ns<__half>(unsigned long long);
template cudaError_t launch_fused_tma_seam16_storage<__half>(const void*, void*, const StepArgs&,
                                                         int, const CUtensorMap*, int, int*,
                                                         cudaStream_t, MonAcc*);
}  // namespace lbm
