// Fused step kernels for __half population storage (one translation unit per
// storage type so that the variants compile in parallel).
#include "lbm_fused.cuh"

namespace lbm {
template cudaError_t launch_fused_storage<__half>(const void*, void*,
                                              const StepArgs&,
                                              const FusedConfig&,
                                              cudaStream_t);
template cudaError_t launch_fused_batch_storage<__half>(const void*, void*,
                                                    const BatchCase*, int, int,
                                                    bool, bool, const FusedConfig&, int,
                                                    cudaStream_t);
}  // namespace lbm
