// Library-internal declarations shared by the C-ABI layer and the kernel
// translation units.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

constexpr int kDiagSlots = 12;  // accumulated slots of lbm_diagnostics

cudaError_t launch_init_eq(int storage, void* dst, const StepArgs& a,
                           float alpha_R, float alpha_B, const float* rR,
                           const float* rB, const float* u, cudaStream_t s);
cudaError_t launch_set_f(int storage, void* dst, const StepArgs& a,
                         const float* f, cudaStream_t s);
cudaError_t launch_get_f(int storage, const void* src, const StepArgs& a,
                         float* f, cudaStream_t s);
cudaError_t launch_moments(int storage, const void* src, const StepArgs& a,
                           float* rR, float* rB, float* u, cudaStream_t s);
cudaError_t launch_diag(int storage, const void* src, const StepArgs& a,
                        double* part, int nblocks, double* out,
                        cudaStream_t s);
cudaError_t launch_twopass(int storage, const void* src, void* dst,
                           const StepArgs& a, float4* mom, cudaStream_t s);

// Fused z-marching step.  `err` is a device word the kernel may set.
struct FusedConfig {
  int tile_x, tile_y;   // interior cells per CTA (x, y)
  int zchunk;           // planes marched per CTA
};
cudaError_t launch_fused(int storage, const void* src, void* dst,
                         const StepArgs& a, const FusedConfig& cfg,
                         cudaStream_t s);
FusedConfig default_fused_config(const StepArgs& a, int storage);

}  // namespace lbm
