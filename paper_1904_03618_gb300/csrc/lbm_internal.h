// Library-internal declarations shared by the C-ABI layer and the kernel
// translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

constexpr int kDiagSlots = 13;  // accumulated slots of lbm_diagnostics

// Host helpers of the C-ABI layer.  Errors without a context are recorded
// for lbm_last_error(NULL) of the calling thread.
lbm_status validate_params(const lbm_params* p);
StepArgs derive_step_args(const lbm_params* p, long long plane);
lbm_status fail_without_context(lbm_status s, const char* msg);
bool is_device_pointer(const void* ptr);
void clear_thread_error();

cudaError_t launch_init_eq(int storage, void* dst, const StepArgs& a,
                           float alpha_R, float alpha_B, const float* rR,
                           const float* rB, const float* u, cudaStream_t s);
cudaError_t launch_set_f(int storage, void* dst, const StepArgs& a,
                         const float* f, cudaStream_t s);
cudaError_t launch_get_f(int storage, const void* src, const StepArgs& a,
                         float* f, cudaStream_t s);
cudaError_t launch_moments(int storage, const void* src, const StepArgs& a,
                           float* rR, float* rB, float* u, cudaStream_t s);
cudaError_t launch_footprint(int storage, const void* src, const StepArgs& a, int axis,
                             int index, unsigned long long* count, cudaStream_t s);
cudaError_t launch_diag(int storage, const void* src, const StepArgs& a,
                        double* part, int nblocks, double* out,
                        cudaStream_t s);
cudaError_t launch_twopass(int storage, const void* src, void* dst,
                           const StepArgs& a, float4* mom, cudaStream_t s);

// Fused z-marching step.
struct FusedConfig {
  int tile_y;  // CTA rows including the ring: 8 or 16 (interior 30 x (tile_y - 2))
  int zchunk;  // planes marched per CTA (> 0)
  int hold;    // where plane z waits between its two uses: 0 re-pulled from
               // L1/L2, 1 registers, 2 shared memory (tile_y = 8 only),
               // 3 shared memory with cp.async prefetch of plane z + 2
               // (tile_y = 8), 4 shared memory with two tile rows per
               // thread (tile_y = 16), 5 / 6 as 2 with registers capped
               // for 3 / 4 CTAs per SM
};
template <typename T>
cudaError_t launch_fused_storage(const void* src, void* dst, const StepArgs& a,
                                 const FusedConfig& cfg, cudaStream_t s);
cudaError_t launch_fused(int storage, const void* src, void* dst,
                         const StepArgs& a, const FusedConfig& cfg,
                         cudaStream_t s);
FusedConfig default_fused_config(const StepArgs& a, int storage);

// One case of a batch, as the batched kernel sees it.
struct BatchCase {
  StepArgs args;          // plane = the case's padded cell count
  long long pair_base;    // offset of the case, in (red, blue) pairs, within
                          // each population buffer
  int item_start;         // first work item of the case
  int tiles_x, tiles_y;   // 30 x (tile_y - 2) interior tiles
  int pad_;
};
template <typename T>
cudaError_t launch_fused_batch_storage(const void* src, void* dst,
                                       const BatchCase* cases, int ncases,
                                       int total_items, bool walls,
                                       const FusedConfig& cfg, int sms,
                                       cudaStream_t s);
cudaError_t launch_fused_batch(int storage, const void* src, void* dst,
                               const BatchCase* cases, int ncases,
                               int total_items, bool walls,
                               const FusedConfig& cfg, int sms, cudaStream_t s);
bool valid_batch_config(const FusedConfig& c);
bool valid_fused_config(const FusedConfig& c, int storage);

}  // namespace lbm
