// Storage-type dispatch and launch configuration of the fused step.
#include "lbm_internal.h"

namespace lbm {

cudaError_t launch_fused(int storage, const void* src, void* dst,
                         const StepArgs& a, const FusedConfig& cfg,
                         cudaStream_t s) {
  switch (storage) {
    case 0: return launch_fused_storage<float>(src, dst, a, cfg, s);
    case 1: return launch_fused_storage<__half>(src, dst, a, cfg, s);
    case 2: return launch_fused_storage<__nv_bfloat16>(src, dst, a, cfg, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_batch(int storage, const void* src, void* dst,
                               const BatchCase* cases, int ncases,
                               int total_items, bool walls,
                               const FusedConfig& cfg, int sms, cudaStream_t s) {
  switch (storage) {
    case 0: return launch_fused_batch_storage<float>(src, dst, cases, ncases, total_items, walls, cfg, sms, s);
    case 1: return launch_fused_batch_storage<__half>(src, dst, cases, ncases, total_items, walls, cfg, sms, s);
    case 2: return launch_fused_batch_storage<__nv_bfloat16>(src, dst, cases, ncases, total_items, walls, cfg, sms, s);
  }
  return cudaErrorInvalidValue;
}

// Batched kernel variants: (tile_y, hold) = (8, 2), (8, 0), (16, 1).
bool valid_batch_config(const FusedConfig& c) {
  const bool shape = (c.tile_y == 8 && (c.hold == 2 || c.hold == 0)) ||
                     (c.tile_y == 16 && c.hold == 1);
  return shape && c.zchunk > 0;
}

bool valid_fused_config(const FusedConfig& c, int storage) {
  if (c.tile_y != 8 && c.tile_y != 16) return false;
  if (c.hold < 0 || c.hold > 6) return false;
  if ((c.hold == 2 || c.hold == 3 || c.hold >= 5) && c.tile_y != 8) return false;
  if (c.hold == 4 && c.tile_y != 16) return false;
  (void)storage;
  return c.zchunk > 0;
}

// Default: 30 x 6 interior tiles, reduced state held in shared memory, and
// chunks of 12 planes (each chunk re-reads two extra planes for its halo),
// shortened down to 4 planes while the grid has fewer than two CTAs per SM
// over the 152 SMs.  Measured on GB300 at 128^3 (FP32 and FP16 storage):
// 8- and 12-plane chunks are best; 16, 24 and 32 are slower, as are the
// register-capped, two-rows-per-thread and cp.async-pipelined variants.
FusedConfig default_fused_config(const StepArgs& a, int storage) {
  (void)storage;
  FusedConfig c;
  c.tile_y = 8;
  c.hold = 2;
  const long long cols = (long long)((a.nx + 29) / 30) * ((a.ny + 5) / 6);
  int zc = 12;
  while (zc > 4 && cols * ((a.nz + zc - 1) / zc) < 2 * 152) zc /= 2;
  if (zc > a.nz) zc = a.nz;
  c.zchunk = zc;
  return c;
}

}  // namespace lbm
