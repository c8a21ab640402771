// TMA-staged fused step kernels for float population storage (a translation
// unit of its own so that they compile in parallel with the other kernels).
#include "lbm_fused_tma.cuh"

namespace lbm {
template cudaError_t launch_fused_tma_storage<float>(const void*, void*, const StepArgs&,
                                                   const CUtensorMap*, int, int, int,
                                                   int*, cudaStream_t);
template cudaError_t launch_fused_tma_batch_storage<float>(
    const void*, void*, const BatchCase*, int, int, bool, const CUtensorMap*, int, int, int, int*,
    int, cudaStream_t);
template bool tma_config_fits_storage<float>(int, int);
template cudaError_t tma_set_wait_ns<float>(unsigned long long);

// SEAM forms (FP32, periodic in x and y, walls in z allowed): 34 x 15 with
// one stage, 34 x 12 with two.
cudaError_t launch_fused_tma_seam(const void* src, void* dst, const StepArgs& a, int tile_y,
                                  const CUtensorMap* maps6, int zchunk, int* err,
                                  cudaStream_t s, MonAcc* mon) {
  const int zc = zchunk > 0 ? zchunk : a.nz;
  const bool zwalls = a.wz != 0;  // x and y are periodic (seam_eligible)
  if (mon) {  // monitored form: the default 34 x 12 tile only
    if (tile_y != 12) return cudaErrorInvalidValue;
    return zwalls ? launch_tma_seam_v<34, 12, 2, true, true>(src, dst, a, maps6, zc, err, s, mon)
                  : launch_tma_seam_v<34, 12, 2, false, true>(src, dst, a, maps6, zc, err, s,
                                                              mon);
  }
  if (tile_y == 15)
    return zwalls ? launch_tma_seam_v<34, 15, 1, true>(src, dst, a, maps6, zc, err, s)
                  : launch_tma_seam_v<34, 15, 1, false>(src, dst, a, maps6, zc, err, s);
  if (tile_y == 12)
    return zwalls ? launch_tma_seam_v<34, 12, 2, true>(src, dst, a, maps6, zc, err, s)
                  : launch_tma_seam_v<34, 12, 2, false>(src, dst, a, maps6, zc, err, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_tma_seam_batch(const void* src, void* dst, const BatchCase* cases,
                                        int ncases, int total_items, bool walls,
                                        const CUtensorMap* maps6, int zc, int* err, int sms,
                                        cudaStream_t s) {
  return walls ? launch_tma_seam_batch_v<true>(src, dst, cases, ncases, total_items, maps6, zc,
                                               err, sms, s)
               : launch_tma_seam_batch_v<false>(src, dst, cases, ncases, total_items, maps6, zc,
                                                err, sms, s);
}
}  // namespace lbm
