// Library-internal declarations shared by the C-ABI layer and the kernel
// translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// Launch-time facts that belong to a device's context (function attributes,
// occupancy) are cached per device, so that one process may drive several
// GPUs (device ordinals from 64 up share slot 0's cache).
constexpr int kMaxDevices = 64;
inline int device_slot() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) d = 0;
  return d;
}


// NVTX range around a host entry point: the calls show up by name on the
// Nsight Systems timeline; without an attached tool a push / pop is a
// check of one pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kDiagSlots = 13;  // accumulated slots of lbm_diagnostics

// Diagnostics summed inside a monitored step (lbm_step_monitored) over the
// state the step reads: one record per CTA in shared memory, added into one
// global record per step.
struct MonAcc {
  double d[8];      // red mass, blue mass, momentum x, y, z, red-mass moments x, y, z
  unsigned n[4];    // cells: non-finite, total density <= 0, red (rho^N > 0), a colour < 0
  unsigned u2bits;  // largest |u|^2 as float bits (>= 0, so the bits order like the values)
  unsigned pad_[3];
};
// Writes the 16 slots of lbm_diagnostics from a step's record (slot 12 =
// steps, slot 14 = the error word) to out and clears the record.
cudaError_t launch_monitor_out(MonAcc* acc, const int* flags, double steps, double* out,
                               cudaStream_t s);

// Host helpers of the C-ABI layer.  Errors without a context are recorded
// for lbm_last_error(NULL) of the calling thread.
lbm_status validate_params(const lbm_params* p);
// validate_params without the cell-count limit of the two-buffer kernels
// (32-bit pair offsets), for the 64-bit in-place step.
lbm_status validate_params_any_size(const lbm_params* p);
StepArgs derive_step_args(const lbm_params* p, long long plane);
lbm_status fail_without_context(lbm_status s, const char* msg);
// LBM_OK if ptr is device (or managed) memory usable on the current GPU;
// else LBM_ERR_ARG with a message naming `what` (host memory, or device
// memory of another GPU) for lbm_last_error(NULL).
lbm_status require_current_device(const void* ptr, const char* what);
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
// Diagnostics into the 16 result slots out[] of lbm_diagnostics (device
// memory), with steps in [12] and the error word *flags in [14]; part holds
// max_blocks * kDiagSlots doubles, max_blocks from diag_capacity (the blocks
// resident at once); *done is a block counter, zero between launches (the
// kernel re-arms it).
cudaError_t launch_diag(int storage, const void* src, const StepArgs& a,
                        double* part, int max_blocks, unsigned* done,
                        const int* flags, long long steps, double* out,
                        cudaStream_t s);
int diag_capacity(int storage, int sms);
// Moving plates on both faces of `axis` (wall = 2): rebuilds, in buf (the
// state just written by a step), each colour's populations entering from
// beyond a plate (Zou-He velocity nodes, velocities u[low / high]).
cudaError_t launch_plates(int storage, void* buf, const StepArgs& a, int axis,
                          const double u[2][3], cudaStream_t s);
cudaError_t launch_twopass(int storage, const void* src, void* dst,
                           const StepArgs& a, float4* mom, cudaStream_t s);

// Fused z-marching step.
struct FusedConfig {
  int tile_y;  // CTA rows including the ring: 8 or 16 (interior 30 x (tile_y - 2));
               // 16 with hold 7 / 8 is the 16 x 16 thread tile, 15 (hold 7 / 8
               // only) the 34 x 15 tile
  int zchunk;  // planes marched per CTA (> 0)
  int hold;    // where plane z waits between its two uses: 0 re-pulled from
               // L1/L2, 1 registers, 2 shared memory (tile_y = 8 only),
               // 3 shared memory with cp.async prefetch of plane z + 2
               // (tile_y = 8), 4 shared memory with two tile rows per
               // thread (tile_y = 16), 5 / 6 as 2 with registers capped
               // for 3 / 4 CTAs per SM, 7 / 8 shared memory with the
               // pulls staged by tensor copies (TMA) in two / one stages
};
template <typename T>
cudaError_t launch_fused_storage(const void* src, void* dst, const StepArgs& a,
                                 const FusedConfig& cfg, cudaStream_t s);
cudaError_t launch_fused(int storage, const void* src, void* dst,
                         const StepArgs& a, const FusedConfig& cfg,
                         cudaStream_t s);
FusedConfig default_fused_config(const StepArgs& a, int storage);

// TMA-staged fused step (hold 7: two stages, hold 8: one stage).  Tile
// kinds: 0 = 32 x 8 threads (tile_y 8), 1 = 16 x 16 (tile_y 16), 2 = 34 x 15
// (tile_y 15).  Needs an x row of 16-byte multiple length (nx even for
// FP32, nx a multiple of 4 for 16-bit storage); maps[2] are the two tensor
// maps of the source buffer for the tile (tma_build_maps).
bool tma_eligible(const StepArgs& a, int storage);
// The driver's cuTensorMapEncodeTiled, looked up once.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
cudaError_t tensor_map_encoder(EncodeTiledFn* out);
int tma_kind(int tile_y);  // -1 for a tile_y without a TMA form
cudaError_t tma_build_maps(int storage, const void* base, const StepArgs& a, int kind,
                           CUtensorMap maps[2]);
// SEAM forms of the TMA step (34 x 15 threads with one stage, 34 x 12 with
// two; tile_y 15 or 12): FP32 storage, periodic in x and y (walls in z
// allowed), nx >= 34 and
// ny >= 15 (no tile on both seams of an axis), TMA eligible.  Their six maps
// (main 34 and 36 wide, x strip 2 wide, y strips 34 and 36 x 2, corner
// 2 x 2; main and x strip tile_y rows) over the source buffer.
bool seam_eligible(const StepArgs& a, int storage);
cudaError_t tma_build_seam_maps(const void* base, const StepArgs& a, int tile_y,
                                CUtensorMap maps[6]);
// mon (monitored form, tile_y 12 only; else nullptr): the step also adds
// the diagnostics of the state it reads into *mon.
cudaError_t launch_fused_tma_seam(const void* src, void* dst, const StepArgs& a, int tile_y,
                                  const CUtensorMap* maps6, int zchunk, int* err,
                                  cudaStream_t s, MonAcc* mon = nullptr);
// 16-bit SEAM forms (FP16 / BF16, 34 x 15 or 34 x 12 threads, two stages;
// tile_y 15 or 12): periodic in x and y (walls in z allowed), nx a multiple
// of 4, nx >= 34 and ny >= 15.  Four maps over the source buffer: main (38
// rounded up to 40 pairs x tile_y), x strip (4 x tile_y), y strip (40 x 2),
// corner (4 x 2).
bool seam16_eligible(const StepArgs& a, int storage);
cudaError_t tma_build_seam16_maps(int storage, const void* base, const StepArgs& a, int tile_y,
                                  CUtensorMap maps[4]);
template <typename T>
cudaError_t launch_fused_tma_seam16_storage(const void* src, void* dst, const StepArgs& a,
                                            int tile_y, const CUtensorMap* maps4, int zchunk,
                                            int* err, cudaStream_t s, MonAcc* mon);
cudaError_t launch_fused_tma_seam16(int storage, const void* src, void* dst, const StepArgs& a,
                                    int tile_y, const CUtensorMap* maps4, int zchunk, int* err,
                                    cudaStream_t s, MonAcc* mon = nullptr);
// z chunk of the 34 x 12 two-stage SEAM form: the one whose list schedule of
// CTAs over the SMs ends first.
int seam12_zchunk(const StepArgs& a, int sms);
// The same list-schedule model for a 34-wide tile of `rows` interior rows
// (one CTA per SM): 10 for the 34 x 12 tile, 13 for the 34 x 15 tile.
int list_schedule_zchunk(const StepArgs& a, int sms, int rows);
bool tma_config_fits(int storage, int kind, int ns);
// Interior width of a tile (30, or 32 for the 34-wide tiles: tile_y 15, 12).
inline int tile_interior_x(int tile_y) { return tile_y == 15 || tile_y == 12 ? 32 : 30; }
// A batch case the batched SEAM form (34 x 12, two stages) can run: FP32,
// periodic in x and y, TMA eligible, MRT.  Cases narrower than a tile in x
// or y run it too: lanes whose sources wrap across the far seam of a tile
// that spans both seams of an axis pull from global memory.
bool batch_seam_eligible(const StepArgs& a, int storage);
// Default TMA configuration for a single lattice (false: keep the plain one).
bool tma_default_config(const StepArgs& a, int storage, int sms, const bool kind_ok[3],
                        FusedConfig* out);
template <typename T>
bool tma_config_fits_storage(int kind, int ns);
// Give-up limit of the TMA stage waits (0: the default, 20 ms) on the
// current device, per storage type's kernels; for tests of the give-up path.
template <typename T>
cudaError_t tma_set_wait_ns(unsigned long long ns);
// The same for the tensor-core commit waits of the surrogate's GEMM
// (default 200 ms).
cudaError_t mlp_set_wait_ns(unsigned long long ns);

// Device and pinned host allocations of the library, counted; a testing
// hook (lbm_test_fail_allocation) makes the n-th next one fail.
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
cudaError_t host_alloc(void** p, size_t bytes);
void host_free(void* p);
template <typename T>
cudaError_t launch_fused_tma_storage(const void* src, void* dst, const StepArgs& a,
                                     const CUtensorMap* maps, int kind, int ns, int zchunk,
                                     int* err, cudaStream_t s);
cudaError_t launch_fused_tma(int storage, const void* src, void* dst, const StepArgs& a,
                             const CUtensorMap* maps, int kind, int ns, int zchunk, int* err,
                             cudaStream_t s);

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
                                       int total_items, bool walls, bool bgk,
                                       const FusedConfig& cfg, int sms,
                                       cudaStream_t s);
// bgk: every case uses the BGK operator (the (8, hold 2) form only)
cudaError_t launch_fused_batch(int storage, const void* src, void* dst,
                               const BatchCase* cases, int ncases,
                               int total_items, bool walls, bool bgk,
                               const FusedConfig& cfg, int sms, cudaStream_t s);
// Batched TMA step (kind 0 or 2): maps = the device table of the source
// buffer's tensor maps, two per case.
template <typename T>
cudaError_t launch_fused_tma_batch_storage(const void* src, void* dst, const BatchCase* cases,
                                           int ncases, int total_items, bool walls,
                                           const CUtensorMap* maps, int kind, int ns, int zc,
                                           int* err, int sms, cudaStream_t s);
cudaError_t launch_fused_tma_batch(int storage, const void* src, void* dst,
                                   const BatchCase* cases, int ncases, int total_items,
                                   bool walls, const CUtensorMap* maps, int kind, int ns, int zc,
                                   int* err, int sms, cudaStream_t s);
bool valid_batch_config(const FusedConfig& c);
// Batched SEAM step: maps6 = the device table of the source buffer's six
// seam maps (tile_y 12) per case.
cudaError_t launch_fused_tma_seam_batch(const void* src, void* dst, const BatchCase* cases,
                                        int ncases, int total_items, bool walls,
                                        const CUtensorMap* maps6, int zc, int* err, int sms,
                                        cudaStream_t s);
bool valid_fused_config(const FusedConfig& c, int storage);

}  // namespace lbm
