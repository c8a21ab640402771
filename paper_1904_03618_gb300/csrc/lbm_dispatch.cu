// Storage-type dispatch and launch configuration of the fused step.
#include <algorithm>
#include <functional>
#include <vector>

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
                               int total_items, bool walls, bool bgk,
                               const FusedConfig& cfg, int sms, cudaStream_t s) {
  switch (storage) {
    case 0: return launch_fused_batch_storage<float>(src, dst, cases, ncases, total_items, walls, bgk, cfg, sms, s);
    case 1: return launch_fused_batch_storage<__half>(src, dst, cases, ncases, total_items, walls, bgk, cfg, sms, s);
    case 2: return launch_fused_batch_storage<__nv_bfloat16>(src, dst, cases, ncases, total_items, walls, bgk, cfg, sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_tma(int storage, const void* src, void* dst, const StepArgs& a,
                             const CUtensorMap* maps, int kind, int ns, int zchunk, int* err,
                             cudaStream_t s) {
  switch (storage) {
    case 0: return launch_fused_tma_storage<float>(src, dst, a, maps, kind, ns, zchunk, err, s);
    case 1: return launch_fused_tma_storage<__half>(src, dst, a, maps, kind, ns, zchunk, err, s);
    case 2:
      return launch_fused_tma_storage<__nv_bfloat16>(src, dst, a, maps, kind, ns, zchunk, err,
                                                     s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_tma_batch(int storage, const void* src, void* dst,
                                   const BatchCase* cases, int ncases, int total_items,
                                   bool walls, const CUtensorMap* maps, int kind, int ns, int zc,
                                   int* err, int sms, cudaStream_t s) {
  if (kind != 0 && kind != 2) return cudaErrorInvalidValue;
  switch (storage) {
    case 0:
      return launch_fused_tma_batch_storage<float>(src, dst, cases, ncases, total_items, walls,
                                                   maps, kind, ns, zc, err, sms, s);
    case 1:
      return launch_fused_tma_batch_storage<__half>(src, dst, cases, ncases, total_items, walls,
                                                    maps, kind, ns, zc, err, sms, s);
    case 2:
      return launch_fused_tma_batch_storage<__nv_bfloat16>(src, dst, cases, ncases, total_items,
                                                           walls, maps, kind, ns, zc, err, sms,
                                                           s);
  }
  return cudaErrorInvalidValue;
}

int tma_kind(int tile_y) { return tile_y == 8 ? 0 : (tile_y == 16 ? 1 : (tile_y == 15 ? 2 : -1)); }

static const int kTmaTW[3] = {32, 16, 34}, kTmaBY[3] = {8, 16, 15};

bool tma_config_fits(int storage, int kind, int ns) {
  if (kind < 0 || kind > 2 || ns < 1 || ns > 2) return false;
  switch (storage) {
    case 0: return tma_config_fits_storage<float>(kind, ns);
    case 1: return tma_config_fits_storage<__half>(kind, ns);
    case 2: return tma_config_fits_storage<__nv_bfloat16>(kind, ns);
  }
  return false;
}

// Pair bytes of a storage type (red and blue value of one direction and cell).
static int pair_bytes(int storage) { return storage == 0 ? 8 : 4; }

// The TMA forms are built for the MRT operator only (a BGK context runs the
// shared-memory-hold form).
bool tma_eligible(const StepArgs& a, int storage) {
  return ((long long)a.nx * pair_bytes(storage)) % 16 == 0 && a.nz >= 3 && !a.bgk;
}

// Default TMA configuration.  Tile: the one with more interior cells per
// launched thread for this nx x ny (the 34 x 15 tile wins where nx is a
// multiple of 32, the 32 x 8 tile where it is a multiple of 30).  Stages:
// two for FP32, one for 16-bit storage.  z chunk: each CTA refills two halo
// planes (about half a plane of work), and CTAs run in rounds of (SMs x
// CTAs per SM), so the chunk minimises rounds x (zchunk + 1/2).  On GB300 at
// 128^3 this picks the 34 x 15 tile with 12-plane chunks: 14.4 GLUPS (FP32)
// and 15.7 GLUPS (FP16) against 13.1 and 14.6 for the shared-memory hold.
// 16-bit storage on a lattice where the 32 x 8 tile fits better keeps the
// plain shared-memory hold, which is ahead of its TMA form there.
bool tma_default_config(const StepArgs& a, int storage, int sms, const bool kind_ok[3],
                        FusedConfig* out) {
  if (!tma_eligible(a, storage)) return false;
  double best_eff = -1.0;
  int kind = -1;
  for (int k : {0, 2}) {
    if (!kind_ok[k]) continue;
    const int tw = kTmaTW[k], by = kTmaBY[k];
    const double tiles = (double)((a.nx + tw - 3) / (tw - 2)) * ((a.ny + by - 3) / (by - 2));
    const double eff = (double)a.nx * a.ny / (tiles * tw * by);
    if (eff > best_eff * 1.02) {
      best_eff = eff;
      kind = k;
    }
  }
  if (kind < 0) return false;
  const int ns = storage == 0 ? 2 : 1;
  if (storage != 0 && kind == 0) return false;
  if (!tma_config_fits(storage, kind, ns)) return false;
  const int tw = kTmaTW[kind], by = kTmaBY[kind];
  const long long cols = (long long)((a.nx + tw - 3) / (tw - 2)) * ((a.ny + by - 3) / (by - 2));
  const long long slots = (long long)(sms > 0 ? sms : 152) * (kind == 2 ? 1 : 2);
  int best_zc = 12;
  double best_cost = 1e300;
  for (int zc = 6; zc <= 24; ++zc) {
    const long long ctas = cols * ((a.nz + zc - 1) / zc);
    const double cost = (double)((ctas + slots - 1) / slots) * (zc + 1.5);
    if (cost <= best_cost + 1e-9) {
      best_cost = cost;
      best_zc = zc;
    }
  }
  out->tile_y = by;
  out->hold = ns == 2 ? 7 : 8;
  out->zchunk = best_zc < a.nz ? best_zc : a.nz;
  return true;
}

// Two tensor maps over a population buffer seen as a 4-D array of pairs
// [direction][z][y][x] (x fastest; direction stride = the padded plane),
// for a tile of tw x by threads: FP32 map 0 has tw-pair boxes, map 1
// (tw + 2)-pair boxes; 16-bit storage uses tw + 4 pairs rounded up to a
// multiple of 4 (map 1 = map 0).  Boxes are by rows by one plane by one direction, no swizzle; cells
// beyond the array read as zero.
// One tensor map over a population buffer seen as [direction][z][y][x]
// pairs, with a box of w x h pairs (one plane, one direction).
cudaError_t tensor_map_encoder(EncodeTiledFn* out) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return e != cudaSuccess ? e : cudaErrorNotSupported;
    encode = (EncodeTiledFn)fn;
  }
  *out = encode;
  return cudaSuccess;
}

static cudaError_t encode_box(int storage, const void* base, const StepArgs& a, unsigned w,
                              unsigned h, CUtensorMap* map) {
  EncodeTiledFn encode = nullptr;
  const cudaError_t e = tensor_map_encoder(&encode);
  if (e != cudaSuccess) return e;
  const cuuint64_t E = (cuuint64_t)pair_bytes(storage);
  const cuuint64_t dims[4] = {(cuuint64_t)a.nx, (cuuint64_t)a.ny, (cuuint64_t)a.nz, 19};
  const cuuint64_t strides[3] = {E * a.nx, E * a.nx * a.ny, E * (cuuint64_t)a.plane};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt =
      storage == 0 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  const cuuint32_t box[4] = {(cuuint32_t)w, (cuuint32_t)h, 1, 1};
  const CUresult r = encode(map, dt, 4, const_cast<void*>(base), dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tma_build_maps(int storage, const void* base, const StepArgs& a, int kind,
                           CUtensorMap maps[2]) {
  if (kind < 0 || kind > 2) return cudaErrorInvalidValue;
  if (!tma_eligible(a, storage)) return cudaErrorInvalidValue;
  const int tw = kTmaTW[kind], by = kTmaBY[kind];
  for (int m = 0; m < 2; ++m) {
    const unsigned w = (unsigned)(storage == 0 ? (m == 0 ? tw : tw + 2) : (tw + 4 + 3) / 4 * 4);
    cudaError_t e = encode_box(storage, base, a, w, (unsigned)by, &maps[m]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int seam12_zchunk(const StepArgs& a, int sms) { return list_schedule_zchunk(a, sms, 10); }

int list_schedule_zchunk(const StepArgs& a, int sms, int rows) {
  // One CTA per SM; the hardware hands the CTAs out in launch order (tile
  // columns fastest, then z chunks) to whichever SM falls free, so a step
  // lasts as long as that list schedule.  A CTA of p planes costs p + 3
  // plane-times (two halo planes and a pipeline start).  The full chunks all
  // last the same and fill the SMs round by round; the shorter last chunk's
  // CTAs are placed one by one.  Over 6..32 planes at 128^3..256^3 this
  // picks the measured fastest chunk, where counting whole rounds of
  // equal CTAs picked 16 planes at 128^3 (4.5 % slower than 24).  Chunks
  // up to 48 planes: measured against the 32-plane limit it had before,
  // its picks run 3.4 % faster on the 256 x 256 x 1024 lattice, 0.9-2.2 %
  // faster at 128^3 (16-bit) and 192^3 / 256^3, within 0.1 % at 192^3
  // FP32 and 1.6-3.2 % slower at 160^3; beyond 48 planes the CTAs marching
  // neighbouring columns drift apart and the model, which does not see
  // that, goes wrong (128 planes on the 1024-plane lattice: 12 % slower).
  constexpr double kOverhead = 3.0;
  const long long cols = (long long)((a.nx + 31) / 32) * ((a.ny + rows - 1) / rows);
  const int slots = sms > 0 ? sms : 152;
  std::vector<double> heap((size_t)slots);
  int best_zc = 12;
  double best_span = 1e300;
  for (int zc = 6; zc <= 48; ++zc) {
    const long long full = (long long)(a.nz / zc) * cols;
    const int tail = a.nz % zc;
    const double d = zc + kOverhead;
    const long long rounds = full / slots, extra = full % slots;
    for (int j = 0; j < slots; ++j) heap[(size_t)j] = (double)(rounds + (j < extra)) * d;
    double span = (double)(rounds + (extra > 0)) * d;
    if (tail > 0) {
      auto later = std::greater<double>();
      std::make_heap(heap.begin(), heap.end(), later);
      for (long long c = 0; c < cols; ++c) {
        std::pop_heap(heap.begin(), heap.end(), later);
        heap.back() += tail + kOverhead;
        span = std::max(span, heap.back());
        std::push_heap(heap.begin(), heap.end(), later);
      }
    }
    if (span <= best_span + 1e-9) {
      best_span = span;
      best_zc = zc;
    }
  }
  return best_zc < a.nz ? best_zc : a.nz;
}

bool seam_eligible(const StepArgs& a, int storage) {
  return storage == 0 && tma_eligible(a, storage) && !a.wx && !a.wy && a.nx >= kTmaTW[2] &&
         a.ny >= kTmaBY[2];
}

cudaError_t tma_build_seam_maps(const void* base, const StepArgs& a, int tile_y,
                                CUtensorMap maps[6]) {
  // the strips need periodic x and y; the batched form also builds them for
  // cases narrower than a tile (its lanes fall back to global pulls there)
  if (!tma_eligible(a, 0) || a.wx || a.wy || (tile_y != 15 && tile_y != 12))
    return cudaErrorInvalidValue;
  const unsigned tw = (unsigned)kTmaTW[2], by = (unsigned)tile_y;
  const unsigned shape[6][2] = {{tw, by}, {tw + 2, by}, {2, by}, {tw, 2}, {tw + 2, 2}, {2, 2}};
  for (int m = 0; m < 6; ++m) {
    cudaError_t e = encode_box(0, base, a, shape[m][0], shape[m][1], &maps[m]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool seam16_eligible(const StepArgs& a, int storage) {
  return storage != 0 && tma_eligible(a, storage) && !a.wx && !a.wy && a.nx >= kTmaTW[2] &&
         a.ny >= kTmaBY[2];
}

cudaError_t tma_build_seam16_maps(int storage, const void* base, const StepArgs& a, int tile_y,
                                  CUtensorMap maps[4]) {
  if (!seam16_eligible(a, storage) || (tile_y != 15 && tile_y != 12))
    return cudaErrorInvalidValue;
  const unsigned w = (unsigned)(kTmaTW[2] + 4 + 3) / 4 * 4, by = (unsigned)tile_y;
  const unsigned shape[4][2] = {{w, by}, {4, by}, {w, 2}, {4, 2}};
  for (int m = 0; m < 4; ++m) {
    cudaError_t e = encode_box(storage, base, a, shape[m][0], shape[m][1], &maps[m]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_fused_tma_seam16(int storage, const void* src, void* dst, const StepArgs& a,
                                    int tile_y, const CUtensorMap* maps4, int zchunk, int* err,
                                    cudaStream_t s, MonAcc* mon) {
  if (storage == 1)
    return launch_fused_tma_seam16_storage<__half>(src, dst, a, tile_y, maps4, zchunk, err, s,
                                                   mon);
  if (storage == 2)
    return launch_fused_tma_seam16_storage<__nv_bfloat16>(src, dst, a, tile_y, maps4, zchunk,
                                                          err, s, mon);
  return cudaErrorInvalidValue;
}

// Batched kernel variants: (tile_y, hold) = (8, 2), (8, 0), (16, 1), and
// the TMA forms (8 or 15, 7 or 8) where the context built tensor maps.
bool valid_batch_config(const FusedConfig& c) {
  const bool shape = (c.tile_y == 8 && (c.hold == 2 || c.hold == 0)) ||
                     (c.tile_y == 16 && c.hold == 1) ||
                     ((c.tile_y == 8 || c.tile_y == 15) && (c.hold == 7 || c.hold == 8)) ||
                     (c.tile_y == 12 && c.hold == 7);
  return shape && c.zchunk > 0;
}

bool batch_seam_eligible(const StepArgs& a, int storage) {
  return storage == 0 && tma_eligible(a, storage) && !a.wx && !a.wy && !a.bgk;
}

bool valid_fused_config(const FusedConfig& c, int storage) {
  if (c.tile_y == 15) return (c.hold == 7 || c.hold == 8) && c.zchunk > 0;
  if (c.tile_y != 8 && c.tile_y != 16) return false;
  if (c.hold < 0 || c.hold > 8) return false;
  if ((c.hold == 2 || c.hold == 3 || c.hold == 5 || c.hold == 6) && c.tile_y != 8) return false;
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
