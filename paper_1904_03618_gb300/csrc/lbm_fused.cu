// Fused one-kernel step for sm_103a.
//
// A CTA of 32 x BY threads owns a column tile of 30 x (BY - 2) interior
// cells plus a one-cell ring and marches along z over a chunk of planes.
// Each iteration:
//   1. every thread pulls its column's 38 populations of plane z + 1 and
//      writes (rho^N, Qbar_x, Qbar_y, Qbar_z) of that cell into a 4-slot
//      shared-memory window (plane index mod 4);
//   2. one barrier;
//   3. interior threads pull plane z again (the lines were just brought into
//      L1 by step 1 one iteration earlier), form the Eq. 49 gradients from
//      the window (planes z - 1, z, z + 1), collide, recolour and store.
// The ring costs extra L1/L2 reads, not extra HBM traffic: neighbouring CTAs
// read the same lines around the same time.  Four window slots make one
// barrier per plane sufficient: a slot is rewritten four iterations after it
// was filled, when every reader has passed two more barriers.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kTileW = 32;  // threads along x per CTA (one warp)

template <typename T>
__device__ __forceinline__ void pull_sums(const T* __restrict__ src,
                                          const StepArgs& a, int x, int y,
                                          int z, float& rR, float& rB,
                                          float& jx, float& jy, float& jz) {
  float fR[19], fB[19];
  pull_cell<T>(src, a, x, y, z, fR, fB);
  rR = 0.f;
  rB = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    rR += fR[i];
    rB += fB[i];
  }
  float f[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = fR[i] + fB[i];
  jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) +
       (f[13] - f[14]);
  jy = (f[3] - f[4]) + (f[7] - f[8]) + (f[10] - f[9]) + (f[15] - f[16]) +
       (f[17] - f[18]);
  jz = (f[5] - f[6]) + (f[11] - f[12]) + (f[14] - f[13]) + (f[15] - f[16]) +
       (f[18] - f[17]);
}

// Phase field and correction flux of one cell (same arithmetic as macro_of,
// phase_field and qbar_scale).
__device__ __forceinline__ float4 window_entry(const StepArgs& a, float rR,
                                               float rB, float jx, float jy,
                                               float jz) {
  const float rho = rR + rB;
  const float inv = 1.0f / rho;
  const float ux = (jx + 0.5f * (a.fx + rho * a.gx)) * inv;
  const float uy = (jy + 0.5f * (a.fy + rho * a.gy)) * inv;
  const float uz = (jz + 0.5f * (a.fz + rho * a.gz)) * inv;
  const float q = qbar_scale(a, rR, rB);
  return make_float4(phase_field(a, rR, rB), ux * q, uy * q, uz * q);
}

template <typename T, int BY>
__global__ void __launch_bounds__(kTileW* BY)
    k_fused(const T* __restrict__ src, T* __restrict__ dst, StepArgs a,
            int zchunk) {
  __shared__ float4 win[4][BY][kTileW];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * (kTileW - 2), y0 = blockIdx.y * (BY - 2);
  const int zb = blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, a.nz);
  if (zb >= ze) return;

  // Column handled by this thread (ring included), wrapped on periodic axes.
  int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
  bool col_ok = true;
  if (a.wx) col_ok = col_ok && gx >= 0 && gx < a.nx;
  else gx = ((gx % a.nx) + a.nx) % a.nx;
  if (a.wy) col_ok = col_ok && gy >= 0 && gy < a.ny;
  else gy = ((gy % a.ny) + a.ny) % a.ny;

  const int cx = x0 - 1 + tx, cy = y0 - 1 + ty;  // unwrapped
  const bool interior = tx >= 1 && tx <= kTileW - 2 && ty >= 1 &&
                        ty <= BY - 2 && cx < a.nx && cy < a.ny;
  // Eq. 49 neighbours beyond a wall take the centre value.
  const bool xlo = a.wx && cx == 0, xhi = a.wx && cx == a.nx - 1;
  const bool ylo = a.wy && cy == 0, yhi = a.wy && cy == a.ny - 1;

  auto fill = [&](int zl) {
    int zs = zl;
    bool ok = col_ok;
    if (a.wz) ok = ok && zl >= 0 && zl < a.nz;
    else zs = ((zl % a.nz) + a.nz) % a.nz;
    if (ok) {
      float rR, rB, jx, jy, jz;
      pull_sums<T>(src, a, gx, gy, zs, rR, rB, jx, jy, jz);
      win[zl & 3][ty][tx] = window_entry(a, rR, rB, jx, jy, jz);
    }
  };

  fill(zb - 1);
  for (int z = zb; z < ze; ++z) {
    if (z == zb) fill(z);
    fill(z + 1);
    __syncthreads();
    if (interior) {
      const bool zlo = a.wz && z == 0, zhi = a.wz && z == a.nz - 1;
      const float4 ctr = win[z & 3][ty][tx];
      float Gx = 0.f, Gy = 0.f, Gz = 0.f, Qx = 0.f, Qy = 0.f, Qz = 0.f;
#pragma unroll
      for (int i = 1; i < 19; ++i) {
        const int dx = ex(i), dy = ey(i), dz = ez(i);
        const bool beyond = (dx > 0 && xhi) || (dx < 0 && xlo) ||
                            (dy > 0 && yhi) || (dy < 0 && ylo) ||
                            (dz > 0 && zhi) || (dz < 0 && zlo);
        const float4 v = beyond ? ctr : win[(z + dz) & 3][ty + dy][tx + dx];
        const float w = (i <= 6) ? (1.0f / 6.0f) : (1.0f / 12.0f);
        if (dx) {
          Gx += (dx * w) * v.x;
          Qx += (dx * w) * v.y;
        }
        if (dy) {
          Gy += (dy * w) * v.x;
          Qy += (dy * w) * v.z;
        }
        if (dz) {
          Gz += (dz * w) * v.x;
          Qz += (dz * w) * v.w;
        }
      }
      float fR[19], fB[19];
      pull_cell<T>(src, a, cx, cy, z, fR, fB);
      Macro m = macro_of(a, fR, fB);
      collide_cell(a, fR, fB, m, ctr.x, Gx, Gy, Gz, Qx, Qy, Qz);
      store_cell<T>(dst, a, cell_of(a, cx, cy, z), fR, fB);
    }
  }
}

template <typename T, int BY>
static cudaError_t launch_fused_by(const void* src, void* dst,
                                   const StepArgs& a, const FusedConfig& cfg,
                                   cudaStream_t s) {
  dim3 blk(kTileW, BY);
  int zc = cfg.zchunk > 0 ? cfg.zchunk : a.nz;
  dim3 grd((a.nx + kTileW - 3) / (kTileW - 2), (a.ny + BY - 3) / (BY - 2),
           (a.nz + zc - 1) / zc);
  k_fused<T, BY><<<grd, blk, 0, s>>>((const T*)src, (T*)dst, a, zc);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_fused_t(const void* src, void* dst,
                                  const StepArgs& a, const FusedConfig& cfg,
                                  cudaStream_t s) {
  switch (cfg.tile_y) {
    case 8: return launch_fused_by<T, 8>(src, dst, a, cfg, s);
    case 16: return launch_fused_by<T, 16>(src, dst, a, cfg, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused(int storage, const void* src, void* dst,
                         const StepArgs& a, const FusedConfig& cfg,
                         cudaStream_t s) {
  switch (storage) {
    case 0: return launch_fused_t<float>(src, dst, a, cfg, s);
    case 1: return launch_fused_t<__half>(src, dst, a, cfg, s);
    case 2: return launch_fused_t<__nv_bfloat16>(src, dst, a, cfg, s);
  }
  return cudaErrorInvalidValue;
}

// Chunk length along z so that the grid fills the 152 SMs with whole waves
// of two resident CTAs each, without making chunks shorter than 8 planes.
FusedConfig default_fused_config(const StepArgs& a, int storage) {
  (void)storage;
  FusedConfig c;
  c.tile_x = kTileW - 2;
  c.tile_y = 8;
  long long cols = (long long)((a.nx + kTileW - 3) / (kTileW - 2)) *
                   ((a.ny + c.tile_y - 3) / (c.tile_y - 2));
  const long long slots = 152LL * 2;
  long long chunks = (slots + cols - 1) / cols;
  if (chunks < 1) chunks = 1;
  int zc = (int)((a.nz + chunks - 1) / chunks);
  if (zc < 8) zc = 8;
  if (zc > a.nz) zc = a.nz;
  c.zchunk = zc;
  return c;
}

}  // namespace lbm
