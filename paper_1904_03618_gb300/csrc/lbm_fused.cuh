// Fused one-kernel step for sm_103a (included once per storage type).
//
// A CTA of 32 x BY threads owns a column tile of 30 x (BY - 2) interior
// cells plus a one-cell ring and marches along z over a chunk of planes.
// Each iteration:
//   1. every thread pulls its column's populations of plane z + 1 (19
//      red/blue pairs) and writes (rho^N, Qbar_x, Qbar_y, Qbar_z) of that
//      cell into a 4-slot shared-memory window (plane index mod 4);
//   2. one barrier;
//   3. interior threads form the Eq. 49 gradients from the window (planes
//      z - 1, z, z + 1), collide, recolour and store plane z.
// After the pull a cell needs only its total populations f_i = f_i^R +
// f_i^B, rho_R, rho_B and u (24 values): the collision acts on the total
// population and the recolouring needs only the colour densities.  HOLD
// selects where those wait between the pull and the collision: 0 = not
// kept (pulled again from L1/L2), 1 = registers, 2 = shared memory.  The
// ring costs extra L2 reads, not extra HBM traffic: neighbouring CTAs read
// the same lines at about the same time.  Four window slots make one barrier
// per plane sufficient: a slot is rewritten four iterations after it was
// filled, when every reader has passed two more barriers.
//
// k_fused_async is the pipelined form: the pulls of plane z + 2 are issued
// as cp.async copies into a thread-private shared slot before plane z
// collides, so they are in flight during the collision.
//
// Addressing: one base pointer per buffer and 32-bit pair offsets
// (direction * plane + cell); wrapped x / y / z neighbour offsets are
// computed once per column and per plane, so one pulled pair costs an
// integer add, an address multiply-add and one load.
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kTileW = 32;  // threads along x per CTA (one warp)

template <typename T, int I>
__device__ __forceinline__ void add_offsets(const StepArgs& a, float2& v) {
  if (Store<T>::kDeviation) {
    v.x += dev_offset<I>(a, 0);
    v.y += dev_offset<I>(a, 1);
  }
}

// Pull of the 19 pairs of one column / plane, reduced on the fly to
// (f_i = fR_i + fB_i, rho_R, rho_B).  The colour sums run as one paired
// FP32 add per direction (the red and blue values arrive as a pair; each
// component rounds as its scalar add would).
template <typename T, bool WALLS, int I>
struct PullReduce {
  __device__ __forceinline__ static void run(const typename Store<T>::Pair* src,
                                             unsigned plane, const StepArgs& a,
                                             const ColOff& c, const PlaneOff& p,
                                             float* f, float2& rho) {
    const unsigned q = pull_index<WALLS, I>(plane, c, p);
    float2 v = make_float2(0.f, 0.f);
    if (index_ok(a, q, 19ull * plane)) v = Store<T>::to_float2(__ldg(src + q));
    add_offsets<T, I>(a, v);
    rho = __fadd2_rn(rho, v);
    f[I] = v.x + v.y;
    PullReduce<T, WALLS, I + 1>::run(src, plane, a, c, p, f, rho);
  }
};
template <typename T, bool WALLS>
struct PullReduce<T, WALLS, 19> {
  __device__ __forceinline__ static void run(const typename Store<T>::Pair*,
                                             unsigned, const StepArgs&,
                                             const ColOff&, const PlaneOff&,
                                             float*, float2&) {}
};
template <typename T, bool WALLS>
__device__ __forceinline__ void pull_reduce(const typename Store<T>::Pair* src, unsigned plane,
                                            const StepArgs& a, const ColOff& c,
                                            const PlaneOff& p, float* f, float& rR,
                                            float& rB) {
  float2 rho = make_float2(rR, rB);
  PullReduce<T, WALLS, 0>::run(src, plane, a, c, p, f, rho);
  rR = rho.x;
  rB = rho.y;
}

// cp.async of one pair (8 bytes for FP32, 4 bytes for FP16/BF16), global ->
// shared, L1-allocating form.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem),
               "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename T, bool WALLS, int I>
struct PullAsync {
  __device__ __forceinline__ static void run(const typename Store<T>::Pair* src,
                                             unsigned plane, const ColOff& c,
                                             const PlaneOff& p,
                                             typename Store<T>::Pair* raw,
                                             int stride, const StepArgs& a) {
    const unsigned q = pull_index<WALLS, I>(plane, c, p);
    if (index_ok(a, q, 19ull * plane))
      cp_async<sizeof(typename Store<T>::Pair)>(raw + I * stride, src + q);
    PullAsync<T, WALLS, I + 1>::run(src, plane, c, p, raw, stride, a);
  }
};
template <typename T, bool WALLS>
struct PullAsync<T, WALLS, 19> {
  __device__ __forceinline__ static void run(const typename Store<T>::Pair*,
                                             unsigned, const ColOff&,
                                             const PlaneOff&,
                                             typename Store<T>::Pair*, int,
                                             const StepArgs&) {}
};

// Stores the recoloured populations of Eq. 10-11 of one cell, one pair of
// opposite directions at a time (their recolouring terms differ in sign).
template <typename T, int I>
struct StoreRecoloured {
  __device__ __forceinline__ static void run(T* dst, unsigned plane,
                                             const StepArgs& a, unsigned c,
                                             const Recolour& rc,
                                             const float* fs) {
    const float sg = recolour_seg<I>(rc);
    float r1 = rc.wr * fs[I] + sg, b1 = rc.wb * fs[I] - sg;
    float r2 = rc.wr * fs[I + 1] - sg, b2 = rc.wb * fs[I + 1] + sg;
    if (Store<T>::kDeviation) {
      r1 -= dev_offset<I>(a, 0);
      b1 -= dev_offset<I>(a, 1);
      r2 -= dev_offset<I + 1>(a, 0);
      b2 -= dev_offset<I + 1>(a, 1);
    }
    Store<T>::store2(dst + 2 * (size_t)(I * plane + c), r1, b1);
    Store<T>::store2(dst + 2 * (size_t)((I + 1) * plane + c), r2, b2);
    StoreRecoloured<T, I + 2>::run(dst, plane, a, c, rc, fs);
  }
};
template <typename T>
struct StoreRecoloured<T, 19> {
  __device__ __forceinline__ static void run(T*, unsigned, const StepArgs&,
                                             unsigned, const Recolour&,
                                             const float*) {}
};
template <typename T>
__device__ __forceinline__ void store_recoloured(T* dst, unsigned plane,
                                                 const StepArgs& a, unsigned c,
                                                 const Recolour& rc,
                                                 const float* fs) {
  if (!index_ok(a, c, plane)) return;
  float r0 = rc.wr * fs[0], b0 = rc.wb * fs[0];
  if (Store<T>::kDeviation) {
    r0 -= dev_offset<0>(a, 0);
    b0 -= dev_offset<0>(a, 1);
  }
  Store<T>::store2(dst + 2 * (size_t)c, r0, b0);
  StoreRecoloured<T, 1>::run(dst, plane, a, c, rc, fs);
}

// Eq. 49 gradients of rho^N and the correction fluxes at an interior cell
// from the shared window, as weighted differences of opposite neighbours so
// that a uniform field gives an exactly zero gradient.  A neighbour beyond a
// wall takes the centre value.
template <int BY, int TW = kTileW>
__device__ __forceinline__ void window_gradients(
    const float4 (*win)[BY][TW], int z, int ty, int tx, bool xlo, bool xhi,
    bool ylo, bool yhi, bool zlo, bool zhi, float4& ctr, float& Gx, float& Gy,
    float& Gz, float& Qx, float& Qy, float& Qz) {
  ctr = win[z & 3][ty][tx];
  Gx = Gy = Gz = Qx = Qy = Qz = 0.f;
#pragma unroll
  for (int i = 1; i < 19; i += 2) {
    const int dx = ex(i), dy = ey(i), dz = ez(i);
    const bool bp = (dx > 0 && xhi) || (dx < 0 && xlo) || (dy > 0 && yhi) ||
                    (dy < 0 && ylo) || (dz > 0 && zhi) || (dz < 0 && zlo);
    const bool bm = (dx < 0 && xhi) || (dx > 0 && xlo) || (dy < 0 && yhi) ||
                    (dy > 0 && ylo) || (dz < 0 && zhi) || (dz > 0 && zlo);
    const float4 vp = bp ? ctr : win[(z + dz) & 3][ty + dy][tx + dx];
    const float4 vm = bm ? ctr : win[(z - dz) & 3][ty - dy][tx - dx];
    const float w = (i <= 6) ? (1.0f / 6.0f) : (1.0f / 12.0f);
    if (dx) {
      Gx += (dx * w) * (vp.x - vm.x);
      Qx += (dx * w) * (vp.y - vm.y);
    }
    if (dy) {
      Gy += (dy * w) * (vp.x - vm.x);
      Qy += (dy * w) * (vp.z - vm.z);
    }
    if (dz) {
      Gz += (dz * w) * (vp.x - vm.x);
      Qz += (dz * w) * (vp.w - vm.w);
    }
  }
}

// Per-thread geometry shared by the kernels: a CTA tile of TW x BY columns
// (interior (TW - 2) x (BY - 2) plus the one-cell ring).
template <bool WALLS, int BY, int TW = kTileW>
struct Geometry {
  ColOff co;
  bool col_ok, interior, xlo, xhi, ylo, yhi;
  int cx, cy;
  unsigned plane_cells;
  // tile (bx, by) of the lattice's 30 x (BY - 2) interior tiles
  __device__ __forceinline__ Geometry(const StepArgs& a, int tx, int ty, int bx,
                                      int by) {
    const int x0 = bx * (TW - 2), y0 = by * (BY - 2);
    cx = x0 - 1 + tx;
    cy = y0 - 1 + ty;  // unwrapped
    col_ok = true;
    if (WALLS) {
      if (a.wx) col_ok = col_ok && cx >= 0 && cx < a.nx;
      if (a.wy) col_ok = col_ok && cy >= 0 && cy < a.ny;
    }
    const int gx = wrapn(cx, a.nx), gy = wrapn(cy, a.ny);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      co.xo[d] = (unsigned)wrapn(gx + d - 1, a.nx);
      co.yo[d] = (unsigned)wrapn(gy + d - 1, a.ny) * (unsigned)a.nx;
    }
    co.bxl = WALLS && a.wx && gx == 0;
    co.bxh = WALLS && a.wx && gx == a.nx - 1;
    co.byl = WALLS && a.wy && gy == 0;
    co.byh = WALLS && a.wy && gy == a.ny - 1;
    plane_cells = (unsigned)a.nx * (unsigned)a.ny;
    interior = tx >= 1 && tx <= TW - 2 && ty >= 1 && ty <= BY - 2 &&
               cx < a.nx && cy < a.ny;
    xlo = WALLS && a.wx && cx == 0;
    xhi = WALLS && a.wx && cx == a.nx - 1;
    ylo = WALLS && a.wy && cy == 0;
    yhi = WALLS && a.wy && cy == a.ny - 1;
  }
  // zs in [0, nz): the neighbours zs +- 1 wrap by one period at most
  __device__ __forceinline__ PlaneOff plane(const StepArgs& a, int zs) const {
    PlaneOff p;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      p.zo[d] = (unsigned)wrap1(zs + d - 1, a.nz) * plane_cells;
    p.bzl = WALLS && a.wz && zs == 0;
    p.bzh = WALLS && a.wz && zs == a.nz - 1;
    return p;
  }
  __device__ __forceinline__ bool plane_ok(const StepArgs& a, int zl) const {
    return col_ok && (!(WALLS && a.wz) || (zl >= 0 && zl < a.nz));
  }
};

template <int BY, int HOLD>
struct FusedSmem {
  float4 win[4][BY][kTileW];
};
template <int BY>
struct FusedSmem<BY, 2> {
  float4 win[4][BY][kTileW];
  float hold[24][BY - 2][kTileW - 2];  // next plane: f_i, rho_R, rho_B, u
};

// MINB: CTAs per SM the register allocation must allow (launch bounds).
// One work item of the fused step: tile (bx, by), planes [zb, ze).
template <typename T, int BY, bool WALLS, int HOLD, bool BGK = false>
__device__ __forceinline__ void fused_work(const T* __restrict__ src,
                                           T* __restrict__ dst,
                                           const StepArgs& a, int bx, int by,
                                           int zb, int ze,
                                           FusedSmem<BY, HOLD>& sm) {
  using Pair = typename Store<T>::Pair;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const Geometry<WALLS, BY> g(a, tx, ty, bx, by);
  const unsigned plane = (unsigned)a.plane;
  const Pair* srcp = reinterpret_cast<const Pair*>(src);

  // Pulls plane zl (in [zb - 1, ze]) of this column, fills its window slot
  // and returns the reduced state: f (19), then rho_R, rho_B, u (5).
  auto fill = [&](int zl, float* f, float* hu) {
    if (!g.plane_ok(a, zl)) return;
    float rR = 0.f, rB = 0.f;
    pull_reduce<T, WALLS>(srcp, plane, a, g.co, g.plane(a, wrap1(zl, a.nz)),
                                 f, rR, rB);
    const Macro m = macro_total(a, f, rR, rB);
    hu[0] = rR;
    hu[1] = rB;
    hu[2] = m.ux;
    hu[3] = m.uy;
    hu[4] = m.uz;
    sm.win[zl & 3][ty][tx] = stencil_entry(a, m);
  };

  float cf[19], ch[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  {
    float tf[19], th[5];
    fill(zb - 1, tf, th);
    fill(zb, cf, ch);
  }
  for (int z = zb; z < ze; ++z) {
    float nf[19], nh[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    fill(z + 1, nf, nh);
    if constexpr (HOLD == 2) {
      // private slot of this thread (a spill to shared memory): no barrier
      if (g.interior) {
#pragma unroll
        for (int i = 0; i < 19; ++i) sm.hold[i][ty - 1][tx - 1] = nf[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) sm.hold[19 + i][ty - 1][tx - 1] = nh[i];
      }
    }
    __syncthreads();
    if (g.interior) {
      const bool zlo = WALLS && a.wz && z == 0, zhi = WALLS && a.wz && z == a.nz - 1;
      float4 ctr;
      float Gx, Gy, Gz, Qx, Qy, Qz;
      window_gradients<BY>(sm.win, z, ty, tx, g.xlo, g.xhi, g.ylo, g.yhi, zlo, zhi,
                           ctr, Gx, Gy, Gz, Qx, Qy, Qz);
      if (WALLS && a.wetting)
        wetting_rule(a, g.xlo, g.xhi, g.ylo, g.yhi, zlo, zhi, Gx, Gy, Gz);
      Macro m;
      if constexpr (HOLD == 0) {
        float rR = 0.f, rB = 0.f;
        pull_reduce<T, WALLS>(srcp, plane, a, g.co, g.plane(a, z), cf, rR, rB);
        m = macro_total(a, cf, rR, rB);
      } else {
        m = macro_held(a, ch[0], ch[1], ch[2], ch[3], ch[4]);
      }
      const Recolour rc = collide_total<BGK>(a, cf, m, ctr.x, Gx, Gy, Gz, Qx, Qy, Qz);
      store_recoloured<T>(dst, plane, a,
                          (unsigned)z * g.plane_cells + g.co.yo[1] + g.co.xo[1], rc, cf);
    }
    if constexpr (HOLD == 1) {
#pragma unroll
      for (int i = 0; i < 19; ++i) cf[i] = nf[i];
#pragma unroll
      for (int i = 0; i < 5; ++i) ch[i] = nh[i];
    } else if constexpr (HOLD == 2) {
      if (g.interior) {
#pragma unroll
        for (int i = 0; i < 19; ++i) cf[i] = sm.hold[i][ty - 1][tx - 1];
#pragma unroll
        for (int i = 0; i < 5; ++i) ch[i] = sm.hold[19 + i][ty - 1][tx - 1];
      }
    }
  }
}

template <typename T, int BY, bool WALLS, int HOLD, int MINB, bool BGK = false>
__global__ void __launch_bounds__(kTileW* BY, MINB)
    k_fused(const T* __restrict__ src, T* __restrict__ dst,
            const __grid_constant__ StepArgs a, int zchunk) {
  __shared__ FusedSmem<BY, HOLD> sm;
  const int zb = blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, a.nz);
  if (zb >= ze) return;
  fused_work<T, BY, WALLS, HOLD, BGK>(src, dst, a, blockIdx.x, blockIdx.y, zb, ze, sm);
}

// Batched step: many independent lattices ("cases") in one launch.  The
// CTAs are persistent: CTA b takes work items b, b + gridDim.x, ...; the
// items of a case are numbered (chunk, tile y, tile x) with tile x fastest,
// so concurrently running CTAs work on neighbouring tiles of one chunk and
// their ring re-reads hit L2.  The case's parameters are copied into shared
// memory once per item.
template <typename T, int BY, bool WALLS, int HOLD, int MINB, bool BGK = false>
__global__ void __launch_bounds__(kTileW* BY, MINB)
    k_fused_batch(const BatchCase* __restrict__ cases, int ncases,
                  int total_items, const T* __restrict__ src_base,
                  T* __restrict__ dst_base, int zchunk) {
  __shared__ FusedSmem<BY, HOLD> sm;
  __shared__ StepArgs sa;
  __shared__ int s_case, s_item;
  for (int w = blockIdx.x; w < total_items; w += gridDim.x) {
    __syncthreads();  // the previous item is done with sm and sa
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      int lo = 0, hi = ncases - 1;  // last case with item_start <= w
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cases[mid].item_start <= w) lo = mid;
        else hi = mid - 1;
      }
      s_case = lo;
      s_item = w - cases[lo].item_start;
      sa = cases[lo].args;
    }
    __syncthreads();
    const BatchCase& bc = cases[s_case];
    const int tiles_x = bc.tiles_x, tiles_y = bc.tiles_y;
    const int item = s_item;
    const int bx = item % tiles_x, rest = item / tiles_x;
    const int by = rest % tiles_y, chunk = rest / tiles_y;
    const int zb = chunk * zchunk;
    const int ze = min(zb + zchunk, sa.nz);
    const size_t off = 2 * (size_t)bc.pair_base;
    fused_work<T, BY, WALLS, HOLD, BGK>(src_base + off, dst_base + off, sa, bx, by, zb, ze,
                                        sm);
  }
}

// Two columns per thread: a CTA of 32 x 8 threads covers a 32 x 16 column
// tile (interior 30 x 14), thread row ty handling tile rows ty and ty + 8.
// The ring overhead of the moment pass falls from 256/180 to 512/420 and
// each barrier is amortised over two collisions per thread.  The reduced
// state of the next plane waits in shared memory (thread-private slots).
constexpr int kRows2 = 16;
struct Fused2Smem {
  float4 win[4][kRows2][kTileW];
  float hold[2][24][kRows2 - 2][kTileW - 2];  // by plane parity
};

template <typename T, bool WALLS>
__global__ void __launch_bounds__(kTileW * 8, 2)
    k_fused2(const T* __restrict__ src, T* __restrict__ dst,
             const __grid_constant__ StepArgs a, int zchunk) {
  using Pair = typename Store<T>::Pair;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Fused2Smem& sm = *reinterpret_cast<Fused2Smem*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int zb = blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, a.nz);
  if (zb >= ze) return;
  const Geometry<WALLS, kRows2> g0(a, tx, ty, blockIdx.x, blockIdx.y),
      g1(a, tx, ty + 8, blockIdx.x, blockIdx.y);
  const unsigned plane = (unsigned)a.plane;
  const Pair* srcp = reinterpret_cast<const Pair*>(src);

  // Pulls plane zl of the column at tile row `row`: window slot, and for an
  // interior cell its reduced state in the hold slot of the plane's parity
  // (private to this thread).
  auto fill = [&](const Geometry<WALLS, kRows2>& g, int row, int zl) {
    if (!g.plane_ok(a, zl)) return;
    float f[19], rR = 0.f, rB = 0.f;
    pull_reduce<T, WALLS>(srcp, plane, a, g.co, g.plane(a, wrap1(zl, a.nz)), f,
                                 rR, rB);
    const Macro m = macro_total(a, f, rR, rB);
    sm.win[zl & 3][row][tx] = stencil_entry(a, m);
    if (g.interior) {
      float(*h)[kRows2 - 2][kTileW - 2] = sm.hold[zl & 1];
#pragma unroll
      for (int i = 0; i < 19; ++i) h[i][row - 1][tx - 1] = f[i];
      h[19][row - 1][tx - 1] = rR;
      h[20][row - 1][tx - 1] = rB;
      h[21][row - 1][tx - 1] = m.ux;
      h[22][row - 1][tx - 1] = m.uy;
      h[23][row - 1][tx - 1] = m.uz;
    }
  };
  // collision of the interior cell at tile row `row`, plane z
  auto collide = [&](const Geometry<WALLS, kRows2>& g, int row, int z) {
    const bool zlo = WALLS && a.wz && z == 0, zhi = WALLS && a.wz && z == a.nz - 1;
    float4 ctr;
    float Gx, Gy, Gz, Qx, Qy, Qz;
    window_gradients<kRows2>(sm.win, z, row, tx, g.xlo, g.xhi, g.ylo, g.yhi, zlo, zhi,
                             ctr, Gx, Gy, Gz, Qx, Qy, Qz);
    if (WALLS && a.wetting)
      wetting_rule(a, g.xlo, g.xhi, g.ylo, g.yhi, zlo, zhi, Gx, Gy, Gz);
    const float(*h)[kRows2 - 2][kTileW - 2] = sm.hold[z & 1];
    float f[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = h[i][row - 1][tx - 1];
    const Macro m = macro_held(a, h[19][row - 1][tx - 1], h[20][row - 1][tx - 1],
                               h[21][row - 1][tx - 1], h[22][row - 1][tx - 1],
                               h[23][row - 1][tx - 1]);
    const Recolour rc = collide_total<false>(a, f, m, ctr.x, Gx, Gy, Gz, Qx, Qy, Qz);
    store_recoloured<T>(dst, plane, a, (unsigned)z * g.plane_cells + g.co.yo[1] + g.co.xo[1],
                        rc, f);
  };

  fill(g0, ty, zb - 1);
  fill(g1, ty + 8, zb - 1);
  fill(g0, ty, zb);
  fill(g1, ty + 8, zb);
  for (int z = zb; z < ze; ++z) {
    // plane z + 1 fills the other hold parity; plane z's stays readable
    fill(g0, ty, z + 1);
    fill(g1, ty + 8, z + 1);
    __syncthreads();
    if (g0.interior) collide(g0, ty, z);
    if (g1.interior) collide(g1, ty + 8, z);
  }
}

// Pipelined variant (32 x 8 CTA).  Iteration z:
//   A. issue cp.async pulls of plane z + 2 into this thread's raw slot;
//   B. interior threads collide plane z from its held reduced state;
//   C. wait for the copies, reduce plane z + 2 to (f, rho_R, rho_B, u),
//      write its window slot and (interior) its hold slot;
//   D. one barrier.
// The copies of step A are in flight during the collision of step B; the
// raw and hold slots are private to each thread.  Window slot of plane p:
// p mod 4, written in step C of iteration p - 2 and read in iterations
// p - 1 .. p + 1; its next writer runs in iteration p + 2, after the
// barrier that follows the last reader.
constexpr int kAsyncBY = 8;
template <typename T>
struct AsyncSmem {
  float4 win[4][kAsyncBY][kTileW];
  typename Store<T>::Pair raw[19][kAsyncBY][kTileW];
  float hold[2][24][kAsyncBY - 2][kTileW - 2];
};

template <typename T, bool WALLS>
__global__ void __launch_bounds__(kTileW* kAsyncBY, 2)
    k_fused_async(const T* __restrict__ src, T* __restrict__ dst,
                  const __grid_constant__ StepArgs a, int zchunk) {
  constexpr int BY = kAsyncBY;
  using Pair = typename Store<T>::Pair;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AsyncSmem<T>& sm = *reinterpret_cast<AsyncSmem<T>*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int zb = blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, a.nz);
  if (zb >= ze) return;
  const Geometry<WALLS, BY> g(a, tx, ty, blockIdx.x, blockIdx.y);
  const unsigned plane = (unsigned)a.plane;
  const Pair* srcp = reinterpret_cast<const Pair*>(src);
  Pair* raw = &sm.raw[0][ty][tx];
  constexpr int kRawStride = kAsyncBY * kTileW;
  constexpr int hs = (kAsyncBY - 2) * (kTileW - 2);

  auto issue = [&](int zl) -> bool {
    const bool ok = g.plane_ok(a, zl);
    if (ok)
      PullAsync<T, WALLS, 0>::run(srcp, plane, g.co, g.plane(a, wrap1(zl, a.nz)), raw,
                                  kRawStride, a);
    cp_async_commit();
    return ok;
  };
  auto consume = [&](int zl, bool ok) {
    cp_async_wait_all();
    if (!ok) return;
    float f[19], rR = 0.f, rB = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      float2 v = Store<T>::to_float2(raw[i * kRawStride]);
      if (Store<T>::kDeviation) {
        const int s = shell(i);
        v.x += s == 0 ? a.offR0 : (s == 1 ? a.offR1 : a.offR2);
        v.y += s == 0 ? a.offB0 : (s == 1 ? a.offB1 : a.offB2);
      }
      rR += v.x;
      rB += v.y;
      f[i] = v.x + v.y;
    }
    const Macro m = macro_total(a, f, rR, rB);
    sm.win[zl & 3][ty][tx] = stencil_entry(a, m);
    if (g.interior) {
      float* h = &sm.hold[zl & 1][0][ty - 1][tx - 1];
#pragma unroll
      for (int i = 0; i < 19; ++i) h[i * hs] = f[i];
      h[19 * hs] = rR;
      h[20 * hs] = rB;
      h[21 * hs] = m.ux;
      h[22 * hs] = m.uy;
      h[23 * hs] = m.uz;
    }
  };

  for (int zl = zb - 1; zl <= zb + 1; ++zl) consume(zl, issue(zl));
  __syncthreads();
  for (int z = zb; z < ze; ++z) {
    const bool need2 = z + 1 < ze;  // plane z + 2 borders plane z + 1
    const bool ok2 = need2 ? issue(z + 2) : false;
    if (g.interior) {
      const bool zlo = WALLS && a.wz && z == 0, zhi = WALLS && a.wz && z == a.nz - 1;
      float4 ctr;
      float Gx, Gy, Gz, Qx, Qy, Qz;
      window_gradients<BY>(sm.win, z, ty, tx, g.xlo, g.xhi, g.ylo, g.yhi, zlo, zhi,
                           ctr, Gx, Gy, Gz, Qx, Qy, Qz);
      if (WALLS && a.wetting)
        wetting_rule(a, g.xlo, g.xhi, g.ylo, g.yhi, zlo, zhi, Gx, Gy, Gz);
      float f[19];
      const float* h = &sm.hold[z & 1][0][ty - 1][tx - 1];
#pragma unroll
      for (int i = 0; i < 19; ++i) f[i] = h[i * hs];
      const Macro m = macro_held(a, h[19 * hs], h[20 * hs], h[21 * hs], h[22 * hs],
                                 h[23 * hs]);
      const Recolour rc = collide_total<false>(a, f, m, ctr.x, Gx, Gy, Gz, Qx, Qy, Qz);
      store_recoloured<T>(dst, plane, a,
                          (unsigned)z * g.plane_cells + g.co.yo[1] + g.co.xo[1], rc, f);
    }
    if (need2) consume(z + 2, ok2);
    __syncthreads();
  }
}

template <typename T, int BY, bool WALLS, int HOLD,
          int MINB = (BY == 8 && HOLD != 1) ? 2 : 1, bool BGK = false>
static cudaError_t launch_fused_v(const void* src, void* dst,
                                  const StepArgs& a, int zc, cudaStream_t s) {
  dim3 blk(kTileW, BY);
  dim3 grd((a.nx + kTileW - 3) / (kTileW - 2), (a.ny + BY - 3) / (BY - 2),
           (a.nz + zc - 1) / zc);
  k_fused<T, BY, WALLS, HOLD, MINB, BGK><<<grd, blk, 0, s>>>((const T*)src, (T*)dst, a, zc);
  return cudaGetLastError();
}

template <typename T, bool WALLS>
static cudaError_t launch_fused_async(const void* src, void* dst,
                                      const StepArgs& a, int zc,
                                      cudaStream_t s) {
  static bool attr_set[kMaxDevices] = {};
  const int dv = device_slot();
  const int bytes = (int)sizeof(AsyncSmem<T>);
  if (!attr_set[dv]) {
    cudaError_t e = cudaFuncSetAttribute(
        k_fused_async<T, WALLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set[dv] = true;
  }
  dim3 blk(kTileW, kAsyncBY);
  dim3 grd((a.nx + kTileW - 3) / (kTileW - 2), (a.ny + kAsyncBY - 3) / (kAsyncBY - 2),
           (a.nz + zc - 1) / zc);
  k_fused_async<T, WALLS><<<grd, blk, bytes, s>>>((const T*)src, (T*)dst, a, zc);
  return cudaGetLastError();
}

template <typename T, bool WALLS>
static cudaError_t launch_fused2(const void* src, void* dst, const StepArgs& a,
                                 int zc, cudaStream_t s) {
  static bool attr_set[kMaxDevices] = {};
  const int dv = device_slot();
  const int bytes = (int)sizeof(Fused2Smem);
  if (!attr_set[dv]) {
    cudaError_t e = cudaFuncSetAttribute(
        k_fused2<T, WALLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set[dv] = true;
  }
  dim3 blk(kTileW, 8);
  dim3 grd((a.nx + kTileW - 3) / (kTileW - 2), (a.ny + kRows2 - 3) / (kRows2 - 2),
           (a.nz + zc - 1) / zc);
  k_fused2<T, WALLS><<<grd, blk, bytes, s>>>((const T*)src, (T*)dst, a, zc);
  return cudaGetLastError();
}

template <typename T, int BY, bool WALLS>
static cudaError_t launch_fused_h(const void* src, void* dst,
                                  const StepArgs& a, const FusedConfig& cfg,
                                  int zc, cudaStream_t s) {
  switch (cfg.hold) {
    case 0: return launch_fused_v<T, BY, WALLS, 0>(src, dst, a, zc, s);
    case 1: return launch_fused_v<T, BY, WALLS, 1>(src, dst, a, zc, s);
    case 2:
      // the shared-memory hold fits the 48 KB static limit only for BY = 8
      if constexpr (BY == 8) return launch_fused_v<T, BY, WALLS, 2>(src, dst, a, zc, s);
      break;
    case 3:
      if constexpr (BY == 8) return launch_fused_async<T, WALLS>(src, dst, a, zc, s);
      break;
    case 4:
      if constexpr (BY == 16) return launch_fused2<T, WALLS>(src, dst, a, zc, s);
      break;
    case 5:  // as 2, registers capped for three CTAs per SM
      if constexpr (BY == 8) return launch_fused_v<T, BY, WALLS, 2, 3>(src, dst, a, zc, s);
      break;
    case 6:  // as 2, registers capped for four CTAs per SM
      if constexpr (BY == 8) return launch_fused_v<T, BY, WALLS, 2, 4>(src, dst, a, zc, s);
      break;
  }
  return cudaErrorInvalidValue;
}

template <typename T, int BY, bool WALLS, int HOLD, int MINB, bool BGK = false>
static cudaError_t launch_batch_v(const void* src, void* dst, const BatchCase* cases,
                                  int ncases, int total_items, int zc, int sms,
                                  cudaStream_t s) {
  static int per_sm_dev[kMaxDevices] = {};  // resident CTAs per SM, queried once
  int& per_sm = per_sm_dev[device_slot()];
  if (per_sm == 0) {
    int q = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &q, k_fused_batch<T, BY, WALLS, HOLD, MINB, BGK>, kTileW * BY, 0);
    if (e != cudaSuccess) return e;
    per_sm = q < 1 ? 1 : q;
  }
  // one CTA per work item: the hardware hands the next item to whichever
  // SM frees first (a persistent grid's static round-robin shares of
  // unequal items end unevenly)
  const int grid = total_items;
  (void)sms;
  k_fused_batch<T, BY, WALLS, HOLD, MINB, BGK><<<grid, dim3(kTileW, BY), 0, s>>>(
      cases, ncases, total_items, (const T*)src, (T*)dst, zc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fused_batch_storage(const void* src, void* dst,
                                       const BatchCase* cases, int ncases,
                                       int total_items, bool walls, bool bgk,
                                       const FusedConfig& cfg, int sms,
                                       cudaStream_t s) {
  const int zc = cfg.zchunk;
  if (bgk) {  // the BGK operator runs the shared-memory-hold form only
    if (cfg.tile_y != 8 || cfg.hold != 2) return cudaErrorInvalidValue;
    return walls ? launch_batch_v<T, 8, true, 2, 2, true>(src, dst, cases, ncases, total_items, zc, sms, s)
                 : launch_batch_v<T, 8, false, 2, 2, true>(src, dst, cases, ncases, total_items, zc, sms, s);
  }
  if (cfg.tile_y == 8 && cfg.hold == 2)
    return walls ? launch_batch_v<T, 8, true, 2, 2>(src, dst, cases, ncases, total_items, zc, sms, s)
                 : launch_batch_v<T, 8, false, 2, 2>(src, dst, cases, ncases, total_items, zc, sms, s);
  if (cfg.tile_y == 8 && cfg.hold == 0)
    return walls ? launch_batch_v<T, 8, true, 0, 2>(src, dst, cases, ncases, total_items, zc, sms, s)
                 : launch_batch_v<T, 8, false, 0, 2>(src, dst, cases, ncases, total_items, zc, sms, s);
  if (cfg.tile_y == 16 && cfg.hold == 1)
    return walls ? launch_batch_v<T, 16, true, 1, 1>(src, dst, cases, ncases, total_items, zc, sms, s)
                 : launch_batch_v<T, 16, false, 1, 1>(src, dst, cases, ncases, total_items, zc, sms, s);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_fused_storage(const void* src, void* dst,
                                 const StepArgs& a, const FusedConfig& cfg,
                                 cudaStream_t s) {
  const int zc = cfg.zchunk > 0 ? cfg.zchunk : a.nz;
  const bool walls = a.wx || a.wy || a.wz;
  if (a.bgk) {  // the BGK operator runs the shared-memory-hold form only
    if (cfg.tile_y != 8 || cfg.hold != 2) return cudaErrorInvalidValue;
    return walls ? launch_fused_v<T, 8, true, 2, 2, true>(src, dst, a, zc, s)
                 : launch_fused_v<T, 8, false, 2, 2, true>(src, dst, a, zc, s);
  }
  if (cfg.tile_y == 8)
    return walls ? launch_fused_h<T, 8, true>(src, dst, a, cfg, zc, s)
                 : launch_fused_h<T, 8, false>(src, dst, a, cfg, zc, s);
  if (cfg.tile_y == 16)
    return walls ? launch_fused_h<T, 16, true>(src, dst, a, cfg, zc, s)
                 : launch_fused_h<T, 16, false>(src, dst, a, cfg, zc, s);
  return cudaErrorInvalidValue;
}

}  // namespace lbm
