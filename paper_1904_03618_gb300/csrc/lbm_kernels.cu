// Auxiliary kernels (initialisation, state access, moments, FP64
// diagnostics) and the two-pass form of the step, for sm_103a.
//
// Every kernel here maps threads to cells with a 3-D grid (x from the
// thread index, y and z from the block index) and 32-bit cell indices, and
// pulls through the same index function as the fused step (pull_index).
#include "lbm_device.cuh"
#include "lbm_equilibrium.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kAuxBlock = 128;

struct CellPos {
  int x, y, z;
  unsigned c;
};
__device__ __forceinline__ bool cell_pos(const StepArgs& a, CellPos& p) {
  p.x = blockIdx.x * blockDim.x + threadIdx.x;
  p.y = blockIdx.y;
  p.z = blockIdx.z;
  if (p.x >= a.nx) return false;
  p.c = ((unsigned)p.z * (unsigned)a.ny + (unsigned)p.y) * (unsigned)a.nx + (unsigned)p.x;
  return true;
}

// ---------------------------------------------------------------------------
// Scatter of a full state f_i^k(x, t) into the pull-streaming buffer: the
// value f_i(x) is stored exactly where the next pull looks for it
// (pull_index: x - e_i, or, beyond a wall, x itself in direction opp(i)).
// The map is one-to-one.
// ---------------------------------------------------------------------------
template <typename T, int I>
struct ScatterAll {
  __device__ __forceinline__ static void run(T* dst, const StepArgs& a,
                                             const ColOff& co, const PlaneOff& po,
                                             const float* fR, const float* fB) {
    float r = fR[I], b = fB[I];
    if (Store<T>::kDeviation) {
      r -= dev_offset<I>(a, 0);
      b -= dev_offset<I>(a, 1);
    }
    const unsigned q = pull_index<true, I>((unsigned)a.plane, co, po);
    if (index_ok(a, q, 19ull * (unsigned long long)a.plane)) Store<T>::store2(dst + 2 * (size_t)q, r, b);
    ScatterAll<T, I + 1>::run(dst, a, co, po, fR, fB);
  }
};
template <typename T>
struct ScatterAll<T, 19> {
  __device__ __forceinline__ static void run(T*, const StepArgs&, const ColOff&,
                                             const PlaneOff&, const float*,
                                             const float*) {}
};

template <typename T>
__global__ void k_init_eq(T* __restrict__ dst, StepArgs a, float alpha_R,
                          float alpha_B, const float* __restrict__ rho_R,
                          const float* __restrict__ rho_B,
                          const float* __restrict__ u) {
  CellPos p;
  if (!cell_pos(a, p)) return;
  const unsigned N = (unsigned)a.nx * (unsigned)a.ny * (unsigned)a.nz;
  const float ux = u[p.c], uy = u[N + p.c], uz = u[2 * (size_t)N + p.c];
  float fR[19], fB[19];
  equilibrium(rho_R[p.c], alpha_R, ux, uy, uz, a.improved, fR);
  equilibrium(rho_B[p.c], alpha_B, ux, uy, uz, a.improved, fB);
  ScatterAll<T, 0>::run(dst, a, col_off(a, p.x, p.y), plane_off(a, p.z), fR, fB);
}

template <typename T>
__global__ void k_set_f(T* __restrict__ dst, StepArgs a,
                        const float* __restrict__ f) {
  CellPos p;
  if (!cell_pos(a, p)) return;
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  float fR[19], fB[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    fR[i] = f[i * N + p.c];
    fB[i] = f[(19 + i) * N + p.c];
  }
  ScatterAll<T, 0>::run(dst, a, col_off(a, p.x, p.y), plane_off(a, p.z), fR, fB);
}

template <typename T>
__global__ void k_get_f(const T* __restrict__ src, StepArgs a,
                        float* __restrict__ f) {
  CellPos p;
  if (!cell_pos(a, p)) return;
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  float fR[19], fB[19];
  pull_pairs<T>(src, a, p.x, p.y, p.z, fR, fB);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    f[i * N + p.c] = fR[i];
    f[(19 + i) * N + p.c] = fB[i];
  }
}

template <typename T>
__global__ void k_moments(const T* __restrict__ src, StepArgs a,
                          float* __restrict__ rho_R, float* __restrict__ rho_B,
                          float* __restrict__ u) {
  CellPos p;
  if (!cell_pos(a, p)) return;
  const size_t N = (size_t)a.nx * a.ny * a.nz;
  float fR[19], fB[19];
  pull_pairs<T>(src, a, p.x, p.y, p.z, fR, fB);
  const Macro m = macro_of(a, fR, fB);
  if (rho_R) rho_R[p.c] = m.rR;
  if (rho_B) rho_B[p.c] = m.rB;
  if (u) {
    u[p.c] = m.ux;
    u[N + p.c] = m.uy;
    u[2 * N + p.c] = m.uz;
  }
}

// Cells of one lattice plane (normal `axis`, at coordinate `index`) where the
// red colour dominates, rho^N > 0, i.e. rho_R / rho_R^in > rho_B / rho_B^in
// (the order-parameter definition of the phase field).  One thread per plane
// cell, warp ballots, one atomic per warp into the 64-bit count.
template <typename T>
__global__ void k_footprint(const T* __restrict__ src, StepArgs a, int axis, int index,
                            unsigned long long* __restrict__ count) {
  const int n0 = axis == 0 ? a.ny : a.nx;
  const int n1 = axis == 2 ? a.ny : a.nz;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  bool red = false;
  if (e < n0 * n1) {
    const int i = e % n0, j = e / n0;
    const int x = axis == 0 ? index : i;
    const int y = axis == 1 ? index : (axis == 0 ? i : j);
    const int z = axis == 2 ? index : j;
    float fR[19], fB[19];
    pull_pairs<T>(src, a, x, y, z, fR, fB);
    const Macro m = macro_of(a, fR, fB);
    red = m.rR * a.inv_rin_R > m.rB * a.inv_rin_B;
  }
  const unsigned b = __ballot_sync(0xffffffffu, red);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, (unsigned long long)__popc(b));
}

// ---------------------------------------------------------------------------
// Diagnostics with FP64 results.  Work units of one block of 128 (x, y)
// columns times one z range are taken in turn by the resident blocks; a
// thread walks its column over the unit's z range, so the column's offsets
// are formed once and no cell index is divided.  The colour masses and the
// momentum are exact to about FP64 accuracy at FP32 cost (the part's FP64
// rate is far below its FP32 rate): every thread keeps one compensated FP32
// accumulator (Neumaier: running sum plus running error) per direction,
// into which both colours' pulled values are added, and one for all red
// values (57 compensated adds per cell, 40 registers of accumulators).
// The momentum is linear in the per-direction sums, the blue mass is the
// total minus the red mass; both are formed once per thread.  The per-cell
// quantities (finiteness, densities, |u|, the sign of rho^N) come from the
// plain FP32 cell macroscopics the step itself uses, and the red-mass
// centroid moments from the plain per-cell rho_R (centroid to FP32
// accuracy).  Per-thread sums are folded across the warp as compensated
// pairs, across the block in FP64, and the last block folds the block
// partials in a fixed order, so the result is deterministic.
// ---------------------------------------------------------------------------
constexpr int kDiagBlock = 128;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

struct CSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  // adds sign * (o.s + o.c)
  __device__ __forceinline__ void merge(const CSum& o, float sign = 1.f) {
    add(sign * o.s);
    c += sign * o.c;
  }
  // adds x * (o.s + o.c) with the product's rounding error kept (FMA)
  __device__ __forceinline__ void add_scaled(float x, const CSum& o) {
    const float p = x * o.s;
    add(p);
    c += fmaf(x, o.s, -p) + x * o.c;
  }
  // sum over the warp, in lane 0
  __device__ __forceinline__ void warp_fold() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_down_sync(0xffffffffu, s, o);
      const float c2 = __shfl_down_sync(0xffffffffu, c, o);
      add(s2);
      c += c2;
    }
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename T>
__global__ void __launch_bounds__(kDiagBlock, 4)
    k_diag(const T* __restrict__ src, StepArgs a, int zc, unsigned units,
           double* __restrict__ part, unsigned* __restrict__ done,
           const int* __restrict__ flags, double steps, double* __restrict__ out) {
  CSum sT[19];             // per-direction sums of f_i^R + f_i^B (both added)
  CSum sRed;               // sum of every red value
  CSum cx, cy, cz;         // red-mass moments
  unsigned n_nonfinite = 0, n_negative = 0, n_red = 0, n_colour_negative = 0;
  float u2max = 0.f;
  const unsigned nx = (unsigned)a.nx, cols = nx * (unsigned)a.ny;
  const unsigned col_blocks = (cols + kDiagBlock - 1) / kDiagBlock;
  const auto* pairs = reinterpret_cast<const typename Store<T>::Pair*>(src);
  // work unit = (column block, z range); the blocks of one wave take the
  // same z range of neighbouring columns
  for (unsigned u = blockIdx.x; u < units; u += gridDim.x) {
    const unsigned col = (u % col_blocks) * kDiagBlock + threadIdx.x;
    const int z0 = (int)(u / col_blocks) * zc;
    const int z1 = min(a.nz, z0 + zc);
    if (col >= cols) continue;
    const unsigned y = col / nx, x = col - y * nx;
    const ColOff co = col_off(a, (int)x, (int)y);
    CSum colR, colZ;
    for (int z = z0; z < z1; ++z) {
      float fR[19], fB[19];
      PullPairs<T, 0>::run(pairs, a, co, plane_off(a, z), fR, fB);
      // x * 0 is 0 for finite x and NaN for infinities and NaN
      float bad = 0.f;
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        sT[i].add(fR[i]);
        sT[i].add(fB[i]);
        sRed.add(fR[i]);
        bad = fmaf(fR[i], 0.f, bad);
        bad = fmaf(fB[i], 0.f, bad);
      }
      const bool finite = bad == 0.f;
      const Macro m = macro_of(a, fR, fB);
      n_nonfinite += finite ? 0u : 1u;
      n_negative += (m.rho <= 0.f) ? 1u : 0u;
      n_colour_negative += (m.rR < 0.f || m.rB < 0.f) ? 1u : 0u;
      const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
      if (finite && u2 > u2max) u2max = u2;
      n_red += phase_field(a, m.rR, m.rB) > 0.f ? 1u : 0u;
      colR.add(m.rR);
      colZ.add(m.rR * (float)z);
    }
    cx.add_scaled((float)x, colR);
    cy.add_scaled((float)y, colR);
    cz.merge(colZ);
  }
  // blue mass = all values - red values, both as compensated pairs
  CSum mR = sRed, mB, jx, jy, jz;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    mB.merge(sT[i]);
    if (ex(i)) jx.merge(sT[i], (float)ex(i));
    if (ey(i)) jy.merge(sT[i], (float)ey(i));
    if (ez(i)) jz.merge(sT[i], (float)ez(i));
  }
  mB.merge(sRed, -1.f);
  CSum* sums[8] = {&mR, &mB, &jx, &jy, &jz, &cx, &cy, &cz};
#pragma unroll
  for (int k = 0; k < 8; ++k) sums[k]->warp_fold();
  const unsigned full = 0xffffffffu;
  n_nonfinite = __reduce_add_sync(full, n_nonfinite);
  n_negative = __reduce_add_sync(full, n_negative);
  n_red = __reduce_add_sync(full, n_red);
  n_colour_negative = __reduce_add_sync(full, n_colour_negative);
  // u2max >= 0 and never NaN, so its bit pattern orders like the value
  const unsigned u2bits = __reduce_max_sync(full, __float_as_uint(u2max));
  __shared__ double sh[kDiagBlock / 32][kDiagSlots];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    double* w = sh[wid];
    w[0] = mR.value();
    w[1] = mB.value();
    w[2] = jx.value();
    w[3] = jy.value();
    w[4] = jz.value();
    w[5] = (double)n_nonfinite;
    w[6] = (double)n_negative;
    w[7] = sqrt((double)__uint_as_float(u2bits));
    w[8] = (double)n_red;
    w[9] = cx.value();
    w[10] = cy.value();
    w[11] = cz.value();
    w[12] = (double)n_colour_negative;
  }
  __syncthreads();
  if (threadIdx.x < kDiagSlots) {
    const int s = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < kDiagBlock / 32; ++w)
      v = (s == 7) ? fmax(v, sh[w][s]) : v + sh[w][s];
    part[(size_t)blockIdx.x * kDiagSlots + s] = v;
    __threadfence();
  }
  // The last block to finish folds every block's partials: thread t takes
  // the blocks t, t + 128, ... (all slots of a block at once, so its loads
  // are independent), then a fixed shuffle tree and a fixed sum over the
  // warps: the order does not depend on which block came last.  It writes
  // the 16 result slots (centroid divided by the red mass, the step count,
  // the step kernels' error word) and re-arms the counter.
  __shared__ bool last;
  __syncthreads();
  const unsigned nb = gridDim.x;
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == nb - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double fold[kDiagSlots];
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) fold[k] = 0.0;
  for (unsigned b = threadIdx.x; b < nb; b += kDiagBlock) {
    double p[kDiagSlots];
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) p[k] = __ldcg(part + (size_t)b * kDiagSlots + k);
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) fold[k] = (k == 7) ? fmax(fold[k], p[k]) : fold[k] + p[k];
  }
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) {
    const double v = (k == 7) ? warp_max(fold[k]) : warp_sum(fold[k]);
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double fin[kDiagSlots];
    for (int k = 0; k < kDiagSlots; ++k) {
      fin[k] = 0.0;
      for (int w = 0; w < kDiagBlock / 32; ++w)
        fin[k] = (k == 7) ? fmax(fin[k], sh[w][k]) : fin[k] + sh[w][k];
    }
    for (int k = 0; k < 12; ++k) out[k] = fin[k];
    if (fin[0] > 0.0)
      for (int k = 9; k < 12; ++k) out[k] = fin[k] / fin[0];
    out[12] = steps;
    out[13] = fin[12];
    out[14] = (double)__ldcg(flags);
    out[15] = 0.0;
    *done = 0u;
  }
}

// ---------------------------------------------------------------------------
// Moving plates (Sec. IV.A): Zou-He velocity nodes on both faces of one
// axis.  One thread per plate node.  The node's known populations are
// pulled; for each colour k, rho_k = (S_0 + 2 S_out) / (1 - u_n) (S_0: the
// populations parallel to the plate, S_out: those leaving through it, u_n
// the plate's inward normal velocity), and each entering population
// f_i = f_opp(i) + 6 w_i rho_k (e_i . u) - e_i . N with the transverse
// corrections N_t = (1/2) sum_{e_j . n = 0} f_j e_jt - rho_k u_t / 3, which
// make the colour's momentum exactly rho_k u.  f_i is written where the
// next pull of direction i at the node looks (the node's own slot of
// opp(i), as at a wall); no other node reads that slot.
// ---------------------------------------------------------------------------
struct PlateArgs {
  float u[2][3];  // plate velocities (low, high)
  int axis;
};

template <typename T>
__global__ void __launch_bounds__(kAuxBlock)
    k_plates(T* __restrict__ buf, StepArgs a, PlateArgs pl) {
  const int ax = pl.axis, t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
  const int n[3] = {a.nx, a.ny, a.nz};
  const int per_face = n[t1] * n[t2];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * per_face) return;
  const int side = e / per_face, r = e - side * per_face;
  int xyz[3];
  xyz[ax] = side == 0 ? 0 : n[ax] - 1;
  xyz[t1] = r % n[t1];
  xyz[t2] = r / n[t1];
  const int sgn = side == 0 ? 1 : -1;  // inward normal along ax
  const float ux = pl.u[side][0], uy = pl.u[side][1], uz = pl.u[side][2];
  const float uu[3] = {ux, uy, uz};
  const float un = sgn * uu[ax];
  float fR[19], fB[19];
  pull_pairs<T>(buf, a, xyz[0], xyz[1], xyz[2], fR, fB);
  const unsigned c =
      ((unsigned)xyz[2] * (unsigned)a.ny + (unsigned)xyz[1]) * (unsigned)a.nx + (unsigned)xyz[0];
  auto en = [&](int i) { return sgn * (ax == 0 ? ex(i) : (ax == 1 ? ey(i) : ez(i))); };
  auto et = [&](int i, int d) { return d == 0 ? ex(i) : (d == 1 ? ey(i) : ez(i)); };
  float* fk[2] = {fR, fB};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float s0 = 0.f, sout = 0.f, tg[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      const int ni = en(i);
      if (ni == 0) {
        s0 += fk[k][i];
        tg[0] += ex(i) * fk[k][i];
        tg[1] += ey(i) * fk[k][i];
        tg[2] += ez(i) * fk[k][i];
      } else if (ni < 0) {
        sout += fk[k][i];
      }
    }
    const float rho = (s0 + 2.f * sout) / (1.f - un);
    float N[3] = {0.f, 0.f, 0.f};
    N[t1] = 0.5f * tg[t1] - rho * uu[t1] * (1.0f / 3.0f);
    N[t2] = 0.5f * tg[t2] - rho * uu[t2] * (1.0f / 3.0f);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      if (en(i) != 1) continue;
      const float eu = ex(i) * ux + ey(i) * uy + ez(i) * uz;
      const float corr = et(i, 0) * N[0] + et(i, 1) * N[1] + et(i, 2) * N[2];
      const float w = shell(i) == 1 ? (1.0f / 18.0f) : (1.0f / 36.0f);
      fk[k][i] = fk[k][opp(i)] + 6.f * w * rho * eu - corr;
    }
  }
  // write the entering populations (both colours) to their pull slots
  if (!index_ok(a, c, (unsigned long long)a.plane)) return;
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    if (en(i) != 1) continue;
    float rv = fR[i], bv = fB[i];
    if (Store<T>::kDeviation) {
      const int sh = shell(i);
      rv -= sh == 1 ? a.offR1 : a.offR2;
      bv -= sh == 1 ? a.offB1 : a.offB2;
    }
    Store<T>::store2(buf + 2 * ((size_t)opp(i) * (unsigned)a.plane + c), rv, bv);
  }
}

// ---------------------------------------------------------------------------
// Two-pass step.  Pass 1 writes, per cell, (rho^N, Qbar_x, Qbar_y, Qbar_z)
// to a scratch field; pass 2 pulls the populations again, forms the Eq. 49
// gradients from the neighbours' scratch entries and collides.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
    k_twopass_phase(const T* __restrict__ src, StepArgs a,
                    float4* __restrict__ mom) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  float fR[19], fB[19];
  pull_pairs<T>(src, a, x, y, z, fR, fB);
  const Macro m = macro_of(a, fR, fB);
  mom[((unsigned)z * (unsigned)a.ny + (unsigned)y) * (unsigned)a.nx + (unsigned)x] =
      stencil_entry(a, m);
}

// Neighbour x + e of the Eq. 49 stencil; beyond a wall the centre cell.
__device__ __forceinline__ unsigned stencil_cell(const StepArgs& a, int x,
                                                 int y, int z, int dx, int dy,
                                                 int dz, unsigned c) {
  const int xn = x + dx, yn = y + dy, zn = z + dz;
  if ((a.wx && (xn < 0 || xn >= a.nx)) || (a.wy && (yn < 0 || yn >= a.ny)) ||
      (a.wz && (zn < 0 || zn >= a.nz)))
    return c;
  return ((unsigned)wrap1(zn, a.nz) * (unsigned)a.ny + (unsigned)wrap1(yn, a.ny)) *
             (unsigned)a.nx +
         (unsigned)wrap1(xn, a.nx);
}

template <typename T, bool BGK>
__global__ void __launch_bounds__(256)
    k_twopass_collide(const T* __restrict__ src, T* __restrict__ dst,
                      StepArgs a, const float4* __restrict__ mom) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  const unsigned c = ((unsigned)z * (unsigned)a.ny + (unsigned)y) * (unsigned)a.nx + (unsigned)x;
  float fR[19], fB[19];
  pull_pairs<T>(src, a, x, y, z, fR, fB);
  const Macro m = macro_of(a, fR, fB);
  // Eq. 49: d_a psi = 3 sum_i w_i psi(x + e_i) e_ia = (1/6) axis differences
  // + (1/12) diagonal differences, accumulated as differences of opposite
  // neighbours so that a uniform field gives an exactly zero gradient.
  float Gx = 0.f, Gy = 0.f, Gz = 0.f, Qx = 0.f, Qy = 0.f, Qz = 0.f;
#pragma unroll
  for (int i = 1; i < 19; i += 2) {
    const float w = (i <= 6) ? (1.0f / 6.0f) : (1.0f / 12.0f);
    const float4 vp = __ldg(&mom[stencil_cell(a, x, y, z, ex(i), ey(i), ez(i), c)]);
    const float4 vm = __ldg(&mom[stencil_cell(a, x, y, z, -ex(i), -ey(i), -ez(i), c)]);
    if (ex(i)) {
      Gx += (ex(i) * w) * (vp.x - vm.x);
      Qx += (ex(i) * w) * (vp.y - vm.y);
    }
    if (ey(i)) {
      Gy += (ey(i) * w) * (vp.x - vm.x);
      Qy += (ey(i) * w) * (vp.z - vm.z);
    }
    if (ez(i)) {
      Gz += (ez(i) * w) * (vp.x - vm.x);
      Qz += (ez(i) * w) * (vp.w - vm.w);
    }
  }
  if (a.wetting)
    wetting_rule(a, a.wx && x == 0, a.wx && x == a.nx - 1, a.wy && y == 0,
                 a.wy && y == a.ny - 1, a.wz && z == 0, a.wz && z == a.nz - 1, Gx, Gy, Gz);
  const float rn = __ldg(&mom[c]).x;
  collide_cell<BGK>(a, fR, fB, m, rn, Gx, Gy, Gz, Qx, Qy, Qz);
  store_cell<T>(dst, a, c, fR, fB);
}

// ---------------------------------------------------------------------------
// Launchers (host side).
// ---------------------------------------------------------------------------
static inline dim3 aux_grid(const StepArgs& a) {
  return dim3((a.nx + kAuxBlock - 1) / kAuxBlock, a.ny, a.nz);
}

template <typename T>
cudaError_t launch_init_eq_t(void* dst, const StepArgs& a, float alpha_R,
                             float alpha_B, const float* rR, const float* rB,
                             const float* u, cudaStream_t s) {
  k_init_eq<T><<<aux_grid(a), kAuxBlock, 0, s>>>((T*)dst, a, alpha_R, alpha_B, rR, rB, u);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_set_f_t(void* dst, const StepArgs& a, const float* f,
                           cudaStream_t s) {
  k_set_f<T><<<aux_grid(a), kAuxBlock, 0, s>>>((T*)dst, a, f);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_get_f_t(const void* src, const StepArgs& a, float* f,
                           cudaStream_t s) {
  k_get_f<T><<<aux_grid(a), kAuxBlock, 0, s>>>((const T*)src, a, f);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_moments_t(const void* src, const StepArgs& a, float* rR,
                             float* rB, float* u, cudaStream_t s) {
  k_moments<T><<<aux_grid(a), kAuxBlock, 0, s>>>((const T*)src, a, rR, rB, u);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_footprint_t(const void* src, const StepArgs& a, int axis, int index,
                               unsigned long long* count, cudaStream_t s) {
  const int n0 = axis == 0 ? a.ny : a.nx;
  const int n1 = axis == 2 ? a.ny : a.nz;
  const unsigned blocks = (unsigned)((n0 * n1 + kAuxBlock - 1) / kAuxBlock);
  k_footprint<T><<<blocks, kAuxBlock, 0, s>>>((const T*)src, a, axis, index, count);
  return cudaGetLastError();
}
// Grid of the diagnostics: work units of one column block x one z range,
// taken in turn by at most max_blocks blocks (the partials scratch holds
// that many; max_blocks is the number resident at once).  The z split
// minimises rounds x planes per unit, rounds = units / blocks rounded up,
// so that no block walks a whole extra column while the others idle.
template <typename T>
cudaError_t launch_diag_t(const void* src, const StepArgs& a, double* part,
                          int max_blocks, unsigned* done, const int* flags,
                          long long steps, double* out, cudaStream_t s) {
  const long long cols = (long long)a.nx * a.ny;
  const long long cb = (cols + kDiagBlock - 1) / kDiagBlock;
  long long best_zs = 1;
  double best = -1.0;
  for (long long zs = 1; zs <= a.nz; ++zs) {
    const long long zc = (a.nz + zs - 1) / zs;
    if ((zs - 1) * zc >= a.nz) continue;       // same split as a smaller zs
    const long long units = cb * zs;
    const long long rounds = (units + max_blocks - 1) / max_blocks;
    const double cost = (double)rounds * ((double)zc + 0.25);
    if (best < 0.0 || cost < best) {
      best = cost;
      best_zs = zs;
    }
  }
  const int zc = (int)((a.nz + best_zs - 1) / best_zs);
  const long long zs = (a.nz + zc - 1) / zc;
  const long long units = cb * zs;
  const int blocks = (int)(units < max_blocks ? units : max_blocks);
  k_diag<T><<<blocks, kDiagBlock, 0, s>>>((const T*)src, a, zc, (unsigned)units, part,
                                          done, flags, (double)steps, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_plates_t(void* buf, const StepArgs& a, int axis, const double u[2][3],
                            cudaStream_t s) {
  PlateArgs pl;
  pl.axis = axis;
  for (int side = 0; side < 2; ++side)
    for (int d = 0; d < 3; ++d) pl.u[side][d] = (float)u[side][d];
  const int n[3] = {a.nx, a.ny, a.nz};
  const long long nodes = 2LL * n[(axis + 1) % 3] * n[(axis + 2) % 3];
  const unsigned blocks = (unsigned)((nodes + kAuxBlock - 1) / kAuxBlock);
  k_plates<T><<<blocks, kAuxBlock, 0, s>>>((T*)buf, a, pl);
  return cudaGetLastError();
}
template <typename T>
int diag_capacity_t(int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_diag<T>,
                                                    kDiagBlock, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * sms;
}
template <typename T>
cudaError_t launch_twopass_t(const void* src, void* dst, const StepArgs& a,
                             float4* mom, cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grd((a.nx + 31) / 32, (a.ny + 7) / 8, a.nz);
  k_twopass_phase<T><<<grd, blk, 0, s>>>((const T*)src, a, mom);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.bgk)
    k_twopass_collide<T, true><<<grd, blk, 0, s>>>((const T*)src, (T*)dst, a, mom);
  else
    k_twopass_collide<T, false><<<grd, blk, 0, s>>>((const T*)src, (T*)dst, a, mom);
  return cudaGetLastError();
}

#define LBM_DISPATCH(storage, FN, ...)                                 \
  switch (storage) {                                                   \
    case 0: return FN<float>(__VA_ARGS__);                             \
    case 1: return FN<__half>(__VA_ARGS__);                            \
    case 2: return FN<__nv_bfloat16>(__VA_ARGS__);                     \
  }                                                                    \
  return cudaErrorInvalidValue;

cudaError_t launch_init_eq(int storage, void* dst, const StepArgs& a,
                           float alpha_R, float alpha_B, const float* rR,
                           const float* rB, const float* u, cudaStream_t s) {
  LBM_DISPATCH(storage, launch_init_eq_t, dst, a, alpha_R, alpha_B, rR, rB, u,
               s)
}
cudaError_t launch_set_f(int storage, void* dst, const StepArgs& a,
                         const float* f, cudaStream_t s) {
  LBM_DISPATCH(storage, launch_set_f_t, dst, a, f, s)
}
cudaError_t launch_get_f(int storage, const void* src, const StepArgs& a,
                         float* f, cudaStream_t s) {
  LBM_DISPATCH(storage, launch_get_f_t, src, a, f, s)
}
cudaError_t launch_moments(int storage, const void* src, const StepArgs& a,
                           float* rR, float* rB, float* u, cudaStream_t s) {
  LBM_DISPATCH(storage, launch_moments_t, src, a, rR, rB, u, s)
}
cudaError_t launch_footprint(int storage, const void* src, const StepArgs& a, int axis,
                             int index, unsigned long long* count, cudaStream_t s) {
  LBM_DISPATCH(storage, launch_footprint_t, src, a, axis, index, count, s)
}
cudaError_t launch_diag(int storage, const void* src, const StepArgs& a,
                        double* part, int max_blocks, unsigned* done,
                        const int* flags, long long steps, double* out,
                        cudaStream_t s) {
  LBM_DISPATCH(storage, launch_diag_t, src, a, part, max_blocks, done, flags, steps,
               out, s)
}
cudaError_t launch_plates(int storage, void* buf, const StepArgs& a, int axis,
                          const double u[2][3], cudaStream_t s) {
  if (axis < 0 || axis > 2) return cudaErrorInvalidValue;
  LBM_DISPATCH(storage, launch_plates_t, buf, a, axis, u, s)
}
int diag_capacity(int storage, int sms) {
  switch (storage) {
    case 1: return diag_capacity_t<__half>(sms);
    case 2: return diag_capacity_t<__nv_bfloat16>(sms);
    default: return diag_capacity_t<float>(sms);
  }
}
cudaError_t launch_twopass(int storage, const void* src, void* dst,
                           const StepArgs& a, float4* mom, cudaStream_t s) {
  LBM_DISPATCH(storage, launch_twopass_t, src, dst, a, mom, s)
}

// A monitored step's record -> the 16 slots of lbm_diagnostics (steps: the
// steps completed before the state the step read); the record is cleared
// for the next step.
__global__ void k_monitor_out(MonAcc* __restrict__ acc, const int* __restrict__ flags,
                              double steps, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < 5; ++k) out[k] = acc->d[k];
  out[5] = (double)acc->n[0];
  out[6] = (double)acc->n[1];
  out[7] = sqrt((double)__uint_as_float(acc->u2bits));
  out[8] = (double)acc->n[2];
  for (int k = 5; k < 8; ++k) out[4 + k] = acc->d[0] > 0.0 ? acc->d[k] / acc->d[0] : acc->d[k];
  out[12] = steps;
  out[13] = (double)acc->n[3];
  out[14] = (double)*flags;
  out[15] = 0.0;
  for (int k = 0; k < 8; ++k) acc->d[k] = 0.0;
  for (int k = 0; k < 4; ++k) acc->n[k] = 0u;
  acc->u2bits = 0u;
}
cudaError_t launch_monitor_out(MonAcc* acc, const int* flags, double steps, double* out,
                               cudaStream_t s) {
  k_monitor_out<<<1, 32, 0, s>>>(acc, flags, steps, out);
  return cudaGetLastError();
}

}  // namespace lbm
