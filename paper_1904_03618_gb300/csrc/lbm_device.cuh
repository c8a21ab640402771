// Device-side building blocks of the colour-gradient MRT-LB step
// (Wen, Li, Yu & Luo, arXiv:1904.03618) for sm_103a.
//
// The collision is written for the total population f = f^R + f^B: the
// relaxation matrix S (Eq. 44) depends only on the cell's phase field, so
// summing Eq. 41 over the two colours gives one 19-moment update
//   m* = m - S (m - sum_k m^{k,eq}) + (I - S/2)(sum_k C^k + F_hat) + S P_hat
// followed by f* = f + M^-1 (m* - m) (Eq. 42, 12, 53).  All moment-space
// quantities are closed forms of the raw-moment basis of Eq. 43:
//   m^eq   Appendix rows 0-15; rows 16-18 as M f^eq (the printed rows 16-18
//          differ from M f^eq at O(u^2); the paper defines m^eq = M f^eq);
//          third-order rows carry p_k u (Eq. 19), i.e. the Eq. 18 high-order
//          term with coefficient 3 (the printed 3/2 gives half of Eq. 19);
//   C      Eq. 45-48, rows 4-6 only;
//   F_hat  M times the Guo forcing term (force density F, u shifted by F/2);
//   P_hat  M times the summed perturbation of Eq. 8, executed through S as
//          Eq. 53 prescribes.
// M^-1 is applied in its sparse closed form (99 non-zeros).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---------------------------------------------------------------------------
// Step arguments, derived on the host from lbm_params.
// ---------------------------------------------------------------------------
struct StepArgs {
  int nx, ny, nz;
  int wx, wy, wz;           // wall flags per axis
  long long plane;          // elements per (colour, direction) plane
  int improved;
  int bgk;                      // 1: every non-conserved rate is 1 / tau_v (Eq. 20)
  float inv_rin_R, inv_rin_B;   // 1 / rho_k^in (below Eq. 8)
  float cs2_R, cs2_B;           // (c_s^k)^2 = (1 - alpha_k) / 2 (Eq. 13)
  float q_R, q_B;               // 1 - 3 (c_s^k)^2 (below Eq. 49)
  float tau_R, tau_B;           // Eq. 52 end values
  float tau_h;                  // 2 tau_R tau_B / (tau_R + tau_B)
  float par_a, par_b;           // slopes of g^R, g^B at rho^N = 0
  float par_a2, par_b2;         // par_a / (2 delta), par_b / (2 delta)
  float delta;                  // Eq. 52
  int has_force;                // any non-zero force or gravity component
  int wetting;                  // contact-angle rule at wall-adjacent cells
  float cos_t, sin_t;           // cos and sin of the contact angle
  float s_e, s_q, s_pi;         // 1/tau_e, 1/tau_q, 1/tau_pi (Eq. 44)
  float half_A;                 // (A_R + A_B) / 2, Eq. 8 summed over colours
  float beta;                   // Eq. 10-11
  float fx, fy, fz;             // uniform force density
  float gx, gy, gz;             // gravity
  // deviation storage offsets ref_k * phi_i^k for (rest, axis, diagonal)
  float offR0, offR1, offR2, offB0, offB1, offB2;
  // checked builds (LBM_CHECKED): count of out-of-range indices, else null
  unsigned* oob;
};

// Checked builds (compiled with -DLBM_CHECKED, the stand-in for a memory
// checker): the step kernels test every computed population index against
// its buffer before the access, count an index out of range in *a.oob and
// skip that access.  Normal builds compile the test away.
#ifdef LBM_CHECKED
__device__ __forceinline__ bool index_ok(const StepArgs& a, unsigned long long i,
                                         unsigned long long n) {
  if (i < n) return true;
  if (a.oob) atomicAdd(a.oob, 1u);
  return false;
}
#else
__device__ __forceinline__ constexpr bool index_ok(const StepArgs&, unsigned long long,
                                                   unsigned long long) {
  return true;
}
#endif

// ---------------------------------------------------------------------------
// D3Q19 lattice of Eq. 5, as compile-time functions of the direction index.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ex(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int ez(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
// Opposite pairs are (1,2), (3,4), ..., (17,18).
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
}
// 0 = rest, 1 = axis (|e| = 1), 2 = diagonal (|e| = sqrt 2)
__host__ __device__ constexpr int shell(int i) {
  return i == 0 ? 0 : (i <= 6 ? 1 : 2);
}

// ---------------------------------------------------------------------------
// Storage formats.  The red and blue values of one direction and cell are
// adjacent (one 8-byte FP32 pair or one 4-byte half pair), so one access
// moves both colours.  FP32 stores f itself; FP16 / BF16 store the deviation
// f - ref_k phi_i^k and are converted to FP32 on load.
// ---------------------------------------------------------------------------
template <typename T>
struct Store;

template <>
struct Store<float> {
  static constexpr bool kDeviation = false;
  using Pair = float2;
  __device__ __forceinline__ static float2 load2(const float* p) {
    return __ldg(reinterpret_cast<const float2*>(p));
  }
  __device__ __forceinline__ static void store2(float* p, float r, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(r, b);
  }
  __device__ __forceinline__ static float2 to_float2(float2 v) { return v; }
};
template <>
struct Store<__half> {
  static constexpr bool kDeviation = true;
  using Pair = __half2;
  __device__ __forceinline__ static float2 load2(const __half* p) {
    return __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
  }
  __device__ __forceinline__ static void store2(__half* p, float r, float b) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(r, b);
  }
  __device__ __forceinline__ static float2 to_float2(__half2 v) {
    return __half22float2(v);
  }
};
template <>
struct Store<__nv_bfloat16> {
  static constexpr bool kDeviation = true;
  using Pair = __nv_bfloat162;
  __device__ __forceinline__ static float2 load2(const __nv_bfloat16* p) {
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
  }
  __device__ __forceinline__ static void store2(__nv_bfloat16* p, float r,
                                                float b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(r, b);
  }
  __device__ __forceinline__ static float2 to_float2(__nv_bfloat162 v) {
    return __bfloat1622float2(v);
  }
};

template <int I>
__device__ __forceinline__ float dev_offset(const StepArgs& a, int k) {
  constexpr int s = shell(I);
  if (k == 0) return s == 0 ? a.offR0 : (s == 1 ? a.offR1 : a.offR2);
  return s == 0 ? a.offB0 : (s == 1 ? a.offB1 : a.offB2);
}

// Reciprocal through the special-function unit (relative error of a few ulp,
// far below the FP32 parity bar); the IEEE-exact division is a multi-
// instruction sequence on the critical path of every cell.
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }

// ---------------------------------------------------------------------------
// Indexing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap1(int v, int n) {
  return v < 0 ? v + n : (v >= n ? v - n : v);
}
// Wrapped neighbour offsets of one column / plane (index d + 1 for x + d).
struct ColOff {
  unsigned xo[3], yo[3];
  bool bxl, bxh, byl, byh;  // pull source beyond a wall (x-1 < 0, x+1 >= n)
};
struct PlaneOff {
  unsigned zo[3];
  bool bzl, bzh;
};

__device__ __forceinline__ int wrapn(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Pair index of the pulled value of direction I: f_I(x) comes from x - e_I,
// or, beyond a wall, from direction opp(I) of x itself (halfway bounce-back).
template <bool WALLS, int I>
__device__ __forceinline__ unsigned pull_index(unsigned plane, const ColOff& c,
                                               const PlaneOff& p) {
  unsigned cs = p.zo[1 - ez(I)] + c.yo[1 - ey(I)] + c.xo[1 - ex(I)];
  unsigned q = I;
  if (WALLS) {
    const bool out = (ex(I) > 0 && c.bxl) || (ex(I) < 0 && c.bxh) ||
                     (ey(I) > 0 && c.byl) || (ey(I) < 0 && c.byh) ||
                     (ez(I) > 0 && p.bzl) || (ez(I) < 0 && p.bzh);
    if (out) {
      cs = p.zo[1] + c.yo[1] + c.xo[1];
      q = opp(I);
    }
  }
  return q * plane + cs;
}

// Offsets of the cell (x, y, z), all in range, for pull_index.
__device__ __forceinline__ ColOff col_off(const StepArgs& a, int x, int y) {
  ColOff c;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    c.xo[d] = (unsigned)wrap1(x + d - 1, a.nx);
    c.yo[d] = (unsigned)wrap1(y + d - 1, a.ny) * (unsigned)a.nx;
  }
  c.bxl = a.wx && x == 0;
  c.bxh = a.wx && x == a.nx - 1;
  c.byl = a.wy && y == 0;
  c.byh = a.wy && y == a.ny - 1;
  return c;
}
__device__ __forceinline__ PlaneOff plane_off(const StepArgs& a, int z) {
  PlaneOff p;
  const unsigned pc = (unsigned)a.nx * (unsigned)a.ny;
#pragma unroll
  for (int d = 0; d < 3; ++d) p.zo[d] = (unsigned)wrap1(z + d - 1, a.nz) * pc;
  p.bzl = a.wz && z == 0;
  p.bzh = a.wz && z == a.nz - 1;
  return p;
}

// Pull of both colours of all 19 directions of one cell (walls handled at
// run time), converted to FP32 with the deviation offsets added back.
template <typename T, int I>
struct PullPairs {
  __device__ __forceinline__ static void run(const typename Store<T>::Pair* src,
                                             const StepArgs& a, const ColOff& c,
                                             const PlaneOff& p, float* fR,
                                             float* fB) {
    const unsigned q = pull_index<true, I>((unsigned)a.plane, c, p);
    float2 v = make_float2(0.f, 0.f);
    if (index_ok(a, q, 19ull * (unsigned long long)a.plane))
      v = Store<T>::to_float2(__ldg(src + q));
    if (Store<T>::kDeviation) {
      v.x += dev_offset<I>(a, 0);
      v.y += dev_offset<I>(a, 1);
    }
    fR[I] = v.x;
    fB[I] = v.y;
    PullPairs<T, I + 1>::run(src, a, c, p, fR, fB);
  }
};
template <typename T>
struct PullPairs<T, 19> {
  __device__ __forceinline__ static void run(const typename Store<T>::Pair*,
                                             const StepArgs&, const ColOff&,
                                             const PlaneOff&, float*, float*) {}
};
template <typename T>
__device__ __forceinline__ void pull_pairs(const T* src, const StepArgs& a, int x,
                                           int y, int z, float* fR, float* fB) {
  PullPairs<T, 0>::run(reinterpret_cast<const typename Store<T>::Pair*>(src), a,
                       col_off(a, x, y), plane_off(a, z), fR, fB);
}

// Store of the post-recolouring populations at the cell itself (the next
// step pulls them).
template <typename T>
__device__ __forceinline__ void store_cell(T* __restrict__ dst,
                                           const StepArgs& a, unsigned c,
                                           const float* fR, const float* fB) {
  if (!index_ok(a, c, (unsigned long long)a.plane)) return;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    float r = fR[i], b = fB[i];
    if (Store<T>::kDeviation) {
      const int s = shell(i);
      r -= s == 0 ? a.offR0 : (s == 1 ? a.offR1 : a.offR2);
      b -= s == 0 ? a.offB0 : (s == 1 ? a.offB1 : a.offB2);
    }
    Store<T>::store2(dst + 2 * ((size_t)i * (unsigned)a.plane + c), r, b);
  }
}

// ---------------------------------------------------------------------------
// Cell macroscopics (Eq. 4 with the forcing shift; rho^N below Eq. 8).
// ---------------------------------------------------------------------------
struct Macro {
  float rR, rB, rho, inv_rho, ux, uy, uz, Fx, Fy, Fz;
};

// From the total populations f_i = f_i^R + f_i^B and the colour densities.
__device__ __forceinline__ Macro macro_total(const StepArgs& a, const float* f,
                                             float rR, float rB) {
  Macro m;
  const float jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) +
                   (f[11] - f[12]) + (f[13] - f[14]);
  const float jy = (f[3] - f[4]) + (f[7] - f[8]) + (f[10] - f[9]) +
                   (f[15] - f[16]) + (f[17] - f[18]);
  const float jz = (f[5] - f[6]) + (f[11] - f[12]) + (f[14] - f[13]) +
                   (f[15] - f[16]) + (f[18] - f[17]);
  m.rR = rR;
  m.rB = rB;
  m.rho = rR + rB;
  m.inv_rho = fast_rcp(m.rho);
  m.Fx = a.fx + m.rho * a.gx;
  m.Fy = a.fy + m.rho * a.gy;
  m.Fz = a.fz + m.rho * a.gz;
  m.ux = (jx + 0.5f * m.Fx) * m.inv_rho;
  m.uy = (jy + 0.5f * m.Fy) * m.inv_rho;
  m.uz = (jz + 0.5f * m.Fz) * m.inv_rho;
  return m;
}

// Macroscopics from held values (colour densities and velocity).
__device__ __forceinline__ Macro macro_held(const StepArgs& a, float rR,
                                            float rB, float ux, float uy,
                                            float uz) {
  Macro m;
  m.rR = rR;
  m.rB = rB;
  m.rho = rR + rB;
  m.inv_rho = fast_rcp(m.rho);
  m.Fx = a.fx + m.rho * a.gx;
  m.Fy = a.fy + m.rho * a.gy;
  m.Fz = a.fz + m.rho * a.gz;
  m.ux = ux;
  m.uy = uy;
  m.uz = uz;
  return m;
}

// Reduces the pulled colour populations to (f = fR + fB, rho_R, rho_B), all
// that the collision and recolouring of the cell need.
__device__ __forceinline__ void reduce_colours(const float* fR, const float* fB,
                                               float* f, float& rR, float& rB) {
  rR = 0.f;
  rB = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    rR += fR[i];
    rB += fB[i];
    f[i] = fR[i] + fB[i];
  }
}

__device__ __forceinline__ Macro macro_of(const StepArgs& a, const float* fR,
                                          const float* fB) {
  float f[19], rR, rB;
  reduce_colours(fR, fB, f, rR, rB);
  return macro_total(a, f, rR, rB);
}

__device__ __forceinline__ float phase_field(const StepArgs& a, float rR,
                                             float rB) {
  float r = rR * a.inv_rin_R, b = rB * a.inv_rin_B;
  return (r - b) * fast_rcp(r + b);
}

// Sum over colours of rho_k (1 - 3 c_s^k^2): Qbar_alpha = u_alpha * this.
__device__ __forceinline__ float qbar_scale(const StepArgs& a, float rR,
                                            float rB) {
  return a.q_R * rR + a.q_B * rB;
}

// Window entry of the Eq. 49 stencils: (rho^N, Qbar_x, Qbar_y, Qbar_z).
__device__ __forceinline__ float4 stencil_entry(const StepArgs& a,
                                                const Macro& m) {
  const float q = qbar_scale(a, m.rR, m.rB);
  return make_float4(phase_field(a, m.rR, m.rB), m.ux * q, m.uy * q, m.uz * q);
}

// Eq. 52 with the parabolic g^R, g^B (continuous, zero slope at +-delta,
// harmonic mean at rho^N = 0).
__device__ __forceinline__ float tau_v_of(const StepArgs& a, float rn) {
  if (rn > a.delta) return a.tau_R;
  if (rn > 0.f) return a.tau_h + rn * (a.par_a - a.par_a2 * rn);
  if (rn >= -a.delta)
    return a.tau_h + rn * (a.par_b + a.par_b2 * rn);
  return a.tau_B;
}

// Contact-angle rule at a fluid cell next to a wall: the colour gradient
// keeps its magnitude and its direction along the wall and is turned to
// the angle pi - theta from the inward wall normal (theta through the red
// fluid).  lo/hi flag the walls the cell touches on each axis; the normal
// of an edge or corner cell is the normalised sum.  A gradient with no
// component along the wall is left unchanged.
__device__ __forceinline__ void wetting_rule(const StepArgs& a, bool xlo, bool xhi,
                                             bool ylo, bool yhi, bool zlo, bool zhi,
                                             float& Gx, float& Gy, float& Gz) {
  float nx = (xlo ? 1.f : 0.f) - (xhi ? 1.f : 0.f);
  float ny = (ylo ? 1.f : 0.f) - (yhi ? 1.f : 0.f);
  float nz = (zlo ? 1.f : 0.f) - (zhi ? 1.f : 0.f);
  const float nn = nx * nx + ny * ny + nz * nz;
  if (nn == 0.f) return;
  const float in = rsqrtf(nn);
  nx *= in;
  ny *= in;
  nz *= in;
  const float gn = Gx * nx + Gy * ny + Gz * nz;
  const float tx = Gx - gn * nx, ty = Gy - gn * ny, tz = Gz - gn * nz;
  const float tt = tx * tx + ty * ty + tz * tz;
  const float g2 = Gx * Gx + Gy * Gy + Gz * Gz;
  if (tt <= 0.f || g2 <= 0.f) return;
  const float gm = sqrtf(g2), it = rsqrtf(tt);
  Gx = gm * (-a.cos_t * nx + a.sin_t * tx * it);
  Gy = gm * (-a.cos_t * ny + a.sin_t * ty * it);
  Gz = gm * (-a.cos_t * nz + a.sin_t * tz * it);
}

// ---------------------------------------------------------------------------
// Recolouring coefficients of Eq. 10-11 for one cell:
//   f_i^{R,+} = wr f*_i + seg_i,  f_i^{B,+} = wb f*_i - seg_i,
//   seg_i = beta rho_R rho_B / rho^2 cos(phi_i) sum_k rho_k phi_i^k
//         = c_shell(i) * (e_i . n),
// since sum_k rho_k phi_i^k = p/6 on the axes and p/12 on the diagonals and
// cos(phi_i) = e_i . n / |e_i| (|e_i| = 1 or sqrt 2).
// ---------------------------------------------------------------------------
struct Recolour {
  float wr, wb, nx, ny, nz, cax, cdg;
};

template <int I>
__device__ __forceinline__ float recolour_seg(const Recolour& rc) {
  if (I == 0) return 0.f;
  const float en = ex(I) * rc.nx + ey(I) * rc.ny + ez(I) * rc.nz;
  return (shell(I) == 1 ? rc.cax : rc.cdg) * en;
}

// ---------------------------------------------------------------------------
// Collision + perturbation of the total population of one cell.  On entry
// f holds the pulled f_i = f_i^R + f_i^B; on exit the post-perturbation
// f*_i (Eq. 12 summed over colours).  Returns the recolouring coefficients.
// grad = grad rho^N and Q = (d_x Qbar_x, d_y Qbar_y, d_z Qbar_z), both from
// the Eq. 49 stencil.
// ---------------------------------------------------------------------------
// BGK: the operator of Eq. 20 (Lambda = I / tau_v), a compile-time choice:
// in the MRT form the rates of rows 4 and 10-18 are launch constants, so
// their relaxation does not wait for tau_v.
template <bool BGK = false>
__device__ __forceinline__ Recolour collide_total(const StepArgs& a, float* f,
                                                  const Macro& mc, float rhoN,
                                                  float Gx, float Gy, float Gz,
                                                  float Qx, float Qy,
                                                  float Qz) {
  const float rho = mc.rho, ux = mc.ux, uy = mc.uy, uz = mc.uz;
  const float Fx = mc.Fx, Fy = mc.Fy, Fz = mc.Fz;

  // raw moments of Eq. 43, rows 4..18
  const float a12 = f[1] + f[2], a34 = f[3] + f[4], a56 = f[5] + f[6];
  const float Sxy = (f[7] + f[8]) + (f[9] + f[10]);
  const float Sxz = (f[11] + f[12]) + (f[13] + f[14]);
  const float Syz = (f[15] + f[16]) + (f[17] + f[18]);
  float m[19];
  m[4] = a12 + a34 + a56 + 2.f * (Sxy + Sxz + Syz);
  m[5] = 2.f * a12 - a34 - a56 + Sxy + Sxz - 2.f * Syz;
  m[6] = a34 - a56 + Sxy - Sxz;
  m[7] = (f[7] + f[8]) - (f[9] + f[10]);
  m[8] = (f[11] + f[12]) - (f[13] + f[14]);
  m[9] = (f[15] + f[16]) - (f[17] + f[18]);
  m[10] = (f[7] - f[8]) - (f[9] - f[10]);
  m[11] = (f[7] - f[8]) + (f[9] - f[10]);
  m[12] = (f[11] - f[12]) - (f[13] - f[14]);
  m[13] = (f[11] - f[12]) + (f[13] - f[14]);
  m[14] = (f[15] - f[16]) - (f[17] - f[18]);
  m[15] = (f[15] - f[16]) + (f[17] - f[18]);
  m[16] = Sxy;
  m[17] = Sxz;
  m[18] = Syz;

  // equilibria summed over colours; p = sum_k rho_k (c_s^k)^2
  const float p = a.cs2_R * mc.rR + a.cs2_B * mc.rB;
  const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
  const float pc = a.improved ? p : rho * (1.0f / 3.0f);
  float e[19];
  e[4] = 3.f * p + rho * (ux2 + uy2 + uz2);
  e[5] = rho * (2.f * ux2 - uy2 - uz2);
  e[6] = rho * (uy2 - uz2);
  e[7] = rho * ux * uy;
  e[8] = rho * ux * uz;
  e[9] = rho * uy * uz;
  e[10] = pc * uy;
  e[11] = pc * ux;
  e[12] = pc * uz;
  e[13] = pc * ux;
  e[14] = pc * uz;
  e[15] = pc * uy;
  const float twop = 2.f * p;
  e[16] = (twop + rho * (2.f * ux2 + 2.f * uy2 - uz2)) * (1.0f / 6.0f);
  e[17] = (twop + rho * (2.f * ux2 + 2.f * uz2 - uy2)) * (1.0f / 6.0f);
  e[18] = (twop + rho * (2.f * uy2 + 2.f * uz2 - ux2)) * (1.0f / 6.0f);

  // source in moment space: correction C (rows 4-6) + Guo force F_hat
  float src[19];
#pragma unroll
  for (int r = 4; r < 19; ++r) src[r] = 0.f;
  if (a.has_force) {
    const float Fux = Fx * ux, Fuy = Fy * uy, Fuz = Fz * uz;
    src[4] = 2.f * (Fux + Fuy + Fuz);
    src[5] = 2.f * (2.f * Fux - Fuy - Fuz);
    src[6] = 2.f * (Fuy - Fuz);
    src[7] = Fx * uy + Fy * ux;
    src[8] = Fx * uz + Fz * ux;
    src[9] = Fy * uz + Fz * uy;
    const float third = 1.0f / 3.0f;
    src[10] = Fy * third;
    src[11] = Fx * third;
    src[12] = Fz * third;
    src[13] = Fx * third;
    src[14] = Fz * third;
    src[15] = Fy * third;
    src[16] = (2.f * Fux + 2.f * Fuy - Fuz) * third;
    src[17] = (2.f * Fux + 2.f * Fuz - Fuy) * third;
    src[18] = (2.f * Fuy + 2.f * Fuz - Fux) * third;
  }
  if (a.improved) {
    src[4] += Qx + Qy + Qz;
    src[5] += 2.f * Qx - Qy - Qz;
    src[6] += Qy - Qz;
  }

  // perturbation moments (A/2)|G| pi(n), pi from M applied to Eq. 8
  const float G2 = Gx * Gx + Gy * Gy + Gz * Gz;
  const bool has_g = G2 >= 1e-24f;
  const float ig = has_g ? rsqrtf(G2) : 0.f;
  const float hA = a.half_A;
  float P4 = 0.f, P5 = 0.f, P6 = 0.f, P7 = 0.f, P8 = 0.f, P9 = 0.f, P16 = 0.f,
        P17 = 0.f, P18 = 0.f;
  if (has_g) {
    const float k29 = hA * ig * (2.0f / 9.0f);
    const float k19 = hA * ig * (1.0f / 9.0f);
    const float Gx2 = Gx * Gx, Gy2 = Gy * Gy, Gz2 = Gz * Gz;
    P4 = -(4.0f / 9.0f) * hA * (G2 * ig);
    P5 = k29 * (2.f * Gx2 - Gy2 - Gz2);
    P6 = k29 * (Gy2 - Gz2);
    P7 = k29 * Gx * Gy;
    P8 = k29 * Gx * Gz;
    P9 = k29 * Gy * Gz;
    P16 = -k19 * Gz2;
    P17 = -k19 * Gy2;
    P18 = -k19 * Gx2;
  }

  // relaxation rates (Eq. 44) with the variable tau_v of Eq. 52; the BGK
  // operator of Eq. 20 is Lambda = I / tau_v, every rate 1 / tau_v (the
  // conserved rows carry only F, whatever their rate)
  const float s_v = fast_rcp(tau_v_of(a, rhoN));
  const float s_e = BGK ? s_v : a.s_e;
  const float s_q = BGK ? s_v : a.s_q;
  const float s_pi = BGK ? s_v : a.s_pi;

  // change of moments dm = m* - m (rows 1-3: F; row 0: 0)
  float d[19];
  d[4] = -s_e * (m[4] - e[4]) + (1.f - 0.5f * s_e) * src[4] + s_e * P4;
#pragma unroll
  for (int r = 5; r <= 9; ++r)
    d[r] = -s_v * (m[r] - e[r]) + (1.f - 0.5f * s_v) * src[r];
  d[5] += s_v * P5;
  d[6] += s_v * P6;
  d[7] += s_v * P7;
  d[8] += s_v * P8;
  d[9] += s_v * P9;
#pragma unroll
  for (int r = 10; r <= 15; ++r)
    d[r] = -s_q * (m[r] - e[r]) + (1.f - 0.5f * s_q) * src[r];
#pragma unroll
  for (int r = 16; r <= 18; ++r)
    d[r] = -s_pi * (m[r] - e[r]) + (1.f - 0.5f * s_pi) * src[r];
  d[16] += s_pi * P16;
  d[17] += s_pi * P17;
  d[18] += s_pi * P18;
  d[1] = Fx;
  d[2] = Fy;
  d[3] = Fz;

  // f* = f + M^-1 dm (sparse closed form of the inverse of Eq. 43)
  const float h = 0.5f, q = 0.25f;
  const float c46 = d[4] * (1.0f / 6.0f);
  const float c5a = d[5] * (1.0f / 6.0f), c5b = d[5] * (1.0f / 12.0f);
  const float c6 = d[6] * 0.25f;
  f[0] += -d[4] + d[16] + d[17] + d[18];
  {
    const float base = c46 + c5a - h * (d[16] + d[17]);
    const float odd = h * (d[1] - d[11] - d[13]);
    f[1] += base + odd;
    f[2] += base - odd;
  }
  {
    const float base = c46 - c5b + c6 - h * (d[16] + d[18]);
    const float odd = h * (d[2] - d[10] - d[15]);
    f[3] += base + odd;
    f[4] += base - odd;
  }
  {
    const float base = c46 - c5b - c6 - h * (d[17] + d[18]);
    const float odd = h * (d[3] - d[12] - d[14]);
    f[5] += base + odd;
    f[6] += base - odd;
  }
  f[7] += q * (d[7] + d[10] + d[11] + d[16]);
  f[8] += q * (d[7] - d[10] - d[11] + d[16]);
  f[9] += q * (-d[7] - d[10] + d[11] + d[16]);
  f[10] += q * (-d[7] + d[10] - d[11] + d[16]);
  f[11] += q * (d[8] + d[12] + d[13] + d[17]);
  f[12] += q * (d[8] - d[12] - d[13] + d[17]);
  f[13] += q * (-d[8] - d[12] + d[13] + d[17]);
  f[14] += q * (-d[8] + d[12] - d[13] + d[17]);
  f[15] += q * (d[9] + d[14] + d[15] + d[18]);
  f[16] += q * (d[9] - d[14] - d[15] + d[18]);
  f[17] += q * (-d[9] - d[14] + d[15] + d[18]);
  f[18] += q * (-d[9] + d[14] - d[15] + d[18]);

  Recolour rc;
  rc.wr = mc.rR * mc.inv_rho;
  rc.wb = mc.rB * mc.inv_rho;
  rc.nx = rc.ny = rc.nz = rc.cax = rc.cdg = 0.f;
  if (has_g) {
    rc.nx = Gx * ig;
    rc.ny = Gy * ig;
    rc.nz = Gz * ig;
    const float cb = a.beta * rc.wr * rc.wb * p;
    rc.cax = cb * (1.0f / 6.0f);
    rc.cdg = cb * (1.0f / (12.0f * 1.41421356237309515f));
  }
  return rc;
}

template <int I>
struct RecolourAll {
  __device__ __forceinline__ static void run(const Recolour& rc,
                                             const float* fs, float* fR,
                                             float* fB) {
    const float sg = recolour_seg<I>(rc);
    fR[I] = rc.wr * fs[I] + sg;
    fB[I] = rc.wb * fs[I] - sg;
    RecolourAll<I + 1>::run(rc, fs, fR, fB);
  }
};
template <>
struct RecolourAll<19> {
  __device__ __forceinline__ static void run(const Recolour&, const float*,
                                             float*, float*) {}
};

// Collision + perturbation + recolouring of one cell given both colours.  On
// entry fR, fB hold the pulled populations; on exit the post-recolouring
// f^{k,+}.
template <bool BGK = false>
__device__ __forceinline__ void collide_cell(const StepArgs& a, float* fR,
                                             float* fB, const Macro& mc,
                                             float rhoN, float Gx, float Gy,
                                             float Gz, float Qx, float Qy,
                                             float Qz) {
  float f[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = fR[i] + fB[i];
  const Recolour rc = collide_total<BGK>(a, f, mc, rhoN, Gx, Gy, Gz, Qx, Qy, Qz);
  RecolourAll<0>::run(rc, f, fR, fB);
}

}  // namespace lbm
