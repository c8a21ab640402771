// lbm_step_inplace and its companions: the time step on ONE population
// array, updated in place with the AA access pattern.  Half the population
// memory of the two-buffer context (168 bytes per cell with the scratch,
// against 304), and 64-bit cell indices, so a lattice is bounded by device
// memory alone.
//
// Layout: f[(k * 19 + i) * N + cell], k = 0 red, 1 blue,
// cell = (z * ny + y) * nx + x; FP32, or FP16 / BF16 holding the deviation
// f - ref_k phi_i^k from the colour's rest state (the offsets of the
// two-buffer context; opposite directions share an offset, so the AA swap
// of slots keeps each value's offset).  A state has a parity:
//   even: slot (i, x) holds f_i(x, t), the population after streaming;
//   odd:  slot (opp(i), x) holds f_i^+(x, t - 1), the post-collision value
//         before streaming, so f_i(x, t) sits at slot (opp(i), x - e_i) or,
//         where x - e_i lies beyond a wall (halfway bounce-back), at slot
//         (i, x).
// A step from an even state reads a cell's 38 values from its own slots,
// collides and writes f_i^+(x) to slot (opp(i), x): the state turns odd and
// no value moves between cells.  A step from an odd state reads f_i(x, t)
// where the odd layout keeps it, collides and writes f_i^+(x) to slot
// (i, x + e_i) -- slot (opp(i), x) where x + e_i lies beyond a wall --
// which is where the next even state keeps f_i(x + e_i, t + 1).  In both,
// the slot written for direction i is the slot read for direction opp(i):
// every cell writes exactly the 38 slots it read, so one thread per cell
// that reads all of them before writing any races with no other thread.
//
// The colour-gradient step also needs the moments of the 18 neighbours at
// time t (the Eq. 49 stencils of rho^N and Qbar), and a neighbour's slots
// may already hold time t + 1 when a cell runs.  So each step is two
// passes: the phase field (rho^N, Qbar) of every cell into a caller-owned
// scratch of 16 bytes per cell, then the in-place collision.  Algorithmic
// traffic per cell and step: 152 B read + 16 B written, then 152 + 16 B
// read and 152 B written -- 488 B, against the 304 B of the fused
// two-buffer step.
#include <cstdint>

#include "lbm_device.cuh"
#include "lbm_equilibrium.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kInplaceBlock = 128;

struct Site {
  int x, y, z;
  long long c;
};

// Threads along x, blocks along y and z (ny, nz <= 65535).
__device__ __forceinline__ bool site_of(const StepArgs& a, Site& s) {
  s.x = blockIdx.x * blockDim.x + threadIdx.x;
  s.y = blockIdx.y;
  s.z = blockIdx.z;
  if (s.x >= a.nx) return false;
  s.c = ((long long)s.z * a.ny + s.y) * a.nx + s.x;
  return true;
}

// The cell's neighbourhood along each axis, element d + 1 for the offset
// d = -1, 0, +1: the wrapped x coordinate, the row offset y * nx and the
// plane offset z * nx * ny of the neighbour, -1 where it lies beyond a
// wall.  Computed once per thread; with the direction loops unrolled every
// neighbour index below is then two adds and three sign tests.
struct Nbr {
  int x[3];
  long long y[3], z[3];
};

__device__ __forceinline__ Nbr neighbourhood(const StepArgs& a, const Site& s) {
  Nbr n;
  const long long row = a.nx, plane = (long long)a.nx * a.ny;
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    const int xn = s.x + d, yn = s.y + d, zn = s.z + d;
    n.x[d + 1] = (xn < 0 || xn >= a.nx) ? (a.wx ? -1 : wrap1(xn, a.nx)) : xn;
    const int yw = (yn < 0 || yn >= a.ny) ? (a.wy ? -1 : wrap1(yn, a.ny)) : yn;
    const int zw = (zn < 0 || zn >= a.nz) ? (a.wz ? -1 : wrap1(zn, a.nz)) : zn;
    n.y[d + 1] = yw < 0 ? -1 : yw * row;
    n.z[d + 1] = zw < 0 ? -1 : zw * plane;
  }
  return n;
}

// Cell index of x + (dx, dy, dz), |d| <= 1, wrapped on periodic axes; -1
// where it lies beyond a wall.
__device__ __forceinline__ long long site_shift(const Nbr& n, int dx, int dy, int dz) {
  const int x = n.x[dx + 1];
  const long long y = n.y[dy + 1], z = n.z[dz + 1];
  return (x < 0 || y < 0 || z < 0) ? -1 : z + y + x;
}

// Offset, within one colour, of the slot that holds f_i(x, t) in a state of
// the given parity.
template <int ODD>
__device__ __forceinline__ long long slot_of(const Nbr& n, const Site& s, int i,
                                             long long N) {
  if (!ODD) return (long long)i * N + s.c;
  const long long src = site_shift(n, -ex(i), -ey(i), -ez(i));
  return src < 0 ? (long long)i * N + s.c : (long long)opp(i) * N + src;
}

// One stored value: FP32 as is; 16-bit as the deviation from the offset of
// population direction i (shell of i) of colour k.
__device__ __forceinline__ float ip_offset(const StepArgs& a, int k, int i) {
  const int s = shell(i);
  if (k == 0) return s == 0 ? a.offR0 : (s == 1 ? a.offR1 : a.offR2);
  return s == 0 ? a.offB0 : (s == 1 ? a.offB1 : a.offB2);
}
__device__ __forceinline__ float ip_widen(float v) { return v; }
__device__ __forceinline__ float ip_widen(__half v) { return __half2float(v); }
__device__ __forceinline__ float ip_widen(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T ip_narrow(float v);
template <>
__device__ __forceinline__ float ip_narrow<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half ip_narrow<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 ip_narrow<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <typename T>
__device__ __forceinline__ float ip_load(const T* p, const StepArgs& a, int k, int i) {
  const float v = ip_widen(*p);
  return Store<T>::kDeviation ? v + ip_offset(a, k, i) : v;
}
template <typename T>
__device__ __forceinline__ void ip_store(T* p, float v, const StepArgs& a, int k, int i) {
  *p = ip_narrow<T>(Store<T>::kDeviation ? v - ip_offset(a, k, i) : v);
}

template <int ODD, typename T>
__device__ __forceinline__ void load_site(const T* f, const StepArgs& a, const Nbr& n,
                                          const Site& s, long long N, float* fR, float* fB) {
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const long long o = slot_of<ODD>(n, s, i, N);
    fR[i] = ip_load(f + o, a, 0, i);
    fB[i] = ip_load(f + 19 * N + o, a, 1, i);
  }
}

template <typename T>
__global__ void __launch_bounds__(kInplaceBlock)
    k_inplace_init(T* __restrict__ f, StepArgs a, long long N, float alpha_R,
                   float alpha_B, const float* __restrict__ rho_R,
                   const float* __restrict__ rho_B, const float* __restrict__ u) {
  Site s;
  if (!site_of(a, s)) return;
  const float ux = u[s.c], uy = u[N + s.c], uz = u[2 * N + s.c];
  float fR[19], fB[19];
  equilibrium(rho_R[s.c], alpha_R, ux, uy, uz, a.improved, fR);
  equilibrium(rho_B[s.c], alpha_B, ux, uy, uz, a.improved, fB);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    ip_store(f + (long long)i * N + s.c, fR[i], a, 0, i);
    ip_store(f + (long long)(19 + i) * N + s.c, fB[i], a, 1, i);
  }
}

// An even state from FP32 populations f_in[(k * 19 + i) * N + cell].
template <typename T>
__global__ void __launch_bounds__(kInplaceBlock)
    k_inplace_set(T* __restrict__ f, StepArgs a, long long N, const float* __restrict__ f_in) {
  Site s;
  if (!site_of(a, s)) return;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    ip_store(f + (long long)i * N + s.c, f_in[(long long)i * N + s.c], a, 0, i);
    ip_store(f + (long long)(19 + i) * N + s.c, f_in[(long long)(19 + i) * N + s.c], a, 1, i);
  }
}

// Pass 1: (rho^N, Qbar) of every cell at time t.
template <int ODD, typename T>
__global__ void __launch_bounds__(kInplaceBlock)
    k_inplace_phase(const T* __restrict__ f, StepArgs a, long long N,
                    float4* __restrict__ phase) {
  Site s;
  if (!site_of(a, s)) return;
  const Nbr nb = neighbourhood(a, s);
  float fR[19], fB[19];
  load_site<ODD>(f, a, nb, s, N, fR, fB);
  phase[s.c] = stencil_entry(a, macro_of(a, fR, fB));
}

// Pass 2: Eq. 49 gradients from the phase field (a neighbour beyond a wall
// takes the cell's own entry), collision, perturbation and recolouring, and
// the in-place write.  f is read and written by this kernel: plain loads.
// Four blocks per SM (at most 128 registers, 16 warps; the odd form spills
// 16 bytes): 7 % faster than the 139-144 registers and 12 warps the
// compiler picks unbounded.
template <int ODD, bool BGK, typename T>
__global__ void __launch_bounds__(kInplaceBlock, 4)
    k_inplace_collide(T* f, StepArgs a, long long N, const float4* __restrict__ phase) {
  Site s;
  if (!site_of(a, s)) return;
  const Nbr nb = neighbourhood(a, s);
  float fR[19], fB[19];
  load_site<ODD>(f, a, nb, s, N, fR, fB);
  const Macro m = macro_of(a, fR, fB);
  const float4 ctr = phase[s.c];
  float Gx = 0.f, Gy = 0.f, Gz = 0.f, Qx = 0.f, Qy = 0.f, Qz = 0.f;
#pragma unroll
  for (int i = 1; i < 19; i += 2) {
    const long long np = site_shift(nb, ex(i), ey(i), ez(i));
    const long long nm = site_shift(nb, -ex(i), -ey(i), -ez(i));
    const float4 vp = np < 0 ? ctr : phase[np];
    const float4 vm = nm < 0 ? ctr : phase[nm];
    const float w = (i <= 6) ? (1.0f / 6.0f) : (1.0f / 12.0f);
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
    wetting_rule(a, a.wx && s.x == 0, a.wx && s.x == a.nx - 1, a.wy && s.y == 0,
                 a.wy && s.y == a.ny - 1, a.wz && s.z == 0, a.wz && s.z == a.nz - 1, Gx, Gy,
                 Gz);
  collide_cell<BGK>(a, fR, fB, m, ctr.x, Gx, Gy, Gz, Qx, Qy, Qz);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const long long o = slot_of<ODD>(nb, s, opp(i), N);
    ip_store(f + o, fR[i], a, 0, i);
    ip_store(f + 19 * N + o, fB[i], a, 1, i);
  }
}

// f_i(x, t) in the even layout and / or the moments (Eq. 4 with the forcing
// shift), from a state of either parity.
template <int ODD, typename T>
__global__ void __launch_bounds__(kInplaceBlock)
    k_inplace_read(const T* __restrict__ f, StepArgs a, long long N,
                   float* __restrict__ f_out, float* __restrict__ rho_R,
                   float* __restrict__ rho_B, float* __restrict__ u) {
  Site s;
  if (!site_of(a, s)) return;
  const Nbr nb = neighbourhood(a, s);
  float fR[19], fB[19];
  load_site<ODD>(f, a, nb, s, N, fR, fB);
  if (f_out) {
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      f_out[(long long)i * N + s.c] = fR[i];
      f_out[(long long)(19 + i) * N + s.c] = fB[i];
    }
  }
  if (rho_R || rho_B || u) {
    const Macro m = macro_of(a, fR, fB);
    if (rho_R) rho_R[s.c] = m.rR;
    if (rho_B) rho_B[s.c] = m.rB;
    if (u) {
      u[s.c] = m.ux;
      u[N + s.c] = m.uy;
      u[2 * N + s.c] = m.uz;
    }
  }
}

dim3 site_grid(const lbm_params* p) {
  return dim3((unsigned)((p->nx + kInplaceBlock - 1) / kInplaceBlock), (unsigned)p->ny,
              (unsigned)p->nz);
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + nb && y < x + na;
}

lbm_status check_params(const lbm_params* p, const char* no_plates_msg) {
  const lbm_status st = validate_params_any_size(p);
  if (st != LBM_OK) return st;
  if (p->wall[0] == 2 || p->wall[1] == 2 || p->wall[2] == 2)
    return fail_without_context(LBM_ERR_ARG, no_plates_msg);
  return LBM_OK;
}

size_t value_bytes(const lbm_params* p) { return p->storage == LBM_F32 ? 4 : 2; }

// The launches of one storage type (the element type of f).
template <typename T>
cudaError_t ip_init(const lbm_params* p, const StepArgs& a, long long N, void* f,
                    const float* rR, const float* rB, const float* u, cudaStream_t s) {
  k_inplace_init<T><<<site_grid(p), kInplaceBlock, 0, s>>>(
      (T*)f, a, N, (float)p->alpha_R, (float)p->alpha_B, rR, rB, u);
  return cudaGetLastError();
}
template <typename T>
cudaError_t ip_set(const lbm_params* p, const StepArgs& a, long long N, void* f,
                   const float* f_in, cudaStream_t s) {
  k_inplace_set<T><<<site_grid(p), kInplaceBlock, 0, s>>>((T*)f, a, N, f_in);
  return cudaGetLastError();
}
template <typename T>
cudaError_t ip_step(const lbm_params* p, const StepArgs& a, long long N, void* fv, int parity,
                    float4* phase, cudaStream_t s) {
  T* f = (T*)fv;
  const dim3 g = site_grid(p);
  if (parity) {
    k_inplace_phase<1, T><<<g, kInplaceBlock, 0, s>>>(f, a, N, phase);
    if (a.bgk)
      k_inplace_collide<1, true, T><<<g, kInplaceBlock, 0, s>>>(f, a, N, phase);
    else
      k_inplace_collide<1, false, T><<<g, kInplaceBlock, 0, s>>>(f, a, N, phase);
  } else {
    k_inplace_phase<0, T><<<g, kInplaceBlock, 0, s>>>(f, a, N, phase);
    if (a.bgk)
      k_inplace_collide<0, true, T><<<g, kInplaceBlock, 0, s>>>(f, a, N, phase);
    else
      k_inplace_collide<0, false, T><<<g, kInplaceBlock, 0, s>>>(f, a, N, phase);
  }
  return cudaGetLastError();
}
template <typename T>
cudaError_t ip_read(const lbm_params* p, const StepArgs& a, long long N, const void* fv,
                    int parity, float* f_out, float* rR, float* rB, float* u, cudaStream_t s) {
  const T* f = (const T*)fv;
  if (parity)
    k_inplace_read<1, T><<<site_grid(p), kInplaceBlock, 0, s>>>(f, a, N, f_out, rR, rB, u);
  else
    k_inplace_read<0, T><<<site_grid(p), kInplaceBlock, 0, s>>>(f, a, N, f_out, rR, rB, u);
  return cudaGetLastError();
}

}  // namespace
}  // namespace lbm

// The entry points dispatch on p->storage to the element type of f.
#define LBM_IP_DISPATCH(p, call)                                              \
  ((p)->storage == LBM_F16    ? call<__half>                                  \
   : (p)->storage == LBM_BF16 ? call<__nv_bfloat16>                           \
                              : call<float>)

extern "C" lbm_status lbm_inplace_init(const lbm_params* p, const float* rho_R,
                                       const float* rho_B, const float* u, void* f,
                                       void* cuda_stream) {
  lbm::NvtxRange nvtx_range_("lbm_inplace_init");
  using namespace lbm;
  clear_thread_error();
  lbm_status st =
      check_params(p, "lbm_inplace_init: moving plates (wall = 2) are not supported in place");
  if (st != LBM_OK) return st;
  if (!rho_R || !rho_B || !u || !f)
    return fail_without_context(LBM_ERR_ARG, "lbm_inplace_init: NULL array");
  if (((uintptr_t)f & (value_bytes(p) - 1)) != 0)
    return fail_without_context(LBM_ERR_ARG, "lbm_inplace_init: f misaligned for its values");
  if ((st = require_current_device(rho_R, "lbm_inplace_init: rho_R")) != LBM_OK ||
      (st = require_current_device(rho_B, "lbm_inplace_init: rho_B")) != LBM_OK ||
      (st = require_current_device(u, "lbm_inplace_init: u")) != LBM_OK ||
      (st = require_current_device(f, "lbm_inplace_init: f")) != LBM_OK)
    return st;
  const long long N = (long long)p->nx * p->ny * p->nz;
  const size_t fb = (size_t)N * 38 * value_bytes(p), nb = (size_t)N * sizeof(float);
  if (overlap(f, fb, rho_R, nb) || overlap(f, fb, rho_B, nb) || overlap(f, fb, u, 3 * nb))
    return fail_without_context(LBM_ERR_ARG, "lbm_inplace_init: f overlaps an input field");
  const StepArgs a = derive_step_args(p, N);
  if (LBM_IP_DISPATCH(p, ip_init)(p, a, N, f, rho_R, rho_B, u, (cudaStream_t)cuda_stream) !=
      cudaSuccess)
    return fail_without_context(LBM_ERR_CUDA, "lbm_inplace_init: kernel launch failed");
  return LBM_OK;
}

extern "C" lbm_status lbm_inplace_set(const lbm_params* p, const float* f_in, void* f,
                                      void* cuda_stream) {
  lbm::NvtxRange nvtx_range_("lbm_inplace_set");
  using namespace lbm;
  clear_thread_error();
  lbm_status st =
      check_params(p, "lbm_inplace_set: moving plates (wall = 2) are not supported in place");
  if (st != LBM_OK) return st;
  if (!f_in || !f) return fail_without_context(LBM_ERR_ARG, "lbm_inplace_set: NULL array");
  if (((uintptr_t)f & (value_bytes(p) - 1)) != 0)
    return fail_without_context(LBM_ERR_ARG, "lbm_inplace_set: f misaligned for its values");
  if ((st = require_current_device(f_in, "lbm_inplace_set: f_in")) != LBM_OK ||
      (st = require_current_device(f, "lbm_inplace_set: f")) != LBM_OK)
    return st;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (overlap(f, (size_t)N * 38 * value_bytes(p), f_in, (size_t)N * 38 * sizeof(float)))
    return fail_without_context(LBM_ERR_ARG, "lbm_inplace_set: f and f_in overlap");
  const StepArgs a = derive_step_args(p, N);
  if (LBM_IP_DISPATCH(p, ip_set)(p, a, N, f, f_in, (cudaStream_t)cuda_stream) != cudaSuccess)
    return fail_without_context(LBM_ERR_CUDA, "lbm_inplace_set: kernel launch failed");
  return LBM_OK;
}

extern "C" lbm_status lbm_step_inplace(const lbm_params* p, void* f, int parity, int nsteps,
                                       void* scratch, void* cuda_stream) {
  lbm::NvtxRange nvtx_range_("lbm_step_inplace");
  using namespace lbm;
  clear_thread_error();
  lbm_status st =
      check_params(p, "lbm_step_inplace: moving plates (wall = 2) are not supported in place");
  if (st != LBM_OK) return st;
  if (parity != 0 && parity != 1)
    return fail_without_context(LBM_ERR_ARG, "lbm_step_inplace: parity must be 0 or 1");
  if (nsteps < 0)
    return fail_without_context(LBM_ERR_ARG, "lbm_step_inplace: nsteps must be >= 0");
  if (!f || !scratch)
    return fail_without_context(LBM_ERR_ARG, "lbm_step_inplace: NULL array");
  if (((uintptr_t)scratch & 15u) != 0 || ((uintptr_t)f & (value_bytes(p) - 1)) != 0)
    return fail_without_context(LBM_ERR_ARG,
                                "lbm_step_inplace: scratch must be 16-byte aligned and f "
                                "aligned for its values");
  if ((st = require_current_device(f, "lbm_step_inplace: f")) != LBM_OK ||
      (st = require_current_device(scratch, "lbm_step_inplace: scratch")) != LBM_OK)
    return st;
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (overlap(f, (size_t)N * 38 * value_bytes(p), scratch, (size_t)N * sizeof(float4)))
    return fail_without_context(LBM_ERR_ARG, "lbm_step_inplace: f and scratch overlap");
  const StepArgs a = derive_step_args(p, N);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  float4* phase = (float4*)scratch;
  for (int k = 0; k < nsteps; ++k, parity ^= 1)
    if (LBM_IP_DISPATCH(p, ip_step)(p, a, N, f, parity, phase, s) != cudaSuccess)
      return fail_without_context(LBM_ERR_CUDA, "lbm_step_inplace: kernel launch failed");
  return LBM_OK;
}

extern "C" lbm_status lbm_inplace_read(const lbm_params* p, const void* f, int parity,
                                       float* f_out, float* rho_R, float* rho_B, float* u,
                                       void* cuda_stream) {
  lbm::NvtxRange nvtx_range_("lbm_inplace_read");
  using namespace lbm;
  clear_thread_error();
  lbm_status st =
      check_params(p, "lbm_inplace_read: moving plates (wall = 2) are not supported in place");
  if (st != LBM_OK) return st;
  if (parity != 0 && parity != 1)
    return fail_without_context(LBM_ERR_ARG, "lbm_inplace_read: parity must be 0 or 1");
  if (!f || (!f_out && !rho_R && !rho_B && !u))
    return fail_without_context(LBM_ERR_ARG, "lbm_inplace_read: NULL f or no output");
  if (((uintptr_t)f & (value_bytes(p) - 1)) != 0)
    return fail_without_context(LBM_ERR_ARG, "lbm_inplace_read: f misaligned for its values");
  const long long N = (long long)p->nx * p->ny * p->nz;
  const size_t fb = (size_t)N * 38 * value_bytes(p), ob = (size_t)N * 38 * sizeof(float),
               nb = (size_t)N * sizeof(float);
  const void* outs[4] = {f_out, rho_R, rho_B, u};
  const size_t sizes[4] = {ob, nb, nb, 3 * nb};
  for (int k = 0; k < 4; ++k)
    for (int l = k + 1; l < 4; ++l)
      if (outs[k] && outs[l] && overlap(outs[k], sizes[k], outs[l], sizes[l]))
        return fail_without_context(LBM_ERR_ARG, "lbm_inplace_read: two outputs overlap");
  if ((st = require_current_device(f, "lbm_inplace_read: f")) != LBM_OK) return st;
  for (int k = 0; k < 4; ++k) {
    if (!outs[k]) continue;
    if ((st = require_current_device(outs[k], "lbm_inplace_read: an output")) != LBM_OK)
      return st;
    if (overlap(f, fb, outs[k], sizes[k]))
      return fail_without_context(LBM_ERR_ARG, "lbm_inplace_read: an output overlaps f");
  }
  const StepArgs a = derive_step_args(p, N);
  if (LBM_IP_DISPATCH(p, ip_read)(p, a, N, f, parity, f_out, rho_R, rho_B, u,
                                  (cudaStream_t)cuda_stream) != cudaSuccess)
    return fail_without_context(LBM_ERR_CUDA, "lbm_inplace_read: kernel launch failed");
  return LBM_OK;
}
