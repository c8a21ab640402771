// Auxiliary kernels (initialisation, state access, moments, FP64
// diagnostics) and the two-pass form of the step, for sm_103a.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Scatter of a full state f_i^k(x, t) into the pull-streaming buffer: the
// value f_i(x) is stored where the next pull looks for it, i.e. at
// x - e_i (wrapped), or, when x - e_i lies beyond a wall, at x in direction
// opp(i) (halfway bounce-back).  The map is one-to-one.
// ---------------------------------------------------------------------------
template <typename T, int I>
__device__ __forceinline__ void scatter_one(T* __restrict__ dst,
                                            const StepArgs& a, int x, int y,
                                            int z, long long c, float vr,
                                            float vb) {
  int xs = x - ex(I), ys = y - ey(I), zs = z - ez(I);
  bool out = (a.wx && (xs < 0 || xs >= a.nx)) ||
             (a.wy && (ys < 0 || ys >= a.ny)) ||
             (a.wz && (zs < 0 || zs >= a.nz));
  long long cs;
  int d;
  if (out) {
    cs = c;
    d = opp(I);
  } else {
    cs = cell_of(a, wrap1(xs, a.nx), wrap1(ys, a.ny), wrap1(zs, a.nz));
    d = I;
  }
  if (Store<T>::kDeviation) {
    vr -= dev_offset<I>(a, 0);
    vb -= dev_offset<I>(a, 1);
  }
  Store<T>::store2(dst + pidx2(a, d, cs), vr, vb);
}

template <typename T, int I>
struct ScatterAll {
  __device__ __forceinline__ static void run(T* __restrict__ dst,
                                             const StepArgs& a, int x, int y,
                                             int z, long long c,
                                             const float* fR,
                                             const float* fB) {
    scatter_one<T, I>(dst, a, x, y, z, c, fR[I], fB[I]);
    ScatterAll<T, I + 1>::run(dst, a, x, y, z, c, fR, fB);
  }
};
template <typename T>
struct ScatterAll<T, 19> {
  __device__ __forceinline__ static void run(T* __restrict__,
                                             const StepArgs&, int, int, int,
                                             long long, const float*,
                                             const float*) {}
};

// Equilibrium of one colour: Eq. 18 with the high-order term coefficient 3
// (improved) or Eq. 6 (original).  phi_i^k of Eq. 13, c = 1.
__device__ __forceinline__ void equilibrium(float rho, float alpha, float ux,
                                            float uy, float uz, int improved,
                                            float* fe) {
  const float cs2 = 0.5f * (1.f - alpha);
  const float uu = ux * ux + uy * uy + uz * uz;
  const float ph[3] = {alpha, (1.f - alpha) * (1.0f / 12.0f),
                       (1.f - alpha) * (1.0f / 24.0f)};
  const float w[3] = {1.0f / 3.0f, 1.0f / 18.0f, 1.0f / 36.0f};
  const float hk = improved ? 3.f * (3.f * cs2 - 1.f) : 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const float eu = ex(i) * ux + ey(i) * uy + ez(i) * uz;
    const int s = shell(i);
    const float ee = (float)s;  // |e|^2 = 0, 1, 2
    float br = 3.f * eu + 4.5f * eu * eu - 1.5f * uu + hk * eu * (3.f * ee - 5.f);
    fe[i] = rho * (ph[s] + w[s] * br);
  }
}

__device__ __forceinline__ bool cell_coords(const StepArgs& a, long long c,
                                            int& x, int& y, int& z) {
  long long N = (long long)a.nx * a.ny * a.nz;
  if (c >= N) return false;
  x = (int)(c % a.nx);
  long long r = c / a.nx;
  y = (int)(r % a.ny);
  z = (int)(r / a.ny);
  return true;
}

template <typename T>
__global__ void k_init_eq(T* __restrict__ dst, StepArgs a, float alpha_R,
                          float alpha_B, const float* __restrict__ rho_R,
                          const float* __restrict__ rho_B,
                          const float* __restrict__ u) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!cell_coords(a, c, x, y, z)) return;
  long long N = (long long)a.nx * a.ny * a.nz;
  float ux = u[c], uy = u[N + c], uz = u[2 * N + c];
  float fR[19], fB[19];
  equilibrium(rho_R[c], alpha_R, ux, uy, uz, a.improved, fR);
  equilibrium(rho_B[c], alpha_B, ux, uy, uz, a.improved, fB);
  ScatterAll<T, 0>::run(dst, a, x, y, z, c, fR, fB);
}

template <typename T>
__global__ void k_set_f(T* __restrict__ dst, StepArgs a,
                        const float* __restrict__ f) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!cell_coords(a, c, x, y, z)) return;
  long long N = (long long)a.nx * a.ny * a.nz;
  float fR[19], fB[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    fR[i] = f[(long long)i * N + c];
    fB[i] = f[(long long)(19 + i) * N + c];
  }
  ScatterAll<T, 0>::run(dst, a, x, y, z, c, fR, fB);
}

template <typename T>
__global__ void k_get_f(const T* __restrict__ src, StepArgs a,
                        float* __restrict__ f) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!cell_coords(a, c, x, y, z)) return;
  long long N = (long long)a.nx * a.ny * a.nz;
  float fR[19], fB[19];
  pull_cell<T>(src, a, x, y, z, fR, fB);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    f[(long long)i * N + c] = fR[i];
    f[(long long)(19 + i) * N + c] = fB[i];
  }
}

template <typename T>
__global__ void k_moments(const T* __restrict__ src, StepArgs a,
                          float* __restrict__ rho_R, float* __restrict__ rho_B,
                          float* __restrict__ u) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int x, y, z;
  if (!cell_coords(a, c, x, y, z)) return;
  long long N = (long long)a.nx * a.ny * a.nz;
  float fR[19], fB[19];
  pull_cell<T>(src, a, x, y, z, fR, fB);
  Macro m = macro_of(a, fR, fB);
  if (rho_R) rho_R[c] = m.rR;
  if (rho_B) rho_B[c] = m.rB;
  if (u) {
    u[c] = m.ux;
    u[N + c] = m.uy;
    u[2 * N + c] = m.uz;
  }
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: per-block partial sums (warp shuffles, then shared
// memory) into a scratch array, then one block folds the partials in a
// fixed order, so the result is deterministic.
// ---------------------------------------------------------------------------
constexpr int kDiagBlock = 256;

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

template <typename T>
__global__ void __launch_bounds__(kDiagBlock)
    k_diag_partial(const T* __restrict__ src, StepArgs a,
                   double* __restrict__ part) {
  double acc[kDiagSlots];
#pragma unroll
  for (int s = 0; s < kDiagSlots; ++s) acc[s] = 0.0;
  long long N = (long long)a.nx * a.ny * a.nz;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_coords(a, c, x, y, z);
    float fR[19], fB[19];
    pull_cell<T>(src, a, x, y, z, fR, fB);
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 19; ++i)
      finite = finite && isfinite(fR[i]) && isfinite(fB[i]);
    Macro m = macro_of(a, fR, fB);
    double rR = 0, rB = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      rR += (double)fR[i];
      rB += (double)fB[i];
      double fi = (double)fR[i] + (double)fB[i];
      jx += ex(i) * fi;
      jy += ey(i) * fi;
      jz += ez(i) * fi;
    }
    acc[0] += rR;
    acc[1] += rB;
    acc[2] += jx;
    acc[3] += jy;
    acc[4] += jz;
    acc[5] += finite ? 0.0 : 1.0;
    acc[6] += (m.rR < 0.f || m.rB < 0.f) ? 1.0 : 0.0;
    double um = sqrt((double)m.ux * m.ux + (double)m.uy * m.uy +
                     (double)m.uz * m.uz);
    if (finite && um > acc[7]) acc[7] = um;
    acc[8] += phase_field(a, m.rR, m.rB) > 0.f ? 1.0 : 0.0;
    acc[9] += rR * x;
    acc[10] += rR * y;
    acc[11] += rR * z;
  }
  __shared__ double sh[kDiagBlock / 32][kDiagSlots];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < kDiagSlots; ++s) {
    double v = (s == 7) ? warp_max(acc[s]) : warp_sum(acc[s]);
    if (lane == 0) sh[wid][s] = v;
  }
  __syncthreads();
  if (threadIdx.x < kDiagSlots) {
    int s = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < kDiagBlock / 32; ++w)
      v = (s == 7) ? fmax(v, sh[w][s]) : v + sh[w][s];
    part[(long long)blockIdx.x * kDiagSlots + s] = v;
  }
}

__global__ void k_diag_final(const double* __restrict__ part, int nblocks,
                             double* __restrict__ out) {
  int s = threadIdx.x;
  if (s >= kDiagSlots) return;
  double v = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    double p = part[(long long)b * kDiagSlots + s];
    v = (s == 7) ? fmax(v, p) : v + p;
  }
  out[s] = v;
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
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  float fR[19], fB[19];
  pull_cell<T>(src, a, x, y, z, fR, fB);
  Macro m = macro_of(a, fR, fB);
  float q = qbar_scale(a, m.rR, m.rB);
  mom[cell_of(a, x, y, z)] =
      make_float4(phase_field(a, m.rR, m.rB), m.ux * q, m.uy * q, m.uz * q);
}

// Neighbour x + e of the Eq. 49 stencil; beyond a wall the centre cell.
__device__ __forceinline__ long long stencil_cell(const StepArgs& a, int x,
                                                  int y, int z, int dx, int dy,
                                                  int dz, long long c) {
  int xn = x + dx, yn = y + dy, zn = z + dz;
  if ((a.wx && (xn < 0 || xn >= a.nx)) || (a.wy && (yn < 0 || yn >= a.ny)) ||
      (a.wz && (zn < 0 || zn >= a.nz)))
    return c;
  return cell_of(a, wrap1(xn, a.nx), wrap1(yn, a.ny), wrap1(zn, a.nz));
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_twopass_collide(const T* __restrict__ src, T* __restrict__ dst,
                      StepArgs a, const float4* __restrict__ mom) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  int z = blockIdx.z;
  if (x >= a.nx || y >= a.ny) return;
  long long c = cell_of(a, x, y, z);
  float fR[19], fB[19];
  pull_cell<T>(src, a, x, y, z, fR, fB);
  Macro m = macro_of(a, fR, fB);
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
  float rn = __ldg(&mom[c]).x;
  collide_cell(a, fR, fB, m, rn, Gx, Gy, Gz, Qx, Qy, Qz);
  store_cell<T>(dst, a, c, fR, fB);
}

// ---------------------------------------------------------------------------
// Launchers (host side).
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int b) {
  return (unsigned)((n + b - 1) / b);
}

template <typename T>
cudaError_t launch_init_eq_t(void* dst, const StepArgs& a, float alpha_R,
                             float alpha_B, const float* rR, const float* rB,
                             const float* u, cudaStream_t s) {
  long long N = (long long)a.nx * a.ny * a.nz;
  k_init_eq<T><<<blocks_for(N, 128), 128, 0, s>>>((T*)dst, a, alpha_R, alpha_B,
                                                   rR, rB, u);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_set_f_t(void* dst, const StepArgs& a, const float* f,
                           cudaStream_t s) {
  long long N = (long long)a.nx * a.ny * a.nz;
  k_set_f<T><<<blocks_for(N, 128), 128, 0, s>>>((T*)dst, a, f);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_get_f_t(const void* src, const StepArgs& a, float* f,
                           cudaStream_t s) {
  long long N = (long long)a.nx * a.ny * a.nz;
  k_get_f<T><<<blocks_for(N, 128), 128, 0, s>>>((const T*)src, a, f);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_moments_t(const void* src, const StepArgs& a, float* rR,
                             float* rB, float* u, cudaStream_t s) {
  long long N = (long long)a.nx * a.ny * a.nz;
  k_moments<T><<<blocks_for(N, 128), 128, 0, s>>>((const T*)src, a, rR, rB, u);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_diag_t(const void* src, const StepArgs& a, double* part,
                          int nblocks, double* out, cudaStream_t s) {
  k_diag_partial<T><<<nblocks, kDiagBlock, 0, s>>>((const T*)src, a, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_diag_final<<<1, 32, 0, s>>>(part, nblocks, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_twopass_t(const void* src, void* dst, const StepArgs& a,
                             float4* mom, cudaStream_t s) {
  dim3 blk(32, 8);
  dim3 grd((a.nx + 31) / 32, (a.ny + 7) / 8, a.nz);
  k_twopass_phase<T><<<grd, blk, 0, s>>>((const T*)src, a, mom);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_twopass_collide<T><<<grd, blk, 0, s>>>((const T*)src, (T*)dst, a, mom);
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
cudaError_t launch_diag(int storage, const void* src, const StepArgs& a,
                        double* part, int nblocks, double* out,
                        cudaStream_t s) {
  LBM_DISPATCH(storage, launch_diag_t, src, a, part, nblocks, out, s)
}
cudaError_t launch_twopass(int storage, const void* src, void* dst,
                           const StepArgs& a, float4* mom, cudaStream_t s) {
  LBM_DISPATCH(storage, launch_twopass_t, src, dst, a, mom, s)
}

}  // namespace lbm
