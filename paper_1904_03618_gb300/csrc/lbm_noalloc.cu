// lbm_step_noalloc: one time step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: memory-budgeted or pre-allocated
// services that forbid new device allocations after start-up, and
// embedders that own every device buffer themselves.  For them this entry point runs the two-pass form of
// the step (phase-field pass, then collision) on caller-owned input and
// output population arrays, with its only scratch -- the phase field of
// rho^N and the correction fluxes, 16 bytes per cell -- in the file-scope
// device array below.  That array is part of the library's device image:
// every GPU that loads the library holds it (4 MiB) until the process
// exits.
//
// The host code never uses the array's name as a device address (on the
// host it is only a stand-in symbol); the device address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call made on
// it, and again whenever the CUDA context current on that device differs
// from the one the address was taken in (after cudaDeviceReset, or when an
// embedder makes a context of its own current, the library's device image
// is loaded again at another address).
#include <mutex>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr long long kNoAllocMaxCells = 1LL << 18;  // 262,144 cells, e.g. 64^3

// Shared by every call on a device; holds the last call's phase field.
static __device__ __align__(256) float4 g_noalloc_phase[kNoAllocMaxCells];

// Per device: the context the address was looked up in, and the address.
CUcontext g_phase_ctx[kMaxDevices];
float4* g_phase_addr[kMaxDevices];
std::mutex g_phase_mutex;

// The driver context current on this thread (the runtime makes the
// device's primary context current on its first call), through the
// runtime's driver entry point; nullptr if it cannot be read.
CUcontext current_context() {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  static GetCurrentFn get_current = nullptr;
  if (!get_current) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    get_current = (GetCurrentFn)fn;
  }
  CUcontext ctx = nullptr;
  return get_current(&ctx) == CUDA_SUCCESS ? ctx : nullptr;
}

// Phase pass: (rho^N, Qbar) of every cell from f_i^k(x, t), read in place
// (the input is the state after streaming, layout [k][i][cell]).
__global__ void k_noalloc_phase(const float* __restrict__ f, StepArgs a,
                                float4* __restrict__ phase) {
  const long long N = (long long)a.nx * a.ny * a.nz;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float fR[19], fB[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    fR[i] = __ldg(f + (long long)i * N + c);
    fB[i] = __ldg(f + (long long)(19 + i) * N + c);
  }
  const Macro m = macro_of(a, fR, fB);
  phase[c] = stencil_entry(a, m);
}

__device__ __forceinline__ long long neighbour(const StepArgs& a, int x, int y,
                                               int z, int dx, int dy, int dz,
                                               long long c) {
  const int xn = x + dx, yn = y + dy, zn = z + dz;
  if ((a.wx && (xn < 0 || xn >= a.nx)) || (a.wy && (yn < 0 || yn >= a.ny)) ||
      (a.wz && (zn < 0 || zn >= a.nz)))
    return -1;
  return ((long long)wrap1(zn, a.nz) * a.ny + wrap1(yn, a.ny)) * a.nx +
         wrap1(xn, a.nx);
}

// Collision pass: Eq. 49 gradients from the phase field, collision,
// perturbation and recolouring, then push streaming into f_out (halfway
// bounce-back where x + e_i lies beyond a wall).
template <bool BGK>
__global__ void k_noalloc_collide(const float* __restrict__ f,
                                  float* __restrict__ fout, StepArgs a,
                                  const float4* __restrict__ phase) {
  const long long N = (long long)a.nx * a.ny * a.nz;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int x = (int)(c % a.nx), y = (int)((c / a.nx) % a.ny),
            z = (int)(c / ((long long)a.nx * a.ny));
  float fR[19], fB[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    fR[i] = __ldg(f + (long long)i * N + c);
    fB[i] = __ldg(f + (long long)(19 + i) * N + c);
  }
  const Macro m = macro_of(a, fR, fB);
  const float4 ctr = __ldg(&phase[c]);
  float Gx = 0.f, Gy = 0.f, Gz = 0.f, Qx = 0.f, Qy = 0.f, Qz = 0.f;
#pragma unroll
  for (int i = 1; i < 19; i += 2) {
    const long long np = neighbour(a, x, y, z, ex(i), ey(i), ez(i), c);
    const long long nm = neighbour(a, x, y, z, -ex(i), -ey(i), -ez(i), c);
    const float4 vp = np < 0 ? ctr : __ldg(&phase[np]);
    const float4 vm = nm < 0 ? ctr : __ldg(&phase[nm]);
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
    wetting_rule(a, a.wx && x == 0, a.wx && x == a.nx - 1, a.wy && y == 0,
                 a.wy && y == a.ny - 1, a.wz && z == 0, a.wz && z == a.nz - 1, Gx, Gy, Gz);
  collide_cell<BGK>(a, fR, fB, m, ctr.x, Gx, Gy, Gz, Qx, Qy, Qz);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const long long d = neighbour(a, x, y, z, ex(i), ey(i), ez(i), c);
    const int q = d < 0 ? opp(i) : i;
    const long long cd = d < 0 ? c : d;
    fout[(long long)q * N + cd] = fR[i];
    fout[(long long)(19 + q) * N + cd] = fB[i];
  }
}

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_step_noalloc(const lbm_params* p, const float* f_in,
                                       float* f_out, void* cuda_stream) {
  using namespace lbm;
  clear_thread_error();
  lbm_status st = validate_params(p);
  if (st != LBM_OK) return st;
  if (p->wall[0] == 2 || p->wall[1] == 2 || p->wall[2] == 2)
    return fail_without_context(LBM_ERR_ARG,
                                "lbm_step_noalloc: moving plates (wall = 2) are not supported");
  const long long N = (long long)p->nx * p->ny * p->nz;
  if (N > kNoAllocMaxCells)
    return fail_without_context(
        LBM_ERR_ARG,
        "lbm_step_noalloc: nx*ny*nz exceeds its fixed scratch of 262144 cells "
        "(4 MiB); use lbm_create/lbm_step for larger lattices");
  if (!f_in || !f_out)
    return fail_without_context(LBM_ERR_ARG, "lbm_step_noalloc: NULL population array");
  const size_t bytes = (size_t)N * 38 * sizeof(float);
  const char* a0 = (const char*)f_in;
  const char* b0 = (const char*)f_out;
  if (a0 < b0 + bytes && b0 < a0 + bytes)
    return fail_without_context(LBM_ERR_ARG, "lbm_step_noalloc: f_in and f_out overlap");
  if ((st = require_current_device(f_in, "lbm_step_noalloc: f_in")) != LBM_OK ||
      (st = require_current_device(f_out, "lbm_step_noalloc: f_out")) != LBM_OK)
    return st;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail_without_context(LBM_ERR_CUDA, "lbm_step_noalloc: no usable current device");
  float4* phase = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_phase_mutex);
    const CUcontext ctx = current_context();
    if (!g_phase_addr[dev] || !ctx || ctx != g_phase_ctx[dev]) {
      // with this device and this context current
      float4* ptr = nullptr;
      e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_phase);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        g_phase_addr[dev] = nullptr;
        return fail_without_context(LBM_ERR_CUDA,
                                    "lbm_step_noalloc: cudaGetSymbolAddress of the scratch failed");
      }
      g_phase_addr[dev] = ptr;
      // the lookup has made the device's context current if none was
      g_phase_ctx[dev] = current_context();
    }
    phase = g_phase_addr[dev];
  }
  lbm_params q = *p;
  q.storage = LBM_F32;
  const StepArgs a = derive_step_args(&q, N);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const unsigned blocks = (unsigned)((N + 127) / 128);
  k_noalloc_phase<<<blocks, 128, 0, s>>>(f_in, a, phase);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    if (a.bgk)
      k_noalloc_collide<true><<<blocks, 128, 0, s>>>(f_in, f_out, a, phase);
    else
      k_noalloc_collide<false><<<blocks, 128, 0, s>>>(f_in, f_out, a, phase);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return fail_without_context(LBM_ERR_CUDA, "lbm_step_noalloc: kernel launch failed");
  return LBM_OK;
}
