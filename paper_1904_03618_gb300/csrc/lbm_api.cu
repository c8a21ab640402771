// C ABI of the library (declared in include/lbm.h): parameter validation,
// device memory, stream ordering, host/device pointer handling and error
// reporting around the kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using lbm::StepArgs;

// One lattice of a context.  A single-lattice context has one case.
struct CaseRec {
  lbm_params p;
  StepArgs args;        // args.plane = the case's padded cell count
  long long N;          // cells
  long long pair_base;  // offset of the case within each buffer, in pairs
  int initialized;
};

struct lbm_ctx {
  CaseRec* cases;
  int ncases;
  int storage, kernel;
  lbm::FusedConfig fused;
  cudaStream_t stream;
  int device, sms;
  size_t elem;              // bytes per stored population value
  long long total_pairs;    // pairs per buffer over all cases
  long long max_cells;      // largest case
  bool any_walls;
  void* pop[2];             // ping-pong population buffers
  int cur;                  // buffer holding the current state (pull layout)
  float4* phase;            // two-pass scratch: (rho^N, Qbar) per cell
  double* diag_part;        // per-block partial sums of the diagnostics
  double* diag_out;         // folded sums and the error word (device)
  unsigned* diag_done;      // block counter of the diagnostics kernel
  double* diag_host;        // pinned host copy of diag_out
  // lbm_step_diagnostics_async runs the diagnostics on a stream of their own
  // (created on first use), so that they overlap the next step, which only
  // reads the buffer they read; a launch that writes a buffer first waits
  // for the last diagnostics that read it (diag_ev[b], pending diag_pend[b]).
  cudaStream_t dstream;
  cudaEvent_t step_ev, diag_ev[2];
  bool diag_pend[2];
  int diag_blocks;
  float* staging;           // device staging for host-pointer transfers
  size_t staging_floats;
  lbm::BatchCase* d_cases;  // device case table of the batched kernel
  unsigned long long* foot; // per-case plane counts (lbm_batch_footprint)
  int* d_flags;             // device error word of the kernels' bounded waits
  unsigned* d_oob;          // checked builds: out-of-range index count
  lbm::MonAcc* d_mon;       // monitored steps: the step's diagnostics record
  double* d_mon_out;        // its 16 slots
  bool tma_ok[3];           // tensor maps built, per tile kind (single lattice)
  CUtensorMap tmaps[2][3][2];  // [buffer][tile kind][map]: TMA maps
  CUtensorMap smaps[2][2][6];  // [tile: 0 = 34 x 15, 1 = 34 x 12][buffer][map]: SEAM forms
  bool seam_ok;                // smaps built (FP32, periodic in x and y)
  CUtensorMap smaps16[2][2][4];  // [tile: 0 = 34 x 15, 1 = 34 x 12][buffer][map]: 16-bit SEAM
  bool seam16_ok;                // smaps16 built (FP16 / BF16, periodic in x and y)
  CUtensorMap* d_bmaps[2][3];  // batches: [buffer][tile kind] -> device table, 2 per case
  bool batch_tma_ok[3];        // batch tables built, per tile kind
  CUtensorMap* d_seam_bmaps[2];  // batches: [buffer] -> six seam maps (tile_y 12) per case
  bool batch_seam_ok;            // every case runs the batched SEAM form
  int total_items;
  int plate_axis;           // axis of the moving plates (wall = 2), or -1
  double plate_u[2][3];     // their velocities (low, high)
  cudaGraphExec_t graph;    // two captured steps (buffer 0 -> 1 -> 0)
  int use_graph;
  long long steps;
  char err[512];
};

static thread_local char g_create_err[512];

static lbm_status fail(lbm_ctx* c, lbm_status s, const char* fmt, ...) {
  char* dst = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return s;
}

static lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
  return fail(c, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LBM_CUDA(ctx, call, what)                       \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

// Allocation layer: every device and pinned-host allocation of the library
// goes through these, so that the live count is known and a test can make
// the n-th next allocation fail (as cudaMalloc does when memory runs out).
static std::atomic<long long> g_live_allocs{0};
static std::atomic<int> g_fail_countdown{0};

static bool injected_failure() {
  int n = g_fail_countdown.load();
  while (n > 0) {
    if (g_fail_countdown.compare_exchange_weak(n, n - 1)) return n == 1;
  }
  return false;
}

namespace lbm {
cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) ++g_live_allocs;
  return e;
}
void dev_free(void* p) {
  if (!p) return;
  cudaFree(p);
  --g_live_allocs;
}
cudaError_t host_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMallocHost(p, bytes);
  if (e == cudaSuccess) ++g_live_allocs;
  return e;
}
void host_free(void* p) {
  if (!p) return;
  cudaFreeHost(p);
  --g_live_allocs;
}
}  // namespace lbm

extern "C" void lbm_test_fail_allocation(int n) { g_fail_countdown.store(n > 0 ? n : 0); }
extern "C" long long lbm_test_live_allocations(void) { return g_live_allocs.load(); }

extern "C" lbm_status lbm_test_index_checks(lbm_ctx* c, int* checked, unsigned* out_of_range) {
  if (!c || !checked || !out_of_range) return c ? fail(c, LBM_ERR_ARG, "NULL output") : LBM_ERR_ARG;
#ifdef LBM_CHECKED
  *checked = 1;
  LBM_CUDA(c, cudaMemcpyAsync(out_of_range, c->d_oob, sizeof(unsigned), cudaMemcpyDeviceToHost,
                              c->stream),
           "cudaMemcpyAsync");
  LBM_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
#else
  *checked = 0;
  *out_of_range = 0;
#endif
  return LBM_OK;
}

extern "C" lbm_status lbm_test_set_wait_limits(unsigned long long stage_ns,
                                               unsigned long long mma_ns) {
  cudaError_t e = lbm::tma_set_wait_ns<float>(stage_ns);
  if (e == cudaSuccess) e = lbm::tma_set_wait_ns<__half>(stage_ns);
  if (e == cudaSuccess) e = lbm::tma_set_wait_ns<__nv_bfloat16>(stage_ns);
  if (e == cudaSuccess) e = lbm::mlp_set_wait_ns(mma_ns);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

// Where a caller's pointer lives, seen from the GPU the work runs on.
// Device memory of another GPU is refused by every entry point that hands
// caller pointers to a kernel: without peer access the kernel would fault.
enum PtrWhere { kPtrHost = 0, kPtrHere = 1, kPtrOtherDevice = 2 };

// Test hook (lbm_test_fake_pointer_attributes): a fixed answer in place of
// cudaPointerGetAttributes and cudaGetDevice, so that the checks can be
// exercised on machines with one GPU or none.
static std::atomic<int> g_fake_on{0};
static std::atomic<int> g_fake_type{0}, g_fake_device{0}, g_fake_current{0};

// The device the context-free entry points run on (the current one).
static int current_device() {
  if (g_fake_on.load()) return g_fake_current.load();
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return d;
}

static PtrWhere pointer_where(const void* ptr, int run_device, int* owner) {
  int type, device;
  if (g_fake_on.load()) {
    type = g_fake_type.load();
    device = g_fake_device.load();
  } else {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
      cudaGetLastError();
      return kPtrHost;
    }
    type = at.type;
    device = at.device;
  }
  *owner = device;
  if (type == cudaMemoryTypeManaged) return kPtrHere;
  if (type != cudaMemoryTypeDevice) return kPtrHost;
  return device == run_device ? kPtrHere : kPtrOtherDevice;
}

// Context API: *device = the pointer may be read or written by the
// context's kernels; host memory is staged; another GPU's memory fails.
static lbm_status caller_memory(lbm_ctx* c, const void* ptr, const char* what,
                                bool* device);

// Every check but the 32-bit pair-offset limit of the two-buffer kernels.
static lbm_status validate_any_size(const lbm_params* p) {
  if (!p) return fail(nullptr, LBM_ERR_ARG, "params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1)
    return fail(nullptr, LBM_ERR_ARG, "nx, ny, nz must be >= 1");
  if (p->ny > 65535 || p->nz > 65535)
    return fail(nullptr, LBM_ERR_ARG, "ny and nz must be <= 65535");
  for (int a = 0; a < 3; ++a)
    if (p->wall[a] < 0 || p->wall[a] > 2)
      return fail(nullptr, LBM_ERR_ARG, "wall[%d] must be 0, 1 or 2", a);
  for (int a = 0; a < 3; ++a) {
    if (p->wall[a] != 2) continue;
    const int n[3] = {p->nx, p->ny, p->nz};
    if (p->wall[(a + 1) % 3] != 0 || p->wall[(a + 2) % 3] != 0)
      return fail(nullptr, LBM_ERR_ARG,
                  "moving plates (wall[%d] = 2) need the other two axes periodic", a);
    if (n[a] < 3)
      return fail(nullptr, LBM_ERR_ARG, "moving plates need at least 3 layers between them");
    for (int side = 0; side < 2; ++side)
      for (int d = 0; d < 3; ++d)
        if (!(fabs(p->wall_u[side][d]) < 0.5))
          return fail(nullptr, LBM_ERR_ARG, "wall_u components must be finite and below 0.5");
  }
  if (p->improved != 0 && p->improved != 1)
    return fail(nullptr, LBM_ERR_ARG, "improved must be 0 or 1");
  if (p->storage < LBM_F32 || p->storage > LBM_BF16)
    return fail(nullptr, LBM_ERR_ARG, "storage must be LBM_F32, LBM_F16 or LBM_BF16");
  if (p->kernel != LBM_KERNEL_FUSED && p->kernel != LBM_KERNEL_TWO_PASS)
    return fail(nullptr, LBM_ERR_ARG, "kernel must be LBM_KERNEL_FUSED or LBM_KERNEL_TWO_PASS");
  if (p->wetting != 0 && p->wetting != 1)
    return fail(nullptr, LBM_ERR_ARG, "wetting must be 0 or 1");
  if (p->collision != LBM_COLLISION_MRT && p->collision != LBM_COLLISION_BGK)
    return fail(nullptr, LBM_ERR_ARG, "collision must be LBM_COLLISION_MRT or LBM_COLLISION_BGK");
  if (p->wetting && !(p->contact_angle_deg > 0 && p->contact_angle_deg < 180))
    return fail(nullptr, LBM_ERR_ARG, "contact_angle_deg must lie in (0, 180)");
  if (!(p->rho_in_R > 0) || !(p->rho_in_B > 0))
    return fail(nullptr, LBM_ERR_ARG, "rho_in_R and rho_in_B must be > 0");
  if (!(p->alpha_R >= 0 && p->alpha_R < 1) || !(p->alpha_B >= 0 && p->alpha_B < 1))
    return fail(nullptr, LBM_ERR_ARG, "alpha_R and alpha_B must lie in [0, 1)");
  const double taus[5] = {p->tau_R, p->tau_B, p->tau_e, p->tau_q, p->tau_pi};
  const char* names[5] = {"tau_R", "tau_B", "tau_e", "tau_q", "tau_pi"};
  for (int i = 0; i < 5; ++i)
    if (!(taus[i] > 0.5) || !isfinite(taus[i]))
      return fail(nullptr, LBM_ERR_ARG, "%s must be finite and > 1/2", names[i]);
  if (!(p->A_R >= 0) || !(p->A_B >= 0) || !isfinite(p->A_R) || !isfinite(p->A_B))
    return fail(nullptr, LBM_ERR_ARG, "A_R and A_B must be finite and >= 0");
  if (!(p->beta >= 0 && p->beta <= 1))
    return fail(nullptr, LBM_ERR_ARG, "beta must lie in [0, 1]");
  if (!(p->delta > 0 && p->delta <= 1))
    return fail(nullptr, LBM_ERR_ARG, "delta must lie in (0, 1]");
  for (int a = 0; a < 3; ++a)
    if (!isfinite(p->force[a]) || !isfinite(p->gravity[a]))
      return fail(nullptr, LBM_ERR_ARG, "force and gravity must be finite");
  if (!isfinite(p->ref_R) || !isfinite(p->ref_B))
    return fail(nullptr, LBM_ERR_ARG, "ref_R and ref_B must be finite");
  return LBM_OK;
}

static lbm_status validate(const lbm_params* p) {
  const lbm_status st = validate_any_size(p);
  if (st != LBM_OK) return st;
  long long N = (long long)p->nx * p->ny * p->nz;
  // pair offsets (direction * padded plane + cell) are 32-bit
  if ((N + 64) * 19 >= (1LL << 32))
    return fail(nullptr, LBM_ERR_ARG, "lattice too large: nx*ny*nz must be below 226,000,000");
  return LBM_OK;
}

static StepArgs derive_args(const lbm_params* p, long long plane) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.wx = p->wall[0];
  a.wy = p->wall[1];
  a.wz = p->wall[2];
  a.plane = plane;
  a.improved = p->improved;
  a.bgk = p->collision == LBM_COLLISION_BGK ? 1 : 0;
  a.inv_rin_R = (float)(1.0 / p->rho_in_R);
  a.inv_rin_B = (float)(1.0 / p->rho_in_B);
  double csR = 0.5 * (1.0 - p->alpha_R), csB = 0.5 * (1.0 - p->alpha_B);
  a.cs2_R = (float)csR;
  a.cs2_B = (float)csB;
  a.q_R = (float)(1.0 - 3.0 * csR);
  a.q_B = (float)(1.0 - 3.0 * csB);
  a.tau_R = (float)p->tau_R;
  a.tau_B = (float)p->tau_B;
  double th = 2.0 * p->tau_R * p->tau_B / (p->tau_R + p->tau_B);
  a.tau_h = (float)th;
  a.par_a = (float)(2.0 * (p->tau_R - th) / p->delta);
  a.par_b = (float)(2.0 * (th - p->tau_B) / p->delta);
  a.par_a2 = (float)(2.0 * (p->tau_R - th) / p->delta / (2.0 * p->delta));
  a.par_b2 = (float)(2.0 * (th - p->tau_B) / p->delta / (2.0 * p->delta));
  a.delta = (float)p->delta;
  a.s_e = (float)(1.0 / p->tau_e);
  a.s_q = (float)(1.0 / p->tau_q);
  a.s_pi = (float)(1.0 / p->tau_pi);
  a.half_A = (float)(0.5 * (p->A_R + p->A_B));
  a.beta = (float)p->beta;
  a.fx = (float)p->force[0];
  a.fy = (float)p->force[1];
  a.fz = (float)p->force[2];
  a.gx = (float)p->gravity[0];
  a.gy = (float)p->gravity[1];
  a.gz = (float)p->gravity[2];
  a.wetting = p->wetting && (p->wall[0] || p->wall[1] || p->wall[2]);
  const double th_rad = p->contact_angle_deg * 3.14159265358979323846 / 180.0;
  a.cos_t = (float)cos(th_rad);
  a.sin_t = (float)sin(th_rad);
  a.has_force = (p->force[0] != 0 || p->force[1] != 0 || p->force[2] != 0 ||
                 p->gravity[0] != 0 || p->gravity[1] != 0 || p->gravity[2] != 0);
  if (p->storage != LBM_F32) {
    a.offR0 = (float)(p->ref_R * p->alpha_R);
    a.offR1 = (float)(p->ref_R * (1.0 - p->alpha_R) / 12.0);
    a.offR2 = (float)(p->ref_R * (1.0 - p->alpha_R) / 24.0);
    a.offB0 = (float)(p->ref_B * p->alpha_B);
    a.offB1 = (float)(p->ref_B * (1.0 - p->alpha_B) / 12.0);
    a.offB2 = (float)(p->ref_B * (1.0 - p->alpha_B) / 24.0);
  }
  return a;
}

// Shared with the other host translation units (declared in lbm_internal.h).
namespace lbm {
lbm_status validate_params(const lbm_params* p) { return validate(p); }
lbm_status validate_params_any_size(const lbm_params* p) { return validate_any_size(p); }
StepArgs derive_step_args(const lbm_params* p, long long plane) {
  return derive_args(p, plane);
}
lbm_status fail_without_context(lbm_status s, const char* msg) {
  return fail(nullptr, s, "%s", msg);
}
lbm_status require_current_device(const void* ptr, const char* what) {
  const int cur = current_device();
  int owner = -1;
  switch (pointer_where(ptr, cur, &owner)) {
    case kPtrHere:
      return LBM_OK;
    case kPtrOtherDevice:
      return fail(nullptr, LBM_ERR_ARG,
                  "%s is device memory of GPU %d, but GPU %d is current: make the GPU that "
                  "owns the arrays current before the call",
                  what, owner, cur);
    default:
      return fail(nullptr, LBM_ERR_ARG, "%s must be device memory", what);
  }
}
void clear_thread_error() { g_create_err[0] = 0; }
}  // namespace lbm

static void release(lbm_ctx* c) {
  if (!c) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (c->device >= 0) cudaSetDevice(c->device);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  lbm::dev_free(c->pop[0]);
  lbm::dev_free(c->pop[1]);
  lbm::dev_free(c->phase);
  lbm::dev_free(c->diag_part);
  lbm::dev_free(c->diag_out);
  lbm::dev_free(c->diag_done);
  lbm::host_free(c->diag_host);
  lbm::dev_free(c->staging);
  lbm::dev_free(c->d_cases);
  lbm::dev_free(c->foot);
  lbm::dev_free(c->d_flags);
  lbm::dev_free(c->d_oob);
  lbm::dev_free(c->d_mon);
  lbm::dev_free(c->d_mon_out);
  for (int b = 0; b < 2; ++b)
    for (int w = 0; w < 3; ++w) lbm::dev_free(c->d_bmaps[b][w]);
  for (int b = 0; b < 2; ++b) lbm::dev_free(c->d_seam_bmaps[b]);
  delete[] c->cases;
  if (prev >= 0) cudaSetDevice(prev);
}

static void drop_graph(lbm_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
}

// Rebuilds the batched kernel's device case table for the current fused
// configuration (tile counts and item numbering depend on it).
static lbm_status upload_case_table(lbm_ctx* c) {
  if (c->ncases <= 1) return LBM_OK;
  lbm::BatchCase* h = new (std::nothrow) lbm::BatchCase[c->ncases];
  if (!h) return fail(c, LBM_ERR_OOM, "host allocation failed");
  const int ty = c->fused.tile_y, zc = c->fused.zchunk;
  long long items = 0;
  for (int k = 0; k < c->ncases; ++k) {
    const CaseRec& r = c->cases[k];
    h[k].args = r.args;
    h[k].pair_base = r.pair_base;
    h[k].item_start = (int)items;
    const int iw = lbm::tile_interior_x(ty);
    h[k].tiles_x = (r.p.nx + iw - 1) / iw;
    h[k].tiles_y = (r.p.ny + ty - 3) / (ty - 2);
    h[k].pad_ = 0;
    items += (long long)h[k].tiles_x * h[k].tiles_y * ((r.p.nz + zc - 1) / zc);
  }
  if (items >= (1LL << 31)) {
    delete[] h;
    return fail(c, LBM_ERR_ARG, "batch too large: more than 2^31 work items");
  }
  cudaError_t e = cudaMemcpyAsync(c->d_cases, h, sizeof(lbm::BatchCase) * c->ncases,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  delete[] h;
  if (e != cudaSuccess) return cuda_fail(c, e, "upload of the case table");
  c->total_items = (int)items;
  drop_graph(c);
  return LBM_OK;
}

static lbm_status create_ctx(const lbm_params* ps, int ncases, void* cuda_stream,
                             lbm_ctx** out) {
  g_create_err[0] = 0;
  if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ps || ncases < 1) return fail(nullptr, LBM_ERR_ARG, "need at least one case");
  for (int k = 0; k < ncases; ++k) {
    lbm_status st = validate(&ps[k]);
    if (st != LBM_OK) {
      if (ncases > 1) {
        char buf[512];
        snprintf(buf, sizeof(buf), "case %d: %s", k, g_create_err);
        return fail(nullptr, st, "%s", buf);
      }
      return st;
    }
    if (ps[k].storage != ps[0].storage || ps[k].kernel != ps[0].kernel ||
        ps[k].collision != ps[0].collision)
      return fail(nullptr, LBM_ERR_ARG,
                  "all cases of a batch need the same storage, kernel and collision");
  }
  if (ncases > 1 && ps[0].kernel != LBM_KERNEL_FUSED)
    return fail(nullptr, LBM_ERR_ARG, "batches run the fused kernel only");
  if (ncases > 1)
    for (int k = 0; k < ncases; ++k)
      for (int a = 0; a < 3; ++a)
        if (ps[k].wall[a] == 2)
          return fail(nullptr, LBM_ERR_ARG, "moving plates (wall = 2) need a single lattice");
  lbm_ctx* c = new (std::nothrow) lbm_ctx;
  if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
  memset(c, 0, sizeof(*c));
  c->cases = new (std::nothrow) CaseRec[ncases];
  if (!c->cases) {
    delete c;
    return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
  }
  c->ncases = ncases;
  c->storage = ps[0].storage;
  c->kernel = ps[0].kernel;
  c->plate_axis = -1;
  for (int a = 0; a < 3; ++a)
    if (ps[0].wall[a] == 2) c->plate_axis = a;
  for (int side = 0; side < 2; ++side)
    for (int d = 0; d < 3; ++d) c->plate_u[side][d] = ps[0].wall_u[side][d];
  c->device = -1;
  c->stream = (cudaStream_t)cuda_stream;
  c->use_graph = 1;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete[] c->cases;
    delete c;
    return fail(nullptr, LBM_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
  }
  c->elem = c->storage == LBM_F32 ? 4 : 2;
  long long pairs = 0;
  for (int k = 0; k < ncases; ++k) {
    CaseRec& r = c->cases[k];
    r.p = ps[k];
    r.N = (long long)r.p.nx * r.p.ny * r.p.nz;
    const long long plane = (r.N + 63) / 64 * 64;  // 256-byte aligned planes
    r.args = derive_args(&r.p, plane);
    r.pair_base = pairs;
    r.initialized = 0;
    pairs += 19 * plane;
    if (r.N > c->max_cells) c->max_cells = r.N;
    c->any_walls = c->any_walls || r.p.wall[0] || r.p.wall[1] || r.p.wall[2];
  }
  c->total_pairs = pairs;
  c->fused = lbm::default_fused_config(c->cases[0].args, c->storage);
  if (ncases > 1) c->fused.zchunk = 12;
  const size_t bytes = (size_t)pairs * 2 * c->elem;
  lbm_status st = LBM_OK;
  for (int b = 0; b < 2 && st == LBM_OK; ++b)
    if (lbm::dev_alloc((void**)&c->pop[b], bytes) != cudaSuccess)
      st = fail(nullptr, LBM_ERR_OOM, "cudaMalloc of %zu bytes failed", bytes);
  if (st == LBM_OK && c->kernel == LBM_KERNEL_TWO_PASS &&
      lbm::dev_alloc((void**)&c->phase, sizeof(float4) * (size_t)c->max_cells) != cudaSuccess)
    st = fail(nullptr, LBM_ERR_OOM, "cudaMalloc of the phase field failed");
  if (st == LBM_OK) {
    c->diag_blocks = lbm::diag_capacity(c->storage, c->sms);
    if (lbm::dev_alloc((void**)&c->diag_part, sizeof(double) * lbm::kDiagSlots * c->diag_blocks) != cudaSuccess ||
        lbm::dev_alloc((void**)&c->diag_out, sizeof(double) * 16) != cudaSuccess ||
        lbm::dev_alloc((void**)&c->diag_done, sizeof(unsigned)) != cudaSuccess ||
        lbm::host_alloc((void**)&c->diag_host, sizeof(double) * 16) != cudaSuccess ||
        cudaMemset(c->diag_done, 0, sizeof(unsigned)) != cudaSuccess)
      st = fail(nullptr, LBM_ERR_OOM, "cudaMalloc of diagnostics scratch failed");
  }
  if (st == LBM_OK) {
    if (lbm::dev_alloc((void**)&c->d_flags, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_flags, 0, sizeof(int)) != cudaSuccess)
      st = fail(nullptr, LBM_ERR_OOM, "cudaMalloc of the error word failed");
  }
#ifdef LBM_CHECKED
  if (st == LBM_OK) {
    if (lbm::dev_alloc((void**)&c->d_oob, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(c->d_oob, 0, sizeof(unsigned)) != cudaSuccess)
      st = fail(nullptr, LBM_ERR_OOM, "cudaMalloc of the index-check count failed");
    for (int k = 0; k < ncases && st == LBM_OK; ++k) c->cases[k].args.oob = c->d_oob;
  }
#endif
  if (st == LBM_OK && ncases == 1 && c->kernel == LBM_KERNEL_FUSED &&
      lbm::tma_eligible(c->cases[0].args, c->storage)) {
    for (int w = 0; w < 3; ++w) {
      c->tma_ok[w] = true;
      for (int b = 0; b < 2 && c->tma_ok[w]; ++b)
        c->tma_ok[w] = lbm::tma_build_maps(c->storage, c->pop[b], c->cases[0].args, w,
                                           c->tmaps[b][w]) == cudaSuccess;
    }
    if (c->tma_ok[2] && lbm::seam_eligible(c->cases[0].args, c->storage)) {
      c->seam_ok = true;
      for (int t = 0; t < 2 && c->seam_ok; ++t)
        for (int b = 0; b < 2 && c->seam_ok; ++b)
          c->seam_ok = lbm::tma_build_seam_maps(c->pop[b], c->cases[0].args, t == 0 ? 15 : 12,
                                                c->smaps[t][b]) == cudaSuccess;
    }
    cudaGetLastError();
    lbm::FusedConfig t;
    if (lbm::tma_default_config(c->cases[0].args, c->storage, c->sms, c->tma_ok, &t))
      c->fused = t;
    if (c->seam_ok) {
      // periodic FP32 lattices: the 34 x 12 tile with two stages and the
      // seams staged by tensor copies
      c->fused.tile_y = 12;
      c->fused.hold = 7;
      c->fused.zchunk = lbm::seam12_zchunk(c->cases[0].args, c->sms);
    }
    if (lbm::seam16_eligible(c->cases[0].args, c->storage)) {
      c->seam16_ok = true;
      for (int t = 0; t < 2 && c->seam16_ok; ++t)
        for (int b = 0; b < 2 && c->seam16_ok; ++b)
          c->seam16_ok = lbm::tma_build_seam16_maps(c->storage, c->pop[b], c->cases[0].args,
                                                    t == 0 ? 15 : 12,
                                                    c->smaps16[t][b]) == cudaSuccess;
      cudaGetLastError();
      if (c->seam16_ok && c->fused.tile_y == 15 && c->fused.hold == 8) {
        // the 16-bit seam form: two stages, the list-schedule chunk
        c->fused.hold = 7;
        c->fused.zchunk = lbm::list_schedule_zchunk(c->cases[0].args, c->sms, 13);
      }
    }
  }
  if (st == LBM_OK && ncases > 1) {
    // tensor maps of every case for the batched TMA step (tile kinds 0, 2)
    bool all = true;
    for (int k = 0; k < ncases && all; ++k)
      all = lbm::tma_eligible(c->cases[k].args, c->storage);
    CUtensorMap* hm = all ? new (std::nothrow) CUtensorMap[2 * (size_t)ncases] : nullptr;
    for (int w : {0, 2}) {
      bool ok = hm != nullptr;
      for (int b = 0; b < 2 && ok; ++b) {
        for (int k = 0; k < ncases && ok; ++k)
          ok = lbm::tma_build_maps(c->storage,
                                   (char*)c->pop[b] + (size_t)c->cases[k].pair_base * 2 * c->elem,
                                   c->cases[k].args, w, hm + 2 * k) == cudaSuccess;
        ok = ok && lbm::dev_alloc((void**)&c->d_bmaps[b][w], sizeof(CUtensorMap) * 2 * ncases) == cudaSuccess &&
             cudaMemcpy(c->d_bmaps[b][w], hm, sizeof(CUtensorMap) * 2 * ncases,
                        cudaMemcpyHostToDevice) == cudaSuccess;
      }
      c->batch_tma_ok[w] = ok;
    }
    delete[] hm;
    cudaGetLastError();
    // Batch default: the TMA form of the 34 x 15 tile, 32-plane chunks, one
    // stage for FP32 and two for 16-bit storage (GB300, 512-case droplet
    // sweep: 11.4 and 14.6 GLUPS against 10.0 and 12.5 for the 32 x 8
    // shared-memory hold).
    const int ns = c->storage == LBM_F32 ? 1 : 2;
    if (c->batch_tma_ok[2] && lbm::tma_config_fits(c->storage, 2, ns)) {
      c->fused.tile_y = 15;
      c->fused.zchunk = 32;
      c->fused.hold = ns == 2 ? 7 : 8;
    }
    // FP32 batches periodic in x and y: the SEAM form of the 34 x 12 tile
    // with two stages, six maps per case and buffer
    bool seam = true;
    for (int k = 0; k < ncases && seam; ++k)
      seam = lbm::batch_seam_eligible(c->cases[k].args, c->storage);
    CUtensorMap* hs = seam ? new (std::nothrow) CUtensorMap[6 * (size_t)ncases] : nullptr;
    seam = hs != nullptr;
    for (int b = 0; b < 2 && seam; ++b) {
      for (int k = 0; k < ncases && seam; ++k)
        seam = lbm::tma_build_seam_maps(
                   (char*)c->pop[b] + (size_t)c->cases[k].pair_base * 2 * c->elem,
                   c->cases[k].args, 12, hs + 6 * k) == cudaSuccess;
      seam = seam &&
             lbm::dev_alloc((void**)&c->d_seam_bmaps[b], sizeof(CUtensorMap) * 6 * ncases) ==
                 cudaSuccess &&
             cudaMemcpy(c->d_seam_bmaps[b], hs, sizeof(CUtensorMap) * 6 * ncases,
                        cudaMemcpyHostToDevice) == cudaSuccess;
    }
    delete[] hs;
    cudaGetLastError();
    // an option for the autotuner, not the default: on the 512-case droplet
    // sweep (GB300) the 34 x 15 one-stage form above runs 11.5 ms per step
    // against 13.5 ms for this one at its best chunk (48 planes): most of
    // the sweep's cells are in 96^3 cases, whose 34 x 12 tiles are ragged
    // in y and carry more ring per cell
    c->batch_seam_ok = seam;
  }
  if (st == LBM_OK && ncases > 1 &&
      lbm::dev_alloc((void**)&c->d_cases, sizeof(lbm::BatchCase) * ncases) != cudaSuccess)
    st = fail(nullptr, LBM_ERR_OOM, "cudaMalloc of the case table failed");
  if (st == LBM_OK) {
    st = upload_case_table(c);
    if (st != LBM_OK) {
      char buf[512];
      snprintf(buf, sizeof(buf), "%s", c->err);
      st = fail(nullptr, st, "%s", buf);
    }
  }
  if (st != LBM_OK) {
    cudaGetLastError();
    release(c);
    delete c;
    return st;
  }
  c->err[0] = 0;
  *out = c;
  return LBM_OK;
}

extern "C" lbm_status lbm_create(const lbm_params* p, void* cuda_stream,
                                 lbm_ctx** out) {
  lbm::NvtxRange nvtx_range_("lbm_create");
  return create_ctx(p, 1, cuda_stream, out);
}

extern "C" lbm_status lbm_create_batch(const lbm_params* cases, int ncases,
                                       void* cuda_stream, lbm_ctx** out) {
  lbm::NvtxRange nvtx_range_("lbm_create_batch");
  return create_ctx(cases, ncases, cuda_stream, out);
}

extern "C" void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  if (c->dstream) {
    cudaStreamSynchronize(c->dstream);
    cudaStreamDestroy(c->dstream);
    cudaEventDestroy(c->step_ev);
    cudaEventDestroy(c->diag_ev[0]);
    cudaEventDestroy(c->diag_ev[1]);
  }
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  release(c);
  delete c;
}

extern "C" const char* lbm_last_error(const lbm_ctx* c) {
  return c ? c->err : g_create_err;
}

extern "C" int lbm_num_cases(const lbm_ctx* c) { return c ? c->ncases : 0; }

static lbm_status ensure_staging(lbm_ctx* c, size_t floats) {
  if (c->staging_floats >= floats) return LBM_OK;
  lbm::dev_free(c->staging);
  c->staging = nullptr;
  c->staging_floats = 0;
  drop_graph(c);
  if (lbm::dev_alloc((void**)&c->staging, floats * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LBM_ERR_OOM, "cudaMalloc of %zu staging floats failed", floats);
  }
  c->staging_floats = floats;
  return LBM_OK;
}

static lbm_status caller_memory(lbm_ctx* c, const void* ptr, const char* what,
                                bool* device) {
  int owner = -1;
  switch (pointer_where(ptr, c->device, &owner)) {
    case kPtrHere:
      *device = true;
      return LBM_OK;
    case kPtrOtherDevice:
      return fail(c, LBM_ERR_ARG,
                  "%s is device memory of GPU %d, but the context runs on GPU %d", what,
                  owner, c->device);
    default:
      *device = false;
      return LBM_OK;
  }
}

// Makes `n` floats at `ptr` (host or device) readable by kernels: returns
// ptr itself for device memory, else a staging copy at `slot` floats.
static lbm_status device_input(lbm_ctx* c, const float* ptr, size_t n,
                               size_t slot, const float** out) {
  bool dev = false;
  lbm_status st = caller_memory(c, ptr, "an input field", &dev);
  if (st != LBM_OK) return st;
  if (dev) {
    *out = ptr;
    return LBM_OK;
  }
  LBM_CUDA(c, cudaMemcpyAsync(c->staging + slot, ptr, n * sizeof(float),
                              cudaMemcpyHostToDevice, c->stream),
           "cudaMemcpyAsync H2D");
  *out = c->staging + slot;
  return LBM_OK;
}

// A single lattice whose state is set anew starts without the error word of
// the bounded waits of earlier steps (a batch keeps it: its cases were
// stepped together, and the word does not say which failed).
static lbm_status fresh_state(lbm_ctx* c) {
  if (c->ncases == 1)
    LBM_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream), "cudaMemsetAsync");
  return LBM_OK;
}

// Buffer b of case k, as a byte pointer.
static char* case_buffer(lbm_ctx* c, int b, int k) {
  return (char*)c->pop[b] + (size_t)c->cases[k].pair_base * 2 * c->elem;
}

static lbm_status check_case(lbm_ctx* c, int k) {
  if (k < 0 || k >= c->ncases)
    return fail(c, LBM_ERR_ARG, "case index %d out of range [0, %d)", k, c->ncases);
  return LBM_OK;
}

// The context stream waits for the asynchronous diagnostics that still read
// buffer b (b < 0: both buffers, and the diagnostics scratch).
static lbm_status settle_diag(lbm_ctx* c, int b) {
  for (int q = 0; q < 2; ++q) {
    if ((b >= 0 && q != b) || !c->diag_pend[q]) continue;
    LBM_CUDA(c, cudaStreamWaitEvent(c->stream, c->diag_ev[q], 0), "cudaStreamWaitEvent");
    c->diag_pend[q] = false;
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_init_fields(lbm_ctx* c, int k, const float* rho_R,
                                            const float* rho_B, const float* u) {
  lbm::NvtxRange nvtx_range_("lbm_batch_init_fields");
  if (!c) return LBM_ERR_ARG;
  lbm_status st = check_case(c, k);
  if (st != LBM_OK) return st;
  if (!rho_R || !rho_B || !u) return fail(c, LBM_ERR_ARG, "NULL field pointer");
  if ((st = settle_diag(c, -1)) != LBM_OK) return st;
  CaseRec& r = c->cases[k];
  const size_t N = (size_t)r.N;
  bool dR_dev = false, dB_dev = false, dU_dev = false;
  if ((st = caller_memory(c, rho_R, "rho_R", &dR_dev)) != LBM_OK ||
      (st = caller_memory(c, rho_B, "rho_B", &dB_dev)) != LBM_OK ||
      (st = caller_memory(c, u, "u", &dU_dev)) != LBM_OK)
    return st;
  const bool all_dev = dR_dev && dB_dev && dU_dev;
  if (!all_dev && (st = ensure_staging(c, 5 * N)) != LBM_OK) return st;
  const float *dR, *dB, *dU;
  if ((st = device_input(c, rho_R, N, 0, &dR)) != LBM_OK) return st;
  if ((st = device_input(c, rho_B, N, N, &dB)) != LBM_OK) return st;
  if ((st = device_input(c, u, 3 * N, 2 * N, &dU)) != LBM_OK) return st;
  LBM_CUDA(c, lbm::launch_init_eq(c->storage, case_buffer(c, c->cur, k), r.args,
                                  (float)r.p.alpha_R, (float)r.p.alpha_B, dR, dB, dU,
                                  c->stream),
           "init kernel");
  if ((st = fresh_state(c)) != LBM_OK) return st;
  r.initialized = 1;
  c->steps = 0;
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_init_fields(lbm_ctx* c, const float* rho_R,
                                      const float* rho_B, const float* u,
                                      const unsigned char* solid) {
  lbm::NvtxRange nvtx_range_("lbm_init_fields");
  if (!c) return LBM_ERR_ARG;
  if (solid) return fail(c, LBM_ERR_ARG, "solid masks are not supported; use wall[]");
  return lbm_batch_init_fields(c, 0, rho_R, rho_B, u);
}

// mon (monitored steps, the seam forms' default tiles only): the step also
// sums the diagnostics of the state it reads into *mon.
static lbm_status launch_step(lbm_ctx* c, int from, lbm::MonAcc* mon = nullptr) {
  const void* src = c->pop[from];
  void* dst = c->pop[from ^ 1];
  cudaError_t e;
  if (c->ncases > 1 && c->fused.tile_y == 12 && c->fused.hold == 7) {
    e = c->batch_seam_ok
            ? lbm::launch_fused_tma_seam_batch(src, dst, c->d_cases, c->ncases, c->total_items,
                                               c->any_walls, c->d_seam_bmaps[from],
                                               c->fused.zchunk, c->d_flags, c->sms, c->stream)
            : cudaErrorInvalidValue;
  } else if (c->ncases > 1 && (c->fused.hold == 7 || c->fused.hold == 8)) {
    const int w = lbm::tma_kind(c->fused.tile_y);
    e = (w == 0 || w == 2) && c->batch_tma_ok[w]
            ? lbm::launch_fused_tma_batch(c->storage, src, dst, c->d_cases, c->ncases,
                                          c->total_items, c->any_walls, c->d_bmaps[from][w], w,
                                          c->fused.hold == 7 ? 2 : 1, c->fused.zchunk,
                                          c->d_flags, c->sms, c->stream)
            : cudaErrorInvalidValue;
  } else if (c->ncases > 1)
    e = lbm::launch_fused_batch(c->storage, src, dst, c->d_cases, c->ncases,
                                c->total_items, c->any_walls, c->cases[0].args.bgk != 0,
                                c->fused, c->sms, c->stream);
  else if (c->kernel == LBM_KERNEL_TWO_PASS)
    e = lbm::launch_twopass(c->storage, src, dst, c->cases[0].args, c->phase, c->stream);
  else if (c->seam16_ok && c->fused.hold == 7 &&
           (c->fused.tile_y == 15 || c->fused.tile_y == 12))
    e = lbm::launch_fused_tma_seam16(c->storage, src, dst, c->cases[0].args, c->fused.tile_y,
                                     c->smaps16[c->fused.tile_y == 15 ? 0 : 1][from],
                                     c->fused.zchunk, c->d_flags, c->stream, mon);
  else if (c->seam_ok && ((c->fused.hold == 8 && c->fused.tile_y == 15) ||
                           (c->fused.hold == 7 && c->fused.tile_y == 12)))
    e = lbm::launch_fused_tma_seam(src, dst, c->cases[0].args, c->fused.tile_y,
                                   c->smaps[c->fused.tile_y == 15 ? 0 : 1][from],
                                   c->fused.zchunk, c->d_flags, c->stream, mon);
  else if (c->fused.hold == 7 || c->fused.hold == 8) {
    const int w = lbm::tma_kind(c->fused.tile_y);
    e = w >= 0 && c->tma_ok[w]
            ? lbm::launch_fused_tma(c->storage, src, dst, c->cases[0].args, c->tmaps[from][w],
                                    w, c->fused.hold == 7 ? 2 : 1, c->fused.zchunk,
                                    c->d_flags, c->stream)
            : cudaErrorInvalidValue;
  }
  else
    e = lbm::launch_fused(c->storage, src, dst, c->cases[0].args, c->fused, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
  if (c->plate_axis >= 0) {
    e = lbm::launch_plates(c->storage, dst, c->cases[0].args, c->plate_axis, c->plate_u,
                           c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "moving-plate kernel launch");
  }
  return LBM_OK;
}

// Two steps (buffer 0 -> 1 -> 0) captured once into a CUDA graph.
static lbm_status ensure_graph(lbm_ctx* c) {
  if (c->graph) return LBM_OK;
  cudaGraph_t g = nullptr;
  LBM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal),
           "cudaStreamBeginCapture");
  lbm_status st = launch_step(c, 0);
  if (st == LBM_OK) st = launch_step(c, 1);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  return LBM_OK;
}

extern "C" lbm_status lbm_step(lbm_ctx* c, int n) {
  lbm::NvtxRange nvtx_range_("lbm_step");
  if (!c) return LBM_ERR_ARG;
  if (n < 0) return fail(c, LBM_ERR_ARG, "n must be >= 0");
  for (int k = 0; k < c->ncases; ++k)
    if (!c->cases[k].initialized)
      return fail(c, LBM_ERR_STATE, "lbm_step before every case was initialised (case %d)", k);
  {  // one step writes the other buffer only; more steps write both
    lbm_status sd = settle_diag(c, n == 1 ? (c->cur ^ 1) : -1);
    if (sd != LBM_OK) return sd;
  }
  // CUDA graphs need a capturable stream (not the legacy default stream).
  const bool graphs = c->use_graph && c->stream != nullptr && n >= 4;
  lbm_status st;
  if (graphs) {
    // Bring the state to buffer 0; before the first capture also run two
    // plain steps, so that one-time kernel attribute and occupancy queries
    // happen outside stream capture.
    const int plain = (c->cur == 1 ? 1 : 0) + (c->graph ? 0 : 2);
    for (int q = 0; q < plain; ++q) {
      if ((st = launch_step(c, c->cur)) != LBM_OK) return st;
      c->cur ^= 1;
      c->steps += 1;
      n -= 1;
    }
    if ((st = ensure_graph(c)) != LBM_OK) return st;
    for (; n >= 2; n -= 2) {
      LBM_CUDA(c, cudaGraphLaunch(c->graph, c->stream), "cudaGraphLaunch");
      c->steps += 2;
    }
  }
  for (; n > 0; --n) {
    if ((st = launch_step(c, c->cur)) != LBM_OK) return st;
    c->cur ^= 1;
    c->steps += 1;
  }
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_set_graphs(lbm_ctx* c, int enable) {
  if (!c) return LBM_ERR_ARG;
  c->use_graph = enable ? 1 : 0;
  if (!enable) drop_graph(c);
  return LBM_OK;
}

static bool case_ready(lbm_ctx* c, int k) { return c->cases[k].initialized != 0; }

extern "C" lbm_status lbm_batch_moments(lbm_ctx* c, int k, float* rho_R,
                                        float* rho_B, float* u) {
  lbm::NvtxRange nvtx_range_("lbm_batch_moments");
  if (!c) return LBM_ERR_ARG;
  lbm_status st = check_case(c, k);
  if (st != LBM_OK) return st;
  if (!case_ready(c, k)) return fail(c, LBM_ERR_STATE, "moments before init");
  const CaseRec& r = c->cases[k];
  const size_t N = (size_t)r.N;
  float* outs[3] = {rho_R, rho_B, u};
  const size_t sizes[3] = {N, N, 3 * N};
  const size_t slots[3] = {0, N, 2 * N};
  bool host[3];
  bool any_host = false;
  for (int q = 0; q < 3; ++q) {
    bool dev = false;
    if (outs[q] && (st = caller_memory(c, outs[q], "a moments output", &dev)) != LBM_OK)
      return st;
    host[q] = outs[q] && !dev;
    any_host = any_host || host[q];
  }
  if (any_host && (st = ensure_staging(c, 5 * N)) != LBM_OK) return st;
  float* k_out[3];
  for (int q = 0; q < 3; ++q)
    k_out[q] = !outs[q] ? nullptr : (host[q] ? c->staging + slots[q] : outs[q]);
  LBM_CUDA(c, lbm::launch_moments(c->storage, case_buffer(c, c->cur, k), r.args,
                                  k_out[0], k_out[1], k_out[2], c->stream),
           "moments kernel");
  for (int q = 0; q < 3; ++q)
    if (host[q])
      LBM_CUDA(c, cudaMemcpyAsync(outs[q], k_out[q], sizes[q] * sizeof(float),
                                  cudaMemcpyDeviceToHost, c->stream),
               "cudaMemcpyAsync D2H");
  if (any_host) LBM_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_moments(lbm_ctx* c, float* rho_R, float* rho_B,
                                  float* u) {
  lbm::NvtxRange nvtx_range_("lbm_moments");
  return lbm_batch_moments(c, 0, rho_R, rho_B, u);
}

static lbm_status enqueue_diag(lbm_ctx* c, int k, cudaStream_t s) {
  const CaseRec& r = c->cases[k];
  LBM_CUDA(c, lbm::launch_diag(c->storage, case_buffer(c, c->cur, k), r.args,
                               c->diag_part, c->diag_blocks, c->diag_done, c->d_flags,
                               c->steps, c->diag_out, s),
           "diagnostics kernel");
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_diagnostics(lbm_ctx* c, int k, double out[16]) {
  lbm::NvtxRange nvtx_range_("lbm_batch_diagnostics");
  if (!c || !out) return c ? fail(c, LBM_ERR_ARG, "out is NULL") : LBM_ERR_ARG;
  lbm_status st = check_case(c, k);
  if (st != LBM_OK) return st;
  if (!case_ready(c, k)) return fail(c, LBM_ERR_STATE, "diagnostics before init");
  if ((st = settle_diag(c, -1)) != LBM_OK) return st;  // shares the scratch
  if ((st = enqueue_diag(c, k, c->stream)) != LBM_OK) return st;
  LBM_CUDA(c, cudaMemcpyAsync(c->diag_host, c->diag_out, sizeof(double) * 16,
                              cudaMemcpyDeviceToHost, c->stream),
           "cudaMemcpyAsync D2H");
  LBM_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  for (int i = 0; i < 16; ++i) out[i] = c->diag_host[i];
  c->err[0] = 0;
  const int flags = (int)out[14];
  if (flags)
    return fail(c, LBM_ERR_TIMEOUT,
                "a bounded wait of the step kernel gave up (code %d); results are invalid", flags);
  if (out[5] != 0.0 || out[6] != 0.0)
    return fail(c, LBM_ERR_UNSTABLE,
                "%.0f cells with non-finite populations, %.0f with total density <= 0",
                out[5], out[6]);
  return LBM_OK;
}

extern "C" lbm_status lbm_step_diagnostics_async(lbm_ctx* c, int n, double* out) {
  lbm::NvtxRange nvtx_range_("lbm_step_diagnostics_async");
  if (!c || !out) return c ? fail(c, LBM_ERR_ARG, "out is NULL") : LBM_ERR_ARG;
  if (!c->dstream) {
    LBM_CUDA(c, cudaStreamCreateWithFlags(&c->dstream, cudaStreamNonBlocking),
             "cudaStreamCreateWithFlags");
    LBM_CUDA(c, cudaEventCreateWithFlags(&c->step_ev, cudaEventDisableTiming),
             "cudaEventCreateWithFlags");
    for (int q = 0; q < 2; ++q)
      LBM_CUDA(c, cudaEventCreateWithFlags(&c->diag_ev[q], cudaEventDisableTiming),
               "cudaEventCreateWithFlags");
  }
  lbm_status st = lbm_step(c, n);
  if (st != LBM_OK) return st;
  // the diagnostics of the state just reached, on their own stream after
  // the step; they read buffer cur, which the next step only reads
  LBM_CUDA(c, cudaEventRecord(c->step_ev, c->stream), "cudaEventRecord");
  LBM_CUDA(c, cudaStreamWaitEvent(c->dstream, c->step_ev, 0), "cudaStreamWaitEvent");
  if ((st = enqueue_diag(c, 0, c->dstream)) != LBM_OK) return st;
  LBM_CUDA(c, cudaMemcpyAsync(out, c->diag_out, sizeof(double) * 16, cudaMemcpyDefault,
                              c->dstream),
           "cudaMemcpyAsync of the diagnostics");
  LBM_CUDA(c, cudaEventRecord(c->diag_ev[c->cur], c->dstream), "cudaEventRecord");
  c->diag_pend[c->cur] = true;
  c->err[0] = 0;
  return LBM_OK;
}

// The monitored form exists for the seam kernels' default tiles, with z
// chunks of at most 255 planes (a thread's counts are packed in bytes).
static bool monitor_fused(const lbm_ctx* c) {
  const int zc = c->fused.zchunk > 0 ? c->fused.zchunk : c->cases[0].p.nz;
  return c->ncases == 1 && c->kernel == LBM_KERNEL_FUSED && c->fused.hold == 7 && zc <= 255 &&
         ((c->seam_ok && c->storage == LBM_F32 && c->fused.tile_y == 12) ||
          (c->seam16_ok && c->storage != LBM_F32 && c->fused.tile_y == 15));
}

extern "C" lbm_status lbm_step_monitored(lbm_ctx* c, int n, double* out) {
  lbm::NvtxRange nvtx_range_("lbm_step_monitored");
  if (!c || !out) return c ? fail(c, LBM_ERR_ARG, "out is NULL") : LBM_ERR_ARG;
  if (n < 0) return fail(c, LBM_ERR_ARG, "n must be >= 0");
  if (c->ncases != 1)
    return fail(c, LBM_ERR_ARG, "lbm_step_monitored: single-lattice contexts only");
  if (!c->cases[0].initialized) return fail(c, LBM_ERR_STATE, "lbm_step_monitored before init");
  lbm_status st = settle_diag(c, -1);
  if (st != LBM_OK) return st;
  const bool fused = monitor_fused(c);
  if (fused && !c->d_mon) {
    if (lbm::dev_alloc((void**)&c->d_mon, sizeof(lbm::MonAcc)) != cudaSuccess ||
        lbm::dev_alloc((void**)&c->d_mon_out, sizeof(double) * 16) != cudaSuccess) {
      cudaGetLastError();
      lbm::dev_free(c->d_mon);
      c->d_mon = nullptr;
      return fail(c, LBM_ERR_OOM, "cudaMalloc of the monitor record failed");
    }
    LBM_CUDA(c, cudaMemsetAsync(c->d_mon, 0, sizeof(lbm::MonAcc), c->stream), "cudaMemsetAsync");
  }
  for (int k = 0; k < n; ++k) {
    double* o = out + 16 * (size_t)k;
    if (fused) {
      if ((st = launch_step(c, c->cur, c->d_mon)) != LBM_OK) return st;
      LBM_CUDA(c, lbm::launch_monitor_out(c->d_mon, c->d_flags, (double)c->steps, c->d_mon_out,
                                          c->stream),
               "monitor kernel");
      LBM_CUDA(c, cudaMemcpyAsync(o, c->d_mon_out, sizeof(double) * 16, cudaMemcpyDefault,
                                  c->stream),
               "cudaMemcpyAsync of the monitor");
    } else {
      // other kernel forms: the diagnostics pass over the state, then the step
      if ((st = enqueue_diag(c, 0, c->stream)) != LBM_OK) return st;
      LBM_CUDA(c, cudaMemcpyAsync(o, c->diag_out, sizeof(double) * 16, cudaMemcpyDefault,
                                  c->stream),
               "cudaMemcpyAsync of the diagnostics");
      if ((st = launch_step(c, c->cur)) != LBM_OK) return st;
    }
    c->cur ^= 1;
    c->steps += 1;
  }
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_sync(lbm_ctx* c) {
  lbm::NvtxRange nvtx_range_("lbm_sync");
  if (!c) return LBM_ERR_ARG;
  if (c->dstream) LBM_CUDA(c, cudaStreamSynchronize(c->dstream), "stream sync");
  for (int q = 0; q < 2; ++q) c->diag_pend[q] = false;
  LBM_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_diagnostics(lbm_ctx* c, double out[16]) {
  return lbm_batch_diagnostics(c, 0, out);
}

extern "C" lbm_status lbm_batch_footprint(lbm_ctx* c, int axis, int index,
                                          long long* counts) {
  lbm::NvtxRange nvtx_range_("lbm_batch_footprint");
  if (!c || !counts) return c ? fail(c, LBM_ERR_ARG, "counts is NULL") : LBM_ERR_ARG;
  if (axis < 0 || axis > 2) return fail(c, LBM_ERR_ARG, "axis must be 0, 1 or 2");
  for (int k = 0; k < c->ncases; ++k) {
    const lbm_params& p = c->cases[k].p;
    const int n = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
    if (index < 0 || index >= n)
      return fail(c, LBM_ERR_ARG, "plane index %d outside case %d (extent %d)", index, k, n);
    if (!case_ready(c, k)) return fail(c, LBM_ERR_STATE, "footprint before init (case %d)", k);
  }
  if (!c->foot)
    LBM_CUDA(c, lbm::dev_alloc((void**)&c->foot, sizeof(unsigned long long) * c->ncases), "cudaMalloc");
  LBM_CUDA(c, cudaMemsetAsync(c->foot, 0, sizeof(unsigned long long) * c->ncases, c->stream),
           "cudaMemsetAsync");
  for (int k = 0; k < c->ncases; ++k)
    LBM_CUDA(c, lbm::launch_footprint(c->storage, case_buffer(c, c->cur, k), c->cases[k].args,
                                      axis, index, c->foot + k, c->stream),
             "footprint kernel");
  static_assert(sizeof(long long) == sizeof(unsigned long long), "64-bit counts");
  LBM_CUDA(c, cudaMemcpyAsync(counts, c->foot, sizeof(long long) * c->ncases,
                              cudaMemcpyDefault, c->stream),
           "cudaMemcpyAsync D2H");
  LBM_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  return LBM_OK;
}

extern "C" lbm_status lbm_batch_get_f(lbm_ctx* c, int k, float* f) {
  lbm::NvtxRange nvtx_range_("lbm_batch_get_f");
  if (!c || !f) return c ? fail(c, LBM_ERR_ARG, "f is NULL") : LBM_ERR_ARG;
  lbm_status st = check_case(c, k);
  if (st != LBM_OK) return st;
  if (!case_ready(c, k)) return fail(c, LBM_ERR_STATE, "get_f before init");
  const CaseRec& r = c->cases[k];
  const size_t n = 38 * (size_t)r.N;
  bool dev = false;
  if ((st = caller_memory(c, f, "f", &dev)) != LBM_OK) return st;
  if (dev) {
    LBM_CUDA(c, lbm::launch_get_f(c->storage, case_buffer(c, c->cur, k), r.args, f,
                                  c->stream),
             "get_f kernel");
  } else {
    if ((st = ensure_staging(c, n)) != LBM_OK) return st;
    LBM_CUDA(c, lbm::launch_get_f(c->storage, case_buffer(c, c->cur, k), r.args,
                                  c->staging, c->stream),
             "get_f kernel");
    LBM_CUDA(c, cudaMemcpyAsync(f, c->staging, n * sizeof(float),
                                cudaMemcpyDeviceToHost, c->stream),
             "cudaMemcpyAsync D2H");
    LBM_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  }
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_get_f(lbm_ctx* c, float* f) { return lbm_batch_get_f(c, 0, f); }

extern "C" lbm_status lbm_batch_set_f(lbm_ctx* c, int k, const float* f) {
  lbm::NvtxRange nvtx_range_("lbm_batch_set_f");
  if (!c || !f) return c ? fail(c, LBM_ERR_ARG, "f is NULL") : LBM_ERR_ARG;
  lbm_status st = check_case(c, k);
  if (st != LBM_OK) return st;
  if ((st = settle_diag(c, -1)) != LBM_OK) return st;
  CaseRec& r = c->cases[k];
  const size_t n = 38 * (size_t)r.N;
  const float* src = f;
  bool dev = false;
  if ((st = caller_memory(c, f, "f", &dev)) != LBM_OK) return st;
  if (!dev) {
    if ((st = ensure_staging(c, n)) != LBM_OK) return st;
    LBM_CUDA(c, cudaMemcpyAsync(c->staging, f, n * sizeof(float),
                                cudaMemcpyHostToDevice, c->stream),
             "cudaMemcpyAsync H2D");
    src = c->staging;
  }
  LBM_CUDA(c, lbm::launch_set_f(c->storage, case_buffer(c, c->cur, k), r.args, src,
                                c->stream),
           "set_f kernel");
  if ((st = fresh_state(c)) != LBM_OK) return st;
  r.initialized = 1;
  c->steps = 0;
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_set_f(lbm_ctx* c, const float* f) { return lbm_batch_set_f(c, 0, f); }

extern "C" size_t lbm_population_bytes(const lbm_ctx* c) {
  return c ? (size_t)c->total_pairs * 2 * c->elem : 0;
}

extern "C" lbm_status lbm_get_populations(lbm_ctx* c, void* dst) {
  lbm::NvtxRange nvtx_range_("lbm_get_populations");
  if (!c || !dst) return c ? fail(c, LBM_ERR_ARG, "dst is NULL") : LBM_ERR_ARG;
  for (int k = 0; k < c->ncases; ++k)
    if (!case_ready(c, k)) return fail(c, LBM_ERR_STATE, "lbm_get_populations before init");
  LBM_CUDA(c, cudaMemcpyAsync(dst, c->pop[c->cur], lbm_population_bytes(c),
                              cudaMemcpyDefault, c->stream),
           "cudaMemcpyAsync");
  LBM_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_set_populations(lbm_ctx* c, const void* src) {
  lbm::NvtxRange nvtx_range_("lbm_set_populations");
  if (!c || !src) return c ? fail(c, LBM_ERR_ARG, "src is NULL") : LBM_ERR_ARG;
  {
    lbm_status st = settle_diag(c, -1);
    if (st != LBM_OK) return st;
  }
  LBM_CUDA(c, cudaMemcpyAsync(c->pop[c->cur], src, lbm_population_bytes(c),
                              cudaMemcpyDefault, c->stream),
           "cudaMemcpyAsync");
  {
    lbm_status st = fresh_state(c);
    if (st != LBM_OK) return st;
  }
  LBM_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
  for (int k = 0; k < c->ncases; ++k) c->cases[k].initialized = 1;
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" size_t lbm_plane_bytes(const lbm_ctx* c) {
  if (!c || c->ncases != 1) return 0;
  const CaseRec& r = c->cases[0];
  return (size_t)19 * r.p.nx * r.p.ny * 2 * c->elem;
}

// One strided copy: direction i's planes z0 .. z0 + n - 1 are contiguous in
// the buffer (cell = (z ny + y) nx + x), direction planes r.args.plane pairs
// apart; the caller's side holds the 19 runs back to back.
static lbm_status plane_copy(lbm_ctx* c, int z0, int n, void* host_side, bool to_caller) {
  if (!c) return LBM_ERR_ARG;
  if (c->ncases != 1) return fail(c, LBM_ERR_ARG, "plane copies need a single-lattice context");
  if (!host_side) return fail(c, LBM_ERR_ARG, "NULL plane buffer");
  const CaseRec& r = c->cases[0];
  if (z0 < 0 || n < 1 || z0 + n > r.p.nz)
    return fail(c, LBM_ERR_ARG, "planes [%d, %d) outside [0, %d)", z0, z0 + n, r.p.nz);
  if (!r.initialized) return fail(c, LBM_ERR_STATE, "plane copy before init");
  bool dev = false;
  lbm_status st = caller_memory(c, host_side, "the plane buffer", &dev);
  if (st != LBM_OK) return st;
  // writing the current buffer waits for diagnostics still reading it
  if (!to_caller && (st = settle_diag(c, c->cur)) != LBM_OK) return st;
  const size_t pair = 2 * c->elem;
  const size_t cells = (size_t)r.p.nx * r.p.ny;
  const size_t run = (size_t)n * cells * pair;
  char* buf = (char*)c->pop[c->cur] + (size_t)z0 * cells * pair;
  const size_t pitch = (size_t)r.args.plane * pair;
  if (to_caller)
    LBM_CUDA(c, cudaMemcpy2DAsync(host_side, run, buf, pitch, run, 19, cudaMemcpyDefault,
                                  c->stream),
             "cudaMemcpy2DAsync");
  else
    LBM_CUDA(c, cudaMemcpy2DAsync(buf, pitch, host_side, run, run, 19, cudaMemcpyDefault,
                                  c->stream),
             "cudaMemcpy2DAsync");
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_get_planes(lbm_ctx* c, int z0, int n, void* dst) {
  lbm::NvtxRange nvtx_range_("lbm_get_planes");
  return plane_copy(c, z0, n, dst, true);
}

extern "C" lbm_status lbm_set_planes(lbm_ctx* c, int z0, int n, const void* src) {
  lbm::NvtxRange nvtx_range_("lbm_set_planes");
  return plane_copy(c, z0, n, const_cast<void*>(src), false);
}

extern "C" lbm_status lbm_set_fused_config(lbm_ctx* c, int tile_y, int zchunk,
                                           int hold) {
  if (!c) return LBM_ERR_ARG;
  lbm::FusedConfig f;
  f.tile_y = tile_y;
  f.hold = hold;
  f.zchunk = zchunk == 0
                 ? (c->ncases > 1 ? 12 : lbm::default_fused_config(c->cases[0].args, c->storage).zchunk)
                 : zchunk;
  const bool batch_tma =
      (hold == 7 || hold == 8) && (tile_y == 8 || tile_y == 15) &&
      c->batch_tma_ok[lbm::tma_kind(tile_y)] &&
      lbm::tma_config_fits(c->storage, lbm::tma_kind(tile_y), hold == 7 ? 2 : 1);
  const bool single_tma =
      lbm::tma_kind(f.tile_y) >= 0 && c->tma_ok[lbm::tma_kind(f.tile_y)] &&
      lbm::tma_config_fits(c->storage, lbm::tma_kind(f.tile_y), f.hold == 7 ? 2 : 1);
  const bool ok =
      zchunk >= 0 &&
      (c->ncases > 1
           ? lbm::valid_batch_config(f) && ((hold != 7 && hold != 8) || batch_tma)
           : lbm::valid_fused_config(f, c->storage) && ((hold != 7 && hold != 8) || single_tma));
  if (tile_y == 12) {  // the two-stage SEAM form only
    if (c->ncases > 1) {
      if (!(c->batch_seam_ok && hold == 7 && zchunk >= 0))
        return fail(c, LBM_ERR_ARG,
                    "tile_y 12 is the batched seam form (hold 7) of FP32 batches whose cases "
                    "are periodic in x and y (MRT, nx a multiple of 2)");
      c->fused = f;
      drop_graph(c);
      lbm_status st = upload_case_table(c);
      if (st != LBM_OK) return st;
      c->err[0] = 0;
      return LBM_OK;
    }
    if (!((c->seam_ok || c->seam16_ok) && hold == 7 && zchunk >= 0))
      return fail(c, LBM_ERR_ARG,
                  "tile_y 12 is the two-stage seam form (hold 7) of single periodic lattices "
                  "with nx a multiple of 2 (FP32) or 4 (16-bit), nx >= 34 and ny >= 15");
    if (zchunk == 0) f.zchunk = lbm::seam12_zchunk(c->cases[0].args, c->sms);
    c->fused = f;
    drop_graph(c);
    c->err[0] = 0;
    return LBM_OK;
  }
  if (ok && c->cases[0].args.bgk && (f.tile_y != 8 || f.hold != 2))
    return fail(c, LBM_ERR_ARG,
                "the BGK operator runs the shared-memory-hold form only (tile_y 8, hold 2)");
  if (!ok)
    return fail(c, LBM_ERR_ARG,
                c->ncases > 1
                    ? "invalid batch configuration ((tile_y, hold) = (8, 2), (8, 0), (16, 1), "
                      "or (8 or 15, 7 or 8) where every case has tensor maps; zchunk >= 0)"
                    : "invalid fused configuration (tile_y 8, 15 or 16, zchunk >= 0, hold "
                      "0..8; hold 2, 3, 5, 6 need tile_y 8, hold 4 needs tile_y 16, tile_y 15 "
                      "needs hold 7 or 8; hold 7 and 8 need nx * pair bytes a multiple of 16 "
                      "and a tile whose stages fit shared memory)");
  c->fused = f;
  drop_graph(c);
  lbm_status st = upload_case_table(c);
  if (st != LBM_OK) return st;
  c->err[0] = 0;
  return LBM_OK;
}

extern "C" lbm_status lbm_get_fused_config(const lbm_ctx* c, int* tile_y,
                                           int* zchunk, int* hold) {
  if (!c || !tile_y || !zchunk || !hold) return LBM_ERR_ARG;
  *tile_y = c->fused.tile_y;
  *zchunk = c->fused.zchunk;
  *hold = c->fused.hold;
  return LBM_OK;
}

extern "C" lbm_status lbm_default_fused_config(const lbm_params* p, int sms, int* tile_y,
                                               int* zchunk, int* hold) {
  g_create_err[0] = 0;
  lbm_status st = validate(p);
  if (st != LBM_OK) return st;
  if (!tile_y || !zchunk || !hold)
    return fail(nullptr, LBM_ERR_ARG, "lbm_default_fused_config: NULL output");
  if (sms < 0) return fail(nullptr, LBM_ERR_ARG, "lbm_default_fused_config: sms must be >= 0");
  // the choice lbm_create makes for a single lattice, with every tensor map
  // encoded (they do on every lattice tma_eligible / seam_eligible admit)
  const long long N = (long long)p->nx * p->ny * p->nz;
  const StepArgs a = derive_args(p, (N + 63) / 64 * 64);
  lbm::FusedConfig f = lbm::default_fused_config(a, p->storage);
  if (p->kernel == LBM_KERNEL_FUSED && lbm::tma_eligible(a, p->storage)) {
    const bool maps_ok[3] = {true, true, true};
    lbm::FusedConfig t;
    if (lbm::tma_default_config(a, p->storage, sms, maps_ok, &t)) f = t;
    if (lbm::seam_eligible(a, p->storage)) {
      f.tile_y = 12;
      f.hold = 7;
      f.zchunk = lbm::seam12_zchunk(a, sms);
    }
    if (lbm::seam16_eligible(a, p->storage) && f.tile_y == 15 && f.hold == 8) {
      f.hold = 7;
      f.zchunk = lbm::list_schedule_zchunk(a, sms, 13);
    }
  }
  *tile_y = f.tile_y;
  *zchunk = f.zchunk;
  *hold = f.hold;
  return LBM_OK;
}

extern "C" int lbm_launches_per_step(const lbm_ctx* c) {
  if (!c) return 0;
  return ((c->ncases == 1 && c->kernel == LBM_KERNEL_TWO_PASS) ? 2 : 1) +
         (c->plate_axis >= 0 ? 1 : 0);
}

extern "C" void lbm_test_fake_pointer_attributes(int enable, int type, int device,
                                                 int current_device) {
  g_fake_type.store(type);
  g_fake_device.store(device);
  g_fake_current.store(current_device);
  g_fake_on.store(enable ? 1 : 0);
}
