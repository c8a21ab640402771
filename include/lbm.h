/*
 * lbm.h -- C ABI of the GB300 (sm_103a) implementation of the improved
 * three-dimensional colour-gradient MRT lattice Boltzmann time step of
 * Wen, Li, Yu & Luo, "Improved three-dimensional color-gradient lattice
 * Boltzmann model for immiscible multiphase flows" (arXiv:1904.03618).
 *
 * The operation behind this interface is one time step of Eq. 1-2 for two
 * fluids ("red" k = R and "blue" k = B) on the D3Q19 lattice of Eq. 5:
 *   pull streaming (Sec. II.A, below Eq. 13), moments (Eq. 4), phase field
 *   rho^N (below Eq. 8), isotropic colour and correction gradients (Eq. 49),
 *   variable shear relaxation time (Eq. 52), MRT collision in moment space
 *   with the improved equilibrium (Eq. 18-19, Appendix) and the correction
 *   term (Eq. 41, 45-48), the surface-tension perturbation applied through
 *   the collision matrix (Eq. 8, 53), and recolouring (Eq. 10-11).
 *
 * Conventions for every entry point:
 *   - A lattice has nx * ny * nz cells, x fastest: cell = (z * ny + y) * nx + x.
 *   - Scalar fields are float32 arrays of N = nx*ny*nz values; vector fields
 *     are three consecutive planes (x, y, z components), 3*N values.
 *   - Population arrays f_i^k are float32, layout [k][i][cell], k = 0 red,
 *     1 blue, i = 0..18 in the order of Eq. 5: 38*N values.
 *   - Pointers marked "host or device" may point to either; the library
 *     detects which (CUDA unified addressing) and copies accordingly.
 *     Device memory must belong to the GPU the work runs on (the context's
 *     GPU, or the current one for the calls without a context): a pointer
 *     to another GPU's memory is refused with LBM_ERR_ARG before any launch.
 *     Caller-owned memory is only read or written during the call's stream
 *     work and never retained.
 *   - All work is ordered on the stream given to lbm_create (or to the
 *     stateless calls).  Calls that return data to a host pointer
 *     synchronise that stream before returning; others return as soon as
 *     the work is queued.  Nothing is ordered across streams: device memory
 *     the caller wrote (or will reuse) on another stream must be ordered
 *     against this one by the caller (an event and cudaStreamWaitEvent).
 *   - Every function returns an lbm_status; nothing aborts, traps or exits.
 *     On failure lbm_last_error() describes the cause.
 *   - Lattice units throughout: delta_x = delta_t = c = 1.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, library-owned */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,      /* invalid argument or parameter                    */
  LBM_ERR_OOM = -2,      /* device or host allocation failed                 */
  LBM_ERR_CUDA = -3,     /* a CUDA runtime call failed                       */
  LBM_ERR_UNSTABLE = -4, /* non-finite value or negative density detected    */
  LBM_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up               */
  LBM_ERR_STATE = -6     /* call out of order (e.g. step before init)        */
} lbm_status;

typedef enum {
  LBM_F32 = 0,  /* populations stored as float32                            */
  LBM_F16 = 1,  /* stored as IEEE half deviations f - ref_k * phi_i^k         */
  LBM_BF16 = 2  /* stored as bfloat16 deviations f - ref_k * phi_i^k          */
} lbm_storage;

typedef enum {
  LBM_KERNEL_FUSED = 0,   /* one kernel per step: z-marching tile, halo moments
                             recomputed in shared memory                     */
  LBM_KERNEL_TWO_PASS = 1 /* two kernels per step: phase field and correction
                             flux written to a scratch field, then collision */
} lbm_kernel;

typedef enum {
  LBM_COLLISION_MRT = 0, /* the paper's MRT operator: Eq. 40-44 with tau_e,
                            tau_q, tau_pi and the variable tau_v of Eq. 52,
                            perturbation by Eq. 53                           */
  LBM_COLLISION_BGK = 1  /* BGK with the correction term, Eq. 20: every
                            non-conserved moment relaxes at 1 / tau_v of Eq. 52
                            (tau_e, tau_q, tau_pi unused), the correction and
                            force under (1 - 1/(2 tau_v)), the Eq. 8
                            perturbation divided by tau_v -- Lambda = I / tau_v
                            in Eq. 40 and 53, as the paper notes            */
} lbm_collision;

/* Model and lattice parameters.  Defaults used by the paper are in
   brackets; see the cited equations for meaning. */
typedef struct {
  int nx, ny, nz;      /* lattice size, each >= 1, ny and nz <= 65535,
                          nx*ny*nz < 226 million (the in-place calls:
                          limited by device memory only)                    */
  int wall[3];         /* per axis: 0 periodic, 1 halfway bounce-back walls on
                          both faces (wall at -1/2 and n - 1/2); Sec. IV.B-D;
                          2 moving plates through the first and last layer
                          (Zou-He velocity nodes, Sec. IV.A) with velocities
                          wall_u -- at most one such axis, the other two
                          periodic, single lattices only                    */
  int improved;        /* 1: Eq. 18 equilibrium + Eq. 45 correction (the
                          improved model); 0: Eq. 6, no correction (the
                          "original model" of Sec. IV.A)                     */
  int storage;         /* lbm_storage                                        */
  int kernel;          /* lbm_kernel                                         */
  int wetting;         /* 0: neutral walls (contact angle 90 degrees, Sec.
                          IV.D: neighbours beyond a wall take the centre value
                          in Eq. 49); 1: contact angle contact_angle_deg --
                          at a fluid cell next to a wall the colour gradient
                          keeps its magnitude and its direction along the wall
                          and is turned to the angle pi - theta from the
                          inward wall normal (theta measured through the red
                          fluid) before the perturbation and recolouring use
                          it.  The paper has only the neutral wall.          */
  double rho_in_R, rho_in_B; /* rho_k^in in rho^N, below Eq. 8 (> 0)         */
  double alpha_R, alpha_B;   /* alpha_k of Eq. 13, in [0, 1)                 */
  double tau_R, tau_B;       /* tau_v^R, tau_v^B of Eq. 52 (> 1/2)            */
  double tau_e, tau_q, tau_pi; /* Eq. 44 [1.0] (> 1/2)                       */
  double A_R, A_B;     /* Eq. 8; surface tension 2 (A_R + A_B) / 9 (Eq. 53)  */
  double beta;         /* recolouring parameter of Eq. 10-11, in [0, 1]      */
  double delta;        /* interface half-width of Eq. 52 [0.98], in (0, 1]   */
  double force[3];     /* uniform body-force density (Sec. IV.B)             */
  double gravity[3];   /* acceleration g; adds the force density rho * g
                          (Sec. IV.C)                                        */
  double ref_R, ref_B; /* reference densities of the FP16/BF16 deviation
                          storage (ignored for LBM_F32): colour k is stored as
                          f_i^k - ref_k * phi_i^k                            */
  double contact_angle_deg; /* theta in (0, 180) when wetting = 1            */
  int collision;       /* lbm_collision [LBM_COLLISION_MRT]                  */
  int reserved;        /* 0                                                  */
  double wall_u[2][3]; /* velocity of the low and the high plate of the
                          wall = 2 axis (its normal component moves fluid
                          through the plate).  After every step the
                          populations of each colour entering from beyond a
                          plate are rebuilt so that the node carries
                          rho_k * wall_u (mass from the normal velocity,
                          bounce-back of the non-equilibrium part along the
                          normal, transverse momentum corrections); the plate
                          velocity carries no forcing shift                  */
} lbm_params;

/* Creates a context: validates p, allocates the two population buffers and
   scratch on the current CUDA device, and binds `cuda_stream` (a
   cudaStream_t; NULL = the legacy default stream).  *out receives the
   context; on failure *out is NULL.  Errors: LBM_ERR_ARG for an invalid p
   (the message names the field), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_create(const lbm_params *p, void *cuda_stream, lbm_ctx **out);

/* Sets the populations to the equilibrium of each colour (Eq. 18, or Eq. 6
   when improved = 0) for the given fields, as in the paper's initialisation
   "brought to the equilibrium state" (Sec. IV.A).  rho_R, rho_B: N floats;
   u: 3*N floats; all host or device.  solid must be NULL (walls are the
   per-axis flags of lbm_params).  Resets the step counter to 0.
   Errors: LBM_ERR_ARG (NULL field, non-NULL solid), LBM_ERR_CUDA. */
lbm_status lbm_init_fields(lbm_ctx *ctx, const float *rho_R,
                           const float *rho_B, const float *u,
                           const unsigned char *solid);

/* Advances n >= 0 time steps (Eq. 1-2, Eq. 10-13, Eq. 40-53, streaming).
   Queued on the context stream; returns without waiting.
   Errors: LBM_ERR_ARG (n < 0), LBM_ERR_STATE (no init yet), LBM_ERR_CUDA. */
lbm_status lbm_step(lbm_ctx *ctx, int n);

/* Writes the macroscopic fields at the current time level (after
   streaming): rho_R, rho_B (N floats each) and u (3*N floats), with
   u = (sum_i sum_k e_i f_i^k + F/2) / rho (Eq. 4, forcing shift), F the
   total force density.  Any output pointer may be NULL to skip it; each is
   host or device. */
lbm_status lbm_moments(lbm_ctx *ctx, float *rho_R, float *rho_B, float *u);

/* FP64 whole-lattice diagnostics into the host array out[16]:
   [0] sum rho_R   [1] sum rho_B   [2..4] sum_i sum_k e_i f_i^k (momentum)
   [5] count of cells with a non-finite population
   [6] count of cells with total density rho <= 0
   [7] max |u|     [8] count of cells with rho^N > 0
   [9..11] red-mass centroid (sum rho_R x / sum rho_R, lattice coordinates,
           no periodic unwrapping)
   [12] number of completed steps
   [13] count of cells with rho_R < 0 or rho_B < 0 (small negative colour
        densities in the minority phase are a normal effect of the
        recolouring, Eq. 10-11; informational)
   [14] error word of the step kernels' bounded waits (0: none); it stays
        set until a single lattice's state is set anew (lbm_init_fields,
        lbm_set_f, lbm_set_populations), for a batch until it is destroyed
   [15] 0 (reserved).
   The colour masses and the momentum are exact to about FP64 accuracy
   (compensated FP32 accumulators per direction and thread, FP64 across
   threads); the centroid and |u| come from the FP32 cell
   moments.  One kernel launch and one 128-byte copy; synchronises the
   context stream.  Returns LBM_ERR_TIMEOUT if [14] is non-zero, else
   LBM_ERR_UNSTABLE if [5] or [6] is non-zero (out is filled either way). */
lbm_status lbm_diagnostics(lbm_ctx *ctx, double out[16]);

/* Monitored stepping without host waits: advances n >= 0 steps (as
   lbm_step, on the context stream) and queues the diagnostics of the state
   they reach (case 0 of a batch) and an asynchronous copy of their 16 slots
   (as lbm_diagnostics) into out, which may be pinned host memory or device
   memory (pageable host memory makes the copy synchronous).  The
   diagnostics run on a stream of the library's own (created on first use)
   after the step, so that they overlap the next step, which only reads the
   buffer they read; a later launch that writes that buffer waits for them.
   Returns after queueing: out is valid after lbm_sync.  State errors are
   reported in the slots ([5], [6], [14]), not by the return value.
   Errors: LBM_ERR_ARG (out NULL, n < 0), LBM_ERR_STATE, LBM_ERR_CUDA. */
lbm_status lbm_step_diagnostics_async(lbm_ctx *ctx, int n, double *out);

/* Monitored stepping with the diagnostics computed inside the step: n >= 0
   steps (as lbm_step), where step k (k = 0 .. n-1) also reports the
   diagnostics of the state it reads -- the state after k steps of this
   call -- into out[16 k .. 16 k + 15] (the slots of lbm_diagnostics; slot
   [12] = the steps completed before that state), out being pinned host or
   device memory (pageable host memory makes the copies synchronous).  For
   a single lattice on the seam forms' default tiles (FP32 periodic in x
   and y, FP16 / BF16 periodic in x and y with nx a multiple of 4) the step
   kernel sums them from the moments it already holds, so monitoring adds
   no pass over the populations: per warp in FP32 (the masses and momentum
   to about 1e-7 relative, not the compensated sums of lbm_diagnostics),
   across warps and CTAs in FP64, by atomics (the last bits can vary from
   run to run); the counts, max |u| and centroid as lbm_diagnostics.  Other
   contexts run the lbm_diagnostics pass before each step.  Queued on the
   context stream without a host wait: out is valid after lbm_sync.  The
   state after the last step is not reported (lbm_diagnostics gives it).
   Errors: LBM_ERR_ARG (out NULL, n < 0, a batch), LBM_ERR_STATE,
   LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_step_monitored(lbm_ctx *ctx, int n, double *out);

/* Waits until all work queued by the context (its stream and the stream of
   the asynchronous diagnostics) has finished. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Copies f_i^k(x, t) -- the populations after streaming at the current
   time level, the paper's state variable -- as float32 [2][19][N] into f
   (host or device), converting from the storage format. */
lbm_status lbm_get_f(lbm_ctx *ctx, float *f);

/* Sets the state from f_i^k(x, t) given as float32 [2][19][N] (host or
   device), converting to the storage format.  Resets the step counter. */
lbm_status lbm_set_f(lbm_ctx *ctx, const float *f);

/* Size in bytes of one raw population buffer (the checkpoint unit).  The
   internal layout is [direction][cell][colour]: the red and blue values of
   one direction and cell are adjacent; each direction plane is padded. */
size_t lbm_population_bytes(const lbm_ctx *ctx);

/* Raw checkpoint of the current population buffer: dst (host or device)
   receives lbm_population_bytes() bytes in the library's internal layout
   (storage format, pull-streaming order).  Restoring it with
   lbm_set_populations into a context created with the same parameters
   resumes the run bit-identically.  The step counter is not part of it.
   Both synchronise the context stream. */
lbm_status lbm_get_populations(lbm_ctx *ctx, void *dst);
lbm_status lbm_set_populations(lbm_ctx *ctx, const void *src);

/* Halo planes of a z-slab decomposition of one lattice over several
   contexts (one per GPU or per slab); the paper has no counterpart.  A
   slab's context covers its own planes plus two ghost planes on each side
   that has a neighbour, with wall[2] = 1: a cell's update reads the stored
   state within two planes, so after every step the two outermost planes
   of each neighbour's own range, copied into the ghost planes, make the
   slab's own planes evolve exactly as in the undivided lattice (the ghost
   planes themselves are overwritten by the next copy).
   lbm_get_planes copies the stored planes z0 .. z0 + n - 1 of the current
   state into dst, lbm_set_planes copies src into them: raw storage format
   (the buffer the next step pulls from; FP16 / BF16 as stored
   deviations), layout [i][z][y][x][colour], n * lbm_plane_bytes() bytes.
   Single-lattice contexts only; 0 <= z0, n >= 1, z0 + n <= nz.  dst / src
   are host or device memory (device memory of the context's GPU); the copy
   is queued on the context stream and the calls return without waiting
   (pageable host memory makes the copy synchronous).
   lbm_plane_bytes: bytes of one plane, 19 * nx * ny * 2 * element size. */
size_t lbm_plane_bytes(const lbm_ctx *ctx);
lbm_status lbm_get_planes(lbm_ctx *ctx, int z0, int n, void *dst);
lbm_status lbm_set_planes(lbm_ctx *ctx, int z0, int n, const void *src);

/* Launch configuration of the fused kernel (LBM_KERNEL_FUSED), the knob the
   autotuner turns; results are identical for every valid configuration.
   Batch contexts accept (tile_y, hold) = (8, 2), (8, 0), (16, 1) and, when
   every case has an x row of 16-byte multiple length, the TMA forms (8 or
   15, 7 or 8); their default is then (15, 32, 8) for FP32 and (15, 32, 7)
   for 16-bit storage.
   tile_y: CTA rows including the one-cell ring, 8 or 16 (the interior tile
   is 30 x (tile_y - 2) cells), or 15 (below).  zchunk: planes marched per CTA, 0 = the
   library's default for this lattice.  hold: where the populations of a
   plane wait between the moment pass and the collision: 0 pulled again, 1
   registers, 2 shared memory (tile_y = 8 only), 3 shared memory filled by
   asynchronous copies issued two planes ahead (tile_y = 8 only), 4 shared
   memory with each thread handling two tile rows (tile_y = 16 only), 5 and
   6 as 2 with registers capped for three and four CTAs per SM, 7 and 8 as
   2 with each plane's pulls staged in shared memory by tensor copies (TMA)
   issued two planes (7) or one plane (8) ahead, for single lattices with
   nx * 8 bytes (FP32) or nx * 4 bytes (FP16/BF16) a multiple of 16;
   tile_y = 8 is a 32 x 8 thread tile, tile_y = 16 a 16 x 16 thread tile
   (interior 14 x 14; with hold 7 for 16-bit storage only) and tile_y = 15
   (hold 7 and 8 only) a 34 x 15 thread tile (interior 32 x 13, one CTA per
   SM).  On FP32 single lattices periodic in x and y (walls in z allowed)
   with nx >= 34 and ny >= 15, the TMA forms stage the cells beyond the
   periodic x / y seams by tensor copies of the lattice's far side instead
   of pulling them from global memory (the seam forms): tile_y = 15 with
   hold 8 (one stage), and tile_y = 12 with hold 7 -- a 34 x 12 thread tile
   (interior 32 x 10) with two stages, accepted only there and the default
   there.  The TMA waits are bounded and report LBM_ERR_TIMEOUT through
   lbm_diagnostics.
   Errors: LBM_ERR_ARG. */
lbm_status lbm_set_fused_config(lbm_ctx *ctx, int tile_y, int zchunk, int hold);
lbm_status lbm_get_fused_config(const lbm_ctx *ctx, int *tile_y, int *zchunk,
                                int *hold);

/* The fused configuration lbm_create picks for a single lattice with these
   parameters on a GPU with `sms` streaming multiprocessors (0: 152, the
   GB300), computed on the host without a GPU: the same rules, with every
   tensor map taken as encodable (which holds on every lattice the TMA
   eligibility rules admit).  For the 34 x 12 seam form the z chunk is the
   one whose list schedule of CTAs over the SMs ends first: one CTA per SM,
   handed out in launch order to the first SM that falls free, each costing
   its planes + 3 plane-times.  Errors: LBM_ERR_ARG (invalid parameters,
   NULL output, sms < 0), described by lbm_last_error(NULL). */
lbm_status lbm_default_fused_config(const lbm_params *p, int sms, int *tile_y,
                                    int *zchunk, int *hold);

/* Number of kernel launches one lbm_step(ctx, 1) issues (1 for the fused
   kernel, 2 for the two-pass form). */
int lbm_launches_per_step(const lbm_ctx *ctx);

/* ---- Batches: many independent lattices advanced together --------------
   A batch context holds `ncases` lattices ("cases"), each with its own
   lbm_params (size, walls, densities, alpha, relaxation times, surface
   tension, beta, forces); all cases share storage (p->storage) and run the
   fused kernel.  lbm_step advances every case by n steps with one kernel
   launch per step: persistent CTAs take (case, z-chunk, tile) work items in
   turn, so cases of uneven sizes share the GPU without idle tails; in the
   TMA forms each case's pulls are staged by tensor copies described by
   per-case tensor maps held in device memory.  Cases
   must be initialised (lbm_batch_init_fields or lbm_batch_set_f) before
   lbm_step.  The single-lattice calls (lbm_init_fields, lbm_moments,
   lbm_diagnostics, lbm_get_f, lbm_set_f) act on case 0 of a batch. */
lbm_status lbm_create_batch(const lbm_params *cases, int ncases,
                            void *cuda_stream, lbm_ctx **out);
int lbm_num_cases(const lbm_ctx *ctx);
lbm_status lbm_batch_init_fields(lbm_ctx *ctx, int case_index,
                                 const float *rho_R, const float *rho_B,
                                 const float *u);
lbm_status lbm_batch_moments(lbm_ctx *ctx, int case_index, float *rho_R,
                             float *rho_B, float *u);
lbm_status lbm_batch_diagnostics(lbm_ctx *ctx, int case_index,
                                 double out[16]);
/* For every case, the number of cells of the lattice plane normal to `axis`
   (0 = x, 1 = y, 2 = z) at coordinate `index` where the red colour dominates
   (rho^N > 0, rho^N as defined below Eq. 8), at the current time level.  With a
   wall at z = 0 and index 0 this is the wetted footprint of a red drop on
   the floor (area in lattice cells); the paper has no counterpart.  counts:
   ncases long longs, host or device.  index must lie inside every case;
   synchronises the stream. */
lbm_status lbm_batch_footprint(lbm_ctx *ctx, int axis, int index,
                               long long *counts);
lbm_status lbm_batch_get_f(lbm_ctx *ctx, int case_index, float *f);
lbm_status lbm_batch_set_f(lbm_ctx *ctx, int case_index, const float *f);

/* lbm_step(ctx, n) with n >= 4 on a non-default stream replays two steps
   captured once into a CUDA graph (the first such call also runs two plain
   steps before capturing).  enable = 0 launches every step directly.  The
   result does not depend on it. */
lbm_status lbm_set_graphs(lbm_ctx *ctx, int enable);

/* One time step that allocates no device memory, for callers that cannot
   call cudaMalloc (services whose device memory is fixed at start-up,
   embedders that own every device buffer).  The paper has no counterpart:
   it is a deployment variant of the two-pass step above, with the same
   result.
   f_in: f_i^k(x, t) after streaming, float32 [2][19][N], device memory;
   f_out: receives f_i^k(x, t + 1) in the same layout, device memory, must
   not overlap f_in.  p->storage and p->kernel are ignored (FP32).  Work is
   queued on cuda_stream (a cudaStream_t, NULL = legacy default stream); the
   call returns without waiting.  The scratch (16 bytes per cell) is a fixed
   device array of 262,144 cells (4 MiB) inside the library, held by every
   GPU that loads the library until the process exits: lattices with
   nx*ny*nz > 262,144 are rejected with LBM_ERR_ARG.  The first call on each
   device looks up that array's device address (with the device current),
   and a call looks it up again when the CUDA context current on the device
   is not the one of the last lookup (after cudaDeviceReset, or when an
   embedder makes a context of its own current, the library is loaded again
   at another address).  All calls on a device share the array and it
   keeps the last call's contents (every entry a call reads is written by
   that call first), so calls that overlap
   on the GPU -- e.g. on two streams at once -- race.  Errors (LBM_ERR_ARG,
   LBM_ERR_CUDA) are described by lbm_last_error(NULL) of the calling
   thread; f_in or f_out in host memory, or in device memory of a GPU other
   than the current one, is LBM_ERR_ARG. */
lbm_status lbm_step_noalloc(const lbm_params *p, const float *f_in,
                            float *f_out, void *cuda_stream);

/* ---- In-place step (AA access pattern) ----------------------------------
   The step of Eq. 1-2 (the same collision, forcing, perturbation,
   recolouring, walls, wetting rule and BGK option as lbm_step) on ONE
   population array [2][19][N] (k = 0 red, 1 blue; cell = (z * ny + y) * nx
   + x) of p->storage's values -- FP32 populations, or FP16 / BF16
   deviations f - ref_k phi_i^k from the colour's rest state, with the
   offsets of a context of the same parameters (p->ref_R, p->ref_B) --
   updated in place: 152 bytes per cell in FP32 (76 in 16 bits) plus a
   16-byte scratch, against 304 (152) for the two buffers of a context.  Cell indices are
   64-bit: nx*ny*nz is limited by device memory only (ny, nz <= 65535).  The
   paper streams between two arrays; this is a deployment variant with the
   same result up to FP32 rounding.
   A state has a parity.  Even (0): f[k][i][x] = f_i^k(x, t), after
   streaming, the layout of lbm_set_f / lbm_get_f (stored as above).  Each
   stored value keeps its direction's offset in both parities (opposite
   directions share an offset).  Odd (1): f[k][opp(i)][x]
   = f_i^{k,+}(x, t - 1), the post-collision value before streaming, so
   f_i^k(x, t) is found at f[k][opp(i)][x - e_i], or at f[k][i][x] where
   x - e_i lies beyond a wall; e_i in the order of Eq. 5, where opp pairs
   the directions (1,2), (3,4), ..., (17,18).  A step turns one parity into the
   other; the caller keeps track of it (after lbm_step_inplace with n steps
   the parity is (parity + n) mod 2).
   Each step runs two kernels: the phase field (rho^N, Qbar) of every cell
   into the scratch, then the in-place collision (488 bytes of memory
   traffic per cell, against 304 for lbm_step's fused kernel).
   Moving plates (wall = 2) are rejected with LBM_ERR_ARG; p->kernel is
   ignored.  f must be aligned to its value size.  All arrays are device
   memory of the
   current GPU owned by the caller; work is queued on cuda_stream (a cudaStream_t, NULL = legacy
   default stream) and the calls return without waiting.  Errors
   (LBM_ERR_ARG, LBM_ERR_CUDA) are described by lbm_last_error(NULL) of the
   calling thread. */

/* Equilibrium populations (Eq. 18 with the improved coefficient when
   p->improved, else Eq. 6) of the fields rho_R, rho_B (N floats each) and
   u (u_x, u_y, u_z planes, 3N floats) written into f as an even state.  f
   must not overlap the fields. */
lbm_status lbm_inplace_init(const lbm_params *p, const float *rho_R,
                            const float *rho_B, const float *u, void *f,
                            void *cuda_stream);

/* An even state from FP32 populations f_in[2][19][N] (the layout of
   lbm_set_f), stored in p->storage's format (16-bit: the deviations rounded
   to nearest even).  f must not overlap f_in. */
lbm_status lbm_inplace_set(const lbm_params *p, const float *f_in, void *f,
                           void *cuda_stream);

/* nsteps >= 0 time steps of the state f of the given parity (0 or 1), in
   place.  scratch: N float4 (16 bytes per cell, 16-byte aligned), not
   overlapping f; its contents on entry are ignored. */
lbm_status lbm_step_inplace(const lbm_params *p, void *f, int parity,
                            int nsteps, void *scratch, void *cuda_stream);

/* Reads the state f of the given parity: f_out (may be NULL) receives
   f_i^k(x, t) in the even layout, rho_R, rho_B (N floats) and u (3N)
   (each may be NULL) the moments of lbm_moments (u with the half-force
   shift of Eq. 4).  At least one output; none may overlap f or another
   output. */
lbm_status lbm_inplace_read(const lbm_params *p, const void *f, int parity,
                            float *f_out, float *rho_R, float *rho_B,
                            float *u, void *cuda_stream);

/* ---- Surrogate network (tensor cores) -----------------------------------
   A fully connected network x -> tanh(x W_1 + b_1) -> ... (depth hidden
   layers of `width`) -> (. W_out + b_out), trained with mean squared error
   sum((y - t)^2) / (batch * n_out) and Adam (beta1 0.9, beta2 0.999, eps
   1e-8).  It maps impact parameters to a spreading-factor series and screens
   parameter sweeps; the lattice Boltzmann step remains its fallback and the
   reference its error is measured against.  The paper has no counterpart.  Every matrix product
   runs on the 5th-generation tensor cores (tcgen05, BF16 operands, FP32
   accumulation); weights, gradients, Adam moments and activations are FP32.
   Parameters are one flat FP32 vector, layer by layer: W_l (fan_in x
   fan_out, row-major, W[i][j] maps input i to output j), then b_l.
   x (batch x n_in), t and y (batch x n_out) are row-major float32; x and t
   must be device memory, y and the parameter / gradient arrays may be host
   or device.  Work is queued on cuda_stream; calls returning values to the
   host synchronise it.  1 <= n_in, width, n_out <= 256, 0 <= depth <= 64,
   1 <= batch <= max_batch.  LBM_ERR_TIMEOUT reports a bounded wait for the
   tensor cores that gave up (nothing traps). */
typedef struct lbm_mlp lbm_mlp;
lbm_status lbm_mlp_create(int n_in, int width, int depth, int n_out,
                          int max_batch, void *cuda_stream, lbm_mlp **out);
size_t lbm_mlp_num_params(const lbm_mlp *m);
/* Copies the parameters in and resets the Adam state, the step count and
   the record of a bounded wait that gave up. */
lbm_status lbm_mlp_set_params(lbm_mlp *m, const float *theta);
lbm_status lbm_mlp_get_params(lbm_mlp *m, float *theta);
/* y = network(x); synchronises the stream (LBM_ERR_TIMEOUT if a GEMM's
   bounded wait gave up). */
lbm_status lbm_mlp_forward(lbm_mlp *m, const float *x, int batch, float *y);
/* Loss (host float, nullable) and gradient (num_params floats, nullable). */
lbm_status lbm_mlp_loss_grad(lbm_mlp *m, const float *x, const float *t,
                             int batch, float *loss, float *grad);
/* Forward, backward and one Adam step with learning rate lr; loss
   (nullable) receives the loss before the step (synchronises). */
lbm_status lbm_mlp_train_step(lbm_mlp *m, const float *x, const float *t,
                              int batch, float lr, float *loss);
void lbm_mlp_destroy(lbm_mlp *m);
const char *lbm_mlp_last_error(const lbm_mlp *m);

/* The network's matrix product on its own: C(m, n) = sum_k A(m, k) B(k, n)
   with A(m, k) = A[m*sa_m + k*sa_k], B(k, n) = B[k*sb_k + n*sb_n],
   C[m*sc_m + n]; device pointers, operands rounded to BF16, FP32
   accumulation, 1 <= N <= 256.  For K > 256 the product is split over K
   and the partial sums are added into C with atomics (C is zeroed first),
   so the FP32 summation order, and with it the last bits of C, can differ
   from call to call; within the bound K 2^-24 sum_k |A(m, k) B(k, n)| of
   the exact product of the rounded operands either way.  err (device int)
   is set to 1 if a bounded wait gave up.  Queued on cuda_stream. */
lbm_status lbm_gemm_bf16(const float *A, long long sa_m, long long sa_k,
                         const float *B, long long sb_k, long long sb_n,
                         float *C, long long sc_m, int M, int N, int K,
                         int *err, void *cuda_stream);

/* Releases everything the context owns.  NULL is allowed. */
void lbm_destroy(lbm_ctx *ctx);

/* Testing hook of the pointer checks, for machines with one GPU or none;
   the paper has no counterpart.  enable = 1: until it is called again with
   enable = 0, every pointer the library classifies is taken to be memory
   of CUDA memory type `type` (a cudaMemoryType value: 1 host, 2 device, 3
   managed) on GPU `device`, and `current_device` is taken to be the current
   GPU, without asking the CUDA runtime.  Process-wide; not for use while
   other threads call the library. */
void lbm_test_fake_pointer_attributes(int enable, int type, int device,
                                      int current_device);

/* Testing hook of the bounded device waits; the paper has no counterpart.
   Sets, on the current GPU, how long the step kernels' waits for their
   tensor copies (stage_ns, default 20 ms) and the surrogate GEMM's waits
   for its tensor-core commits (mma_ns, default 200 ms) last before they
   give up and report LBM_ERR_TIMEOUT (0 restores a default; a limit
   below 1000 ns, shorter than a tick of the GPU's global timer, gives up
   at the first poll that finds the copies or MMAs outstanding).  The wait
   that follows a give-up, for the block's own copies or MMAs still in
   flight, keeps its full limit.  Synchronises the device; call it while no
   work of the library runs. */
lbm_status lbm_test_set_wait_limits(unsigned long long stage_ns,
                                    unsigned long long mma_ns);

/* Testing hooks of the allocation paths; the paper has no counterpart.
   lbm_test_fail_allocation(n), n > 0: the n-th device or pinned host
   allocation the library makes from now on fails as cudaMalloc does when
   memory runs out (n <= 0: none).  lbm_test_live_allocations: allocations
   the library has made and not yet released. */
void lbm_test_fail_allocation(int n);
long long lbm_test_live_allocations(void);

/* Testing hook of the checked build (the library compiled with
   -DLBM_CHECKED, a stand-in for a memory checker, which is not run on the
   GPUs this library is tested on); the paper has no counterpart.  In that
   build the step kernels test every computed population index (pulls,
   stores, the seam and plate writes) against its buffer and the TMA copies'
   x coordinates against the 16-byte rule before the access, count a
   failure and skip the access.  *checked: 1 in the checked build, 0
   otherwise; *out_of_range: the failures counted since ctx was created (0
   in a normal build).  Synchronises ctx's stream. */
lbm_status lbm_test_index_checks(lbm_ctx *ctx, int *checked, unsigned *out_of_range);

/* Testing hook of the surrogate GEMM's launch plan; the paper has no
   counterpart.  out = {form, columns per CTA, column blocks or K splits,
   CTAs per column block or per split} as lbm_gemm_bf16 would launch the
   product on a GPU with `sms` SMs.  K <= 256 (the persistent
   warp-specialised kernel, B resident): form 1 is the TMA-fed form (A
   K-contiguous, sa_k = 1, with a row stride sa_m a multiple of 4 floats,
   a_aligned16 nonzero for a 16-byte aligned A, M >= 128 and K >= 32; it
   falls back to form 0 when the driver cannot encode the tensor map), form
   0 the register form.  K > 256 (a plain product, as lbm_gemm_bf16 makes):
   form 2, the register form split over ceil(K / 256) grid slices of 256
   K each that add into C; form 3 (zeros after it), the one-tile-per-CTA
   kernel, when the slices would exceed 65,535.  Host only: no CUDA call.
   LBM_ERR_ARG for out == NULL, M, N, K or sms out of range (N <= 256). */
lbm_status lbm_test_gemm_plan(int M, int N, int K, long long sa_m, long long sa_k,
                              int a_aligned16, int sms, int out[4]);

/* Text of the last error on ctx (never NULL; "" after success).  With
   ctx == NULL, the last error of a failed lbm_create in this thread. */
const char *lbm_last_error(const lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
