// TMA-pipelined fused step for sm_103a (included once per storage type).
//
// Same z-march as k_fused with the shared-memory hold (four-slot window of
// (rho^N, Qbar), one barrier per plane), on a CTA tile of TW x BY threads,
// interior (TW - 2) x (BY - 2) plus the one-cell ring: 32 x 8 (two CTAs per
// SM), 16 x 16 (two CTAs per SM, two tile rows per warp) or 34 x 15 (one CTA
// of 16 warps per SM; 32-wide interiors tile lattices whose nx is a multiple
// of 32 without a ragged column of tiles, and the ring lanes are spread over
// all warps), but the pulls of a plane do not come from per-thread global
// loads.  One thread issues, per
// plane and direction i, one tensor copy (cp.async.bulk.tensor, TMA) of the
// box of source cells x - e_i of the tile's columns into a shared-memory
// stage.  With NS = 2 stages the copies of plane z + 2 are in flight while
// plane z + 1 is reduced and plane z collides; with NS = 1 the copies of
// plane z + 1 are issued after plane z's barrier and land during its
// collision.  Each thread reads its 19 pairs from shared memory at fixed
// offsets (row ty, column tx + const) with no address arithmetic.
//
// Box geometry (pairs = red/blue values of one direction and cell):
//   FP32 (8-byte pairs): directions with e_ix = +1 start at x0 - 2, with
//     e_ix = -1 at x0, both TW pairs wide; e_ix = 0 starts at x0 - 2 and is
//     TW + 2 pairs wide.  x0 = (TW - 2) bx is even, so every start is
//     16-byte aligned.
//   FP16 / BF16 (4-byte pairs): every box starts at (x0 - 2) rounded down to
//     a multiple of 4 pairs and is TW + 4 pairs wide, rounded up to a
//     multiple of 4.
//   Rows y0 - 1 - e_iy ... (BY rows); plane z - e_iz, wrapped periodically
//   in z.  Each box is padded to a multiple of 128 bytes in the stage.
// A copy whose box reaches beyond the lattice in x or y fills zeros there
// (TMA bounds handling); in the plain form the cells whose sources lie
// beyond the lattice in x or y -- the periodic wrap and bounce-back links,
// i.e. cells on the first and last row and column -- pull from global memory
// as k_fused does (the SEAM form below stages the periodic ones), and so do
// the first and last plane of a lattice with walls in z (they get no
// copies).
//
// Periodic seams (SEAM form: FP32, lattices periodic in x and y -- walls in
// z allowed, their first and last plane pulled from global memory; a 34 x 15
// tile with one stage or a 34 x 12 tile with two).  A tensor copy cannot wrap around a periodic axis, so a tile on a
// seam gets, per direction, up to three more copies into its stage: the two
// columns beyond the x seam (a 2 x BY box read from the other side of the
// lattice), the two rows beyond the y seam (a W x 2 box) and the 2 x 2
// corner.  A direction's main box and its strips share one block of the
// stage; each lane looks up its 19 pairs through nine byte offsets, one per
// (e_x, e_y), fixed per chunk, so a seam tile reads shared memory exactly
// like an inner one and no lane pulls from global memory.
//
// Waits on the stage mbarriers are bounded (kTmaWaitNs); a wait that
// gives up sets *err, waits (bounded) for the CTA's copies still in flight
// and leaves the CTA.
#pragma once

#include <cuda.h>

#include "lbm_fused.cuh"

namespace lbm {

// A stage's copies land within microseconds; a wait gives up after
// g_tma_wait_ns, kTmaWaitNs unless a test has shortened it to exercise the
// give-up path (tma_set_wait_ns).  The drain after a give-up always waits
// up to kTmaWaitNs, so that no CTA leaves with its own copies in flight.
constexpr unsigned long long kTmaWaitNs = 20ull * 1000 * 1000;
static __device__ unsigned long long g_tma_wait_ns = kTmaWaitNs;

// Sets g_tma_wait_ns of this translation unit on the current device (0:
// the default); instantiated once per storage type's unit.
template <typename T>
cudaError_t tma_set_wait_ns(unsigned long long ns) {
  const unsigned long long v = ns ? ns : kTmaWaitNs;
  return cudaMemcpyToSymbol(g_tma_wait_ns, &v, sizeof v);
}

template <typename T>
__host__ __device__ constexpr int tma_pair_bytes() {
  return (int)sizeof(typename Store<T>::Pair);
}
// Box width of direction i, in pairs, for a tile TW threads wide (16-bit
// boxes rounded up to whole 16-byte rows).
template <typename T, int TW>
__host__ __device__ constexpr int tma_width(int i) {
  return tma_pair_bytes<T>() == 8 ? (ex(i) == 0 ? TW + 2 : TW) : (TW + 4 + 3) / 4 * 4;
}
// Bytes of direction i's box in a stage, padded to a multiple of 128 so
// that every box starts 128-byte aligned.
template <typename T, int TW, int BY>
__host__ __device__ constexpr int tma_box_bytes(int i) {
  return (tma_width<T, TW>(i) * BY * tma_pair_bytes<T>() + 127) / 128 * 128;
}
template <typename T, int TW, int BY>
__host__ __device__ constexpr int tma_box_off(int i) {
  int o = 0;
  for (int j = 0; j < i; ++j) o += tma_box_bytes<T, TW, BY>(j);
  return o;
}
// SEAM form: per direction one block = main box (up to TW + 2 pairs wide) |
// x strip (2 x BY) | y strip (up to (TW + 2) x 2) | corner (2 x 2), each part
// 128-byte aligned; the main box of a TW-wide direction leaves its block's
// tail unused.
template <int TW, int BY>
__host__ __device__ constexpr int seam_main_bytes(int w) {
  return (w * BY * 8 + 127) / 128 * 128;
}
template <int TW, int BY>
__host__ __device__ constexpr int seam_xs_off(int w) {
  return seam_main_bytes<TW, BY>(w);
}
template <int TW, int BY>
__host__ __device__ constexpr int seam_ys_off(int w) {
  return seam_xs_off<TW, BY>(w) + (2 * BY * 8 + 127) / 128 * 128;
}
template <int TW, int BY>
__host__ __device__ constexpr int seam_cs_off(int w) {
  return seam_ys_off<TW, BY>(w) + ((TW + 2) * 2 * 8 + 127) / 128 * 128;
}
template <int TW, int BY>
__host__ __device__ constexpr int seam_block_bytes() {
  return seam_cs_off<TW, BY>(TW + 2) + 128;
}
// 16-bit SEAM form (4-byte pairs; TMA boxes start on 16-byte boundaries, so
// strips are four pairs wide): per direction one block = main box (W16 =
// TW + 4 rounded up to 4 pairs, from x = (x0 - 2) & ~3) | x strip (4 x BY,
// from x = nx - 4 at the low seam, 0 at the high one) | y strip (W16 x 2) |
// corner (4 x 2), each part 128-byte aligned.
template <int TW>
__host__ __device__ constexpr int s16_w() {
  return (TW + 4 + 3) / 4 * 4;
}
template <int TW, int BY>
__host__ __device__ constexpr int s16_xs_off() {
  return (s16_w<TW>() * BY * 4 + 127) / 128 * 128;
}
template <int TW, int BY>
__host__ __device__ constexpr int s16_ys_off() {
  return s16_xs_off<TW, BY>() + (4 * BY * 4 + 127) / 128 * 128;
}
template <int TW, int BY>
__host__ __device__ constexpr int s16_cs_off() {
  return s16_ys_off<TW, BY>() + (s16_w<TW>() * 2 * 4 + 127) / 128 * 128;
}
template <int TW, int BY>
__host__ __device__ constexpr int s16_block_bytes() {
  return s16_cs_off<TW, BY>() + 128;
}
template <typename T, int TW, int BY, bool SEAM = false>
__host__ __device__ constexpr int tma_stage_bytes() {
  return SEAM ? 19 * (tma_pair_bytes<T>() == 8 ? seam_block_bytes<TW, BY>()
                                                : s16_block_bytes<TW, BY>())
              : tma_box_off<T, TW, BY>(19);
}
// Bytes the 19 copies of a plane deliver (the boxes without their padding):
// the transaction count the stage's mbarrier expects.
template <typename T, int TW, int BY>
__host__ __device__ constexpr int tma_stage_tx_bytes() {
  int b = 0;
  for (int i = 0; i < 19; ++i) b += tma_width<T, TW>(i) * BY * tma_pair_bytes<T>();
  return b;
}
// Which of the two tensor maps direction i uses (FP32: 0 = TW wide, 1 =
// TW + 2 wide; 16-bit pairs: map 0 only).
template <typename T>
__host__ __device__ constexpr int tma_map(int i) {
  return tma_pair_bytes<T>() == 8 && ex(i) == 0 ? 1 : 0;
}

constexpr int kTmaSmemLimit = 227 * 1024;  // dynamic shared memory per CTA
template <int TW, int BY>
__host__ __device__ constexpr int tma_win_bytes() {
  return 4 * BY * TW * 16;
}
template <int TW, int BY>
__host__ __device__ constexpr int tma_hold_bytes(int vals) {
  return vals * (BY - 2) * (TW - 2) * 4;
}
// Values a cell holds between its pull and its collision: f (19), rho_R,
// rho_B and, where shared memory allows, u (recomputed from f otherwise).
template <typename T, int TW, int BY, int NS, bool SEAM = false>
__host__ __device__ constexpr int tma_hold_vals() {
  return NS * tma_stage_bytes<T, TW, BY, SEAM>() + tma_win_bytes<TW, BY>() +
                     tma_hold_bytes<TW, BY>(24) + 16 <=
                 (TW * BY > 256 ? kTmaSmemLimit : 113 * 1024)
             ? 24
             : 21;
}
template <typename T, int TW, int BY, int NS, bool SEAM = false>
__host__ __device__ constexpr int tma_smem_bytes() {
  return NS * tma_stage_bytes<T, TW, BY, SEAM>() + tma_win_bytes<TW, BY>() +
         tma_hold_bytes<TW, BY>(tma_hold_vals<T, TW, BY, NS, SEAM>()) + 16;
}
// Resident CTAs per SM the configuration is laid out for.
template <int TW, int BY>
__host__ __device__ constexpr int tma_ctas_per_sm() {
  return TW * BY > 256 ? 1 : 2;
}
template <typename T, int TW, int BY, int NS, bool SEAM = false>
__host__ __device__ constexpr bool tma_fits() {
  return tma_smem_bytes<T, TW, BY, NS, SEAM>() <=
         (tma_ctas_per_sm<TW, BY>() == 1 ? kTmaSmemLimit : 113 * 1024);
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try(unsigned mbar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_test(unsigned mbar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}
// The give-up limit of this launch, read once per CTA (a volatile read:
// only the host writes it, so its initial value is no constant).
__device__ __forceinline__ unsigned long long tma_wait_limit() {
  return *(const volatile unsigned long long*)&g_tma_wait_ns;
}
// Bounded wait for a phase of a stage mbarrier: `limit` ns of wall time on
// the global timer.  A limit below 1000 ns (shorter than a tick of that
// timer, and than the time a blocking try_wait may suspend the thread) is a
// test of the give-up path: one non-blocking poll decides.
__device__ __forceinline__ bool tma_wait(unsigned mbar, unsigned parity,
                                         unsigned long long limit = kTmaWaitNs) {
  if (limit < 1000) return mbar_test(mbar, parity);
  if (mbar_try(mbar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try(mbar, parity))
    if (global_ns() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int x, int y,
                                            int z, int d, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(d),
      "r"(mbar)
      : "memory");
}

// Issues the 19 copies of one plane into a stage.
template <typename T, int TW, int BY, int I>
struct TmaIssue {
  __device__ __forceinline__ static void run(unsigned stage, const CUtensorMap* m0,
                                             const CUtensorMap* m1, int x0, int y0, int zz,
                                             int nz, unsigned mbar) {
    int x;
    if constexpr (tma_pair_bytes<T>() == 8)
      x = ex(I) < 0 ? x0 : x0 - 2;
    else
      x = (x0 - 2) & ~3;
    tma_load_4d(stage + tma_box_off<T, TW, BY>(I), tma_map<T>(I) ? m1 : m0, x,
                y0 - 1 - ey(I), wrap1(zz - ez(I), nz), I, mbar);
    TmaIssue<T, TW, BY, I + 1>::run(stage, m0, m1, x0, y0, zz, nz, mbar);
  }
};
template <typename T, int TW, int BY>
struct TmaIssue<T, TW, BY, 19> {
  __device__ __forceinline__ static void run(unsigned, const CUtensorMap*, const CUtensorMap*,
                                             int, int, int, int, unsigned) {}
};

// SEAM form: the strip maps (x strip 2 x BY, y strips TW x 2 and (TW + 2) x 2,
// corner 2 x 2) of the source buffer.
struct SeamStripMaps {
  const CUtensorMap *xs, *ys0, *ys1, *cs;
};
// SEAM form, one thread: the main boxes of a plane into their blocks (as
// TmaIssue, compile-time direction and map) ...
template <int TW, int BY, int I>
struct TmaIssueSeamMain {
  __device__ __forceinline__ static void run(unsigned block0, const CUtensorMap* m0,
                                             const CUtensorMap* m1, int x0, int y0, int zz,
                                             int nz, unsigned mbar) {
    tma_load_4d(block0 + (unsigned)(I * seam_block_bytes<TW, BY>()), ex(I) == 0 ? m1 : m0,
                ex(I) < 0 ? x0 : x0 - 2, y0 - 1 - ey(I), wrap1(zz - ez(I), nz), I, mbar);
    TmaIssueSeamMain<TW, BY, I + 1>::run(block0, m0, m1, x0, y0, zz, nz, mbar);
  }
};
template <int TW, int BY>
struct TmaIssueSeamMain<TW, BY, 19> {
  __device__ __forceinline__ static void run(unsigned, const CUtensorMap*, const CUtensorMap*,
                                             int, int, int, int, unsigned) {}
};
// ... and, on a seam tile only, the strips a lane can read: x strip from
// source x = xs for the directions whose sources cross that seam (e_x >= 0
// at the low seam, xlo; e_x <= 0 at the high one), y strip from source y =
// ys likewise, the corner where both cross (xs or ys < 0: none).
template <int I>
__device__ __forceinline__ bool seam_crosses(int e, bool lo) {
  return lo ? e >= 0 : e <= 0;
}
template <int TW, int BY, int I>
struct TmaIssueStrips {
  __device__ __forceinline__ static void run(unsigned block0, const SeamStripMaps& sm, int x0,
                                             int y0, int zz, int nz, int xs, int ys, bool xlo,
                                             bool ylo, unsigned mbar) {
    constexpr int w = ex(I) == 0 ? TW + 2 : TW;
    const unsigned blk = block0 + (unsigned)(I * seam_block_bytes<TW, BY>());
    const int x = ex(I) < 0 ? x0 : x0 - 2;
    const int y = y0 - 1 - ey(I);
    const int z = wrap1(zz - ez(I), nz);
    const bool cx = xs >= 0 && seam_crosses<I>(ex(I), xlo);
    const bool cy = ys >= 0 && seam_crosses<I>(ey(I), ylo);
    if (cx) tma_load_4d(blk + seam_xs_off<TW, BY>(w), sm.xs, xs, y, z, I, mbar);
    if (cy)
      tma_load_4d(blk + seam_ys_off<TW, BY>(w), ex(I) == 0 ? sm.ys1 : sm.ys0, x, ys, z, I, mbar);
    if (cx && cy) tma_load_4d(blk + seam_cs_off<TW, BY>(w), sm.cs, xs, ys, z, I, mbar);
    TmaIssueStrips<TW, BY, I + 1>::run(block0, sm, x0, y0, zz, nz, xs, ys, xlo, ylo, mbar);
  }
};
template <int TW, int BY>
struct TmaIssueStrips<TW, BY, 19> {
  __device__ __forceinline__ static void run(unsigned, const SeamStripMaps&, int, int, int, int,
                                             int, int, bool, bool, unsigned) {}
};
// Bytes one plane's copies deliver on a tile with or without x / y strips
// (xlo / ylo: the tile's seam is the low one of its axis).
template <int TW, int BY>
__host__ __device__ constexpr int seam_tx_bytes(bool xstrip, bool ystrip, bool xlo, bool ylo) {
  int b = 0;
  for (int i = 0; i < 19; ++i) {
    const int w = ex(i) == 0 ? TW + 2 : TW;
    const bool cx = xstrip && (xlo ? ex(i) >= 0 : ex(i) <= 0);
    const bool cy = ystrip && (ylo ? ey(i) >= 0 : ey(i) <= 0);
    b += w * BY * 8;
    if (cx) b += 2 * BY * 8;
    if (cy) b += w * 2 * 8;
    if (cx && cy) b += 2 * 2 * 8;
  }
  return b;
}
// Byte offset, within a direction's block, of the pair a lane reads for a
// direction (ex, ey): its source cell (cx - ex, cy - ey) in the main box, or
// beyond a periodic seam in the x strip, the y strip or the corner.  Lanes
// whose source lies further out (beyond the ring, unused) read the main box.
template <int TW, int BY>
__device__ __forceinline__ unsigned seam_lane_off(int tx, int ty, int cx, int cy, int ex_,
                                                  int ey_, int nx, int ny) {
  const int w = ex_ == 0 ? TW + 2 : TW;
  const int col = tx + (ex_ == 0 ? 1 : 0);
  const int sx = cx - ex_, sy = cy - ey_;
  const bool xin = sx >= 0 && sx < nx, yin = sy >= 0 && sy < ny;
  const int xc = sx < 0 ? sx + 2 : sx - nx, yc = sy < 0 ? sy + 2 : sy - ny;
  // only lanes of the ring and the interior (whose moments are used) look
  // beyond a seam; the strips copied are the ones those lanes need
  const bool used = cx >= -1 && cx <= nx && cy >= -1 && cy <= ny;
  const bool xok = used && xc >= 0 && xc < 2, yok = used && yc >= 0 && yc < 2;
  int off = (ty * w + col) * 8;
  if (!xin && yin && xok) off = seam_xs_off<TW, BY>(w) + (ty * 2 + xc) * 8;
  if (xin && !yin && yok) off = seam_ys_off<TW, BY>(w) + (yc * w + col) * 8;
  if (!xin && !yin && xok && yok) off = seam_cs_off<TW, BY>(w) + (yc * 2 + xc) * 8;
  return (unsigned)off;
}
// SEAM form of StageReduce: the pair of direction I at its lane offset.
template <int TW, int BY, int I>
struct StageReduceSeam {
  __device__ __forceinline__ static void run(const unsigned char* stage, const unsigned* loff,
                                             float* f, float2& rho) {
    const float2 v = *reinterpret_cast<const float2*>(
        stage + I * seam_block_bytes<TW, BY>() + loff[(ex(I) + 1) * 3 + (ey(I) + 1)]);
    rho = __fadd2_rn(rho, v);
    f[I] = v.x + v.y;
    StageReduceSeam<TW, BY, I + 1>::run(stage, loff, f, rho);
  }
};
template <int TW, int BY>
struct StageReduceSeam<TW, BY, 19> {
  __device__ __forceinline__ static void run(const unsigned char*, const unsigned*, float*,
                                             float2&) {}
};

// 16-bit SEAM form, one thread: the main boxes of a plane (one map) ...
template <int TW, int BY, int I>
struct TmaIssueSeamMain16 {
  __device__ __forceinline__ static void run(unsigned block0, const CUtensorMap* m0, int x0,
                                             int y0, int zz, int nz, unsigned mbar) {
    tma_load_4d(block0 + (unsigned)(I * s16_block_bytes<TW, BY>()), m0, (x0 - 2) & ~3,
                y0 - 1 - ey(I), wrap1(zz - ez(I), nz), I, mbar);
    TmaIssueSeamMain16<TW, BY, I + 1>::run(block0, m0, x0, y0, zz, nz, mbar);
  }
};
template <int TW, int BY>
struct TmaIssueSeamMain16<TW, BY, 19> {
  __device__ __forceinline__ static void run(unsigned, const CUtensorMap*, int, int, int, int,
                                             unsigned) {}
};
// ... and, on a seam tile, the strips a lane can read (xs: first pair of the
// x strip, nx - 4 or 0; ys: first row of the y strip, ny - 2 or 0; < 0: none).
template <int TW, int BY, int I>
struct TmaIssueStrips16 {
  __device__ __forceinline__ static void run(unsigned block0, const SeamStripMaps& sm, int x0,
                                             int y0, int zz, int nz, int xs, int ys, bool xlo,
                                             bool ylo, unsigned mbar) {
    const unsigned blk = block0 + (unsigned)(I * s16_block_bytes<TW, BY>());
    const int y = y0 - 1 - ey(I);
    const int z = wrap1(zz - ez(I), nz);
    const bool cx = xs >= 0 && seam_crosses<I>(ex(I), xlo);
    const bool cy = ys >= 0 && seam_crosses<I>(ey(I), ylo);
    if (cx) tma_load_4d(blk + s16_xs_off<TW, BY>(), sm.xs, xs, y, z, I, mbar);
    if (cy) tma_load_4d(blk + s16_ys_off<TW, BY>(), sm.ys0, (x0 - 2) & ~3, ys, z, I, mbar);
    if (cx && cy) tma_load_4d(blk + s16_cs_off<TW, BY>(), sm.cs, xs, ys, z, I, mbar);
    TmaIssueStrips16<TW, BY, I + 1>::run(block0, sm, x0, y0, zz, nz, xs, ys, xlo, ylo, mbar);
  }
};
template <int TW, int BY>
struct TmaIssueStrips16<TW, BY, 19> {
  __device__ __forceinline__ static void run(unsigned, const SeamStripMaps&, int, int, int, int,
                                             int, int, bool, bool, unsigned) {}
};
template <int TW, int BY>
__host__ __device__ constexpr int seam16_tx_bytes(bool xstrip, bool ystrip, bool xlo, bool ylo) {
  int b = 0;
  for (int i = 0; i < 19; ++i) {
    const bool cx = xstrip && (xlo ? ex(i) >= 0 : ex(i) <= 0);
    const bool cy = ystrip && (ylo ? ey(i) >= 0 : ey(i) <= 0);
    b += s16_w<TW>() * BY * 4;
    if (cx) b += 4 * BY * 4;
    if (cy) b += s16_w<TW>() * 2 * 4;
    if (cx && cy) b += 4 * 2 * 4;
  }
  return b;
}
// Byte offset, within a direction's block, of the pair a lane reads for a
// direction (ex, ey) in the 16-bit SEAM form (see seam_lane_off).
template <int TW, int BY>
__device__ __forceinline__ unsigned seam16_lane_off(int tx, int ty, int cx, int cy, int ex_,
                                                    int ey_, int nx, int ny) {
  constexpr int W = s16_w<TW>();
  const int col = tx + 3 - ex_;  // the main box starts at x0 - 4 (x0 a multiple of 4)
  const int sx = cx - ex_, sy = cy - ey_;
  const bool xin = sx >= 0 && sx < nx, yin = sy >= 0 && sy < ny;
  const int xi = sx < 0 ? sx + 4 : sx - nx, yc = sy < 0 ? sy + 2 : sy - ny;
  const bool used = cx >= -1 && cx <= nx && cy >= -1 && cy <= ny;
  const bool xok = used && xi >= 0 && xi < 4, yok = used && yc >= 0 && yc < 2;
  int off = (ty * W + col) * 4;
  if (!xin && yin && xok) off = s16_xs_off<TW, BY>() + (ty * 4 + xi) * 4;
  if (xin && !yin && yok) off = s16_ys_off<TW, BY>() + (yc * W + col) * 4;
  if (!xin && !yin && xok && yok) off = s16_cs_off<TW, BY>() + (yc * 4 + xi) * 4;
  return (unsigned)off;
}
template <typename T, int TW, int BY, int I>
struct StageReduceSeam16 {
  __device__ __forceinline__ static void run(const unsigned char* stage, const unsigned* loff,
                                             const StepArgs& a, float* f, float2& rho) {
    using Pair = typename Store<T>::Pair;
    float2 v = Store<T>::to_float2(*reinterpret_cast<const Pair*>(
        stage + I * s16_block_bytes<TW, BY>() + loff[(ex(I) + 1) * 3 + (ey(I) + 1)]));
    add_offsets<T, I>(a, v);
    rho = __fadd2_rn(rho, v);
    f[I] = v.x + v.y;
    StageReduceSeam16<T, TW, BY, I + 1>::run(stage, loff, a, f, rho);
  }
};
template <typename T, int TW, int BY>
struct StageReduceSeam16<T, TW, BY, 19> {
  __device__ __forceinline__ static void run(const unsigned char*, const unsigned*,
                                             const StepArgs&, float*, float2&) {}
};

// Reads the 19 pairs of one cell from a stage, reduced on the fly to
// (f_i = fR_i + fB_i, rho_R, rho_B).  col0 = tx (FP32) or tx + 1 + o (16-bit).
template <typename T, int TW, int BY, int I>
struct StageReduce {
  __device__ __forceinline__ static void run(const unsigned char* stage, int ty, int col0,
                                             const StepArgs& a, float* f, float2& rho) {
    using Pair = typename Store<T>::Pair;
    int col;
    if constexpr (tma_pair_bytes<T>() == 8)
      col = col0 + (ex(I) == 0 ? 1 : 0);
    else
      col = col0 - ex(I);
    const Pair* box = reinterpret_cast<const Pair*>(stage + tma_box_off<T, TW, BY>(I));
    float2 v = Store<T>::to_float2(box[ty * tma_width<T, TW>(I) + col]);
    add_offsets<T, I>(a, v);
    rho = __fadd2_rn(rho, v);  // (rho_R, rho_B) as one paired add
    f[I] = v.x + v.y;
    StageReduce<T, TW, BY, I + 1>::run(stage, ty, col0, a, f, rho);
  }
};
template <typename T, int TW, int BY>
struct StageReduce<T, TW, BY, 19> {
  __device__ __forceinline__ static void run(const unsigned char*, int, int, const StepArgs&,
                                             float*, float2&) {}
};

// Thread -> cell of a TW x BY tile: the interior cells first, row by row
// (one tile row per warp when TW - 2 = 32), then the ring (top row, bottom
// row, left column, right column).  The collision runs only in interior
// cells, so its warps have every lane busy, and the ring's moment-only work
// fills warps of its own, which skip the collision.
template <int TW, int BY>
__device__ __forceinline__ void tile_cell(int L, int& tx, int& ty) {
  constexpr int IW = TW - 2, IH = BY - 2;
  if (L < IW * IH) {
    tx = 1 + L % IW;
    ty = 1 + L / IW;
    return;
  }
  int r = L - IW * IH;
  if (r < TW) {
    tx = r;
    ty = 0;
    return;
  }
  r -= TW;
  if (r < TW) {
    tx = r;
    ty = BY - 1;
    return;
  }
  r -= TW;
  tx = r < IH ? 0 : TW - 1;
  ty = 1 + (r < IH ? r : r - IH);
}
// The thread that issues a plane's tensor copies: the first ring thread (a
// ring warp has no collision to delay).
template <int TW, int BY>
__host__ __device__ constexpr int tma_issuer() {
  return (TW - 2) * (BY - 2);
}

// Monitored steps: each lane adds the diagnostics of its interior cell's
// state (the state the step reads) to FP32 sums in registers; every
// kMonFold planes (and after the last) each warp folds its lanes with FP32
// shuffles (paired adds) and lane 0 adds the fold into the warp's own slot
// of the CTA's record (FP32, the colour masses with Kahan compensation: no
// atomics and no FP64 -- the FP64 pipe is narrow on this GPU; a per-plane
// FP64 fold cost the step more than its collision).  After the chunk the
// kernel adds the slots in FP64 into the step's global record.  The
// momentum is the raw sum_i e_i f_i (the velocity without its half-force
// shift); a NaN or an infinity in any population reaches rho or u, so
// their finiteness marks the cell; rho^N is the cell's phase-field entry
// of the window.
constexpr int kMonWarps = 16;  // warps of the largest monitored CTA (34 x 15)
struct MonSlot {
  float s[8], c[8];  // sums and their Kahan compensations (MonAcc::d order)
  unsigned n[4];
  unsigned u2bits;
};
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
// A lane's sums over the planes since the warp last folded.  A lane keeps
// its column (x, y) over the chunk, so its red-mass moments in x and y are
// x and y times its red mass: only the z moment has a sum of its own.
constexpr int kMonFold = 4;  // planes per fold (the packed counts stay below 256)
struct MonLane {
  float2 p[3] = {};   // (red mass, blue mass), (momentum x, y), (momentum z, sum rho_R z)
  unsigned cnt = 0u;  // bytes: non-finite, rho <= 0, red, a colour < 0
  float u2 = 0.f;     // largest finite |u|^2
};
__device__ __forceinline__ void monitor_lane_add(MonLane& l, const Macro& m, float phi, int z) {
  const bool finite = isfinite(m.rho) && isfinite(m.ux) && isfinite(m.uy) && isfinite(m.uz);
  l.p[0] = __fadd2_rn(l.p[0], make_float2(m.rR, m.rB));
  l.p[1] = __fadd2_rn(l.p[1], make_float2(m.rho * m.ux - 0.5f * m.Fx,
                                          m.rho * m.uy - 0.5f * m.Fy));
  l.p[2] = __fadd2_rn(l.p[2], make_float2(m.rho * m.uz - 0.5f * m.Fz, m.rR * (float)z));
  l.cnt += (finite ? 0u : 1u) | ((m.rho <= 0.f ? 1u : 0u) << 8) |
           ((phi > 0.f ? 1u : 0u) << 16) | ((m.rR < 0.f || m.rB < 0.f ? 1u : 0u) << 24);
  if (finite) l.u2 = fmaxf(l.u2, m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
}
// Folds the warp's lanes (x, y: the lane's column; a lane without interior
// cells has zero sums) into its slot and clears the lanes' sums; every lane
// of the warp calls it.  The CTA's last warp can be partial (34 x 12 and
// 34 x 15 threads): its missing lanes count as exited, which the full-mask
// shuffles allow, but a lane whose partner is missing reads an undefined
// value, so that warp's fold -- ring cells only, whose sums are zero -- is
// not stored.  nthreads: the CTA's threads.
__device__ __forceinline__ void monitor_fold(MonSlot* slots, MonLane& l, int x, int y,
                                             int tid, int nthreads) {
  constexpr unsigned full = 0xffffffffu;
  float2 q[4] = {l.p[0], l.p[1], make_float2(l.p[2].x, l.p[0].x * (float)x),
                 make_float2(l.p[0].x * (float)y, l.p[2].y)};
  // the fold in pairs: two shuffles and one paired FP32 add per pair
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      q[k] = __fadd2_rn(q[k], make_float2(__shfl_xor_sync(full, q[k].x, off),
                                          __shfl_xor_sync(full, q[k].y, off)));
  // the four counts of a warp (at most 32 kMonFold each) fit their bytes
  const unsigned cnt = __reduce_add_sync(full, l.cnt);
  const unsigned ub = __reduce_max_sync(full, __float_as_uint(l.u2));
  if ((tid & 31) == 0 && (tid & ~31) + 32 <= nthreads) {
    MonSlot& w = slots[tid >> 5];
    // compensated adds for the colour masses, whose drift is what a monitor
    // watches; plain FP32 adds for the rest
    kahan_add(w.s[0], w.c[0], q[0].x);
    kahan_add(w.s[1], w.c[1], q[0].y);
    w.s[2] += q[1].x;
    w.s[3] += q[1].y;
    w.s[4] += q[2].x;
    w.s[5] += q[2].y;
    w.s[6] += q[3].x;
    w.s[7] += q[3].y;
#pragma unroll
    for (int k = 0; k < 4; ++k) w.n[k] += (cnt >> (8 * k)) & 0xffu;
    w.u2bits = max(w.u2bits, ub);
  }
  l = MonLane();
}
// The CTA's record (kMonWarps slots): cleared before the chunk, added into
// the step's global record after it (both bracketed by the kernel's
// barriers).
__device__ __forceinline__ void monitor_clear(MonSlot* slots, int tid) {
  for (int i = tid; i < kMonWarps; i += 32) {
    MonSlot& w = slots[i];
    for (int k = 0; k < 8; ++k) w.s[k] = w.c[k] = 0.f;
    for (int k = 0; k < 4; ++k) w.n[k] = 0u;
    w.u2bits = 0u;
  }
}
__device__ __forceinline__ void monitor_flush(const MonSlot* slots, MonAcc* g, int tid) {
  if (tid < 8) {
    double v = 0.0;
    for (int w = 0; w < kMonWarps; ++w) v += (double)slots[w].s[tid] - (double)slots[w].c[tid];
    atomicAdd(&g->d[tid], v);
  } else if (tid < 12) {
    unsigned v = 0u;
    for (int w = 0; w < kMonWarps; ++w) v += slots[w].n[tid - 8];
    atomicAdd(&g->n[tid - 8], v);
  } else if (tid == 12) {
    unsigned v = 0u;
    for (int w = 0; w < kMonWarps; ++w) v = max(v, slots[w].u2bits);
    atomicMax(&g->u2bits, v);
  }
}

// One work item of the TMA-staged step: tile (bx, by) of the lattice `a`,
// planes [zb, ze).  The CTA's stage mbarriers are initialised; G0 counts
// the fills of the CTA's earlier items (their stage use), so that the
// stages and mbarrier phases continue across items.  map0 / map1: the
// source buffer's tensor maps (param or global space).  Returns false after
// a wait gave up (*err set, the CTA's copies drained).
// FALLBACK (SEAM form, batches): a tile that spans both seams of an axis
// (a case narrower than the tile's interior) gets the strips of its low
// seam only; its lanes whose sources lie beyond the high seam pull from
// global memory.
template <typename T, bool WALLS, int TW, int BY, int NS, bool SEAM = false,
          bool FALLBACK = false, bool MON = false>
__device__ __forceinline__ bool tma_chunk(const T* __restrict__ src, T* __restrict__ dst,
                                          const StepArgs& a, const CUtensorMap* map0,
                                          const CUtensorMap* map1, int bx, int by, int zb,
                                          int ze, unsigned char* smem, unsigned G0,
                                          int* __restrict__ err, unsigned long long wait_ns,
                                          const SeamStripMaps* strips = nullptr,
                                          MonSlot* mon = nullptr) {
  static_assert(!SEAM || tma_pair_bytes<T>() == 8 || (TW - 2) % 4 == 0,
                "the 16-bit SEAM form needs tile columns on 16-byte boundaries");
  constexpr int SB = tma_stage_bytes<T, TW, BY, SEAM>();
  constexpr int HV = tma_hold_vals<T, TW, BY, NS, SEAM>();
  using Pair = typename Store<T>::Pair;
  unsigned char* stage0 = smem;
  float4(*win)[BY][TW] = reinterpret_cast<float4(*)[BY][TW]>(smem + NS * SB);
  float(*hold)[BY - 2][TW - 2] =
      reinterpret_cast<float(*)[BY - 2][TW - 2]>(smem + NS * SB + tma_win_bytes<TW, BY>());
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(
      smem + NS * SB + tma_win_bytes<TW, BY>() + tma_hold_bytes<TW, BY>(HV));

  const int tid = threadIdx.y * TW + threadIdx.x;
  int tx, ty;
  tile_cell<TW, BY>(tid, tx, ty);
  const Geometry<WALLS, BY, TW> g(a, tx, ty, bx, by);
  const unsigned plane = (unsigned)a.plane;
  const Pair* srcp = reinterpret_cast<const Pair*>(src);
  const int x0 = bx * (TW - 2), y0 = by * (BY - 2);
  // every source x - e_i, y - e_i of this column lies inside the lattice
  const bool col_fast = g.cx >= 1 && g.cx <= a.nx - 2 && g.cy >= 1 && g.cy <= a.ny - 2;
  // SEAM form: strip sources of this tile (< 0: none) and the lane's nine
  // offsets; the copies deliver TX bytes per plane
  int TX = tma_stage_tx_bytes<T, TW, BY>();
  int seam_xs = -1, seam_ys = -1;
  unsigned loff[9];
  if constexpr (SEAM && tma_pair_bytes<T>() == 8) {
    const int cx = x0 - 1 + tx, cy = y0 - 1 + ty;
    if (x0 < 2) seam_xs = a.nx - 2;
    else if (x0 + TW - 2 >= a.nx - 1) seam_xs = 0;
    if (y0 < 2) seam_ys = a.ny - 2;
    else if (y0 + BY - 2 >= a.ny - 1) seam_ys = 0;
    TX = seam_tx_bytes<TW, BY>(seam_xs >= 0, seam_ys >= 0, x0 < 2, y0 < 2);
#pragma unroll
    for (int e = 0; e < 9; ++e)
      loff[e] = seam_lane_off<TW, BY>(tx, ty, cx, cy, e / 3 - 1, e % 3 - 1, a.nx, a.ny);
  } else if constexpr (SEAM) {  // 16-bit pairs: strips four pairs wide
    const int cx = x0 - 1 + tx, cy = y0 - 1 + ty;
    if (x0 < 2) seam_xs = a.nx - 4;
    else if (x0 + TW - 2 >= a.nx - 1) seam_xs = 0;
    if (y0 < 2) seam_ys = a.ny - 2;
    else if (y0 + BY - 2 >= a.ny - 1) seam_ys = 0;
    TX = seam16_tx_bytes<TW, BY>(seam_xs >= 0, seam_ys >= 0, x0 < 2, y0 < 2);
#pragma unroll
    for (int e = 0; e < 9; ++e)
      loff[e] = seam16_lane_off<TW, BY>(tx, ty, cx, cy, e / 3 - 1, e % 3 - 1, a.nx, a.ny);
  }
  bool lane_global = false;
  if constexpr (SEAM && FALLBACK) {
    const int cx = x0 - 1 + tx, cy = y0 - 1 + ty;
    lane_global = (x0 < 2 && x0 + TW - 2 >= a.nx - 1 && cx >= a.nx - 1) ||
                  (y0 < 2 && y0 + BY - 2 >= a.ny - 1 && cy >= a.ny - 1);
  }
  int col0 = tx;
  if constexpr (tma_pair_bytes<T>() != 8) col0 = tx + 1 + ((x0 - 2) - ((x0 - 2) & ~3));
  const unsigned st_base = smem_addr(stage0), mb_base = smem_addr(mbar);
  // fill k of this item is the CTA's fill G0 + k: its stage and the parity
  // of the mbarrier phase it completes
  auto stage_of = [&](int k) { return NS == 2 ? (int)((G0 + (unsigned)k) & 1u) : 0; };
  auto st_addr = [&](int k) { return st_base + (unsigned)(stage_of(k) * SB); };
  auto mb = [&](int k) { return mb_base + 8u * (unsigned)stage_of(k); };
  auto par = [&](int k) {
    const unsigned n = G0 + (unsigned)k;
    return (NS == 2 ? n >> 1 : n) & 1u;
  };

  // fill index k = plane zb - 1 + k; with walls in z the first and last
  // plane are pulled from global memory (bounce-back links) and get no copies
  const int K = ze - zb + 2;
  auto staged = [&](int zl) {
    if (!(WALLS && a.wz)) return true;
    return zl >= 1 && zl <= a.nz - 2;
  };
  auto issue_one = [&](int k) {  // one thread
    const int zl = zb - 1 + k;
    const unsigned m = mb(k);
#ifdef LBM_CHECKED
    // the copies' x coordinates (x0 and x0 - 2 for 8-byte pairs, rounded
    // down to 4 pairs for 4-byte pairs; the seam strips' from nx) must start
    // on 16 bytes: a misaligned one is counted and its plane not copied
    // (the stage wait then gives up and reports)
    if (tma_pair_bytes<T>() == 8 ? ((x0 & 1) != 0 || (SEAM && (a.nx & 1) != 0))
                                 : (SEAM && (a.nx & 3) != 0)) {
      index_ok(a, 1, 0);
      return;
    }
#endif
    if (staged(zl)) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(m),
                   "r"(TX)
                   : "memory");
      if constexpr (SEAM && tma_pair_bytes<T>() == 8) {
        TmaIssueSeamMain<TW, BY, 0>::run(st_addr(k), map0, map1, x0, y0, wrap1(zl, a.nz), a.nz,
                                         m);
        if (seam_xs >= 0 || seam_ys >= 0)
          TmaIssueStrips<TW, BY, 0>::run(st_addr(k), *strips, x0, y0, wrap1(zl, a.nz), a.nz,
                                         seam_xs, seam_ys, x0 < 2, y0 < 2, m);
      } else if constexpr (SEAM) {
        TmaIssueSeamMain16<TW, BY, 0>::run(st_addr(k), map0, x0, y0, wrap1(zl, a.nz), a.nz, m);
        if (seam_xs >= 0 || seam_ys >= 0)
          TmaIssueStrips16<TW, BY, 0>::run(st_addr(k), *strips, x0, y0, wrap1(zl, a.nz), a.nz,
                                           seam_xs, seam_ys, x0 < 2, y0 < 2, m);
      } else {
        TmaIssue<T, TW, BY, 0>::run(st_addr(k), map0, map1, x0, y0, wrap1(zl, a.nz), a.nz, m);
      }
    } else {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(m) : "memory");
    }
  };
  auto issue = [&](int k) {
    if (tid == tma_issuer<TW, BY>()) issue_one(k);
  };
  // Pulls plane zl: window slot and reduced state (f, rho_R, rho_B, u).
  auto fill = [&](int k, float* f, float* hu) {
    const int zl = zb - 1 + k;
    if (!g.plane_ok(a, zl)) return;
    float rR = 0.f, rB = 0.f;
    bool from_stage = false;
    if constexpr (SEAM) {
      // every lane (the first and last plane of z walls: global)
      if (staged(zl) && !lane_global) {
        float2 rho = make_float2(0.f, 0.f);
        if constexpr (tma_pair_bytes<T>() == 8)
          StageReduceSeam<TW, BY, 0>::run(stage0 + stage_of(k) * SB, loff, f, rho);
        else
          StageReduceSeam16<T, TW, BY, 0>::run(stage0 + stage_of(k) * SB, loff, a, f, rho);
        rR = rho.x;
        rB = rho.y;
        from_stage = true;
      }
    } else {
      if (col_fast && staged(zl)) {
        float2 rho = make_float2(0.f, 0.f);
        StageReduce<T, TW, BY, 0>::run(stage0 + stage_of(k) * SB, ty, col0, a, f, rho);
        rR = rho.x;
        rB = rho.y;
        from_stage = true;
      }
    }
    if (!from_stage)
      pull_reduce<T, WALLS>(srcp, plane, a, g.co, g.plane(a, wrap1(zl, a.nz)), f, rR, rB);
    const Macro m = macro_total(a, f, rR, rB);
    hu[0] = rR;
    hu[1] = rB;
    hu[2] = m.ux;
    hu[3] = m.uy;
    hu[4] = m.uz;
    win[zl & 3][ty][tx] = stencil_entry(a, m);
  };
  // after a failed wait: the copies of fills k .. k + NS - 1 may be in flight
  auto drain = [&](int k) {
    if (tid == tma_issuer<TW, BY>()) atomicExch(err, 1);
    for (int j = k; j < k + NS && j < K; ++j) tma_wait(mb(j), par(j), kTmaWaitNs);
  };

  float cf[19], ch[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  if constexpr (NS == 2) {
    issue(0);
    issue(1);
    float tf[19], th[5];
    bool ok = tma_wait(mb(0), par(0), wait_ns);
    if (ok) fill(0, tf, th);
    ok = ok && tma_wait(mb(1), par(1), wait_ns);
    if (ok) fill(1, cf, ch);
    if (!__syncthreads_and(ok ? 1 : 0)) {
      drain(0);
      return false;
    }
    if (K > 2) issue(2);
    if (K > 3) issue(3);
  } else {
    issue(0);
    float tf[19], th[5];
    bool ok = tma_wait(mb(0), par(0), wait_ns);
    if (ok) fill(0, tf, th);
    if (!__syncthreads_and(ok ? 1 : 0)) {
      drain(0);
      return false;
    }
    issue(1);
    ok = tma_wait(mb(1), par(1), wait_ns);
    if (ok) fill(1, cf, ch);
    if (!__syncthreads_and(ok ? 1 : 0)) {
      drain(1);
      return false;
    }
    if (K > 2) issue(2);
  }
  MonLane ml;  // monitored form: this lane's sums since the last fold
  for (int k = 2; k < K; ++k) {
    const int z = zb + k - 2;  // plane that collides; plane z + 1 is filled
    float nf[19], nh[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const bool got = tma_wait(mb(k), par(k), wait_ns);
    if (got) {
      fill(k, nf, nh);
      if (g.interior) {  // private slot of this thread
#pragma unroll
        for (int i = 0; i < 19; ++i) hold[i][ty - 1][tx - 1] = nf[i];
#pragma unroll
        for (int i = 0; i < HV - 19; ++i) hold[19 + i][ty - 1][tx - 1] = nh[i];
      }
    }
    if (!__syncthreads_and(got ? 1 : 0)) {
      drain(k);
      return false;
    }
    // the stage of fill k is consumed by every thread: refill it
    if (k + NS < K) issue(k + NS);
    if (g.interior) {
      const bool zlo = WALLS && a.wz && z == 0, zhi = WALLS && a.wz && z == a.nz - 1;
      float4 ctr;
      float Gx, Gy, Gz, Qx, Qy, Qz;
      window_gradients<BY, TW>(win, z, ty, tx, g.xlo, g.xhi, g.ylo, g.yhi, zlo, zhi, ctr, Gx,
                               Gy, Gz, Qx, Qy, Qz);
      if (WALLS && a.wetting)
        wetting_rule(a, g.xlo, g.xhi, g.ylo, g.yhi, zlo, zhi, Gx, Gy, Gz);
      const Macro m = HV == 24 ? macro_held(a, ch[0], ch[1], ch[2], ch[3], ch[4])
                               : macro_total(a, cf, ch[0], ch[1]);
      if constexpr (MON) monitor_lane_add(ml, m, ctr.x, z);
      const Recolour rc = collide_total<false>(a, cf, m, ctr.x, Gx, Gy, Gz, Qx, Qy, Qz);
      store_recoloured<T>(dst, plane, a, (unsigned)z * g.plane_cells + g.co.yo[1] + g.co.xo[1],
                          rc, cf);
#pragma unroll
      for (int i = 0; i < 19; ++i) cf[i] = hold[i][ty - 1][tx - 1];
#pragma unroll
      for (int i = 0; i < HV - 19; ++i) ch[i] = hold[19 + i][ty - 1][tx - 1];
    }
    if constexpr (MON)
      if ((k - 2) % kMonFold == kMonFold - 1 || k == K - 1)
        monitor_fold(mon, ml, g.cx, g.cy, tid, TW * BY);
  }
  return true;
}

__device__ __forceinline__ void tma_init_barriers(unsigned char* mbar_bytes, int ns) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    for (int q = 0; q < ns; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(mbar_bytes + 8 * q))
                   : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
}

template <typename T, int TW, int BY, int NS, bool SEAM = false>
__device__ __forceinline__ unsigned char* tma_mbar_bytes(unsigned char* smem) {
  return smem + NS * tma_stage_bytes<T, TW, BY, SEAM>() + tma_win_bytes<TW, BY>() +
         tma_hold_bytes<TW, BY>(tma_hold_vals<T, TW, BY, NS, SEAM>());
}

template <typename T, bool WALLS, int TW, int BY, int NS>
__global__ void __launch_bounds__(TW* BY, (tma_ctas_per_sm<TW, BY>()))
    k_fused_tma(const T* __restrict__ src, T* __restrict__ dst,
                const __grid_constant__ StepArgs a, const __grid_constant__ CUtensorMap map0,
                const __grid_constant__ CUtensorMap map1, int zchunk, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int zb = blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, a.nz);
  if (zb >= ze) return;
  if (smem_addr(smem) & 127u) {  // the copies need 128-byte aligned boxes
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(err, 2);
    return;
  }
  tma_init_barriers(tma_mbar_bytes<T, TW, BY, NS>(smem), NS);
  __syncthreads();
  tma_chunk<T, WALLS, TW, BY, NS>(src, dst, a, &map0, &map1, blockIdx.x, blockIdx.y, zb, ze,
                                  smem, 0u, err, tma_wait_limit());
}

// SEAM form (FP32, periodic in x and y, one stage): the source buffer's six
// tensor maps (main TW, main TW + 2, x strip, y strip TW, y strip TW + 2,
// corner), each a kernel parameter of its own like the other forms' maps.
// MON: also the diagnostics of the state read, added into *gmon.
template <int TW, int BY, int NS, bool WALLS, bool MON = false>
__global__ void __launch_bounds__(TW* BY, 1)
    k_fused_tma_seam(const float* __restrict__ src, float* __restrict__ dst,
                     const __grid_constant__ StepArgs a,
                     const __grid_constant__ CUtensorMap map0,
                     const __grid_constant__ CUtensorMap map1,
                     const __grid_constant__ CUtensorMap mxs,
                     const __grid_constant__ CUtensorMap mys0,
                     const __grid_constant__ CUtensorMap mys1,
                     const __grid_constant__ CUtensorMap mcs, int zchunk,
                     int* __restrict__ err, MonAcc* __restrict__ gmon) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int zb = blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, a.nz);
  if (zb >= ze) return;
  if (smem_addr(smem) & 127u) {  // the copies need 128-byte aligned blocks
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(err, 2);
    return;
  }
  const int tid = threadIdx.y * TW + threadIdx.x;
  MonSlot* macc = nullptr;  // the CTA's record, a slot per warp (monitored form only)
  if constexpr (MON) {
    static_assert(TW * BY <= 32 * kMonWarps, "one record slot per warp");
    __shared__ MonSlot macc_s[kMonWarps];
    macc = macc_s;
    if (tid < 32) monitor_clear(macc, tid);
  }
  tma_init_barriers(tma_mbar_bytes<float, TW, BY, NS, true>(smem), NS);
  __syncthreads();
  const SeamStripMaps strips = {&mxs, &mys0, &mys1, &mcs};
  const bool ok = tma_chunk<float, WALLS, TW, BY, NS, true, false, MON>(
      src, dst, a, &map0, &map1, blockIdx.x, blockIdx.y, zb, ze, smem, 0u, err,
      tma_wait_limit(), &strips, macc);
  if constexpr (MON) {
    __syncthreads();
    if (ok) monitor_flush(macc, gmon, tid);
  }
}

template <int TW, int BY, int NS, bool WALLS, bool MON = false>
static cudaError_t launch_tma_seam_v(const void* src, void* dst, const StepArgs& a,
                                     const CUtensorMap* maps6, int zc, int* err,
                                     cudaStream_t s, MonAcc* mon = nullptr) {
  static_assert(tma_fits<float, TW, BY, NS, true>(), "SEAM stages do not fit");
  static bool attr_set[kMaxDevices] = {};
  const int dv = device_slot();
  constexpr int bytes = tma_smem_bytes<float, TW, BY, NS, true>();
  if (!attr_set[dv]) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_tma_seam<TW, BY, NS, WALLS, MON>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set[dv] = true;
  }
  dim3 blk(TW, BY);
  dim3 grd((a.nx + TW - 3) / (TW - 2), (a.ny + BY - 3) / (BY - 2), (a.nz + zc - 1) / zc);
  k_fused_tma_seam<TW, BY, NS, WALLS, MON><<<grd, blk, bytes, s>>>(
      (const float*)src, (float*)dst, a, maps6[0], maps6[1], maps6[2], maps6[3], maps6[4],
      maps6[5], zc, err, mon);
  return cudaGetLastError();
}

// 16-bit SEAM form (FP16 / BF16 deviation storage, periodic in x and y,
// walls in z allowed): the source buffer's four maps (main W16 x BY, x strip
// 4 x BY, y strip W16 x 2, corner 4 x 2) as kernel parameters.
template <typename T, int TW, int BY, int NS, bool WALLS, bool MON = false>
__global__ void __launch_bounds__(TW* BY, 1)
    k_fused_tma_seam16(const T* __restrict__ src, T* __restrict__ dst,
                       const __grid_constant__ StepArgs a,
                       const __grid_constant__ CUtensorMap map0,
                       const __grid_constant__ CUtensorMap mxs,
                       const __grid_constant__ CUtensorMap mys,
                       const __grid_constant__ CUtensorMap mcs, int zchunk,
                       int* __restrict__ err, MonAcc* __restrict__ gmon) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int zb = blockIdx.z * zchunk;
  const int ze = min(zb + zchunk, a.nz);
  if (zb >= ze) return;
  if (smem_addr(smem) & 127u) {  // the copies need 128-byte aligned blocks
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(err, 2);
    return;
  }
  const int tid = threadIdx.y * TW + threadIdx.x;
  MonSlot* macc = nullptr;  // the CTA's record, a slot per warp (monitored form only)
  if constexpr (MON) {
    static_assert(TW * BY <= 32 * kMonWarps, "one record slot per warp");
    __shared__ MonSlot macc_s[kMonWarps];
    macc = macc_s;
    if (tid < 32) monitor_clear(macc, tid);
  }
  tma_init_barriers(tma_mbar_bytes<T, TW, BY, NS, true>(smem), NS);
  __syncthreads();
  const SeamStripMaps strips = {&mxs, &mys, &mys, &mcs};
  const bool ok = tma_chunk<T, WALLS, TW, BY, NS, true, false, MON>(
      src, dst, a, &map0, &map0, blockIdx.x, blockIdx.y, zb, ze, smem, 0u, err,
      tma_wait_limit(), &strips, macc);
  if constexpr (MON) {
    __syncthreads();
    if (ok) monitor_flush(macc, gmon, tid);
  }
}

template <typename T, int TW, int BY, int NS, bool WALLS, bool MON = false>
static cudaError_t launch_tma_seam16_v(const void* src, void* dst, const StepArgs& a,
                                       const CUtensorMap* maps4, int zc, int* err,
                                       cudaStream_t s, MonAcc* mon = nullptr) {
  static_assert(tma_fits<T, TW, BY, NS, true>(), "16-bit SEAM stages do not fit");
  static bool attr_set[kMaxDevices] = {};
  const int dv = device_slot();
  constexpr int bytes = tma_smem_bytes<T, TW, BY, NS, true>();
  if (!attr_set[dv]) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_tma_seam16<T, TW, BY, NS, WALLS, MON>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set[dv] = true;
  }
  dim3 blk(TW, BY);
  dim3 grd((a.nx + TW - 3) / (TW - 2), (a.ny + BY - 3) / (BY - 2), (a.nz + zc - 1) / zc);
  k_fused_tma_seam16<T, TW, BY, NS, WALLS, MON><<<grd, blk, bytes, s>>>(
      (const T*)src, (T*)dst, a, maps4[0], maps4[1], maps4[2], maps4[3], zc, err, mon);
  return cudaGetLastError();
}

// 16-bit SEAM forms: tile_y 15 (34 x 15) or 12 (34 x 12), two stages.
template <typename T>
cudaError_t launch_fused_tma_seam16_storage(const void* src, void* dst, const StepArgs& a,
                                            int tile_y, const CUtensorMap* maps4, int zchunk,
                                            int* err, cudaStream_t s, MonAcc* mon) {
  const int zc = zchunk > 0 ? zchunk : a.nz;
  const bool zwalls = a.wz != 0;
  if (mon) {  // monitored form: the default 34 x 15 tile only
    if (tile_y != 15) return cudaErrorInvalidValue;
    return zwalls ? launch_tma_seam16_v<T, 34, 15, 2, true, true>(src, dst, a, maps4, zc, err,
                                                                 s, mon)
                  : launch_tma_seam16_v<T, 34, 15, 2, false, true>(src, dst, a, maps4, zc,
                                                                  err, s, mon);
  }
  if (tile_y == 15)
    return zwalls ? launch_tma_seam16_v<T, 34, 15, 2, true>(src, dst, a, maps4, zc, err, s)
                  : launch_tma_seam16_v<T, 34, 15, 2, false>(src, dst, a, maps4, zc, err, s);
  if (tile_y == 12)
    return zwalls ? launch_tma_seam16_v<T, 34, 12, 2, true>(src, dst, a, maps4, zc, err, s)
                  : launch_tma_seam16_v<T, 34, 12, 2, false>(src, dst, a, maps4, zc, err, s);
  return cudaErrorInvalidValue;
}

// Batched TMA step: persistent CTAs take the work items (case, z chunk,
// tile row, tile column) -- tile column fastest, so that CTAs running at
// the same time march neighbouring tiles of one chunk and share their halo
// lines in L2.  Per item the case's StepArgs are copied to shared memory;
// its tensor maps come from a device table (two per case for the source
// buffer), made visible to the tensor-map proxy before use.
template <typename T, bool WALLS, int TW, int BY, int NS>
__global__ void __launch_bounds__(TW* BY, (tma_ctas_per_sm<TW, BY>()))
    k_fused_tma_batch(const BatchCase* __restrict__ cases, int ncases, int total_items,
                      const CUtensorMap* __restrict__ maps, const T* __restrict__ src_base,
                      T* __restrict__ dst_base, int zchunk, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ StepArgs sa;
  __shared__ int s_case, s_item;
  if (smem_addr(smem) & 127u) {
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(err, 2);
    return;
  }
  tma_init_barriers(tma_mbar_bytes<T, TW, BY, NS>(smem), NS);
  const unsigned long long wait_ns = tma_wait_limit();
  unsigned G0 = 0;
  for (int w = blockIdx.x; w < total_items; w += gridDim.x) {
    __syncthreads();  // the previous item is done with the shared state
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
      const CUtensorMap* m = maps + 2 * lo;
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(m)
                   : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(m + 1)
                   : "memory");
    }
    __syncthreads();
    const BatchCase& bc = cases[s_case];
    const int item = s_item;
    const int bx = item % bc.tiles_x, rest = item / bc.tiles_x;
    const int by = rest % bc.tiles_y, chunk = rest / bc.tiles_y;
    const int zb = chunk * zchunk;
    const int ze = min(zb + zchunk, sa.nz);
    const size_t off = 2 * (size_t)bc.pair_base;
    if (!tma_chunk<T, WALLS, TW, BY, NS>(src_base + off, dst_base + off, sa, maps + 2 * s_case,
                                         maps + 2 * s_case + 1, bx, by, zb, ze, smem, G0, err,
                                         wait_ns))
      return;
    G0 += (unsigned)(ze - zb + 2);
  }
}

// Batched SEAM step (FP32, every case periodic in x and y): as
// k_fused_tma_batch on the 34 x 12 tile with two stages, the six seam maps
// of each case (main 34 and 36 wide, x strip, y strips, corner) from a
// device table, six per case; cases narrower than the tile run through the
// FALLBACK lanes.
template <bool WALLS>
__global__ void __launch_bounds__(34 * 12, 1)
    k_fused_tma_seam_batch(const BatchCase* __restrict__ cases, int ncases, int total_items,
                           const CUtensorMap* __restrict__ maps, const float* __restrict__ src_base,
                           float* __restrict__ dst_base, int zchunk, int* __restrict__ err) {
  constexpr int TW = 34, BY = 12, NS = 2;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ StepArgs sa;
  __shared__ int s_case, s_item;
  if (smem_addr(smem) & 127u) {
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicExch(err, 2);
    return;
  }
  tma_init_barriers(tma_mbar_bytes<float, TW, BY, NS, true>(smem), NS);
  const unsigned long long wait_ns = tma_wait_limit();
  unsigned G0 = 0;
  for (int w = blockIdx.x; w < total_items; w += gridDim.x) {
    __syncthreads();  // the previous item is done with the shared state
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
      const CUtensorMap* m = maps + 6 * lo;
      for (int q = 0; q < 6; ++q)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(m + q)
                     : "memory");
    }
    __syncthreads();
    const BatchCase& bc = cases[s_case];
    const int item = s_item;
    const int bx = item % bc.tiles_x, rest = item / bc.tiles_x;
    const int by = rest % bc.tiles_y, chunk = rest / bc.tiles_y;
    const int zb = chunk * zchunk;
    const int ze = min(zb + zchunk, sa.nz);
    const size_t off = 2 * (size_t)bc.pair_base;
    const CUtensorMap* m = maps + 6 * s_case;
    const SeamStripMaps strips = {m + 2, m + 3, m + 4, m + 5};
    if (!tma_chunk<float, WALLS, TW, BY, NS, true, true>(src_base + off, dst_base + off, sa,
                                                         m, m + 1, bx, by, zb, ze, smem, G0,
                                                         err, wait_ns, &strips))
      return;
    G0 += (unsigned)(ze - zb + 2);
  }
}

template <bool WALLS>
static cudaError_t launch_tma_seam_batch_v(const void* src, void* dst, const BatchCase* cases,
                                           int ncases, int total_items, const CUtensorMap* maps,
                                           int zc, int* err, int sms, cudaStream_t s) {
  static_assert(tma_fits<float, 34, 12, 2, true>(), "SEAM stages do not fit");
  static bool attr_set[kMaxDevices] = {};
  const int dv = device_slot();
  constexpr int bytes = tma_smem_bytes<float, 34, 12, 2, true>();
  if (!attr_set[dv]) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_tma_seam_batch<WALLS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    attr_set[dv] = true;
  }
  // one CTA per work item: the hardware hands the next item to whichever
  // SM frees first (a persistent grid taking items round-robin ran the
  // 512-case droplet sweep 20-30 % slower: its static shares of unequal
  // items end unevenly)
  const int grid = total_items;
  (void)sms;
  k_fused_tma_seam_batch<WALLS><<<grid, dim3(34, 12), bytes, s>>>(
      cases, ncases, total_items, maps, (const float*)src, (float*)dst, zc, err);
  return cudaGetLastError();
}

// Tensor maps are built on the host (lbm_dispatch.cu); the launcher only
// sets the dynamic shared-memory limit once per instantiation.
template <typename T, bool WALLS, int TW, int BY, int NS>
static cudaError_t launch_tma_v(const void* src, void* dst, const StepArgs& a,
                                const CUtensorMap* maps, int zc, int* err, cudaStream_t s) {
  if constexpr (!tma_fits<T, TW, BY, NS>()) {
    return cudaErrorInvalidValue;
  } else {
    static bool attr_set[kMaxDevices] = {};
    const int dv = device_slot();
    constexpr int bytes = tma_smem_bytes<T, TW, BY, NS>();
    if (!attr_set[dv]) {
      cudaError_t e = cudaFuncSetAttribute(k_fused_tma<T, WALLS, TW, BY, NS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e != cudaSuccess) return e;
      attr_set[dv] = true;
    }
    dim3 blk(TW, BY);
    dim3 grd((a.nx + TW - 3) / (TW - 2), (a.ny + BY - 3) / (BY - 2), (a.nz + zc - 1) / zc);
    k_fused_tma<T, WALLS, TW, BY, NS><<<grd, blk, bytes, s>>>((const T*)src, (T*)dst, a, maps[0],
                                                             maps[1], zc, err);
    return cudaGetLastError();
  }
}

template <typename T, bool WALLS>
static cudaError_t launch_tma_w(const void* src, void* dst, const StepArgs& a,
                                const CUtensorMap* maps, int kind, int ns, int zc, int* err,
                                cudaStream_t s) {
  switch (kind * 2 + (ns - 1)) {
    case 0: return launch_tma_v<T, WALLS, 32, 8, 1>(src, dst, a, maps, zc, err, s);
    case 1: return launch_tma_v<T, WALLS, 32, 8, 2>(src, dst, a, maps, zc, err, s);
    case 2: return launch_tma_v<T, WALLS, 16, 16, 1>(src, dst, a, maps, zc, err, s);
    case 3: return launch_tma_v<T, WALLS, 16, 16, 2>(src, dst, a, maps, zc, err, s);
    case 4: return launch_tma_v<T, WALLS, 34, 15, 1>(src, dst, a, maps, zc, err, s);
    case 5: return launch_tma_v<T, WALLS, 34, 15, 2>(src, dst, a, maps, zc, err, s);
  }
  return cudaErrorInvalidValue;
}

// kind: tile 0 = 32 x 8, 1 = 16 x 16, 2 = 34 x 15 threads; ns: stages (1, 2);
// maps: the two tensor maps of the source buffer for that tile.
template <typename T>
cudaError_t launch_fused_tma_storage(const void* src, void* dst, const StepArgs& a,
                                     const CUtensorMap* maps, int kind, int ns, int zchunk,
                                     int* err, cudaStream_t s) {
  const int zc = zchunk > 0 ? zchunk : a.nz;
  const bool walls = a.wx || a.wy || a.wz;
  return walls ? launch_tma_w<T, true>(src, dst, a, maps, kind, ns, zc, err, s)
               : launch_tma_w<T, false>(src, dst, a, maps, kind, ns, zc, err, s);
}

template <typename T, bool WALLS, int TW, int BY, int NS>
static cudaError_t launch_tma_batch_v(const void* src, void* dst, const BatchCase* cases,
                                      int ncases, int total_items, const CUtensorMap* maps,
                                      int zc, int* err, int sms, cudaStream_t s) {
  if constexpr (!tma_fits<T, TW, BY, NS>()) {
    return cudaErrorInvalidValue;
  } else {
    static int per_sm_dev[kMaxDevices] = {};  // resident CTAs per SM, queried once
    int& per_sm = per_sm_dev[device_slot()];
    constexpr int bytes = tma_smem_bytes<T, TW, BY, NS>();
    if (per_sm == 0) {
      cudaError_t e = cudaFuncSetAttribute(k_fused_tma_batch<T, WALLS, TW, BY, NS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e != cudaSuccess) return e;
      int q = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &q, k_fused_tma_batch<T, WALLS, TW, BY, NS>, TW * BY, bytes);
      if (e != cudaSuccess) return e;
      per_sm = q < 1 ? 1 : q;
    }
    // one CTA per work item (see launch_tma_seam_batch_v)
    const int grid = total_items;
    (void)sms;
    k_fused_tma_batch<T, WALLS, TW, BY, NS><<<grid, dim3(TW, BY), bytes, s>>>(
        cases, ncases, total_items, maps, (const T*)src, (T*)dst, zc, err);
    return cudaGetLastError();
  }
}

// Batched TMA step; kind 0 (32 x 8) or 2 (34 x 15), ns stages; maps: the
// device table of the source buffer's tensor maps, two per case.
template <typename T>
cudaError_t launch_fused_tma_batch_storage(const void* src, void* dst, const BatchCase* cases,
                                           int ncases, int total_items, bool walls,
                                           const CUtensorMap* maps, int kind, int ns, int zc,
                                           int* err, int sms, cudaStream_t s) {
  switch ((kind == 2 ? 2 : 0) + (ns - 1) + (walls ? 4 : 0)) {
    case 0: return launch_tma_batch_v<T, false, 32, 8, 1>(src, dst, cases, ncases, total_items, maps, zc, err, sms, s);
    case 1: return launch_tma_batch_v<T, false, 32, 8, 2>(src, dst, cases, ncases, total_items, maps, zc, err, sms, s);
    case 2: return launch_tma_batch_v<T, false, 34, 15, 1>(src, dst, cases, ncases, total_items, maps, zc, err, sms, s);
    case 3: return launch_tma_batch_v<T, false, 34, 15, 2>(src, dst, cases, ncases, total_items, maps, zc, err, sms, s);
    case 4: return launch_tma_batch_v<T, true, 32, 8, 1>(src, dst, cases, ncases, total_items, maps, zc, err, sms, s);
    case 5: return launch_tma_batch_v<T, true, 32, 8, 2>(src, dst, cases, ncases, total_items, maps, zc, err, sms, s);
    case 6: return launch_tma_batch_v<T, true, 34, 15, 1>(src, dst, cases, ncases, total_items, maps, zc, err, sms, s);
    case 7: return launch_tma_batch_v<T, true, 34, 15, 2>(src, dst, cases, ncases, total_items, maps, zc, err, sms, s);
  }
  return cudaErrorInvalidValue;
}

// Whether (kind, ns) fits the shared memory for the storage type.
template <typename T>
bool tma_config_fits_storage(int kind, int ns) {
  switch (kind * 2 + (ns - 1)) {
    case 0: return tma_fits<T, 32, 8, 1>();
    case 1: return tma_fits<T, 32, 8, 2>();
    case 2: return tma_fits<T, 16, 16, 1>();
    case 3: return tma_fits<T, 16, 16, 2>();
    case 4: return tma_fits<T, 34, 15, 1>();
    case 5: return tma_fits<T, 34, 15, 2>();
  }
  return false;
}

}  // namespace lbm
