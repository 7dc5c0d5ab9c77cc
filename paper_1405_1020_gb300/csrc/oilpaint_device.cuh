// oilpaint_device.cuh -- device code of the sm_103a oil-paint filter.
//
// The filter is section 4 of Mukherjee, arXiv 1405.1020 (histogram-based oil
// paint): per output pixel, a histogram of the intensity levels of the
// (2r+1)^2 neighbours with a count and R, G, B sums per level, the most
// populated level (lowest on a tie), and that level's truncated mean colour.
// The paper rebuilds the histogram from scratch for every pixel (O(r^2)
// visits); here it is a running histogram that slides down a column of
// output pixels: one step adds the entering image row segment and removes the
// leaving one, 2(2r+1) bin updates per output pixel (Huang's running
// histogram), which gives exactly the same counts and sums.
//
// Data path, per CTA tile of TW output columns x tile_h output rows:
//   1. pack prepass (earlier kernel): every pixel becomes one 32-bit word
//      holding its level and R, G, B (format 0: level << 24 | R << 16 |
//      G << 8 | B for one column per thread; formats 1 and 2 laid out so that
//      a bin delta is one or two masks, for the K-column and column paths),
//      so the level (section 4's quantisation) is computed once per pixel,
//      not once per window visit;
//   2. halo staging: chunks of `ch` packed rows, (TW + 2r) columns rounded to
//      16 bytes, are copied by TMA (cp.async.bulk.tensor.2d) into a ring of
//      shared-memory slots; an mbarrier per slot signals arrival (bounded
//      waits);
//   3. the histograms slide down the tile: one per output column and thread
//      (run_tile), or per thread a window histogram plus difference
//      histograms covering K = 2 or 4 output columns (run_tile_delta, L <=
//      32), or one per image column with the levels across a warp's lanes
//      (run_tile_cols); bins are laid out so the 32 lanes of a warp hit 32
//      different banks whatever their levels;
//   4. argmax: the first level of the largest count (ties to the lowest), as
//      a max over (count, reversed level) keys or a strict > scan;
//   5. the three channel means and the byte stores.
//
// Bins (selected per image by the radius):
//   variant A (r <= 15, window <= 961 pixels): one 64-bit word per bin whose
//       fields (a 10-bit count and three 18-bit sums, 961*255 < 2^18) cannot
//       overflow into each other, so one 64-bit add or subtract updates all
//       four quantities (field order per word format, below);
//   variant B (r <= 44, window <= 7921 pixels): a 64-bit word of three 21-bit
//       sums (7921*255 < 2^21) plus a separate count (16 bits on the K-column
//       path, 32 bits elsewhere).
#pragma once

#include <cuda.h>
#include <stdint.h>

#include <type_traits>

namespace opk {

constexpr int kVarA = 0;
constexpr int kVarB = 1;
constexpr int kMaxRadiusA = 15;
constexpr int kMaxRadiusB = 44;
// A batch splits its images into at most this many groups (radius above
// kMaxRadiusA or not, levels above kBatchLevelSplit or not), each run by its
// own persistent launch sized for the group's largest radius and level count.
constexpr int kBatchGroups = 4;
constexpr uint32_t kBatchLevelSplit = 20;

// bits of the device error word
constexpr uint32_t kErrTimeout = 1u;
// Words of the timeout diagnostic record: [0] set once, then image w, h,
// tile x0, y0, y1, chunk k, chunks, global chunk, slots, expected parity,
// chunks issued, barrier word lo, hi, r | L << 16, box width | ch << 16.
constexpr int kDiagWords = 16;

// One image, as the kernels see it.
struct __align__(16) ImgDesc {
  const uint8_t *in;        // device, rows `stride` bytes apart
  uint8_t *out;             // device, rows `ostride` bytes apart
  uint32_t *packed;         // device, h*ppitch words (pack prepass output)
  const CUtensorMap *tmap;  // device copy of the packed image's tensor map (batch path)
  uint32_t w, h, stride, bpp;
  int32_t r;
  uint32_t L, mode, ppitch;  // mode bit 0: divide by 3 first; bit 1: literal
  uint32_t tile_h, tiles_x, boxw, variant;
  uint32_t ostride;  // output row pitch in bytes
  uint32_t kcols;    // 1: one column per thread (word format 0); 2 or 4: difference
                     // histograms over kcols columns per thread (word formats 1, 2)
  int32_t xshift;    // x of the first tile (0, or -3..0 so that x0 - r is 4-aligned)
  uint32_t fmt;      // packed word format: 0 one column per thread, 1 (r <= 15) and 2
                     // (r > 15) difference and column histograms
  uint32_t path;     // 0: histograms per thread; 1: column histograms, levels across lanes
  uint32_t fused;    // 1: the tensor map reads the input image itself (4-byte pixels) and
                     // each ring chunk is converted to packed words in shared memory;
                     // 0: it reads the packed image the pack prepass wrote
  // output window: columns [ox0, ox1), rows [oy0, oy1) (the whole image, or
  // in literal mode the pixels at least r from every edge); tiles cover the
  // rows from oy0
  int32_t ox0, ox1, oy0, oy1;
};

constexpr uint32_t kModeIntDiv3 = 1u;
// Literal mode: the section-4 listing as printed -- white (level L) is
// counted outside the levels the argmax reads, nothing is written when no
// level below L occurs, and only the colour bytes are written.
constexpr uint32_t kModeLiteral = 2u;

// The difference-histogram path needs r <= 15 (64-bit bins) and L <= 32
// (5-bit level field next to the valid bit).
constexpr int kDeltaMaxRadius = 44;
constexpr uint32_t kDeltaMaxLevels = 32;
// The direct path (run_tile_direct, path 4): radius 0, 1 or 2, any L <= 256.
constexpr uint32_t kPathDirect = 4;
constexpr int kDirectMaxRadius = 2;
// The straight-line difference-histogram path (run_tile_deltak): variant-A
// bins, K/2 <= r <= 15 for K = 2, 4 or 8 columns per thread (r >= 4 for
// K = 8), L <= 32 (L <= 64 for K = 2).
constexpr int kDeltaKMaxRadius = 15;
constexpr uint32_t kDeltaK2MaxLevels = 64;
__host__ __device__ constexpr int deltak_min_radius(int k) {
  return k == 8 ? 4 : (k == 4 ? 2 : 1);
}

// Halo boxes up to kMaxBox2dWords words wide are 2-D TMA copies; wider ones
// (up to kMaxBoxWords) use the 3-D view of the packed image (tma_load_3d),
// which reads the padding words at the end of each packed row: the pack
// prepass writes them as zero.
constexpr uint32_t kMaxBox2dWords = 256;
constexpr uint32_t kMaxBoxWords = 1024;

// Geometry of the shared-memory halo ring, fixed per launch.  Chunk k of a
// tile brings the ch rows entering the window during its steps and the ch
// rows leaving it (2r+1 rows earlier, read again from L2 rather than kept),
// so the ring never holds more than pf + 1 chunks whatever the radius.
struct RingCfg {
  uint32_t ch;          // rows per chunk (TMA box height)
  uint32_t pf;          // chunks in flight ahead of the one being consumed
  uint32_t nslot;       // ring slots = pf + 1
  uint32_t half_bytes;  // bytes of one half (entering or leaving rows), multiple of 128
  uint32_t slot_bytes;  // 2 * half_bytes
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Checked builds (-DOPK_CHECKED=1, the library's bounds-checking variant;
// no GPU sanitizer is used).  Every shared-memory access through the helpers
// below is checked against the running kernel's dynamic shared memory and its
// alignment, every global pixel access against the image, and every TMA
// copy's x coordinate against the 16-byte rule.  A violation sets a bit in
// g_check_error (read and cleared by the host after each run) and the access
// is skipped instead of faulting.
#ifndef OPK_CHECKED
#define OPK_CHECKED 0
#endif

#if OPK_CHECKED
static __device__ uint32_t g_check_error;
extern __shared__ uint8_t opk_dyn_smem[];

__device__ __forceinline__ void check_fail(uint32_t bit) { atomicOr(&g_check_error, bit); }

__device__ __forceinline__ bool smem_ok(uint32_t addr, uint32_t bytes) {
  uint32_t dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const uint32_t lo = smem_addr(opk_dyn_smem);
  const uint32_t align = bytes < 8u ? bytes : 8u;
  const bool ok = addr >= lo && addr + bytes <= lo + dyn && (addr & (align - 1u)) == 0u;
  if (!ok) check_fail(1u);
  return ok;
}
#define OPK_SMEM_OK(a, n) smem_ok((a), (n))
#else
#define OPK_SMEM_OK(a, n) true
#endif

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete; gives up after
// timeout_ns nanoseconds of the global timer and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > timeout_ns) return false;
  }
}

// Makes the tensor-map proxy re-read a 128-byte tensor map in global memory:
// the batch path rewrites its device-resident tensor maps between launches
// (by host copies), and a descriptor cached from an earlier launch would
// describe another image and another box size.
__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap *map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                   reinterpret_cast<uint64_t>(map))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2-D tiled TMA load of a {box_w, box_h} box at element coordinates (x, y)
// of the tensor map into shared memory at dst, completing on mbarrier bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int32_t x,
                                            int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// 3-D tiled TMA load: the packed image seen as {4 words, ppitch / 4 groups,
// rows}, a box of {4, boxw / 4, ch} at group g, row y.  It lands in shared
// memory exactly as the 2-D box of boxw words would, and serves halo rows
// wider than the 256 elements a box dimension may hold.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int32_t g,
                                            int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(g), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  if (!OPK_SMEM_OK(addr, 4u)) return 0u;
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ void lds_v2(uint32_t addr, uint32_t &lo, uint32_t &hi) {
  if (!OPK_SMEM_OK(addr, 8u)) {
    lo = hi = 0u;
    return;
  }
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(addr));
}

__device__ __forceinline__ void lds_v4(uint32_t addr, uint32_t (&v)[4]) {
  if (!OPK_SMEM_OK(addr, 16u)) {
    v[0] = v[1] = v[2] = v[3] = 0u;
    return;
  }
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(addr));
}

__device__ __forceinline__ void sts_v4(uint32_t addr, const uint32_t (&v)[4]) {
  if (!OPK_SMEM_OK(addr, 16u)) return;
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]),
               "r"(v[2]), "r"(v[3])
               : "memory");
}

__device__ __forceinline__ void sts_zero64(uint32_t addr) {
  if (!OPK_SMEM_OK(addr, 8u)) return;
  asm volatile("st.shared.v2.u32 [%0], {%1, %1};" ::"r"(addr), "r"(0u));
}

__device__ __forceinline__ void sts_zero32(uint32_t addr) {
  if (!OPK_SMEM_OK(addr, 4u)) return;
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(0u));
}

__device__ __forceinline__ uint32_t lds_u16(uint32_t addr) {
  if (!OPK_SMEM_OK(addr, 2u)) return 0u;
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ void sts_u16(uint32_t addr, uint32_t v) {
  if (!OPK_SMEM_OK(addr, 2u)) return;
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"(static_cast<uint16_t>(v)));
}


// Raw shared-memory accesses of the histogram helpers (volatile asm: they
// keep their program order among themselves, so a read after a write of the
// same bin sees it; the arithmetic between them is plain C++, scheduled
// freely).  Bins are 64-bit words updated by 64-bit integer adds.
__device__ __forceinline__ uint64_t ld_bin(uint32_t addr) {
  uint64_t v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void st_bin(uint32_t addr, uint64_t v) {
  asm volatile("st.shared.u64 [%0], %1;" ::"r"(addr), "l"(v));
}
__device__ __forceinline__ uint32_t ld_w32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void st_w32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ uint32_t ld_w16(uint32_t addr) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ void st_w16(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"(static_cast<uint16_t>(v)));
}
__device__ __forceinline__ uint64_t u64_of(uint32_t lo, uint32_t hi) {
  return static_cast<uint64_t>(hi) << 32 | lo;
}

// 64-bit read-modify-write of one histogram bin.
__device__ __forceinline__ void bin_add64(uint32_t addr, uint32_t dlo, uint32_t dhi) {
  if (!OPK_SMEM_OK(addr, 8u)) return;
  st_bin(addr, ld_bin(addr) + u64_of(dlo, dhi));
}

__device__ __forceinline__ void bin_sub64(uint32_t addr, uint32_t dlo, uint32_t dhi) {
  if (!OPK_SMEM_OK(addr, 8u)) return;
  st_bin(addr, ld_bin(addr) - u64_of(dlo, dhi));
}

__device__ __forceinline__ void cnt_add(uint32_t addr, uint32_t d) {
  if (!OPK_SMEM_OK(addr, 4u)) return;
  st_w32(addr, ld_w32(addr) + d);
}

// Two 64-bit additions issued together (addr_a != addr_b).
__device__ __forceinline__ void bin_add64x2(uint32_t addr_a, uint32_t alo, uint32_t ahi,
                                            uint32_t addr_b, uint32_t blo, uint32_t bhi) {
  if (!OPK_SMEM_OK(addr_a, 8u) || !OPK_SMEM_OK(addr_b, 8u)) return;
  const uint64_t a = ld_bin(addr_a), b = ld_bin(addr_b);
  st_bin(addr_a, a + u64_of(alo, ahi));
  st_bin(addr_b, b + u64_of(blo, bhi));
}

// +(alo, ahi) at A and -(blo, bhi) at B as one two-deep update that is
// right whether or not A == B: both loads are issued first, and when the
// two bins coincide the subtraction is applied to the sum, which the second
// store (to the same bin) leaves in place.
__device__ __forceinline__ void bin_addsub64_chain(uint32_t A, uint32_t alo, uint32_t ahi,
                                                   uint32_t B, uint32_t blo, uint32_t bhi) {
  if (!OPK_SMEM_OK(A, 8u) || !OPK_SMEM_OK(B, 8u)) return;
  const uint64_t a0 = ld_bin(A), b0 = ld_bin(B);
  const uint64_t a = a0 + u64_of(alo, ahi);
  const uint64_t b = (A == B ? a : b0) - u64_of(blo, bhi);
  st_bin(A, a);
  st_bin(B, b);
}

// +(alo, ahi) at A, then +(blo, bhi) at B, where A and B may coincide (the
// second addition applies to the first's sum): both loads first.
__device__ __forceinline__ void bin_add64x2_chain(uint32_t A, uint32_t alo, uint32_t ahi,
                                                  uint32_t B, uint32_t blo, uint32_t bhi) {
  if (!OPK_SMEM_OK(A, 8u) || !OPK_SMEM_OK(B, 8u)) return;
  const uint64_t a0 = ld_bin(A), b0 = ld_bin(B);
  const uint64_t a = a0 + u64_of(alo, ahi);
  const uint64_t b = (A == B ? a : b0) + u64_of(blo, bhi);
  st_bin(A, a);
  st_bin(B, b);
}

// Two such chained pairs issued together (A, B in one histogram; C, D in
// another): four loads first.
__device__ __forceinline__ void bin_add64x4_chain(uint32_t A, uint32_t alo, uint32_t ahi,
                                                  uint32_t B, uint32_t blo, uint32_t bhi,
                                                  uint32_t C, uint32_t clo, uint32_t chi,
                                                  uint32_t D, uint32_t dlo, uint32_t dhi) {
  if (!OPK_SMEM_OK(A, 8u) || !OPK_SMEM_OK(B, 8u) || !OPK_SMEM_OK(C, 8u) || !OPK_SMEM_OK(D, 8u))
    return;
  const uint64_t a0 = ld_bin(A), b0 = ld_bin(B), c0 = ld_bin(C), d0 = ld_bin(D);
  const uint64_t a = a0 + u64_of(alo, ahi), c = c0 + u64_of(clo, chi);
  const uint64_t b = (A == B ? a : b0) + u64_of(blo, bhi);
  const uint64_t d = (C == D ? c : d0) + u64_of(dlo, dhi);
  st_bin(A, a);
  st_bin(B, b);
  st_bin(C, c);
  st_bin(D, d);
}

// Two such updates issued together (A, B in one histogram; C, D in
// another): four loads first.
__device__ __forceinline__ void bin_addsub64x2_chain(uint32_t A, uint32_t alo, uint32_t ahi,
                                                     uint32_t B, uint32_t blo, uint32_t bhi,
                                                     uint32_t C, uint32_t clo, uint32_t chi,
                                                     uint32_t D, uint32_t dlo, uint32_t dhi) {
  if (!OPK_SMEM_OK(A, 8u) || !OPK_SMEM_OK(B, 8u) || !OPK_SMEM_OK(C, 8u) || !OPK_SMEM_OK(D, 8u))
    return;
  const uint64_t a0 = ld_bin(A), b0 = ld_bin(B), c0 = ld_bin(C), d0 = ld_bin(D);
  const uint64_t a = a0 + u64_of(alo, ahi), c = c0 + u64_of(clo, chi);
  const uint64_t b = (A == B ? a : b0) - u64_of(blo, bhi);
  const uint64_t d = (C == D ? c : d0) - u64_of(dlo, dhi);
  st_bin(A, a);
  st_bin(B, b);
  st_bin(C, c);
  st_bin(D, d);
}

// Variant B bins (64-bit sums at As / Bs, 32-bit counts at Ac / Bc): +(alo,
// ahi, ac) at A and -(blo, bhi, bc) at B, all loads first; As == Bs implies
// Ac == Bc, and then the subtraction applies to the sum (as
// bin_addsub64_chain).
__device__ __forceinline__ void binb_addsub_chain(uint32_t As, uint32_t Ac, uint32_t alo,
                                                  uint32_t ahi, uint32_t ac, uint32_t Bs,
                                                  uint32_t Bc, uint32_t blo, uint32_t bhi,
                                                  uint32_t bc) {
  if (!OPK_SMEM_OK(As, 8u) || !OPK_SMEM_OK(Ac, 4u) || !OPK_SMEM_OK(Bs, 8u) ||
      !OPK_SMEM_OK(Bc, 4u))
    return;
  const uint64_t a0 = ld_bin(As);
  const uint32_t ca0 = ld_w32(Ac);
  const uint64_t b0 = ld_bin(Bs);
  const uint32_t cb0 = ld_w32(Bc);
  const bool same = As == Bs;
  const uint64_t a = a0 + u64_of(alo, ahi);
  const uint32_t ca = ca0 + ac;
  const uint64_t b = (same ? a : b0) - u64_of(blo, bhi);
  const uint32_t cb = (same ? ca : cb0) - bc;
  st_bin(As, a);
  st_w32(Ac, ca);
  st_bin(Bs, b);
  st_w32(Bc, cb);
}

// ------------------------------------------------------------ pack prepass

// Section 4's intensity level of one pixel, clamped to L-1 (literal mode:
// not clamped, so pure white gives L).
__device__ __forceinline__ uint32_t level_of(uint32_t R, uint32_t G, uint32_t B, uint32_t L,
                                             uint32_t mode) {
  const uint32_t s = R + G + B;
  const uint32_t l = (mode & kModeIntDiv3) ? ((s / 3u) * L) / 255u : (s * L) / 765u;
  if (mode & kModeLiteral) return l;
  return l < L ? l : L - 1u;
}

// Word format 0: level << 24 | R << 16 | G << 8 | B.  In literal mode a
// white pixel carries level L, the histogram's scratch level, which the
// argmax never reads.
__device__ __forceinline__ uint32_t pack_word(uint32_t R, uint32_t G, uint32_t B, uint32_t L,
                                              uint32_t mode) {
  return (level_of(R, G, B, L, mode) << 24) | (R << 16) | (G << 8) | B;
}

// Word format 1 (L <= 64), laid out so that one mask gives the low word and
// one shift and mask the high word of the pixel's bin delta (see dh_delta):
//   bit 0 valid (1 for every image pixel; the zero words TMA supplies outside
//   the image therefore add nothing), bits 1..5 level & 31, 6..9 G >> 4,
//   10..17 R, 18 level >> 5, 20..27 B, 28..31 G & 15.
// Bit 18 lies outside both masks of the delta; it is set only when L > 32,
// which only the two-column straight-line path accepts (the other paths read
// the level as w & 0x3E).
__device__ __forceinline__ uint32_t pack_word_delta(uint32_t R, uint32_t G, uint32_t B,
                                                    uint32_t L, uint32_t mode) {
  const uint32_t l = level_of(R, G, B, L, mode);
  if (l >= L) return 0u;  // literal mode: level L is never read, so it adds nothing
  return 1u | ((l & 31u) << 1) | ((G >> 4) << 6) | (R << 10) | ((l >> 5) << 18) | (B << 20) |
         ((G & 0xFu) << 28);
}

// Word format 2 (L <= 32, 16 <= r <= 44): R @0..7 | level @8..12 |
// B @13..20 | G @21..28 | valid @29 (see DeltaOpsB).
__device__ __forceinline__ uint32_t pack_word_delta_b(uint32_t R, uint32_t G, uint32_t B,
                                                      uint32_t L, uint32_t mode) {
  const uint32_t l = level_of(R, G, B, L, mode);
  if (l >= L) return 0u;  // literal mode: level L adds nothing
  return R | (l << 8) | (B << 13) | (G << 21) | (1u << 29);
}

// Packs row y of image d with threads tid, tid+nthr, ...  Rows whose pixels
// start on a 16-byte (RGBA) or 4-byte (RGB) boundary are read and written
// four pixels at a time; the packed rows always start on a 16-byte boundary
// (the tensor map's base and pitch rule).
__device__ __forceinline__ void pack_row(const ImgDesc &d, uint32_t y, uint32_t tid,
                                         uint32_t nthr) {
  const uint8_t *src = d.in + static_cast<size_t>(y) * d.stride;
  uint32_t *dst = d.packed + static_cast<size_t>(y) * d.ppitch;
  const uint32_t L = d.L, mode = d.mode, w = d.w;
  const uint32_t fmt = d.fmt;
  // the words after the last pixel, up to the 16-byte row pitch, are zero
  // (3-D halo copies read them; zero is the word of no pixel)
  if (tid < d.ppitch - w) dst[w + tid] = 0u;
  auto word = [&](uint32_t R, uint32_t G, uint32_t B) {
    return fmt == 1u   ? pack_word_delta(R, G, B, L, mode)
           : fmt == 2u ? pack_word_delta_b(R, G, B, L, mode)
                       : pack_word(R, G, B, L, mode);
  };
  auto rgba = [&](uint32_t p) { return word(p & 0xFFu, (p >> 8) & 0xFFu, (p >> 16) & 0xFFu); };
  const uintptr_t a = reinterpret_cast<uintptr_t>(src);
  uint32_t x0 = 0;  // first pixel left to the scalar loop
  if (d.bpp == 4 && (a & 15u) == 0) {
    const uint4 *s16 = reinterpret_cast<const uint4 *>(src);
    uint4 *d16 = reinterpret_cast<uint4 *>(dst);
    const uint32_t nq = w >> 2;
    // four 16-byte loads in flight per thread before any conversion
    for (uint32_t q0 = tid; q0 < nq; q0 += 4u * nthr) {
      uint4 p[4];
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        const uint32_t q = q0 + k * nthr;
        if (q < nq) p[k] = __ldg(s16 + q);
      }
#pragma unroll
      for (uint32_t k = 0; k < 4u; ++k) {
        const uint32_t q = q0 + k * nthr;
        if (q < nq) d16[q] = make_uint4(rgba(p[k].x), rgba(p[k].y), rgba(p[k].z), rgba(p[k].w));
      }
    }
    x0 = nq << 2;
  } else if (d.bpp == 3) {
    // Four RGB pixels are three words: R0G0B0R1 G1B1R2G2 B2R3G3B3.  A row
    // that starts m = a & 3 bytes into a word is read as aligned words and
    // shifted by 8m bits (a fourth word is then needed; it lies in the same
    // aligned word as the group's last byte, so it never leaves the row's
    // memory page).  (Two or four groups in flight per thread held more
    // registers than the kernel's occupancy can afford.)
    const uint32_t m = static_cast<uint32_t>(a & 3u);
    const uint32_t *s4 = reinterpret_cast<const uint32_t *>(src - m);
    uint4 *d16 = reinterpret_cast<uint4 *>(dst);
    const uint32_t nq = w >> 2;
    auto run = [&](auto shifted) {
      constexpr bool SH = decltype(shifted)::value;
      const uint32_t sh = 8u * m;
      for (uint32_t q = tid; q < nq; q += nthr) {
        const uint32_t *g4 = s4 + 3u * q;
        const uint32_t w0 = __ldg(g4), w1 = __ldg(g4 + 1u), w2 = __ldg(g4 + 2u);
        uint32_t p0 = w0, p1 = w1, p2 = w2;
        if (SH) {
          const uint32_t w3 = __ldg(g4 + 3u);
          p0 = __funnelshift_r(w0, w1, sh);
          p1 = __funnelshift_r(w1, w2, sh);
          p2 = __funnelshift_r(w2, w3, sh);
        }
        d16[q] = make_uint4(word(p0 & 0xFFu, (p0 >> 8) & 0xFFu, (p0 >> 16) & 0xFFu),
                            word(p0 >> 24, p1 & 0xFFu, (p1 >> 8) & 0xFFu),
                            word((p1 >> 16) & 0xFFu, p1 >> 24, p2 & 0xFFu),
                            word((p2 >> 8) & 0xFFu, (p2 >> 16) & 0xFFu, p2 >> 24));
      }
    };
    if (m)
      run(std::true_type{});
    else
      run(std::false_type{});
    x0 = nq << 2;
  }
  if (d.bpp == 4 && (a & 3u) == 0) {
    const uint32_t *s4 = reinterpret_cast<const uint32_t *>(src);
    for (uint32_t x = x0 + tid; x < w; x += nthr) dst[x] = rgba(__ldg(s4 + x));
    return;
  }
  const uint32_t bpp = d.bpp;
  for (uint32_t x = x0 + tid; x < w; x += nthr) {
    const uint8_t *p = src + x * bpp;
    dst[x] = word(__ldg(p), __ldg(p + 1), __ldg(p + 2));
  }
}

// Fused pack (4-byte input pixels staged raw by the halo copies).  The ring
// slot at shared address `slot` holds the ch entering rows of a chunk, from
// image row ye, and half_bytes further its ch leaving rows, from row yl;
// each row is boxw pixels wide from image column xs (boxw a multiple of 4).
// The CTA's threads convert them in place, four pixels at a time, to the
// packed words the pack prepass would have written (format d.fmt); pixels
// outside the image -- zero-filled by the copy, or the bytes of the row past
// its last pixel -- become word 0, which adds nothing to any histogram.
// The caller synchronises the CTA before and after.
__device__ __forceinline__ void convert_raw_slot(const ImgDesc &d, uint32_t slot,
                                                 uint32_t half_bytes, int xs, int ye, int yl,
                                                 uint32_t ch, uint32_t boxw) {
  const uint32_t groups = boxw >> 2;
  // the direct path's copies bring entering rows only
  const uint32_t rows = (d.path == kPathDirect ? 1u : 2u) * ch;
  const uint32_t nthr = blockDim.x;
  const int w = static_cast<int>(d.w), h = static_cast<int>(d.h);
  const uint32_t L = d.L, mode = d.mode, fmt = d.fmt;
  uint32_t hr = 0, q = threadIdx.x;  // half-row (entering rows, then leaving rows), group
  while (q >= groups) {
    q -= groups;
    ++hr;
  }
  while (hr < rows) {
    const bool leaving = hr >= ch;
    const uint32_t rr = leaving ? hr - ch : hr;
    const int y = (leaving ? yl : ye) + static_cast<int>(rr);
    const uint32_t addr = slot + (leaving ? half_bytes : 0u) + (rr * boxw + 4u * q) * 4u;
    const int x = xs + static_cast<int>(4u * q);
    const bool row_in = y >= 0 && y < h;
    uint32_t v[4];
    lds_v4(addr, v);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t p = v[e];
      const uint32_t R = p & 0xFFu, G = (p >> 8) & 0xFFu, B = (p >> 16) & 0xFFu;
      const uint32_t wd = fmt == 1u   ? pack_word_delta(R, G, B, L, mode)
                          : fmt == 2u ? pack_word_delta_b(R, G, B, L, mode)
                                      : pack_word(R, G, B, L, mode);
      v[e] = (row_in && x + e >= 0 && x + e < w) ? wd : 0u;
    }
    sts_v4(addr, v);
    q += nthr;
    while (q >= groups) {
      q -= groups;
      ++hr;
    }
  }
}

// --------------------------------------------------------- histogram bins

// Variant A delta of packed word w: count +1 @54, R @36, G @18, B @0.
__device__ __forceinline__ void delta_a(uint32_t w, uint32_t &lo, uint32_t &hi) {
  lo = (w & 0xFFu) | ((w << 10) & 0x03FC0000u);
  hi = ((w >> 12) & 0x00000FF0u) | 0x00400000u;
}

// Variant B delta of the 64-bit sums: R @42, G @21, B @0.
__device__ __forceinline__ void delta_b(uint32_t w, uint32_t &lo, uint32_t &hi) {
  lo = (w & 0xFFu) | ((w << 13) & 0x1FE00000u);
  hi = (w >> 6) & 0x0003FC00u;
}

// One histogram owned by one thread (one output column per thread, word
// format 0): level l of thread t lives at sums + l * NT * 8 (+ cnts + l * NT
// * 4 for variant B), so the 32 lanes of a warp always touch 32 consecutive
// bins whatever their levels.  Level L exists but the argmax never reads it
// (literal mode's white pixels land there).
template <int NT, int VAR>
struct Hist {
  static constexpr uint32_t kStride64 = NT * 8u;
  static constexpr uint32_t kStride32 = NT * 4u;
  uint32_t sums;     // smem address of level 0's 64-bit bin
  uint32_t cnts;     // smem address of level 0's count (variant B)

  __device__ __forceinline__ void clear(uint32_t L) const {
    for (uint32_t l = 0; l < L; ++l) {
      sts_zero64(sums + l * kStride64);
      if (VAR == kVarB) sts_zero32(cnts + l * kStride32);
    }
  }
  __device__ __forceinline__ void delta(uint32_t w, uint32_t &lo, uint32_t &hi) const {
    if (VAR == kVarA)
      delta_a(w, lo, hi);
    else
      delta_b(w, lo, hi);
  }
  __device__ __forceinline__ void add(uint32_t w) const {
    const uint32_t lvl = w >> 24;
    uint32_t lo, hi;
    delta(w, lo, hi);
    bin_add64(sums + lvl * kStride64, lo, hi);
    if (VAR == kVarB) cnt_add(cnts + lvl * kStride32, 1u);
  }
  __device__ __forceinline__ void sub(uint32_t w) const {
    const uint32_t lvl = w >> 24;
    uint32_t lo, hi;
    delta(w, lo, hi);
    bin_sub64(sums + lvl * kStride64, lo, hi);
    if (VAR == kVarB) cnt_add(cnts + lvl * kStride32, 0xFFFFFFFFu);
  }
  // Adds pixel win and removes pixel wout as one two-deep update; when both
  // fall in the same level the removal applies to the sum (chained).
  __device__ __forceinline__ void addsub(uint32_t win, uint32_t wout) const {
    const uint32_t la = win >> 24, lb = wout >> 24;
    uint32_t alo, ahi, blo, bhi;
    delta(win, alo, ahi);
    delta(wout, blo, bhi);
    if (VAR == kVarA)
      bin_addsub64_chain(sums + la * kStride64, alo, ahi, sums + lb * kStride64, blo, bhi);
    else
      binb_addsub_chain(sums + la * kStride64, cnts + la * kStride32, alo, ahi, 1u,
                        sums + lb * kStride64, cnts + lb * kStride32, blo, bhi, 1u);
  }
  // Count of level l, for variant A kept in place in bits 22..31 of the high
  // word (comparing these words compares counts).
  __device__ __forceinline__ uint32_t count_key(uint32_t l) const {
    if (VAR == kVarA) return lds_u32(sums + l * kStride64 + 4u) & 0xFFC00000u;
    return lds_u32(cnts + l * kStride32);
  }
  __device__ __forceinline__ void bin(uint32_t l, uint32_t &lo, uint32_t &hi) const {
    lds_v2(sums + l * kStride64, lo, hi);
  }
};

// Channel sums and count of a word-format-0 bin.
template <int VAR>
__device__ __forceinline__ void unpack_bin(uint32_t lo, uint32_t hi, uint32_t cnt_b,
                                           uint32_t &cnt, uint32_t &R, uint32_t &G,
                                           uint32_t &B) {
  if (VAR == kVarA) {
    cnt = hi >> 22;
    R = (hi >> 4) & 0x3FFFFu;
    G = ((hi & 0xFu) << 14) | (lo >> 18);
    B = lo & 0x3FFFFu;
  } else {
    cnt = cnt_b;
    R = hi >> 10;
    G = (lo >> 21) | ((hi & 0x3FFu) << 11);
    B = lo & 0x1FFFFFu;
  }
}

// ------------------------------------------- difference-histogram bins
//
// Difference-histogram bins.  Both kinds are linear in the pixel (modulo
// 2^64 / 2^32), so the signed fields of a difference histogram are
// harmless: the sum of a window's bins decodes exactly.
//
// Variant A (r <= 15, word format 1), one 64-bit bin:
//   count:10 @0 | R:18 @10 | G:18 @28 | B:18 @46.
// The count sits at the bottom of the LOW word, so the low word of a sum of
// bins is the sum of their low words: adding the low words of a window
// histogram and of difference histograms gives an exact count without
// touching the high words.  A pixel's delta is one mask of its word (low
// word, with the valid bit landing on the count) and one shift and mask
// (high word); zero words (outside the image) have a zero delta.
//
// Variant B (16 <= r <= 44, word format 2), a 64-bit sums bin
//   R:21 @0 | G:21 @21 | B:21 @42   (89^2 * 255 < 2^21)
// plus a count in a second array laid out like the sums: 16 bits at a
// quarter of the stride on the K-column path (a bin's count address is
// (sums address >> 2) + cd for one CTA-wide constant cd), 32 bits at half
// the stride on the column path.

__device__ __forceinline__ void dh_delta(uint32_t w, uint32_t &lo, uint32_t &hi) {
  lo = w & 0xF003FC01u;
  hi = (w >> 6) & 0x003FC00Fu;
}

// Address of w's bin in a histogram whose level 0 is at `base` and whose
// levels are LS bytes apart: the level field sits at bits 1..5, so
// (w & 0x3E) * LS / 2.
template <uint32_t LS>
__device__ __forceinline__ uint32_t dh_addr(uint32_t base, uint32_t w) {
  return base + (w & 0x3Eu) * (LS / 2u);
}

__device__ __forceinline__ void neg64(uint32_t &lo, uint32_t &hi) {
  const uint64_t v = 0ull - (static_cast<uint64_t>(hi) << 32 | lo);
  lo = static_cast<uint32_t>(v);
  hi = static_cast<uint32_t>(v >> 32);
}

// Variant A operations on histograms given by the address of the thread's
// level-0 bin, levels LS bytes apart.
template <uint32_t LS>
struct DeltaOpsA {
  __device__ __forceinline__ void add(uint32_t base, uint32_t w) const {
    uint32_t lo, hi;
    dh_delta(w, lo, hi);
    bin_add64(dh_addr<LS>(base, w), lo, hi);
  }
  __device__ __forceinline__ void sub(uint32_t base, uint32_t w) const {
    uint32_t lo, hi;
    dh_delta(w, lo, hi);
    bin_sub64(dh_addr<LS>(base, w), lo, hi);
  }
  // +w0 +w1 in one histogram as one two-deep update (their bins may coincide).
  __device__ __forceinline__ void add2(uint32_t base, uint32_t w0, uint32_t w1) const {
    uint32_t alo, ahi, blo, bhi;
    dh_delta(w0, alo, ahi);
    dh_delta(w1, blo, bhi);
    bin_add64x2_chain(dh_addr<LS>(base, w0), alo, ahi, dh_addr<LS>(base, w1), blo, bhi);
  }
  // +w0 +w1 in histogram p and +w2 +w3 in histogram q != p, four deep.
  __device__ __forceinline__ void add2x2(uint32_t p, uint32_t w0, uint32_t w1, uint32_t q,
                                         uint32_t w2, uint32_t w3) const {
    uint32_t alo, ahi, blo, bhi, clo, chi, dlo, dhi;
    dh_delta(w0, alo, ahi);
    dh_delta(w1, blo, bhi);
    dh_delta(w2, clo, chi);
    dh_delta(w3, dlo, dhi);
    bin_add64x4_chain(dh_addr<LS>(p, w0), alo, ahi, dh_addr<LS>(p, w1), blo, bhi,
                      dh_addr<LS>(q, w2), clo, chi, dh_addr<LS>(q, w3), dlo, dhi);
  }
  // +win -wout in one histogram as one two-deep update (the bins of the two
  // words may coincide).
  __device__ __forceinline__ void addsub(uint32_t base, uint32_t win, uint32_t wout) const {
    uint32_t alo, ahi, blo, bhi;
    dh_delta(win, alo, ahi);
    dh_delta(wout, blo, bhi);
    bin_addsub64_chain(dh_addr<LS>(base, win), alo, ahi, dh_addr<LS>(base, wout), blo, bhi);
  }
  // +win_p -wout_p in histogram p and +win_q -wout_q in histogram q != p as
  // one four-deep update.
  __device__ __forceinline__ void addsub_x2(uint32_t p, uint32_t win_p, uint32_t wout_p,
                                            uint32_t q, uint32_t win_q, uint32_t wout_q) const {
    uint32_t alo, ahi, blo, bhi, clo, chi, dlo, dhi;
    dh_delta(win_p, alo, ahi);
    dh_delta(wout_p, blo, bhi);
    dh_delta(win_q, clo, chi);
    dh_delta(wout_q, dlo, dhi);
    bin_addsub64x2_chain(dh_addr<LS>(p, win_p), alo, ahi, dh_addr<LS>(p, wout_p), blo, bhi,
                         dh_addr<LS>(q, win_q), clo, chi, dh_addr<LS>(q, wout_q), dlo, dhi);
  }
  // (+/-)wp at histogram p and (+/-)wq at histogram q != p.
  template <bool NEG_P, bool NEG_Q>
  __device__ __forceinline__ void pm_x2(uint32_t p, uint32_t wp, uint32_t q, uint32_t wq) const {
    uint32_t plo, phi, qlo, qhi;
    dh_delta(wp, plo, phi);
    dh_delta(wq, qlo, qhi);
    if (NEG_P) neg64(plo, phi);
    if (NEG_Q) neg64(qlo, qhi);
    bin_add64x2(dh_addr<LS>(p, wp), plo, phi, dh_addr<LS>(q, wq), qlo, qhi);
  }
};

// Two additions at two distinct bins (signs folded into the deltas).
__device__ __forceinline__ void binb_add_x2(uint32_t As, uint32_t Ac, uint32_t alo, uint32_t ahi,
                                            uint32_t ac, uint32_t Bs, uint32_t Bc, uint32_t blo,
                                            uint32_t bhi, uint32_t bc) {
  if (!OPK_SMEM_OK(As, 8u) || !OPK_SMEM_OK(Ac, 4u) || !OPK_SMEM_OK(Bs, 8u) ||
      !OPK_SMEM_OK(Bc, 4u))
    return;
  const uint64_t a0 = ld_bin(As);
  const uint32_t ca0 = ld_w32(Ac);
  const uint64_t b0 = ld_bin(Bs);
  const uint32_t cb0 = ld_w32(Bc);
  st_bin(As, a0 + u64_of(alo, ahi));
  st_w32(Ac, ca0 + ac);
  st_bin(Bs, b0 + u64_of(blo, bhi));
  st_w32(Bc, cb0 + bc);
}

__device__ __forceinline__ void binb_add(uint32_t As, uint32_t Ac, uint32_t lo, uint32_t hi,
                                         uint32_t c) {
  if (!OPK_SMEM_OK(As, 8u) || !OPK_SMEM_OK(Ac, 4u)) return;
  const uint64_t a0 = ld_bin(As);
  const uint32_t ca0 = ld_w32(Ac);
  st_bin(As, a0 + u64_of(lo, hi));
  st_w32(Ac, ca0 + c);
}

// Variant B bins with 16-bit counts (the K-column path: a window's count is
// at most 89^2 = 7921, and the difference histograms' counts are kept mod
// 2^16, which the window sums undo): binb_add, binb_add_x2 and
// binb_addsub_chain with 2-byte count accesses (a 16-bit load zero-extends
// into the 32-bit register; a 16-bit store keeps its low half).
__device__ __forceinline__ void binb16_add(uint32_t As, uint32_t Ac, uint32_t lo, uint32_t hi,
                                           uint32_t c) {
  if (!OPK_SMEM_OK(As, 8u) || !OPK_SMEM_OK(Ac, 2u)) return;
  const uint64_t a0 = ld_bin(As);
  const uint32_t ca0 = ld_w16(Ac);
  st_bin(As, a0 + u64_of(lo, hi));
  st_w16(Ac, ca0 + c);
}

__device__ __forceinline__ void binb16_add_x2(uint32_t As, uint32_t Ac, uint32_t alo,
                                              uint32_t ahi, uint32_t ac, uint32_t Bs,
                                              uint32_t Bc, uint32_t blo, uint32_t bhi,
                                              uint32_t bc) {
  if (!OPK_SMEM_OK(As, 8u) || !OPK_SMEM_OK(Ac, 2u) || !OPK_SMEM_OK(Bs, 8u) ||
      !OPK_SMEM_OK(Bc, 2u))
    return;
  const uint64_t a0 = ld_bin(As);
  const uint32_t ca0 = ld_w16(Ac);
  const uint64_t b0 = ld_bin(Bs);
  const uint32_t cb0 = ld_w16(Bc);
  st_bin(As, a0 + u64_of(alo, ahi));
  st_w16(Ac, ca0 + ac);
  st_bin(Bs, b0 + u64_of(blo, bhi));
  st_w16(Bc, cb0 + bc);
}

__device__ __forceinline__ void binb16_addsub_chain(uint32_t As, uint32_t Ac, uint32_t alo,
                                                    uint32_t ahi, uint32_t ac, uint32_t Bs,
                                                    uint32_t Bc, uint32_t blo, uint32_t bhi,
                                                    uint32_t bc) {
  if (!OPK_SMEM_OK(As, 8u) || !OPK_SMEM_OK(Ac, 2u) || !OPK_SMEM_OK(Bs, 8u) ||
      !OPK_SMEM_OK(Bc, 2u))
    return;
  const uint64_t a0 = ld_bin(As);
  const uint32_t ca0 = ld_w16(Ac);
  const uint64_t b0 = ld_bin(Bs);
  const uint32_t cb0 = ld_w16(Bc);
  const bool same = As == Bs;
  const uint64_t a = a0 + u64_of(alo, ahi);
  const uint32_t ca = ca0 + ac;
  const uint64_t b = (same ? a : b0) - u64_of(blo, bhi);
  const uint32_t cb = (same ? ca : cb0) - bc;
  st_bin(As, a);
  st_w16(Ac, ca);
  st_bin(Bs, b);
  st_w16(Bc, cb);
}

// Word format 2 (L <= 32): R @0..7 | level @8..12 | B @13..20 | G @21..28 |
// valid @29.  Sums delta: low word one mask (R, G), high word one shift and
// mask (B << 10); count delta: the valid bit.
__device__ __forceinline__ void dhb_delta(uint32_t w, uint32_t &lo, uint32_t &hi, uint32_t &c) {
  lo = w & 0x1FE000FFu;
  hi = (w >> 3) & 0x0003FC00u;
  c = w >> 29;
}

// Variant B operations; counts of CW bytes (4, or 2 on the K-column path)
// laid out like the sums at CW/8 of their stride.
template <uint32_t LS, uint32_t CW = 4u>
struct DeltaOpsB {
  static_assert(CW == 2u || CW == 4u, "count width");
  uint32_t cd;  // count address = (sums address * CW / 8) + cd

  // level field (bits 8..12) times the level stride LS
  __device__ __forceinline__ uint32_t saddr(uint32_t base, uint32_t w) const {
    return base + (((w & 0x1F00u) * LS) >> 8);
  }
  __device__ __forceinline__ uint32_t caddr(uint32_t s) const {
    return (s >> (CW == 2u ? 2 : 1)) + cd;
  }
  __device__ __forceinline__ void bin_add(uint32_t s, uint32_t lo, uint32_t hi, uint32_t c) const {
    if constexpr (CW == 2u)
      binb16_add(s, caddr(s), lo, hi, c);
    else
      binb_add(s, caddr(s), lo, hi, c);
  }

  __device__ __forceinline__ void add(uint32_t base, uint32_t w) const {
    uint32_t lo, hi, c;
    dhb_delta(w, lo, hi, c);
    bin_add(saddr(base, w), lo, hi, c);
  }
  __device__ __forceinline__ void sub(uint32_t base, uint32_t w) const {
    uint32_t lo, hi, c;
    dhb_delta(w, lo, hi, c);
    neg64(lo, hi);
    bin_add(saddr(base, w), lo, hi, 0u - c);
  }
  __device__ __forceinline__ void add2(uint32_t base, uint32_t w0, uint32_t w1) const {
    add(base, w0);
    add(base, w1);
  }
  __device__ __forceinline__ void add2x2(uint32_t p, uint32_t w0, uint32_t w1, uint32_t q,
                                         uint32_t w2, uint32_t w3) const {
    add2(p, w0, w1);
    add2(q, w2, w3);
  }
  __device__ __forceinline__ void addsub(uint32_t base, uint32_t win, uint32_t wout) const {
    uint32_t alo, ahi, ac, blo, bhi, bc;
    dhb_delta(win, alo, ahi, ac);
    dhb_delta(wout, blo, bhi, bc);
    const uint32_t as = saddr(base, win), bs = saddr(base, wout);
    if constexpr (CW == 2u)
      binb16_addsub_chain(as, caddr(as), alo, ahi, ac, bs, caddr(bs), blo, bhi, bc);
    else
      binb_addsub_chain(as, caddr(as), alo, ahi, ac, bs, caddr(bs), blo, bhi, bc);
  }
  // Two histograms: issued as two two-deep updates (a four-deep one would
  // need 20 operands and more registers than it saves latency here).
  __device__ __forceinline__ void addsub_x2(uint32_t p, uint32_t win_p, uint32_t wout_p,
                                            uint32_t q, uint32_t win_q, uint32_t wout_q) const {
    addsub(p, win_p, wout_p);
    addsub(q, win_q, wout_q);
  }
  template <bool NEG_P, bool NEG_Q>
  __device__ __forceinline__ void pm_x2(uint32_t p, uint32_t wp, uint32_t q, uint32_t wq) const {
    uint32_t plo, phi, pc, qlo, qhi, qc;
    dhb_delta(wp, plo, phi, pc);
    dhb_delta(wq, qlo, qhi, qc);
    if (NEG_P) {
      neg64(plo, phi);
      pc = 0u - pc;
    }
    if (NEG_Q) {
      neg64(qlo, qhi);
      qc = 0u - qc;
    }
    const uint32_t ps = saddr(p, wp), qs = saddr(q, wq);
    if constexpr (CW == 2u)
      binb16_add_x2(ps, caddr(ps), plo, phi, pc, qs, caddr(qs), qlo, qhi, qc);
    else
      binb_add_x2(ps, caddr(ps), plo, phi, pc, qs, caddr(qs), qlo, qhi, qc);
  }
};

// ------------------------------------------------------------ division

// Truncating n / d for the channel means.  r <= 15 (n < 2^18, d <= 961):
// Granlund and Montgomery's multiply-high by m = ceil(2^31 / d), looked up
// in a table built at compile time, q = floor(2n * m / 2^32); with
// e = m*d - 2^31 < d the error term n*e / 2^31 stays below 2^28 / 2^31 < 1,
// so q is exact.  Larger radii use integer division.  The table lives in
// global memory (read through the L1 cache) rather than in each CTA's
// shared memory, which the histograms need.
constexpr uint32_t kRcpEntries = 962;  // d = 0..961 (entry 0 unused)

struct RcpTable {
  uint32_t m[kRcpEntries];
};

constexpr RcpTable make_rcp_table() {
  RcpTable t{};
  for (uint32_t d = 1; d < kRcpEntries; ++d)
    t.m[d] = static_cast<uint32_t>(((1ull << 31) + d - 1u) / d);
  return t;
}

__device__ const RcpTable g_rcp = make_rcp_table();

__device__ __forceinline__ uint32_t rcp_of(uint32_t d) { return __ldg(&g_rcp.m[d]); }

template <int VAR>
__device__ __forceinline__ uint32_t div_mean(uint32_t n, uint32_t d, uint32_t m) {
  if (VAR == kVarA) return __umulhi(n << 1, m);
  return n / d;
}

// ----------------------------------------------------------------- tiles

// Shared-memory carve-up common to all kernels.  `smem` is the dynamic
// shared memory base; every region starts on a 128-byte boundary.
struct SmemMap {
  uint32_t bars;  // nslot mbarriers
  uint32_t ring;  // nslot * slot_bytes
  uint32_t sums;  // histogram bins
  uint32_t cnts;  // variant B counts
  uint8_t *ring_ptr;
};

__device__ __forceinline__ SmemMap carve_smem(uint8_t *smem, const RingCfg &rc,
                                              uint32_t nhist_bins) {
  SmemMap s;
  const uint32_t base = smem_addr(smem);
  const uint32_t a = (base + 127u) & ~127u;
  s.bars = a;
  s.ring = a + ((rc.nslot * 8u + 127u) & ~127u);
  s.sums = s.ring + rc.nslot * rc.slot_bytes;
  s.cnts = s.sums + nhist_bins * 8u;
  s.ring_ptr = smem + (s.ring - base);
  return s;
}

// Writes the output pixel (x, y): R, G, B and, with 4 bytes per pixel, alpha.
__device__ __forceinline__ void store_pixel(const ImgDesc &d, int x, int y, uint32_t R,
                                            uint32_t G, uint32_t B, uint32_t alpha) {
#if OPK_CHECKED
  if (x < 0 || y < 0 || x >= static_cast<int>(d.w) || y >= static_cast<int>(d.h)) {
    check_fail(2u);
    return;
  }
#endif
  uint8_t *o = d.out + static_cast<size_t>(y) * d.ostride + static_cast<size_t>(x) * d.bpp;
  if (d.bpp == 4 && !(d.mode & kModeLiteral)) {
    const uint32_t v = R | (G << 8) | (B << 16) | (alpha << 24);
    if ((reinterpret_cast<uintptr_t>(o) & 3u) == 0) {
      *reinterpret_cast<uint32_t *>(o) = v;
    } else {
      o[0] = static_cast<uint8_t>(R);
      o[1] = static_cast<uint8_t>(G);
      o[2] = static_cast<uint8_t>(B);
      o[3] = static_cast<uint8_t>(alpha);
    }
  } else {
    o[0] = static_cast<uint8_t>(R);
    o[1] = static_cast<uint8_t>(G);
    o[2] = static_cast<uint8_t>(B);
  }
}

__device__ __forceinline__ uint32_t load_alpha(const ImgDesc &d, int x, int y) {
#if OPK_CHECKED
  if (x < 0 || y < 0 || x >= static_cast<int>(d.w) || y >= static_cast<int>(d.h)) {
    check_fail(2u);
    return 0u;
  }
#endif
  return __ldg(d.in + static_cast<size_t>(y) * d.stride + static_cast<size_t>(x) * 4u + 3u);
}

// The halo-ring protocol of one tile.  Step s = 0 .. nsteps-1 adds entering
// row E0 + s and removes leaving row E0 + s - (2r+1).  Chunk k covers steps
// [k*ch, (k+1)*ch): its entering and leaving rows arrive by two TMA copies of
// d.boxw columns from image column xs (a multiple of 4) into ring slot
// (chunk_ctr + k) % nslot, whose mbarrier completes its phase
// ((chunk_ctr + k) / nslot) & 1.  chunk_ctr counts the chunks this CTA has
// consumed and is advanced by the tile.  For each step, step(s, e, l) gets
// the ring rows of the entering and leaving row, column 0 = image column xs.
// Returns false if a copy did not arrive within timeout_ns: the error bit is
// set, the first such event is described in diag (16 words, may be null),
// and the copies still in flight are waited for (bounded) before returning.
// tmap_global: the tensor map lives in global memory (batch path) and may
// have been rewritten since an earlier launch; it is fenced before use.
template <class Step>
__device__ __forceinline__ bool ring_pass(const ImgDesc &d, const CUtensorMap *tmap, int xs,
                                          int E0, int nsteps, const RingCfg &rc,
                                          const SmemMap &sm, uint32_t &chunk_ctr,
                                          uint32_t *err, uint64_t timeout_ns, uint32_t *diag,
                                          bool tmap_global, int x0, int y0, int y1,
                                          Step &&step) {
  const int t = threadIdx.x;
  const int r = d.r;
  const int ch = static_cast<int>(rc.ch);
  const int nchunks = (nsteps + ch - 1) / ch;
  const uint32_t box_bytes = d.boxw * rc.ch * 4u;
  const uint32_t boxw = d.boxw;

  auto issue = [&](int k) {
    const uint32_t g = chunk_ctr + static_cast<uint32_t>(k);
    const uint32_t slot = g % rc.nslot;
    const uint32_t bar = sm.bars + slot * 8u;
    const uint32_t dst = sm.ring + slot * rc.slot_bytes;
#if OPK_CHECKED
    // x a multiple of 4 words (16 bytes); both halves inside the ring slot
    if ((xs & 3) != 0 || box_bytes > rc.half_bytes || !OPK_SMEM_OK(dst, rc.slot_bytes)) {
      check_fail(4u);
      return;  // nothing armed: the wait for this chunk runs out and reports a timeout
    }
#endif
    // the direct path (4) keeps its windows in registers: entering rows only
    const bool leaving = d.path != kPathDirect;
    mbar_arrive_expect_tx(bar, (leaving ? 2u : 1u) * box_bytes);
    if (boxw > kMaxBox2dWords) {  // xs is a multiple of 4: a whole group
      tma_load_3d(dst, tmap, xs >> 2, E0 + k * ch, bar);
      if (leaving) tma_load_3d(dst + rc.half_bytes, tmap, xs >> 2, E0 + k * ch - 2 * r - 1, bar);
    } else {
      tma_load_2d(dst, tmap, xs, E0 + k * ch, bar);
      if (leaving) tma_load_2d(dst + rc.half_bytes, tmap, xs, E0 + k * ch - 2 * r - 1, bar);
    }
  };

  __syncthreads();  // the previous tile no longer reads the ring
  int issued = min(static_cast<int>(rc.pf), nchunks);
  if (t == 0) {
    if (tmap_global) fence_tensormap_acquire(tmap);
    fence_proxy_async_smem();
    for (int k = 0; k < issued; ++k) issue(k);
  }

  const uint32_t *ring = reinterpret_cast<const uint32_t *>(sm.ring_ptr);
  const uint32_t slot_words = rc.slot_bytes / 4u;
  const uint32_t half_words = rc.half_bytes / 4u;

  for (int k = 0; k < nchunks; ++k) {
    const uint32_t g = chunk_ctr + static_cast<uint32_t>(k);
    const bool ok = mbar_wait_bounded(sm.bars + (g % rc.nslot) * 8u, (g / rc.nslot) & 1u,
                                      timeout_ns);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicOr(err, kErrTimeout);
        if (diag && atomicCAS(diag, 0u, 1u) == 0u) {
          const uint32_t slot = g % rc.nslot;
          uint32_t blo, bhi;
          asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                       : "=r"(blo), "=r"(bhi)
                       : "r"(sm.bars + slot * 8u));
          const uint32_t rec[15] = {d.w, d.h, static_cast<uint32_t>(x0),
                                    static_cast<uint32_t>(y0), static_cast<uint32_t>(y1),
                                    static_cast<uint32_t>(k), static_cast<uint32_t>(nchunks), g,
                                    rc.nslot, (g / rc.nslot) & 1u, static_cast<uint32_t>(issued),
                                    blo, bhi, static_cast<uint32_t>(r) | (d.L << 16),
                                    d.boxw | (rc.ch << 16)};
          for (int i = 0; i < 15; ++i) diag[1 + i] = rec[i];
          __threadfence();
        }
        // wait, again bounded, for the copies still in flight
        for (int j = k; j < issued; ++j) {
          const uint32_t gj = chunk_ctr + static_cast<uint32_t>(j);
          mbar_wait_bounded(sm.bars + (gj % rc.nslot) * 8u, (gj / rc.nslot) & 1u, timeout_ns);
        }
      }
      __syncthreads();
      return false;
    }
    // every thread has finished chunk k-1, whose slot receives chunk k + pf
    if (k + static_cast<int>(rc.pf) < nchunks) {
      if (t == 0) {
        fence_proxy_async_smem();
        issue(k + static_cast<int>(rc.pf));
      }
      ++issued;
    }
    if (d.fused) {  // raw input pixels: convert the chunk in place
      convert_raw_slot(d, sm.ring + (g % rc.nslot) * rc.slot_bytes, rc.half_bytes, xs,
                       E0 + k * ch, E0 + k * ch - 2 * r - 1, rc.ch, boxw);
      __syncthreads();
    }
    const uint32_t *base_e = ring + (g % rc.nslot) * slot_words;
    const uint32_t *base_l = base_e + half_words;
    const int s_end = min((k + 1) * ch, nsteps);
    for (int s = k * ch; s < s_end; ++s) {
      const uint32_t off = static_cast<uint32_t>(s - k * ch) * boxw;
      step(s, base_e + off, base_l + off);
    }
  }
  chunk_ctr += static_cast<uint32_t>(nchunks);
  return true;
}

// Direct path (path 4), radius R = 0, 1 or 2, any L <= 256: no histogram.  A
// window holds at most (2R+1)^2 = 25 pixels, so its most frequent level is
// found by comparing the pixels' 8-bit levels pairwise (section 4's count per
// level, restricted to the levels present), at a cost independent of L.
// Thread t owns column xa = x0 + t and keeps its window's packed words
// (format 0) in registers, oldest row first, sliding down the tile: each
// step shifts the rows up and appends the entering row from the ring; the
// leaving row is simply dropped (the ring carries entering rows only).  A
// cell outside the image, or in literal mode a white pixel (level L), gets
// the level 256 + k: it matches no other cell, its count stays 0, and it
// cannot win.  Keys (count << 9) | (511 - level) give the largest count and,
// on ties, the lowest level; the winning level's channel sums are summed
// over the matching cells and divided exactly (counts <= 25).
template <int NT, int R>
__device__ bool run_tile_direct(const ImgDesc &d, const CUtensorMap *tmap, int x0, int y0,
                                int y1, const RingCfg &rc, const SmemMap &sm,
                                uint32_t &chunk_ctr, uint32_t *err, uint64_t timeout_ns) {
  static_assert(R >= 0 && R <= kDirectMaxRadius, "direct path radius");
  constexpr int N = 2 * R + 1;
  constexpr int K = N * N;
  const int t = threadIdx.x;
  const int W = static_cast<int>(d.w), H = static_cast<int>(d.h);
  const uint32_t L = d.L;
  const int xa = x0 + t;
  const int xs = (x0 - R) & ~3;  // box start, rounded down to 16 bytes
  const int jl = xa - R - xs;    // ring index of column xa - R
  const int E0 = y0 - R;
  const int nsteps = (y1 - y0) + 2 * R;
  const bool col_out = xa >= d.ox0 && xa < d.ox1;
  uint32_t colmask = 0;  // bit c: column xa - R + c lies in the image
#pragma unroll
  for (int c = 0; c < N; ++c)
    if (xa - R + c >= 0 && xa - R + c < W) colmask |= 1u << c;
  uint32_t win[K];
  uint32_t rowmask = 0;  // bit i: window row i lies in the image
#pragma unroll
  for (int k = 0; k < K; ++k) win[k] = 0u;

  return ring_pass(
      d, tmap, xs, E0, nsteps, rc, sm, chunk_ctr, err, timeout_ns, nullptr, false, x0, y0, y1,
      [&](int s, const uint32_t *rowe, const uint32_t *) {
        const int e = E0 + s;  // entering row
#pragma unroll
        for (int k = 0; k < K - N; ++k) win[k] = win[k + N];
        const uint32_t *pe = rowe + jl;
#pragma unroll
        for (int c = 0; c < N; ++c) win[K - N + c] = pe[c];
        rowmask = (rowmask >> 1) | ((e >= 0 && e < H) ? (1u << (N - 1)) : 0u);
        if (s < 2 * R || !col_out) return;
        const int y = e - R;  // the output row, complete now
        const uint32_t alpha = d.bpp == 4 ? load_alpha(d, xa, y) : 0u;
        uint32_t lv[K];
        uint32_t inmask = (1u << K) - 1u;  // bit k: cell k takes part
        constexpr uint32_t kAll = (1u << N) - 1u;
        if (rowmask == kAll && colmask == kAll && !(d.mode & kModeLiteral)) {
          // inside the image, every level below L: every cell takes part
#pragma unroll
          for (int k = 0; k < K; ++k) lv[k] = win[k] >> 24;
        } else {
          inmask = 0u;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const uint32_t l = win[k] >> 24;
            const bool in = ((rowmask >> (k / N)) & (colmask >> (k % N)) & 1u) && l < L;
            lv[k] = in ? l : 256u + static_cast<uint32_t>(k);
            inmask |= in ? 1u << k : 0u;
          }
        }
        // every pair compared once, both counts updated (one candidate at a
        // time against every cell, with one count live, measured 5% slower
        // at r = 2)
        uint32_t cnt[K];
#pragma unroll
        for (int k = 0; k < K; ++k) cnt[k] = (inmask >> k) & 1u;
#pragma unroll
        for (int a = 0; a < K; ++a)
#pragma unroll
          for (int b = a + 1; b < K; ++b) {
            const uint32_t eq = lv[a] == lv[b] ? 1u : 0u;
            cnt[a] += eq;
            cnt[b] += eq;
          }
        uint32_t best = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) best = max(best, (cnt[k] << 9) | (511u - lv[k]));
        if (best < 512u) return;  // no level below L in the window (literal mode only)
        const uint32_t m = 511u - (best & 511u), n = best >> 9;
        uint32_t Rs = 0, Gs = 0, Bs = 0;
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (lv[k] == m) {
            Rs += (win[k] >> 16) & 0xFFu;
            Gs += (win[k] >> 8) & 0xFFu;
            Bs += win[k] & 0xFFu;
          }
        const uint32_t mul = rcp_of(n);
        store_pixel(d, xa, y, div_mean<kVarA>(Rs, n, mul), div_mean<kVarA>(Gs, n, mul),
                    div_mean<kVarA>(Bs, n, mul), alpha);
      });
}

// One output column per thread: tile [x0, x0 + NT) x [y0, y1), thread t owns
// column x0 + t and a running histogram of its window (2(2r+1) updates per
// output pixel); border threads clip their windows to the image.
template <int NT, int VAR>
__device__ bool run_tile(const ImgDesc &d, const CUtensorMap *tmap, int x0, int y0, int y1,
                         const RingCfg &rc, const SmemMap &sm, uint32_t &chunk_ctr,
                         uint32_t *err, uint64_t timeout_ns, uint32_t *diag = nullptr,
                         bool tmap_global = false) {
  const int t = threadIdx.x;
  const int r = d.r;
  const int W = static_cast<int>(d.w), H = static_cast<int>(d.h);
  const uint32_t L = d.L;
  const int xa = x0 + t;
  const int xs = (x0 - r) & ~3;  // box start, rounded down to 16 bytes
  const int cl = xa - r, cr = xa + r;
  const bool active = xa < W;
  const bool interior = cl >= 0 && cr < W;
  const int jl = cl - xs;  // ring index of column cl (>= 0)
  const int E0 = y0 - r;
  const int nsteps = (y1 - y0) + 2 * r;
  const int j0 = interior ? 0 : max(cl, 0) - cl;
  const int j1 = interior ? 2 * r + 1 : (active ? min(cr, W - 1) - cl + 1 : 0);

  Hist<NT, VAR> h;
  h.sums = sm.sums + static_cast<uint32_t>(t) * 8u;
  h.cnts = sm.cnts + static_cast<uint32_t>(t) * 4u;
  h.clear(L);

  return ring_pass(
      d, tmap, xs, E0, nsteps, rc, sm, chunk_ctr, err, timeout_ns, diag, tmap_global, x0, y0,
      y1, [&](int s, const uint32_t *rowe, const uint32_t *rowl) {
        const int e = E0 + s;         // entering row
        const int l = e - 2 * r - 1;  // leaving row
        const bool do_add = e >= 0 && e < H;
        const bool do_rm = l >= 0 && l >= E0 && l < H;
        // output row e - r is complete and column xa is in the output window
        const bool out_now = s >= 2 * r && xa >= d.ox0 && xa < d.ox1;
        const uint32_t *pe = rowe + jl;
        const uint32_t *pl = rowl + jl;
        // the alpha byte is fetched before the updates so its latency is hidden
        const uint32_t alpha = (out_now && d.bpp == 4) ? load_alpha(d, xa, e - r) : 0u;
        if (do_add && do_rm) {
          int j = j0;
          for (; j + 4 <= j1; j += 4) {
            const uint32_t a0 = pe[j], a1 = pe[j + 1], a2 = pe[j + 2], a3 = pe[j + 3];
            const uint32_t b0 = pl[j], b1 = pl[j + 1], b2 = pl[j + 2], b3 = pl[j + 3];
            h.addsub(a0, b0);
            h.addsub(a1, b1);
            h.addsub(a2, b2);
            h.addsub(a3, b3);
          }
          for (; j < j1; ++j) h.addsub(pe[j], pl[j]);
        } else if (do_add) {
          for (int j = j0; j < j1; ++j) h.add(pe[j]);
        } else if (do_rm) {
          for (int j = j0; j < j1; ++j) h.sub(pl[j]);
        }
        if (out_now) {
          // the first level of the largest count (the strict > scan from
          // level 0).  VAR A: max over keys (count, 255 - level), the count
          // in place in bits 22..31 of the high word -- one or and one max
          // per level; VAR B keeps the scan (its counts would need a shift,
          // and it measured slower as keys).
          uint32_t m = 0, bcount = 0;
          if constexpr (VAR == kVarA) {
            uint32_t best = 0;
            for (uint32_t lv = 0; lv < L; ++lv) best = max(best, h.count_key(lv) | (255u - lv));
            m = 255u - (best & 0xFFu);
            bcount = best >> 22;
          } else {
            for (uint32_t lv = 0; lv < L; ++lv) {
              const uint32_t kk = h.count_key(lv);
              if (kk > bcount) {
                bcount = kk;
                m = lv;
              }
            }
          }
          // no level below L in the window (literal mode only)
          if (bcount != 0u) {
            uint32_t lo, hi, cnt, R, G, B;
            h.bin(m, lo, hi);
            unpack_bin<VAR>(lo, hi, VAR == kVarB ? bcount : 0u, cnt, R, G, B);
            const uint32_t mul = VAR == kVarA ? rcp_of(cnt) : 0u;
            store_pixel(d, xa, e - r, div_mean<VAR>(R, cnt, mul), div_mean<VAR>(G, cnt, mul),
                        div_mean<VAR>(B, cnt, mul), alpha);
          }
        }
      });
}

// K-word vector load from a ring row (K-aligned index, rows 16-byte aligned).
template <int K>
struct VecOf;
template <>
struct VecOf<2> {
  using T = uint2;
  static __device__ __forceinline__ uint32_t at(const uint2 &v, int q) { return q ? v.y : v.x; }
};
template <>
struct VecOf<4> {
  using T = uint4;
  static __device__ __forceinline__ uint32_t at(const uint4 &v, int q) {
    return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
  }
};

// One step's updates of a difference-histogram thread with one window
// histogram H at h0 and D_i at h0 + i*hstride (see run_tile_delta), from the
// ring words 0 .. 2r+K-1 of its entering row pe and, when RM, its leaving
// row pl.  Word j (image column xa - r + j) feeds
//   the window histogram H when j <= 2r,
//   D_{j+1} negatively (its left column leaves) when j <= K-2,
//   D_{j-2r} positively (its right column) when j >= 2r+1.
// Groups of K words are loaded as one vector; the groups that only feed H
// skip the tests.
template <int K, bool RM, class Ops>
__device__ __forceinline__ void delta_step(const Ops &ops, const uint32_t *pe, const uint32_t *pl,
                                           int r, uint32_t h0, uint32_t hstride) {
  using V = typename VecOf<K>::T;
  const int last = 2 * r + K - 1;
  const int ngroups = last / K + 1;
  auto upd = [&](uint32_t base, uint32_t e, uint32_t l) {
    if (RM)
      ops.addsub(base, e, l);
    else
      ops.add(base, e);
  };
  auto updneg = [&](uint32_t base, uint32_t e, uint32_t l) {
    if (RM)
      ops.addsub(base, l, e);
    else
      ops.sub(base, e);
  };
  auto word = [&](int j, uint32_t e, uint32_t l) {
    if (j <= 2 * r) upd(h0, e, l);
    if (j <= K - 2) updneg(h0 + static_cast<uint32_t>(j + 1) * hstride, e, l);
    if (j >= 2 * r + 1 && j <= last) upd(h0 + static_cast<uint32_t>(j - 2 * r) * hstride, e, l);
  };
  auto load = [&](const uint32_t *p) { return *reinterpret_cast<const V *>(p); };
  V a = load(pe), b = V{};
  if (RM) b = load(pl);
#pragma unroll
  for (int q = 0; q < K; ++q) word(q, VecOf<K>::at(a, q), VecOf<K>::at(b, q));
  int g = 1;
#pragma unroll 2
  for (; (g + 1) * K - 1 <= 2 * r; ++g) {
    a = load(pe + g * K);
    if (RM) {
      b = load(pl + g * K);
#pragma unroll
      for (int q = 0; q < K; ++q) upd(h0, VecOf<K>::at(a, q), VecOf<K>::at(b, q));
    } else {
#pragma unroll
      for (int q = 0; q < K; q += 2) ops.add2(h0, VecOf<K>::at(a, q), VecOf<K>::at(a, q + 1));
    }
  }
  for (; g < ngroups; ++g) {
    a = load(pe + g * K);
    if (RM) b = load(pl + g * K);
#pragma unroll
    for (int q = 0; q < K; ++q) word(g * K + q, VecOf<K>::at(a, q), VecOf<K>::at(b, q));
  }
}

// The same step with the window histogram split by word parity: H_even at
// h0 (words 0, 2, .., 2r), H_odd at h0 + hstride (words 1, 3, .., 2r-1) and
// D_i at h0 + (1+i)*hstride.  The two halves are independent, so each
// update of an even word is issued together with one of an odd word (four
// bins in flight instead of two); the last even word pairs with the first
// D update and the D updates pair among themselves.
template <int K, bool RM, class Ops>
__device__ __forceinline__ void delta_step_split(const Ops &ops, const uint32_t *pe,
                                                 const uint32_t *pl, int r, uint32_t h0,
                                                 uint32_t hstride) {
  using V = typename VecOf<K>::T;
  const uint32_t hev = h0, hod = h0 + hstride;
  auto dh = [&](int i) { return h0 + static_cast<uint32_t>(1 + i) * hstride; };
  auto at = [](const V &v, int q) { return VecOf<K>::at(v, q); };
  auto load = [&](const uint32_t *p) { return *reinterpret_cast<const V *>(p); };
  // +e -l in histograms p and q (p != q)
  auto both = [&](uint32_t p, uint32_t ep, uint32_t lp, uint32_t q, uint32_t eq, uint32_t lq) {
    if (RM)
      ops.addsub_x2(p, ep, lp, q, eq, lq);
    else
      ops.template pm_x2<false, false>(p, ep, q, eq);
  };
  // +e -l in histogram p and the column leaving D_i: +l -e in histogram q
  auto with_leaving = [&](uint32_t p, uint32_t ep, uint32_t lp, uint32_t q, uint32_t eq,
                          uint32_t lq) {
    if (RM)
      ops.addsub_x2(p, ep, lp, q, lq, eq);
    else
      ops.template pm_x2<false, true>(p, ep, q, eq);
  };
  const int nfull = (2 * r + 1) / K;  // groups made only of window words
  const V a0 = load(pe);
  V b0 = V{};
  if (RM) b0 = load(pl);
  int g = 0;
  if (nfull > 0) {
#pragma unroll
    for (int q = 0; q < K; q += 2) both(hev, at(a0, q), at(b0, q), hod, at(a0, q + 1), at(b0, q + 1));
    g = 1;
  }
#pragma unroll 2
  for (; g < nfull; ++g) {
    const V a = load(pe + g * K);
    V b = V{};
    if (RM) b = load(pl + g * K);
    if (!RM && K == 4) {
      // the fill only adds: H_even's two words chain, as do H_odd's
      ops.add2x2(hev, at(a, 0), at(a, 2), hod, at(a, 1), at(a, 3));
    } else {
#pragma unroll
      for (int q = 0; q < K; q += 2)
        both(hev, at(a, q), at(b, q), hod, at(a, q + 1), at(b, q + 1));
    }
  }
  // the c = 2r + 1 - nfull*K remaining window words (c odd, 1 <= c < K);
  // the last is even and goes to H_even together with D_1's leaving word 0
  V ta = a0, tb = b0;
  if (nfull > 0) {
    ta = load(pe + nfull * K);
    if (RM) tb = load(pl + nfull * K);
  }
  uint32_t es = at(ta, 0), ls = at(tb, 0);
  if (K == 4 && 2 * r + 1 - nfull * K == 3) {
    both(hev, at(ta, 0), at(tb, 0), hod, at(ta, 1), at(tb, 1));
    es = at(ta, 2);
    ls = at(tb, 2);
  }
  with_leaving(hev, es, ls, dh(1), at(a0, 0), at(b0, 0));
  const uint32_t *pe2 = pe + 2 * r + 1, *pl2 = pl + 2 * r + 1;
  if (K == 2) {
    const uint32_t e = pe2[0], l = RM ? pl2[0] : 0u;
    if (RM)
      ops.addsub(dh(1), e, l);
    else
      ops.add(dh(1), e);
  } else {
    // D_2, D_3 lose words 1, 2; D_1, D_2, D_3 gain words 2r+1, 2r+2, 2r+3
    if (RM)
      ops.addsub_x2(dh(2), at(b0, 1), at(a0, 1), dh(3), at(b0, 2), at(a0, 2));
    else
      ops.template pm_x2<true, true>(dh(2), at(a0, 1), dh(3), at(a0, 2));
    const uint32_t e1 = pe2[0], e2 = pe2[1], e3 = pe2[2];
    const uint32_t l1 = RM ? pl2[0] : 0u, l2 = RM ? pl2[1] : 0u, l3 = RM ? pl2[2] : 0u;
    both(dh(1), e1, l1, dh(2), e2, l2);
    if (RM)
      ops.addsub(dh(3), e3, l3);
    else
      ops.add(dh(3), e3);
  }
}

// Into how many histograms the K-column path splits the window histogram
// (by column parity): with four columns per thread a second, independent
// update chain pays for the extra histogram; with two columns the extra
// histogram costs more occupancy than the chain gains, and a four-way split
// of the four-column window histogram measured slower still (two more
// histograms per thread, one resident CTA fewer per SM).  Variant B bins
// (10 bytes) never split: split, the K = 4 path ran 5-22% slower at r = 16..44
// (5 instead of 7 resident CTAs per SM at r = 20, L = 20).
constexpr int kSplit2 = 1;
constexpr int kSplit4 = 2;
__host__ __device__ constexpr int hsplit(int k, int var) {
  return var == kVarA ? (k == 4 ? kSplit4 : kSplit2) : 1;
}

// K output columns per thread through difference histograms (r <= 44,
// L <= 32; VAR A for r <= 15 with word format 1, VAR B above with word
// format 2).  Thread t owns columns xa .. xa+K-1 with xa = x0 + K*t; x0 - r
// is a multiple of 4 (tiles start at d.xshift), so every thread's window
// starts on a 16-byte boundary of the ring.  It keeps
//   H    the histogram of the window of column xa (2r+1 columns; split into
//        hsplit(K, VAR) histograms by column index where that is above 1),
//   D_i  (i = 1..K-1) the histogram of column xa+i+r minus that of column
//        xa+i-1-r, so that the window histogram of column xa+i is
//        H + D_1 + ... + D_i.
// A step costs 2(2r+1) + 4(K-1) bin updates for K outputs.  Histograms are
// L levels of NT bins, interleaved level-major (a level's NH rows of NT bins
// are adjacent, thread-minor); VAR B keeps its 16-bit counts in a second
// array of the same shape.  The argmax runs over running sums of counts (VAR A: the
// histograms' low words, whose bottom 10 bits are the counts) with keys
// (count, 31 - level), so the lowest level wins ties under max.  Pixels
// outside the image are TMA zero fill whose delta is zero, so no thread
// clips its window.
template <int NT, int K, int VAR>
__device__ bool run_tile_delta(const ImgDesc &d, const CUtensorMap *tmap, int x0, int y0,
                               int y1, const RingCfg &rc, const SmemMap &sm,
                               uint32_t &chunk_ctr, uint32_t *err, uint64_t timeout_ns,
                               uint32_t *diag = nullptr, bool tmap_global = false) {
  static_assert(K == 2 || K == 4, "two or four columns per thread");
  constexpr int NB = hsplit(K, VAR);  // histograms making up H
  static_assert(NB == 1 || NB == 2, "split of H");
  constexpr int NH = NB + K - 1;
  const int t = threadIdx.x;
  const int r = d.r;
  const uint32_t L = d.L;
  const int xa = x0 + K * t;
  const int xs = x0 - r;  // a multiple of 4 by the choice of d.xshift
  const int jl = K * t;
  const int E0 = y0 - r;
  const int nsteps = (y1 - y0) + 2 * r;
  // Level-major layout: level lv of histogram i, thread t at
  // sums + lv * NH*NT*8 + i * NT*8 + t * 8, so the NH bins a thread reads for
  // one level of the argmax lie at fixed offsets from one address.
  constexpr uint32_t LS = NH * NT * 8u;
  const uint32_t lstride = LS;       // between levels of one histogram
  const uint32_t hstride = NT * 8u;  // between histograms
  const uint32_t h0 = sm.sums + static_cast<uint32_t>(t) * 8u;
  // VAR B counts (16 bits): same shape at a quarter of the stride, after the sums
  const uint32_t cbase = sm.sums + L * LS;
  const uint32_t cd = cbase - (sm.sums >> 2);
  using Ops = typename std::conditional<VAR == kVarA, DeltaOpsA<LS>, DeltaOpsB<LS, 2u>>::type;
  Ops ops;
  if constexpr (VAR == kVarB) ops.cd = cd;
  auto hist = [&](int i) { return h0 + static_cast<uint32_t>(i) * hstride; };
  auto cnt_of = [&](uint32_t s) { return (s >> 2) + cd; };
#pragma unroll
  for (int i = 0; i < NH; ++i)
    for (uint32_t lv = 0; lv < L; ++lv) {
      sts_zero64(hist(i) + lv * lstride);
      if (VAR == kVarB) sts_u16(cnt_of(hist(i) + lv * lstride), 0u);
    }

  return ring_pass(
      d, tmap, xs, E0, nsteps, rc, sm, chunk_ctr, err, timeout_ns, diag, tmap_global, x0, y0,
      y1, [&](int s, const uint32_t *rowe, const uint32_t *rowl) {
        const bool rm = s >= 2 * r + 1;  // the leaving row was added by this tile
        const bool out_now = s >= 2 * r;
        const int y = E0 + s - r;
        const uint32_t *pe = rowe + jl;
        const uint32_t *pl = rowl + jl;
        uint32_t alpha[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const int x = xa + i;
          alpha[i] = (out_now && d.bpp == 4 && x >= d.ox0 && x < d.ox1) ? load_alpha(d, x, y) : 0u;
        }
        if constexpr (NB == 2) {
          if (rm)
            delta_step_split<K, true>(ops, pe, pl, r, h0, hstride);
          else
            delta_step_split<K, false>(ops, pe, pl, r, h0, hstride);
        } else {
          if (rm)
            delta_step<K, true>(ops, pe, pl, r, h0, hstride);
          else
            delta_step<K, false>(ops, pe, pl, r, h0, hstride);
        }
        if (!out_now) return;
        // count of level lv in histogram i (VAR A: the low word, count in bits 0..9)
        auto count_word = [&](int i, uint32_t lv) {
          const uint32_t a = hist(i) + lv * lstride;
          if constexpr (VAR == kVarA)
            return lds_u32(a);
          else
            return lds_u16(cnt_of(a));
        };
        // the shift keeps the count's bits and drops the rest (VAR A: the
        // sums above the 10-bit count; VAR B: the wrap of the 16-bit counts)
        constexpr int CSH = VAR == kVarA ? 22 : 16;
        uint32_t best[K];
#pragma unroll
        for (int i = 0; i < K; ++i) best[i] = 0u;
        for (uint32_t lv = 0; lv < L; ++lv) {
          uint32_t acc = count_word(0, lv);
#pragma unroll
          for (int b = 1; b < NB; ++b) acc += count_word(b, lv);
          // key of window i = (count_i << CSH) | (31 - lv); the key of window
          // i follows from that of window i-1 by adding D_i's count word
          // shifted into place (the shift drops VAR A's sums above the count,
          // and the tag bits below CSH are untouched)
          uint32_t key = (acc << CSH) | (31u - lv);
          best[0] = max(best[0], key);
#pragma unroll
          for (int i = 1; i < K; ++i) {
            key += count_word(NB - 1 + i, lv) << CSH;
            best[i] = max(best[i], key);
          }
        }
        // the reciprocals are fetched first, so that their latency overlaps
        // the loads of the winning bins
        uint32_t mulv[K];
#pragma unroll
        for (int i = 0; i < K; ++i) mulv[i] = VAR == kVarA ? rcp_of(best[i] >> CSH) : 0u;
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const int x = xa + i;
          if (x < d.ox0 || x >= d.ox1) continue;
          const uint32_t m = 31u - (best[i] & 31u);
          const uint32_t cnt = best[i] >> CSH;
          if (cnt == 0u) continue;  // no level below L (literal mode only)
          uint64_t v = 0;
#pragma unroll
          for (int j = 0; j < NB + i; ++j) {
            uint32_t lo, hi;
            lds_v2(hist(j) + m * lstride, lo, hi);
            v += static_cast<uint64_t>(hi) << 32 | lo;
          }
          const uint32_t lo = static_cast<uint32_t>(v);
          const uint32_t hi = static_cast<uint32_t>(v >> 32);
          if (VAR == kVarA) {
            const uint32_t R = (lo >> 10) & 0x3FFFFu;
            const uint32_t G = (lo >> 28) | ((hi & 0x3FFFu) << 4);
            const uint32_t B = hi >> 14;
            const uint32_t mul = mulv[i];
            store_pixel(d, x, y, __umulhi(R << 1, mul), __umulhi(G << 1, mul),
                        __umulhi(B << 1, mul), alpha[i]);
          } else {
            const uint32_t R = lo & 0x1FFFFFu;
            const uint32_t G = (lo >> 21) | ((hi & 0x3FFu) << 11);
            const uint32_t B = (hi >> 10) & 0x1FFFFFu;
            store_pixel(d, x, y, R / cnt, G / cnt, B / cnt, alpha[i]);
          }
        }
      });
}

// ------------------------------------------------ eight columns per thread
//
// K = 8 output columns per thread (run_tile_delta8): variant-A bins and word
// format 1, 4 <= r <= 15, L <= 32, the radius a template parameter so that a
// step is straight-line code.  Thread t owns columns xa .. xa+7 (xa = x0 + 8t)
// and keeps the histogram of the window of column xa, split by the parity of
// the window column into He and Ho (two independent update chains), and
// D_1 .. D_7, the histograms of column xa+i+r minus column xa+i-1-r:
// 2(2r+1) + 28 bin updates per 8 outputs (11.25 per output at r = 15,
// against 18.5 with four columns).  With eight windows the argmax would read
// nine count words per level, so the counts of D_1 .. D_7 are kept a second
// time, as signed bytes packed into two words per level and thread (DC:
// D_1..D_4 at bits 8(i-1) of word 0, D_5..D_7 at bits 8(i-5) of word 1; a
// pixel adds its valid bit there, so the zero words outside the image count
// nothing), and a level costs four loads: the low words of He and Ho and the
// two DC words.  A D_i count lies in [-31, 31] (two columns of at most 31
// pixels), so the prefix sums of the bytes of one word lie in [-124, 124]:
// multiplying the word by 0x01010101 replaces each byte by the sum of the
// bytes up to it (the word is linear in its signed bytes mod 2^32), and
// adding 0x80808080 then maps every prefix to an unsigned byte with no carry
// between bytes.
//
// The updates are issued in blocks of up to three bin pairs (one on He, one
// on Ho, one on a D_i with its pair of DC words), all loads first.  The two
// bins of a pair may coincide; the second's delta then includes the first's
// (decided from the addresses alone, before the loads), so that the second
// store, which lands last, holds both updates and no bin's load-add-store
// chain waits on another's.
//
// Shared memory (after the ring): 64-bit bins [level][histogram][thread],
// histograms He, Ho, D_1..D_7 numbered 0..8, then the DC words
// [level][word][thread].

// A 64-bit bin update (shared address, delta) and a 32-bit one.
struct Upd64 {
  uint32_t a;
  uint64_t d;
};
struct Upd32 {
  uint32_t a, v;
};

// Pairs (A, B) on He, (C, D) on Ho and (E, F) on a D_i with its count words
// (G, H): A, C, E, G add; B and D subtract (SUB) or add; F and H subtract.
// All loads first, then the stores in slot order.
template <bool SUB>
__device__ __forceinline__ void blk_hhd(const Upd64 &A, const Upd64 &B, const Upd64 &C,
                                        const Upd64 &D, const Upd64 &E, const Upd64 &F,
                                        const Upd32 &G, const Upd32 &H) {
  if (!OPK_SMEM_OK(A.a, 8u) || !OPK_SMEM_OK(B.a, 8u) || !OPK_SMEM_OK(C.a, 8u) ||
      !OPK_SMEM_OK(D.a, 8u) || !OPK_SMEM_OK(E.a, 8u) || !OPK_SMEM_OK(F.a, 8u) ||
      !OPK_SMEM_OK(G.a, 4u) || !OPK_SMEM_OK(H.a, 4u))
    return;
  const uint64_t a = ld_bin(A.a), b = ld_bin(B.a), c = ld_bin(C.a), d = ld_bin(D.a);
  const uint64_t e = ld_bin(E.a), f = ld_bin(F.a);
  const uint32_t g = ld_w32(G.a), h = ld_w32(H.a);
  st_bin(A.a, a + A.d);
  st_bin(B.a, SUB ? b - B.d : b + B.d);
  st_bin(C.a, c + C.d);
  st_bin(D.a, SUB ? d - D.d : d + D.d);
  st_bin(E.a, e + E.d);
  st_bin(F.a, f - F.d);
  st_w32(G.a, g + G.v);
  st_w32(H.a, h - H.v);
}

// Pairs (A, B) and (C, D) on two histograms.
template <bool SUB>
__device__ __forceinline__ void blk_hh(const Upd64 &A, const Upd64 &B, const Upd64 &C,
                                       const Upd64 &D) {
  if (!OPK_SMEM_OK(A.a, 8u) || !OPK_SMEM_OK(B.a, 8u) || !OPK_SMEM_OK(C.a, 8u) ||
      !OPK_SMEM_OK(D.a, 8u))
    return;
  const uint64_t a = ld_bin(A.a), b = ld_bin(B.a), c = ld_bin(C.a), d = ld_bin(D.a);
  st_bin(A.a, a + A.d);
  st_bin(B.a, SUB ? b - B.d : b + B.d);
  st_bin(C.a, c + C.d);
  st_bin(D.a, SUB ? d - D.d : d + D.d);
}

// Pair (A, B) on He or Ho, pair (E, F) on a D_i with its count words (G, H).
template <bool SUB>
__device__ __forceinline__ void blk_hd(const Upd64 &A, const Upd64 &B, const Upd64 &E,
                                       const Upd64 &F, const Upd32 &G, const Upd32 &H) {
  if (!OPK_SMEM_OK(A.a, 8u) || !OPK_SMEM_OK(B.a, 8u) || !OPK_SMEM_OK(E.a, 8u) ||
      !OPK_SMEM_OK(F.a, 8u) || !OPK_SMEM_OK(G.a, 4u) || !OPK_SMEM_OK(H.a, 4u))
    return;
  const uint64_t a = ld_bin(A.a), b = ld_bin(B.a), e = ld_bin(E.a), f = ld_bin(F.a);
  const uint32_t g = ld_w32(G.a), h = ld_w32(H.a);
  st_bin(A.a, a + A.d);
  st_bin(B.a, SUB ? b - B.d : b + B.d);
  st_bin(E.a, e + E.d);
  st_bin(F.a, f - F.d);
  st_w32(G.a, g + G.v);
  st_w32(H.a, h - H.v);
}

// Pair (A, B) on one histogram.
template <bool SUB>
__device__ __forceinline__ void blk_h(const Upd64 &A, const Upd64 &B) {
  if (!OPK_SMEM_OK(A.a, 8u) || !OPK_SMEM_OK(B.a, 8u)) return;
  const uint64_t a = ld_bin(A.a), b = ld_bin(B.a);
  st_bin(A.a, a + A.d);
  st_bin(B.a, SUB ? b - B.d : b + B.d);
}

// As blk_hd and blk_h, with the window pair (A, B) chained instead of
// alias-safe: B's delta is its own, and when A == B the second update
// applies to the first's sum (one select after the loads, two instructions
// fewer than computing the alias-safe delta).
template <bool SUB>
__device__ __forceinline__ void blk_hd_chain(const Upd64 &A, const Upd64 &B, const Upd64 &E,
                                             const Upd64 &F, const Upd32 &G, const Upd32 &H) {
  if (!OPK_SMEM_OK(A.a, 8u) || !OPK_SMEM_OK(B.a, 8u) || !OPK_SMEM_OK(E.a, 8u) ||
      !OPK_SMEM_OK(F.a, 8u) || !OPK_SMEM_OK(G.a, 4u) || !OPK_SMEM_OK(H.a, 4u))
    return;
  const uint64_t a0 = ld_bin(A.a), b0 = ld_bin(B.a), e = ld_bin(E.a), f = ld_bin(F.a);
  const uint32_t g = ld_w32(G.a), h = ld_w32(H.a);
  const uint64_t a = a0 + A.d;
  const uint64_t b = A.a == B.a ? a : b0;
  st_bin(A.a, a);
  st_bin(B.a, SUB ? b - B.d : b + B.d);
  st_bin(E.a, e + E.d);
  st_bin(F.a, f - F.d);
  st_w32(G.a, g + G.v);
  st_w32(H.a, h - H.v);
}

template <bool SUB>
__device__ __forceinline__ void blk_h_chain(const Upd64 &A, const Upd64 &B) {
  if (!OPK_SMEM_OK(A.a, 8u) || !OPK_SMEM_OK(B.a, 8u)) return;
  const uint64_t a0 = ld_bin(A.a), b0 = ld_bin(B.a);
  const uint64_t a = a0 + A.d;
  const uint64_t b = A.a == B.a ? a : b0;
  st_bin(A.a, a);
  st_bin(B.a, SUB ? b - B.d : b + B.d);
}

// Pair (E, F) on a D_i (E adds, F subtracts) with its count words (G, H).
__device__ __forceinline__ void blk_d(const Upd64 &E, const Upd64 &F, const Upd32 &G,
                                      const Upd32 &H) {
  if (!OPK_SMEM_OK(E.a, 8u) || !OPK_SMEM_OK(F.a, 8u) || !OPK_SMEM_OK(G.a, 4u) ||
      !OPK_SMEM_OK(H.a, 4u))
    return;
  const uint64_t e = ld_bin(E.a), f = ld_bin(F.a);
  const uint32_t g = ld_w32(G.a), h = ld_w32(H.a);
  st_bin(E.a, e + E.d);
  st_bin(F.a, f - F.d);
  st_w32(G.a, g + G.v);
  st_w32(H.a, h - H.v);
}

// One thread's histograms and count words for K output columns per thread
// (K = 2, 4 or 8), the window histogram split into NB = 1 or 2 parts (by the
// parity of the window column; NB = 1 for K = 2), and the updates of one
// packed word (word format 1).  Histograms 0 .. NB-1 are the window
// histogram's parts, NB - 1 + i is D_i.  The count words hold, for K = 4 and
// 8, the counts of D_1 .. D_4 (word 0) and D_5 .. D_7 (word 1) of one level;
// for K = 2 (L <= 64) the counts of D_1 at four consecutive levels (byte
// lv & 3 of word lv / 4).  The level is read as the 5-bit field at bits 1..5
// (L <= 32) or, for K = 2, with bit 18 as its sixth bit.
template <int NT, int K, int NB>
struct DeltaK {
  static_assert((K == 2 && NB == 1) || ((K == 4 || K == 8) && (NB == 1 || NB == 2)),
                "K columns, NB window parts");
  static constexpr int kHists = NB + K - 1;
  static constexpr int kDCWords = (K - 1 + 3) / 4;  // per level (K = 4, 8)
  static constexpr uint32_t kHS = NT * 8u;                   // between histograms
  static constexpr uint32_t kLS = kHists * kHS;              // between levels (bins)
  static constexpr uint32_t kDW = NT * 4u;                   // between DC words
  static constexpr uint32_t kDLS = kDCWords * kDW;           // between levels (DC, K = 4, 8)
  uint32_t h0;   // the first window part's level-0 bin of this thread
  uint32_t dc0;  // this thread's first DC word

  // twice word w's level
  static __device__ __forceinline__ uint32_t lv2(uint32_t w) {
    if constexpr (K == 2)
      return (w & 0x3Eu) | ((w >> 12) & 0x40u);
    else
      return w & 0x3Eu;
  }
  // +w in histogram k
  __device__ __forceinline__ Upd64 add(int k, uint32_t w) const {
    uint32_t lo, hi;
    dh_delta(w, lo, hi);
    return Upd64{h0 + static_cast<uint32_t>(k) * kHS + lv2(w) * (kLS / 2u), u64_of(lo, hi)};
  }
  // the second update of a pair whose first is `first`, of word w in
  // histogram k, to be subtracted (SUB) or added; when both land on one bin
  // it also carries the first's delta
  template <bool SUB>
  __device__ __forceinline__ Upd64 second(const Upd64 &first, int k, uint32_t w) const {
    const Upd64 u = add(k, w);
    const uint64_t x = u.a == first.a ? first.d : 0ull;
    return Upd64{u.a, SUB ? u.d - x : u.d + x};
  }
  // D_i's count word at word w's level and the word's valid bit moved to
  // D_i's byte (K = 4, 8) or to the level's byte (K = 2)
  __device__ __forceinline__ Upd32 cnt(int i, uint32_t w) const {
    if constexpr (K == 2) {
      const uint32_t l2 = lv2(w);  // 2 * level
      return Upd32{dc0 + (l2 >> 3) * kDW, (w & 1u) << ((l2 & 6u) << 2)};
    } else {
      return Upd32{dc0 + static_cast<uint32_t>((i - 1) >> 2) * kDW + lv2(w) * (kDLS / 2u),
                   (w & 1u) << (8 * ((i - 1) & 3))};
    }
  }
  // D_i: +a -b (sums and count)
  __device__ __forceinline__ void dpair(int i, uint32_t a, uint32_t b, Upd64 &E, Upd64 &F,
                                        Upd32 &G, Upd32 &H) const {
    E = add(NB - 1 + i, a);
    F = second<true>(E, NB - 1 + i, b);
    G = cnt(i, a);
    H = cnt(i, b);
    if (H.a == G.a) H.v -= G.v;
  }
};

// One step of run_tile_deltak from the ring words 0 .. 2R+K-1 (read as
// 16-byte groups, 8-byte for K = 2) of the entering row pe and (RM) the
// leaving row pl.  Word j
// feeds the window histogram when j <= 2R (with NB = 2: part 0 for even j,
// part 1 for odd j), D_{j+1} negatively (its left column leaves the window)
// when j <= K-2, and D_{j-2R} positively (its right column enters) when
// j >= 2R+1; R >= K/2 keeps the words 0 .. K-2 inside the window and apart
// from the right words.  While the window fills (RM false) rows only enter.
template <int NT, int K, int NB, int R, bool RM>
__device__ __forceinline__ void deltak_step(const DeltaK<NT, K, NB> &o, const uint32_t *pe,
                                            const uint32_t *pl) {
  // groups of GW words covering words 0 .. 2R+K-1: 16 bytes, or 8 for K = 2
  // (a two-column thread's window starts on an 8-byte boundary only)
  constexpr int GW = K == 2 ? 2 : 4;
  constexpr int NG = (2 * R + K + GW - 1) / GW;
  constexpr int ND = 2 * (K - 1);  // D pairs of a step
  uint32_t e[GW * NG], l[GW * NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    if constexpr (GW == 4) {
      const uint4 v = *reinterpret_cast<const uint4 *>(pe + 4 * g);
      e[4 * g] = v.x;
      e[4 * g + 1] = v.y;
      e[4 * g + 2] = v.z;
      e[4 * g + 3] = v.w;
      if (RM) {
        const uint4 u = *reinterpret_cast<const uint4 *>(pl + 4 * g);
        l[4 * g] = u.x;
        l[4 * g + 1] = u.y;
        l[4 * g + 2] = u.z;
        l[4 * g + 3] = u.w;
      } else {
        l[4 * g] = l[4 * g + 1] = l[4 * g + 2] = l[4 * g + 3] = 0u;
      }
    } else {
      const uint2 v = *reinterpret_cast<const uint2 *>(pe + 2 * g);
      e[2 * g] = v.x;
      e[2 * g + 1] = v.y;
      if (RM) {
        const uint2 u = *reinterpret_cast<const uint2 *>(pl + 2 * g);
        l[2 * g] = u.x;
        l[2 * g + 1] = u.y;
      } else {
        l[2 * g] = l[2 * g + 1] = 0u;
      }
    }
  }
  Upd64 A, B, C, D, E, F;
  Upd32 G, H;
  if constexpr (RM) {
    // D pair k: the left words (k < K-1: D_{k+1} +l_k -e_k), then the right
    // words (k >= K-1: D_{k-K+2} +e -l at word 2R + k - K + 2)
    auto dp = [&](int k) {
      if (k < K - 1)
        o.dpair(k + 1, l[k], e[k], E, F, G, H);
      else
        o.dpair(k - K + 2, e[2 * R + k - K + 2], l[2 * R + k - K + 2], E, F, G, H);
    };
    if constexpr (NB == 2) {
      // block b: part-0 pair at word 2b, part-1 pair at word 2b+1 (b < R), D pair b
#pragma unroll
      for (int b = 0; b <= R; ++b) {
        A = o.add(0, e[2 * b]);
        B = o.template second<true>(A, 0, l[2 * b]);
        if (b < R) {
          C = o.add(1, e[2 * b + 1]);
          D = o.template second<true>(C, 1, l[2 * b + 1]);
          if (b < ND) {
            dp(b);
            blk_hhd<true>(A, B, C, D, E, F, G, H);
          } else {
            blk_hh<true>(A, B, C, D);
          }
        } else if (b < ND) {
          dp(b);
          blk_hd<true>(A, B, E, F, G, H);
        } else {
          blk_h<true>(A, B);
        }
      }
#pragma unroll
      for (int k = R + 1; k < ND; ++k) {
        dp(k);
        blk_d(E, F, G, H);
      }
    } else {
      // block j: the window pair at word j (chained), D pair j
#pragma unroll
      for (int j = 0; j <= 2 * R; ++j) {
        A = o.add(0, e[j]);
        B = o.add(0, l[j]);
        if (j < ND) {
          dp(j);
          blk_hd_chain<true>(A, B, E, F, G, H);
        } else {
          blk_h_chain<true>(A, B);
        }
      }
#pragma unroll
      for (int k = 2 * R + 1; k < ND; ++k) {
        dp(k);
        blk_d(E, F, G, H);
      }
    }
  } else {
    // D pair q: D_{q+1} +(word 2R + q + 1) -(word q)
    if constexpr (NB == 2) {
      // part-0 pairs of even words (4q, 4q + 2), part-1 pairs of odd words
      // (4q + 1, 4q + 3)
      constexpr int NPE = (R + 1) / 2, NPO = R / 2;
      constexpr int NQ = NPE > NPO ? NPE : NPO;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const bool he = q < NPE, ho = q < NPO, hd = q < K - 1;
        if (he) {
          A = o.add(0, e[4 * q]);
          B = o.template second<false>(A, 0, e[4 * q + 2]);
        }
        if (ho) {
          C = o.add(1, e[4 * q + 1]);
          D = o.template second<false>(C, 1, e[4 * q + 3]);
        }
        if (hd) o.dpair(q + 1, e[2 * R + q + 1], e[q], E, F, G, H);
        if (he && ho && hd)
          blk_hhd<false>(A, B, C, D, E, F, G, H);
        else if (he && ho)
          blk_hh<false>(A, B, C, D);
        else if (he && hd)
          blk_hd<false>(A, B, E, F, G, H);
        else if (ho && hd)
          blk_hd<false>(C, D, E, F, G, H);
        else if (he)
          blk_h<false>(A, B);
        else if (ho)
          blk_h<false>(C, D);
      }
      if ((R + 1) % 2) {
        A = o.add(0, e[2 * R]);
        bin_add64(A.a, static_cast<uint32_t>(A.d), static_cast<uint32_t>(A.d >> 32));
      }
      if (R % 2) {
        C = o.add(1, e[2 * R - 1]);
        bin_add64(C.a, static_cast<uint32_t>(C.d), static_cast<uint32_t>(C.d >> 32));
      }
#pragma unroll
      for (int q = NQ; q < K - 1; ++q) {
        o.dpair(q + 1, e[2 * R + q + 1], e[q], E, F, G, H);
        blk_d(E, F, G, H);
      }
    } else {
      // window pairs (2q, 2q + 1) (chained), then the last window word 2R
#pragma unroll
      for (int q = 0; q < R; ++q) {
        A = o.add(0, e[2 * q]);
        B = o.add(0, e[2 * q + 1]);
        if (q < K - 1) {
          o.dpair(q + 1, e[2 * R + q + 1], e[q], E, F, G, H);
          blk_hd_chain<false>(A, B, E, F, G, H);
        } else {
          blk_h_chain<false>(A, B);
        }
      }
      A = o.add(0, e[2 * R]);
      bin_add64(A.a, static_cast<uint32_t>(A.d), static_cast<uint32_t>(A.d >> 32));
#pragma unroll
      for (int q = R; q < K - 1; ++q) {
        o.dpair(q + 1, e[2 * R + q + 1], e[q], E, F, G, H);
        blk_d(E, F, G, H);
      }
    }
  }
}

// K output columns per thread (see above); the tile [x0, x0 + K NT) x
// [y0, y1), x0 - R a multiple of 4 (tiles start at d.xshift), so every
// thread's window starts on a 16-byte boundary of the ring.  Pixels outside
// the image are zero words (TMA fill, and the zeroed row padding), whose
// delta is zero.
template <int NT, int K, int NB, int R>
__device__ bool run_tile_deltak(const ImgDesc &d, const CUtensorMap *tmap, int x0, int y0, int y1,
                                const RingCfg &rc, const SmemMap &sm, uint32_t &chunk_ctr,
                                uint32_t *err, uint64_t timeout_ns, uint32_t *diag = nullptr,
                                bool tmap_global = false) {
  using O = DeltaK<NT, K, NB>;
  const int t = threadIdx.x;
  const uint32_t L = d.L;
  const int xa = x0 + K * t;
  const int xs = x0 - R;  // a multiple of 4 by the choice of d.xshift
  const int jl = K * t;
  const int E0 = y0 - R;
  const int nsteps = (y1 - y0) + 2 * R;
  O o;
  o.h0 = sm.sums + static_cast<uint32_t>(t) * 8u;
  o.dc0 = sm.sums + L * O::kLS + static_cast<uint32_t>(t) * 4u;
  for (uint32_t lv = 0; lv < L; ++lv) {
#pragma unroll
    for (int i = 0; i < O::kHists; ++i)
      sts_zero64(o.h0 + lv * O::kLS + static_cast<uint32_t>(i) * O::kHS);
    if constexpr (K != 2) {
#pragma unroll
      for (int w = 0; w < O::kDCWords; ++w)
        sts_zero32(o.dc0 + lv * O::kDLS + static_cast<uint32_t>(w) * O::kDW);
    }
  }
  if constexpr (K == 2)  // one count word per four levels
    for (uint32_t q = 0; q < (L + 3u) / 4u; ++q) sts_zero32(o.dc0 + q * O::kDW);

  return ring_pass(
      d, tmap, xs, E0, nsteps, rc, sm, chunk_ctr, err, timeout_ns, diag, tmap_global, x0, y0,
      y1, [&](int s, const uint32_t *rowe, const uint32_t *rowl) {
        const bool rm = s >= 2 * R + 1;  // the leaving row was added by this tile
        const bool out_now = s >= 2 * R;
        const int y = E0 + s - R;
        const uint32_t *pe = rowe + jl;
        const uint32_t *pl = rowl + jl;
        uint32_t alpha[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const int x = xa + i;
          alpha[i] = (out_now && d.bpp == 4 && x >= d.ox0 && x < d.ox1) ? load_alpha(d, x, y) : 0u;
        }
        if (rm)
          deltak_step<NT, K, NB, R, true>(o, pe, pl);
        else
          deltak_step<NT, K, NB, R, false>(o, pe, pl);
        if (!out_now) return;
        // keys (count << 22) | (31 - level): the lowest level wins ties under max
        uint32_t best[K];
#pragma unroll
        for (int i = 0; i < K; ++i) best[i] = 0u;
        // the level tag: 6 bits (L <= 64) for two columns, else 5
        constexpr uint32_t kTag = K == 2 ? 63u : 31u;
        if constexpr (K == 2) {
          // windows 0 and 1 as the halves of one word: 16-bit keys
          // (count << 6) | (63 - level), below 2^16 for count <= 961; window
          // 1 adds D_1's signed count times 64 to the high half, whose sum
          // stays in [0, 2^16).  The four levels' counts share a word as
          // signed bytes, linear mod 2^32 (a negative byte borrows from the
          // next), so the word plus 0x80808080 holds each count plus 128 as
          // an unsigned byte, no carry between them.
          uint32_t b01 = 0u;
          for (uint32_t lq = 0; lq < L; lq += 4u) {
            const uint32_t dw = lds_u32(o.dc0 + (lq >> 2) * O::kDW) + 0x80808080u;
#pragma unroll
            for (uint32_t k = 0; k < 4u; ++k) {
              const uint32_t lv = lq + k;
              if (lv >= L) break;
              const uint32_t c = lds_u32(o.h0 + lv * O::kLS);
              // (count + 128) << 22, less 128 << 22: the count times 64 in the high half
              const uint32_t x = (((dw >> (8u * k)) & 0xFFu) << 22) - (128u << 22);
              const uint32_t k0 = ((c << 6) & 0xFFC0u) | (63u - lv);
              b01 = __viaddmax_u16x2(k0 * 0x00010001u, x, b01);
            }
          }
          auto key32 = [](uint32_t h) { return (h & 0xFFC0u) << 16 | (h & 63u); };
          best[0] = key32(b01 & 0xFFFFu);
          best[1] = key32(b01 >> 16);
        } else if constexpr (K == 4) {
          // two windows per word: 16-bit keys (count << 5) | (31 - level)
          // (count <= 961, so a key is below 2^15), max per halfword
          uint32_t b01 = 0u, b23 = 0u;
#pragma unroll 4
          for (uint32_t lv = 0; lv < L; ++lv) {
            uint32_t c = lds_u32(o.h0 + lv * O::kLS);
            if (NB == 2) c += lds_u32(o.h0 + lv * O::kLS + O::kHS);
            // byte k of p: 128 + the count of D_1 + .. + D_{k+1}
            const uint32_t p = lds_u32(o.dc0 + lv * O::kDLS) * 0x01010101u + 0x80808080u;
            const uint32_t k0 = ((c << 5) & 0x7FE0u) | (31u - lv);
            // window 1 (high half of b01) adds byte 0, windows 2 and 3 (b23)
            // bytes 1 and 2, each still carrying its bias of 128, i.e. 4096
            // in the key: the same for every level of a window, so it leaves
            // the argmax alone, keeps every halfword within 16 bits (at most
            // 30783 + 4096) and is taken off once after the loop
            const uint32_t x01 = __byte_perm(p, 0u, 0x4044u) << 5;  // byte 0 -> high half
            const uint32_t x23 = __byte_perm(p, 0u, 0x4241u) << 5;  // bytes 1, 2 -> low, high
            b01 = __viaddmax_u16x2(k0 * 0x00010001u, x01, b01);
            b23 = __viaddmax_u16x2(k0 * 0x00010001u, x23, b23);
          }
          // back to the 32-bit keys (count << 22) | tag of the general code
          auto key32 = [](uint32_t h) { return (h & 0xFFE0u) << 17 | (h & 31u); };
          best[0] = key32(b01 & 0xFFFFu);
          best[1] = key32((b01 >> 16) - 4096u);
          best[2] = key32((b23 & 0xFFFFu) - 4096u);
          best[3] = key32((b23 >> 16) - 4096u);
        } else {
#pragma unroll 4
        for (uint32_t lv = 0; lv < L; ++lv) {
          // the window parts' low words: the counts sit in bits 0..9, so the
          // low 10 bits of the sum are the window's count
          uint32_t c = lds_u32(o.h0 + lv * O::kLS);
          if (NB == 2) c += lds_u32(o.h0 + lv * O::kLS + O::kHS);
          const uint32_t k0 = (c << 22) | (31u - lv);
          best[0] = max(best[0], k0);
          // byte k of p: 128 + the count of D_{4w+1} + .. + D_{4w+k+1} for DC
          // word w; the key of window 4w + k + 1 adds that prefix to the key
          // of window 4w
          uint32_t kw = k0;
#pragma unroll
          for (int w = 0; w < O::kDCWords; ++w) {
            const uint32_t p =
                lds_u32(o.dc0 + lv * O::kDLS + static_cast<uint32_t>(w) * O::kDW) * 0x01010101u +
                0x80808080u;
            const uint32_t kb = kw - (128u << 22);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int i = 4 * w + k + 1;
              if (i < K) {
                const uint32_t ki = kb + (((p >> (8 * k)) & 0xFFu) << 22);
                best[i] = max(best[i], ki);
                if (k == 3) kw = ki;
              }
            }
          }
        }
        }
        // the reciprocals first, so that their latency overlaps the loads
        // of the winning bins
        uint32_t mulv[K];
#pragma unroll
        for (int i = 0; i < K; ++i) mulv[i] = rcp_of(best[i] >> 22);
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const int x = xa + i;
          if (x < d.ox0 || x >= d.ox1) continue;
          const uint32_t m = kTag - (best[i] & kTag);
          if ((best[i] >> 22) == 0u) continue;  // no level below L (literal mode only)
          uint64_t v = 0;
#pragma unroll
          for (int j = 0; j < NB + i; ++j) {  // the window parts, D_1 .. D_i
            uint32_t lo, hi;
            lds_v2(o.h0 + m * O::kLS + static_cast<uint32_t>(j) * O::kHS, lo, hi);
            v += static_cast<uint64_t>(hi) << 32 | lo;
          }
          const uint32_t lo = static_cast<uint32_t>(v);
          const uint32_t hi = static_cast<uint32_t>(v >> 32);
          const uint32_t Rs = (lo >> 10) & 0x3FFFFu;
          const uint32_t Gs = (lo >> 28) | ((hi & 0x3FFFu) << 4);
          const uint32_t Bs = hi >> 14;
          const uint32_t mul = mulv[i];
          store_pixel(d, x, y, __umulhi(Rs << 1, mul), __umulhi(Gs << 1, mul),
                      __umulhi(Bs << 1, mul), alpha[i]);
        }
      });
}

// Shared-memory layout of the column path after the ring (all sizes in
// bytes, Lp = L | 1 levels per histogram so that a column's histogram is an
// odd number of 8-byte bins long and 32 lanes updating 32 neighbouring
// columns spread over the banks):
//   colhist  [ncols][Lp] 8-byte bins  (ncols = T + 2r image columns)
//   winners  [NW][32]    8-byte bins  (each warp's last 32 winning bins)
// and for variant B the column histograms' counts (4 bytes, same layout at
// half the stride).
__host__ __device__ constexpr uint32_t cols_levels(uint32_t L) { return L | 1u; }
__host__ __device__ constexpr uint32_t cols_sums_bytes(uint32_t ncols, uint32_t nw, uint32_t L) {
  return (ncols * cols_levels(L) + nw * 32u) * 8u;
}

// Column histograms with the levels across a warp's lanes (r <= 44, L <= 32;
// VAR A bins and word format 1 for r <= 15, VAR B and format 2 above).  A CTA
// of NW warps owns the tile [x0, x0 + T) x [y0, y1), T = NW * 32 * TWK, and
// keeps one histogram per image column x0 - r .. x0 + T + r - 1 over the
// window's 2r + 1 rows.  Per row step:
//   A. all threads slide the column histograms down one row (+ the entering
//      pixel, - the leaving one: 2 bin updates per column);
//   B. warp w sums the 2r + 1 column histograms of its first window, then
//      sweeps its 32 * TWK output columns of the row: lane l holds level l of
//      the current window in registers; an output is one max-reduction over
//      the lanes of (count, 31 - l) keys (the lowest level wins ties), after
//      which the winning lane stores its bin in slot k of 32, and moving one
//      column right adds the entering column's histogram and subtracts the
//      leaving one (one 64-bit add and subtract per lane).  After 32 outputs
//      lane k reads slot k and all lanes compute their means and store
//      together.
// The sweep's work per output pixel does not depend on r.  Pixels outside the image
// are TMA zero fill, whose delta is zero.
template <int NW, int TWK, int VAR>
__device__ bool run_tile_cols(const ImgDesc &d, const CUtensorMap *tmap, int x0, int y0, int y1,
                              const RingCfg &rc, const SmemMap &sm, uint32_t &chunk_ctr,
                              uint32_t *err, uint64_t timeout_ns, uint32_t *diag = nullptr,
                              bool tmap_global = false) {
  constexpr int NT = 32 * NW;
  constexpr int TW = 32 * TWK;  // output columns per warp
  constexpr int T = NW * TW;
  constexpr uint32_t FULL = 0xFFFFFFFFu;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int r = d.r;
  const uint32_t L = d.L;
  const uint32_t Lp = cols_levels(L);
  const uint32_t S = Lp * 8u;  // bytes between two columns' histograms
  const int ncols = T + 2 * r;
  const int xs = x0 - r;  // a multiple of 4 by the choice of d.xshift
  const int E0 = y0 - r;
  const int nsteps = (y1 - y0) + 2 * r;
  const uint32_t colb = sm.sums;
  const uint32_t winb = colb + static_cast<uint32_t>(ncols) * S;  // 32 winner slots per warp
  const uint32_t sums_end = winb + NW * 32u * 8u;
  // VAR B counts: the same layout at half the stride
  const uint32_t cbase = (sums_end + 127u) & ~127u;
  const uint32_t cd = cbase - (colb >> 1);
  const uint8_t *gbase = sm.ring_ptr - sm.ring;  // generic address of shared address 0
  using Ops = typename std::conditional<VAR == kVarA, DeltaOpsA<8u>, DeltaOpsB<8u>>::type;
  Ops ops;
  if constexpr (VAR == kVarB) ops.cd = cd;
  // zero the column histograms (all Lp levels)
  {
    const uint32_t words = static_cast<uint32_t>(ncols) * Lp * 2u;
    for (uint32_t i = t; i < words; i += NT) sts_zero32(colb + i * 4u);
    if (VAR == kVarB)
      for (uint32_t i = t; i < words / 2u; i += NT) sts_zero32(cbase + i * 4u);
  }
  const bool lv_ok = static_cast<uint32_t>(lane) < L;
  const uint32_t tag = 31u - static_cast<uint32_t>(lane);
  const uint32_t mywin = winb + static_cast<uint32_t>(warp) * 32u * 8u;

  return ring_pass(
      d, tmap, xs, E0, nsteps, rc, sm, chunk_ctr, err, timeout_ns, diag, tmap_global, x0, y0,
      y1, [&](int s, const uint32_t *rowe, const uint32_t *rowl) {
        const bool rm = s >= 2 * r + 1;  // the leaving row was added by this tile
        // A. column histograms, then this warp's start window
        for (int j = t; j < ncols; j += NT) {
          const uint32_t base = colb + static_cast<uint32_t>(j) * S;
          if (rm)
            ops.addsub(base, rowe[j], rowl[j]);
          else
            ops.add(base, rowe[j]);
        }
        __syncthreads();
        if (s >= 2 * r) {
          // B. sweep this warp's outputs of row y
          const int y = E0 + s - r;
          const int xw = x0 + warp * TW;
          const uint8_t *cp = gbase + colb + static_cast<uint32_t>(lane) * 8u;
          const uint8_t *cc = gbase + (colb >> 1) + cd + static_cast<uint32_t>(lane) * 4u;
          // the window of column xw: the sum of its 2r + 1 column histograms
          uint64_t acc = 0;
          uint32_t cnt = 0;
          if (lv_ok) {
            for (int j = warp * TW; j <= warp * TW + 2 * r; ++j) {
              acc += *reinterpret_cast<const uint64_t *>(cp + static_cast<uint32_t>(j) * S);
              if (VAR == kVarB)
                cnt += *reinterpret_cast<const uint32_t *>(cc + static_cast<uint32_t>(j) * (S / 2u));
            }
          }
          // the winning lane leaves its bin for output k in slot k
          uint64_t *wslot = reinterpret_cast<uint64_t *>(const_cast<uint8_t *>(gbase + mywin));
          uint32_t Wk = 0;
#pragma unroll
          for (int bt = 0; bt < TWK; ++bt) {
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
              const uint32_t lo = static_cast<uint32_t>(acc);
              uint32_t key = 0u;
              if (lv_ok) key = (VAR == kVarA ? (lo << 22) : (cnt << 5)) | tag;
              const uint32_t kmax = __reduce_max_sync(FULL, key);
              const int m = static_cast<int>(31u - (kmax & 31u));
              if (lane == m) wslot[k] = acc;
              if (lane == k) Wk = kmax;
              // move one column right: + column x + r + 1, - column x - r
              const int kk = bt * 32 + k;
              if (kk + 1 < TW && lv_ok) {
                const uint32_t jin = static_cast<uint32_t>(warp * TW + kk + 2 * r + 1);
                const uint32_t jout = static_cast<uint32_t>(warp * TW + kk);
                acc += *reinterpret_cast<const uint64_t *>(cp + jin * S);
                acc -= *reinterpret_cast<const uint64_t *>(cp + jout * S);
                if (VAR == kVarB) {
                  cnt += *reinterpret_cast<const uint32_t *>(cc + jin * (S / 2u));
                  cnt -= *reinterpret_cast<const uint32_t *>(cc + jout * (S / 2u));
                }
              }
            }
            // lane k of this batch owns output xw + 32 bt + k
            __syncwarp();
            const uint64_t wv = wslot[lane];
            __syncwarp();  // slots are rewritten by the next batch
            const uint32_t Wlo = static_cast<uint32_t>(wv), Whi = static_cast<uint32_t>(wv >> 32);
            const int x = xw + bt * 32 + lane;
            const uint32_t c = VAR == kVarA ? (Wk >> 22) : (Wk >> 5);  // the winner's count
            if (x >= d.ox0 && x < d.ox1 && c != 0u) {
              const uint32_t alpha = d.bpp == 4 ? load_alpha(d, x, y) : 0u;
              if (VAR == kVarA) {
                const uint32_t R = (Wlo >> 10) & 0x3FFFFu;
                const uint32_t G = (Wlo >> 28) | ((Whi & 0x3FFFu) << 4);
                const uint32_t B = Whi >> 14;
                const uint32_t mul = rcp_of(c);
                store_pixel(d, x, y, __umulhi(R << 1, mul), __umulhi(G << 1, mul),
                            __umulhi(B << 1, mul), alpha);
              } else {
                const uint32_t R = Wlo & 0x1FFFFFu;
                const uint32_t G = (Wlo >> 21) | ((Whi & 0x3FFu) << 11);
                const uint32_t B = (Whi >> 10) & 0x1FFFFFu;
                store_pixel(d, x, y, R / c, G / c, B / c, alpha);
              }
            }
          }
        }
        __syncthreads();  // the next step's A rewrites what B read
      });
}

// Barrier init; ends with a CTA barrier.
__device__ __forceinline__ void init_cta(const SmemMap &sm, const RingCfg &rc) {
  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < rc.nslot; ++s) mbar_init(sm.bars + s * 8u, 1u);
    mbar_fence_init();
  }
  __syncthreads();
}

}  // namespace opk
