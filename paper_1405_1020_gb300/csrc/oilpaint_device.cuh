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
//        level << 24 | R << 16 | G << 8 | B
//      so the level (section 4's quantisation) is computed once per pixel,
//      not once per window visit;
//   2. halo staging: chunks of `ch` packed rows, (TW + 2r) columns rounded to
//      16 bytes, are copied by TMA (cp.async.bulk.tensor.2d) into a ring of
//      shared-memory slots; an mbarrier per slot signals arrival;
//   3. thread t owns output column x0 + t and a private histogram in shared
//      memory laid out [level][thread] (so the 32 lanes of a warp always hit
//      32 different banks whatever their levels); it slides down the tile;
//   4. argmax over the L bins with a strict > scan from level 0;
//   5. the three channel means and the byte stores.
//
// Bins (selected per image by the radius):
//   variant A (r <= 15, window <= 961 pixels): one 64-bit word per bin,
//       count:10 @54 | sumR:18 @36 | sumG:18 @18 | sumB:18 @0.
//       No field can overflow into the next (961*255 < 2^18, 961 < 2^10), so
//       one 64-bit add or subtract updates all four quantities.
//   variant B (r <= 44, window <= 7921 pixels): a 64-bit word
//       sumR:21 @42 | sumG:21 @21 | sumB:21 @0 (7921*255 < 2^21) plus a
//       separate 32-bit count.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace opk {

constexpr int kVarA = 0;
constexpr int kVarB = 1;
constexpr int kMaxRadiusA = 15;
constexpr int kMaxRadiusB = 44;

// bits of the device error word
constexpr uint32_t kErrTimeout = 1u;

// One image, as the kernels see it.
struct __align__(16) ImgDesc {
  const uint8_t *in;        // device, h*stride bytes
  uint8_t *out;             // device, h*stride bytes
  uint32_t *packed;         // device, h*ppitch words (pack prepass output)
  const CUtensorMap *tmap;  // device copy of the packed image's tensor map (batch path)
  uint32_t w, h, stride, bpp;
  int32_t r;
  uint32_t L, mode, ppitch;  // mode: 0 = paper level, 1 = divide by 3 first
  uint32_t tile_h, tiles_x, boxw, variant;
};

// Geometry of the shared-memory halo ring, fixed per launch.
struct RingCfg {
  uint32_t ch;          // rows per chunk (TMA box height)
  uint32_t pf;          // chunks in flight ahead of the one being consumed
  uint32_t nslot;       // ring slots, >= pf + ceil((2r+1)/ch) + 1
  uint32_t slot_bytes;  // bytes per slot, multiple of 128
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

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

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ void lds_v2(uint32_t addr, uint32_t &lo, uint32_t &hi) {
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(addr));
}

__device__ __forceinline__ void sts_zero64(uint32_t addr) {
  asm volatile("st.shared.v2.u32 [%0], {%1, %1};" ::"r"(addr), "r"(0u));
}

__device__ __forceinline__ void sts_zero32(uint32_t addr) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(0u));
}

// 64-bit read-modify-write of one histogram bin.  All histogram accesses are
// volatile asm, so they keep their program order among themselves; the ring
// reads are ordinary loads and may be scheduled around them.
__device__ __forceinline__ void bin_add64(uint32_t addr, uint32_t dlo, uint32_t dhi) {
  asm volatile(
      "{\n\t.reg .u32 a, b;\n\t"
      "ld.shared.v2.u32 {a, b}, [%0];\n\t"
      "add.cc.u32 a, a, %1;\n\t"
      "addc.u32 b, b, %2;\n\t"
      "st.shared.v2.u32 [%0], {a, b};\n\t}" ::"r"(addr),
      "r"(dlo), "r"(dhi));
}

__device__ __forceinline__ void bin_sub64(uint32_t addr, uint32_t dlo, uint32_t dhi) {
  asm volatile(
      "{\n\t.reg .u32 a, b;\n\t"
      "ld.shared.v2.u32 {a, b}, [%0];\n\t"
      "sub.cc.u32 a, a, %1;\n\t"
      "subc.u32 b, b, %2;\n\t"
      "st.shared.v2.u32 [%0], {a, b};\n\t}" ::"r"(addr),
      "r"(dlo), "r"(dhi));
}

__device__ __forceinline__ void cnt_add(uint32_t addr, uint32_t d) {
  asm volatile(
      "{\n\t.reg .u32 a;\n\t"
      "ld.shared.u32 a, [%0];\n\t"
      "add.u32 a, a, %1;\n\t"
      "st.shared.u32 [%0], a;\n\t}" ::"r"(addr),
      "r"(d));
}

// ------------------------------------------------------------ pack prepass

// Section 4's intensity level of one pixel, clamped to L-1.
__device__ __forceinline__ uint32_t level_of(uint32_t R, uint32_t G, uint32_t B, uint32_t L,
                                             uint32_t mode) {
  const uint32_t s = R + G + B;
  const uint32_t l = mode ? ((s / 3u) * L) / 255u : (s * L) / 765u;
  return l < L ? l : L - 1u;
}

__device__ __forceinline__ uint32_t pack_word(uint32_t R, uint32_t G, uint32_t B, uint32_t L,
                                              uint32_t mode) {
  return (level_of(R, G, B, L, mode) << 24) | (R << 16) | (G << 8) | B;
}

// Packs row y of image d with threads tid, tid+nthr, ...
__device__ __forceinline__ void pack_row(const ImgDesc &d, uint32_t y, uint32_t tid,
                                         uint32_t nthr) {
  const uint8_t *src = d.in + static_cast<size_t>(y) * d.stride;
  uint32_t *dst = d.packed + static_cast<size_t>(y) * d.ppitch;
  const uint32_t L = d.L, mode = d.mode, w = d.w;
  if (d.bpp == 4 && (reinterpret_cast<uintptr_t>(src) & 3u) == 0) {
    const uint32_t *s4 = reinterpret_cast<const uint32_t *>(src);
    for (uint32_t x = tid; x < w; x += nthr) {
      const uint32_t p = __ldg(s4 + x);
      dst[x] = pack_word(p & 0xFFu, (p >> 8) & 0xFFu, (p >> 16) & 0xFFu, L, mode);
    }
  } else {
    const uint32_t bpp = d.bpp;
    for (uint32_t x = tid; x < w; x += nthr) {
      const uint8_t *p = src + x * bpp;
      dst[x] = pack_word(__ldg(p), __ldg(p + 1), __ldg(p + 2), L, mode);
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

template <int TW, int VAR>
struct Hist {
  // byte distance between consecutive levels of one thread's histogram
  static constexpr uint32_t kLevelStride64 = TW * 8u;
  static constexpr uint32_t kLevelStride32 = TW * 4u;
  uint32_t sums;  // smem address of this thread's level-0 64-bit bin
  uint32_t cnts;  // smem address of this thread's level-0 count (variant B)

  __device__ __forceinline__ void clear(uint32_t L) const {
    for (uint32_t l = 0; l < L; ++l) {
      sts_zero64(sums + l * kLevelStride64);
      if (VAR == kVarB) sts_zero32(cnts + l * kLevelStride32);
    }
  }
  __device__ __forceinline__ void add(uint32_t w) const {
    const uint32_t lvl = w >> 24;
    uint32_t lo, hi;
    if (VAR == kVarA) {
      delta_a(w, lo, hi);
      bin_add64(sums + lvl * kLevelStride64, lo, hi);
    } else {
      delta_b(w, lo, hi);
      bin_add64(sums + lvl * kLevelStride64, lo, hi);
      cnt_add(cnts + lvl * kLevelStride32, 1u);
    }
  }
  __device__ __forceinline__ void sub(uint32_t w) const {
    const uint32_t lvl = w >> 24;
    uint32_t lo, hi;
    if (VAR == kVarA) {
      delta_a(w, lo, hi);
      bin_sub64(sums + lvl * kLevelStride64, lo, hi);
    } else {
      delta_b(w, lo, hi);
      bin_sub64(sums + lvl * kLevelStride64, lo, hi);
      cnt_add(cnts + lvl * kLevelStride32, 0xFFFFFFFFu);
    }
  }
  // Most populated level (lowest on a tie) and its truncated channel means.
  __device__ __forceinline__ void mode_colour(uint32_t L, uint32_t &oR, uint32_t &oG,
                                              uint32_t &oB) const {
    uint32_t m = 0, cnt, R, G, B, lo, hi;
    if (VAR == kVarA) {
      uint32_t best = 0;  // count field of the best bin, kept in place (bits 22..31)
      for (uint32_t l = 0; l < L; ++l) {
        const uint32_t k = lds_u32(sums + l * kLevelStride64 + 4u) & 0xFFC00000u;
        if (k > best) {
          best = k;
          m = l;
        }
      }
      lds_v2(sums + m * kLevelStride64, lo, hi);
      cnt = hi >> 22;
      R = (hi >> 4) & 0x3FFFFu;
      G = ((hi & 0xFu) << 14) | (lo >> 18);
      B = lo & 0x3FFFFu;
    } else {
      uint32_t best = 0;
      for (uint32_t l = 0; l < L; ++l) {
        const uint32_t c = lds_u32(cnts + l * kLevelStride32);
        if (c > best) {
          best = c;
          m = l;
        }
      }
      cnt = best;
      lds_v2(sums + m * kLevelStride64, lo, hi);
      R = hi >> 10;
      G = (lo >> 21) | ((hi & 0x3FFu) << 11);
      B = lo & 0x1FFFFFu;
    }
    oR = R / cnt;
    oG = G / cnt;
    oB = B / cnt;
  }
};

// ----------------------------------------------------------------- tiles

// Shared-memory carve-up common to both kernels.  `smem` is the dynamic
// shared memory base; returns the 128-byte aligned addresses.
struct SmemMap {
  uint32_t bars;  // nslot mbarriers
  uint32_t ring;  // nslot * slot_bytes
  uint32_t sums;  // L * TW * 8
  uint32_t cnts;  // L * TW * 4 (variant B)
  uint8_t *ring_ptr;
};

__device__ __forceinline__ SmemMap carve_smem(uint8_t *smem, const RingCfg &rc, uint32_t tw,
                                              uint32_t lmax) {
  SmemMap s;
  const uint32_t base = smem_addr(smem);
  const uint32_t a = (base + 127u) & ~127u;
  s.bars = a;
  s.ring = a + ((rc.nslot * 8u + 127u) & ~127u);
  s.sums = s.ring + rc.nslot * rc.slot_bytes;
  s.cnts = s.sums + lmax * tw * 8u;
  s.ring_ptr = smem + (s.ring - base);
  return s;
}

// Output tile [x0, x0+TW) x [y0, y1) of image d.  Chunk k of the tile holds
// the entering rows [y0 - r + k*ch, y0 - r + (k+1)*ch); it lives in ring
// slot (chunk_ctr + k) % nslot, whose mbarrier completes its phase
// ((chunk_ctr + k) / nslot) & 1.  chunk_ctr counts the chunks this CTA has
// consumed so far and is advanced by the tile.  Returns false if a halo copy
// did not arrive within timeout_ns (error recorded in *err).
template <int TW, int VAR>
__device__ bool run_tile(const ImgDesc &d, const CUtensorMap *tmap, int x0, int y0, int y1,
                         const RingCfg &rc, const SmemMap &sm, uint32_t &chunk_ctr,
                         uint32_t *err, uint64_t timeout_ns) {
  const int t = threadIdx.x;
  const int r = d.r;
  const int W = static_cast<int>(d.w), H = static_cast<int>(d.h);
  const int x = x0 + t;
  const int xs = (x0 - r) & ~3;  // box start, rounded down to 16 bytes
  const int clo = max(x - r, 0), chi = min(x + r, W - 1);
  const int nseg = x < W ? chi - clo + 1 : 0;
  const int jlo = clo - xs;
  const int E0 = y0 - r;  // first entering row
  const int nsteps = (y1 - y0) + 2 * r;
  const int ch = static_cast<int>(rc.ch);
  const int nchunks = (nsteps + ch - 1) / ch;
  const uint32_t box_bytes = d.boxw * rc.ch * 4u;

  Hist<TW, VAR> hist;
  hist.sums = sm.sums + static_cast<uint32_t>(t) * 8u;
  hist.cnts = sm.cnts + static_cast<uint32_t>(t) * 4u;
  hist.clear(d.L);

  auto issue = [&](int k) {
    const uint32_t g = chunk_ctr + static_cast<uint32_t>(k);
    const uint32_t slot = g % rc.nslot;
    const uint32_t bar = sm.bars + slot * 8u;
    mbar_arrive_expect_tx(bar, box_bytes);
    tma_load_2d(sm.ring + slot * rc.slot_bytes, tmap, xs, E0 + k * ch, bar);
  };

  __syncthreads();  // the previous tile no longer reads the ring
  int issued = 0;
  if (t == 0) {
    fence_proxy_async_smem();
    for (; issued < static_cast<int>(rc.pf) && issued < nchunks; ++issued) issue(issued);
  }
  issued = min(static_cast<int>(rc.pf), nchunks);

  const uint32_t *ring = reinterpret_cast<const uint32_t *>(sm.ring_ptr);
  const uint32_t slot_words = rc.slot_bytes / 4u;
  auto row_ptr = [&](int e) -> const uint32_t * {
    const int rel = e - E0;
    const uint32_t slot = (chunk_ctr + static_cast<uint32_t>(rel / ch)) % rc.nslot;
    return ring + slot * slot_words + static_cast<uint32_t>(rel % ch) * d.boxw + jlo;
  };

  for (int k = 0; k < nchunks; ++k) {
    const uint32_t g = chunk_ctr + static_cast<uint32_t>(k);
    const bool ok = mbar_wait_bounded(sm.bars + (g % rc.nslot) * 8u, (g / rc.nslot) & 1u,
                                      timeout_ns);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        atomicOr(err, kErrTimeout);
        // wait, again bounded, for the copies still in flight
        for (int j = k; j < issued; ++j) {
          const uint32_t gj = chunk_ctr + static_cast<uint32_t>(j);
          mbar_wait_bounded(sm.bars + (gj % rc.nslot) * 8u, (gj / rc.nslot) & 1u, timeout_ns);
        }
      }
      __syncthreads();
      return false;
    }
    if (k + static_cast<int>(rc.pf) < nchunks) {
      if (t == 0) {
        fence_proxy_async_smem();
        issue(k + static_cast<int>(rc.pf));
      }
      ++issued;
    }
    const int s_end = min((k + 1) * ch, nsteps);
    for (int s = k * ch; s < s_end; ++s) {
      const int e = E0 + s;         // entering row
      const int l = e - 2 * r - 1;  // leaving row
      const bool do_add = e >= 0 && e < H;
      const bool do_rm = l >= 0 && l >= E0 && l < H;
      if (do_add && do_rm) {
        const uint32_t *pe = row_ptr(e);
        const uint32_t *pl = row_ptr(l);
        int j = 0;
        for (; j + 4 <= nseg; j += 4) {
          const uint32_t a0 = pe[j], a1 = pe[j + 1], a2 = pe[j + 2], a3 = pe[j + 3];
          const uint32_t b0 = pl[j], b1 = pl[j + 1], b2 = pl[j + 2], b3 = pl[j + 3];
          hist.sub(b0);
          hist.add(a0);
          hist.sub(b1);
          hist.add(a1);
          hist.sub(b2);
          hist.add(a2);
          hist.sub(b3);
          hist.add(a3);
        }
        for (; j < nseg; ++j) {
          const uint32_t a = pe[j], b = pl[j];
          hist.sub(b);
          hist.add(a);
        }
      } else if (do_add) {
        const uint32_t *pe = row_ptr(e);
        for (int j = 0; j < nseg; ++j) hist.add(pe[j]);
      } else if (do_rm) {
        const uint32_t *pl = row_ptr(l);
        for (int j = 0; j < nseg; ++j) hist.sub(pl[j]);
      }
      if (s >= 2 * r && x < W) {
        const int y = e - r;
        uint32_t R, G, B;
        hist.mode_colour(d.L, R, G, B);
        uint8_t *o = d.out + static_cast<size_t>(y) * d.stride + static_cast<size_t>(x) * d.bpp;
        if (d.bpp == 4) {
          const uint32_t a =
              __ldg(d.in + static_cast<size_t>(y) * d.stride + static_cast<size_t>(x) * 4u + 3u);
          const uint32_t v = R | (G << 8) | (B << 16) | (a << 24);
          if ((reinterpret_cast<uintptr_t>(o) & 3u) == 0) {
            *reinterpret_cast<uint32_t *>(o) = v;
          } else {
            o[0] = static_cast<uint8_t>(R);
            o[1] = static_cast<uint8_t>(G);
            o[2] = static_cast<uint8_t>(B);
            o[3] = static_cast<uint8_t>(a);
          }
        } else {
          o[0] = static_cast<uint8_t>(R);
          o[1] = static_cast<uint8_t>(G);
          o[2] = static_cast<uint8_t>(B);
        }
      }
    }
  }
  chunk_ctr += static_cast<uint32_t>(nchunks);
  return true;
}

__device__ __forceinline__ void init_ring_barriers(const SmemMap &sm, const RingCfg &rc) {
  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < rc.nslot; ++s) mbar_init(sm.bars + s * 8u, 1u);
    mbar_fence_init();
  }
  __syncthreads();
}

}  // namespace opk
