// oilpaint_internal.h -- launchers shared by the C-ABI layer and the kernel TU.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "oilpaint_device.cuh"

namespace opk {

// Histogram variant for a radius (A up to 15, B up to 44), -1 if unsupported.
inline int variant_for_radius(int r) {
  if (r < 0) return -1;
  if (r <= kMaxRadiusA) return kVarA;
  if (r <= kMaxRadiusB) return kVarB;
  return -1;
}

// Bytes per histogram bin per thread for a variant.
inline uint32_t bin_bytes(int variant) { return variant == kVarA ? 8u : 12u; }

// Ring geometry: pf + 1 slots, each holding the ch entering rows and the ch
// leaving rows of one chunk (two halves, each 128-byte aligned).
inline RingCfg make_ring(int r, uint32_t ch, uint32_t pf, uint32_t boxw) {
  (void)r;
  RingCfg rc;
  rc.ch = ch;
  rc.pf = pf;
  rc.nslot = pf + 1u;
  rc.half_bytes = (boxw * ch * 4u + 127u) & ~127u;
  rc.slot_bytes = 2u * rc.half_bytes;
  return rc;
}

// Box width (words) of the halo copy of a TW-wide tile at radius r: covers
// columns [x0 - r, x0 + TW + r) from the 16-byte boundary at or below x0 - r.
// x0 is a multiple of TW (hence of 4), so the offset is (-r) mod 4.
inline uint32_t box_width(uint32_t tw, int r) {
  const uint32_t off = static_cast<uint32_t>((-r) & 3);
  return (off + tw + 2u * static_cast<uint32_t>(r) + 3u) & ~3u;
}

inline bool delta_eligible(int r, uint32_t L) {
  return r >= 0 && r <= kDeltaMaxRadius && L >= 1 && L <= kDeltaMaxLevels;
}

// The straight-line difference-histogram path (paths 2 and 3; K = 2, 4 or
// 8 columns per thread, one kernel per radius): variant-A bins, L <= 32 (64
// for K = 2, window histogram in one part only), and r >= K/2 so that the
// left difference words 0 .. K-2 lie inside the window and apart from the
// right ones.
inline bool deltak_eligible(int k, int r, uint32_t L) {
  return (k == 2 || k == 4 || k == 8) && r >= deltak_min_radius(k) && r <= kDeltaKMaxRadius &&
         L >= 1 && L <= (k == 2 ? kDeltaK2MaxLevels : kDeltaMaxLevels);
}

// Box width (words) of a difference-histogram tile: thread t reads K-word
// groups from ring index K*t up to the group holding word 2r+K-1.
inline uint32_t delta_box_width(uint32_t nt, int k, int r) {
  const uint32_t ng = (2u * static_cast<uint32_t>(r) + static_cast<uint32_t>(k) - 1u) /
                          static_cast<uint32_t>(k) + 1u;
  const uint32_t w = static_cast<uint32_t>(k) * (nt - 1u + ng);
  return (w + 3u) & ~3u;
}

// Launch geometry of one image: path (0 histograms per thread, 1 column
// histograms, 4 the direct path of radius 0 to 2, 2 and 3 the straight-line
// difference histograms with the
// window histogram in one or two parts), threads per CTA, columns per thread
// (path 0: 2 or 4 only where the difference-histogram path applies; path 1:
// outputs per warp / 32; paths 2 and 3: 4 or 8), tile width, the x of the
// first tile, tiles per row, the halo box width, the histogram variant and
// the packed word format.
struct Geometry {
  int path;
  int r;
  uint32_t nt;
  int kcols;
  uint32_t tile_w;
  int32_t xshift;
  uint32_t tiles_x;
  uint32_t boxw;
  int variant;
  uint32_t fmt;
};

inline Geometry image_geometry(int path, uint32_t nt, int kcols_wanted, int r, uint32_t L,
                               uint32_t w) {
  Geometry g;
  g.nt = nt;
  g.r = r;
  g.variant = variant_for_radius(r);
  // the direct path: radius 0, 1 or 2, any L, one column per thread
  if (path == static_cast<int>(kPathDirect)) {
    if (r >= 0 && r <= kDirectMaxRadius && kcols_wanted == 1) {
      g.path = path;
      g.kcols = 1;
      g.tile_w = nt;
      g.xshift = 0;
      g.boxw = box_width(nt, r);
      g.fmt = 0u;
      g.variant = kVarA;
      g.tiles_x = (w + nt - 1u) / nt;
      return g;
    }
    path = 0;
  }
  // eight columns per thread exist only on the straight-line path (in two parts)
  if (path == 0 && kcols_wanted == 8) path = 3;
  if (path == 2 || path == 3) {
    g.path = deltak_eligible(kcols_wanted, r, L) ? path : 0;
    if (g.path) {
      g.kcols = kcols_wanted;
      g.tile_w = nt * static_cast<uint32_t>(g.kcols);
      g.xshift = (r & 3) ? (r & 3) - 4 : 0;
      g.boxw = delta_box_width(nt, g.kcols, r);
      g.fmt = 1u;
      g.tiles_x = static_cast<uint32_t>((static_cast<int64_t>(w) - g.xshift + g.tile_w - 1) /
                                        g.tile_w);
      return g;
    }
    path = 0;
    if (kcols_wanted == 8) kcols_wanted = 1;
  }
  g.path = (path == 1 && delta_eligible(r, L)) ? 1 : 0;
  if (g.path == 1) {
    g.kcols = kcols_wanted == 2 ? 2 : 1;
    g.tile_w = nt * static_cast<uint32_t>(g.kcols);
    g.xshift = (r & 3) ? (r & 3) - 4 : 0;
    g.boxw = (g.tile_w + 2u * static_cast<uint32_t>(r) + 3u) & ~3u;
  } else {
    g.kcols = (kcols_wanted > 1 && kcols_wanted <= 4 && delta_eligible(r, L)) ? kcols_wanted : 1;
    g.tile_w = nt * static_cast<uint32_t>(g.kcols);
    if (g.kcols > 1) {
      // first tile at x0 = xshift with x0 - r a multiple of 4
      g.xshift = (r & 3) ? (r & 3) - 4 : 0;
      g.boxw = delta_box_width(nt, g.kcols, r);
    } else {
      g.xshift = 0;
      g.boxw = box_width(nt, r);
    }
  }
  g.fmt = (g.path == 1 || g.kcols > 1) ? (g.variant == kVarA ? 1u : 2u) : 0u;
  g.tiles_x = static_cast<uint32_t>((static_cast<int64_t>(w) - g.xshift + g.tile_w - 1) /
                                    g.tile_w);
  return g;
}

// Shared bytes of the column path's histograms (column sums, winner slots;
// variant B adds the counts after a 128-byte boundary).
inline size_t cols_hist_bytes(const Geometry &g, int r, uint32_t L) {
  const uint32_t ncols = g.tile_w + 2u * static_cast<uint32_t>(r);
  const size_t sums = cols_sums_bytes(ncols, g.nt / 32u, L);
  if (g.variant == kVarA) return sums;
  return ((sums + 127u) & ~static_cast<size_t>(127u)) + sums / 2u;
}

// Blocks of the single-image pack launch: one per image row (256 threads
// each).  Fewer blocks looping over several rows each (as many as fit one
// wave) measured slower: a block's rows are then packed one after another,
// each waiting for its own loads.
inline int pack_grid_for(uint32_t rows, int /*sms*/) {
  return static_cast<int>(rows ? rows : 1u);
}

// Histogram bytes of a CTA on the straight-line path: per level and thread
// nb + k - 1 histograms of 8-byte bins and (k - 1)/4 rounded up count words
// (k = 2: one count word per four levels).
inline size_t deltak_hist_bytes(uint32_t nt, int k, int nb, uint32_t L) {
  if (k == 2)  // two histograms, one count word per four levels
    return (static_cast<size_t>(16) * L + (L + 3u) / 4u * 4u) * nt;
  return static_cast<size_t>((nb + k - 1) * 8 + (k - 1 + 3) / 4 * 4) * L * nt;
}

// Histogram bytes of a CTA on path kcols (1: one histogram of L + 1 levels
// per thread, bins of the variant's size; 2 or 4: kcols histograms, one
// more where the window histogram is split, of L levels per thread, bins of
// 8 bytes (variant A) or 8 + 2 bytes (variant B)).
inline size_t hist_bytes(uint32_t nt, int kcols, uint32_t L, int variant) {
  // (column path: cols_hist_bytes; straight-line path: deltak_hist_bytes)
  if (kcols > 1) {
    const size_t nh = static_cast<size_t>(kcols) + static_cast<size_t>(hsplit(kcols, variant)) - 1u;
    // variant B: 8-byte sums and a 16-bit count per bin
    return nh * L * nt * (variant == kVarA ? 8u : 10u);
  }
  return static_cast<size_t>(L + 1u) * nt * bin_bytes(variant);
}

// Dynamic shared memory of a filter CTA given its histogram bytes (plus 128
// bytes of alignment slack).
inline size_t tile_smem_bytes(size_t hist, const RingCfg &rc) {
  return 128u + ((rc.nslot * 8u + 127u) & ~127u) + static_cast<size_t>(rc.nslot) * rc.slot_bytes +
         hist;
}

// Output window of an image: the whole image, or with the literal-mode bit
// (2) the pixels at least r from every edge -- empty when w <= 2r or h <= 2r.
struct Window {
  int32_t x0, x1, y0, y1;
  uint32_t rows() const { return y1 > y0 ? static_cast<uint32_t>(y1 - y0) : 0u; }
};

inline Window output_window(uint32_t w, uint32_t h, int r, uint32_t flags) {
  Window o{0, static_cast<int32_t>(w), 0, static_cast<int32_t>(h)};
  if (flags & kModeLiteral) {
    if (static_cast<int64_t>(w) > 2ll * r && static_cast<int64_t>(h) > 2ll * r)
      o = Window{r, static_cast<int32_t>(w) - r, r, static_cast<int32_t>(h) - r};
    else
      o = Window{0, 0, 0, 0};
  }
  return o;
}

inline void set_window(ImgDesc &d, const Window &o) {
  d.ox0 = o.x0;
  d.ox1 = o.x1;
  d.oy0 = o.y0;
  d.oy1 = o.y1;
}

// Tensor map of a packed image (defined with the C ABI): w x h 32-bit
// words, rows ppitch words apart, copied in {boxw, ch} boxes; elements out
// of range read as zero.  False if the driver's encoder is unavailable or
// refuses the map.
bool encode_packed_map(CUtensorMap *map, const uint32_t *packed, uint32_t w, uint32_t h,
                       uint32_t ppitch, uint32_t boxw, uint32_t ch);

// The same for any image of 32-bit words (the packed image, or for the fused
// pack the input pixels of a 4-byte-per-pixel image): w x h words, rows
// pitch_bytes apart.  False unless base and pitch are multiples of 16 bytes.
bool encode_word_map(CUtensorMap *map, const void *base, uint32_t w, uint32_t h,
                     uint64_t pitch_bytes, uint32_t boxw, uint32_t ch);

// Tile height for an image of H output rows cut into tiles_x tile columns
// when `slots` CTAs can be resident at once: minimises waves x steps per
// tile, where a tile of h output rows takes h + 2r steps (2r of them only
// fill the running histogram) and a wave is `slots` tiles side by side.
uint32_t auto_tile_h(uint32_t H, uint32_t tiles_x, int r, uint64_t slots);

// Launchers; each returns cudaSuccess or the launch error.
cudaError_t launch_pack_single(const ImgDesc &d, int grid, cudaStream_t s);
// nt threads per CTA (32, 64, 96, 128); kcols 1 (one column per thread,
// histogram variant `variant`) or 2 / 4 (difference histograms); with
// d.path == 1 the column-histogram kernel with nt / 32 warps sweeping
// 32 * kcols outputs each
cudaError_t launch_tile(uint32_t nt, int kcols, int variant, const ImgDesc &d,
                        const CUtensorMap &map, const RingCfg &rc, dim3 grid, size_t smem,
                        uint32_t *err, uint64_t timeout_ns, cudaStream_t s);
// d_n: device pointer to the number of images (the batch tables are
// device-resident); the launch also zeroes the nqueues ticket counters at
// d_queues for the filter launches that follow it.
cudaError_t launch_pack_batch(const ImgDesc *d_descs, const uint32_t *d_row_prefix,
                              const uint32_t *d_n, uint32_t *d_queues, uint32_t nqueues, int grid,
                              cudaStream_t s);
// d_grp: device pointer to one group's image count, with the index of its
// first descriptor kBatchGroups words and of its first tile-prefix entry
// 2 kBatchGroups words further on.
cudaError_t launch_persistent(uint32_t nt, int kcols, const ImgDesc *d_descs,
                              const uint32_t *d_tile_prefix, const uint32_t *d_grp,
                              uint32_t *d_queue, const RingCfg &rc, uint32_t lmax, int grid,
                              size_t smem, uint32_t *err, uint64_t timeout_ns, cudaStream_t s);
cudaError_t launch_selftest_wait(uint32_t *d_err, uint64_t timeout_ns, cudaStream_t s);
// The straight-line difference-histogram path (paths 2 and 3, d.kcols = 2,
// 4 or 8, nt = 32 or 64 threads, one kernel per radius in K's range, variant
// A, d.L within K's limit); cudaErrorInvalidValue otherwise.
cudaError_t launch_deltak(uint32_t nt, const ImgDesc &d, const CUtensorMap &map,
                          const RingCfg &rc, dim3 grid, size_t smem, uint32_t *err,
                          uint64_t timeout_ns, cudaStream_t s);
cudaError_t set_deltak_smem_limit(size_t bytes);
int deltak_occupancy(uint32_t nt, int k, int nb, size_t smem);
// One straight-line kernel (nullptr outside the tables): nt threads, nb
// window parts, radius r; defined in oilpaint_delta4.cu / oilpaint_delta8.cu.
using DeltaKFn = void (*)(const CUtensorMap, const ImgDesc, const RingCfg, uint32_t *, uint64_t);
DeltaKFn deltak_kernel_k2(uint32_t nt, int nb, int r);
DeltaKFn deltak_kernel_k4(uint32_t nt, int nb, int r);
DeltaKFn deltak_kernel_k8(uint32_t nt, int nb, int r);
// Checked builds: the bounds-check violation bits since the last call
// (1 shared memory, 2 image pixels, 4 TMA copy), cleared; 0 otherwise.
cudaError_t take_check_error(uint32_t *bits);

// Raise the dynamic shared-memory limit of every filter kernel instance to
// `bytes`; returns the error of the first failing call.
cudaError_t set_tile_smem_limit(size_t bytes);
// Resident CTAs per SM of the plain (kcols 1: variant), difference-histogram
// (kcols 2, 4) or persistent kernel.
int tile_occupancy(uint32_t nt, bool persistent, int kcols, int variant, size_t smem);
// ... of the column-histogram kernel: nt = 32 * warps, twk = outputs per warp / 32.
int tile_occupancy_cols(uint32_t nt, int twk, int variant, size_t smem);
// ... of the direct kernel (path 4) of nt threads at radius r.
int direct_occupancy(uint32_t nt, int r, size_t smem);

// Histogram bytes and resident CTAs of an image's single-image kernel.
inline size_t geometry_hist_bytes(const Geometry &g, int r, uint32_t L) {
  if (g.path == static_cast<int>(kPathDirect)) return 0;  // windows in registers
  if (g.path == 2 || g.path == 3) return deltak_hist_bytes(g.nt, g.kcols, g.path - 1, L);
  return g.path == 1 ? cols_hist_bytes(g, r, L) : hist_bytes(g.nt, g.kcols, L, g.variant);
}
inline int geometry_occupancy(const Geometry &g, size_t smem) {
  if (g.path == static_cast<int>(kPathDirect)) return direct_occupancy(g.nt, g.r, smem);
  if (g.path == 2 || g.path == 3) return deltak_occupancy(g.nt, g.kcols, g.path - 1, smem);
  return g.path == 1 ? tile_occupancy_cols(g.nt, g.kcols, g.variant, smem)
                     : tile_occupancy(g.nt, false, g.kcols, g.variant, smem);
}

}  // namespace opk
