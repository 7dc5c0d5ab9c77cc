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

// Dynamic shared memory of a filter CTA of nt threads with cpt output columns
// per thread (plus 128 bytes of alignment slack).
inline size_t tile_smem_bytes(uint32_t nt, int cpt, uint32_t lmax, int variant_max,
                              const RingCfg &rc) {
  const size_t nhist = cpt == 1 ? 1u : 3u;
  // L levels plus one scratch level per histogram
  return 128u + ((rc.nslot * 8u + 127u) & ~127u) + static_cast<size_t>(rc.nslot) * rc.slot_bytes +
         kRcpBytes + nhist * (lmax + 1u) * nt * bin_bytes(variant_max);
}

// Launchers; each returns cudaSuccess or the launch error.
cudaError_t launch_pack_single(const ImgDesc &d, int grid, cudaStream_t s);
// nt threads per CTA (32, 64, 96, 128), cpt output columns per thread (1, 2)
cudaError_t launch_tile_plain(uint32_t nt, int cpt, int variant, const ImgDesc &d,
                              const CUtensorMap &map, const RingCfg &rc, dim3 grid, size_t smem,
                              uint32_t *err, uint64_t timeout_ns, cudaStream_t s);
// d_n: device pointer to the number of images (the batch tables are device-resident).
cudaError_t launch_pack_batch(const ImgDesc *d_descs, const uint32_t *d_row_prefix,
                              const uint32_t *d_n, uint32_t *d_queue, int grid, cudaStream_t s);
cudaError_t launch_persistent(uint32_t nt, int cpt, const ImgDesc *d_descs,
                              const uint32_t *d_tile_prefix, const uint32_t *d_n,
                              uint32_t *d_queue, const RingCfg &rc, uint32_t lmax, int grid,
                              size_t smem, uint32_t *err, uint64_t timeout_ns, cudaStream_t s);
cudaError_t launch_selftest_wait(uint32_t *d_err, uint64_t timeout_ns, cudaStream_t s);

// Raise the dynamic shared-memory limit of every filter kernel instance to
// `bytes`; returns the error of the first failing call.
cudaError_t set_tile_smem_limit(size_t bytes);
// Resident CTAs per SM of the plain (variant) or persistent (variant < 0) kernel.
int tile_occupancy(uint32_t nt, int cpt, int variant, size_t smem);

}  // namespace opk
