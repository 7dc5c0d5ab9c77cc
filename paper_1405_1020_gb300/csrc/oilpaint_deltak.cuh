// oilpaint_deltak.cuh -- kernels and launch tables of the straight-line
// difference-histogram path (run_tile_deltak in oilpaint_device.cuh): one
// kernel per radius, per CTA of 32 or 64 threads, per window split (NB = 1
// or 2 parts; 1 for K = 2), for K = 2, 4 or 8 output columns per thread.
// Each K is compiled in a translation unit of its own (oilpaint_delta2.cu,
// oilpaint_delta4.cu, oilpaint_delta8.cu) so that they compile in parallel.
#pragma once

#include <utility>

#include "oilpaint_internal.h"

namespace opk {

template <int NT, int K, int NB, int R>
__global__ void __launch_bounds__(NT, 1)
    tile_deltak_kernel(const __grid_constant__ CUtensorMap tmap, const ImgDesc d,
                       const RingCfg rc, uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  const SmemMap sm = carve_smem(smem, rc, 0u);
  init_cta(sm, rc);
  uint32_t ctr = 0;
  const int x0 = d.xshift + static_cast<int>(blockIdx.x) * NT * K;
  const int y0 = d.oy0 + static_cast<int>(blockIdx.y * d.tile_h);
  const int y1 = min(y0 + static_cast<int>(d.tile_h), d.oy1);
  run_tile_deltak<NT, K, NB, R>(d, &tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns);
}

// The kernel of radius r (K's radius range), or nullptr.
template <int NT, int K, int NB, int R0, int... Rs>
DeltaKFn deltak_kernel_for(int r, std::integer_sequence<int, Rs...>) {
  static constexpr DeltaKFn fns[sizeof...(Rs)] = {&tile_deltak_kernel<NT, K, NB, R0 + Rs>...};
  const int i = r - R0;
  return (i >= 0 && i < static_cast<int>(sizeof...(Rs))) ? fns[i] : nullptr;
}

template <int K>
DeltaKFn deltak_kernel(uint32_t nt, int nb, int r) {
  constexpr int R0 = deltak_min_radius(K);
  using Seq = std::make_integer_sequence<int, kDeltaKMaxRadius - R0 + 1>;
  if constexpr (K == 2) {  // the window histogram in one part only
    if (nb != 1) return nullptr;
    if (nt == 32) return deltak_kernel_for<32, K, 1, R0>(r, Seq{});
    if (nt == 64) return deltak_kernel_for<64, K, 1, R0>(r, Seq{});
  } else {
    if (nt == 32) return nb == 1 ? deltak_kernel_for<32, K, 1, R0>(r, Seq{})
                                 : deltak_kernel_for<32, K, 2, R0>(r, Seq{});
    if (nt == 64) return nb == 1 ? deltak_kernel_for<64, K, 1, R0>(r, Seq{})
                                 : deltak_kernel_for<64, K, 2, R0>(r, Seq{});
  }
  return nullptr;
}

}  // namespace opk
