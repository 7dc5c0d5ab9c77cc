// oilpaint_delta8.cu -- the eight-columns-per-thread filter kernel
// (run_tile_delta8 in oilpaint_device.cuh) and its launcher: one kernel per
// radius 4..15 and per CTA of 32 or 64 threads, so that the update steps
// are straight-line code.  Kept in a translation unit of its own so that it
// compiles in parallel with the other kernels.
#include "oilpaint_internal.h"

namespace opk {

template <int NT, int R>
__global__ void __launch_bounds__(NT, 1)
    tile_delta8_kernel(const __grid_constant__ CUtensorMap tmap, const ImgDesc d,
                       const RingCfg rc, uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  const SmemMap sm = carve_smem(smem, rc, 0u);
  init_cta(sm, rc);
  uint32_t ctr = 0;
  const int x0 = d.xshift + static_cast<int>(blockIdx.x) * NT * 8;
  const int y0 = d.oy0 + static_cast<int>(blockIdx.y * d.tile_h);
  const int y1 = min(y0 + static_cast<int>(d.tile_h), d.oy1);
  run_tile_delta8<NT, R>(d, &tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns);
}

namespace {

using KernelFn = void (*)(const CUtensorMap, const ImgDesc, const RingCfg, uint32_t *, uint64_t);

template <int NT, int... Rs>
struct Table {
  static constexpr KernelFn fns[sizeof...(Rs)] = {&tile_delta8_kernel<NT, Rs>...};
};

template <int NT>
KernelFn kernel_for(int r) {
  using T = Table<NT, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15>;
  static_assert(kDelta8MinRadius == 4 && kDelta8MaxRadius == 15, "one kernel per radius");
  if (r < kDelta8MinRadius || r > kDelta8MaxRadius) return nullptr;
  return T::fns[r - kDelta8MinRadius];
}

KernelFn kernel_for(uint32_t nt, int r) {
  if (nt == 32) return kernel_for<32>(r);
  if (nt == 64) return kernel_for<64>(r);
  return nullptr;
}

}  // namespace

cudaError_t launch_delta8(uint32_t nt, const ImgDesc &d, const CUtensorMap &map,
                          const RingCfg &rc, dim3 grid, size_t smem, uint32_t *err,
                          uint64_t timeout_ns, cudaStream_t s) {
  const KernelFn f = kernel_for(nt, d.r);
  if (!f || d.variant != static_cast<uint32_t>(kVarA) || d.L > kDeltaMaxLevels)
    return cudaErrorInvalidValue;
  f<<<grid, nt, smem, s>>>(map, d, rc, err, timeout_ns);
  return cudaGetLastError();
}

cudaError_t set_delta8_smem_limit(size_t bytes) {
  for (uint32_t nt : {32u, 64u})
    for (int r = kDelta8MinRadius; r <= kDelta8MaxRadius; ++r) {
      const cudaError_t e = cudaFuncSetAttribute(kernel_for(nt, r),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(bytes));
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

int delta8_occupancy(uint32_t nt, size_t smem) {
  const KernelFn f = kernel_for(nt, kDelta8MaxRadius);  // the same resources at every radius
  if (!f) return 0;
  int n = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, static_cast<int>(nt), smem) ==
                 cudaSuccess
             ? n
             : 0;
}

}  // namespace opk
