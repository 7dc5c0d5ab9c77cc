// oilpaint_kernels.cu -- kernel entry points and their launchers.
//
//   pack_single_kernel / pack_batch_kernel  the pack prepass (one image / a
//                                           batch; the batch form also resets
//                                           the tile-queue counter)
//   tile_plain_kernel<TW, VAR>              one CTA per output tile
//   persistent_kernel<TW>                   grid-sized CTAs pulling
//                                           (image, tile) tickets from a
//                                           device atomic until the queue of a
//                                           whole batch is empty
//   selftest_wait_kernel                    exercises the bounded mbarrier wait
#include "oilpaint_internal.h"

namespace opk {

__global__ void __launch_bounds__(256) pack_single_kernel(const ImgDesc d) {
  for (uint32_t y = blockIdx.x; y < d.h; y += gridDim.x) pack_row(d, y, threadIdx.x, blockDim.x);
}

// Largest i in [0, n) with prefix[i] <= g (prefix strictly increasing, prefix[0] = 0).
__device__ __forceinline__ uint32_t find_image(const uint32_t *__restrict__ prefix, uint32_t n,
                                               uint32_t g) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1u) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256)
    pack_batch_kernel(const ImgDesc *__restrict__ descs, const uint32_t *__restrict__ row_prefix,
                      const uint32_t *__restrict__ d_n, uint32_t *queue) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *queue = 0u;
  const uint32_t n = __ldg(d_n);
  if (n == 0) return;
  const uint32_t total = __ldg(row_prefix + n);
  for (uint32_t g = blockIdx.x; g < total; g += gridDim.x) {
    const uint32_t i = find_image(row_prefix, n, g);
    const ImgDesc d = descs[i];
    pack_row(d, g - __ldg(row_prefix + i), threadIdx.x, blockDim.x);
  }
}

template <int TW, int VAR>
__global__ void __launch_bounds__(TW)
    tile_plain_kernel(const __grid_constant__ CUtensorMap tmap, const ImgDesc d, const RingCfg rc,
                      uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  const SmemMap sm = carve_smem(smem, rc, TW, d.L);
  init_ring_barriers(sm, rc);
  uint32_t ctr = 0;
  const int x0 = static_cast<int>(blockIdx.x) * TW;
  const int y0 = static_cast<int>(blockIdx.y * d.tile_h);
  const int y1 = min(y0 + static_cast<int>(d.tile_h), static_cast<int>(d.h));
  run_tile<TW, VAR>(d, &tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns);
}

template <int TW>
__global__ void __launch_bounds__(TW)
    persistent_kernel(const ImgDesc *__restrict__ descs, const uint32_t *__restrict__ tile_prefix,
                      const uint32_t *__restrict__ d_n, uint32_t *queue, const RingCfg rc,
                      uint32_t lmax, uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint32_t s_job[2];
  const SmemMap sm = carve_smem(smem, rc, TW, lmax);
  init_ring_barriers(sm, rc);
  const uint32_t n = __ldg(d_n);
  if (n == 0) return;
  const uint32_t total = __ldg(tile_prefix + n);
  uint32_t ctr = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t ticket = atomicAdd(queue, 1u);
      uint32_t img = 0xFFFFFFFFu, local = 0;
      if (ticket < total) {
        img = find_image(tile_prefix, n, ticket);
        local = ticket - __ldg(tile_prefix + img);
      }
      s_job[0] = img;
      s_job[1] = local;
    }
    __syncthreads();
    const uint32_t img = s_job[0], local = s_job[1];
    if (img == 0xFFFFFFFFu) break;
    const ImgDesc d = descs[img];
    const int x0 = static_cast<int>(local % d.tiles_x) * TW;
    const int y0 = static_cast<int>((local / d.tiles_x) * d.tile_h);
    const int y1 = min(y0 + static_cast<int>(d.tile_h), static_cast<int>(d.h));
    const bool ok = d.variant == kVarA
                        ? run_tile<TW, kVarA>(d, d.tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns)
                        : run_tile<TW, kVarB>(d, d.tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns);
    if (!ok) break;
  }
}

__global__ void selftest_wait_kernel(uint32_t *err, uint64_t timeout_ns) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_addr(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1u);
    mbar_fence_init();
  }
  __syncthreads();
  // Nothing arrives on this barrier, so its phase 0 never completes.
  const bool ok = mbar_wait_bounded(b, 0u, timeout_ns);
  if (!ok && threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_pack_single(const ImgDesc &d, int grid, cudaStream_t s) {
  pack_single_kernel<<<grid, 256, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_pack_batch(const ImgDesc *d_descs, const uint32_t *d_row_prefix,
                              const uint32_t *d_n, uint32_t *d_queue, int grid, cudaStream_t s) {
  pack_batch_kernel<<<grid, 256, 0, s>>>(d_descs, d_row_prefix, d_n, d_queue);
  return cudaGetLastError();
}

template <int TW>
static cudaError_t launch_plain_tw(int variant, const ImgDesc &d, const CUtensorMap &map,
                                   const RingCfg &rc, dim3 grid, size_t smem, uint32_t *err,
                                   uint64_t timeout_ns, cudaStream_t s) {
  if (variant == kVarA)
    tile_plain_kernel<TW, kVarA><<<grid, TW, smem, s>>>(map, d, rc, err, timeout_ns);
  else
    tile_plain_kernel<TW, kVarB><<<grid, TW, smem, s>>>(map, d, rc, err, timeout_ns);
  return cudaGetLastError();
}

cudaError_t launch_tile_plain(uint32_t tw, int variant, const ImgDesc &d, const CUtensorMap &map,
                              const RingCfg &rc, dim3 grid, size_t smem, uint32_t *err,
                              uint64_t timeout_ns, cudaStream_t s) {
  switch (tw) {
    case 32: return launch_plain_tw<32>(variant, d, map, rc, grid, smem, err, timeout_ns, s);
    case 64: return launch_plain_tw<64>(variant, d, map, rc, grid, smem, err, timeout_ns, s);
    case 128: return launch_plain_tw<128>(variant, d, map, rc, grid, smem, err, timeout_ns, s);
    case 256: return launch_plain_tw<256>(variant, d, map, rc, grid, smem, err, timeout_ns, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_persistent(uint32_t tw, const ImgDesc *d_descs, const uint32_t *d_tile_prefix,
                              const uint32_t *d_n, uint32_t *d_queue, const RingCfg &rc, uint32_t lmax,
                              int grid, size_t smem, uint32_t *err, uint64_t timeout_ns,
                              cudaStream_t s) {
  switch (tw) {
    case 32:
      persistent_kernel<32><<<grid, 32, smem, s>>>(d_descs, d_tile_prefix, d_n, d_queue, rc, lmax,
                                                   err, timeout_ns);
      break;
    case 64:
      persistent_kernel<64><<<grid, 64, smem, s>>>(d_descs, d_tile_prefix, d_n, d_queue, rc, lmax,
                                                   err, timeout_ns);
      break;
    case 128:
      persistent_kernel<128><<<grid, 128, smem, s>>>(d_descs, d_tile_prefix, d_n, d_queue, rc,
                                                     lmax, err, timeout_ns);
      break;
    case 256:
      persistent_kernel<256><<<grid, 256, smem, s>>>(d_descs, d_tile_prefix, d_n, d_queue, rc,
                                                     lmax, err, timeout_ns);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_selftest_wait(uint32_t *d_err, uint64_t timeout_ns, cudaStream_t s) {
  selftest_wait_kernel<<<1, 32, 0, s>>>(d_err, timeout_ns);
  return cudaGetLastError();
}

template <int TW>
static cudaError_t set_limit_tw(size_t bytes) {
  const int b = static_cast<int>(bytes);
  cudaError_t e = cudaFuncSetAttribute(tile_plain_kernel<TW, kVarA>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(tile_plain_kernel<TW, kVarB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(persistent_kernel<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              b);
}

cudaError_t set_tile_smem_limit(uint32_t tw, size_t bytes) {
  switch (tw) {
    case 32: return set_limit_tw<32>(bytes);
    case 64: return set_limit_tw<64>(bytes);
    case 128: return set_limit_tw<128>(bytes);
    case 256: return set_limit_tw<256>(bytes);
    default: return cudaErrorInvalidValue;
  }
}

template <int TW>
static int occupancy_tw(int variant, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (variant == kVarA)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tile_plain_kernel<TW, kVarA>, TW, smem);
  else if (variant == kVarB)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tile_plain_kernel<TW, kVarB>, TW, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persistent_kernel<TW>, TW, smem);
  return e == cudaSuccess ? n : 0;
}

int tile_occupancy(uint32_t tw, int variant, size_t smem) {
  switch (tw) {
    case 32: return occupancy_tw<32>(variant, smem);
    case 64: return occupancy_tw<64>(variant, smem);
    case 128: return occupancy_tw<128>(variant, smem);
    case 256: return occupancy_tw<256>(variant, smem);
    default: return 0;
  }
}

}  // namespace opk
