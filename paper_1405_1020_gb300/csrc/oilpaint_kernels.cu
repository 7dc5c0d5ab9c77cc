// oilpaint_kernels.cu -- kernel entry points and their launchers.
//
//   pack_single_kernel / pack_batch_kernel  the pack prepass (one image, a
//                                           row per block / a batch, a row per
//                                           warp; the batch form also resets
//                                           the groups' tile-queue counters)
//   tile_plain_kernel<NT, VAR>              one CTA per output tile, one output
//                                           column per thread (NT threads)
//   tile_delta_kernel<NT, K, VAR>           one CTA per output tile, K output
//                                           columns per thread through
//                                           difference histograms (one kernel
//                                           per radius instead: oilpaint_delta4.cu,
//                                           oilpaint_delta8.cu)
//   tile_cols_kernel<NW, TWK, VAR>          one CTA per output tile, column
//                                           histograms swept by NW warps
//   persistent_kernel<NT, K>                grid-sized CTAs pulling
//                                           (image, tile) tickets from one
//                                           batch group's device atomic until
//                                           its queue is empty
//   selftest_wait_kernel                    exercises the bounded mbarrier wait
#include "oilpaint_internal.h"

namespace opk {

// Both pack kernels are held to 40 registers (6 blocks of 256 per SM) and
// the single-image launch takes one row per block: the pack streams its
// input once, so the loads in flight per SM decide its speed.  At 48
// registers and three rows per block the 12 MP RGBA pack took 24 us and the
// RGB one about 30 us; with more blocks resident and one row each, 22 us and
// 24 us.
__global__ void __launch_bounds__(256, 6) pack_single_kernel(const ImgDesc d) {
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

__global__ void __launch_bounds__(256, 6)
    pack_batch_kernel(const ImgDesc *__restrict__ descs, const uint32_t *__restrict__ row_prefix,
                      const uint32_t *__restrict__ d_n, uint32_t *queues, uint32_t nqueues) {
  // the filter launches that follow start their ticket queues from zero
  if (blockIdx.x == 0 && threadIdx.x < nqueues) queues[threadIdx.x] = 0u;
  const uint32_t n = __ldg(d_n);
  if (n == 0) return;
  const uint32_t total = __ldg(row_prefix + n);
  // One row per warp: a batch's rows are short and each starts with a
  // dependent search and descriptor load, so many rows in flight per block
  // hide those latencies (one row per block left the launch at 45% of the
  // copy bandwidth on the 64-image batch).
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < total; g += nwarps) {
    const uint32_t i = find_image(row_prefix, n, g);
    const ImgDesc d = descs[i];
    pack_row(d, g - __ldg(row_prefix + i), lane, 32u);
  }
}

template <int NT, int VAR>
__global__ void __launch_bounds__(NT, 1)
    tile_plain_kernel(const __grid_constant__ CUtensorMap tmap, const ImgDesc d, const RingCfg rc,
                      uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  const SmemMap sm = carve_smem(smem, rc, (d.L + 1u) * NT);
  init_cta(sm, rc);
  uint32_t ctr = 0;
  const int x0 = static_cast<int>(blockIdx.x) * NT;
  const int y0 = d.oy0 + static_cast<int>(blockIdx.y * d.tile_h);
  const int y1 = min(y0 + static_cast<int>(d.tile_h), d.oy1);
  run_tile<NT, VAR>(d, &tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns);
}

template <int NT, int K, int VAR>
__global__ void __launch_bounds__(NT, 1)
    tile_delta_kernel(const __grid_constant__ CUtensorMap tmap, const ImgDesc d, const RingCfg rc,
                      uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  const SmemMap sm = carve_smem(smem, rc, 0u);
  init_cta(sm, rc);
  uint32_t ctr = 0;
  const int x0 = d.xshift + static_cast<int>(blockIdx.x) * NT * K;
  const int y0 = d.oy0 + static_cast<int>(blockIdx.y * d.tile_h);
  const int y1 = min(y0 + static_cast<int>(d.tile_h), d.oy1);
  run_tile_delta<NT, K, VAR>(d, &tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns);
}

// Radius 2's window and counts fit 128 registers per thread (then 4 CTAs of
// 128 threads per SM); unbounded, the unrolled comparisons take all 255.
template <int NT, int R>
__global__ void __launch_bounds__(NT, R < 2 ? 1 : 65536 / (NT * 128))
    tile_direct_kernel(const __grid_constant__ CUtensorMap tmap, const ImgDesc d,
                       const RingCfg rc, uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  const SmemMap sm = carve_smem(smem, rc, 0u);
  init_cta(sm, rc);
  uint32_t ctr = 0;
  const int x0 = static_cast<int>(blockIdx.x) * NT;
  const int y0 = d.oy0 + static_cast<int>(blockIdx.y * d.tile_h);
  const int y1 = min(y0 + static_cast<int>(d.tile_h), d.oy1);
  run_tile_direct<NT, R>(d, &tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns);
}

template <int NW, int TWK, int VAR>
__global__ void __launch_bounds__(32 * NW, 1)
    tile_cols_kernel(const __grid_constant__ CUtensorMap tmap, const ImgDesc d, const RingCfg rc,
                     uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  const SmemMap sm = carve_smem(smem, rc, 0u);
  init_cta(sm, rc);
  uint32_t ctr = 0;
  const int x0 = d.xshift + static_cast<int>(blockIdx.x) * (32 * NW * TWK);
  const int y0 = d.oy0 + static_cast<int>(blockIdx.y * d.tile_h);
  const int y1 = min(y0 + static_cast<int>(d.tile_h), d.oy1);
  run_tile_cols<NW, TWK, VAR>(d, &tmap, x0, y0, y1, rc, sm, ctr, err, timeout_ns);
}

// K = 1: every image on the one-column path; K = 2 or 4: images with
// d.kcols == K on the difference-histogram path, the others on the
// one-column path.  Shared memory is sized by the host for the largest.
// d_grp points at the group's image count; kBatchGroups and 2 kBatchGroups
// words further on lie the index of its first descriptor and of its first
// tile-prefix entry, so one fixed launch serves any batch composition.
template <int NT, int K>
__global__ void __launch_bounds__(NT, 1)
    persistent_kernel(const ImgDesc *__restrict__ descs, const uint32_t *__restrict__ tile_prefix,
                      const uint32_t *__restrict__ d_grp, uint32_t *queue, const RingCfg rc,
                      uint32_t lmax, uint32_t *err, uint64_t timeout_ns) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint32_t s_job[2];
  const SmemMap sm = carve_smem(smem, rc, (lmax + 1u) * NT);
  init_cta(sm, rc);
  const uint32_t n = __ldg(d_grp);
  if (n == 0) return;
  descs += __ldg(d_grp + kBatchGroups);
  tile_prefix += __ldg(d_grp + 2 * kBatchGroups);
  const uint32_t total = __ldg(tile_prefix + n);
  uint32_t ctr = 0;
  // the batch's control block keeps a timeout diagnostic record 8 words
  // after the error word
  uint32_t *diag = err + 7;
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
    const int tw = NT * static_cast<int>(d.kcols);
    const int x0 = d.xshift + static_cast<int>(local % d.tiles_x) * tw;
    const int y0 = d.oy0 + static_cast<int>((local / d.tiles_x) * d.tile_h);
    const int y1 = min(y0 + static_cast<int>(d.tile_h), d.oy1);
    bool ok;
    if (K > 1 && d.kcols == static_cast<uint32_t>(K)) {
      constexpr int KD = K > 1 ? K : 2;
      ok = d.variant == kVarA
               ? run_tile_delta<NT, KD, kVarA>(d, d.tmap, x0, y0, y1, rc, sm, ctr, err,
                                               timeout_ns, diag, true)
               : run_tile_delta<NT, KD, kVarB>(d, d.tmap, x0, y0, y1, rc, sm, ctr, err,
                                               timeout_ns, diag, true);
    } else {
      // this image's counts follow its own L + 1 levels of sums
      SmemMap smi = sm;
      smi.cnts = sm.sums + (d.L + 1u) * NT * 8u;
      ok = d.variant == kVarA ? run_tile<NT, kVarA>(d, d.tmap, x0, y0, y1, rc, smi, ctr, err,
                                                    timeout_ns, diag, true)
                              : run_tile<NT, kVarB>(d, d.tmap, x0, y0, y1, rc, smi, ctr, err,
                                                    timeout_ns, diag, true);
    }
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
                              const uint32_t *d_n, uint32_t *d_queues, uint32_t nqueues, int grid,
                              cudaStream_t s) {
  if (nqueues > 256u) return cudaErrorInvalidValue;
  pack_batch_kernel<<<grid, 256, 0, s>>>(d_descs, d_row_prefix, d_n, d_queues, nqueues);
  return cudaGetLastError();
}

template <int NT>
static void plain_n(int variant, const ImgDesc &d, const CUtensorMap &map, const RingCfg &rc,
                    dim3 grid, size_t smem, uint32_t *err, uint64_t timeout_ns, cudaStream_t s) {
  if (variant == kVarA)
    tile_plain_kernel<NT, kVarA><<<grid, NT, smem, s>>>(map, d, rc, err, timeout_ns);
  else
    tile_plain_kernel<NT, kVarB><<<grid, NT, smem, s>>>(map, d, rc, err, timeout_ns);
}

template <int NT>
static void delta_n(int k, const ImgDesc &d, const CUtensorMap &map, const RingCfg &rc,
                    dim3 grid, size_t smem, uint32_t *err, uint64_t timeout_ns, cudaStream_t s) {
  const bool a = d.variant == static_cast<uint32_t>(kVarA);
  if (k == 4) {
    if (a)
      tile_delta_kernel<NT, 4, kVarA><<<grid, NT, smem, s>>>(map, d, rc, err, timeout_ns);
    else
      tile_delta_kernel<NT, 4, kVarB><<<grid, NT, smem, s>>>(map, d, rc, err, timeout_ns);
  } else {
    if (a)
      tile_delta_kernel<NT, 2, kVarA><<<grid, NT, smem, s>>>(map, d, rc, err, timeout_ns);
    else
      tile_delta_kernel<NT, 2, kVarB><<<grid, NT, smem, s>>>(map, d, rc, err, timeout_ns);
  }
}

template <int NW>
static void cols_n(int twk, int variant, const ImgDesc &d, const CUtensorMap &map,
                   const RingCfg &rc, dim3 grid, size_t smem, uint32_t *err, uint64_t timeout_ns,
                   cudaStream_t s) {
  const bool a = variant == kVarA;
  if (twk == 2) {
    if (a)
      tile_cols_kernel<NW, 2, kVarA><<<grid, 32 * NW, smem, s>>>(map, d, rc, err, timeout_ns);
    else
      tile_cols_kernel<NW, 2, kVarB><<<grid, 32 * NW, smem, s>>>(map, d, rc, err, timeout_ns);
  } else {
    if (a)
      tile_cols_kernel<NW, 1, kVarA><<<grid, 32 * NW, smem, s>>>(map, d, rc, err, timeout_ns);
    else
      tile_cols_kernel<NW, 1, kVarB><<<grid, 32 * NW, smem, s>>>(map, d, rc, err, timeout_ns);
  }
}

// The direct kernel of nt threads and radius r (nullptr outside the table).
using DirectFn = void (*)(const CUtensorMap, const ImgDesc, const RingCfg, uint32_t *, uint64_t);
static DirectFn direct_fn(uint32_t nt, int r) {
  static constexpr DirectFn fns[4][kDirectMaxRadius + 1] = {
      {tile_direct_kernel<32, 0>, tile_direct_kernel<32, 1>, tile_direct_kernel<32, 2>},
      {tile_direct_kernel<64, 0>, tile_direct_kernel<64, 1>, tile_direct_kernel<64, 2>},
      {tile_direct_kernel<96, 0>, tile_direct_kernel<96, 1>, tile_direct_kernel<96, 2>},
      {tile_direct_kernel<128, 0>, tile_direct_kernel<128, 1>, tile_direct_kernel<128, 2>}};
  const int i = nt == 32 ? 0 : nt == 64 ? 1 : nt == 96 ? 2 : nt == 128 ? 3 : -1;
  if (i < 0 || r < 0 || r > kDirectMaxRadius) return nullptr;
  return fns[i][r];
}

int direct_occupancy(uint32_t nt, int r, size_t smem) {
  const DirectFn f = direct_fn(nt, r);
  if (!f) return 0;
  int n = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, static_cast<int>(nt), smem) ==
                 cudaSuccess
             ? n
             : 0;
}

cudaError_t launch_tile(uint32_t nt, int kcols, int variant, const ImgDesc &d,
                        const CUtensorMap &map, const RingCfg &rc, dim3 grid, size_t smem,
                        uint32_t *err, uint64_t timeout_ns, cudaStream_t s) {
  if (d.path == kPathDirect) {
    const DirectFn f = direct_fn(nt, d.r);
    if (!f || kcols != 1 || d.fmt != 0u) return cudaErrorInvalidValue;
    f<<<grid, nt, smem, s>>>(map, d, rc, err, timeout_ns);
    return cudaGetLastError();
  }
  if (d.path == 1u) {
    if (kcols != 1 && kcols != 2) return cudaErrorInvalidValue;
    switch (nt) {
      case 32: cols_n<1>(kcols, variant, d, map, rc, grid, smem, err, timeout_ns, s); break;
      case 64: cols_n<2>(kcols, variant, d, map, rc, grid, smem, err, timeout_ns, s); break;
      case 128: cols_n<4>(kcols, variant, d, map, rc, grid, smem, err, timeout_ns, s); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  if (d.path == 2u || d.path == 3u)
    return launch_deltak(nt, d, map, rc, grid, smem, err, timeout_ns, s);
  if (kcols != 1 && kcols != 2 && kcols != 4) return cudaErrorInvalidValue;
  switch (nt) {
    case 32:
      kcols == 1 ? plain_n<32>(variant, d, map, rc, grid, smem, err, timeout_ns, s)
                 : delta_n<32>(kcols, d, map, rc, grid, smem, err, timeout_ns, s);
      break;
    case 64:
      kcols == 1 ? plain_n<64>(variant, d, map, rc, grid, smem, err, timeout_ns, s)
                 : delta_n<64>(kcols, d, map, rc, grid, smem, err, timeout_ns, s);
      break;
    case 96:
      kcols == 1 ? plain_n<96>(variant, d, map, rc, grid, smem, err, timeout_ns, s)
                 : delta_n<96>(kcols, d, map, rc, grid, smem, err, timeout_ns, s);
      break;
    case 128:
      kcols == 1 ? plain_n<128>(variant, d, map, rc, grid, smem, err, timeout_ns, s)
                 : delta_n<128>(kcols, d, map, rc, grid, smem, err, timeout_ns, s);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NT>
static void persistent_n(int k, const ImgDesc *d_descs, const uint32_t *d_tile_prefix,
                         const uint32_t *d_grp, uint32_t *d_queue, const RingCfg &rc,
                         uint32_t lmax, int grid, size_t smem, uint32_t *err,
                         uint64_t timeout_ns, cudaStream_t s) {
  if (k == 4)
    persistent_kernel<NT, 4><<<grid, NT, smem, s>>>(d_descs, d_tile_prefix, d_grp, d_queue, rc,
                                                    lmax, err, timeout_ns);
  else if (k == 2)
    persistent_kernel<NT, 2><<<grid, NT, smem, s>>>(d_descs, d_tile_prefix, d_grp, d_queue, rc,
                                                    lmax, err, timeout_ns);
  else
    persistent_kernel<NT, 1><<<grid, NT, smem, s>>>(d_descs, d_tile_prefix, d_grp, d_queue, rc,
                                                    lmax, err, timeout_ns);
}

cudaError_t launch_persistent(uint32_t nt, int kcols, const ImgDesc *d_descs,
                              const uint32_t *d_tile_prefix, const uint32_t *d_grp,
                              uint32_t *d_queue, const RingCfg &rc, uint32_t lmax, int grid,
                              size_t smem, uint32_t *err, uint64_t timeout_ns, cudaStream_t s) {
  if (kcols != 1 && kcols != 2 && kcols != 4) return cudaErrorInvalidValue;
  switch (nt) {
    case 32:
      persistent_n<32>(kcols, d_descs, d_tile_prefix, d_grp, d_queue, rc, lmax, grid, smem, err,
                       timeout_ns, s);
      break;
    case 64:
      persistent_n<64>(kcols, d_descs, d_tile_prefix, d_grp, d_queue, rc, lmax, grid, smem, err,
                       timeout_ns, s);
      break;
    case 96:
      persistent_n<96>(kcols, d_descs, d_tile_prefix, d_grp, d_queue, rc, lmax, grid, smem, err,
                       timeout_ns, s);
      break;
    case 128:
      persistent_n<128>(kcols, d_descs, d_tile_prefix, d_grp, d_queue, rc, lmax, grid, smem, err,
                        timeout_ns, s);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t take_check_error(uint32_t *bits) {
#if OPK_CHECKED
  uint32_t v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_check_error, sizeof(v));
  if (e == cudaSuccess && v) {
    const uint32_t z = 0;
    e = cudaMemcpyToSymbol(g_check_error, &z, sizeof(z));
  }
  *bits = v;
  return e;
#else
  *bits = 0;
  return cudaSuccess;
#endif
}

cudaError_t launch_selftest_wait(uint32_t *d_err, uint64_t timeout_ns, cudaStream_t s) {
  selftest_wait_kernel<<<1, 32, 0, s>>>(d_err, timeout_ns);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t set_limit_n(int b) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(tile_plain_kernel<NT, kVarA>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tile_plain_kernel<NT, kVarB>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tile_delta_kernel<NT, 2, kVarA>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tile_delta_kernel<NT, 4, kVarA>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tile_delta_kernel<NT, 2, kVarB>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tile_delta_kernel<NT, 4, kVarB>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(persistent_kernel<NT, 1>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(persistent_kernel<NT, 2>, a, b)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(persistent_kernel<NT, 4>, a, b);
}

template <int NW>
static cudaError_t set_limit_cols(int b) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(tile_cols_kernel<NW, 1, kVarA>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tile_cols_kernel<NW, 1, kVarB>, a, b)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(tile_cols_kernel<NW, 2, kVarA>, a, b)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(tile_cols_kernel<NW, 2, kVarB>, a, b);
}

cudaError_t set_tile_smem_limit(size_t bytes) {
  const int b = static_cast<int>(bytes);
  cudaError_t e;
  if ((e = set_deltak_smem_limit(bytes)) != cudaSuccess) return e;
  for (uint32_t nt : {32u, 64u, 96u, 128u})
    for (int r = 0; r <= kDirectMaxRadius; ++r)
      if ((e = cudaFuncSetAttribute(direct_fn(nt, r), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    b)) != cudaSuccess)
        return e;
  if ((e = set_limit_cols<1>(b)) != cudaSuccess) return e;
  if ((e = set_limit_cols<2>(b)) != cudaSuccess) return e;
  if ((e = set_limit_cols<4>(b)) != cudaSuccess) return e;
  if ((e = set_limit_n<32>(b)) != cudaSuccess) return e;
  if ((e = set_limit_n<64>(b)) != cudaSuccess) return e;
  if ((e = set_limit_n<96>(b)) != cudaSuccess) return e;
  return set_limit_n<128>(b);
}

template <class F>
static int occ_of(F f, int nt, size_t smem) {
  int n = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, nt, smem) == cudaSuccess ? n : 0;
}

template <int NT>
static int occupancy_n(bool persistent, int kcols, int variant, size_t smem) {
  if (persistent) {
    if (kcols == 4) return occ_of(persistent_kernel<NT, 4>, NT, smem);
    if (kcols == 2) return occ_of(persistent_kernel<NT, 2>, NT, smem);
    return occ_of(persistent_kernel<NT, 1>, NT, smem);
  }
  if (kcols == 4)
    return variant == kVarA ? occ_of(tile_delta_kernel<NT, 4, kVarA>, NT, smem)
                            : occ_of(tile_delta_kernel<NT, 4, kVarB>, NT, smem);
  if (kcols == 2)
    return variant == kVarA ? occ_of(tile_delta_kernel<NT, 2, kVarA>, NT, smem)
                            : occ_of(tile_delta_kernel<NT, 2, kVarB>, NT, smem);
  return variant == kVarA ? occ_of(tile_plain_kernel<NT, kVarA>, NT, smem)
                          : occ_of(tile_plain_kernel<NT, kVarB>, NT, smem);
}

template <int NW>
static int occupancy_cols(int twk, int variant, size_t smem) {
  const bool a = variant == kVarA;
  if (twk == 2)
    return a ? occ_of(tile_cols_kernel<NW, 2, kVarA>, 32 * NW, smem)
             : occ_of(tile_cols_kernel<NW, 2, kVarB>, 32 * NW, smem);
  return a ? occ_of(tile_cols_kernel<NW, 1, kVarA>, 32 * NW, smem)
           : occ_of(tile_cols_kernel<NW, 1, kVarB>, 32 * NW, smem);
}

int tile_occupancy_cols(uint32_t nt, int twk, int variant, size_t smem) {
  switch (nt) {
    case 32: return occupancy_cols<1>(twk, variant, smem);
    case 64: return occupancy_cols<2>(twk, variant, smem);
    case 128: return occupancy_cols<4>(twk, variant, smem);
    default: return 0;
  }
}

static DeltaKFn deltak_fn(uint32_t nt, int k, int nb, int r) {
  return k == 2   ? deltak_kernel_k2(nt, nb, r)
         : k == 4 ? deltak_kernel_k4(nt, nb, r)
         : k == 8 ? deltak_kernel_k8(nt, nb, r)
                  : nullptr;
}

cudaError_t launch_deltak(uint32_t nt, const ImgDesc &d, const CUtensorMap &map,
                          const RingCfg &rc, dim3 grid, size_t smem, uint32_t *err,
                          uint64_t timeout_ns, cudaStream_t s) {
  const DeltaKFn f = deltak_fn(nt, static_cast<int>(d.kcols), static_cast<int>(d.path) - 1,
                                   d.r);
  if (!f || d.variant != static_cast<uint32_t>(kVarA) ||
      d.L > (d.kcols == 2u ? kDeltaK2MaxLevels : kDeltaMaxLevels))
    return cudaErrorInvalidValue;
  f<<<grid, nt, smem, s>>>(map, d, rc, err, timeout_ns);
  return cudaGetLastError();
}

cudaError_t set_deltak_smem_limit(size_t bytes) {
  for (int k : {2, 4, 8})
    for (uint32_t nt : {32u, 64u})
      for (int nb : {1, 2})
        for (int r = deltak_min_radius(k); r <= kDeltaKMaxRadius; ++r) {
          if (k == 2 && nb == 2) continue;
          const cudaError_t e =
              cudaFuncSetAttribute(deltak_fn(nt, k, nb, r),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(bytes));
          if (e != cudaSuccess) return e;
        }
  return cudaSuccess;
}

int deltak_occupancy(uint32_t nt, int k, int nb, size_t smem) {
  // the same resources at every radius of one (nt, k, nb)
  const DeltaKFn f = deltak_fn(nt, k, nb, kDeltaKMaxRadius);
  if (!f) return 0;
  int n = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, static_cast<int>(nt), smem) ==
                 cudaSuccess
             ? n
             : 0;
}

int tile_occupancy(uint32_t nt, bool persistent, int kcols, int variant, size_t smem) {
  switch (nt) {
    case 32: return occupancy_n<32>(persistent, kcols, variant, smem);
    case 64: return occupancy_n<64>(persistent, kcols, variant, smem);
    case 96: return occupancy_n<96>(persistent, kcols, variant, smem);
    case 128: return occupancy_n<128>(persistent, kcols, variant, smem);
    default: return 0;
  }
}

}  // namespace opk
