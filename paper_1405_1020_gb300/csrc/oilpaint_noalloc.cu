// oilpaint_noalloc.cu -- op_run_noalloc: the filter without any device
// allocation.
//
// Who needs it: some callers cannot allocate device memory at all.  A plugin
// running inside a host application that owns every byte of device memory
// through its own pool (a foreign cudaMalloc fails, or breaks the host's
// budget), code on a latency-critical path where the implicit device-wide
// synchronisation of cudaMalloc/cudaFree is not acceptable, and processes
// whose free memory another allocator has already claimed.  op_run needs a
// packed-word workspace of 4 bytes per pixel and, unless the caller hands it
// one, allocates it; this entry point instead uses a fixed scratch array
// compiled into the library.
//
// The scratch array is a file-scope __device__ array of kNoAllocWords 32-bit
// words (16 MiB).  This file is a module of its own, and the CUDA runtime
// loads a module (and with it places the array in device memory) the first
// time the module is used on a device -- here, the first
// cudaGetSymbolAddress of a call on that device, or the first after a
// cudaDeviceReset.  That first call therefore needs 16 MiB of free device
// memory and fails with OP_E_CUDA without it; later calls find the array in
// place and allocate nothing.  The array stays until the process exits (or
// the device is reset).
//
// Host code cannot use the array's name as a device address (in host code
// it names a host-side stand-in), so every call asks the runtime for the
// device address with cudaGetSymbolAddress, on the current device.  Every
// call shares the array and it keeps the last call's contents; the pack
// prepass rewrites every word the filter then reads, and the error word is
// cleared at the start of each call.  Calls that overlap on the GPU (two
// host threads, two streams) race on the array.
#include <algorithm>

#include "oilpaint.h"
#include "oilpaint_internal.h"

// The scratch: packed words of the image being filtered, and the device
// error word of the bounded waits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[OP_NOALLOC_MAX_WORDS];
static __device__ __align__(256) uint32_t g_noalloc_error;

namespace {

constexpr size_t kNoAllocWords = OP_NOALLOC_MAX_WORDS;
constexpr uint64_t kWaitTimeoutNs = 1000000000ull;

// A CUDA call failed: clear the runtime's last error, so that it is not
// reported again by a later, unrelated launch check, and return OP_E_CUDA.
int cuda_failed() {
  (void)cudaGetLastError();
  return OP_E_CUDA;
}

}  // namespace

extern "C" int op_run_noalloc(const uint8_t *d_in, uint8_t *d_out, uint32_t width,
                              uint32_t height, uint32_t stride, uint32_t bpp, int32_t radius,
                              uint32_t levels, uint32_t flags, void *stream) {
  if (!d_in || !d_out || width < 1 || height < 1 || width > OP_MAX_DIM || height > OP_MAX_DIM ||
      (bpp != 3 && bpp != 4) || static_cast<uint64_t>(stride) < static_cast<uint64_t>(width) * bpp ||
      radius < 0 || radius > OP_MAX_RADIUS || levels < 1 || levels > OP_MAX_LEVELS ||
      (flags & ~(OP_LEVEL_INTDIV3 | OP_LITERAL | OP_FUSED_PACK)) ||
      ((flags & OP_LITERAL) && levels > OP_LITERAL_MAX_LEVELS))
    return OP_E_INVALID;
  const size_t bytes = static_cast<size_t>(height) * stride;
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
  if (a < b + bytes && b < a + bytes) return OP_E_INVALID;
  const uint32_t ppitch = (width + 3u) & ~3u;
  if (static_cast<uint64_t>(ppitch) * height > kNoAllocWords) return OP_E_UNSUPPORTED;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_failed();
  // The arrays' device addresses on the current device (the first call on a
  // device loads this file's module there; see above).
  void *p_scratch = nullptr, *p_err = nullptr;
  if (cudaGetSymbolAddress(&p_scratch, g_noalloc_scratch) != cudaSuccess ||
      cudaGetSymbolAddress(&p_err, g_noalloc_error) != cudaSuccess)
    return cuda_failed();
  uint32_t *packed = static_cast<uint32_t *>(p_scratch);
  uint32_t *d_err = static_cast<uint32_t *>(p_err);
  op_config_t cfg;
  int st = op_default_config(radius, levels, &cfg);
  if (st != OP_OK) {
    if (st == OP_E_CUDA) (void)cudaGetLastError();
    return st;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cuda_failed();

  const int cpt = (cfg.cols_per_thread == 2 || cfg.cols_per_thread == 4)
                      ? static_cast<int>(cfg.cols_per_thread)
                      : 1;
  const opk::Geometry g = opk::image_geometry(static_cast<int>(cfg.path),
                                              cfg.tile_w / static_cast<uint32_t>(cpt), cpt,
                                              radius, levels, width);
  const uint32_t boxw = g.boxw;
  const opk::RingCfg rc = opk::make_ring(radius, cfg.chunk_rows, cfg.prefetch, boxw);
  const size_t smem = opk::tile_smem_bytes(opk::geometry_hist_bytes(g, radius, levels), rc);

  opk::ImgDesc d{};
  d.in = d_in;
  d.out = d_out;
  d.packed = packed;
  d.tmap = nullptr;
  d.w = width;
  d.h = height;
  d.stride = stride;
  d.ostride = stride;
  d.bpp = bpp;
  d.r = radius;
  d.L = levels;
  d.mode = flags & (OP_LEVEL_INTDIV3 | OP_LITERAL);
  d.ppitch = ppitch;
  d.tiles_x = g.tiles_x;
  const opk::Window win = opk::output_window(width, height, radius, flags);
  opk::set_window(d, win);
  if (win.rows() == 0u) return OP_OK;  // literal mode: no pixel is r from every edge
  if (cfg.tile_h) {
    d.tile_h = std::min(cfg.tile_h, win.rows());
  } else {
    const int occ = std::max(1, opk::geometry_occupancy(g, smem));
    d.tile_h = opk::auto_tile_h(win.rows(), d.tiles_x, radius, static_cast<uint64_t>(occ) * sms);
  }
  d.boxw = boxw;
  d.variant = static_cast<uint32_t>(g.variant);
  d.kcols = static_cast<uint32_t>(g.kcols);
  d.xshift = g.xshift;
  d.fmt = g.fmt;
  d.path = static_cast<uint32_t>(g.path);

  CUtensorMap map;
  if (!opk::encode_packed_map(&map, packed, width, height, ppitch, boxw, cfg.chunk_rows))
    return cuda_failed();

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s) != cudaSuccess) return cuda_failed();
  const int pack_grid = opk::pack_grid_for(height, sms);
  if (opk::launch_pack_single(d, pack_grid, s) != cudaSuccess) return cuda_failed();
  const dim3 grid(d.tiles_x, (win.rows() + d.tile_h - 1) / d.tile_h);
  if (opk::launch_tile(g.nt, g.kcols, g.variant, d, map, rc, grid, smem, d_err, kWaitTimeoutNs,
                       s) != cudaSuccess)
    return cuda_failed();
  uint32_t err = 0;
  if (cudaMemcpyAsync(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_failed();
  if (err) return OP_E_TIMEOUT;
  uint32_t bits = 0;
  if (opk::take_check_error(&bits) != cudaSuccess) return cuda_failed();
  return bits ? OP_E_BOUNDS : OP_OK;
}
