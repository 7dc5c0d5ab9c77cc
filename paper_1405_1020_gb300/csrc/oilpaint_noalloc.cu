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
// words (16 MiB): every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device address
// (in host code it names a host-side stand-in), so the device address is
// taken once per device with cudaGetSymbolAddress, with that device current,
// on the first call made on it.  Every call shares the array and it keeps the
// last call's contents; the pack prepass rewrites every word the filter then
// reads, and the error word is cleared at the start of each call.  Calls that
// overlap on the GPU (two host threads, two streams) race on the array.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "oilpaint.h"
#include "oilpaint_internal.h"

// The scratch: packed words of the image being filtered, and the device
// error word of the bounded waits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[OP_NOALLOC_MAX_WORDS];
static __device__ __align__(256) uint32_t g_noalloc_error;

namespace {

constexpr size_t kNoAllocWords = OP_NOALLOC_MAX_WORDS;
constexpr int kMaxDevices = 64;
constexpr uint64_t kWaitTimeoutNs = 1000000000ull;

struct DeviceScratch {
  bool ready = false;
  uint32_t *packed = nullptr;  // device address of g_noalloc_scratch
  uint32_t *err = nullptr;     // device address of g_noalloc_error
};

std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

// Looks the scratch addresses up for device `dev` (the current device).
int scratch_for(int dev, DeviceScratch *out) {
  if (dev < 0 || dev >= kMaxDevices) return OP_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceScratch &s = g_dev[dev];
  if (!s.ready) {
    void *p = nullptr, *e = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return OP_E_CUDA;
    if (cudaGetSymbolAddress(&e, g_noalloc_error) != cudaSuccess) return OP_E_CUDA;
    s.packed = static_cast<uint32_t *>(p);
    s.err = static_cast<uint32_t *>(e);
    s.ready = true;
  }
  *out = s;
  return OP_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Output rows per CTA: the fewest waves of resident CTAs times the steps of
// one tile (h output rows cost h + 2r steps).
uint32_t pick_tile_h(uint32_t H, uint32_t tiles_x, int r, uint64_t slots) {
  double best = 1e300;
  uint32_t best_h = H;
  for (uint32_t t = 1; t <= H; ++t) {
    const uint32_t th = (H + t - 1) / t;
    if (t > 1 && (H + th - 1) / th != t) continue;
    const uint64_t waves = (static_cast<uint64_t>(tiles_x) * t + slots - 1) / slots;
    const double cost = static_cast<double>(waves) * (th + 2.0 * r);
    if (cost < best) {
      best = cost;
      best_h = th;
    }
  }
  return best_h;
}

}  // namespace

extern "C" int op_run_noalloc(const uint8_t *d_in, uint8_t *d_out, uint32_t width,
                              uint32_t height, uint32_t stride, uint32_t bpp, int32_t radius,
                              uint32_t levels, uint32_t flags, void *stream) {
  if (!d_in || !d_out || width < 1 || height < 1 || width > OP_MAX_DIM || height > OP_MAX_DIM ||
      (bpp != 3 && bpp != 4) || static_cast<uint64_t>(stride) < static_cast<uint64_t>(width) * bpp ||
      radius < 0 || radius > OP_MAX_RADIUS || levels < 1 || levels > OP_MAX_LEVELS ||
      (flags & ~(OP_LEVEL_INTDIV3 | OP_LITERAL)) ||
      ((flags & OP_LITERAL) && levels > OP_LITERAL_MAX_LEVELS))
    return OP_E_INVALID;
  const size_t bytes = static_cast<size_t>(height) * stride;
  const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
  if (a < b + bytes && b < a + bytes) return OP_E_INVALID;
  const uint32_t ppitch = (width + 3u) & ~3u;
  if (static_cast<uint64_t>(ppitch) * height > kNoAllocWords) return OP_E_UNSUPPORTED;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OP_E_CUDA;
  DeviceScratch sc;
  int st = scratch_for(dev, &sc);
  if (st != OP_OK) return st;
  op_config_t cfg;
  st = op_default_config(radius, levels, &cfg);
  if (st != OP_OK) return st;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return OP_E_CUDA;

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
  d.packed = sc.packed;
  d.tmap = nullptr;
  d.w = width;
  d.h = height;
  d.stride = stride;
  d.ostride = stride;
  d.bpp = bpp;
  d.r = radius;
  d.L = levels;
  d.mode = flags;
  d.ppitch = ppitch;
  d.tiles_x = g.tiles_x;
  const opk::Window win = opk::output_window(width, height, radius, flags);
  opk::set_window(d, win);
  if (win.rows() == 0u) return OP_OK;  // literal mode: no pixel is r from every edge
  if (cfg.tile_h) {
    d.tile_h = std::min(cfg.tile_h, win.rows());
  } else {
    const int occ = std::max(1, opk::geometry_occupancy(g, smem));
    d.tile_h = pick_tile_h(win.rows(), d.tiles_x, radius, static_cast<uint64_t>(occ) * sms);
  }
  d.boxw = boxw;
  d.variant = static_cast<uint32_t>(g.variant);
  d.kcols = static_cast<uint32_t>(g.kcols);
  d.xshift = g.xshift;
  d.fmt = g.fmt;
  d.path = static_cast<uint32_t>(g.path);

  auto fn = encode_fn();
  if (!fn) return OP_E_CUDA;
  CUtensorMap map;
  cuuint64_t dims[2] = {width, height};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ppitch) * 4u};
  cuuint32_t box[2] = {boxw, cfg.chunk_rows};
  cuuint32_t estr[2] = {1, 1};
  if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, sc.packed, dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return OP_E_CUDA;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(sc.err, 0, sizeof(uint32_t), s) != cudaSuccess) return OP_E_CUDA;
  const int pack_grid = opk::pack_grid_for(height, sms);
  if (opk::launch_pack_single(d, pack_grid, s) != cudaSuccess) return OP_E_CUDA;
  const dim3 grid(d.tiles_x, (win.rows() + d.tile_h - 1) / d.tile_h);
  if (opk::launch_tile(g.nt, g.kcols, g.variant, d, map, rc, grid, smem, sc.err, kWaitTimeoutNs,
                       s) != cudaSuccess)
    return OP_E_CUDA;
  uint32_t err = 0;
  if (cudaMemcpyAsync(&err, sc.err, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return OP_E_CUDA;
  if (err) return OP_E_TIMEOUT;
  uint32_t bits = 0;
  if (opk::take_check_error(&bits) != cudaSuccess) return OP_E_CUDA;
  return bits ? OP_E_BOUNDS : OP_OK;
}
