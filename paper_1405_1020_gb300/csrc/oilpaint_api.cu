// oilpaint_api.cu -- the C ABI declared in include/oilpaint.h.
//
// Host side only: argument checks, launch configuration (tuning table,
// automatic tile height), workspace management, TMA tensor-map encoding,
// the batch descriptor tables and the CUDA-graph capture of a batch run.
// All filtering happens in the kernels of oilpaint_kernels.cu.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "oilpaint.h"
#include "oilpaint_internal.h"

using opk::ImgDesc;
using opk::RingCfg;

namespace opk {

namespace {

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

}  // namespace

bool encode_packed_map(CUtensorMap *map, const uint32_t *packed, uint32_t w, uint32_t h,
                       uint32_t ppitch, uint32_t boxw, uint32_t ch) {
  return encode_word_map(map, packed, w, h, static_cast<uint64_t>(ppitch) * 4u, boxw, ch);
}

bool encode_word_map(CUtensorMap *map, const void *base, uint32_t w, uint32_t h,
                     uint64_t pitch_bytes, uint32_t boxw, uint32_t ch) {
  auto fn = encode_fn();
  if (!fn) return false;
  if (pitch_bytes % 16u || reinterpret_cast<uintptr_t>(base) % 16u) return false;
  CUresult r;
  if (boxw <= kMaxBox2dWords) {
    cuuint64_t dims[2] = {w, h};
    cuuint64_t strides[1] = {pitch_bytes};
    cuuint32_t box[2] = {boxw, ch};
    cuuint32_t estr[2] = {1, 1};
    r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(base), dims, strides,
           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    // {4 words, ceil(w / 4) groups, rows}: the same rows, read in groups of
    // four words, so that a box row may be up to 4 * 256 words wide.  The
    // last group of a row may reach up to 3 words past word w - 1; they lie
    // inside the row because the pitch is a multiple of 16 bytes and holds
    // w words.
    if (boxw % 4u || boxw > kMaxBoxWords || pitch_bytes < 16u * ((w + 3u) / 4u)) return false;
    cuuint64_t dims[3] = {4, (w + 3u) / 4u, h};
    cuuint64_t strides[2] = {16, pitch_bytes};
    cuuint32_t box[3] = {4, boxw / 4u, ch};
    cuuint32_t estr[3] = {1, 1, 1};
    r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<void *>(base), dims, strides,
           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  return r == CUDA_SUCCESS;
}

uint32_t auto_tile_h(uint32_t H, uint32_t tiles_x, int r, uint64_t slots) {
  double best = 1e300;
  uint32_t best_h = H;
  if (slots < 1) slots = 1;
  // Only the distinct heights ceil(H / t) matter, each with the smallest t
  // giving it, in increasing t (O(sqrt H) of them; ties keep the smaller t):
  // after height th the next is reached at t = ceil(H / (th - 1)).
  for (uint32_t t = 1; t <= H;) {
    const uint32_t th = (H + t - 1) / t;
    const uint64_t tiles = static_cast<uint64_t>(tiles_x) * t;
    const uint64_t waves = (tiles + slots - 1) / slots;
    const double cost = static_cast<double>(waves) * (th + 2.0 * r);
    if (cost < best) {
      best = cost;
      best_h = th;
    }
    if (th == 1) break;
    t = (H + th - 2) / (th - 1);
  }
  return best_h;
}

}  // namespace opk

namespace {

thread_local int g_last_error = OP_OK;
constexpr uint64_t kWaitTimeoutNs = 1000000000ull;  // bounded device waits give up after 1 s

// ------------------------------------------------------------ device info

struct DevInfo {
  int sms = 0;
  size_t smem_optin = 0;
};

int device_info(int dev, DevInfo *out) {
  static std::mutex mu;
  static std::map<int, DevInfo> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) {
    *out = it->second;
    return OP_OK;
  }
  DevInfo di;
  int v = 0;
  if (cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return OP_E_CUDA;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return OP_E_CUDA;
  di.smem_optin = static_cast<size_t>(v);
  // The dynamic shared-memory limit is raised once per device to the maximum.
  if (opk::set_tile_smem_limit(di.smem_optin - 1024u) != cudaSuccess) return OP_E_CUDA;
  cache[dev] = di;
  *out = di;
  return OP_OK;
}

// NVTX range over one host call (a no-op unless a profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// ------------------------------------------------------------ configs

std::mutex g_tune_mu;
std::map<std::pair<int, uint32_t>, op_config_t> g_tune;
// batch groups, keyed by the group's largest radius and level count
std::map<std::pair<int, uint32_t>, op_config_t> g_batch_tune;

// Output columns per thread and threads per CTA of a configuration.
int cols_per_thread(const op_config_t &c) {
  return (c.cols_per_thread == 2 || c.cols_per_thread == 4 || c.cols_per_thread == 8)
             ? static_cast<int>(c.cols_per_thread)
             : 1;
}
uint32_t threads_of(const op_config_t &c) {
  return c.tile_w / static_cast<uint32_t>(cols_per_thread(c));
}

// Range checks that need no device.
bool config_in_range(const op_config_t &c) {
  if (c.path > 4u) return false;
  if (c.path == 4u && cols_per_thread(c) != 1) return false;  // direct: one column per thread
  if (c.cols_per_thread != 0 && c.cols_per_thread != 1 && c.cols_per_thread != 2 &&
      c.cols_per_thread != 4 && c.cols_per_thread != 8)
    return false;
  const uint32_t cpt = static_cast<uint32_t>(cols_per_thread(c));
  if (c.tile_w % cpt) return false;
  const uint32_t nt = c.tile_w / cpt;
  if (nt != 32 && nt != 64 && nt != 96 && nt != 128) return false;
  // the straight-line paths (2, 3): 4 or 8 columns of 32 or 64 threads, or 2
  // columns on path 2; eight columns exist only there (path 0 with 8 columns
  // means path 3)
  if ((c.path == 2u || c.path == 3u || cpt == 8u) && (nt > 64 || (cpt != 4u && cpt != 8u))) {
    // two columns: path 2 only (the window histogram in one part)
    if (!(c.path == 2u && cpt == 2u && nt <= 64)) return false;
  }
  if (cpt == 8u && c.path == 1u) return false;
  if (c.path == 1u && (cpt == 4u || nt == 96u)) return false;  // 1, 2 or 4 warps x 32 or 64
  if (c.chunk_rows < 1 || c.chunk_rows > 32 || c.prefetch < 1 || c.prefetch > 4) return false;
  return c.tile_h <= OP_MAX_DIM;
}

opk::Geometry geometry_of(const op_config_t &c, int r, uint32_t L, uint32_t w) {
  return opk::image_geometry(static_cast<int>(c.path), threads_of(c), cols_per_thread(c), r, L,
                             w);
}

size_t smem_of(const opk::Geometry &g, const op_config_t &c, int r, uint32_t L) {
  const RingCfg rc = opk::make_ring(r, c.chunk_rows, c.prefetch, g.boxw);
  return opk::tile_smem_bytes(opk::geometry_hist_bytes(g, r, L), rc);
}

size_t smem_for(const op_config_t &c, int r, uint32_t L) {
  return smem_of(geometry_of(c, r, L, 1u), c, r, L);
}

// What a persistent CTA of configuration c needs to run every image of
// radius <= max_r and levels <= max_L: the widest halo box and the largest
// histogram area over the one-column path (any image) and, for 2 or 4
// columns per thread, the difference-histogram path (r <= 15, L <= 32).
struct BatchNeeds {
  uint32_t boxw;
  size_t hist;
};

BatchNeeds batch_needs(const op_config_t &c, int max_r, uint32_t max_L) {
  const uint32_t nt = threads_of(c);
  const int k = cols_per_thread(c);
  BatchNeeds n;
  n.boxw = opk::box_width(nt, max_r);
  n.hist = opk::hist_bytes(nt, 1, max_L, opk::variant_for_radius(max_r));
  if (k > 1) {
    const int rd = std::min(max_r, static_cast<int>(opk::kDeltaMaxRadius));
    const uint32_t Ld = std::min(max_L, static_cast<uint32_t>(opk::kDeltaMaxLevels));
    n.boxw = std::max(n.boxw, opk::delta_box_width(nt, k, rd));
    // the largest delta histogram over the radii a batch may hold
    n.hist = std::max(n.hist, opk::hist_bytes(nt, k, Ld, opk::variant_for_radius(rd)));
    n.hist = std::max(n.hist, opk::hist_bytes(nt, k, Ld, opk::kVarA));
  }
  return n;
}

size_t batch_smem(const op_config_t &c, const BatchNeeds &n) {
  return opk::tile_smem_bytes(n.hist, opk::make_ring(0, c.chunk_rows, c.prefetch, n.boxw));
}

// Range checks plus "runs as asked and fits one CTA" for radius r, L levels.
int check_config(const op_config_t &c, int r, uint32_t L, const DevInfo &di) {
  if (!config_in_range(c)) return OP_E_INVALID;
  const opk::Geometry g = geometry_of(c, r, L, 1u);
  // the path and columns asked for must apply (K columns and the column
  // histograms need L <= 32, the straight-line path its radius range)
  const int want_path = (c.path == 0u && cols_per_thread(c) == 8) ? 3 : static_cast<int>(c.path);
  if (g.path != want_path || g.kcols != cols_per_thread(c)) return OP_E_UNSUPPORTED;
  if (g.boxw > opk::kMaxBoxWords) return OP_E_UNSUPPORTED;
  if (smem_of(g, c, r, L) > di.smem_optin - 1024u) return OP_E_UNSUPPORTED;
  return OP_OK;
}

// Built-in default: the direct path at radius 1 and 2 with many levels, else
// the first of a preference list that runs and whose shared
// memory leaves room for >= 2 CTAs per SM, one halo chunk in flight: the
// straight-line difference histograms (64 threads x 4 columns, the window
// histogram in one part, 2-row chunks) where they apply (2 <= r <= 15,
// L <= 32), then difference histograms over 4 or 2 columns per thread
// (r <= 44, L <= 32), then one column per thread (8-row chunks).
op_config_t builtin_config(int r, uint32_t L, const DevInfo &di) {
  // The direct path at r = 0 (the pixel itself: 12 MP 0.049 ms against
  // 0.109 ms) and where its cost, independent of L, beats the L-level
  // argmax of the histogram paths (12 MP at r = 1: 0.19 ms against 0.125 ms
  // at L = 20, 0.17 ms at L = 32 and 0.34 ms at L = 64; at r = 2: 0.80 ms
  // against 0.67 ms at L = 128 and 1.50 ms at L = 256).
  if (r == 0 || (r == 1 && L > 40u) || (r == 2 && L > 150u)) {
    const op_config_t c = {64, 0, 8, 1, 1, 4};  // 64 threads, 8-row chunks, 1 in flight
    if (check_config(c, r, L, di) == OP_OK) return c;
  }
  // threads, columns per thread, path, halo chunk rows
  static const uint32_t prefs[][4] = {{64, 4, 2, 2}, {32, 4, 0, 8}, {64, 2, 0, 8}, {128, 1, 0, 8},
                                      {96, 1, 0, 8},  {64, 1, 0, 8}, {32, 1, 0, 8}};
  for (const auto &p : prefs) {
    op_config_t c = {p[0] * p[1], 0, p[3], 1, p[1], p[2]};
    if (check_config(c, r, L, di) != OP_OK) continue;
    if (smem_for(c, r, L) * 2 <= di.smem_optin) return c;
  }
  return op_config_t{32, 0, 4, 1, 1, 0};
}

int pick_config(int r, uint32_t L, const DevInfo &di, op_config_t *out) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({r, L});
    if (it != g_tune.end() && check_config(it->second, r, L, di) == OP_OK) {
      *out = it->second;
      return OP_OK;
    }
  }
  *out = builtin_config(r, L, di);
  return check_config(*out, r, L, di);
}

uint32_t effective_tile_h(const op_config_t &c, uint32_t w, uint32_t h, int r, uint32_t L,
                          const DevInfo &di) {
  if (c.tile_h) return std::min(c.tile_h, h);
  const opk::Geometry g = geometry_of(c, r, L, w);
  const int occ = std::max(1, opk::geometry_occupancy(g, smem_of(g, c, r, L)));
  return opk::auto_tile_h(h, g.tiles_x, r, static_cast<uint64_t>(occ) * di.sms);
}

bool valid_image(uint32_t w, uint32_t h, uint32_t stride, uint32_t bpp, int32_t r, uint32_t L,
                 uint32_t flags) {
  if (w < 1 || h < 1 || w > OP_MAX_DIM || h > OP_MAX_DIM) return false;
  if (bpp != 3 && bpp != 4) return false;
  if (static_cast<uint64_t>(stride) < static_cast<uint64_t>(w) * bpp) return false;
  if (r < 0 || r > OP_MAX_RADIUS) return false;
  if (L < 1 || L > OP_MAX_LEVELS) return false;
  if (flags & ~(OP_LEVEL_INTDIV3 | OP_LITERAL | OP_FUSED_PACK)) return false;
  if ((flags & OP_LITERAL) && L > OP_LITERAL_MAX_LEVELS) return false;
  return true;
}

uint32_t packed_pitch(uint32_t w) { return (w + 3u) & ~3u; }

bool ranges_overlap(const void *a, const void *b, size_t n) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + n && y < x + n;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return OP_OK;
  return e == cudaErrorMemoryAllocation ? OP_E_NOMEM : OP_E_CUDA;
}

}  // namespace

// ============================================================== single image

struct op_s {
  uint32_t w, h, stride, bpp;
  int32_t r;
  uint32_t L, flags;
  int device;
  DevInfo di;
  op_config_t cfg;
  uint32_t tile_h;  // effective tile height of cfg (auto_tile_h when cfg.tile_h == 0)
  uint32_t ppitch;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  CUtensorMap map;
  bool map_valid = false;
  // tensor maps over the input image for the fused pack, for the last two
  // input pointers (op_run_host_async alternates between two)
  CUtensorMap raw_map[2];
  const void *raw_ptr[2] = {nullptr, nullptr};
  uint32_t raw_next = 0;
  uint32_t *d_err = nullptr;
  cudaEvent_t prof_ev = nullptr;
  // host-buffer path: two staging slots, each an input and an output image,
  // and three internal streams (copy in, filter, copy out) so that
  // consecutive calls overlap one image's copies with another's filter
  struct HostPipe {
    bool ready = false;
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    uint8_t *d_in[2] = {nullptr, nullptr}, *d_out[2] = {nullptr, nullptr};
    cudaEvent_t in_done[2] = {nullptr, nullptr}, run_done[2] = {nullptr, nullptr},
                out_done[2] = {nullptr, nullptr};
    uint32_t next = 0;  // slot of the next call
  } hp;
};

namespace {

void host_pipe_free(op_s::HostPipe &hp) {
  cudaStream_t ss[3] = {hp.s_in, hp.s_run, hp.s_out};
  for (cudaStream_t x : ss)
    if (x) cudaStreamSynchronize(x);
  for (int b = 0; b < 2; ++b) {
    cudaFree(hp.d_in[b]);
    cudaFree(hp.d_out[b]);
    if (hp.in_done[b]) cudaEventDestroy(hp.in_done[b]);
    if (hp.run_done[b]) cudaEventDestroy(hp.run_done[b]);
    if (hp.out_done[b]) cudaEventDestroy(hp.out_done[b]);
  }
  for (cudaStream_t x : ss)
    if (x) cudaStreamDestroy(x);
  hp = op_s::HostPipe();
}

int host_pipe_init(op_s::HostPipe &hp, size_t bytes) {
  if (hp.ready) return OP_OK;
  cudaError_t e = cudaSuccess;
  const unsigned sf = cudaStreamNonBlocking;
  const unsigned ef = cudaEventDisableTiming;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp.s_in, sf);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp.s_run, sf);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp.s_out, sf);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(&hp.d_in[b], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&hp.d_out[b], bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.in_done[b], ef);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.run_done[b], ef);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp.out_done[b], ef);
  }
  if (e != cudaSuccess) {
    host_pipe_free(hp);
    return cuda_status(e);
  }
  hp.ready = true;
  return OP_OK;
}

}  // namespace

extern "C" {

int op_last_error(void) { return g_last_error; }

const char *op_status_string(int status) {
  switch (status) {
    case OP_OK: return "ok";
    case OP_E_INVALID: return "invalid argument";
    case OP_E_CUDA: return "CUDA error";
    case OP_E_NOMEM: return "out of memory";
    case OP_E_TIMEOUT: return "device wait timed out";
    case OP_E_UNSUPPORTED: return "unsupported configuration";
    case OP_E_BOUNDS: return "bounds check failed (checked build)";
    default: return "unknown status";
  }
}

op_t *op_create_ex(uint32_t width, uint32_t height, uint32_t stride, uint32_t bpp, int32_t radius,
                   uint32_t levels, uint32_t flags) {
  if (!valid_image(width, height, stride, bpp, radius, levels, flags)) {
    g_last_error = OP_E_INVALID;
    return nullptr;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    g_last_error = OP_E_CUDA;
    return nullptr;
  }
  DevInfo di;
  int st = device_info(dev, &di);
  if (st != OP_OK) {
    g_last_error = st;
    return nullptr;
  }
  op_config_t cfg;
  st = pick_config(radius, levels, di, &cfg);
  if (st != OP_OK) {
    g_last_error = st;
    return nullptr;
  }
  op_t *op = new (std::nothrow) op_t();
  if (!op) {
    g_last_error = OP_E_NOMEM;
    return nullptr;
  }
  op->w = width;
  op->h = height;
  op->stride = stride;
  op->bpp = bpp;
  op->r = radius;
  op->L = levels;
  op->flags = flags;
  op->device = dev;
  op->di = di;
  op->cfg = cfg;
  op->tile_h = effective_tile_h(op->cfg, width,
                                std::max(1u, opk::output_window(width, height, radius, flags).rows()),
                                radius, levels, di);
  op->ppitch = packed_pitch(width);
  if (cudaMalloc(&op->d_err, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(op->d_err, 0, sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(op->d_err);
    delete op;
    g_last_error = OP_E_NOMEM;
    return nullptr;
  }
  g_last_error = OP_OK;
  return op;
}

op_t *op_create(uint32_t width, uint32_t height, uint32_t stride, int32_t radius,
                uint32_t levels) {
  const uint32_t bpp =
      (static_cast<uint64_t>(stride) >= 4ull * width && stride % 4u == 0) ? 4u : 3u;
  return op_create_ex(width, height, stride, bpp, radius, levels, OP_LEVEL_PAPER);
}

int op_get_config(const op_t *op, op_config_t *cfg) {
  if (!op || !cfg) return OP_E_INVALID;
  *cfg = op->cfg;
  return OP_OK;
}

int op_set_config(op_t *op, const op_config_t *cfg) {
  if (!op || !cfg) return OP_E_INVALID;
  const int st = check_config(*cfg, op->r, op->L, op->di);
  if (st != OP_OK) return st;
  op->cfg = *cfg;
  op->tile_h = effective_tile_h(
      op->cfg, op->w, std::max(1u, opk::output_window(op->w, op->h, op->r, op->flags).rows()),
      op->r, op->L, op->di);
  op->map_valid = false;
  op->raw_ptr[0] = op->raw_ptr[1] = nullptr;
  return OP_OK;
}

int op_default_config(int32_t radius, uint32_t levels, op_config_t *cfg) {
  if (!cfg || radius < 0 || radius > OP_MAX_RADIUS || levels < 1 || levels > OP_MAX_LEVELS)
    return OP_E_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OP_E_CUDA;
  DevInfo di;
  const int st = device_info(dev, &di);
  if (st != OP_OK) return st;
  return pick_config(radius, levels, di, cfg);
}

int op_tune_table_set(int32_t radius, uint32_t levels, const op_config_t *cfg) {
  if (!cfg || radius < 0 || radius > OP_MAX_RADIUS || levels < 1 || levels > OP_MAX_LEVELS)
    return OP_E_INVALID;
  if (!config_in_range(*cfg)) return OP_E_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[{radius, levels}] = *cfg;
  return OP_OK;
}

int op_batch_tune_table_set(int32_t max_radius, uint32_t max_levels, const op_config_t *cfg) {
  if (max_radius < 0 || max_radius > OP_MAX_RADIUS || max_levels < 1 ||
      max_levels > OP_MAX_LEVELS)
    return OP_E_INVALID;
  if (cfg && (!config_in_range(*cfg) || cfg->path != 0u)) return OP_E_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (cfg)
    g_batch_tune[{max_radius, max_levels}] = *cfg;
  else
    g_batch_tune.erase({max_radius, max_levels});
  return OP_OK;
}

size_t op_workspace_size(const op_t *op) {
  if (!op) return 0;
  return static_cast<size_t>(op->ppitch) * op->h * 4u;
}

int op_set_workspace(op_t *op, void *d_ws, size_t bytes) {
  if (!op || !d_ws || bytes < op_workspace_size(op) || (reinterpret_cast<uintptr_t>(d_ws) & 15u))
    return OP_E_INVALID;
  if (op->ws_owned) cudaFree(op->ws);
  op->ws = d_ws;
  op->ws_bytes = bytes;
  op->ws_owned = false;
  op->map_valid = false;
  op->raw_ptr[0] = op->raw_ptr[1] = nullptr;
  return OP_OK;
}

static int ensure_workspace(op_t *op) {
  if (op->ws) return OP_OK;
  void *p = nullptr;
  const cudaError_t e = cudaMalloc(&p, op_workspace_size(op));
  if (e != cudaSuccess) return cuda_status(e);
  op->ws = p;
  op->ws_bytes = op_workspace_size(op);
  op->ws_owned = true;
  op->map_valid = false;
  op->raw_ptr[0] = op->raw_ptr[1] = nullptr;
  return OP_OK;
}

int op_run(op_t *op, const uint8_t *d_in, uint8_t *d_out, void *stream) {
  NvtxRange nvtx("op_run");
  if (!op || !d_in || !d_out) return OP_E_INVALID;
  const size_t bytes = static_cast<size_t>(op->h) * op->stride;
  if (ranges_overlap(d_in, d_out, bytes)) return OP_E_INVALID;
  const op_config_t &c = op->cfg;
  const opk::Geometry g = geometry_of(c, op->r, op->L, op->w);
  // Fused pack (OP_FUSED_PACK): the filter's copies read the input pixels
  // themselves (the map over the input is encoded once per input pointer)
  // and the packed workspace is not needed.
  const CUtensorMap *map = &op->map;
  bool fused = op->bpp == 4 && (op->flags & OP_FUSED_PACK) && op->stride % 16u == 0u &&
               reinterpret_cast<uintptr_t>(d_in) % 16u == 0u;
  if (fused) {
    int k = op->raw_ptr[0] == d_in ? 0 : op->raw_ptr[1] == d_in ? 1 : -1;
    if (k < 0) {
      k = static_cast<int>(op->raw_next);
      op->raw_next ^= 1u;
      op->raw_ptr[k] = nullptr;
      if (opk::encode_word_map(&op->raw_map[k], d_in, op->w, op->h, op->stride, g.boxw,
                               c.chunk_rows))
        op->raw_ptr[k] = d_in;
      else
        k = -1;  // the driver refused this map: run the prepass instead
    }
    fused = k >= 0;
    if (fused) map = &op->raw_map[k];
  }
  if (!fused) {
    const int st = ensure_workspace(op);
    if (st != OP_OK) return st;
    if (!op->map_valid) {
      if (!opk::encode_packed_map(&op->map, static_cast<const uint32_t *>(op->ws), op->w, op->h,
                                  op->ppitch, g.boxw, c.chunk_rows))
        return OP_E_CUDA;
      op->map_valid = true;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ImgDesc d{};
  d.in = d_in;
  d.out = d_out;
  d.packed = static_cast<uint32_t *>(op->ws);
  d.tmap = nullptr;
  d.w = op->w;
  d.h = op->h;
  d.stride = op->stride;
  d.ostride = op->stride;
  d.bpp = op->bpp;
  d.r = op->r;
  d.L = op->L;
  d.mode = op->flags & (OP_LEVEL_INTDIV3 | OP_LITERAL);
  d.fused = fused ? 1u : 0u;
  d.ppitch = op->ppitch;
  d.tiles_x = g.tiles_x;
  d.tile_h = op->tile_h;
  d.boxw = g.boxw;
  d.variant = static_cast<uint32_t>(g.variant);
  d.kcols = static_cast<uint32_t>(g.kcols);
  d.xshift = g.xshift;
  d.fmt = g.fmt;
  d.path = static_cast<uint32_t>(g.path);
  const opk::Window win = opk::output_window(op->w, op->h, op->r, op->flags);
  opk::set_window(d, win);
  if (win.rows() == 0u) return OP_OK;  // literal mode: no pixel is r from every edge
  const RingCfg rc = opk::make_ring(op->r, c.chunk_rows, c.prefetch, g.boxw);
  const size_t smem = smem_of(g, c, op->r, op->L);
  cudaError_t e;
  if (!fused) {
    e = opk::launch_pack_single(d, opk::pack_grid_for(op->h, op->di.sms), s);
    if (e != cudaSuccess) return OP_E_CUDA;
  }
  if (op->prof_ev && cudaEventRecord(op->prof_ev, s) != cudaSuccess) return OP_E_CUDA;
  const dim3 grid(d.tiles_x, (win.rows() + d.tile_h - 1) / d.tile_h);
  e = opk::launch_tile(g.nt, g.kcols, g.variant, d, *map, rc, grid, smem, op->d_err,
                       kWaitTimeoutNs, s);
  return e == cudaSuccess ? OP_OK : OP_E_CUDA;
}

int op_run_host_async(op_t *op, const uint8_t *h_in, uint8_t *h_out, void *stream) {
  NvtxRange nvtx("op_run_host_async");
  if (!op || !h_in || !h_out) return OP_E_INVALID;
  const size_t bytes = static_cast<size_t>(op->h) * op->stride;
  if (ranges_overlap(h_in, h_out, bytes)) return OP_E_INVALID;
  op_s::HostPipe &hp = op->hp;
  int st = host_pipe_init(hp, bytes);
  if (st != OP_OK) return st;
  const uint32_t b = hp.next;
  hp.next ^= 1u;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t row = static_cast<size_t>(op->w) * op->bpp;
  // slot b's input may be overwritten once the filter that read it is done,
  // its output once the copy that read it is done; events never recorded
  // yet are complete
  if (cudaStreamWaitEvent(hp.s_in, hp.run_done[b], 0) != cudaSuccess ||
      cudaMemcpyAsync(hp.d_in[b], h_in, bytes, cudaMemcpyHostToDevice, hp.s_in) != cudaSuccess ||
      cudaEventRecord(hp.in_done[b], hp.s_in) != cudaSuccess ||
      cudaStreamWaitEvent(hp.s_run, hp.in_done[b], 0) != cudaSuccess ||
      cudaStreamWaitEvent(hp.s_run, hp.out_done[b], 0) != cudaSuccess)
    return OP_E_CUDA;
  st = op_run(op, hp.d_in[b], hp.d_out[b], hp.s_run);
  if (st != OP_OK) return st;
  if (cudaEventRecord(hp.run_done[b], hp.s_run) != cudaSuccess ||
      cudaStreamWaitEvent(hp.s_out, hp.run_done[b], 0) != cudaSuccess ||
      cudaMemcpy2DAsync(h_out, op->stride, hp.d_out[b], op->stride, row, op->h,
                        cudaMemcpyDeviceToHost, hp.s_out) != cudaSuccess ||
      cudaEventRecord(hp.out_done[b], hp.s_out) != cudaSuccess ||
      cudaStreamWaitEvent(s, hp.out_done[b], 0) != cudaSuccess)
    return OP_E_CUDA;
  return OP_OK;
}

int op_run_host(op_t *op, const uint8_t *h_in, uint8_t *h_out, void *stream) {
  const int st = op_run_host_async(op, h_in, h_out, stream);
  if (st != OP_OK) return st;
  return op_sync_status(op, stream);
}

int op_set_profile_event(op_t *op, void *event) {
  if (!op) return OP_E_INVALID;
  op->prof_ev = static_cast<cudaEvent_t>(event);
  return OP_OK;
}

int op_sync_status(op_t *op, void *stream) {
  if (!op) return OP_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return OP_E_CUDA;
  uint32_t err = 0;
  if (cudaMemcpy(&err, op->d_err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
    return OP_E_CUDA;
  if (err) {
    if (cudaMemset(op->d_err, 0, sizeof(err)) != cudaSuccess) return OP_E_CUDA;
    return OP_E_TIMEOUT;
  }
  uint32_t bits = 0;
  if (opk::take_check_error(&bits) != cudaSuccess) return OP_E_CUDA;
  return bits ? OP_E_BOUNDS : OP_OK;
}

int op_destroy(op_t *op) {
  if (!op) return OP_OK;
  if (op->ws_owned) cudaFree(op->ws);
  host_pipe_free(op->hp);
  cudaFree(op->d_err);
  delete op;
  return OP_OK;
}

}  // extern "C"

// ============================================================== batch

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct op_batch_s {
  uint32_t max_images;
  uint64_t max_pixels;
  int32_t max_r;
  uint32_t max_L;
  int device;
  DevInfo di;
  // Images are split by radius (above 15: variant-B bins) and by level count
  // (above kBatchLevelSplit: larger histograms) into up to four groups.  Each
  // group is one persistent launch with its own configuration, shared-memory
  // size, grid, ticket queue and table segment, so images with small
  // histograms are not held to the occupancy of the largest ones.  Groups
  // other than the first run on side streams forked from the caller's, the
  // costliest first, so the cheaper groups fill the tails of the others.
  bool split_r = false, split_L = false;
  int groups = 1;
  int32_t group_r[opk::kBatchGroups] = {};
  uint32_t group_L[opk::kBatchGroups] = {};
  op_config_t gcfg[opk::kBatchGroups] = {};
  RingCfg rc[opk::kBatchGroups] = {};
  size_t smem[opk::kBatchGroups] = {};
  int grid_persist[opk::kBatchGroups] = {};
  int grid_pack = 0;
  uint32_t gn[opk::kBatchGroups] = {};
  cudaStream_t side[opk::kBatchGroups - 1] = {};
  cudaEvent_t fork = nullptr, join[opk::kBatchGroups - 1] = {};
  // workspace layout
  size_t off_ctrl, off_hdr, off_descs, off_maps, off_tile_prefix, off_row_prefix, off_packed,
      total;
  size_t stage_bytes;  // hdr .. row_prefix, copied in one transfer
  uint8_t *ws = nullptr;
  bool ws_owned = false;
  bool ctrl_clean = false;
  uint8_t *h_stage = nullptr;  // pinned mirror of [hdr .. row_prefix]
  cudaEvent_t stage_done = nullptr;
  uint32_t n = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;

  int group_of(int32_t r, uint32_t L) const {
    const int rb = split_r && r > opk::kMaxRadiusA ? 1 : 0;
    const int lb = split_L && L > opk::kBatchLevelSplit ? 1 : 0;
    return rb * (split_L ? 2 : 1) + lb;
  }
};

namespace {

// Control block words: [1] error word, [2 .. 2 + kBatchGroups) the groups'
// ticket queues, [8 .. 24) the timeout diagnostic record.
constexpr uint32_t kCtrlWords = 24;
constexpr uint32_t kCtrlQueue = 2;
// Header words: image count of each group, index of its first descriptor,
// index of its first tile-prefix entry, then the batch's image count.
constexpr uint32_t kHdrCount = 0;
constexpr uint32_t kHdrDesc = opk::kBatchGroups;
constexpr uint32_t kHdrPrefix = 2 * opk::kBatchGroups;
constexpr uint32_t kHdrTotal = 3 * opk::kBatchGroups;
constexpr uint32_t kHdrWords = kHdrTotal + 1;

// Whether configuration c runs every image of a group bounded by radius r and
// L levels in one persistent CTA; its shared memory and CTAs per SM if so.
bool batch_group_fits(const op_config_t &c, int32_t r, uint32_t L, const DevInfo &di,
                      size_t *smem, int *occ) {
  if (!config_in_range(c) || c.path != 0u || cols_per_thread(c) > 4) return false;
  const BatchNeeds nd = batch_needs(c, r, L);
  const size_t sm = batch_smem(c, nd);
  if (nd.boxw > opk::kMaxBoxWords || sm > di.smem_optin - 1024u) return false;
  const int o = opk::tile_occupancy(threads_of(c), true, cols_per_thread(c), -1, sm);
  if (o < 1) return false;
  *smem = sm;
  *occ = o;
  return true;
}

}  // namespace

extern "C" {

op_batch_t *op_batch_create(uint32_t max_images, uint64_t max_pixels, int32_t max_radius,
                            uint32_t max_levels, const op_config_t *cfg) {
  if (max_images < 1 || max_images > (1u << 20) || max_pixels < 1 || max_radius < 0 ||
      max_radius > OP_MAX_RADIUS || max_levels < 1 || max_levels > OP_MAX_LEVELS ||
      max_pixels > (1ull << 34)) {
    g_last_error = OP_E_INVALID;
    return nullptr;
  }
  if (cfg && (!config_in_range(*cfg))) {
    g_last_error = OP_E_INVALID;
    return nullptr;
  }
  if (cfg && cfg->path != 0u) {  // the persistent kernel keeps histograms per thread
    g_last_error = OP_E_UNSUPPORTED;
    return nullptr;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    g_last_error = OP_E_CUDA;
    return nullptr;
  }
  DevInfo di;
  int st = device_info(dev, &di);
  if (st != OP_OK) {
    g_last_error = st;
    return nullptr;
  }
  op_batch_t *b = new (std::nothrow) op_batch_t();
  if (!b) {
    g_last_error = OP_E_NOMEM;
    return nullptr;
  }
  b->max_images = max_images;
  b->max_pixels = max_pixels;
  b->max_r = max_radius;
  b->max_L = max_levels;
  b->device = dev;
  b->di = di;
  b->split_r = max_radius > opk::kMaxRadiusA;
  b->split_L = max_levels > opk::kBatchLevelSplit;
  b->groups = (b->split_r ? 2 : 1) * (b->split_L ? 2 : 1);
  for (int rb = 0; rb <= (b->split_r ? 1 : 0); ++rb)
    for (int lb = 0; lb <= (b->split_L ? 1 : 0); ++lb) {
      const int g = rb * (b->split_L ? 2 : 1) + lb;
      b->group_r[g] = rb ? max_radius : std::min(max_radius, int32_t{opk::kMaxRadiusA});
      b->group_L[g] = lb ? max_levels : std::min(max_levels, opk::kBatchLevelSplit);
    }
  for (int g = 0; g < b->groups; ++g) {
    const int32_t r = b->group_r[g];
    const uint32_t L = b->group_L[g];
    size_t sm = 0;
    int occ = 0;
    bool found = false;
    if (cfg) {
      found = batch_group_fits(*cfg, r, L, di, &sm, &occ);
      b->gcfg[g] = *cfg;
    } else {
      // Default: the first that fits a persistent CTA of the batch tuning
      // table's entry for the group's bounds, the single-image table's entry
      // for an image of those bounds, and a preference list (on GB300 the
      // mixed batches ran fastest with 64 threads x 2 columns and 2-row
      // halo chunks where neither table has an entry).
      std::vector<op_config_t> cands;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_batch_tune.find({r, L});
        if (it != g_batch_tune.end()) cands.push_back(it->second);
        it = g_tune.find({r, L});
        if (it != g_tune.end()) cands.push_back(it->second);
      }
      static const uint32_t prefs[][2] = {{64, 2}, {32, 2}, {32, 4}, {64, 1}, {32, 1}};
      for (const auto &p : prefs) cands.push_back(op_config_t{p[0] * p[1], 0, 2, 1, p[1], 0});
      for (op_config_t c : cands) {
        c.tile_h = 0;
        if (batch_group_fits(c, r, L, di, &sm, &occ)) {
          b->gcfg[g] = c;
          found = true;
          break;
        }
      }
    }
    if (!found) {
      delete b;
      g_last_error = OP_E_UNSUPPORTED;
      return nullptr;
    }
    const BatchNeeds nd = batch_needs(b->gcfg[g], r, L);
    b->rc[g] = opk::make_ring(r, b->gcfg[g].chunk_rows, b->gcfg[g].prefetch, nd.boxw);
    b->smem[g] = sm;
    b->grid_persist[g] = occ * di.sms;
  }
  b->grid_pack = 6 * di.sms;  // the pack kernels' resident blocks per SM (launch bounds)
  size_t o = 0;
  b->off_ctrl = o;
  o = align_up(o + kCtrlWords * sizeof(uint32_t), kAlign);
  b->off_hdr = o;
  o = align_up(o + kHdrWords * sizeof(uint32_t), kAlign);
  b->off_descs = o;  // all images, grouped, in run order
  o = align_up(o + static_cast<size_t>(max_images) * sizeof(ImgDesc), kAlign);
  b->off_maps = o;
  o = align_up(o + static_cast<size_t>(max_images) * sizeof(CUtensorMap), kAlign);
  b->off_tile_prefix = o;  // one segment of n_g + 1 entries per group
  o = align_up(o + (static_cast<size_t>(max_images) + opk::kBatchGroups) * sizeof(uint32_t),
               kAlign);
  b->off_row_prefix = o;  // over all images, for the pack kernel
  o = align_up(o + (static_cast<size_t>(max_images) + 1) * sizeof(uint32_t), kAlign);
  b->off_packed = o;
  b->stage_bytes = o - b->off_hdr;
  o = align_up(o + static_cast<size_t>(max_pixels) * 4u + static_cast<size_t>(max_images) * kAlign,
               kAlign);
  b->total = o;
  bool ok = cudaMallocHost(&b->h_stage, b->stage_bytes) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->stage_done, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int g = 1; g < b->groups && ok; ++g)
    ok = cudaStreamCreateWithFlags(&b->side[g - 1], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[g - 1], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    op_batch_destroy(b);
    g_last_error = OP_E_NOMEM;
    return nullptr;
  }
  g_last_error = OP_OK;
  return b;
}

size_t op_batch_workspace_size(const op_batch_t *b) { return b ? b->total : 0; }

int op_batch_get_config(const op_batch_t *b, op_config_t *cfg) {
  if (!b || !cfg) return OP_E_INVALID;
  *cfg = b->gcfg[0];
  cfg->tile_h = 0;
  return OP_OK;
}

int op_batch_group_count(const op_batch_t *b) { return b ? b->groups : OP_E_INVALID; }

int op_batch_get_group(const op_batch_t *b, uint32_t group, op_config_t *cfg,
                       int32_t *max_radius, uint32_t *max_levels) {
  if (!b || group >= static_cast<uint32_t>(b->groups)) return OP_E_INVALID;
  if (cfg) {
    *cfg = b->gcfg[group];
    cfg->tile_h = 0;
  }
  if (max_radius) *max_radius = b->group_r[group];
  if (max_levels) *max_levels = b->group_L[group];
  return OP_OK;
}

int op_batch_set_workspace(op_batch_t *b, void *d_ws, size_t bytes) {
  if (!b || !d_ws || bytes < b->total || (reinterpret_cast<uintptr_t>(d_ws) & (kAlign - 1)))
    return OP_E_INVALID;
  if (b->ws_owned) cudaFree(b->ws);
  b->ws = static_cast<uint8_t *>(d_ws);
  b->ws_owned = false;
  b->ctrl_clean = false;
  if (b->exec) {  // a captured graph points at the old workspace
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  return OP_OK;
}

int op_batch_set(op_batch_t *b, const op_image_t *images, uint32_t n, void *stream) {
  NvtxRange nvtx("op_batch_set");
  if (!b || (n && !images) || n > b->max_images) return OP_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!b->ws) {
    void *p = nullptr;
    const cudaError_t e = cudaMalloc(&p, b->total);
    if (e != cudaSuccess) return cuda_status(e);
    b->ws = static_cast<uint8_t *>(p);
    b->ws_owned = true;
    b->ctrl_clean = false;
  }
  // validate the images and place each in its group
  std::vector<uint32_t> order(n);
  std::vector<int> grp(n);
  std::vector<opk::Geometry> geo(n);
  std::vector<double> tile_cost(n);
  std::vector<uint32_t> tile_h(n);
  uint64_t padded = 0;
  for (uint32_t i = 0; i < n; ++i) {
    const op_image_t &im = images[i];
    const uint32_t ostride = im.out_stride ? im.out_stride : im.stride;
    if (!im.in || !im.out ||
        !valid_image(im.width, im.height, im.stride, im.bpp, im.radius, im.levels, im.flags) ||
        static_cast<uint64_t>(ostride) < static_cast<uint64_t>(im.width) * im.bpp ||
        im.radius > b->max_r || im.levels > b->max_L)
      return OP_E_INVALID;
    // the bytes each image actually spans: (h-1) pitches plus one row of pixels
    const size_t row = static_cast<size_t>(im.width) * im.bpp;
    const uintptr_t ia = reinterpret_cast<uintptr_t>(im.in);
    const uintptr_t oa = reinterpret_cast<uintptr_t>(im.out);
    const size_t in_span = static_cast<size_t>(im.height - 1) * im.stride + row;
    const size_t out_span = static_cast<size_t>(im.height - 1) * ostride + row;
    if (ia < oa + out_span && oa < ia + in_span) return OP_E_INVALID;
    padded += static_cast<uint64_t>(packed_pitch(im.width)) * im.height;
    uint32_t th = 0;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find({im.radius, im.levels});
      if (it != g_tune.end()) th = it->second.tile_h;
    }
    tile_h[i] = th;  // 0: chosen below from the image's share of the GPU
    grp[i] = b->group_of(im.radius, im.levels);
    const op_config_t &c = b->gcfg[grp[i]];
    geo[i] = opk::image_geometry(0, threads_of(c), cols_per_thread(c), im.radius, im.levels,
                                 im.width);
    order[i] = i;
  }
  if (padded > b->max_pixels) return OP_E_INVALID;
  // Tile heights: an image gets its pixel share of its group's resident
  // CTAs (two waves' worth when the group holds several images, so that the
  // ticket queue can balance them; one for a lone image) and the waves model
  // of the single-image path picks its tile height for that many slots.  A
  // lone small request thus spreads over the GPU in short tiles (latency),
  // a large mixed batch keeps tall tiles (less refill per output row).
  {
    double gpix[opk::kBatchGroups] = {};
    uint32_t gnum[opk::kBatchGroups] = {};
    for (uint32_t i = 0; i < n; ++i) {
      gpix[grp[i]] += static_cast<double>(images[i].width) * images[i].height;
      ++gnum[grp[i]];
    }
    for (uint32_t i = 0; i < n; ++i) {
      const op_image_t &im = images[i];
      const uint32_t rows = opk::output_window(im.width, im.height, im.radius, im.flags).rows();
      uint32_t th = tile_h[i];
      if (th == 0) {
        const int g = grp[i];
        const double share = static_cast<double>(im.width) * im.height / gpix[g] *
                             b->grid_persist[g] * (gnum[g] > 1 ? 2.0 : 1.0);
        th = opk::auto_tile_h(std::max(1u, rows), geo[i].tiles_x, im.radius,
                         std::max<uint64_t>(1u, static_cast<uint64_t>(share)));
      }
      th = std::max(1u, std::min(th, rows));
      tile_h[i] = th;
      // per step a tile slides one window column (4r + 2 bin updates) and
      // K - 1 difference columns (4 each); per output row it scans K argmaxes
      const double r = im.radius, k = geo[i].kcols;
      tile_cost[i] = (th + 2.0 * r) * (4.0 * r + 2.0 + 4.0 * (k - 1.0)) +
                     th * k * (im.levels + 10.0);
    }
  }
  // grouped, most expensive tiles first within a group
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) {
    return grp[a] != grp[c] ? grp[a] < grp[c] : tile_cost[a] > tile_cost[c];
  });
  // the previous op_batch_set's copy must have left the pinned staging buffer
  if (cudaEventSynchronize(b->stage_done) != cudaSuccess) return OP_E_CUDA;
  auto host = [&](size_t off) { return b->h_stage + (off - b->off_hdr); };
  uint32_t *hdr = reinterpret_cast<uint32_t *>(host(b->off_hdr));
  ImgDesc *hd = reinterpret_cast<ImgDesc *>(host(b->off_descs));
  CUtensorMap *hm = reinterpret_cast<CUtensorMap *>(host(b->off_maps));
  uint32_t *htp = reinterpret_cast<uint32_t *>(host(b->off_tile_prefix));
  uint32_t *hrp = reinterpret_cast<uint32_t *>(host(b->off_row_prefix));
  const CUtensorMap *dmaps = reinterpret_cast<const CUtensorMap *>(b->ws + b->off_maps);
  size_t poff = b->off_packed;
  uint64_t rows = 0;
  uint32_t k = 0;
  for (int g = 0; g < opk::kBatchGroups; ++g) {
    const uint32_t first = k;
    uint64_t tiles = 0;
    for (; k < n && grp[order[k]] == g; ++k) {
      const uint32_t i = order[k];
      const op_image_t &im = images[i];
      ImgDesc d{};
      d.in = im.in;
      d.out = im.out;
      d.packed = reinterpret_cast<uint32_t *>(b->ws + poff);
      d.tmap = dmaps + k;
      d.w = im.width;
      d.h = im.height;
      d.stride = im.stride;
      d.ostride = im.out_stride ? im.out_stride : im.stride;
      d.bpp = im.bpp;
      d.r = im.radius;
      d.L = im.levels;
      d.mode = im.flags & (OP_LEVEL_INTDIV3 | OP_LITERAL);
      d.ppitch = packed_pitch(im.width);
      d.tile_h = tile_h[i];
      const opk::Geometry &ge = geo[i];
      d.tiles_x = ge.tiles_x;
      d.boxw = ge.boxw;
      d.variant = static_cast<uint32_t>(ge.variant);
      d.kcols = static_cast<uint32_t>(ge.kcols);
      d.xshift = ge.xshift;
      d.fmt = ge.fmt;
      d.path = 0u;
      const opk::Window win = opk::output_window(d.w, d.h, d.r, d.mode);
      opk::set_window(d, win);
      if (!opk::encode_packed_map(&hm[k], d.packed, d.w, d.h, d.ppitch, d.boxw, b->rc[g].ch))
        return OP_E_CUDA;
      hd[k] = d;
      htp[k + g] = static_cast<uint32_t>(tiles);
      hrp[k] = static_cast<uint32_t>(rows);
      tiles += static_cast<uint64_t>(d.tiles_x) * ((win.rows() + d.tile_h - 1) / d.tile_h);
      rows += d.h;
      poff = align_up(poff + static_cast<size_t>(d.ppitch) * d.h * 4u, kAlign);
    }
    if (tiles >= 0xFFFFFFFFull) return OP_E_INVALID;
    htp[k + g] = static_cast<uint32_t>(tiles);  // the segment's end
    hdr[kHdrCount + g] = k - first;
    hdr[kHdrDesc + g] = first;
    hdr[kHdrPrefix + g] = first + g;
    b->gn[g] = k - first;
  }
  if (k != n || poff > b->total || rows >= 0xFFFFFFFFull) return OP_E_INVALID;
  hrp[n] = static_cast<uint32_t>(rows);
  hdr[kHdrTotal] = n;
  if (!b->ctrl_clean) {
    if (cudaMemsetAsync(b->ws + b->off_ctrl, 0, kCtrlWords * sizeof(uint32_t), s) != cudaSuccess)
      return OP_E_CUDA;
    b->ctrl_clean = true;
  }
  if (cudaMemcpyAsync(b->ws + b->off_hdr, b->h_stage, b->stage_bytes, cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaEventRecord(b->stage_done, s) != cudaSuccess)
    return OP_E_CUDA;
  b->n = n;
  return OP_OK;
}

int op_batch_run(op_batch_t *b, void *stream) {
  NvtxRange nvtx("op_batch_run");
  if (!b || !b->ws) return OP_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t *ctrl = reinterpret_cast<uint32_t *>(b->ws + b->off_ctrl);
  const uint32_t *hdr = reinterpret_cast<const uint32_t *>(b->ws + b->off_hdr);
  const ImgDesc *descs = reinterpret_cast<const ImgDesc *>(b->ws + b->off_descs);
  const uint32_t *tp = reinterpret_cast<const uint32_t *>(b->ws + b->off_tile_prefix);
  const uint32_t *rp = reinterpret_cast<const uint32_t *>(b->ws + b->off_row_prefix);
  // Fixed grids; the image counts and the tables are read from device
  // memory, so the launches do not depend on the current batch and a
  // captured graph stays valid across op_batch_set calls.  (Packing each
  // group on its own stream, overlapping the other groups' filters, measured
  // no faster on the 64-image batch and less steady.)
  if (opk::launch_pack_batch(descs, rp, hdr + kHdrTotal, ctrl + kCtrlQueue, opk::kBatchGroups,
                             b->grid_pack, s) != cudaSuccess)
    return OP_E_CUDA;
  auto launch = [&](int g, cudaStream_t st) {
    const op_config_t &c = b->gcfg[g];
    return opk::launch_persistent(threads_of(c), cols_per_thread(c), descs, tp, hdr + g,
                                  ctrl + kCtrlQueue + g, b->rc[g], b->group_L[g],
                                  b->grid_persist[g], b->smem[g], ctrl + 1, kWaitTimeoutNs, st);
  };
  if (b->groups > 1 && cudaEventRecord(b->fork, s) != cudaSuccess) return OP_E_CUDA;
  // the costlier groups (larger radius, then more levels) first, each on its
  // side stream
  for (int g = b->groups - 1; g >= 1; --g) {
    cudaStream_t st = b->side[g - 1];
    if (cudaStreamWaitEvent(st, b->fork, 0) != cudaSuccess || launch(g, st) != cudaSuccess ||
        cudaEventRecord(b->join[g - 1], st) != cudaSuccess)
      return OP_E_CUDA;
  }
  if (launch(0, s) != cudaSuccess) return OP_E_CUDA;
  for (int g = 1; g < b->groups; ++g)
    if (cudaStreamWaitEvent(s, b->join[g - 1], 0) != cudaSuccess) return OP_E_CUDA;
  return OP_OK;
}

int op_batch_capture(op_batch_t *b, void *stream) {
  if (!b || !b->ws) return OP_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return OP_E_CUDA;
  const int st = op_batch_run(b, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != OP_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != OP_OK ? st : OP_E_CUDA;
  }
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    b->exec = nullptr;
    return OP_E_CUDA;
  }
  b->graph = g;
  return OP_OK;
}

int op_batch_launch_graph(op_batch_t *b, void *stream) {
  NvtxRange nvtx("op_batch_launch_graph");
  if (!b || !b->exec) return OP_E_INVALID;
  return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? OP_OK
                                                                                      : OP_E_CUDA;
}

int op_batch_sync_status(op_batch_t *b, void *stream) {
  if (!b || !b->ws) return OP_E_INVALID;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return OP_E_CUDA;
  uint32_t err = 0;
  uint32_t *d_err = reinterpret_cast<uint32_t *>(b->ws + b->off_ctrl) + 1;
  if (cudaMemcpy(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
    return OP_E_CUDA;
  if (err) {
    if (cudaMemset(d_err, 0, sizeof(err)) != cudaSuccess) return OP_E_CUDA;
    return OP_E_TIMEOUT;
  }
  uint32_t bits = 0;
  if (opk::take_check_error(&bits) != cudaSuccess) return OP_E_CUDA;
  return bits ? OP_E_BOUNDS : OP_OK;
}

int op_batch_destroy(op_batch_t *b) {
  if (!b) return OP_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int g = 0; g < opk::kBatchGroups - 1; ++g) {
    if (b->side[g]) {
      cudaStreamSynchronize(b->side[g]);
      cudaStreamDestroy(b->side[g]);
    }
    if (b->join[g]) cudaEventDestroy(b->join[g]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->stage_done) cudaEventDestroy(b->stage_done);
  if (b->ws_owned) cudaFree(b->ws);
  cudaFreeHost(b->h_stage);
  delete b;
  return OP_OK;
}

int op_selftest_wait_timeout(uint64_t timeout_ns, void *stream) {
  if (timeout_ns < 1 || timeout_ns > 2000000000ull) return OP_E_INVALID;
  uint32_t *d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(uint32_t)) != cudaSuccess) return OP_E_NOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = OP_OK;
  if (cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s) != cudaSuccess ||
      opk::launch_selftest_wait(d_err, timeout_ns, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    st = OP_E_CUDA;
  } else {
    uint32_t err = 0;
    if (cudaMemcpy(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = OP_E_CUDA;
    else if (err & opk::kErrTimeout)
      st = OP_E_TIMEOUT;
  }
  cudaFree(d_err);
  return st;
}

}  // extern "C"
