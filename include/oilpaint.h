/*
 * oilpaint.h -- C ABI of the GB300 (sm_103a) histogram oil-paint filter.
 *
 * The filter is the one of section 4 of S. Mukherjee, "Study on performance
 * improvement of oil paint image filter algorithm using Parallel Pattern
 * Library" (arXiv 1405.1020), whose interface there is
 * ApplyOilPaintOnBuffer(in, width, height, intensity_level, radius, out).
 * For every output pixel (x, y):
 *   - each neighbour in the (2r+1) x (2r+1) window centred on (x, y) gets the
 *     intensity level floor((R+G+B) * L / 765), clamped to L-1 (section 4's
 *     ((r+g+b)*intensity_level/3.0)/255 is the same integer for every sum and
 *     every L in 1..256; pure white, the one sum that reaches L, joins the top
 *     level).  OP_LEVEL_INTDIV3 selects floor(floor((R+G+B)/3) * L / 255)
 *     instead, also clamped;
 *   - neighbours outside the image are skipped (the window shrinks at the
 *     border; every pixel of the image is written);
 *   - the level with the largest count wins, the lowest level on a tie;
 *   - each output channel is the truncated mean of that level's pixels.
 * With 4 bytes per pixel the 4th byte is copied from the input pixel.  Bytes
 * between width*bpp and stride in a row are never written.
 *
 * Conventions for every call:
 *   - "device pointer" means memory the CUDA device can address (cudaMalloc,
 *     a torch CUDA tensor's data_ptr(), ...); "host pointer" means ordinary or
 *     pinned host memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); every *_run call is asynchronous on it and never synchronises;
 *   - calls return OP_OK (0) or a negative OP_E_* status; nothing aborts;
 *   - errors found on the device while a kernel runs (a bounded wait that ran
 *     out) set a sticky per-object error word that op_sync_status /
 *     op_batch_sync_status report and clear;
 *   - an op_t or op_batch_t is not thread safe: one host thread at a time.
 *   - the device used is the one current (cudaSetDevice) when the object is
 *     created; calls must be made with that device current.
 */
#ifndef OILPAINT_H
#define OILPAINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define OP_OK 0
#define OP_E_INVALID (-1)     /* bad argument (NULL, size out of range, aliasing, ...) */
#define OP_E_CUDA (-2)        /* a CUDA runtime call or kernel launch failed */
#define OP_E_NOMEM (-3)       /* host or device allocation failed */
#define OP_E_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define OP_E_UNSUPPORTED (-5) /* valid request the library cannot run here (e.g. shared memory) */
#define OP_E_BOUNDS (-6)      /* the bounds-checking build (liboilpaint_checked.so) found
                                 a shared-memory, pixel or TMA access out of range and
                                 skipped it; reported by the sync calls */

/* ---- flags for op_create_ex / op_image_t.flags -------------------------- */
#define OP_LEVEL_PAPER 0u   /* level = min(floor((R+G+B)*L/765), L-1)        (section 4) */
#define OP_LEVEL_INTDIV3 1u /* level = min(floor(floor((R+G+B)/3)*L/255), L-1)          */
/*
 * OP_LITERAL (flag bit, with either level mode): the section-4 listing as
 * printed instead of the default readings.  Only pixels at least `radius`
 * from every edge are written (none when width or height <= 2*radius); the
 * level is not clamped, so pure white (R+G+B = 765) lands on level L, which
 * the argmax (levels 0..L-1) never reads; a pixel whose window has no level
 * below L is not written; only the three colour bytes are written (alpha and
 * the border keep whatever the output buffer held).  Needs
 * levels <= OP_LITERAL_MAX_LEVELS (the listing's arrays hold 255 levels).
 */
#define OP_LITERAL 2u
#define OP_LITERAL_MAX_LEVELS 254u
/*
 * OP_FUSED_PACK (flag bit): no separate pack launch.  For an image of 4 bytes
 * per pixel whose input pointer and stride are multiples of 16 bytes, op_run
 * then runs one launch: the filter's halo copies read the input pixels
 * themselves and each copied chunk is converted to the packed words in
 * shared memory (the same words, so the same output bytes), and the packed
 * workspace is neither allocated nor written.  It saves 4 * width * height
 * bytes of device memory but is slower on GB300 (4000 x 3000, r = 15, L = 20:
 * 0.367 ms per image against 0.287 ms with the prepass; 23-33% slower at
 * r = 1..12): the conversion runs in the filter, which is bound by its
 * shared-memory pipe, for every halo row it copies, entering and leaving.
 * Other images, the batch API and op_run_noalloc ignore the flag.
 */
#define OP_FUSED_PACK 4u

/* ---- limits ------------------------------------------------------------- */
#define OP_MAX_RADIUS 44   /* 255*(2r+1)^2 must fit the 21-bit per-level channel sums */
#define OP_MAX_LEVELS 256  /* levels are stored in 8 bits */
#define OP_MAX_DIM 65535u  /* width and height */

typedef struct op_s op_t;

/*
 * Launch configuration of the filter kernel.  op_create picks it from the
 * tuning table (see op_tune_table_set); the autotuner overrides it.
 *   tile_w          output columns per CTA = threads x cols_per_thread, with
 *                   32, 64, 96 or 128 threads;
 *   tile_h          output rows per CTA (0 = chosen from the image size and
 *                   the number of resident CTAs);
 *   chunk_rows      input rows per TMA halo copy, 1..32;
 *   prefetch        halo copies in flight ahead of the one being consumed, 1..4;
 *   cols_per_thread output columns per thread: 1 (one running histogram of
 *                   the window per output column), 2, 4 or 8 (difference
 *                   histograms: each thread keeps the window histogram H of
 *                   its first column and, for each next column i, the
 *                   histogram D_i of the column entering minus the column
 *                   leaving the window, so the window of column i is
 *                   H + D_1 + ... + D_i; 2(2r+1) + 4(K-1) bin updates per K
 *                   outputs instead of 2(2r+1) per output); 0 = 1.  2, 4 and
 *                   8 need levels <= 32, else the configuration is refused
 *                   (OP_E_UNSUPPORTED) by op_set_config; a batch runs its
 *                   other images on the one-column path.  8 exists only on
 *                   path 3 (path 0 with 8 columns means path 3).
 *   path            0: histograms kept per thread (the fields above);
 *                   1: column histograms with the levels across a warp's
 *                   lanes (Perreault and Hebert's constant-time column
 *                   histograms: work per pixel independent of r): a CTA
 *                   keeps one histogram per image column of its tile and
 *                   halo, each warp sweeps
 *                   32 * cols_per_thread output columns of every row
 *                   (cols_per_thread 1 or 2), tile_w / cols_per_thread =
 *                   32, 64 or 128 threads; needs levels <= 32;
 *                   2 and 3: the difference histograms of 4 or 8 columns
 *                   per thread compiled once per radius (straight-line
 *                   steps), with the counts of D_1 .. D_{K-1} also kept as
 *                   bytes packed into one word per level and per four
 *                   columns, so that the argmax reads two words per level;
 *                   the window histogram in one part (path 2) or split by
 *                   column parity into two (path 3); 32 or 64 threads;
 *                   needs levels <= 32 and K/2 <= radius <= 15 (radius >= 4
 *                   for 8 columns), else OP_E_UNSUPPORTED.  Not for batches;
 *                   4: direct, no histogram (radius 0, 1 or 2, any levels, one
 *                   column per thread, 32..128 threads): each thread keeps
 *                   its window's (2r+1)^2 packed pixels in registers and
 *                   counts their 8-bit levels by pairwise comparison, so the
 *                   work per pixel does not depend on L; other radii are
 *                   refused (OP_E_UNSUPPORTED).  Not for batches.
 * The halo copy of a tile is at most 1024 columns wide (copies wider than
 * 256 columns read the packed image as groups of 4 words): tile_w + 2r + up
 * to 3 columns for one column per thread and for path 1, K * (threads - 1 +
 * ceil((2r+K-1)/K) + 1) rounded up to 4 for K columns per thread.
 */
typedef struct {
  uint32_t tile_w;
  uint32_t tile_h;
  uint32_t chunk_rows;
  uint32_t prefetch;
  uint32_t cols_per_thread;
  uint32_t path;
} op_config_t;

/*
 * op_create -- the 5-argument form (section 4's interface plus the row
 * pitch).  width, height in pixels (1..OP_MAX_DIM); stride = bytes between
 * rows; bytes per pixel are 4 if stride >= 4*width and stride % 4 == 0, else
 * 3; 0 <= radius <= OP_MAX_RADIUS; 1 <= levels <= OP_MAX_LEVELS.  Level mode
 * OP_LEVEL_PAPER.  Returns a handle owned by the caller (free with
 * op_destroy), or NULL with the reason in op_last_error().
 */
op_t *op_create(uint32_t width, uint32_t height, uint32_t stride, int32_t radius, uint32_t levels);

/* op_create_ex -- explicit bytes per pixel (3 or 4, stride >= width*bpp) and
 * flags (OP_LEVEL_PAPER or OP_LEVEL_INTDIV3, optionally | OP_LITERAL).  Otherwise
 * as op_create. */
op_t *op_create_ex(uint32_t width, uint32_t height, uint32_t stride, uint32_t bpp, int32_t radius,
                   uint32_t levels, uint32_t flags);

/* Status of the last op_create / op_create_ex / op_batch_create on this host
 * thread (OP_OK after a success). */
int op_last_error(void);

/* Static, human-readable name of a status code. */
const char *op_status_string(int status);

/* Current launch configuration of `op` into *cfg. */
int op_get_config(const op_t *op, op_config_t *cfg);

/* Replace the launch configuration.  OP_E_INVALID for values out of range,
 * OP_E_UNSUPPORTED if its shared memory does not fit one CTA on this device.
 * The workspace size does not depend on the configuration. */
int op_set_config(op_t *op, const op_config_t *cfg);

/* Configuration op_create would pick for (radius, levels) on the current
 * device: the tuning-table entry if one is set, else the built-in default. */
int op_default_config(int32_t radius, uint32_t levels, op_config_t *cfg);

/* Record a tuned configuration for (radius, levels) in this process's table
 * (read by later op_create / op_batch_set calls).  Not persisted. */
int op_tune_table_set(int32_t radius, uint32_t levels, const op_config_t *cfg);

/* Record a tuned configuration for a batch group whose largest radius and
 * level count are (max_radius, max_levels) (see op_batch_create); read by
 * later op_batch_create calls with cfg NULL, before the single-image table.
 * path must be 0; cfg NULL removes the entry.  Not persisted. */
int op_batch_tune_table_set(int32_t max_radius, uint32_t max_levels, const op_config_t *cfg);

/* Bytes of device workspace op_run needs: the packed-word image of
 * section 4's per-pixel level and colour (one 32-bit word per pixel, rows
 * padded to 16 bytes). */
size_t op_workspace_size(const op_t *op);

/* Give `op` caller-owned device workspace of `bytes` >= op_workspace_size,
 * 16-byte aligned; it must stay valid while runs that use it are in flight.
 * Without it op_run allocates its own on first use (freed by op_destroy);
 * runs that take the fused pack (OP_FUSED_PACK) use none. */
int op_set_workspace(op_t *op, void *d_ws, size_t bytes);

/*
 * op_run -- filter one image, asynchronously on `stream`.  d_in, d_out:
 * device pointers to height*stride bytes each, non-overlapping.  Launches the
 * pack prepass and the tiled filter kernel (the filter alone under
 * OP_FUSED_PACK, where it applies).  OP_E_CUDA if a launch fails.
 */
int op_run(op_t *op, const uint8_t *d_in, uint8_t *d_out, void *stream);

/*
 * op_run_host -- the same filter on host buffers: copies h_in to device
 * memory owned by `op`, runs, copies the result to h_out and synchronises
 * `stream` before returning (op_run_host_async followed by op_sync_status).
 * h_in, h_out: host pointers to height*stride bytes (page-locked memory makes
 * the copies faster and lets them overlap).  Only pixel bytes of h_out are
 * written; its row padding is left untouched.  Device staging memory and
 * three internal streams are created on the first call and freed by
 * op_destroy.
 */
int op_run_host(op_t *op, const uint8_t *h_in, uint8_t *h_out, void *stream);

/*
 * op_run_host_async -- enqueue the host-buffer filter and return.  The copy
 * of h_in, the filter and the copy to h_out run on the op's own streams
 * through one of two staging slots, so consecutive calls pipeline: one
 * image's copies in and out overlap another's filter.  `stream` is made to
 * wait for this call's copy to h_out, so synchronising it (or
 * op_sync_status) waits for the result; h_in is read without waiting for
 * `stream` (host data is ready when the call is made).  h_in and h_out must
 * stay valid, and h_in unchanged, until then; page-locked memory is needed
 * for the copies to be asynchronous.  Not thread-safe per op.
 */
int op_run_host_async(op_t *op, const uint8_t *h_in, uint8_t *h_out, void *stream);

/* Profiling hook: when `event` (a cudaEvent_t passed as void*) is not NULL,
 * every later op_run records it on the run's stream between the pack prepass
 * and the filter kernel, so that events recorded by the caller before and
 * after op_run time the two kernels separately (with OP_FUSED_PACK there is
 * one launch, and the event is recorded just before it).  NULL turns it off.
 * The event stays owned by the caller. */
int op_set_profile_event(op_t *op, void *event);

/* Synchronise `stream`, then report and clear the sticky device error word
 * of `op`: OP_OK, OP_E_TIMEOUT, or OP_E_CUDA if the stream reported an error. */
int op_sync_status(op_t *op, void *stream);

/* Free `op` and everything it allocated.  NULL is accepted.  The caller
 * must make sure no run using it is still in flight. */
int op_destroy(op_t *op);

/* ---- batched, persistent form ------------------------------------------- */

/* One image of a batch.  in/out: device pointers; the input's rows are
 * `stride` bytes apart, the output's `out_stride` bytes apart (0 = stride),
 * so the input may be a strided crop of a larger image and the output packed.
 * The (height-1) pitches plus one row of pixels that each spans must not
 * overlap.  Other fields as op_create_ex. */
typedef struct {
  const uint8_t *in;
  uint8_t *out;
  uint32_t width, height, stride, bpp;
  int32_t radius;
  uint32_t levels;
  uint32_t flags;
  uint32_t out_stride;
} op_image_t;

typedef struct op_batch_s op_batch_t;

/*
 * op_batch_create -- a batch runner for up to `max_images` images holding at
 * most `max_pixels` pixels in total, every radius <= max_radius and level
 * count <= max_levels.  The images of a run are split into up to four
 * groups -- radius above 15 or not (when max_radius > 15), levels above 20
 * or not (when max_levels > 20) -- and each group is one persistent kernel
 * launch whose CTAs take (image, tile) tickets from the group's device-side
 * atomic counter until its queue is empty; the groups' launches run
 * concurrently on streams forked from the caller's.  cfg: tile_w,
 * chunk_rows, prefetch and cols_per_thread of every group's launch (path
 * must be 0); NULL = per group, the first that fits of the batch tuning
 * table's entry for the group's largest radius and level count
 * (op_batch_tune_table_set), the single-image table's entry for them and a
 * built-in default.  tile_h is chosen per image.  With 2 or 4 columns per thread,
 * images of <= 32 levels take the difference-histogram path and the others
 * one column per thread with tile_w / cols_per_thread threads.  Returns NULL
 * with op_last_error() on failure (OP_E_UNSUPPORTED: cfg does not fit a
 * group's largest image in one CTA).
 */
op_batch_t *op_batch_create(uint32_t max_images, uint64_t max_pixels, int32_t max_radius,
                            uint32_t max_levels, const op_config_t *cfg);

/* Launch configuration of the first group's persistent kernel into *cfg
 * (tile_h is 0: it is chosen per image). */
int op_batch_get_config(const op_batch_t *b, op_config_t *cfg);

/* Number of image groups of the batch (1, 2 or 4), or OP_E_INVALID. */
int op_batch_group_count(const op_batch_t *b);

/* Group `group`'s launch configuration and the largest radius and level
 * count it holds (each output pointer may be NULL); OP_E_INVALID if group
 * is out of range. */
int op_batch_get_group(const op_batch_t *b, uint32_t group, op_config_t *cfg,
                       int32_t *max_radius, uint32_t *max_levels);

/* Device workspace a batch needs: descriptors, tensor maps, tile tables and
 * the packed-word images of max_pixels pixels. */
size_t op_batch_workspace_size(const op_batch_t *b);

/* Caller-owned workspace (device pointer, >= op_batch_workspace_size bytes,
 * 256-byte aligned).  Without it the batch allocates its own on first set. */
int op_batch_set_workspace(op_batch_t *b, void *d_ws, size_t bytes);

/*
 * op_batch_set -- describe the images of the next run(s): validates them,
 * builds per-image descriptors, TMA tensor maps and the tile queue on the
 * host, and copies them to the device workspace asynchronously on `stream`.
 * A captured graph (op_batch_capture) reads these device tables, so it stays
 * valid across op_batch_set calls.  n may be 0 (runs then do nothing).
 */
int op_batch_set(op_batch_t *b, const op_image_t *images, uint32_t n, void *stream);

/* Launch the batch's pack kernel and one persistent filter kernel per group
 * (1 + groups launches, fixed grids) on `stream` and, forked from it and
 * joined back into it, the batch's side streams. */
int op_batch_run(op_batch_t *b, void *stream);

/* Capture op_batch_run's launches into a CUDA graph owned by `b` (replacing
 * any earlier one).  `stream` must not be capturing already. */
int op_batch_capture(op_batch_t *b, void *stream);

/* Replay the captured graph on `stream`; OP_E_INVALID if none. */
int op_batch_launch_graph(op_batch_t *b, void *stream);

/* As op_sync_status, for the batch's error word. */
int op_batch_sync_status(op_batch_t *b, void *stream);

/* Free the batch (graph, host staging, owned workspace).  NULL accepted. */
int op_batch_destroy(op_batch_t *b);

/* ---- self-test of the bounded device wait -------------------------------- */

/*
 * op_selftest_wait_timeout -- launches one CTA that waits, through the same
 * bounded mbarrier wait the filter kernels use, on a barrier that nothing
 * completes, with a limit of `timeout_ns` nanoseconds (1..2e9).  The wait
 * gives up, the kernel records OP_E_TIMEOUT in a device word and returns;
 * this call synchronises `stream` and returns that status.  It exercises the
 * error path without faulting or hanging the device.
 */
int op_selftest_wait_timeout(uint64_t timeout_ns, void *stream);

/* ---- allocation-free entry point ------------------------------------------
 * The paper has no counterpart to this call: it exists for callers that
 * cannot allocate device memory -- a plugin inside a host application that
 * owns all device memory through its own pool, code on a latency-critical
 * path that cannot afford the device-wide synchronisation of cudaMalloc and
 * cudaFree, or a process whose free memory another allocator already holds.
 */

/* Words of the fixed scratch array behind op_run_noalloc: 16 MiB, held by
 * every GPU that loads this library until the process exits. */
#define OP_NOALLOC_MAX_WORDS (4u * 1024u * 1024u)

/*
 * op_run_noalloc -- the filter of op_run on one image without allocating:
 * no cudaMalloc, no cudaFree, no allocating library call.  Its packed-word
 * scratch is a file-scope device array of OP_NOALLOC_MAX_WORDS words inside
 * the library, so the image must satisfy ((width + 3) & ~3) * height <=
 * OP_NOALLOC_MAX_WORDS (e.g. 2048 x 2048); larger images return
 * OP_E_UNSUPPORTED.  Other arguments as op_create_ex / op_run; d_in and d_out
 * are device pointers the caller owns (height * stride bytes each).
 * The call is synchronous: it returns after `stream` has completed the work.
 * Returns OP_OK; OP_E_INVALID (a NULL pointer, a size, radius, level count
 * or flag out of range, stride < width * bpp, overlapping buffers);
 * OP_E_UNSUPPORTED (image larger than the array, or no launch configuration
 * fits this device); OP_E_TIMEOUT (a bounded device wait gave up);
 * OP_E_BOUNDS (bounds-checking build only); OP_E_CUDA (a CUDA call failed;
 * the runtime's last error is cleared before returning).
 * The first call on a device (and the first after a cudaDeviceReset) loads
 * the library part that holds the array onto that device: the CUDA runtime
 * then places the 16 MiB array in device memory, so that call needs that
 * much free memory and returns OP_E_CUDA without it.  Make that first call
 * before any stream capture.  Later calls find the array in place and
 * allocate nothing.
 * All calls share the one array and it keeps the last call's contents;
 * calls that overlap on the GPU (other host threads, other streams) race on
 * it and must be serialised by the caller.
 */
int op_run_noalloc(const uint8_t *d_in, uint8_t *d_out, uint32_t width, uint32_t height,
                   uint32_t stride, uint32_t bpp, int32_t radius, uint32_t levels,
                   uint32_t flags, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* OILPAINT_H */
