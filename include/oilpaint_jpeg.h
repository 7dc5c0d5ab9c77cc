/*
 * oilpaint_jpeg.h -- JPEG in, oil-paint filter, JPEG out, on the GPU.
 *
 * The paper's application (section 3) wraps its filter between a JPEG decoder
 * and encoder: `Decode` turns a JPEG file into a pixel buffer with its width,
 * height and row stride (section 3.2, "Decoder"), `Encode` writes a buffer back
 * as a JPEG file ("Encoder"), and `ApplyOilPaintOnFile` runs decode, filter and
 * encode in turn and logs the time of each phase ("Application of Image
 * Filter").  This library is that pipeline with the decoder and encoder on the
 * GPU (NVIDIA nvJPEG) and the filter run through op_create_ex / op_run of
 * oilpaint.h, so a decoded image never leaves device memory:
 *
 *   JPEG bytes (host) --nvJPEG decode--> RGB (device, 3 bytes per pixel,
 *   interleaved, rows `pitch` bytes apart) --op_run--> filtered RGB (device)
 *   --nvJPEG encode--> JPEG bytes (host)
 *
 * The library is liboilpaint_jpeg.so, built beside liboilpaint.so when the
 * toolkit has nvJPEG; it links both.  The filter's arithmetic, arguments and
 * edge rules are those of op_create_ex (radius, levels, flags as there); the
 * pixel order is R, G, B, which the filter treats like the paper's
 * B, G, R buffer (the level uses the channel sum, and the means are per
 * channel).
 *
 * Conventions (as oilpaint.h):
 *   - calls return OP_OK (0) or a negative status: the OP_E_* codes of
 *     oilpaint.h plus OP_E_CODEC and OP_E_NOSPACE below; nothing aborts;
 *   - pointers named d_* are device pointers; JPEG byte buffers are host
 *     memory (pageable or pinned);
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that return encoded bytes or a timing synchronise that
 *     stream before they return; op_jpeg_decode does not (its device work is
 *     queued on `stream`, the host-side parse is done when it returns), but
 *     a decode first waits for the device work of the context's previous
 *     decode, whose staging buffers it reuses.  Every decode in this library
 *     follows that rule, op_jpeg_filter's and op_jpeg_filter_batch's
 *     included.
 *   - one op_jpeg_t serves one host thread at a time.
 */
#ifndef OILPAINT_JPEG_H
#define OILPAINT_JPEG_H

#include <stddef.h>
#include <stdint.h>

#include "oilpaint.h"

#ifdef __cplusplus
extern "C" {
#endif

#define OP_E_CODEC (-7)   /* nvJPEG rejected the stream (not a JPEG, truncated,
                             an unsupported coding) or failed to encode */
#define OP_E_NOSPACE (-8) /* the output byte buffer is too small; *out_bytes
                             holds the size needed */

/* Chroma subsampling of the encoded output (the values of nvJPEG's
 * nvjpegChromaSubsampling_t). */
#define OP_JPEG_CSS_444 0
#define OP_JPEG_CSS_422 1
#define OP_JPEG_CSS_420 2

typedef struct op_jpeg op_jpeg_t;

/* Per-phase device times of the last op_jpeg_filter / op_jpeg_filter_file /
 * op_jpeg_filter_batch call, in milliseconds, from CUDA events recorded on its stream around each
 * phase (the counterpart of the paper's decode / process / encode tick counts
 * in ApplyOilPaintOnFile).  decode_ms includes the host-side parse nvJPEG does
 * inside the decode call, because the events bracket the call. */
typedef struct {
    float decode_ms;
    float filter_ms;
    float encode_ms;
} op_jpeg_timing_t;

/* Create a codec context on the current device: an nvJPEG handle, decode and
 * encode states and encoder parameters.  NULL on failure; op_jpeg_last_error()
 * then gives OP_E_CODEC (nvJPEG could not be initialised) or OP_E_NOMEM.
 * `stream` only orders the encoder's setup work. */
op_jpeg_t *op_jpeg_create(void *stream);

/* Status of the last op_jpeg_create on this host thread. */
int op_jpeg_last_error(void);

/* Width, height and component count (1 or 3) of a JPEG stream, read from its
 * headers.  Each output pointer may be NULL.  OP_E_INVALID for NULL data or
 * zero length, OP_E_CODEC if the headers do not parse. */
int op_jpeg_info(op_jpeg_t *jp, const uint8_t *data, size_t len, uint32_t *width,
                 uint32_t *height, uint32_t *components);

/* Decode a JPEG stream into interleaved RGB at d_rgb (height rows of
 * `pitch` bytes, pitch >= 3 * width; bytes past 3 * width in a row are not
 * written).  A grayscale stream decodes to R = G = B.  OP_E_INVALID for a
 * NULL pointer or a pitch below 3 * width, OP_E_CODEC if nvJPEG rejects the
 * stream. */
int op_jpeg_decode(op_jpeg_t *jp, const uint8_t *data, size_t len, uint8_t *d_rgb,
                   uint32_t pitch, void *stream);

/* Upper bound on the encoded size of a width x height image at `quality`
 * (1..100) and `sampling` (OP_JPEG_CSS_*), for sizing output buffers. */
int op_jpeg_encode_bound(op_jpeg_t *jp, uint32_t width, uint32_t height, int quality,
                         int sampling, size_t *bytes);

/* Encode interleaved RGB at d_rgb (rows `pitch` bytes apart) as a baseline
 * JPEG at `quality` (1..100) with `sampling`.  The bytes go to out[0..cap);
 * *out_bytes receives their count.  OP_E_NOSPACE if cap is too small (then
 * *out_bytes is the size needed and out is untouched); OP_E_INVALID for bad
 * arguments; OP_E_CODEC if nvJPEG fails.  Synchronises `stream`. */
int op_jpeg_encode(op_jpeg_t *jp, const uint8_t *d_rgb, uint32_t width, uint32_t height,
                   uint32_t pitch, int quality, int sampling, uint8_t *out, size_t cap,
                   size_t *out_bytes, void *stream);

/* The pipeline on byte buffers: decode `in`, filter (radius, levels, flags as
 * op_create_ex), encode at quality / sampling into out[0..cap), count in
 * *out_bytes.  If d_filtered is not NULL the filtered RGB is written there
 * (rows of filtered_pitch >= 3 * width bytes) and encoded from there;
 * otherwise the context's own device buffers are used (kept and grown across
 * calls; the filter handle is kept while the image size and parameters stay
 * the same).  Returns the first failing step's status: OP_E_CODEC from
 * decode or encode, the op_create_ex / op_run / op_sync_status status of the
 * filter, OP_E_NOSPACE as op_jpeg_encode.  Synchronises `stream`; the phase
 * times are then available from op_jpeg_last_timing. */
int op_jpeg_filter(op_jpeg_t *jp, const uint8_t *in, size_t in_len, int32_t radius,
                   uint32_t levels, uint32_t flags, int quality, int sampling, uint8_t *out,
                   size_t cap, size_t *out_bytes, uint8_t *d_filtered, uint32_t filtered_pitch,
                   void *stream);

/* ApplyOilPaintOnFile: read the JPEG file in_path, run op_jpeg_filter, write
 * the result to out_path (created or truncated).  OP_E_INVALID if in_path
 * cannot be read or out_path cannot be written; otherwise as op_jpeg_filter. */
int op_jpeg_filter_file(op_jpeg_t *jp, const char *in_path, const char *out_path,
                        int32_t radius, uint32_t levels, uint32_t flags, int quality,
                        int sampling, void *stream);

/* Most images one op_jpeg_filter_batch call takes. */
#define OP_JPEG_MAX_BATCH 64

/* The pipeline over n JPEG streams (section 3.2's ApplyOilPaintOnFile over a
 * set of files): the streams are decoded together, then each image is
 * filtered (radius, levels, flags as op_create_ex) and encoded at quality /
 * sampling in turn.  in[i] (in_len[i] bytes, host) is image i; its encoded
 * result goes to out[i][0..cap[i]) (host) with its length in out_bytes[i],
 * and its status in status[i] (OP_OK, or the first failing step's status as
 * op_jpeg_filter gives it; on OP_E_NOSPACE out_bytes[i] is the size needed).
 *
 * Decoding: the streams nvJPEG's hardware decoder takes (baseline, one scan,
 * not 4:1:0 or 4:1:1 sampling; checked per stream with
 * nvjpegDecodeBatchedSupported) are decoded in one nvjpegDecodeBatched call on
 * the GPU's JPEG decoder engines, the others with the decode of
 * op_jpeg_decode; where the engine is absent, or the batched call fails, every
 * stream takes that decode.  The engine's output was byte-identical to the
 * other decoder's on the streams tested (see the tests).  The hardware
 * context is created by the first call that needs it and kept.
 *
 * Device memory: the decoded images of a call are held together (the sum of
 * height x pitch over the images, pitch = 3 * width rounded up to 16 bytes),
 * in a buffer of the context that is kept and grown across calls.
 *
 * Returns OP_OK when every image succeeded, otherwise the status of the first
 * image that failed (status[] says which; the others are still processed).
 * OP_E_INVALID, with nothing processed and status[] untouched, for a NULL
 * context or array, n = 0, n > OP_JPEG_MAX_BATCH, a quality outside 1..100
 * or an unknown sampling; a NULL in[i] (or a NULL out[i] with cap[i] > 0)
 * fails image i alone, with OP_E_INVALID.  Synchronises `stream`;
 * op_jpeg_last_timing then gives the batch's decode time and the sums of
 * the images' filter and encode times. */
int op_jpeg_filter_batch(op_jpeg_t *jp, uint32_t n, const uint8_t *const *in,
                         const size_t *in_len, int32_t radius, uint32_t levels, uint32_t flags,
                         int quality, int sampling, uint8_t *const *out, const size_t *cap,
                         size_t *out_bytes, int *status, void *stream);

/* Phase times of the last successful op_jpeg_filter / op_jpeg_filter_file /
 * op_jpeg_filter_batch; OP_E_INVALID before the first. */
int op_jpeg_last_timing(const op_jpeg_t *jp, op_jpeg_timing_t *t);

/* Release the context, its device buffers and its filter handle (after
 * synchronising the device).  NULL is accepted. */
int op_jpeg_destroy(op_jpeg_t *jp);

#ifdef __cplusplus
}
#endif

#endif /* OILPAINT_JPEG_H */
