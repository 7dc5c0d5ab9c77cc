// oilpaint_jpeg.cu -- the decode -> filter -> encode pipeline of section 3.2
// (Decode, ApplyOilPaintOnBuffer, Encode, ApplyOilPaintOnFile) with nvJPEG as
// the codec and the filter run through the C ABI of oilpaint.h.
//
// Host code only: the decoded image stays in device memory between the
// decoder, the filter's pack and tile kernels and the encoder.  Built as
// liboilpaint_jpeg.so, linked against liboilpaint.so and libnvjpeg, so the
// filter library itself does not depend on nvJPEG.

#include <cuda_runtime.h>
#include <nvjpeg.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "oilpaint_jpeg.h"

struct op_jpeg {
    nvjpegHandle_t handle = nullptr;
    nvjpegJpegState_t dec = nullptr;
    // Recorded after each decode with `dec`: the next decode waits for it,
    // because the state's staging buffers are in use until the device work
    // of the decode that filled them has run.
    cudaEvent_t dec_done = nullptr;
    bool dec_pending = false;
    nvjpegEncoderState_t enc = nullptr;
    nvjpegEncoderParams_t params = nullptr;
    // Device RGB buffers of op_jpeg_filter, grown on demand.
    uint8_t *d_in = nullptr;
    size_t in_cap = 0;
    uint8_t *d_out = nullptr;
    size_t out_cap = 0;
    // Filter handle of the last op_jpeg_filter and the arguments it was made for.
    op_t *op = nullptr;
    uint32_t op_w = 0, op_h = 0, op_pitch = 0, op_levels = 0, op_flags = 0;
    int32_t op_radius = 0;
    // Hardware (JPEG engine) decoder of op_jpeg_filter_batch: its own handle,
    // batched state and stream parser, created on first use; hw_ok is 0
    // before that, 1 when created, -1 when the engine is absent.
    nvjpegHandle_t hw = nullptr;
    nvjpegJpegState_t hw_dec = nullptr;
    nvjpegJpegStream_t hw_parse = nullptr;
    int hw_ok = 0;
    int hw_batch = 0;  // batch size the state was initialised for
    // Decoded images of op_jpeg_filter_batch, held together.
    uint8_t *d_batch = nullptr;
    size_t batch_cap = 0;
    // Events bracketing the three phases.
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    op_jpeg_timing_t timing{};
    bool have_timing = false;
};

namespace {

thread_local int g_last_error = OP_OK;

int from_nvjpeg(nvjpegStatus_t s) {
    switch (s) {
    case NVJPEG_STATUS_SUCCESS: return OP_OK;
    case NVJPEG_STATUS_ALLOCATOR_FAILURE: return OP_E_NOMEM;
    case NVJPEG_STATUS_EXECUTION_FAILED: return OP_E_CUDA;
    default: return OP_E_CODEC;
    }
}

int from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return OP_OK;
    cudaGetLastError();  // leave no sticky-looking error for the caller's next check
    return e == cudaErrorMemoryAllocation ? OP_E_NOMEM : OP_E_CUDA;
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

bool valid_sampling(int s) {
    return s == OP_JPEG_CSS_444 || s == OP_JPEG_CSS_422 || s == OP_JPEG_CSS_420;
}

// Image size and component count from the stream's headers.
int read_info(op_jpeg_t *jp, const uint8_t *data, size_t len, uint32_t *w, uint32_t *h,
              uint32_t *comps) {
    if (!jp || !data || len == 0) return OP_E_INVALID;
    int nc = 0;
    nvjpegChromaSubsampling_t css;
    int ws[NVJPEG_MAX_COMPONENT] = {0}, hs[NVJPEG_MAX_COMPONENT] = {0};
    int st = from_nvjpeg(nvjpegGetImageInfo(jp->handle, data, len, &nc, &css, ws, hs));
    if (st != OP_OK) return st;
    if ((nc != 1 && nc != 3) || ws[0] <= 0 || hs[0] <= 0) return OP_E_CODEC;
    if (w) *w = static_cast<uint32_t>(ws[0]);
    if (h) *h = static_cast<uint32_t>(hs[0]);
    if (comps) *comps = static_cast<uint32_t>(nc);
    return OP_OK;
}

int grow(uint8_t **buf, size_t *cap, size_t need) {
    if (*cap >= need) return OP_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    int st = from_cuda(cudaMalloc(reinterpret_cast<void **>(buf), need));
    if (st == OP_OK) *cap = need;
    return st;
}

int set_params(op_jpeg_t *jp, int quality, int sampling, cudaStream_t s) {
    if (quality < 1 || quality > 100 || !valid_sampling(sampling)) return OP_E_INVALID;
    int st = from_nvjpeg(nvjpegEncoderParamsSetQuality(jp->params, quality, s));
    if (st != OP_OK) return st;
    return from_nvjpeg(nvjpegEncoderParamsSetSamplingFactors(
        jp->params, static_cast<nvjpegChromaSubsampling_t>(sampling), s));
}

// One image through nvJPEG's simple decode.  The decode state is reused
// only after the previous decode's device work has run (it may have been
// queued on another stream, or behind other work on this one).
int decode_into(op_jpeg_t *jp, const uint8_t *data, size_t len, uint8_t *d_rgb, uint32_t pitch,
                cudaStream_t s) {
    if (jp->dec_pending) {
        int st = from_cuda(cudaEventSynchronize(jp->dec_done));
        if (st != OP_OK) return st;
        jp->dec_pending = false;
    }
    nvjpegImage_t dst;
    std::memset(&dst, 0, sizeof(dst));
    dst.channel[0] = d_rgb;
    dst.pitch[0] = pitch;
    int st = from_nvjpeg(nvjpegDecode(jp->handle, jp->dec, data, len, NVJPEG_OUTPUT_RGBI, &dst, s));
    const int rec = from_cuda(cudaEventRecord(jp->dec_done, s));
    if (rec == OP_OK) jp->dec_pending = true;
    return st != OP_OK ? st : rec;
}

// Encode and copy the bitstream out.  The first retrieval only reports the
// length; the stream is synchronised before the copy.
int encode_from(op_jpeg_t *jp, const uint8_t *d_rgb, uint32_t w, uint32_t h, uint32_t pitch,
                uint8_t *out, size_t cap, size_t *out_bytes, cudaStream_t s) {
    nvjpegImage_t src;
    std::memset(&src, 0, sizeof(src));
    src.channel[0] = const_cast<uint8_t *>(d_rgb);
    src.pitch[0] = pitch;
    int st = from_nvjpeg(nvjpegEncodeImage(jp->handle, jp->enc, jp->params, &src,
                                           NVJPEG_INPUT_RGBI, static_cast<int>(w),
                                           static_cast<int>(h), s));
    if (st != OP_OK) return st;
    size_t n = 0;
    st = from_nvjpeg(nvjpegEncodeRetrieveBitstream(jp->handle, jp->enc, nullptr, &n, s));
    if (st != OP_OK) return st;
    st = from_cuda(cudaStreamSynchronize(s));
    if (st != OP_OK) return st;
    *out_bytes = n;
    if (n > cap) return OP_E_NOSPACE;
    st = from_nvjpeg(nvjpegEncodeRetrieveBitstream(jp->handle, jp->enc, out, &n, s));
    if (st != OP_OK) return st;
    *out_bytes = n;
    return from_cuda(cudaStreamSynchronize(s));
}

// The hardware decoder, created on first use; false (and remembered) when
// the GPU has no JPEG engine or nvJPEG cannot drive it.
bool hw_ready(op_jpeg_t *jp) {
    if (jp->hw_ok == 0) {
        bool ok = nvjpegCreateEx(NVJPEG_BACKEND_HARDWARE, nullptr, nullptr, 0, &jp->hw) ==
                  NVJPEG_STATUS_SUCCESS;
        ok = ok && nvjpegJpegStateCreate(jp->hw, &jp->hw_dec) == NVJPEG_STATUS_SUCCESS;
        ok = ok && nvjpegJpegStreamCreate(jp->hw, &jp->hw_parse) == NVJPEG_STATUS_SUCCESS;
        if (!ok) {
            if (jp->hw_parse) nvjpegJpegStreamDestroy(jp->hw_parse);
            if (jp->hw_dec) nvjpegJpegStateDestroy(jp->hw_dec);
            if (jp->hw) nvjpegDestroy(jp->hw);
            jp->hw_parse = nullptr;
            jp->hw_dec = nullptr;
            jp->hw = nullptr;
        }
        cudaGetLastError();
        jp->hw_ok = ok ? 1 : -1;
    }
    return jp->hw_ok == 1;
}

// Whether the hardware decoder takes this stream (nvJPEG reports 0 for yes).
bool hw_takes(op_jpeg_t *jp, const uint8_t *data, size_t len) {
    int unsupported = 1;
    return nvjpegJpegStreamParse(jp->hw, data, len, 0, 0, jp->hw_parse) ==
               NVJPEG_STATUS_SUCCESS &&
           nvjpegDecodeBatchedSupported(jp->hw, jp->hw_parse, &unsupported) ==
               NVJPEG_STATUS_SUCCESS &&
           unsupported == 0;
}

// m streams in one batched call on the hardware decoder.
int hw_decode(op_jpeg_t *jp, int m, const unsigned char *const *data, const size_t *lens,
              nvjpegImage_t *dst, cudaStream_t s) {
    if (jp->hw_batch != m) {
        jp->hw_batch = 0;
        int st = from_nvjpeg(
            nvjpegDecodeBatchedInitialize(jp->hw, jp->hw_dec, m, 1, NVJPEG_OUTPUT_RGBI));
        if (st != OP_OK) return st;
        jp->hw_batch = m;
    }
    return from_nvjpeg(nvjpegDecodeBatched(jp->hw, jp->hw_dec, data, lens, dst, s));
}

// The context's filter handle for these arguments, made anew when the image
// size or the parameters changed.
int ensure_op(op_jpeg_t *jp, uint32_t w, uint32_t h, uint32_t pitch, int32_t radius,
              uint32_t levels, uint32_t flags) {
    if (jp->op && jp->op_w == w && jp->op_h == h && jp->op_pitch == pitch &&
        jp->op_radius == radius && jp->op_levels == levels && jp->op_flags == flags)
        return OP_OK;
    if (jp->op) op_destroy(jp->op);
    jp->op = op_create_ex(w, h, pitch, 3, radius, levels, flags);
    if (!jp->op) return op_last_error();
    jp->op_w = w;
    jp->op_h = h;
    jp->op_pitch = pitch;
    jp->op_radius = radius;
    jp->op_levels = levels;
    jp->op_flags = flags;
    return OP_OK;
}

float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

}  // namespace

extern "C" {

int op_jpeg_last_error(void) { return g_last_error; }

int op_jpeg_destroy(op_jpeg_t *jp) {
    if (!jp) return OP_OK;
    cudaDeviceSynchronize();
    if (jp->op) op_destroy(jp->op);
    if (jp->d_in) cudaFree(jp->d_in);
    if (jp->d_out) cudaFree(jp->d_out);
    for (cudaEvent_t e : jp->ev)
        if (e) cudaEventDestroy(e);
    if (jp->dec_done) cudaEventDestroy(jp->dec_done);
    if (jp->params) nvjpegEncoderParamsDestroy(jp->params);
    if (jp->enc) nvjpegEncoderStateDestroy(jp->enc);
    if (jp->dec) nvjpegJpegStateDestroy(jp->dec);
    if (jp->handle) nvjpegDestroy(jp->handle);
    if (jp->hw_parse) nvjpegJpegStreamDestroy(jp->hw_parse);
    if (jp->hw_dec) nvjpegJpegStateDestroy(jp->hw_dec);
    if (jp->hw) nvjpegDestroy(jp->hw);
    if (jp->d_batch) cudaFree(jp->d_batch);
    cudaGetLastError();
    delete jp;
    return OP_OK;
}

op_jpeg_t *op_jpeg_create(void *stream) {
    op_jpeg_t *jp = new (std::nothrow) op_jpeg_t();
    if (!jp) {
        g_last_error = OP_E_NOMEM;
        return nullptr;
    }
    cudaStream_t s = as_stream(stream);
    int st = from_nvjpeg(nvjpegCreateSimple(&jp->handle));
    if (st == OP_OK) st = from_nvjpeg(nvjpegJpegStateCreate(jp->handle, &jp->dec));
    if (st == OP_OK) st = from_nvjpeg(nvjpegEncoderStateCreate(jp->handle, &jp->enc, s));
    if (st == OP_OK) st = from_nvjpeg(nvjpegEncoderParamsCreate(jp->handle, &jp->params, s));
    if (st == OP_OK) st = set_params(jp, 90, OP_JPEG_CSS_420, s);
    for (int i = 0; i < 4 && st == OP_OK; ++i) st = from_cuda(cudaEventCreate(&jp->ev[i]));
    if (st == OP_OK)
        st = from_cuda(cudaEventCreateWithFlags(&jp->dec_done, cudaEventDisableTiming));
    if (st != OP_OK) {
        op_jpeg_destroy(jp);
        g_last_error = st;
        return nullptr;
    }

    g_last_error = OP_OK;
    return jp;
}

int op_jpeg_info(op_jpeg_t *jp, const uint8_t *data, size_t len, uint32_t *width,
                 uint32_t *height, uint32_t *components) {
    return read_info(jp, data, len, width, height, components);
}

int op_jpeg_decode(op_jpeg_t *jp, const uint8_t *data, size_t len, uint8_t *d_rgb,
                   uint32_t pitch, void *stream) {
    uint32_t w = 0, h = 0;
    if (!d_rgb) return OP_E_INVALID;
    int st = read_info(jp, data, len, &w, &h, nullptr);
    if (st != OP_OK) return st;
    if (static_cast<uint64_t>(pitch) < 3ull * w) return OP_E_INVALID;
    return decode_into(jp, data, len, d_rgb, pitch, as_stream(stream));
}

int op_jpeg_encode_bound(op_jpeg_t *jp, uint32_t width, uint32_t height, int quality,
                         int sampling, size_t *bytes) {
    if (!jp || !bytes || width == 0 || height == 0 || width > 65535u || height > 65535u)
        return OP_E_INVALID;
    int st = set_params(jp, quality, sampling, nullptr);
    if (st != OP_OK) return st;
    return from_nvjpeg(nvjpegEncodeGetBufferSize(jp->handle, jp->params, static_cast<int>(width),
                                                 static_cast<int>(height), bytes));
}

int op_jpeg_encode(op_jpeg_t *jp, const uint8_t *d_rgb, uint32_t width, uint32_t height,
                   uint32_t pitch, int quality, int sampling, uint8_t *out, size_t cap,
                   size_t *out_bytes, void *stream) {
    if (!jp || !d_rgb || !out_bytes || width == 0 || height == 0 || width > 65535u ||
        height > 65535u || static_cast<uint64_t>(pitch) < 3ull * width || (!out && cap > 0))
        return OP_E_INVALID;
    cudaStream_t s = as_stream(stream);
    int st = set_params(jp, quality, sampling, s);
    if (st != OP_OK) return st;
    return encode_from(jp, d_rgb, width, height, pitch, out, cap, out_bytes, s);
}

int op_jpeg_filter(op_jpeg_t *jp, const uint8_t *in, size_t in_len, int32_t radius,
                   uint32_t levels, uint32_t flags, int quality, int sampling, uint8_t *out,
                   size_t cap, size_t *out_bytes, uint8_t *d_filtered, uint32_t filtered_pitch,
                   void *stream) {
    if (!jp || !out_bytes || (!out && cap > 0)) return OP_E_INVALID;
    cudaStream_t s = as_stream(stream);
    uint32_t w = 0, h = 0;
    int st = read_info(jp, in, in_len, &w, &h, nullptr);
    if (st != OP_OK) return st;
    st = set_params(jp, quality, sampling, s);
    if (st != OP_OK) return st;
    // Row pitch: the caller's when it takes the filtered image, else 3w
    // rounded up to 16 bytes.
    uint32_t pitch;
    if (d_filtered) {
        if (static_cast<uint64_t>(filtered_pitch) < 3ull * w) return OP_E_INVALID;
        pitch = filtered_pitch;
    } else {
        pitch = (3u * w + 15u) & ~15u;
    }
    const size_t bytes = static_cast<size_t>(pitch) * h;
    st = grow(&jp->d_in, &jp->in_cap, bytes);
    if (st != OP_OK) return st;
    uint8_t *dst = d_filtered;
    if (!dst) {
        st = grow(&jp->d_out, &jp->out_cap, bytes);
        if (st != OP_OK) return st;
        dst = jp->d_out;
    }
    st = ensure_op(jp, w, h, pitch, radius, levels, flags);
    if (st != OP_OK) return st;
    jp->have_timing = false;
    st = from_cuda(cudaEventRecord(jp->ev[0], s));
    if (st == OP_OK) st = decode_into(jp, in, in_len, jp->d_in, pitch, s);
    if (st == OP_OK) st = from_cuda(cudaEventRecord(jp->ev[1], s));
    if (st == OP_OK) st = op_run(jp->op, jp->d_in, dst, s);
    if (st == OP_OK) st = from_cuda(cudaEventRecord(jp->ev[2], s));
    if (st == OP_OK) st = op_sync_status(jp->op, s);
    if (st == OP_OK) st = encode_from(jp, dst, w, h, pitch, out, cap, out_bytes, s);
    if (st == OP_OK) st = from_cuda(cudaEventRecord(jp->ev[3], s));
    if (st == OP_OK) st = from_cuda(cudaEventSynchronize(jp->ev[3]));
    if (st != OP_OK) return st;
    op_jpeg_timing_t t{};
    st = from_cuda(cudaEventElapsedTime(&t.decode_ms, jp->ev[0], jp->ev[1]));
    if (st == OP_OK) st = from_cuda(cudaEventElapsedTime(&t.filter_ms, jp->ev[1], jp->ev[2]));
    if (st == OP_OK) st = from_cuda(cudaEventElapsedTime(&t.encode_ms, jp->ev[2], jp->ev[3]));
    if (st != OP_OK) return st;
    jp->timing = t;
    jp->have_timing = true;
    return OP_OK;
}

int op_jpeg_filter_file(op_jpeg_t *jp, const char *in_path, const char *out_path,
                        int32_t radius, uint32_t levels, uint32_t flags, int quality,
                        int sampling, void *stream) {
    if (!jp || !in_path || !out_path) return OP_E_INVALID;
    std::vector<uint8_t> in;
    {
        FILE *f = std::fopen(in_path, "rb");
        if (!f) return OP_E_INVALID;
        uint8_t chunk[1 << 16];
        size_t n;
        while ((n = std::fread(chunk, 1, sizeof(chunk), f)) > 0) in.insert(in.end(), chunk, chunk + n);
        const bool bad = std::ferror(f) != 0;
        std::fclose(f);
        if (bad || in.empty()) return OP_E_INVALID;
    }
    uint32_t w = 0, h = 0;
    int st = read_info(jp, in.data(), in.size(), &w, &h, nullptr);
    if (st != OP_OK) return st;
    size_t cap = 0;
    st = op_jpeg_encode_bound(jp, w, h, quality, sampling, &cap);
    if (st != OP_OK) return st;
    std::vector<uint8_t> out(cap);
    size_t n = 0;
    st = op_jpeg_filter(jp, in.data(), in.size(), radius, levels, flags, quality, sampling,
                        out.data(), out.size(), &n, nullptr, 0, stream);
    if (st != OP_OK) return st;
    FILE *f = std::fopen(out_path, "wb");
    if (!f) return OP_E_INVALID;
    const bool ok = std::fwrite(out.data(), 1, n, f) == n;
    return (std::fclose(f) == 0 && ok) ? OP_OK : OP_E_INVALID;
}

int op_jpeg_filter_batch(op_jpeg_t *jp, uint32_t n, const uint8_t *const *in,
                         const size_t *in_len, int32_t radius, uint32_t levels, uint32_t flags,
                         int quality, int sampling, uint8_t *const *out, const size_t *cap,
                         size_t *out_bytes, int *status, void *stream) {
    if (!jp || !in || !in_len || !out || !cap || !out_bytes || !status || n == 0 ||
        n > OP_JPEG_MAX_BATCH || quality < 1 || quality > 100 || !valid_sampling(sampling))
        return OP_E_INVALID;
    cudaStream_t s = as_stream(stream);
    jp->have_timing = false;
    uint32_t w[OP_JPEG_MAX_BATCH], h[OP_JPEG_MAX_BATCH], pitch[OP_JPEG_MAX_BATCH];
    size_t off[OP_JPEG_MAX_BATCH];
    size_t total = 0, most = 0;
    for (uint32_t i = 0; i < n; ++i) {
        out_bytes[i] = 0;
        status[i] = (!in[i] || (!out[i] && cap[i] > 0))
                        ? OP_E_INVALID
                        : read_info(jp, in[i], in_len[i], &w[i], &h[i], nullptr);
        if (status[i] != OP_OK) continue;
        pitch[i] = (3u * w[i] + 15u) & ~15u;
        off[i] = total;
        const size_t bytes = static_cast<size_t>(pitch[i]) * h[i];
        total += bytes;
        if (bytes > most) most = bytes;
    }
    // Steps that every remaining image needs: on failure each takes the status.
    auto fail_rest = [&](int st) {
        for (uint32_t i = 0; i < n; ++i)
            if (status[i] == OP_OK) status[i] = st;
    };
    int st = OP_OK;
    if (total > 0) {
        st = set_params(jp, quality, sampling, s);
        if (st == OP_OK) st = grow(&jp->d_batch, &jp->batch_cap, total);
        if (st == OP_OK) st = grow(&jp->d_out, &jp->out_cap, most);
        if (st == OP_OK) st = from_cuda(cudaEventRecord(jp->ev[0], s));
        if (st != OP_OK) fail_rest(st);
    }
    op_jpeg_timing_t t{};
    if (total > 0 && st == OP_OK) {
        // The hardware decoder's share in one call, then the rest one by one.
        bool on_hw[OP_JPEG_MAX_BATCH] = {};
        const unsigned char *hw_in[OP_JPEG_MAX_BATCH];
        size_t hw_len[OP_JPEG_MAX_BATCH];
        nvjpegImage_t hw_dst[OP_JPEG_MAX_BATCH];
        int m = 0;
        if (hw_ready(jp)) {
            for (uint32_t i = 0; i < n; ++i) {
                if (status[i] != OP_OK || !hw_takes(jp, in[i], in_len[i])) continue;
                on_hw[i] = true;
                hw_in[m] = in[i];
                hw_len[m] = in_len[i];
                std::memset(&hw_dst[m], 0, sizeof(hw_dst[m]));
                hw_dst[m].channel[0] = jp->d_batch + off[i];
                hw_dst[m].pitch[0] = pitch[i];
                ++m;
            }
            if (m > 0 && hw_decode(jp, m, hw_in, hw_len, hw_dst, s) != OP_OK) {
                cudaGetLastError();
                for (uint32_t i = 0; i < n; ++i) on_hw[i] = false;  // all take the other decode
            }
        }
        for (uint32_t i = 0; i < n; ++i)
            if (status[i] == OP_OK && !on_hw[i])
                status[i] = decode_into(jp, in[i], in_len[i], jp->d_batch + off[i], pitch[i], s);
        st = from_cuda(cudaEventRecord(jp->ev[1], s));
        if (st == OP_OK) st = from_cuda(cudaEventSynchronize(jp->ev[1]));
        if (st != OP_OK) fail_rest(st);
        t.decode_ms = elapsed_ms(jp->ev[0], jp->ev[1]);
        // Filter and encode image by image (the encoder synchronises `s`).
        for (uint32_t i = 0; i < n; ++i) {
            if (status[i] != OP_OK) continue;
            uint8_t *src = jp->d_batch + off[i];
            int si = ensure_op(jp, w[i], h[i], pitch[i], radius, levels, flags);
            if (si == OP_OK) si = from_cuda(cudaEventRecord(jp->ev[2], s));
            if (si == OP_OK) si = op_run(jp->op, src, jp->d_out, s);
            if (si == OP_OK) si = from_cuda(cudaEventRecord(jp->ev[3], s));
            if (si == OP_OK) si = op_sync_status(jp->op, s);
            if (si == OP_OK)
                si = encode_from(jp, jp->d_out, w[i], h[i], pitch[i], out[i], cap[i],
                                 &out_bytes[i], s);
            if (si == OP_OK) si = from_cuda(cudaEventRecord(jp->ev[0], s));
            if (si == OP_OK) si = from_cuda(cudaEventSynchronize(jp->ev[0]));
            if (si == OP_OK) {
                t.filter_ms += elapsed_ms(jp->ev[2], jp->ev[3]);
                t.encode_ms += elapsed_ms(jp->ev[3], jp->ev[0]);
            }
            status[i] = si;
        }
    }
    for (uint32_t i = 0; i < n; ++i)
        if (status[i] != OP_OK) return status[i];
    jp->timing = t;
    jp->have_timing = true;
    return OP_OK;
}

int op_jpeg_last_timing(const op_jpeg_t *jp, op_jpeg_timing_t *t) {
    if (!jp || !t || !jp->have_timing) return OP_E_INVALID;
    *t = jp->timing;
    return OP_OK;
}

}  // extern "C"
