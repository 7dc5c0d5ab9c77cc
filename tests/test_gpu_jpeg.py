"""Decode -> filter -> encode (section 3.2's ApplyOilPaintOnFile) on the GPU.

The filter's parity is checked where the pipeline's input is known without
trusting the decoder: flat-block grayscale JPEGs written by
tests/jpeg_fixture.py decode to a known image (checked exactly), and the
pipeline's filtered image equals the oracle on that known image.  On
camera-like photos encoded here the filtered image equals the oracle on the
decoder's output, and the encoded result is the encoder's output for that
filtered image, byte for byte.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1405_1020_gb300 import jpeg as J
from paper_1405_1020_gb300 import synth
from paper_1405_1020_gb300.binding import OP_E_INVALID, OilPaintError

from tests.jpeg_fixture import (flat_gray_image, flat_gray_jpeg, flat_gray_jpeg_progressive,
                                frame_header)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1405_1020_gb300.csrc import build as cbuild
    cbuild.build()
    if cbuild.build_jpeg() is None:
        pytest.skip("nvJPEG is not in this CUDA toolkit")


@pytest.fixture(scope="module")
def pipe():
    _lib_or_skip()
    p = J.JpegPipeline()
    yield p
    p.close()


def _oracle_rgb(rgb: np.ndarray, radius: int, levels: int) -> np.ndarray:
    h, w = rgb.shape[:2]
    buf = np.ascontiguousarray(rgb, dtype=np.uint8).reshape(-1)
    return oracle.oilpaint(buf, w, h, 3 * w, 3, radius, levels, out=buf.copy()).reshape(h, w, 3)


def _psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2)
    return float("inf") if mse == 0 else 10 * np.log10(255.0 ** 2 / mse)


def _blocks(by, bx, seed):
    rng = np.random.default_rng(seed)
    # a few large flat regions with block-level detail, so windows hold ties and edges
    coarse = rng.integers(0, 256, size=((by + 3) // 4, (bx + 3) // 4))
    b = np.kron(coarse, np.ones((4, 4), dtype=np.int64))[:by, :bx]
    jitter = rng.integers(-12, 13, size=(by, bx)) * (rng.random((by, bx)) < 0.3)
    b = np.clip(b + jitter, 0, 255)
    b[0, 0], b[-1, -1] = 0, 255           # extremes of the DC range
    return b.astype(np.uint8)


def test_flat_block_jpeg_decodes_exactly(pipe):
    blocks = _blocks(9, 17, seed=11)
    data = flat_gray_jpeg(blocks)
    hdr = frame_header(data)
    assert (hdr["width"], hdr["height"], hdr["components"]) == (136, 72, 1)
    assert pipe.info(data) == (136, 72, 1)
    got = pipe.decode(data, pitch=3 * 136 + 8)
    torch.cuda.synchronize()
    got = got.cpu().numpy()[:, :3 * 136].reshape(72, 136, 3)
    want = flat_gray_image(blocks)
    for c in range(3):                    # grayscale decodes to R = G = B
        assert np.array_equal(got[..., c], want)


@pytest.mark.parametrize("w,h", [(133, 70), (129, 65), (57, 9)])
def test_flat_block_jpeg_ragged_size_decodes_exactly(pipe, w, h):
    """Sizes that are not multiples of the 8x8 block: the decoder keeps the
    edge blocks' pixels inside the frame only."""
    bx, by = (w + 7) // 8, (h + 7) // 8
    blocks = _blocks(by, bx, seed=w + h)
    data = flat_gray_jpeg(blocks, w, h)
    assert pipe.info(data) == (w, h, 1)
    got = pipe.decode(data).cpu().numpy().reshape(h, w, 3)
    want = flat_gray_image(blocks, w, h)
    for c in range(3):
        assert np.array_equal(got[..., c], want)
    out, rgb = pipe.filter(data, 3, 20, quality=95, sampling=J.OP_JPEG_CSS_444, keep_rgb=True)
    img = np.repeat(want[..., None], 3, axis=2)
    assert np.array_equal(rgb.cpu().numpy().reshape(h, w, 3), _oracle_rgb(img, 3, 20))
    assert frame_header(out)["width"] == w and frame_header(out)["height"] == h


@pytest.mark.parametrize("radius,levels", [(2, 20), (5, 64), (1, 256), (15, 20)])
def test_pipeline_on_flat_blocks_equals_oracle(pipe, radius, levels):
    blocks = _blocks(24, 40, seed=radius * 7 + levels)
    data = flat_gray_jpeg(blocks)
    img = np.repeat(flat_gray_image(blocks)[..., None], 3, axis=2)
    want = _oracle_rgb(img, radius, levels)
    out, rgb = pipe.filter(data, radius, levels, quality=95, sampling=J.OP_JPEG_CSS_444,
                           keep_rgb=True)
    got = rgb.cpu().numpy().reshape(want.shape)
    assert np.array_equal(got, want)
    # the encoded bytes are the encoder's output for that filtered image
    again = pipe.encode(rgb, 320, 192, quality=95, sampling=J.OP_JPEG_CSS_444)
    assert out == again
    hdr = frame_header(out)
    assert (hdr["width"], hdr["height"], hdr["components"]) == (320, 192, 3)


@pytest.mark.parametrize("w,h,sampling,radius,levels", [
    (640, 480, J.OP_JPEG_CSS_420, 4, 20),      # VGA, the paper's smallest size
    (1001, 757, J.OP_JPEG_CSS_420, 15, 20),    # ragged: not a multiple of the 16-pixel MCU
    (803, 611, J.OP_JPEG_CSS_422, 8, 64),
    (517, 389, J.OP_JPEG_CSS_444, 3, 256),
])
def test_pipeline_on_photo_equals_oracle(pipe, w, h, sampling, radius, levels):
    src = synth.camera_like(h, w, seed=w + h, npoly=60, rad_range=(10, 200))
    t = torch.from_numpy(np.ascontiguousarray(src).reshape(h, 3 * w)).cuda()
    data = pipe.encode(t, w, h, quality=90, sampling=sampling)
    hdr = frame_header(data)
    assert (hdr["width"], hdr["height"], hdr["components"]) == (w, h, 3)
    decoded = pipe.decode(data).cpu().numpy().reshape(h, w, 3)
    # a sanity bound (a swapped channel or a shifted row gives ~10 dB): the
    # image's N(0, 6^2) pixel noise alone costs ~30 dB at quality 90
    assert _psnr(decoded, src) > 24.0
    out, rgb = pipe.filter(data, radius, levels, quality=90, sampling=sampling, keep_rgb=True)
    want = _oracle_rgb(decoded, radius, levels)
    got = rgb.cpu().numpy().reshape(h, w, 3)
    assert np.array_equal(got, want)
    assert out == pipe.encode(rgb, w, h, quality=90, sampling=sampling)
    # the pipeline's own buffers (no caller image) give the same bytes
    assert pipe.filter(data, radius, levels, quality=90, sampling=sampling) == out
    t3 = pipe.last_timing()
    assert t3["decode_ms"] > 0 and t3["filter_ms"] > 0 and t3["encode_ms"] > 0


def test_encode_round_trip_fidelity(pipe):
    w, h = 320, 240
    src = synth.camera_like(h, w, seed=5, npoly=20, rad_range=(10, 100), noise=0.0)
    t = torch.from_numpy(np.ascontiguousarray(src).reshape(h, 3 * w)).cuda()
    q95 = pipe.encode(t, w, h, quality=95, sampling=J.OP_JPEG_CSS_444)
    q30 = pipe.encode(t, w, h, quality=30, sampling=J.OP_JPEG_CSS_420)
    assert frame_header(q95)["sampling"] == [(1, 1)] * 3
    assert frame_header(q30)["sampling"][0] == (2, 2)
    assert len(q30) < len(q95)
    p95 = _psnr(pipe.decode(q95).cpu().numpy().reshape(h, w, 3), src)
    p30 = _psnr(pipe.decode(q30).cpu().numpy().reshape(h, w, 3), src)
    assert p95 > 36.0 and p30 > 20.0 and p95 > p30 + 3.0


def test_filter_file(pipe, tmp_path):
    w, h = 400, 300
    src = synth.camera_like(h, w, seed=9, npoly=30, rad_range=(10, 120))
    t = torch.from_numpy(np.ascontiguousarray(src).reshape(h, 3 * w)).cuda()
    data = pipe.encode(t, w, h, quality=92)
    fin, fout = tmp_path / "in.jpg", tmp_path / "out.jpg"
    fin.write_bytes(data)
    pipe.filter_file(str(fin), str(fout), 6, 20, quality=92)
    assert fout.read_bytes() == pipe.filter(data, 6, 20, quality=92)
    with pytest.raises(OilPaintError) as e:
        pipe.filter_file(str(tmp_path / "missing.jpg"), str(fout), 6, 20)
    assert e.value.status == OP_E_INVALID


def test_filter_many_equals_one_at_a_time(pipe):
    datas = []
    for k, (w, h) in enumerate(((320, 240), (101, 77), (640, 480), (64, 64), (333, 251))):
        src = synth.camera_like(h, w, seed=40 + k, npoly=15, rad_range=(5, 80))
        t = torch.from_numpy(np.ascontiguousarray(src).reshape(h, 3 * w)).cuda()
        datas.append(pipe.encode(t, w, h, quality=90))
    datas = datas * 3
    got = J.filter_many(datas, 4, 20, quality=90, workers=4, batch=1)
    assert got == [pipe.filter(d, 4, 20, quality=90) for d in datas]


def test_command_line(pipe, tmp_path, capsys):
    w, h = 300, 200
    src = synth.camera_like(h, w, seed=12, npoly=20, rad_range=(5, 80))
    t = torch.from_numpy(np.ascontiguousarray(src).reshape(h, 3 * w)).cuda()
    data = pipe.encode(t, w, h, quality=90)
    fin, fout = tmp_path / "a.jpg", tmp_path / "b.jpg"
    fin.write_bytes(data)
    assert J.main([str(fin), str(fout), "--radius", "4", "--levels", "16"]) == 0
    assert fout.read_bytes() == pipe.filter(data, 4, 16, quality=90)
    assert '"width": 300' in capsys.readouterr().out


def test_errors(pipe):
    w, h = 64, 48
    src = synth.camera_like(h, w, seed=3, npoly=5, rad_range=(5, 30))
    t = torch.from_numpy(np.ascontiguousarray(src).reshape(h, 3 * w)).cuda()
    data = pipe.encode(t, w, h)
    # not a JPEG: rejected by the header parse on the host
    for junk in (b"\x00" * 64, b"GIF89a" + bytes(100)):
        with pytest.raises(OilPaintError) as e:
            pipe.info(junk)
        assert e.value.status == J.OP_E_CODEC
        with pytest.raises(OilPaintError) as e:
            pipe.filter(junk, 2, 20)
        assert e.value.status == J.OP_E_CODEC
    n = ctypes.c_size_t()
    buf = ctypes.create_string_buffer(16)
    for junk in (b"\x00" * 64, b"\xff\xd8\xff\xd9"):
        assert J.op_jpeg_filter(pipe._h, junk, 2, 20, 0, 90, 0, buf, 16, n) == J.OP_E_CODEC
    assert J.op_jpeg_filter(pipe._h, b"", 2, 20, 0, 90, 0, buf, 16, n) == OP_E_INVALID
    # output buffer too small: the size needed comes back
    st = J.op_jpeg_filter(pipe._h, data, 2, 20, 0, 90, J.OP_JPEG_CSS_420, buf, 16, n)
    assert st == J.OP_E_NOSPACE and n.value > 16
    assert len(pipe.filter(data, 2, 20)) == n.value
    # argument checks
    d = torch.empty((h, 3 * w), dtype=torch.uint8, device="cuda")
    assert J.op_jpeg_decode(pipe._h, data, d.data_ptr(), 3 * w - 1) == OP_E_INVALID
    for q, s in ((0, 0), (101, 0), (90, 3), (90, -1)):
        assert J.op_jpeg_encode(pipe._h, d.data_ptr(), w, h, 3 * w, q, s, buf, 16, n) == OP_E_INVALID
    # the filter's own argument checks come through (radius above the maximum)
    assert J.op_jpeg_filter(pipe._h, data, 45, 20, 0, 90, 0, buf, 16, n) == OP_E_INVALID
    # a fresh context has no timing yet
    with J.JpegPipeline() as fresh:
        with pytest.raises(OilPaintError):
            fresh.last_timing()


def _photo_jpegs(pipe, sizes, seed0, sampling=J.OP_JPEG_CSS_420, quality=90):
    out = []
    for k, (w, h) in enumerate(sizes):
        src = synth.camera_like(h, w, seed=seed0 + k, npoly=15, rad_range=(5, 80))
        t = torch.from_numpy(np.ascontiguousarray(src).reshape(h, 3 * w)).cuda()
        out.append(pipe.encode(t, w, h, quality=quality, sampling=sampling))
    return out


@pytest.mark.parametrize("sampling", [J.OP_JPEG_CSS_444, J.OP_JPEG_CSS_422, J.OP_JPEG_CSS_420])
def test_filter_batch_equals_filter(pipe, sampling):
    # ragged sizes, a grayscale stream among the colour ones; each output must
    # equal the one-image pipeline's (whose filter is checked against the
    # oracle above), whichever decoder the batch gave the stream to
    datas = _photo_jpegs(pipe, ((320, 240), (101, 77), (64, 64), (333, 251), (17, 9)), 60,
                         sampling=sampling)
    datas.insert(2, flat_gray_jpeg(_blocks(9, 13, 7), 99, 70))
    got = pipe.filter_batch(datas, 5, 20, quality=88, sampling=sampling)
    assert got == [pipe.filter(d, 5, 20, quality=88, sampling=sampling) for d in datas]
    t = pipe.last_timing()
    assert t["decode_ms"] > 0 and t["filter_ms"] > 0 and t["encode_ms"] > 0


def test_filter_batch_12mp(pipe):
    # the benchmark's image size, eight streams in one batched decode
    w, h = 4000, 3000
    src = synth.camera_like(h, w, seed=2)
    t = torch.from_numpy(np.ascontiguousarray(src).reshape(h, 3 * w)).cuda()
    data = pipe.encode(t, w, h, quality=90)
    one = pipe.filter(data, 15, 20, quality=90)
    assert pipe.filter_batch([data] * 8, 15, 20, quality=90) == [one] * 8


def test_filter_batch_statuses(pipe):
    datas = _photo_jpegs(pipe, ((96, 80), (50, 41)), 70)
    junk = b"\x00" * 64
    batch = [datas[0], junk, datas[1]]
    with pytest.raises(OilPaintError) as e:
        pipe.filter_batch(batch, 3, 16)
    assert e.value.status == J.OP_E_CODEC and "image 1" in str(e.value)
    # through the C call: per-image statuses; the good images still come out,
    # and an output buffer that is too small reports the size needed
    want = [pipe.filter(d, 3, 16) for d in datas]
    n = 3
    caps = [len(want[0]) + 100, 16, 16]
    bufs = [ctypes.create_string_buffer(c) for c in caps]
    outs = (ctypes.c_void_p * n)(*[ctypes.addressof(b) for b in bufs])
    capa = (ctypes.c_size_t * n)(*caps)
    got = (ctypes.c_size_t * n)()
    status = (ctypes.c_int * n)()
    st = J.op_jpeg_filter_batch(pipe._h, batch, 3, 16, 0, 90, J.OP_JPEG_CSS_420, outs, capa, got,
                                status, None)
    assert st == J.OP_E_CODEC
    assert list(status) == [0, J.OP_E_CODEC, J.OP_E_NOSPACE]
    assert bufs[0].raw[:got[0]] == want[0]
    assert got[2] == len(want[1])
    # arguments checked before anything runs: status[] untouched
    status[0] = 12345
    for bad_n, q in ((0, 90), (J.OP_JPEG_MAX_BATCH + 1, 90), (1, 0), (1, 101)):
        many = [datas[0]] * bad_n
        arr = lambda t: (t * max(bad_n, 1))()  # noqa: E731
        assert J.op_jpeg_filter_batch(pipe._h, many, 3, 16, 0, q, 0, arr(ctypes.c_void_p),
                                      arr(ctypes.c_size_t), arr(ctypes.c_size_t), status,
                                      None) == OP_E_INVALID
    assert status[0] == 12345


def test_filter_many_batched_equals_one_at_a_time(pipe):
    datas = _photo_jpegs(pipe, ((320, 240), (101, 77), (640, 480), (64, 64), (333, 251)), 80)
    datas = datas * 3
    want = [pipe.filter(d, 4, 20, quality=90) for d in datas]
    assert J.filter_many(datas, 4, 20, quality=90, workers=2, batch=4) == want
    with J.JpegPool(3, batch=8) as pool:
        assert pool.filter_many(datas, 4, 20, quality=90) == want
        assert pool.filter_many(datas[:1], 4, 20, quality=90) == want[:1]
    with pytest.raises(ValueError):
        J.JpegPool(1, batch=0)


def test_progressive_flat_block_jpeg_decodes_exactly(pipe):
    blocks = _blocks(8, 11, 21)
    w, h = 83, 61
    data = flat_gray_jpeg_progressive(blocks, w, h)
    assert frame_header(data)["sof"] == 0xC2
    want = flat_gray_image(blocks, w, h)
    got = pipe.decode(data).cpu().numpy().reshape(h, w, 3)
    for c in range(3):
        np.testing.assert_array_equal(got[..., c], want)


def test_filter_batch_mixes_decoders(pipe):
    # progressive streams are not for the JPEG engines (baseline only): in a
    # batch they take the other decoder, behind the engines' share queued on
    # the same stream; every output equals the one-image pipeline's, and the
    # progressive images' filtered pixels equal the oracle's on the known image
    photos = _photo_jpegs(pipe, ((160, 120), (77, 50)), 90)
    b1, b2 = _blocks(7, 10, 31), _blocks(4, 5, 32)
    p1 = flat_gray_jpeg_progressive(b1, 75, 53)
    p2 = flat_gray_jpeg_progressive(b2, 40, 32)
    batch = [photos[0], p1, flat_gray_jpeg(b1, 75, 53), p2, photos[1]]
    for _ in range(3):
        got = pipe.filter_batch(batch, 3, 20, quality=95, sampling=J.OP_JPEG_CSS_444)
        assert got == [pipe.filter(d, 3, 20, quality=95, sampling=J.OP_JPEG_CSS_444)
                       for d in batch]
    for data, blocks, (w, h) in ((p1, b1, (75, 53)), (p2, b2, (40, 32))):
        _, rgb = pipe.filter(data, 3, 20, quality=95, sampling=J.OP_JPEG_CSS_444, keep_rgb=True)
        img = np.repeat(flat_gray_image(blocks, w, h)[..., None], 3, axis=2)
        np.testing.assert_array_equal(rgb.cpu().numpy().reshape(h, w, 3), _oracle_rgb(img, 3, 20))


def test_back_to_back_decodes_on_a_busy_stream(pipe):
    # decodes queued behind tens of milliseconds of other work on their
    # stream, with no synchronisation between them: a decode may not reuse
    # the decoder's state before the previous decode's device work has run
    cases = []
    for k, (by, bx, w, h) in enumerate(((7, 10, 75, 53), (6, 9, 70, 45), (3, 4, 30, 20))):
        blocks = _blocks(by, bx, 50 + k)
        writer = flat_gray_jpeg if k == 1 else flat_gray_jpeg_progressive
        cases.append((writer(blocks, w, h), flat_gray_image(blocks, w, h), w, h))
    stream = torch.cuda.Stream()
    outs = [torch.zeros((h, 3 * w), dtype=torch.uint8, device="cuda") for _, _, w, h in cases]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        torch.cuda._sleep(50_000_000)         # tens of milliseconds of one spinning thread
        for (data, _, w, h), out in zip(cases, outs):
            assert J.op_jpeg_decode(pipe._h, data, out.data_ptr(), 3 * w,
                                    stream.cuda_stream) == 0
    stream.synchronize()
    for (_, want, w, h), out in zip(cases, outs):
        got = out.cpu().numpy().reshape(h, w, 3)
        for c in range(3):
            np.testing.assert_array_equal(got[..., c], want)
