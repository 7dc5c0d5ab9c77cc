"""CUDA path vs the CPU oracle, byte for byte, through the C ABI.

Every comparison covers the whole output buffer: pixel bytes must equal the
oracle's, alpha must be copied, and row padding must keep the fill byte both
sides started from.
"""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from paper_1405_1020_gb300 import binding as B
from paper_1405_1020_gb300 import synth
from paper_1405_1020_gb300.filter import OilPaint
from tests.pins import OUT_FILL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def gpu_filter(buf, w, h, stride, bpp, r, L, mode=0, config=None):
    src = torch.from_numpy(np.ascontiguousarray(buf)).cuda()
    dst = torch.full_like(src, OUT_FILL)
    op = OilPaint(w, h, r, L, bpp=bpp, stride=stride, flags=mode, config=config)
    op.run(src, dst)
    assert op.sync_status() == B.OP_OK
    out = dst.cpu().numpy()
    op.close()
    return out


def cpu_filter(buf, w, h, stride, bpp, r, L, mode=0):
    out = np.full(buf.size, OUT_FILL, np.uint8)
    return oracle.oilpaint(buf, w, h, stride, bpp, r, L, mode=mode, out=out)


def assert_same(got, want, w, h, stride, bpp, what=""):
    if np.array_equal(got, want):
        return
    g = got[: h * stride].reshape(h, stride)
    e = want[: h * stride].reshape(h, stride)
    ys, xs = np.nonzero(g != e)
    msg = f"{what}: {ys.size} bytes differ; first at row {ys[0]}, byte {xs[0]} " \
          f"(pixel {xs[0] // bpp}, channel {xs[0] % bpp}): got {g[ys[0], xs[0]]} want {e[ys[0], xs[0]]}"
    raise AssertionError(msg)


def check_case(img, r, L, bpp=3, pad=0, mode=0, config=None, what=""):
    h, w = img.shape[:2]
    buf, stride = synth.to_strided(img, bpp=bpp, stride=w * bpp + pad)
    got = gpu_filter(buf, w, h, stride, bpp, r, L, mode, config)
    want = cpu_filter(buf, w, h, stride, bpp, r, L, mode)
    assert_same(got, want, w, h, stride, bpp, what or f"{w}x{h} r={r} L={L} bpp={bpp}")


# ---- the workloads ---------------------------------------------------------

def test_uniform_256_r2_L20():
    """256x256 i.i.d. uniform RGB (seed 0), r=2, L=20: whole image."""
    check_case(synth.uniform_rgb(256, 256, seed=0), 2, 20)


@pytest.fixture(scope="module")
def blobs_fhd():
    return synth.blobs_rgb(1080, 1920, seed=1)


@pytest.mark.parametrize("r", list(range(1, 11)))
def test_blobs_1920x1080_radius_sweep(blobs_fhd, r):
    """1920x1080 blobs (seed 1), r = 1..10, L=20: whole image."""
    check_case(blobs_fhd, r, 20)


@pytest.fixture(scope="module")
def camera_12mp():
    img = synth.camera_like(3000, 4000, seed=2)
    buf, stride = synth.to_strided(img, bpp=4, stride=16000)
    return buf, stride


@pytest.mark.parametrize("L", [20, 64, 256])
def test_camera_12mp_rgba_r15_whole_image(camera_12mp, L):
    """4000x3000 RGBA-stride camera-like (seed 2), r=15, L = 20 (the measured
    workload, in the launch configuration the benchmark uses), 64 and 256:
    every byte of the GPU output against the oracle's whole image."""
    buf, stride = camera_12mp
    w, h, r = 4000, 3000, 15
    got = gpu_filter(buf, w, h, stride, 4, r, L)
    want = cpu_filter(buf, w, h, stride, 4, r, L)
    assert_same(got, want, w, h, stride, 4, f"12 MP r=15 L={L}")
    px = oracle.view_pixels(got, w, h, stride, 4)
    assert (px[..., 3] == 255).all()


# ---- fuzz grid ---------------------------------------------------------------

def _fuzz_cases(n=48, seed=7):
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(n):
        w = int(rng.choice([1, 2, 3, 5, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 257, 300]))
        h = int(rng.choice([1, 2, 7, 8, 9, 17, 40, 100, 161, 300]))
        r = int(rng.choice([0, 1, 2, 3, 7, 15, 16, 20, 31, 44]))
        L = int(rng.choice([1, 2, 3, 16, 20, 32, 64, 128, 255, 256]))
        bpp = int(rng.choice([3, 4]))
        pad = int(rng.choice([0, 1, 4, 13]))
        mode = int(rng.integers(0, 2))
        nt = int(rng.choice([32, 64, 96, 128]))
        cpt = int(rng.choice([1, 2, 4]))
        cfg = {"tile_w": nt * cpt, "tile_h": int(rng.choice([0, 1, 5, 16, 64])),
               "chunk_rows": int(rng.choice([1, 2, 3, 8, 16, 32])),
               "prefetch": int(rng.integers(1, 5)), "cols_per_thread": cpt}
        cases.append((k, w, h, r, L, bpp, pad, mode, cfg))
    return cases


@pytest.mark.parametrize("k,w,h,r,L,bpp,pad,mode,cfg", _fuzz_cases())
def test_fuzz(k, w, h, r, L, bpp, pad, mode, cfg):
    img = synth.camera_like(h, w, seed=500 + k, npoly=12, rad_range=(1, 60)) if k % 2 else \
        synth.uniform_rgb(h, w, seed=500 + k)
    try:
        check_case(img, r, L, bpp, pad, mode, cfg)
    except B.OilPaintError as e:
        # the only acceptable refusal: a tile too wide for the radius or shared memory
        assert e.status == B.OP_E_UNSUPPORTED, e


def _delta_fuzz_cases(n=56, seed=11):
    """Cases the difference-histogram path takes (L <= 32, 2 or 4 columns
    per thread; 8-byte bins for r <= 15, variant-B bins above): every r mod 4
    (the tile's x shift), widths around the tile width, one-column and
    one-row images."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(n):
        w = int(rng.choice([1, 2, 3, 4, 5, 7, 31, 61, 64, 67, 127, 128, 131, 190, 256, 259, 400]))
        h = int(rng.choice([1, 2, 3, 9, 16, 33, 100, 211]))
        r = int(rng.integers(0, 16)) if k < 40 else int(rng.integers(16, 45))
        L = int(rng.choice([1, 2, 3, 7, 16, 20, 31, 32]))
        bpp = int(rng.choice([3, 4]))
        pad = int(rng.choice([0, 1, 4, 13]))
        mode = int(rng.integers(0, 2))
        cpt = int(rng.choice([2, 4]))
        nt = int(rng.choice([32, 64] if cpt == 4 else [32, 64, 96, 128]))
        cfg = {"tile_w": nt * cpt, "tile_h": int(rng.choice([0, 1, 3, 16, 64])),
               "chunk_rows": int(rng.choice([1, 2, 3, 8, 16, 32])),
               "prefetch": int(rng.integers(1, 5)), "cols_per_thread": cpt}
        cases.append((k, w, h, r, L, bpp, pad, mode, cfg))
    return cases


@pytest.mark.parametrize("k,w,h,r,L,bpp,pad,mode,cfg", _delta_fuzz_cases())
def test_fuzz_difference_histograms(k, w, h, r, L, bpp, pad, mode, cfg):
    img = synth.camera_like(h, w, seed=900 + k, npoly=12, rad_range=(1, 60)) if k % 2 else \
        synth.uniform_rgb(h, w, seed=900 + k)
    try:
        check_case(img, r, L, bpp, pad, mode, cfg)
    except B.OilPaintError as e:
        # refused only when the ring of halo copies plus the K histograms
        # exceeds a CTA's shared memory (an upper estimate of it here)
        assert e.status == B.OP_E_UNSUPPORTED, e
        K, nt = cfg["cols_per_thread"], cfg["tile_w"] // cfg["cols_per_thread"]
        ng = (2 * r + K - 1) // K + 1
        boxw = -(-K * (nt - 1 + ng) // 4) * 4
        half = -(-boxw * cfg["chunk_rows"] * 4 // 128) * 128
        nh = K + (1 if K == 4 and r <= 15 else 0)  # four 8-byte columns split H
        hist = (nh * L + 1) * nt * (8 if r <= 15 else 12)
        slots = cfg["prefetch"] + 1
        smem = 128 + -(-slots * 8 // 128) * 128 + 2 * half * slots + hist
        assert smem > 226 * 1024, (cfg, r, L, smem)


def _straight_cases(n=120, seed=17):
    """The straight-line difference-histogram path (one kernel per radius):
    2, 4 or 8 columns per thread, the window histogram in one part (path 2)
    or two (path 3; eight columns on path 0 mean path 3; two columns: path 2
    only, with up to 64 levels, the sixth level bit), every radius of each
    width's range and both parities (where in a 16-byte group the right
    difference words start), widths around the tile widths, one-row and short
    images, both level modes and literal mode, tile heights, halo chunk
    heights and prefetch depths."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(n):
        K = (4, 8, 2)[k % 3]
        path = {8: int(rng.choice([0, 2, 3])), 4: int(rng.choice([2, 3])), 2: 2}[K]
        w = int(rng.choice([1, 3, 8, 9, 31, 127, 129, 200, 255, 256, 257, 263, 500, 511, 512,
                            513, 700, 1030]))
        h = int(rng.choice([1, 2, 5, 16, 33, 90, 161]))
        r = int(rng.integers({8: 4, 4: 2, 2: 1}[K], 16))
        L = int(rng.choice([1, 2, 3, 7, 16, 20, 31, 32] + ([33, 47, 63, 64] if K == 2 else [])))
        bpp = int(rng.choice([3, 4]))
        pad = int(rng.choice([0, 1, 4, 13]))
        mode = int(rng.choice([0, 1, B.OP_LITERAL, B.OP_LITERAL | 1]))
        nt = int(rng.choice([32, 64]))
        cfg = {"tile_w": nt * K, "tile_h": int(rng.choice([0, 1, 3, 16, 64])),
               "chunk_rows": int(rng.choice([1, 2, 3, 8])), "prefetch": int(rng.integers(1, 3)),
               "cols_per_thread": K, "path": path}
        cases.append((k, w, h, r, L, bpp, pad, mode, cfg))
    return cases


@pytest.mark.parametrize("k,w,h,r,L,bpp,pad,mode,cfg", _straight_cases())
def test_fuzz_straight_line_path(k, w, h, r, L, bpp, pad, mode, cfg):
    img = synth.camera_like(h, w, seed=1700 + k, npoly=12, rad_range=(1, 60)) if k % 4 < 2 else \
        synth.uniform_rgb(h, w, seed=1700 + k)
    if k % 3 == 0:  # runs of white pixels (level L - 1, or level L in literal mode)
        img[np.random.default_rng(k).random((h, w)) < 0.2] = 255
    try:
        check_case(img, r, L, bpp, pad, mode, cfg)
    except B.OilPaintError as e:
        # refused only when the halo ring plus the histograms (nb + K - 1 of
        # 8-byte bins and (K - 1) / 4 count words per level and thread)
        # exceed a CTA's shared memory
        assert e.status == B.OP_E_UNSUPPORTED, e
        K = cfg["cols_per_thread"]
        nb = 1 if cfg["path"] == 2 else 2
        nt = cfg["tile_w"] // K
        boxw = -(-K * (nt - 1 + (2 * r + K - 1) // K + 1) // 4) * 4
        half = -(-boxw * cfg["chunk_rows"] * 4 // 128) * 128
        slots = cfg["prefetch"] + 1
        hist = (((nb + K - 1) * 8 + -(-(K - 1) // 4) * 4) * L if K > 2 else
                16 * L + -(-L // 4) * 4) * nt
        smem = 128 + -(-slots * 8 // 128) * 128 + 2 * half * slots + hist
        assert smem > 226 * 1024, (cfg, r, L, smem)


@pytest.mark.parametrize("r", list(range(1, 16)))
def test_straight_line_every_radius(r):
    """Every radius of the straight-line path, two, four and eight columns
    per thread, the window histogram in one and two parts, 32 and 64 threads,
    RGB and RGBA, on an image whose width is not a tile multiple; two columns
    also at 64 levels."""
    img = synth.camera_like(97, 601, seed=40 + r, npoly=30, rad_range=(3, 150))
    for nt, L in ((32, 20), (64, 64)):
        check_case(img, r, L, bpp=4 if L == 20 else 3, pad=0 if L == 20 else 7,
                   config={"tile_w": 2 * nt, "cols_per_thread": 2, "chunk_rows": 2, "path": 2})
    for K in (4, 8):
        if r < {4: 2, 8: 4}[K]:
            continue
        for path, nt, bpp, pad, ch in ((2, 32, 4, 0, 2), (3, 64, 3, 5, 1), (2, 64, 3, 1, 1),
                                       (3, 32, 4, 8, 3)):
            check_case(img, r, 20, bpp=bpp, pad=pad,
                       config={"tile_w": K * nt, "cols_per_thread": K, "chunk_rows": ch,
                               "path": path})


@pytest.mark.parametrize("K,path,r,L,status", [
    (8, 0, 3, 20, B.OP_E_UNSUPPORTED), (8, 2, 16, 20, B.OP_E_UNSUPPORTED),
    (8, 3, 15, 33, B.OP_E_UNSUPPORTED), (4, 2, 1, 20, B.OP_E_UNSUPPORTED),
    (4, 3, 16, 20, B.OP_E_UNSUPPORTED), (4, 2, 15, 64, B.OP_E_UNSUPPORTED),
    (8, 0, 0, 1, B.OP_E_UNSUPPORTED), (2, 2, 0, 20, B.OP_E_UNSUPPORTED),
    (2, 2, 16, 20, B.OP_E_UNSUPPORTED), (2, 2, 15, 65, B.OP_E_UNSUPPORTED),
    (2, 3, 5, 20, B.OP_E_INVALID)])
def test_straight_line_refused_outside_its_range(K, path, r, L, status):
    op = OilPaint(300, 40, r, L)
    with pytest.raises(B.OilPaintError) as e:
        op.set_config({"tile_w": 32 * K, "cols_per_thread": K, "path": path})
    assert e.value.status == status
    op.close()


def _direct_cases(n=108, seed=23):
    """The direct path (path 4: radius 0, 1 or 2, windows in registers, levels
    compared pairwise): every level count class up to 256, widths around the
    tile widths and narrower than a tile, one-row and short images, both
    level modes and literal mode, thread counts, tile heights, halo chunk
    heights and prefetch depths."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(n):
        r = (1, 2, 0)[k % 3]
        mode = int(rng.choice([0, 1, B.OP_LITERAL, B.OP_LITERAL | 1]))
        Ls = [1, 2, 3, 7, 16, 20, 32, 33, 64, 100, 255, 256]
        L = int(rng.choice([x for x in Ls if not (mode & B.OP_LITERAL) or x <= 254]))
        w = int(rng.choice([1, 2, 3, 5, 31, 32, 33, 63, 64, 65, 95, 96, 97, 128, 129, 300]))
        h = int(rng.choice([1, 2, 3, 4, 5, 17, 64, 129]))
        bpp = int(rng.choice([3, 4]))
        pad = int(rng.choice([0, 1, 4, 13]))
        nt = int(rng.choice([32, 64, 96, 128]))
        cfg = {"tile_w": nt, "tile_h": int(rng.choice([0, 1, 2, 5, 16, 64])),
               "chunk_rows": int(rng.choice([1, 2, 3, 8])), "prefetch": int(rng.integers(1, 3)),
               "cols_per_thread": 1, "path": 4}
        cases.append((k, w, h, r, L, bpp, pad, mode, cfg))
    return cases


@pytest.mark.parametrize("k,w,h,r,L,bpp,pad,mode,cfg", _direct_cases())
def test_fuzz_direct_path(k, w, h, r, L, bpp, pad, mode, cfg):
    if k % 3 == 0:  # few colours: many equal levels and ties
        img = synth.camera_like(h, w, seed=2300 + k, npoly=6, rad_range=(1, 20), noise=0.0)
    elif k % 3 == 1:
        img = synth.uniform_rgb(h, w, seed=2300 + k)
    else:
        img = synth.camera_like(h, w, seed=2300 + k, npoly=12, rad_range=(1, 60))
    if k % 4 == 0:  # runs of white (level L - 1, or level L in literal mode)
        img[np.random.default_rng(k).random((h, w)) < 0.25] = 255
    check_case(img, r, L, bpp, pad, mode, cfg)


@pytest.mark.parametrize("r,L,cfg,status", [
    (3, 20, {"tile_w": 128, "path": 4}, B.OP_E_UNSUPPORTED),
    (15, 256, {"tile_w": 64, "path": 4}, B.OP_E_UNSUPPORTED),
    (1, 20, {"tile_w": 128, "cols_per_thread": 2, "path": 4}, B.OP_E_INVALID),
    (1, 20, {"tile_w": 48, "path": 4}, B.OP_E_INVALID),
])
def test_direct_path_refused_outside_its_range(r, L, cfg, status):
    with pytest.raises(B.OilPaintError) as e:
        OilPaint(100, 50, r, L, bpp=3, stride=300, config=cfg)
    assert e.value.status == status


@pytest.mark.parametrize("r,L", [(1, 20), (2, 256), (1, 256)])
def test_direct_path_whole_12mp_image(camera_12mp, r, L):
    """The 12 MP RGBA camera-like image through the direct path, every byte
    against the oracle."""
    buf, stride = camera_12mp
    w, h = 4000, 3000
    cfg = {"tile_w": 128, "chunk_rows": 4, "prefetch": 1, "path": 4}
    got = gpu_filter(buf, w, h, stride, 4, r, L, config=cfg)
    want = cpu_filter(buf, w, h, stride, 4, r, L)
    assert_same(got, want, w, h, stride, 4, f"12 MP direct r={r} L={L}")


def _column_path_cases(n=48, seed=13):
    """The column-histogram path (path 1, L <= 32): 1, 2 or 4 warps sweeping
    32 or 64 columns each, both bin variants (r <= 15 and above), every
    r mod 4, widths around the tile width."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(n):
        w = int(rng.choice([1, 2, 5, 31, 33, 63, 64, 65, 127, 128, 129, 200, 257, 400]))
        h = int(rng.choice([1, 2, 3, 9, 17, 64, 150]))
        r = int(rng.integers(0, 16)) if k < 32 else int(rng.integers(16, 45))
        L = int(rng.choice([1, 2, 3, 7, 16, 20, 31, 32]))
        bpp = int(rng.choice([3, 4]))
        pad = int(rng.choice([0, 1, 4, 13]))
        mode = int(rng.integers(0, 2))
        twk = int(rng.choice([1, 2]))
        nt = int(rng.choice([32, 64, 128]))
        cfg = {"tile_w": nt * twk, "tile_h": int(rng.choice([0, 1, 3, 16, 64])),
               "chunk_rows": int(rng.choice([1, 2, 3, 8])), "prefetch": int(rng.integers(1, 3)),
               "cols_per_thread": twk, "path": 1}
        cases.append((k, w, h, r, L, bpp, pad, mode, cfg))
    return cases


@pytest.mark.parametrize("k,w,h,r,L,bpp,pad,mode,cfg", _column_path_cases())
def test_fuzz_column_histograms(k, w, h, r, L, bpp, pad, mode, cfg):
    img = synth.camera_like(h, w, seed=1300 + k, npoly=12, rad_range=(1, 60)) if k % 2 else \
        synth.uniform_rgb(h, w, seed=1300 + k)
    try:
        check_case(img, r, L, bpp, pad, mode, cfg)
    except B.OilPaintError as e:
        # refused only when the halo box is wider than 256 columns
        assert e.status == B.OP_E_UNSUPPORTED, e
        assert cfg["tile_w"] + 2 * r + 3 > 256, (cfg, r)


# ---- edge cases --------------------------------------------------------------

@pytest.mark.parametrize("w,h,r,L", [
    (1, 1, 0, 1), (1, 1, 5, 256), (1, 37, 3, 20), (37, 1, 3, 20), (3, 2, 44, 20),
    (128, 128, 15, 256), (128, 128, 16, 256), (129, 65, 44, 256), (300, 45, 44, 1),
    (257, 33, 15, 20), (64, 300, 20, 32),
])
def test_edge_shapes(w, h, r, L):
    img = synth.camera_like(h, w, seed=w * 1000 + h, npoly=8, rad_range=(1, 50))
    check_case(img, r, L, bpp=3, pad=3)
    check_case(img, r, L, bpp=4, pad=0)


@pytest.mark.parametrize("w,h", [(65535, 3), (3, 65535)])
@pytest.mark.parametrize("r,L,cfg", [
    (44, 20, None),
    (15, 20, {"tile_w": 128, "cols_per_thread": 4, "chunk_rows": 2}),
    (20, 32, {"tile_w": 128, "cols_per_thread": 2, "chunk_rows": 4, "tile_h": 1}),
    (7, 64, {"tile_w": 64, "cols_per_thread": 1, "chunk_rows": 8}),
])
def test_maximum_dimensions(w, h, r, L, cfg):
    """Width or height at OP_MAX_DIM: the longest tile rows and columns, the
    most tiles per row (512 of 128 columns), and with one-row tiles the
    largest grid height the launch allows (65535)."""
    rng = np.random.default_rng(w + r)
    img = rng.integers(0, 256, (h, w, 3)).astype(np.uint8)
    img[rng.random((h, w)) < 0.3] = (40, 200, 90)  # runs of one level
    check_case(img, r, L, bpp=3, pad=5, config=cfg)


def test_constant_white_and_black():
    for colour in (255, 0):
        img = np.full((70, 90, 3), colour, np.uint8)
        for L in (1, 20, 256):
            check_case(img, 6, L)


def test_every_config_gives_the_same_bytes():
    img = synth.camera_like(233, 301, seed=9, npoly=30, rad_range=(3, 120))
    h, w = img.shape[:2]
    buf, stride = synth.to_strided(img, bpp=3, stride=w * 3 + 2)
    want = cpu_filter(buf, w, h, stride, 3, 9, 20)
    ran = ran8 = 0
    for nt in (32, 64, 96, 128):
        for cpt in (1, 2, 4, 8):
            if cpt == 8 and nt > 64:
                continue
            for ch in (1, 4, 8, 16):
                for pf in (1, 2, 4):
                    for th in (0, 1, 23, 233):
                        cfg = {"tile_w": nt * cpt, "tile_h": th, "chunk_rows": ch,
                               "prefetch": pf, "cols_per_thread": cpt}
                        try:
                            got = gpu_filter(buf, w, h, stride, 3, 9, 20, config=cfg)
                        except B.OilPaintError as e:
                            # the ring of halo copies does not fit shared memory
                            assert e.status == B.OP_E_UNSUPPORTED, e
                            assert ch * pf >= 16, cfg
                            continue
                        assert_same(got, want, w, h, stride, 3, str(cfg))
                        ran += 1
                        ran8 += cpt == 8
    # every one-column configuration (4 x 4 x 3 x 4) and every configuration
    # whose halo ring is small -- chunk rows x prefetch < 16: 6 of the 12
    # pairs -- runs (10 thread and column combinations of 2, 4 or 8 columns)
    assert ran >= 4 * 4 * 3 * 4 + 10 * 6 * 4 and ran8 >= 2 * 6 * 4


@pytest.mark.parametrize("cpt", [1, 2, 4])
@pytest.mark.parametrize("r,L", [(0, 20), (1, 7), (2, 20), (3, 32), (14, 20), (15, 20),
                                 (16, 20), (20, 32), (15, 256), (44, 64), (13, 3), (15, 33)])
def test_columns_per_thread_both_variants(cpt, r, L):
    """Both histogram variants, one column per thread and both difference-
    histogram widths, with every halo offset (r mod 4), on images whose
    width is not a tile multiple.  Two or four columns per thread are
    refused when L > 32 (and where the halo box or shared memory does not
    fit); with one column per thread, configurations beyond shared memory
    are skipped and one must run."""
    img = synth.camera_like(190, 270, seed=r * L + 1, npoly=25, rad_range=(3, 100))
    ran = 0
    for bpp, pad, nt, ch in ((4, 4, 64, 8), (3, 1, 32, 3)):
        try:
            check_case(img, r, L, bpp=bpp, pad=pad,
                       config={"tile_w": nt * cpt, "cols_per_thread": cpt, "chunk_rows": ch})
            ran += 1
        except B.OilPaintError as e:
            assert e.status == B.OP_E_UNSUPPORTED, e
    if cpt > 1 and L > 32:
        assert ran == 0
    elif cpt == 4:
        assert ran >= 1  # 64 threads x 4 columns: a 256+ box at r >= 1
    else:
        assert ran == 2 or cpt == 1 and ran >= 1


@pytest.mark.parametrize("w,h,r,L", [(300, 40, 15, 20), (301, 41, 14, 20), (97, 50, 13, 16)])
def test_border_threads_several_columns(w, h, r, L):
    """Images narrower than two tiles: most windows reach past an image
    edge into the zero words of the halo copy."""
    img = synth.uniform_rgb(h, w, seed=w + r)
    for nt, k in ((32, 2), (64, 2), (32, 4)):
        check_case(img, r, L, bpp=3, config={"tile_w": k * nt, "cols_per_thread": k})


def test_wide_halo_boxes():
    """Halo rows wider than the 256 elements of a TMA box dimension are copied
    through the three-dimensional view of the packed image (the padding words
    at the end of each packed row read as zero)."""
    for w, r, cfg in ((300, 1, {"tile_w": 256, "cols_per_thread": 2}),
                      (601, 15, {"tile_w": 512, "cols_per_thread": 4, "chunk_rows": 1}),
                      (1029, 13, {"tile_w": 512, "cols_per_thread": 8, "chunk_rows": 2}),
                      (333, 20, {"tile_w": 512, "cols_per_thread": 4, "chunk_rows": 1})):
        check_case(synth.camera_like(40, w, seed=w, npoly=20, rad_range=(2, 80)), r, 20,
                   config=cfg, what=f"{w} wide, r={r}, {cfg}")
        check_case(synth.uniform_rgb(23, w, seed=w), r, 20, bpp=4, pad=12, config=cfg)


def test_run_host_matches_oracle():
    img = synth.blobs_rgb(180, 250, seed=4, nblobs=10, sigma_range=(5, 40))
    h, w = img.shape[:2]
    buf, stride = synth.to_strided(img, bpp=4, stride=w * 4 + 8)
    op = OilPaint(w, h, 5, 20, bpp=4, stride=stride)
    out = np.full(buf.size, OUT_FILL, np.uint8)
    op.run_host(buf, out)
    op.close()
    assert_same(out, cpu_filter(buf, w, h, stride, 4, 5, 20), w, h, stride, 4, "run_host")


def test_run_host_async_pipelined_calls_match_oracle():
    """Five different images through one op back to back, without waiting in
    between: the two staging slots alternate and each call's copies overlap
    another call's filter.  Every output must still equal the oracle's."""
    w, h, r, L = 230, 150, 7, 20
    stride = w * 4 + 8
    op = OilPaint(w, h, r, L, bpp=4, stride=stride)
    ins, outs, wants = [], [], []
    for k in range(5):
        img = synth.camera_like(h, w, seed=700 + k, npoly=20, rad_range=(3, 90))
        buf, _ = synth.to_strided(img, bpp=4, stride=stride)
        wants.append(cpu_filter(buf, w, h, stride, 4, r, L))
        ins.append(torch.from_numpy(buf).pin_memory())
        outs.append(torch.full((buf.size,), OUT_FILL, dtype=torch.uint8).pin_memory())
    stream = torch.cuda.Stream()
    for k in range(5):
        op.run_host_async(ins[k], outs[k], stream)
    assert op.sync_status(stream) == B.OP_OK
    for k in range(5):
        assert_same(outs[k].numpy(), wants[k], w, h, stride, 4, f"async call {k}")
    # and the synchronous form after the asynchronous ones, same op
    out = np.full(ins[0].numel(), OUT_FILL, np.uint8)
    op.run_host(ins[0].numpy(), out)
    assert_same(out, wants[0], w, h, stride, 4, "run_host after async")
    op.close()


def test_invalid_calls_on_device():
    op = OilPaint(64, 32, 3, 20)
    src = torch.zeros(op.nbytes, dtype=torch.uint8, device="cuda")
    assert B.op_run(op.handle, src.data_ptr(), src.data_ptr(), None) == B.OP_E_INVALID
    assert B.op_run(op.handle, src.data_ptr(), src.data_ptr() + 16, None) == B.OP_E_INVALID
    assert B.op_set_workspace(op.handle, src.data_ptr(), 16) == B.OP_E_INVALID
    assert B.op_set_config(op.handle, B.op_config_t.make(48)) == B.OP_E_INVALID
    assert B.op_set_config(op.handle, B.op_config_t.make(64, cols_per_thread=3)) == B.OP_E_INVALID
    assert B.op_set_config(op.handle, B.op_config_t.make(96, cols_per_thread=2)) == B.OP_E_INVALID
    assert B.op_set_config(op.handle, B.op_config_t.make(64, chunk_rows=40)) == B.OP_E_INVALID
    op.close()


def test_bounded_wait_times_out_and_context_survives():
    """A wait on an mbarrier nothing completes gives up after the limit and
    reports OP_E_TIMEOUT; the context keeps working afterwards."""
    assert B.op_selftest_wait_timeout(20_000_000, None) == B.OP_E_TIMEOUT
    check_case(synth.uniform_rgb(50, 60, seed=6), 2, 20)
