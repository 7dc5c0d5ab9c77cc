"""The persistent batched kernel: mixed images in one launch, eagerly and
replayed from a CUDA graph, against the CPU oracle and against solo runs."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from paper_1405_1020_gb300 import binding as B
from paper_1405_1020_gb300 import batchbench, synth
from paper_1405_1020_gb300.filter import TUNING_TABLE, Batch, OilPaint, load_tuning
from tests.pins import OUT_FILL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def make_images(n, seed, max_r=44, levels=(1, 3, 16, 20, 32, 64, 256)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        w = int(rng.integers(1, 260))
        h = int(rng.integers(1, 180))
        r = int(rng.choice([v for v in (0, 1, 2, 5, 15, 16, 20, 44) if v <= max_r]))
        L = int(rng.choice(levels))
        bpp = int(rng.choice([3, 4]))
        pad = int(rng.choice([0, 1, 8]))
        mode = int(rng.integers(0, 2))
        img = synth.camera_like(h, w, seed=seed * 100 + i, npoly=10, rad_range=(2, 80))
        buf, stride = synth.to_strided(img, bpp=bpp, stride=w * bpp + pad)
        out.append(dict(buf=buf, w=w, h=h, stride=stride, bpp=bpp, r=r, L=L, mode=mode))
    return out


def to_device(images):
    for im in images:
        im["src"] = torch.from_numpy(im["buf"]).cuda()
        im["dst"] = torch.full_like(im["src"], OUT_FILL)
    torch.cuda.synchronize()  # the fills ran on the default stream
    return [(im["src"], im["dst"], im["w"], im["h"], im["stride"], im["bpp"], im["r"], im["L"],
             im["mode"]) for im in images]


def oracle_out(im):
    out = np.full(im["buf"].size, OUT_FILL, np.uint8)
    return oracle.oilpaint(im["buf"], im["w"], im["h"], im["stride"], im["bpp"], im["r"],
                           im["L"], mode=im["mode"], out=out)


def check_all(images, what):
    torch.cuda.synchronize()
    for k, im in enumerate(images):
        got = im["dst"].cpu().numpy()
        want = oracle_out(im)
        assert np.array_equal(got, want), (
            f"{what}: image {k} ({im['w']}x{im['h']} r={im['r']} L={im['L']} bpp={im['bpp']})")


def reset(images):
    for im in images:
        im["dst"].fill_(OUT_FILL)
    torch.cuda.synchronize()


def new_batch(images, max_images=64, cfg=None):
    pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
    return Batch(max_images, max(pix, 1) + 4096, 44, 256, config=cfg)


def test_mixed_batch_eager_and_graph():
    images = make_images(24, seed=1)
    descs = to_device(images)
    b = new_batch(images)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.set(descs, stream)
        b.run(stream)
    assert b.sync_status(stream) == B.OP_OK
    check_all(images, "eager")
    reset(images)
    b.capture(stream)
    b.launch_graph(stream)
    assert b.sync_status(stream) == B.OP_OK
    check_all(images, "graph")
    # a different batch through the same graph: the tables are device-resident
    other = make_images(17, seed=2)
    d2 = to_device(other)
    # capacity of the first batch's workspace must hold the second
    if Batch.padded_pixels([(im["w"], im["h"]) for im in other]) <= \
            Batch.padded_pixels([(im["w"], im["h"]) for im in images]) + 4096:
        b.set(d2, stream)
        b.launch_graph(stream)
        assert b.sync_status(stream) == B.OP_OK
        check_all(other, "graph, second batch")
    b.close()


@pytest.mark.parametrize("cfg", [None,
                                 {"tile_w": 64, "chunk_rows": 4, "prefetch": 2},
                                 {"tile_w": 128, "chunk_rows": 16, "prefetch": 1,
                                  "cols_per_thread": 2},
                                 {"tile_w": 128, "chunk_rows": 8, "prefetch": 2,
                                  "cols_per_thread": 4}])
def test_batch_equals_solo_runs(cfg):
    images = make_images(12, seed=3, max_r=20, levels=(16, 20, 32))
    descs = to_device(images)
    pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
    try:
        b = Batch(16, pix + 64, 20, 32, config=cfg)
    except B.OilPaintError as e:
        assert e.status == B.OP_E_UNSUPPORTED
        pytest.skip("configuration does not fit this device")
    b.set(descs)
    b.run()
    assert b.sync_status() == B.OP_OK
    torch.cuda.synchronize()
    for im in images:
        solo = torch.full_like(im["src"], OUT_FILL)
        op = OilPaint(im["w"], im["h"], im["r"], im["L"], bpp=im["bpp"], stride=im["stride"],
                      flags=im["mode"])
        op.run(im["src"], solo)
        assert op.sync_status() == B.OP_OK
        op.close()
        assert torch.equal(solo, im["dst"])
    b.close()


def test_empty_batch_and_reuse():
    b = Batch(4, 10000, 5, 20)
    b.set([])
    b.run()
    assert b.sync_status() == B.OP_OK
    images = make_images(3, seed=4, max_r=5, levels=(20,))
    # keep the set inside the 10000-pixel capacity
    small = [im for im in images if ((im["w"] + 3) // 4 * 4) * im["h"] <= 3000]
    if small:
        descs = to_device(small)
        b.set(descs)
        b.run()
        assert b.sync_status() == B.OP_OK
        check_all(small, "after empty batch")
    b.close()


def test_strided_crops_with_packed_outputs():
    """Inputs that are crops of a larger image (its row pitch) written to
    packed outputs (a different pitch), as the server does."""
    big = synth.camera_like(300, 500, seed=12, npoly=30, rad_range=(5, 150))
    pool = torch.from_numpy(big.reshape(300, -1)).cuda()
    pstride = 500 * 3
    rng = np.random.default_rng(13)
    crops = []
    for i in range(10):
        w, h = int(rng.integers(1, 200)), int(rng.integers(1, 120))
        x0, y0 = int(rng.integers(0, 500 - w + 1)), int(rng.integers(0, 300 - h + 1))
        if i == 0:  # a crop ending at the pool's last byte
            w, h, x0, y0 = 77, 40, 500 - 77, 300 - 40
        crops.append((w, h, x0, y0, int(rng.choice([2, 7, 15])), 20))
    descs, outs = [], []
    for w, h, x0, y0, r, L in crops:
        src = pool.view(-1)[y0 * pstride + x0 * 3:]
        out = torch.full((w * h * 3,), OUT_FILL, dtype=torch.uint8, device="cuda")
        outs.append(out)
        descs.append((src, out, w, h, pstride, 3, r, L, 0, w * 3))
    torch.cuda.synchronize()
    b = Batch(16, 200000, 15, 20)
    b.set(descs)
    b.run()
    assert b.sync_status() == B.OP_OK
    torch.cuda.synchronize()
    for (w, h, x0, y0, r, L), out in zip(crops, outs):
        crop = np.ascontiguousarray(big[y0:y0 + h, x0:x0 + w])
        want = oracle.oilpaint(crop.reshape(-1), w, h, w * 3, 3, r, L,
                               out=np.full(w * h * 3, OUT_FILL, np.uint8))
        assert np.array_equal(out.cpu().numpy(), want), (w, h, x0, y0, r)
    b.close()


def test_batch_rejects_invalid_sets():
    img = torch.zeros(30 * 20 * 3, dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(img)
    b = Batch(2, 4096, 5, 20)
    ok = (img, out, 30, 20, 90, 3, 5, 20)
    with pytest.raises(B.OilPaintError) as e:
        b.set([ok, ok, ok])  # more than max_images
    assert e.value.status == B.OP_E_INVALID
    with pytest.raises(B.OilPaintError):
        b.set([(img, out, 30, 20, 90, 3, 6, 20)])  # radius above the batch maximum
    with pytest.raises(B.OilPaintError):
        b.set([(img, out, 30, 20, 90, 3, 5, 21)])  # levels above the batch maximum
    with pytest.raises(B.OilPaintError):
        b.set([(img, img, 30, 20, 90, 3, 5, 20)])  # in == out
    big = torch.zeros(100 * 50 * 3, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.OilPaintError):
        b.set([(big, torch.zeros_like(big), 100, 50, 300, 3, 5, 20)])  # over the pixel capacity
    b.set([ok])
    b.run()
    assert b.sync_status() == B.OP_OK
    b.close()


@pytest.mark.parametrize("radii", [(16, 20, 44), (0, 2, 15)], ids=["large-only", "small-only"])
def test_batch_with_one_radius_group_empty(radii):
    """A batch created for radii up to 44 (and 32 levels) runs r <= 15 and
    r > 15 in separate groups; either radius side may be empty in a set."""
    images = make_images(9, seed=11 + radii[0], max_r=44, levels=(16, 20, 32))
    rng = np.random.default_rng(radii[1])
    for im in images:
        im["r"] = int(rng.choice(radii))
    descs = to_device(images)
    pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
    b = Batch(16, pix + 64, 44, 32,
              config={"tile_w": 64, "chunk_rows": 2, "prefetch": 1, "cols_per_thread": 2})
    stream = torch.cuda.Stream()
    b.set(descs, stream)
    b.capture(stream)
    b.launch_graph(stream)
    assert b.sync_status(stream) == B.OP_OK
    check_all(images, f"radii {radii}")
    b.close()


def test_four_groups_and_each_group_empty_in_turn():
    """A batch created for radii up to 20 and 32 levels splits its images by
    radius (above 15 or not) and level count (above 20 or not) into four
    groups, each with its own launch configuration; one captured graph
    serves sets in which any one group is empty."""
    images = make_images(16, seed=23, max_r=20, levels=(3, 16, 20, 32))
    for k, im in enumerate(images):  # every group populated
        im["r"] = (2, 15, 16, 20)[k % 4] if k < 8 else im["r"]
        im["L"] = (16, 32)[(k // 4) % 2] if k < 8 else im["L"]
    descs = to_device(images)
    pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
    b = Batch(16, pix + 4096, 20, 32)
    groups = b.groups()
    assert [(g["max_radius"], g["max_levels"]) for g in groups] == [
        (15, 20), (15, 32), (20, 20), (20, 32)]
    assert all(g["config"]["path"] == 0 for g in groups)
    stream = torch.cuda.Stream()
    b.set(descs, stream)
    b.capture(stream)
    b.launch_graph(stream)
    assert b.sync_status(stream) == B.OP_OK
    check_all(images, "four groups")

    def group(im):
        return 2 * (im["r"] > 15) + (im["L"] > 20)

    for g in range(4):
        keep = [k for k, im in enumerate(images) if group(im) != g]
        sub = [images[k] for k in keep]
        reset(sub)
        b.set([descs[k] for k in keep], stream)
        b.launch_graph(stream)
        assert b.sync_status(stream) == B.OP_OK
        check_all(sub, f"group {g} empty")
    b.close()


def test_one_config_for_every_group():
    """A configuration given at creation applies to every group."""
    cfg = {"tile_w": 128, "chunk_rows": 2, "prefetch": 1, "cols_per_thread": 4}
    b = Batch(4, 100000, 44, 64, config=cfg)
    groups = b.groups()
    assert len(groups) == 4
    for g in groups:
        c = g["config"]
        assert (c["tile_w"], c["chunk_rows"], c["prefetch"], c["cols_per_thread"]) == (128, 2, 1, 4)
    assert [(g["max_radius"], g["max_levels"]) for g in groups] == [
        (15, 20), (15, 64), (44, 20), (44, 64)]
    b.close()
    b1 = Batch(4, 100000, 15, 20, config=cfg)
    assert len(b1.groups()) == 1
    b1.close()


def test_batch_tune_table_entry_is_used_where_it_fits():
    """op_batch_create (cfg NULL) takes a group's configuration from the
    batch tuning table when the entry fits the group's largest image in one
    CTA, and falls back to another configuration when it does not."""
    want = {"tile_w": 64, "chunk_rows": 4, "prefetch": 1, "cols_per_thread": 1}
    # 4 columns of 128 threads at r = 44 with 32-row halo chunks, 4 in flight:
    # the ring of halo copies alone exceeds a CTA's shared memory
    wide = {"tile_w": 512, "chunk_rows": 32, "prefetch": 4, "cols_per_thread": 4}
    try:
        B.check(B.op_batch_tune_table_set(15, 20, B.op_config_t.make(**want)), "set")
        b = Batch(4, 100000, 20, 20)
        g = b.groups()
        assert [(x["max_radius"], x["max_levels"]) for x in g] == [(15, 20), (20, 20)]
        got = g[0]["config"]
        assert {k: got[k] for k in want} == want
        b.close()
        B.check(B.op_batch_tune_table_set(44, 32, B.op_config_t.make(**wide)), "set")
        b = Batch(4, 100000, 44, 32)
        got = b.groups()[3]["config"]
        assert (got["tile_w"], got["cols_per_thread"]) != (512, 4)
        b.close()
    finally:
        B.op_batch_tune_table_set(15, 20, None)
        B.op_batch_tune_table_set(44, 32, None)
        load_tuning(TUNING_TABLE)


def test_benchmark_batch_64_images_equal_oracle():
    """The measured mixed batch (64 camera-like RGB images, log-uniform
    320x240..4000x3000 pixels, r in {2,4,8,12,20}, L in {16,20,32}), run the
    way the benchmark runs it -- one graph replay of the grouped persistent
    launches -- against the oracle on every byte of every image."""
    images = batchbench.make_batch(synth.batch_specs(n=64), batchbench.make_pool())
    outs = [torch.full_like(im["src"], OUT_FILL) for im in images]
    torch.cuda.synchronize()
    pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
    b = Batch(64, pix + 4096, max(im["r"] for im in images), max(im["L"] for im in images))
    stream = torch.cuda.Stream()
    try:
        b.set([(im["src"], o, im["w"], im["h"], im["stride"], 3, im["r"], im["L"])
               for im, o in zip(images, outs)], stream)
        b.capture(stream)
        b.launch_graph(stream)
        assert b.sync_status(stream) == B.OP_OK
        assert len(b.groups()) == 4
    finally:
        b.close()
    for k, (im, o) in enumerate(zip(images, outs)):
        buf = im["src"].cpu().numpy()
        want = np.full(buf.size, OUT_FILL, np.uint8)
        oracle.oilpaint(buf, im["w"], im["h"], im["stride"], 3, im["r"], im["L"], out=want)
        assert np.array_equal(o.cpu().numpy(), want), (
            f"image {k} ({im['w']}x{im['h']} r={im['r']} L={im['L']}) differs from the oracle")
