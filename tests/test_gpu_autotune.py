"""The launch-configuration autotuner on the GPU: every candidate it times
writes the oracle's bytes, and the configuration it records is the one the
library then uses."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from paper_1405_1020_gb300 import autotune, synth
from paper_1405_1020_gb300 import binding as B
from paper_1405_1020_gb300.filter import Batch, OilPaint

pytestmark = pytest.mark.gpu

FIELDS = ("tile_w", "tile_h", "chunk_rows", "prefetch", "cols_per_thread", "path")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _pixels(buf, w, h, stride, bpp):
    return np.asarray(buf).reshape(-1)[: h * stride].reshape(h, stride)[:, : w * bpp]


def test_tune_image_candidates_equal_oracle_and_winner_becomes_default():
    # (r, L) = (7, 13): a pair no other test and no committed table entry uses
    w, h, r, L = 333, 211, 7, 13
    img = synth.camera_like(h, w, seed=77, npoly=30, rad_range=(3, 100))
    buf, stride = synth.to_strided(img, bpp=3, stride=w * 3 + 1)
    want = _pixels(oracle.oilpaint(buf, w, h, stride, 3, r, L), w, h, stride, 3)
    cands = [
        {"tile_w": 64, "tile_h": 0, "chunk_rows": 4, "prefetch": 1, "cols_per_thread": 1,
         "path": 0},
        {"tile_w": 128, "tile_h": 0, "chunk_rows": 2, "prefetch": 1, "cols_per_thread": 4,
         "path": 0},
        {"tile_w": 64, "tile_h": 17, "chunk_rows": 2, "prefetch": 2, "cols_per_thread": 2,
         "path": 0},
        {"tile_w": 96, "tile_h": 0, "chunk_rows": 8, "prefetch": 2, "cols_per_thread": 1,
         "path": 0},
        {"tile_w": 64, "tile_h": 0, "chunk_rows": 2, "prefetch": 1, "cols_per_thread": 2,
         "path": 1},
    ]
    verified = []

    def verify(cfg, dst):
        got = _pixels(dst.cpu().numpy(), w, h, stride, 3)
        assert np.array_equal(got, want), f"candidate {cfg} differs from the oracle"
        verified.append(cfg)

    src = torch.from_numpy(buf).cuda()
    res = autotune.tune_image(w, h, 3, stride, r, L, src=src, reps=3, cands=cands,
                              verify=verify)
    assert verified == cands and len(res["results"]) == len(cands)
    assert res["config"] in cands
    assert res["ms"] == min(x["ms"] for x in res["results"])
    # op_default_config and a new op now take the recorded winner
    c = B.op_config_t()
    B.check(B.op_default_config(r, L, c), "op_default_config")
    assert {k: c.as_dict()[k] for k in FIELDS} == {k: res["config"][k] for k in FIELDS}
    op = OilPaint(w, h, r, L, bpp=3, stride=stride)
    try:
        got_cfg = op.config()
        assert all(got_cfg[k] == res["config"][k] for k in FIELDS if k != "tile_h")
        dst = torch.zeros_like(src)
        op.run(src, dst)
        assert op.sync_status() == B.OP_OK
        assert np.array_equal(_pixels(dst.cpu().numpy(), w, h, stride, 3), want)
    finally:
        op.close()


def test_tune_batch_winner_is_used_and_equals_oracle():
    # max radius 9, max levels 20: one group, keyed (9, 20), used by no other test
    specs = [(300, 200, 2, 13), (410, 150, 9, 20), (129, 257, 5, 16), (64, 64, 9, 7)]
    images = []
    for k, (w, h, r, L) in enumerate(specs):
        img = synth.camera_like(h, w, seed=300 + k, npoly=20, rad_range=(3, 90))
        buf, stride = synth.to_strided(img, bpp=3)
        images.append(dict(buf=buf, src=torch.from_numpy(buf).cuda(), w=w, h=h, stride=stride,
                           bpp=3, r=r, L=L))
    cands = [{"tile_w": nt * cpt, "tile_h": 0, "chunk_rows": ch, "prefetch": 1,
              "cols_per_thread": cpt, "path": 0}
             for nt, cpt, ch in ((64, 2, 2), (32, 4, 1), (128, 1, 4))]
    try:
        res = autotune.tune_batch(images, 9, 20, reps=3, cands=cands)
        assert list(res["groups"]) == ["9,20"]
        best = res["groups"]["9,20"]["config"]
        # the winner is a candidate, or the group's untuned default when no
        # candidate beat it; either way it is recorded in the batch table
        assert best in cands or res["ms"] == res["ms_untuned"]
        assert res["ms"] <= res["ms_untuned"]
        pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
        b = Batch(len(images), pix + 4096, 9, 20)
        stream = torch.cuda.Stream()
        outs = [torch.zeros_like(im["src"]) for im in images]
        torch.cuda.synchronize()
        try:
            g = b.groups()
            assert len(g) == 1
            assert all(g[0]["config"][f] == best[f]
                       for f in ("tile_w", "chunk_rows", "prefetch", "cols_per_thread"))
            b.set([(im["src"], o, im["w"], im["h"], im["stride"], 3, im["r"], im["L"])
                   for im, o in zip(images, outs)], stream)
            b.capture(stream)
            b.launch_graph(stream)
            assert b.sync_status(stream) == B.OP_OK
        finally:
            b.close()
        for im, o in zip(images, outs):
            want = oracle.oilpaint(im["buf"], im["w"], im["h"], im["stride"], 3, im["r"], im["L"])
            assert np.array_equal(o.cpu().numpy(), want), (im["w"], im["h"], im["r"], im["L"])
    finally:
        B.check(B.op_batch_tune_table_set(9, 20, None), "op_batch_tune_table_set")
