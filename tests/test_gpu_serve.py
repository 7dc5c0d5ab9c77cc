"""The served path: a continuously batched session whose rounds hold several
requests and overlap on the device, with every request's output equal to the
oracle's filter of its crop."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from paper_1405_1020_gb300 import serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _oracle_crop(img, q):
    crop = np.ascontiguousarray(img[q.y0:q.y0 + q.height, q.x0:q.x0 + q.width])
    buf = crop.reshape(-1)
    return oracle.oilpaint(buf, q.width, q.height, q.width * 3, 3, q.radius, q.levels)


def test_session_equals_oracle_with_batched_overlapping_rounds():
    pool_shape = (2400, 3200)
    img = synth.camera_like(*pool_shape, seed=9, npoly=60, rad_range=(5, 300))
    pool = [torch.from_numpy(img.reshape(pool_shape[0], -1)).cuda()]
    # A burst of large requests (about 50 arriving within 1 ms): each round's
    # kernels run longer than the host takes to form the next round, so the
    # two streams' rounds overlap on the device, and requests that arrive
    # while both streams are busy wait and are batched into one round.
    reqs = synth.poisson_requests(50000.0, 0.001, seed=11, pmin=1e6, pmax=5e6, rmin=2, rmax=6,
                                  pool_shapes=(pool_shape,))
    assert len(reqs) >= 30
    server = serve.OilPaintServer(pool, max_radius=6, max_levels=20, max_round_images=4,
                                  max_round_mpix=20.0)
    try:
        tickets, info = server.serve(reqs, sample_every=1)
    finally:
        server.close()
    assert all(t.t_done is not None and t.error is None for t in tickets)
    # every served output against the oracle on the request's crop
    for t in tickets:
        got = t.out.cpu().numpy()
        assert np.array_equal(got, _oracle_crop(img, t.req)), (
            f"request {t.rid} ({t.req.width}x{t.req.height} r={t.req.radius}) differs "
            f"from the oracle")
    # continuous batching: rounds of several requests, rounds of the two
    # streams in flight on the device at the same time
    sizes = info["round_sizes"]
    assert sum(sizes) == len(tickets)
    assert max(sizes) >= 2, sizes
    spans = info["round_spans"]
    assert len(spans) == info["rounds"]
    assert {s[0] for s in spans} == {0, 1}
    assert serve.overlapping_rounds(spans) >= 2, spans
    st = serve.summarize(tickets, info, 0.0, 0.0)
    assert st.max_round_images == max(sizes) and st.overlapping_rounds >= 2
    assert st.p50_ms > 0 and st.p99_ms >= st.p50_ms


def test_sampled_requests_equal_solo_runs():
    """The benchmark's resampling check (a request re-run alone through
    op_run) on a short session of small requests."""
    pool_shape = (900, 1200)
    img = synth.camera_like(*pool_shape, seed=10, npoly=40, rad_range=(5, 200))
    pool = [torch.from_numpy(img.reshape(pool_shape[0], -1)).cuda()]
    reqs = synth.poisson_requests(400.0, 0.3, seed=12, pmin=2e3, pmax=3e5, rmin=1, rmax=8,
                                  pool_shapes=(pool_shape,))
    server = serve.OilPaintServer(pool, max_radius=8, max_levels=20, max_round_images=16,
                                  max_round_mpix=2.0)
    try:
        tickets, info = server.serve(reqs, sample_every=1)
        assert serve.check_samples(server, tickets) == len(tickets)
    finally:
        server.close()
