"""The served path: every request of a continuously batched session equals
the same request run alone."""
import pytest
import torch

import __graft_entry__
from paper_1405_1020_gb300 import serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_session_results_equal_solo_runs():
    pool_shape = (900, 1200)
    img = synth.camera_like(*pool_shape, seed=9, npoly=40, rad_range=(5, 200))
    pool = [torch.from_numpy(img.reshape(pool_shape[0], -1)).cuda()]
    # high rate, small images: rounds hold several requests and overlap
    reqs = synth.poisson_requests(400.0, 0.5, seed=11, pmin=2e3, pmax=3e5, rmin=1, rmax=8,
                                  pool_shapes=(pool_shape,))
    server = serve.OilPaintServer(pool, max_radius=8, max_levels=20, max_round_images=16,
                                  max_round_mpix=2.0)
    try:
        tickets, info = server.serve(reqs, sample_every=1)
        assert all(t.t_done is not None for t in tickets)
        assert info["rounds"] >= 2
        assert serve.check_samples(server, tickets) == len(tickets)
        st = serve.summarize(tickets, info, 0.0, 0.0)
        assert st.p50_ms > 0 and st.p99_ms >= st.p50_ms
    finally:
        server.close()
