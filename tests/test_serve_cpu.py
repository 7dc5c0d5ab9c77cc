"""Host-side logic of the server: admission under the HBM cap, refusal of
requests that can never fit, round forming, release.  No GPU."""
from paper_1405_1020_gb300 import serve, synth
from paper_1405_1020_gb300.serve import Admission, Ticket


def req(w, h, t=0.0):
    return synth.Request(t, w, h, 3, 20, 0, 0, 0)


def test_admission_respects_cap_and_order():
    one = serve.request_bytes(1000, 1000)
    adm = Admission(cap_bytes=int(2.5 * one), max_round_images=8, max_round_pixels=10**8)
    ts = [Ticket(req(1000, 1000), i) for i in range(4)]
    for t in ts:
        adm.arrive(t)
    got = adm.admit()
    assert [t.rid for t in got] == [0, 1]  # the third would pass the cap
    assert adm.reserved == 2 * one and adm.peak_reserved == 2 * one
    rnd = adm.next_round()
    assert [t.rid for t in rnd] == [0, 1]
    adm.release(rnd[0])
    assert [t.rid for t in adm.admit()] == [2]  # capacity freed by the release
    assert [t.rid for t in adm.waiting] == [3]


def test_refuses_what_can_never_fit():
    adm = Admission(cap_bytes=serve.request_bytes(100, 100), max_round_images=4,
                    max_round_pixels=10**6)
    big = Ticket(req(200, 200), 0)
    adm.arrive(big)
    assert big.error and adm.refused == [big] and not adm.waiting
    wide = Ticket(req(2000, 1000), 1)
    adm2 = Admission(cap_bytes=10**12, max_round_images=4, max_round_pixels=10**6)
    adm2.arrive(wide)
    assert wide.error


def test_round_limits():
    adm = Admission(cap_bytes=10**12, max_round_images=3, max_round_pixels=serve.padded_pixels(100, 100) * 2)
    for i in range(5):
        adm.arrive(Ticket(req(100, 100), i))
    adm.admit()
    assert [t.rid for t in adm.next_round()] == [0, 1]  # pixel limit
    assert [t.rid for t in adm.next_round()] == [2, 3]
    assert [t.rid for t in adm.next_round()] == [4]
    assert adm.next_round() == []


def test_free_memory_gate():
    free = [serve.request_bytes(500, 500) + 1000]
    adm = Admission(cap_bytes=10**12, max_round_images=8, max_round_pixels=10**8,
                    free_bytes=lambda: free[0], headroom=0)
    for i in range(3):
        adm.arrive(Ticket(req(500, 500), i))
    assert [t.rid for t in adm.admit()] == [0]
    free[0] = 10**12
    assert [t.rid for t in adm.admit()] == [1, 2]


def test_poisson_requests_shape():
    rs = synth.poisson_requests(100.0, 2.0, seed=4, pool_shapes=((4400, 6600),))
    assert 120 < len(rs) < 280
    assert all(0.1e6 * 0.9 <= r.width * r.height <= 24e6 * 1.01 for r in rs)
    assert all(r.x0 + r.width <= 6600 and r.y0 + r.height <= 4400 for r in rs)
    assert all(1 <= r.radius <= 20 for r in rs)
    assert [r.t_arrival for r in rs] == sorted(r.t_arrival for r in rs)


def test_overlapping_rounds_counts_cross_stream_overlap_only():
    # (stream slot, images, start ms, done ms)
    spans = [(0, 3, 0.0, 2.0), (1, 2, 1.0, 3.0),   # overlap across streams
             (0, 1, 2.5, 4.0),                     # overlaps round 1
             (0, 4, 5.0, 6.0), (0, 1, 5.5, 7.0),   # same stream: not counted
             (1, 2, 7.0, 8.0)]                     # starts when the last ends
    assert serve.overlapping_rounds(spans) == 3
    assert serve.overlapping_rounds([]) == 0
    assert serve.overlapping_rounds([(0, 1, 0.0, 1.0), (1, 1, 1.0, 2.0)]) == 0
