"""The channel-mean division of the r <= 15 kernels, checked exhaustively.

The kernels divide a channel sum n < 2^18 (at most 961 pixels of 255) by a
count d in 1..961 with Granlund and Montgomery's multiply-high method:
m = ceil(2^31 / d), q = floor(2n * m / 2^32).  This replays that arithmetic
in exact integers for every (n, d) pair the kernels can meet and compares it
with floor division.
"""
import numpy as np


def test_multiply_high_division_is_exact():
    n = np.arange(1 << 18, dtype=np.uint64)
    for d in range(1, 962):
        m = np.uint64(((1 << 31) + d - 1) // d)
        q = ((n << np.uint64(1)) * m) >> np.uint64(32)
        bad = np.nonzero(q != n // np.uint64(d))[0]
        assert bad.size == 0, f"d={d}: first mismatch at n={int(bad[0])}"
