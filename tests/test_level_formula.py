"""Section 4's intensity level, pinned exhaustively.

The paper computes ((r+g+b)*intensity_level/3.0)/255 in double precision and
truncates it to int.  For every R+G+B in 0..765 and L in 1..256 that equals
floor((R+G+B)*L/765); it reaches L only for R+G+B = 765 (pure white), which
both oracles clamp to L-1.
"""
import numpy as np

import oracle
from oracle import oilpaint_np as onp


def paper_double_level(s: int, L: int) -> int:
    # the paper's expression with IEEE doubles, truncated toward zero
    return int(((s * L) / 3.0) / 255)


def test_paper_double_expression_is_the_integer_quotient():
    for L in range(1, 257):
        for s in range(766):
            assert paper_double_level(s, L) == (s * L) // 765
    # only pure white reaches level L
    hits = [(s, L) for L in range(1, 257) for s in range(766) if (s * L) // 765 >= L]
    assert all(s == 765 for s, _ in hits) and len(hits) == 256


def test_oracle_levels_exhaustive_both_modes():
    s = np.arange(766)
    rgb = np.zeros((766, 1, 3), np.int64)
    rgb[:, 0, 0] = np.minimum(s, 255)
    rgb[:, 0, 1] = np.minimum(np.maximum(s - 255, 0), 255)
    rgb[:, 0, 2] = np.maximum(s - 510, 0)
    assert (rgb.sum(-1)[:, 0] == s).all()
    for L in range(1, 257):
        want_paper = np.minimum([paper_double_level(int(v), L) for v in s], L - 1)
        want_div3 = np.minimum((s // 3) * L // 255, L - 1)
        assert np.array_equal(onp.level_map(rgb, L, 0)[:, 0], want_paper)
        assert np.array_equal(onp.level_map(rgb, L, 1)[:, 0], want_div3)
        for v in (0, 1, 76, 77, 254, 255, 382, 383, 510, 764, 765):
            assert oracle.level_of_sum(v, L, 0) == want_paper[v]
            assert oracle.level_of_sum(v, L, 1) == want_div3[v]


def test_mode_example_from_the_readings():
    # R+G+B = 77, L = 20: 77*20/765 = 2.01 -> 2; floor(77/3)*20/255 = 1.96 -> 1
    assert oracle.level_of_sum(77, 20, 0) == 2
    assert oracle.level_of_sum(77, 20, 1) == 1
    assert oracle.level_of_sum(765, 256, 0) == 255
    assert oracle.level_of_sum(765, 1, 0) == 0
