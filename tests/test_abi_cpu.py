"""The C-ABI library builds, loads and exports every declared entry point;
argument checks that happen before any CUDA call behave.  No GPU needed."""
import re
import os

import pytest

from paper_1405_1020_gb300 import binding as B
from paper_1405_1020_gb300.csrc import build as cbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "oilpaint.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(op_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    cbuild.build()
    return B.load()


def test_header_and_binding_agree():
    assert sorted(B.EXPORTS) == declared_functions()


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for st, word in ((0, "ok"), (-1, "invalid"), (-2, "CUDA"), (-3, "memory"), (-4, "timed out"),
                     (-5, "unsupported"), (-6, "bounds")):
        assert word in B.op_status_string(st)


@pytest.mark.parametrize("args", [
    (0, 10, 30, 3, 1, 20, 0),        # width 0
    (10, 0, 30, 3, 1, 20, 0),        # height 0
    (10, 10, 29, 3, 1, 20, 0),       # stride < width*bpp
    (10, 10, 30, 5, 1, 20, 0),       # bpp 5
    (10, 10, 30, 3, -1, 20, 0),      # radius < 0
    (10, 10, 30, 3, 45, 20, 0),      # radius > OP_MAX_RADIUS
    (10, 10, 30, 3, 1, 0, 0),        # L = 0
    (10, 10, 30, 3, 1, 257, 0),      # L > 256
    (10, 10, 30, 3, 1, 20, 8),       # unknown flag (bit 3)
    (10, 10, 30, 3, 1, 255, 2),      # literal mode with L > OP_LITERAL_MAX_LEVELS
    (70000, 10, 210000, 3, 1, 20, 0),  # width > OP_MAX_DIM
])
def test_create_rejects_invalid_arguments(lib, args):
    assert not B.op_create_ex(*args)
    assert B.op_last_error() == B.OP_E_INVALID


def test_null_handles(lib):
    assert B.op_destroy(None) == B.OP_OK
    assert B.op_batch_destroy(None) == B.OP_OK
    assert B.op_run(None, 1, 2, None) == B.OP_E_INVALID
    assert B.op_run_host(None, 1, 2, None) == B.OP_E_INVALID
    assert B.op_run_host_async(None, 1, 2, None) == B.OP_E_INVALID
    assert B.op_sync_status(None, None) == B.OP_E_INVALID
    assert B.op_workspace_size(None) == 0
    assert B.op_batch_workspace_size(None) == 0
    assert B.op_batch_run(None, None) == B.OP_E_INVALID
    assert B.op_batch_launch_graph(None, None) == B.OP_E_INVALID
    cfg = B.op_config_t()
    assert B.op_get_config(None, cfg) == B.OP_E_INVALID


def test_tune_table_validation(lib):
    assert B.op_tune_table_set(3, 20, B.op_config_t.make(48)) == B.OP_E_INVALID
    assert B.op_tune_table_set(3, 20, B.op_config_t.make(96, cols_per_thread=2)) == B.OP_E_INVALID
    assert B.op_tune_table_set(3, 20, B.op_config_t.make(64, cols_per_thread=3)) == B.OP_E_INVALID
    assert B.op_tune_table_set(3, 20, B.op_config_t.make(64, chunk_rows=0)) == B.OP_E_INVALID
    assert B.op_tune_table_set(3, 20, B.op_config_t.make(64, prefetch=5)) == B.OP_E_INVALID
    assert B.op_tune_table_set(99, 20, B.op_config_t.make(64)) == B.OP_E_INVALID
    assert B.op_tune_table_set(3, 20, B.op_config_t.make(64, 32, 4, 2)) == B.OP_OK


def test_batch_tune_table_validation(lib):
    set_ = B.op_batch_tune_table_set
    assert set_(15, 20, B.op_config_t.make(48)) == B.OP_E_INVALID
    assert set_(-1, 20, B.op_config_t.make(64)) == B.OP_E_INVALID
    assert set_(45, 20, B.op_config_t.make(64)) == B.OP_E_INVALID
    assert set_(15, 0, B.op_config_t.make(64)) == B.OP_E_INVALID
    assert set_(15, 257, B.op_config_t.make(64)) == B.OP_E_INVALID
    # the persistent kernel keeps one histogram set per thread: no column path
    assert set_(15, 20, B.op_config_t.make(64, path=1)) == B.OP_E_INVALID
    assert set_(15, 20, B.op_config_t.make(128, 0, 2, 1, 2)) == B.OP_OK
    assert set_(15, 20, None) == B.OP_OK  # removes the entry


def test_selftest_rejects_bad_timeout(lib):
    assert B.op_selftest_wait_timeout(0, None) == B.OP_E_INVALID
    assert B.op_selftest_wait_timeout(3_000_000_000, None) == B.OP_E_INVALID
