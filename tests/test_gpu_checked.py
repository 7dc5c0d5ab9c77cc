"""The bounds-checking build (liboilpaint_checked.so, -DOPK_CHECKED=1): every
shared-memory access of the histogram and ring helpers, every pixel access
and every TMA copy is range-checked on the device; a violation would be
reported as OP_E_BOUNDS.  All kernel paths must run through it with no
check firing and the oracle's bytes."""
import os
import subprocess
import sys

import pytest

from paper_1405_1020_gb300.csrc import build as lib_build

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_path_passes_the_bounds_checks():
    lib_build.build(checked=True)
    env = dict(os.environ, OPK_LIBRARY="checked")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_worker.py")],
                       env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    assert "no bounds check fired" in p.stdout
