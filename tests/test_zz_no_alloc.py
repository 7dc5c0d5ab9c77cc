"""op_run_noalloc: the filter without any device allocation.

Callers that cannot allocate device memory (a plugin inside an application
that owns all device memory through its own pool, a latency-critical path
that cannot take the device-wide synchronisation of cudaMalloc/cudaFree, a
process whose free memory another allocator already holds) call this entry
point; its packed-word scratch is a fixed array inside the library.

Its output must equal op_run's byte for byte (the filter is integer work, so
the tolerance is zero) on consecutive calls that share that array, and images
larger than the array must be refused.  The first call on a device loads the
library part that holds the array, which places the 16 MiB array in device
memory; device free memory may drop by that much across the first call and
must not change across any later one.  The file is collected last so that a
failure here comes after every other test has run; it also passes alone in a
fresh process.
"""
import pytest
import torch

import __graft_entry__
from paper_1405_1020_gb300 import binding as B
from paper_1405_1020_gb300 import synth
from paper_1405_1020_gb300.filter import OilPaint

pytestmark = pytest.mark.gpu

FILL = 0x5A


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _case(w, h, bpp, pad, seed):
    img = synth.camera_like(h, w, seed=seed, npoly=30, rad_range=(5, 200))
    buf, stride = synth.to_strided(img, bpp=bpp, stride=w * bpp + pad)
    return torch.from_numpy(buf).cuda(), stride


def _with_op_run(src, w, h, stride, bpp, r, L, flags):
    out = torch.full_like(src, FILL)
    op = OilPaint(w, h, r, L, bpp=bpp, stride=stride, flags=flags)
    op.run(src, out)
    assert op.sync_status() == B.OP_OK
    op.close()
    return out


def test_noalloc_equals_op_run_on_consecutive_calls():
    cases = [(300, 200, 3, 0, 15, 20, 0, 1), (1000, 700, 4, 12, 4, 32, 1, 2),
             (257, 129, 3, 5, 20, 16, 0, 3)]
    inputs = [(_case(w, h, bpp, pad, seed), w, h, bpp, r, L, fl)
              for w, h, bpp, pad, r, L, fl, seed in cases]
    refs = [_with_op_run(src, w, h, stride, bpp, r, L, fl)
            for (src, stride), w, h, bpp, r, L, fl in inputs]
    # warm-up call: the first call on a device loads the array; free memory
    # may drop by the array's size (rounded up to the allocation granularity)
    (src, stride), w, h, bpp, r, L, fl = inputs[0]
    out = torch.full_like(src, FILL)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    st = B.op_run_noalloc(src.data_ptr(), out.data_ptr(), w, h, stride, bpp, r, L, fl,
                          torch.cuda.current_stream().cuda_stream)
    free_after = torch.cuda.mem_get_info()[0]
    assert st == B.OP_OK, B.status_string(st)
    drop = free_before - free_after
    assert 0 <= drop <= 4 * B.OP_NOALLOC_MAX_WORDS + (4 << 20), drop
    assert torch.equal(out, refs[0])
    # two rounds of calls in a row; each call finds the previous image's
    # words in the shared scratch array
    for _ in range(2):
        for ((src, stride), w, h, bpp, r, L, fl), ref in zip(inputs, refs):
            out = torch.full_like(src, FILL)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            st = B.op_run_noalloc(src.data_ptr(), out.data_ptr(), w, h, stride, bpp, r, L, fl,
                                  torch.cuda.current_stream().cuda_stream)
            free_after = torch.cuda.mem_get_info()[0]
            assert st == B.OP_OK, B.status_string(st)
            assert free_after == free_before, "device memory changed across the call"
            assert torch.equal(out, ref), f"{w}x{h} r={r} L={L} differs from op_run"


def test_noalloc_limit_and_argument_checks():
    w, h = 2048, 2048  # exactly OP_NOALLOC_MAX_WORDS packed words
    assert ((w + 3) // 4 * 4) * h == B.OP_NOALLOC_MAX_WORDS
    src = torch.zeros(h * w * 3, dtype=torch.uint8, device="cuda")
    dst = torch.zeros_like(src)
    s = torch.cuda.current_stream().cuda_stream
    assert B.op_run_noalloc(src.data_ptr(), dst.data_ptr(), w, h, w * 3, 3, 2, 20, 0, s) == B.OP_OK
    assert (dst == 0).all()  # a black image stays black
    big = torch.zeros((h + 1) * w * 3, dtype=torch.uint8, device="cuda")
    big_out = torch.zeros_like(big)
    assert B.op_run_noalloc(big.data_ptr(), big_out.data_ptr(), w, h + 1, w * 3, 3, 2, 20, 0,
                            s) == B.OP_E_UNSUPPORTED
    assert B.op_run_noalloc(src.data_ptr(), src.data_ptr(), w, h, w * 3, 3, 2, 20, 0,
                            s) == B.OP_E_INVALID
    assert B.op_run_noalloc(src.data_ptr(), dst.data_ptr(), w, h, w * 3, 3, 2, 0, 0,
                            s) == B.OP_E_INVALID
    assert B.op_run_noalloc(src.data_ptr(), dst.data_ptr(), w, h, w * 3 - 1, 3, 2, 20, 0,
                            s) == B.OP_E_INVALID
    assert B.op_run_noalloc(None, dst.data_ptr(), w, h, w * 3, 3, 2, 20, 0,
                            s) == B.OP_E_INVALID
