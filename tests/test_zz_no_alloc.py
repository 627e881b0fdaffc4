"""fftseg_exec_noalloc: the no-allocation entry point, for callers that must
not allocate device memory (strict memory budgets, plugins whose host owns
every allocation, real-time threads that cannot afford cudaMalloc).

On two calls in a row (the second reuses the fixed scratch that the first
left behind), its output must match the FP64 oracle per segment, and the
plan-based entry point, within the FP32 tolerance the other tests use, and
fftseg_noalloc_check must report no give-up.  This file sorts last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import siggen
from tests._util import rel_l2, tol_fp32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402


def noalloc_fn():
    from paper_1407_6915_gb300 import build
    build.build()
    fn = fs.lib().fftseg_exec_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p]
    return fn


# 2^19 is the one length whose two factors differ (1024 x 512)
@pytest.mark.parametrize("log_n,nseg,direction,norm", [(17, 7, fs.FORWARD, fs.NORM_NONE),
                                                       (20, 3, fs.INVERSE, fs.NORM_BACKWARD),
                                                       (19, 5, fs.FORWARD, fs.NORM_NONE),
                                                       (18, 5, fs.FORWARD, fs.NORM_ORTHO)])
def test_noalloc_matches_oracle_and_plan_entry_point_twice(log_n, nseg, direction, norm):
    fn = noalloc_fn()
    n = 1 << log_n
    xh = siggen.tones(900 + log_n, nseg * n).reshape(nseg, n)
    x = torch.from_numpy(xh).cuda()
    ref = oracle.fft(xh, direction, norm)
    plan_out = fs.Plan(n, nseg, direction, norm).exec(x).cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full_like(x, complex(3.0, -3.0))
        rc = fn(x.data_ptr(), out.data_ptr(), n, nseg, direction, norm, stream)
        assert rc == fs.OK, fs.last_error()
        torch.cuda.synchronize()
        assert fs.lib().fftseg_noalloc_check() == fs.OK, fs.last_error()
        got = out.cpu().numpy()
        err = rel_l2(got, ref)
        assert err <= tol_fp32(n), (call, err)
        assert rel_l2(got, plan_out) <= tol_fp32(n), call


def test_noalloc_rejects_what_its_scratch_cannot_hold():
    fn = noalloc_fn()
    x = torch.zeros(1 << 21, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for n in (1 << 21, 1 << 16, 3 << 17):
        assert fn(x.data_ptr(), x.data_ptr(), n, 1, fs.FORWARD, fs.NORM_NONE, stream) == fs.E_UNSUPPORTED
        assert "2^17..2^20" in fs.last_error()
    assert fn(x.data_ptr(), x.data_ptr(), 1 << 17, 0, fs.FORWARD, fs.NORM_NONE, stream) == fs.OK
    assert fs.lib().fftseg_noalloc_check() == fs.OK
