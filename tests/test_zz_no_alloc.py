"""fftseg_exec_noalloc: the no-allocation entry point, for callers that must
not allocate device memory (strict memory budgets, plugins whose host owns
every allocation, real-time threads that cannot afford cudaMalloc).

Its output must equal what the plan-based entry point gives for the same
transform, within the FP32 tolerance the other tests use, on two calls in a
row (the second call reuses the fixed scratch that the first one left
behind).  This file sorts last so that a run stopping at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.parametrize("log_n,nseg,direction,norm", [(17, 7, fs.FORWARD, fs.NORM_NONE),
                                                       (20, 3, fs.INVERSE, fs.NORM_BACKWARD),
                                                       (18, 5, fs.FORWARD, fs.NORM_ORTHO)])
def test_noalloc_matches_plan_entry_point_twice(log_n, nseg, direction, norm):
    fn = noalloc_fn()
    n = 1 << log_n
    x = torch.from_numpy(siggen.tones(900 + log_n, nseg * n).reshape(nseg, n)).cuda()
    ref = fs.Plan(n, nseg, direction, norm).exec(x)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full_like(x, complex(3.0, -3.0))
        rc = fn(x.data_ptr(), out.data_ptr(), n, nseg, direction, norm, stream)
        assert rc == fs.OK, fs.last_error()
        torch.cuda.synchronize()
        err = rel_l2(out.cpu().numpy(), ref.cpu().numpy().astype(np.complex128))
        assert err <= tol_fp32(n), (call, err)


def test_noalloc_rejects_what_its_scratch_cannot_hold():
    fn = noalloc_fn()
    x = torch.zeros(1 << 21, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for n in (1 << 21, 1 << 16, 3 << 17):
        assert fn(x.data_ptr(), x.data_ptr(), n, 1, fs.FORWARD, fs.NORM_NONE, stream) == fs.E_UNSUPPORTED
        assert "2^17..2^20" in fs.last_error()
    assert fn(x.data_ptr(), x.data_ptr(), 1 << 17, 0, fs.FORWARD, fs.NORM_NONE, stream) == fs.OK
