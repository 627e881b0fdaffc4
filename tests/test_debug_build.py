"""The self-checking build (-DFFTSEG_DEBUG, libfftseg_debug.so): the
lane-line four-step (also over interleaved units, 2^21..2^24) and
mixed-radix kernels check every shared-memory, ring and tile index they use and report a bad one through fftseg_plan_check
instead of performing it.  On valid inputs the checked build must give the
release build's bits and report nothing."""
import ctypes

import numpy as np
import pytest

import siggen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402


@pytest.fixture(scope="module")
def dbg():
    from paper_1407_6915_gb300 import build
    path = build.build(debug=True)
    L = ctypes.CDLL(path)
    L.fftseg_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint]
    L.fftseg_exec.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.fftseg_plan_check.argtypes = [ctypes.c_void_p]
    L.fftseg_plan_destroy.argtypes = [ctypes.c_void_p]
    L.fftseg_plan_create_frames.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_uint]
    L.fftseg_last_error.restype = ctypes.c_char_p
    return L


def run_debug(L, make, x, out_shape):
    h = ctypes.c_void_p()
    assert make(ctypes.byref(h)) == 0, L.fftseg_last_error()
    y = torch.empty(out_shape, dtype=torch.complex64, device="cuda")
    assert L.fftseg_exec(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    rc = L.fftseg_plan_check(h)
    L.fftseg_plan_destroy(h)
    assert rc == 0, L.fftseg_last_error()  # no index was out of range
    return y.cpu().numpy()


@pytest.mark.parametrize("n,B", [(1 << 16, 70), (1 << 17, 40), (1 << 20, 9), (1 << 21, 33), (1 << 24, 5), (1000, 41),
                                 (3125, 5)])
def test_checked_build_matches_release_bits(dbg, n, B):
    x = torch.from_numpy(siggen.tones(2000 + n % 997, B * n).reshape(B, n)).cuda()
    got = run_debug(dbg, lambda h: dbg.fftseg_plan_create(h, n, B, fs.FORWARD, fs.NORM_NONE, 0, 0, 0), x, (B, n))
    ref = fs.Plan(n, B, fs.FORWARD).exec(x)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got, ref.cpu().numpy())


def test_checked_build_fused_frames(dbg):
    n, hop, F = 1 << 16, 1 << 15, 30
    x = torch.from_numpy(siggen.tones(2100, (F - 1) * hop + n)).cuda()
    got = run_debug(dbg, lambda h: dbg.fftseg_plan_create_frames(h, n, hop, fs.WINDOW_HANN, F, fs.NORM_NONE, 0, 0),
                    x, (F, n))
    ref = fs.FramePlan(n, hop, F, fs.WINDOW_HANN).exec(x)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got, ref.cpu().numpy())
