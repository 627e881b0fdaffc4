"""Lengths that are not powers of two (Bluestein) against the direct-DFT oracle.

The paper's library handles any length (Sec. I: its FFT libraries are general);
here such n run as a cyclic convolution over M = 2^ceil(log2(2n - 1)) points
on the power-of-two kernels.  Bound: the result passes through two M-point
FP32 transforms and three pointwise products, so the FP32 bound is taken for
three transforms of M points, 2e-6 * (3 log2(M) + 3).
"""
import math

import numpy as np
import pytest

import oracle
import siggen
from tests._util import check_guard, guard, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def tol_blue(n):
    M = 1 << math.ceil(math.log2(2 * n - 1))
    return 2e-6 * (3 * math.log2(M) + 3)


def run(plan, x):
    d = torch.from_numpy(x).cuda()
    dt = torch.float32 if plan.out_kind == fs.OUT_POWER else torch.complex64
    buf, y = guard(torch.empty(d.shape, dtype=dt, device="cuda"))  # canaries past the output's end
    plan.exec(d, out=y)
    torch.cuda.synchronize()
    plan.check()
    check_guard(buf)
    return y.cpu().numpy()


@pytest.mark.parametrize("n", [3, 5, 7, 12, 100, 1000, 1001, 4095, 10007])
@pytest.mark.parametrize("direction,norm", [(fs.FORWARD, fs.NORM_NONE), (fs.INVERSE, fs.NORM_BACKWARD),
                                            (fs.FORWARD, fs.NORM_ORTHO)])
def test_bluestein_matches_direct_dft(n, direction, norm):
    B = 5
    x = siggen.tones(1300 + n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, direction, norm, flags=fs.FLAG_BLUESTEIN)
    assert plan.info()["path"] == "bluestein"
    got = run(plan, x)
    ref = oracle.dft(x, direction, norm)
    assert rel_l2(got, ref) <= tol_blue(n), (n, rel_l2(got, ref))


@pytest.mark.parametrize("n,B", [(6, 70000), (1000, 9000), (40009, 4), (100003, 3), (3 * (1 << 20), 2)])
def test_bluestein_chunks_and_large_n(n, B):
    # more segments than one chunk of M-point rows (and than one launch's grid
    # rows at n = 6), and lengths whose M is 2^17 (five passes around the
    # lane-line kernel) up to 2^23; bins spot-checked
    x = siggen.uniform(1400 + n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, fs.FORWARD, flags=fs.FLAG_BLUESTEIN)
    got = run(plan, x)
    segs = np.r_[0, B // 2, B - 1]
    bins = np.unique(np.r_[0, 1, n // 3, n // 2, n - 1, np.arange(0, n, max(1, n // 7))])
    ref = oracle.dft(x[segs], bins=bins)
    assert rel_l2(got[segs][:, bins], ref) <= tol_blue(n)


def test_bluestein_power_and_stream():
    n, B = 3000, 40
    x = siggen.tones(1500, B * n).reshape(B, n)
    plan = fs.Plan(n, B, fs.FORWARD, out_kind=fs.OUT_POWER, flags=fs.FLAG_BLUESTEIN)
    got = run(plan, x)
    X = oracle.dft(x)
    assert rel_l2(got, X.real ** 2 + X.imag ** 2) <= 2 * tol_blue(n)
    # the chunker carries any length: segments of n * 8 bytes
    out = np.zeros(B * n, dtype=np.float32)
    chunks = []

    def rd(ctx, off, dst, nbytes):
        nbytes = min(nbytes, x.nbytes - off)
        if nbytes > 0:
            import ctypes
            ctypes.memmove(dst, x.ctypes.data + off, nbytes)
        return max(nbytes, 0)

    def wr(ctx, off, src, nbytes):
        import ctypes
        ctypes.memmove(out.ctypes.data + off, src, nbytes)
        chunks.append(off)
        return 0

    sp = fs.Plan(n, 16, fs.FORWARD, out_kind=fs.OUT_POWER, flags=fs.FLAG_BLUESTEIN)
    rc, committed = sp.stream(rd, None, wr, None, x.nbytes, 0, 16)
    assert rc == fs.OK and committed == x.nbytes and len(chunks) == 3
    np.testing.assert_array_equal(out.reshape(B, n), got)


@pytest.mark.parametrize("n,B,out_kind", [(3, 1000, fs.OUT_COMPLEX), (100, 37, fs.OUT_POWER),
                                          (1000, 131, fs.OUT_COMPLEX), (2047, 3, fs.OUT_POWER),
                                          (2049, 3, fs.OUT_COMPLEX)])
def test_bluestein_fused_rows(n, B, out_kind):
    # rows with M <= 4096 run in one fused launch with no intermediate rows
    # (ragged last tiles: B is no multiple of 4096 / M); M = 8192 (n = 2049)
    # goes through the five-pass chunks
    M = 1 << math.ceil(math.log2(2 * n - 1))
    x = siggen.tones(1600 + n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, fs.INVERSE, fs.NORM_ORTHO, out_kind=out_kind, flags=fs.FLAG_BLUESTEIN)
    info = plan.info()
    if M <= 4096:
        assert info["launches_per_exec"] == 1 and info["work_bytes"] == 0
    else:
        assert info["launches_per_exec"] > 1 and info["work_bytes"] > 0
    got = run(plan, x)
    X = oracle.dft(x, fs.INVERSE, fs.NORM_ORTHO)
    if out_kind == fs.OUT_POWER:
        assert rel_l2(got, X.real ** 2 + X.imag ** 2) <= 2 * tol_blue(n)
    else:
        assert rel_l2(got, X) <= tol_blue(n)


@pytest.mark.parametrize("n,B,direction,out_kind", [(3001, 33, fs.FORWARD, fs.OUT_COMPLEX),
                                                    (4097, 17, fs.INVERSE, fs.OUT_POWER),
                                                    (9001, 9, fs.FORWARD, fs.OUT_POWER),
                                                    (20011, 5, fs.INVERSE, fs.OUT_COMPLEX),
                                                    (32767, 3, fs.FORWARD, fs.OUT_COMPLEX)])
def test_bluestein_cluster_rows(n, B, direction, out_kind):
    # M = 2^13 .. 2^16: the chirp-in read by the forward cluster transform
    # itself, the product with B and the chirp-out folded into the inverse
    # one; two launches per chunk (one chunk here), bins spot-checked
    M = 1 << math.ceil(math.log2(2 * n - 1))
    assert 1 << 13 <= M <= 1 << 16
    x = siggen.tones(1700 + n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, direction, fs.NORM_ORTHO, out_kind=out_kind, flags=fs.FLAG_BLUESTEIN)
    assert plan.info()["launches_per_exec"] == 2
    got = run(plan, x)
    segs = np.r_[0, B // 2, B - 1]
    bins = np.unique(np.r_[0, 1, n // 3, n // 2, n - 1, np.arange(0, n, max(1, n // 97))])
    X = oracle.dft(x[segs], direction, fs.NORM_ORTHO, bins=bins)
    if out_kind == fs.OUT_POWER:
        assert rel_l2(got[segs][:, bins], X.real ** 2 + X.imag ** 2) <= 2 * tol_blue(n)
    else:
        assert rel_l2(got[segs][:, bins], X) <= tol_blue(n)
