"""GPU parity of the mixed-radix path (lengths n = 2^a 3^b 5^c 7^d <= 4096
that are not powers of two; radix 2, 3, 4, 5, 7 and 8 Stockham stages in one
pass) against the FP64 oracle's direct DFT, per segment, within the FP32
bound 2e-6 log2(n); ragged last tiles, in place, |X|^2 output, streaming,
and the lengths that still go to Bluestein."""
import ctypes

import numpy as np
import pytest

import oracle
import siggen
from tests._util import check_guard, guard, rel_l2, tol_fp32, tol_power

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402

FWD, INV = fs.FORWARD, fs.INVERSE
SMOOTH = [3, 5, 6, 7, 9, 10, 12, 14, 15, 21, 25, 27, 35, 49, 60, 96, 100, 125, 243, 343, 625, 729, 1000,
          1536, 2187, 2401, 3000, 3072, 3125, 4000, 4032]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def run(plan, x, out_dtype=torch.complex64):
    d = torch.from_numpy(x).cuda()
    buf, y = guard(torch.empty(d.shape, dtype=out_dtype, device="cuda"))
    plan.exec(d, out=y)
    torch.cuda.synchronize()
    plan.check()
    check_guard(buf)
    return y.cpu().numpy()


@pytest.mark.parametrize("n", SMOOTH)
@pytest.mark.parametrize("direction,norm", [(FWD, fs.NORM_NONE), (INV, fs.NORM_BACKWARD), (FWD, fs.NORM_ORTHO)])
def test_mixed_radix_matches_direct_dft(n, direction, norm):
    spt = 4096 // n
    B = 3 * spt + max(1, spt // 2)  # several tiles, the last one ragged
    x = siggen.tones(1700 + n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, direction, norm)
    info = plan.info()
    assert info["path"] == "mixed-radix" and info["launches_per_exec"] == 1
    got = run(plan, x)
    assert rel_l2(got, oracle.dft(x, direction, norm)) <= tol_fp32(n), n


@pytest.mark.parametrize("n", [12, 1000, 3125])
def test_mixed_radix_power_in_place_and_bits(n):
    B = 2 * (4096 // n) + 1
    x = siggen.uniform(1800 + n, B * n).reshape(B, n)
    X = oracle.dft(x, FWD, fs.NORM_ORTHO)
    pw = fs.Plan(n, B, FWD, fs.NORM_ORTHO, out_kind=fs.OUT_POWER)
    got = run(pw, x, torch.float32)
    assert rel_l2(got, X.real ** 2 + X.imag ** 2) <= tol_power(n)
    plan = fs.Plan(n, B, FWD, fs.NORM_ORTHO)
    ref = run(plan, x)
    d = torch.from_numpy(x).cuda()
    plan.exec(d, out=d)  # in place
    torch.cuda.synchronize()
    plan.check()
    np.testing.assert_array_equal(d.cpu().numpy(), ref)
    np.testing.assert_array_equal(run(plan, x), ref)  # run to run


def test_mixed_radix_many_tiles_and_round_trip():
    n, B = 1000, 9001  # about 2200 tiles over the persistent grid
    x = siggen.tones(1850, B * n).reshape(B, n)
    fwd = fs.Plan(n, B, FWD)
    inv = fs.Plan(n, B, INV, fs.NORM_BACKWARD)
    got = run(fwd, x)
    segs = np.r_[0:3, B // 2, B - 2, B - 1]
    assert rel_l2(got[segs], oracle.dft(x[segs])) <= tol_fp32(n)
    back = inv.exec(fwd.exec(torch.from_numpy(x).cuda()))
    torch.cuda.synchronize()
    assert rel_l2(back.cpu().numpy(), x) <= 2 * tol_fp32(n)


def test_mixed_radix_streams_bit_equal_to_resident():
    n, B = 3000, 50
    x = siggen.tones(1870, B * n).reshape(B, n)
    plan = fs.Plan(n, 16, FWD)
    resident = fs.Plan(n, B, FWD)
    ref = run(resident, x)
    out = np.zeros(B * n, dtype=np.complex64)

    def rd(ctx, off, dst, nbytes):
        nbytes = max(0, min(nbytes, x.nbytes - off))
        ctypes.memmove(dst, x.ctypes.data + off, nbytes)
        return nbytes

    def wr(ctx, off, src, nbytes):
        ctypes.memmove(out.ctypes.data + off, src, nbytes)
        return 0

    rc, committed = plan.stream(rd, None, wr, None, x.nbytes, 0, 16)
    assert rc == fs.OK and committed == x.nbytes
    np.testing.assert_array_equal(out.reshape(B, n), ref)


def test_other_lengths_still_take_bluestein():
    for n in (11, 4097, 6000, 10007):  # a prime factor above 7, or longer than one tile
        assert fs.Plan(n, 2, FWD).info()["path"] == "bluestein"
    assert fs.Plan(1000, 2, FWD, flags=fs.FLAG_BLUESTEIN).info()["path"] == "bluestein"
