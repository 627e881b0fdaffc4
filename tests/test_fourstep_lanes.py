"""GPU parity of the lane-line persistent four-step kernel (n = 2^16..2^20,
FP32, complex output; the default at 2^17..2^20) against the FP64 oracle,
per segment, on batches that cycle its ring of chunk buffers and end in a
partial chunk; plus in-place runs and run-to-run bit equality (its tiles come
from a queue, so CTAs take different tiles each run, but a tile's arithmetic
does not depend on the CTA that runs it)."""
import numpy as np
import pytest

import oracle
import siggen
from tests._util import check_guard, guard, rel_l2, tol_fp32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402

FWD, INV = fs.FORWARD, fs.INVERSE


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def plan_for(n, B, direction, norm):
    flags = fs.FLAG_FOURSTEP_LANES if n == 1 << 16 else 0
    plan = fs.Plan(n, B, direction, norm, flags=flags)
    assert plan.info()["path"] == "four-step"
    return plan


# segments per 16 MiB chunk: 32, 16, 8, 4, 2; the batches span 4..7 chunks
# (the ring holds 3), the last one partial
@pytest.mark.parametrize("log_n,B", [(16, 101), (17, 61), (18, 29), (19, 15), (20, 13)])
@pytest.mark.parametrize("direction,norm", [(FWD, fs.NORM_NONE), (INV, fs.NORM_BACKWARD), (FWD, fs.NORM_ORTHO)])
def test_lane_line_fourstep_matches_oracle(log_n, B, direction, norm):
    n = 1 << log_n
    x = siggen.tones(1600 + log_n, B * n).reshape(B, n)
    plan = plan_for(n, B, direction, norm)
    d = torch.from_numpy(x).cuda()
    buf, y = guard(d)
    plan.exec(d, out=y)
    torch.cuda.synchronize()
    plan.check()
    check_guard(buf)
    got = y.cpu().numpy()
    assert rel_l2(got, oracle.fft(x, direction, norm)) <= tol_fp32(n)
    # again, and in place: the same bits
    y2 = plan.exec(d)
    plan.exec(d, out=d)
    torch.cuda.synchronize()
    plan.check()
    np.testing.assert_array_equal(y2.cpu().numpy(), got)
    np.testing.assert_array_equal(d.cpu().numpy(), got)


def test_lane_line_fourstep_round_trip_and_partial_batches():
    n, B = 1 << 18, 21
    x = siggen.uniform(1650, B * n).reshape(B, n)
    fwd = plan_for(n, B, FWD, fs.NORM_NONE)
    inv = plan_for(n, B, INV, fs.NORM_BACKWARD)
    d = torch.from_numpy(x).cuda()
    back = inv.exec(fwd.exec(d))
    torch.cuda.synchronize()
    assert rel_l2(back.cpu().numpy(), x) <= 2 * tol_fp32(n)
    full = fwd.exec(d).cpu().numpy()
    for k in (1, 2, 7, 9):  # fewer segments than the plan's batch: a chunk of their own size or a partial chunk
        out = torch.full_like(d, complex(7.0, 7.0))
        fwd.exec(d, out=out, nseg=k)
        torch.cuda.synchronize()
        fwd.check()
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got[:k], full[:k])
        assert (got[k:] == np.complex64(complex(7.0, 7.0))).all()  # untouched past nseg


def test_lane_line_flag_refused_where_it_does_not_apply():
    with pytest.raises(fs.FFTSegError) as e:
        fs.Plan(1 << 21, 2, FWD, flags=fs.FLAG_FOURSTEP_LANES)
    assert e.value.status == fs.E_UNSUPPORTED
    with pytest.raises(fs.FFTSegError):
        fs.Plan(1 << 18, 2, FWD, out_kind=fs.OUT_POWER, flags=fs.FLAG_FOURSTEP_LANES)
