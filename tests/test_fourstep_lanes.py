"""GPU parity of the lane-line persistent four-step kernel (n = 2^16..2^20,
FP32, complex output; the default there) against the FP64 oracle,
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
    plan = fs.Plan(n, B, direction, norm)
    assert plan.info()["path"] == "four-step"
    return plan


# segments per 32 MiB chunk (the default): 64, 32, 16, 8, 4; the batches span
# 5 chunks (the ring holds 3), the last one partial
@pytest.mark.parametrize("log_n,B", [(16, 293), (17, 139), (18, 69), (19, 35), (20, 17)])
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


# |X|^2 from the row pass: the float output box of each row tile (W_B = 32,
# 16 or 8 lines: 128-, 64- and 32-byte rows), several ring chunks, every
# segment compared, nothing written past the output
@pytest.mark.parametrize("log_n,B", [(16, 293), (17, 139), (18, 69), (19, 35), (20, 17)])
@pytest.mark.parametrize("norm", [fs.NORM_NONE, fs.NORM_ORTHO])
def test_lane_line_fourstep_power(log_n, B, norm):
    n = 1 << log_n
    x = siggen.tones(1650 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, FWD, norm, out_kind=fs.OUT_POWER, flags=fs.FLAG_FOURSTEP_L2)
    assert plan.info()["path"] == "four-step" and plan.info()["launches_per_exec"] == 1
    buf, y = guard(torch.empty(B, n, dtype=torch.float32, device="cuda"))
    plan.exec(torch.from_numpy(x).cuda(), out=y)
    torch.cuda.synchronize()
    plan.check()
    check_guard(buf)
    X = oracle.fft(x, FWD, norm)
    assert rel_l2(y.cpu().numpy(), X.real ** 2 + X.imag ** 2) <= 2 * tol_fp32(n)


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


def test_warp_line_flag_refused_where_it_does_not_apply():
    with pytest.raises(fs.FFTSegError) as e:
        fs.Plan(1 << 17, 2, FWD, flags=fs.FLAG_FOURSTEP_WARP_LINES)
    assert e.value.status == fs.E_UNSUPPORTED
    with pytest.raises(fs.FFTSegError):
        fs.Plan(1 << 16, 2, FWD, out_kind=fs.OUT_POWER, flags=fs.FLAG_FOURSTEP_WARP_LINES)


@pytest.mark.parametrize("log_n", [16, 20])
def test_lane_line_fourstep_small_chunks_cycle_the_ring(log_n, monkeypatch):
    # 1 MiB chunks and two chunks of lookahead (a ring of four chunks): the
    # batch cycles the ring many times, so column tiles wait on row tiles often
    monkeypatch.setenv("FFTSEG_WL_CHUNK_MB", "1")
    monkeypatch.setenv("FFTSEG_WL_LOOKAHEAD", "2")
    n = 1 << log_n
    B = 45 if log_n == 16 else 11
    x = siggen.tones(1660 + log_n, B * n).reshape(B, n)
    plan = plan_for(n, B, FWD, fs.NORM_NONE)
    assert plan.info()["work_segs"] == max(1, (1 << 20) // (8 * n))
    got = run_once(plan, x)
    assert rel_l2(got, oracle.fft(x)) <= tol_fp32(n)


def run_once(plan, x):
    y = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    return y.cpu().numpy()


def test_a_dependency_that_never_arrives_ends_in_a_timeout_status():
    # the row tiles of segment 0 wait (with a short limit) for a column-tile
    # count that is never reached: the kernel must give the wait up, complete,
    # and report it through fftseg_plan_check; the plan then works again
    n, B = 1 << 17, 40
    x = torch.from_numpy(siggen.uniform(1670, B * n).reshape(B, n)).cuda()
    stalled = fs.Plan(n, B, FWD, flags=fs.FLAG_TEST_STALL)
    y = stalled.exec(x)
    torch.cuda.synchronize()
    with pytest.raises(fs.FFTSegError) as e:
        stalled.check()
    assert e.value.status == fs.E_TIMEOUT
    stalled.check()  # the flag was cleared by the check that reported it
    ref = plan_for(n, B, FWD, fs.NORM_NONE).exec(x)
    torch.cuda.synchronize()
    # every segment but the first had its dependencies; they are exact
    np.testing.assert_array_equal(y[1:].cpu().numpy(), ref[1:].cpu().numpy())
