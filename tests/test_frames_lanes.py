"""GPU parity of frame plans fused into the lane-line four-step kernel
(n = 2^16..2^20, hop a multiple of N2 = 2^floor(log2(n)/2), complex output):
each frame's column tiles come straight from the signal and the periodic
Hann window is applied as they are read, in one launch.  Checked per frame
against the FP64 oracle (frames_fft), with ragged frame counts, hops below,
at and above n, every norm, guard bands, bit equality with the segment plan
on the windowed frames' rectangular case, and the chunked form for hops
that are not multiples of N2."""
import numpy as np
import pytest

import oracle
import siggen
from tests._util import check_guard, guard, rel_l2, tol_fp32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def run(plan, x, F, n):
    d = torch.from_numpy(x).cuda()
    buf, y = guard(torch.empty(F, n, dtype=torch.complex64, device="cuda"))
    plan.exec(d, out=y)
    torch.cuda.synchronize()
    plan.check()
    check_guard(buf)
    return y.cpu().numpy()


# hop in units of N2 (256 at 2^16 and 2^17, 512 at 2^18 and 2^19, 1024 at 2^20)
@pytest.mark.parametrize("log_n,hop_rows,F", [(16, 128, 77), (16, 1, 300), (16, 320, 40), (17, 100, 70),
                                              (18, 256, 41), (19, 512, 17), (20, 768, 13)])
@pytest.mark.parametrize("window,norm", [(fs.WINDOW_HANN, fs.NORM_NONE), (fs.WINDOW_RECT, fs.NORM_ORTHO),
                                         (fs.WINDOW_HANN, fs.NORM_BACKWARD)])
def test_fused_lane_frames_match_oracle(log_n, hop_rows, F, window, norm):
    n = 1 << log_n
    hop = hop_rows * (1 << (log_n // 2))
    x = siggen.tones(1900 + log_n, (F - 1) * hop + n)
    plan = fs.FramePlan(n, hop, F, window, norm)
    info = plan.info()
    assert info["path"] == "frames" and info["launches_per_exec"] == 1 and info["work_bytes"] == 0
    got = run(plan, x, F, n)
    ref = oracle.frames_fft(x, n, hop, F, window, norm)
    assert rel_l2(got.astype(np.complex128), ref) <= tol_fp32(n)


def test_fused_rect_frames_equal_the_segment_plan_bit_for_bit():
    # rectangular frames at hop = n are the signal's segments: the same kernel,
    # the same bits as the segment plan
    n, F = 1 << 16, 50
    x = siggen.uniform(1950, F * n)
    frames = run(fs.FramePlan(n, n, F, fs.WINDOW_RECT), x, F, n)
    segs = fs.Plan(n, F, fs.FORWARD).exec(torch.from_numpy(x).cuda().view(F, n))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(frames, segs.cpu().numpy())


def test_other_hops_keep_the_chunked_form():
    n, hop, F = 1 << 16, 1000, 60  # not a multiple of N2
    x = siggen.tones(1960, (F - 1) * hop + n)
    plan = fs.FramePlan(n, hop, F, fs.WINDOW_HANN)
    assert plan.info()["launches_per_exec"] > 1
    got = run(plan, x, F, n)
    sample = np.r_[0, F // 2, F - 1]
    ref = np.concatenate([oracle.frames_fft(x[f * hop:], n, hop, 1, fs.WINDOW_HANN) for f in sample])
    assert rel_l2(got[sample].astype(np.complex128), ref) <= tol_fp32(n)


@pytest.mark.parametrize("log_n,hop_rows,F", [(16, 128, 77), (20, 768, 13)])
def test_fused_lane_frames_power(log_n, hop_rows, F):
    # |X|^2 of windowed frames in the same single launch (the row pass's
    # float output boxes)
    n = 1 << log_n
    hop = hop_rows * (1 << (log_n // 2))
    x = siggen.tones(1970 + log_n, (F - 1) * hop + n)
    plan = fs.FramePlan(n, hop, F, fs.WINDOW_HANN, fs.NORM_ORTHO, out_kind=fs.OUT_POWER)
    info = plan.info()
    assert info["launches_per_exec"] == 1 and info["work_bytes"] == 0, info
    got = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    X = oracle.frames_fft(x, n, hop, F, fs.WINDOW_HANN, fs.NORM_ORTHO)
    assert rel_l2(got.cpu().numpy(), X.real ** 2 + X.imag ** 2) <= 2 * tol_fp32(n)


def test_frames_above_2p20_run_chunked_on_the_interleaved_plan():
    # 2^21-point frames: chunks of windowed frames through the interleaved
    # four-step
    n, hop, F = 1 << 21, 1 << 20, 5
    x = siggen.tones(1980, (F - 1) * hop + n)
    plan = fs.FramePlan(n, hop, F, fs.WINDOW_HANN)
    got = run(plan, x, F, n)
    sample = np.r_[0, F - 1]
    ref = np.concatenate([oracle.frames_fft(x[f * hop:], n, hop, 1, fs.WINDOW_HANN) for f in sample])
    assert rel_l2(got[sample].astype(np.complex128), ref) <= tol_fp32(n)
