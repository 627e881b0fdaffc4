"""Overlapping segments (fftseg_plan_create_frames) against the FP64 oracle.

The paper names overlapping FFTs as future work (Sec. VI).  Frame f holds
samples [f*hop, f*hop + n) of the signal, times the window.  Lengths span the
block, cluster and four-step paths of the n-point transform; hops overlap,
tile exactly, skip samples and are odd; frame counts span more than one
32 MiB chunk of the intermediate.
"""
import numpy as np
import pytest

import oracle
import siggen
from tests._util import rel_l2, tol_fp32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(autouse=True)
def small_chunks(monkeypatch):
    # 32 MiB chunks of windowed frames (the default is 512 MiB), so that
    # modest batches span several chunks
    monkeypatch.setenv("FFTSEG_FRAMES_CHUNK_MB", "32")


def signal(seed, samples):
    return siggen.tones(seed, samples)


@pytest.mark.parametrize("log_n,hop_frac", [(4, 0.5), (10, 0.5), (10, 0.25), (12, 0.75), (12, 1.0),
                                            (14, 0.5), (16, 0.5), (16, 1.25)])
@pytest.mark.parametrize("window", [fs.WINDOW_RECT, fs.WINDOW_HANN])
def test_frames_match_oracle(log_n, hop_frac, window):
    n = 1 << log_n
    hop = max(1, int(n * hop_frac))
    F = max(3, (40 << 20) // (8 * n) + 1)  # more than one chunk of the intermediate
    x = signal(40 + log_n, (F - 1) * hop + n)
    plan = fs.FramePlan(n, hop, F, window)
    assert plan.info()["path"] == "frames"
    got = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    assert got.shape == (F, n)
    sample = np.r_[0:2, F // 2, F - 1]
    ref = np.concatenate([oracle.frames_fft(x[f * hop:], n, hop, 1, window) for f in sample])
    assert rel_l2(got.cpu().numpy()[sample].astype(np.complex128), ref) <= tol_fp32(n)


@pytest.mark.parametrize("log_n,hop", [(6, 21), (11, 1001), (13, 4097)])
def test_odd_hops_and_power(log_n, hop):
    n = 1 << log_n
    F = 9
    x = signal(70 + log_n, (F - 1) * hop + n)
    plan = fs.FramePlan(n, hop, F, fs.WINDOW_HANN, norm=fs.NORM_ORTHO, out_kind=fs.OUT_POWER)
    got = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    X = oracle.frames_fft(x, n, hop, F, oracle.WINDOW_HANN, oracle.NORM_ORTHO)
    assert rel_l2(got.cpu().numpy(), X.real ** 2 + X.imag ** 2) <= 2 * tol_fp32(n)


def test_frame_plan_rejections():
    with pytest.raises(fs.FFTSegError):
        fs.FramePlan(1024, 0, 4)  # hop >= 1
    with pytest.raises(fs.FFTSegError):
        fs.FramePlan(1000, 500, 4)  # power-of-two n
    with pytest.raises(fs.FFTSegError):
        fs.FramePlan(1024, 512, 4, window=7)
    with pytest.raises(fs.FFTSegError):
        fs.FramePlan(1024, 512, 4, flags=fs.FLAG_REAL)
    plan = fs.FramePlan(1024, 512, 4)
    buf = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    with pytest.raises(fs.FFTSegError):
        plan.exec_ptr(buf.data_ptr(), buf.data_ptr(), 3)  # out of place only
    with pytest.raises(ValueError):
        plan.exec(torch.zeros(1000, dtype=torch.complex64, device="cuda"), nseg=1)  # not one whole frame
    for total, start in [(8196, 0), (8192, 8), (8192, 4096 * 8 * 2)]:
        # a partial sample; a start that is not a frame's first sample; a start past the last frame
        with pytest.raises(fs.FFTSegError) as e:
            plan.stream(lambda *a: 0, None, lambda *a: 0, None, total, start)
        assert e.value.status == fs.E_INVALID


@pytest.mark.parametrize("log_n,hop,F", [(1, 1, 1000), (2, 3, 777), (5, 7, 300), (9, 256, 51), (12, 4095, 5),
                                         (13, 4096, 5)])
def test_fused_frames(log_n, hop, F):
    # frames of n <= 4096 points run in one launch with no intermediate
    # (ragged last tiles: F is no multiple of 4096 / n); n = 8192 is chunked
    n = 1 << log_n
    x = signal(90 + log_n, (F - 1) * hop + n)
    plan = fs.FramePlan(n, hop, F, fs.WINDOW_HANN, norm=fs.NORM_BACKWARD)
    info = plan.info()
    if n <= 4096:
        assert info["launches_per_exec"] == 1 and info["work_bytes"] == 0
    else:
        assert info["launches_per_exec"] > 1 and info["work_bytes"] > 0
    got = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    X = oracle.frames_fft(x, n, hop, F, oracle.WINDOW_HANN, oracle.NORM_BACKWARD)
    assert rel_l2(got.cpu().numpy().astype(np.complex128), X) <= tol_fp32(max(n, 2))


def test_frames_signal_off_16_bytes_is_rejected():
    # device buffers are 16-byte aligned by contract (the bulk copies rely on
    # it); a signal 8 bytes past a boundary is refused, not read
    n, hop, F = 1024, 512, 4
    x = signal(99, (F - 1) * hop + n + 1)
    xd = torch.from_numpy(x).cuda()[1:]
    assert xd.data_ptr() % 16 == 8
    plan = fs.FramePlan(n, hop, F, fs.WINDOW_HANN)
    with pytest.raises(fs.FFTSegError) as e:
        plan.exec(xd)
    assert e.value.status == fs.E_INVALID
