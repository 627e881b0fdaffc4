"""fftseg_stream over frame plans and real-signal plans, against the same
plans run on the resident signal (bit for bit: the same kernels on the same
frames or segments).

Frames (the paper's overlapping-FFT future work, Sec. VI): a chunk of frames
needs the samples of its first frame up to the end of its last, so
consecutive chunks share n - hop samples; the chunker carries them over
instead of reading them again, and every sample is read once.  Real-signal
plans (the paper's real single-precision records, Sec. III) stream 4n input
bytes per segment and n/2 + 1 bins out.
"""
import ctypes

import numpy as np
import pytest

import siggen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()
    assert torch.cuda.is_available()


class Io:
    """A reader over a host array that records what it was asked for, and a
    writer into a host array."""

    def __init__(self, src, out, limit=None):
        self.src, self.out = src, out
        self.limit = src.nbytes if limit is None else limit  # bytes that exist
        self.reads = []

    def rd(self, ctx, off, dst, nbytes):
        self.reads.append((off, nbytes))
        nbytes = max(0, min(nbytes, self.limit - off))
        if nbytes:
            ctypes.memmove(dst, self.src.ctypes.data + off, nbytes)
        return nbytes

    def wr(self, ctx, off, src, nbytes):
        assert off + nbytes <= self.out.nbytes
        ctypes.memmove(self.out.ctypes.data + off, src, nbytes)
        return 0


def frames_resident(x, n, hop, F, window, out_kind):
    plan = fs.FramePlan(n, hop, F, window, out_kind=out_kind)
    y = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    return y.cpu().numpy()


@pytest.mark.parametrize("n,hop,F,chunk,out_kind", [
    (1024, 256, 301, 64, fs.OUT_COMPLEX),  # overlapping, ragged last chunk
    (1024, 1024, 50, 7, fs.OUT_POWER),     # hop = n: plain segments
    (256, 300, 77, 10, fs.OUT_COMPLEX),    # gaps between frames
    (64, 1, 2000, 333, fs.OUT_COMPLEX),    # hop 1: every chunk is mostly halo
    (8192, 4096, 20, 6, fs.OUT_COMPLEX),   # frames of the chunked n > 4096 path
])
def test_frames_stream_matches_resident(n, hop, F, chunk, out_kind):
    tail = hop // 2  # trailing samples that start no complete frame
    x = siggen.tones(2000 + n + hop, (F - 1) * hop + n + tail)
    ref = frames_resident(x[: (F - 1) * hop + n], n, hop, F, fs.WINDOW_HANN, out_kind)
    out = np.zeros_like(ref)
    io = Io(x, out)
    plan = fs.FramePlan(n, hop, chunk, fs.WINDOW_HANN, out_kind=out_kind)
    rc, committed = plan.stream(io.rd, None, io.wr, None, x.nbytes, 0, chunk)
    assert rc == fs.OK and committed == F * hop * 8
    np.testing.assert_array_equal(out, ref)
    if hop <= n:  # each sample is read once: the halo comes from the previous chunk
        assert sum(b for _, b in io.reads) == ((F - 1) * hop + n) * 8
        ends = [o + b for o, b in io.reads]
        assert all(e == o for e, (o, _) in zip(ends, io.reads[1:]))


def test_frames_stream_resume_and_short_signal():
    n, hop, F, chunk = 512, 128, 200, 32
    x = siggen.tones(2100, (F - 1) * hop + n)
    ref = frames_resident(x, n, hop, F, fs.WINDOW_RECT, fs.OUT_COMPLEX)
    plan = fs.FramePlan(n, hop, chunk, fs.WINDOW_RECT)
    # resume from frame 70: frames before it are left as they were
    out = np.zeros_like(ref)
    rc, committed = plan.stream(Io(x, out).rd, None, Io(x, out).wr, None, x.nbytes, 70 * hop * 8, chunk)
    assert rc == fs.OK and committed == F * hop * 8
    np.testing.assert_array_equal(out[70:], ref[70:])
    assert not out[:70].any()
    # the reader has fewer bytes than total_bytes says: the frames that fit
    # in what it returned are transformed, and the run ends there
    out = np.zeros_like(ref)
    have = (99 * hop + n) * 8 + 40
    io = Io(x, out, limit=have)
    rc, committed = plan.stream(io.rd, None, io.wr, None, x.nbytes, 0, chunk)
    assert rc == fs.OK and committed == 100 * hop * 8
    np.testing.assert_array_equal(out[:100], ref[:100])
    assert not out[100:].any()


def test_frames_stream_writer_failure_then_resume():
    n, hop, F, chunk = 1024, 512, 90, 16
    x = siggen.tones(2200, (F - 1) * hop + n)
    ref = frames_resident(x, n, hop, F, fs.WINDOW_HANN, fs.OUT_COMPLEX)
    out = np.zeros_like(ref)
    calls = []

    def bad_wr(ctx, off, src, nbytes):
        calls.append(off)
        if len(calls) == 3:
            return -1
        ctypes.memmove(out.ctypes.data + off, src, nbytes)
        return 0

    io = Io(x, out)
    plan = fs.FramePlan(n, hop, chunk, fs.WINDOW_HANN)
    rc, committed = plan.stream(io.rd, None, bad_wr, None, x.nbytes, 0, chunk)
    assert rc == fs.E_IO and committed == 2 * chunk * hop * 8
    rc, committed = plan.stream(io.rd, None, io.wr, None, x.nbytes, committed, chunk)
    assert rc == fs.OK and committed == F * hop * 8
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("n,direction,out_kind,B,chunk", [
    (1024, fs.FORWARD, fs.OUT_COMPLEX, 700, 96),  # the fused one-pass kernel
    (4096, fs.FORWARD, fs.OUT_POWER, 90, 16),
    (65536, fs.FORWARD, fs.OUT_COMPLEX, 40, 6),   # chunked inner transform
    (2048, fs.INVERSE, fs.OUT_COMPLEX, 300, 64),
])
def test_real_stream_matches_resident(n, direction, out_kind, B, chunk):
    if direction == fs.FORWARD:
        x = siggen.tones(2300 + n, B * n // 2).view(np.float32).reshape(B, n)
    else:
        x = siggen.tones(2300 + n, B * (n // 2 + 1)).reshape(B, n // 2 + 1)
    plan = fs.Plan(n, B, direction, out_kind=out_kind, flags=fs.FLAG_REAL)
    ref = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    ref = ref.cpu().numpy()
    out = np.zeros_like(ref)
    sp = fs.Plan(n, chunk, direction, out_kind=out_kind, flags=fs.FLAG_REAL)
    io = Io(x, out)
    rc, committed = sp.stream(io.rd, None, io.wr, None, x.nbytes, 0, chunk)
    assert rc == fs.OK and committed == x.nbytes
    np.testing.assert_array_equal(out, ref)
    # a signal that ends inside a segment: the complete segments, then E_PARTIAL
    out[:] = 0
    io = Io(x, out, limit=x.nbytes - x[0].nbytes // 2)
    rc, committed = sp.stream(io.rd, None, io.wr, None, x.nbytes - x[0].nbytes // 2, 0, chunk)
    assert rc == fs.E_PARTIAL and committed == (B - 1) * x[0].nbytes
    np.testing.assert_array_equal(out[: B - 1], ref[: B - 1])
