"""File-backed streaming (fftseg_stream_file): the paper's pipeline end to end
(Sec. III) -- a signal file cut into segments, each transformed, the results
written to a file in positional order.  The file's results equal, bit for bit,
the same plan run on the resident signal, and match the FP64 oracle; a resumed
run completes the output; I/O failures and a partial tail are reported.
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


def resident(x, n, out_kind):
    plan = fs.Plan(n, x.size // n, fs.FORWARD, out_kind=out_kind)
    y = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    return y.cpu().numpy().ravel()


@pytest.mark.parametrize("direct", [True, False])
@pytest.mark.parametrize("n,B,chunk,out_kind", [(256, 300, 64, fs.OUT_COMPLEX), (4096, 70, 16, fs.OUT_COMPLEX),
                                                (1 << 16, 11, 4, fs.OUT_POWER)])
def test_file_stream_equals_resident_and_oracle(tmp_path, n, B, chunk, out_kind, direct):
    x = siggen.tones(950 + n, B * n)
    src, dst = tmp_path / "signal.c64", tmp_path / "spectra.out"
    x.tofile(src)
    plan = fs.Plan(n, chunk, fs.FORWARD, out_kind=out_kind)
    rc, committed = plan.stream_file(src, dst, chunk_segments=chunk, direct=direct)
    assert rc == fs.OK and committed == B * n * 8
    got = np.fromfile(dst, dtype=np.float32 if out_kind == fs.OUT_POWER else np.complex64)
    np.testing.assert_array_equal(got, resident(x, n, out_kind))
    k = np.r_[0, B - 1]
    ref = oracle.fft(x.reshape(B, n)[k])
    if out_kind == fs.OUT_POWER:
        assert rel_l2(got.reshape(B, n)[k], ref.real ** 2 + ref.imag ** 2) <= 2 * tol_fp32(n)
    else:
        assert rel_l2(got.reshape(B, n)[k], ref) <= tol_fp32(n)
    ph = plan.stream_phases()
    assert ph["read_ms"] > 0 and ph["write_ms"] > 0 and ph["wall_ms"] > 0


def test_file_stream_resumes(tmp_path):
    n, B, chunk = 4096, 40, 8
    x = siggen.tones(977, B * n)
    src, dst = tmp_path / "signal.c64", tmp_path / "spectra.out"
    x.tofile(src)
    plan = fs.Plan(n, chunk, fs.FORWARD)
    assert plan.stream_file(src, dst, chunk_segments=chunk)[0] == fs.OK
    full = np.fromfile(dst, dtype=np.complex64)
    # lose the second half of the output, then resume from segment 24
    part = full.copy()
    part[24 * n:] = 0
    part.tofile(dst)
    rc, committed = plan.stream_file(src, dst, start_offset=24 * n * 8, chunk_segments=chunk)
    assert rc == fs.OK and committed == B * n * 8
    np.testing.assert_array_equal(np.fromfile(dst, dtype=np.complex64), full)


def test_file_stream_errors(tmp_path):
    n = 1024
    plan = fs.Plan(n, 4, fs.FORWARD)
    rc, committed = plan.stream_file(tmp_path / "missing.c64", tmp_path / "o.out")
    assert rc == fs.E_IO and committed == 0
    x = siggen.uniform(3, 5 * n + 100)  # five segments and a partial one
    x.tofile(tmp_path / "tail.c64")
    rc, committed = plan.stream_file(tmp_path / "tail.c64", tmp_path / "t.out", chunk_segments=4)
    assert rc == fs.E_PARTIAL and committed == 5 * n * 8
    got = np.fromfile(tmp_path / "t.out", dtype=np.complex64)
    assert got.size == 5 * n
    np.testing.assert_array_equal(got, resident(x[: 5 * n], n, fs.OUT_COMPLEX))


@pytest.mark.parametrize("world", [2, 3])
def test_file_stream_ranges_assemble_the_output(tmp_path, world):
    # the sharded stream's per-rank calls, one after another in one process:
    # each writes its segment range [first, last) at its own output offsets
    from paper_1407_6915_gb300.shard import segment_range, stream_file_sharded
    n, B, chunk = 4096, 23, 4
    x = siggen.tones(991, B * n)
    src, dst = tmp_path / "signal.c64", tmp_path / "spectra.out"
    x.tofile(src)
    ref = resident(x, n, fs.OUT_COMPLEX)
    np.zeros(B * n, dtype=np.complex64).tofile(dst)  # stale content must be overwritten, not truncated
    plan = fs.Plan(n, chunk, fs.FORWARD)
    for r in reversed(range(world)):  # any order: each range lands at its offsets
        first, last = segment_range(B, r, world)
        rc, committed = plan.stream_file(src, dst, start_offset=first * n * 8, end_offset=last * n * 8,
                                         chunk_segments=chunk, keep_output=True)
        assert rc == fs.OK and committed == last * n * 8
    np.testing.assert_array_equal(np.fromfile(dst, dtype=np.complex64), ref)
    # the sharded driver with a no-op barrier, world 1
    dst2 = tmp_path / "one.out"
    rc, committed = stream_file_sharded(plan, src, dst2, 0, 1, lambda: None, chunk_segments=chunk)
    assert rc == fs.OK and committed == B * n * 8
    np.testing.assert_array_equal(np.fromfile(dst2, dtype=np.complex64), ref)


def test_file_stream_frames_real_and_sharded_ranges(tmp_path):
    # a frame plan through the file stream equals the resident frame plan,
    # whole and as two frame ranges (the sharded driver's calls, in order)
    from paper_1407_6915_gb300.shard import stream_file_sharded
    n, hop, F = 1024, 384, 150
    x = siggen.tones(995, (F - 1) * hop + n + 100)  # 100 samples start no frame
    src = tmp_path / "signal.c64"
    x.tofile(src)
    ref = fs.FramePlan(n, hop, F, fs.WINDOW_HANN).exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    plan = fs.FramePlan(n, hop, 32, fs.WINDOW_HANN)
    rc, committed = plan.stream_file(src, tmp_path / "frames.out", chunk_segments=32)
    assert rc == fs.OK and committed == F * hop * 8
    np.testing.assert_array_equal(np.fromfile(tmp_path / "frames.out", dtype=np.complex64).reshape(F, n), ref)
    for r in range(2):
        rc, _ = stream_file_sharded(plan, src, tmp_path / "frames2.out", r, 2, lambda: None, chunk_segments=32)
        assert rc == fs.OK
    np.testing.assert_array_equal(np.fromfile(tmp_path / "frames2.out", dtype=np.complex64).reshape(F, n), ref)
    # a real-signal plan: 4n bytes of float32 samples per segment in
    n, B = 4096, 50
    xr = siggen.tones(996, B * n // 2).view(np.float32).reshape(B, n)
    xr.tofile(tmp_path / "real.f32")
    rplan = fs.Plan(n, B, fs.FORWARD, flags=fs.FLAG_REAL)
    rref = rplan.exec(torch.from_numpy(xr).cuda())
    torch.cuda.synchronize()
    sp = fs.Plan(n, 16, fs.FORWARD, flags=fs.FLAG_REAL)
    rc, committed = sp.stream_file(tmp_path / "real.f32", tmp_path / "real.out", chunk_segments=16)
    assert rc == fs.OK and committed == xr.nbytes
    got = np.fromfile(tmp_path / "real.out", dtype=np.complex64).reshape(B, n // 2 + 1)
    np.testing.assert_array_equal(got, rref.cpu().numpy())


def test_command_line_job(tmp_path):
    # python -m paper_1407_6915_gb300: the whole file through one GPU, as the
    # resident plan would transform it
    from paper_1407_6915_gb300 import __main__ as cli
    n, B = 4096, 40
    x = siggen.tones(997, B * n)
    x.tofile(tmp_path / "in.c64")
    rc = cli.main([str(tmp_path / "in.c64"), str(tmp_path / "out.f32"), "--n", str(n), "--power"])
    assert rc == 0
    got = np.fromfile(tmp_path / "out.f32", dtype=np.float32)
    np.testing.assert_array_equal(got, resident(x, n, fs.OUT_POWER))
