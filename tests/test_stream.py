"""fftseg_stream: the out-of-core chunker against resident fftseg_exec and the oracle.

Sec. III: the file is cut into blocks of segments, each block is transformed
with a batched plan, and outputs are merged in positional order.  Chunk size
(the paper's block size) must not change any result bit; failures are made on
the host (reader/writer callbacks that fail), never on the GPU.
"""
import ctypes

import numpy as np
import pytest

import oracle
import siggen
from tests._util import rel_l2, tol_fp32, tol_power

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()


RD = None


def rd_ptr():
    return siggen.read_fn_ptr()


def wr_ptr():
    return siggen.write_fn_ptr()


def stream_into(plan, total_bytes, chunk, kind=siggen.KIND_TONES, seed=11, start=0, out=None,
                rfail=-1, wfail=-1):
    n = plan.n
    seg_out = n * (4 if plan.out_kind == fs.OUT_POWER else 8)
    nseg_cap = -(-total_bytes // (n * 8))
    if out is None:
        out = np.zeros(nseg_cap * seg_out, dtype=np.uint8)
    src = siggen.source(kind, seed, total_bytes, fail_at_call=rfail)
    snk = siggen.sink(out, fail_at_call=wfail)
    rc, committed = plan.stream(rd_ptr(), ctypes.addressof(src), wr_ptr(), ctypes.addressof(snk),
                                total_bytes, start, chunk)
    return rc, committed, out, snk


@pytest.mark.parametrize("log_n,out_kind", [(10, fs.OUT_COMPLEX), (10, fs.OUT_POWER), (16, fs.OUT_POWER),
                                            (20, fs.OUT_POWER), (13, fs.OUT_COMPLEX)])
def test_stream_equals_resident_exec_and_oracle(log_n, out_kind):
    n = 1 << log_n
    nseg = max(6, (1 << 22) // n) + 1
    total = nseg * n * 8
    plan = fs.Plan(n, 8 if log_n >= 16 else 64, fs.FORWARD, out_kind=out_kind)
    rc, committed, out, snk = stream_into(plan, total, 0)
    assert rc == fs.OK and committed == total
    dt = np.float32 if out_kind == fs.OUT_POWER else np.complex64
    got = out.view(dt).reshape(nseg, n)
    x = siggen.tones(11, nseg * n).reshape(nseg, n)
    # bitwise equal to the resident batched transform (same kernels)
    res = fs.Plan(n, nseg, fs.FORWARD, out_kind=out_kind)
    ref_gpu = res.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, ref_gpu)
    if out_kind == fs.OUT_POWER:
        assert rel_l2(got, oracle.power(x)) <= tol_power(n)
    else:
        assert rel_l2(got, oracle.fft(x)) <= tol_fp32(n)
    ph = plan.stream_phases()
    assert ph["wall_ms"] > 0 and ph["fft_ms"] > 0


def test_chunk_size_does_not_change_bits():
    n = 1024
    nseg = 203
    total = nseg * n * 8
    plan = fs.Plan(n, 64, fs.FORWARD)
    outs = [stream_into(plan, total, c)[2] for c in (1, 7, 64)]
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)


def test_reader_failure_then_resume():
    n, chunk = 1024, 5
    nseg = 60
    total = nseg * n * 8
    plan = fs.Plan(n, chunk, fs.FORWARD)
    full = stream_into(plan, total, chunk)[2]
    rc, committed, out, _ = stream_into(plan, total, chunk, rfail=4)
    assert rc == fs.E_IO
    # chunks 0..3 were read; every one of them is written before returning
    assert committed == 4 * chunk * n * 8
    rc, committed2, out, _ = stream_into(plan, total, chunk, start=committed, out=out)
    assert rc == fs.OK and committed2 == total
    np.testing.assert_array_equal(out, full)


def test_writer_failure_then_resume():
    n, chunk = 4096, 3
    nseg = 40
    total = nseg * n * 8
    plan = fs.Plan(n, chunk, fs.FORWARD)
    full = stream_into(plan, total, chunk)[2]
    rc, committed, out, snk = stream_into(plan, total, chunk, wfail=2)
    assert rc == fs.E_IO
    assert committed == 2 * chunk * n * 8  # writes 0 and 1 succeeded
    rc, committed2, out, _ = stream_into(plan, total, chunk, start=committed, out=out)
    assert rc == fs.OK and committed2 == total
    np.testing.assert_array_equal(out, full)


def test_partial_tail_and_zero_pad():
    n = 1024
    nseg = 10
    total = nseg * n * 8 + 3 * 8  # 3 samples into an eleventh segment
    plan = fs.Plan(n, 4, fs.FORWARD)
    rc, committed, out, _ = stream_into(plan, total, 4)
    assert rc == fs.E_PARTIAL and committed == nseg * n * 8
    padded = fs.Plan(n, 4, fs.FORWARD, flags=fs.FLAG_ZERO_PAD)
    rc, committed, out, _ = stream_into(padded, total, 4)
    assert rc == fs.OK and committed == (nseg + 1) * n * 8
    x = np.zeros((nseg + 1) * n, dtype=np.complex64)
    x[:nseg * n + 3] = siggen.tones(11, nseg * n + 3)
    got = out.view(np.complex64).reshape(nseg + 1, n)
    assert rel_l2(got, oracle.fft(x.reshape(nseg + 1, n))) <= tol_fp32(n)


def test_python_callbacks():
    n, nseg = 256, 37
    x = siggen.uniform(5, nseg * n)
    raw = x.view(np.uint8)
    out = np.zeros(nseg * n * 4, dtype=np.uint8)
    offsets = []

    def reader(ctx, off, dst, nbytes):
        nbytes = min(nbytes, raw.size - off)
        ctypes.memmove(dst, raw.ctypes.data + off, nbytes)
        return nbytes

    def writer(ctx, off, src, nbytes):
        offsets.append(off)
        ctypes.memmove(out.ctypes.data + off, src, nbytes)
        return 0

    plan = fs.Plan(n, 8, fs.FORWARD, out_kind=fs.OUT_POWER)
    rc, committed = plan.stream(reader, None, writer, None, raw.size, 0, 8)
    assert rc == fs.OK and committed == raw.size
    assert offsets == sorted(offsets) and offsets[0] == 0  # positional order
    assert rel_l2(out.view(np.float32).reshape(nseg, n), oracle.power(x.reshape(nseg, n))) <= tol_power(n)


def test_stream_argument_errors():
    plan = fs.Plan(1024, 4, fs.FORWARD)
    src = siggen.source(siggen.KIND_UNIFORM, 1, 8192 * 4)
    snk = siggen.sink(None)
    with pytest.raises(fs.FFTSegError):
        plan.stream(rd_ptr(), ctypes.addressof(src), wr_ptr(), ctypes.addressof(snk), 8192 * 4, 100, 4)
    with pytest.raises(fs.FFTSegError):
        plan.stream(rd_ptr(), ctypes.addressof(src), wr_ptr(), ctypes.addressof(snk), 8192 * 4, 0, 5)


# ------------------------------------------------- lending sources (view)

@pytest.mark.parametrize("log_n,chunk,out_kind", [(10, 64, fs.OUT_COMPLEX), (16, 8, fs.OUT_POWER),
                                                  (17, 4, fs.OUT_COMPLEX)])
def test_stream_view_equals_copying_reader(log_n, chunk, out_kind):
    # a pinned pool lent in place (fftseg_stream_view) gives the same bits as
    # the copying reader over the same bytes, and matches the oracle
    n = 1 << log_n
    nseg = 5 * chunk + 3  # a partial last chunk
    total = nseg * n * 8
    pool = torch.empty(nseg * n, dtype=torch.complex64, pin_memory=True)
    siggen.fill_pointer(siggen.KIND_TONES, 21, 0, nseg * n, pool.data_ptr())
    plan = fs.Plan(n, chunk, fs.FORWARD, out_kind=out_kind)
    seg_out = n * (4 if out_kind == fs.OUT_POWER else 8)
    a = np.zeros(nseg * seg_out, dtype=np.uint8)
    b = np.zeros(nseg * seg_out, dtype=np.uint8)
    # (every ctypes context the C side holds a pointer to stays referenced)
    src, snk_a = siggen.pool_source(pool.data_ptr(), total, total), siggen.sink(a)
    rc, committed = plan.stream_view(siggen.view_fn_ptr(), ctypes.addressof(src), wr_ptr(),
                                     ctypes.addressof(snk_a), total, 0, chunk)
    assert rc == fs.OK and committed == total
    src2, snk_b = siggen.pool_source(pool.data_ptr(), total, total), siggen.sink(b)
    rc, committed = plan.stream(rd_ptr(), ctypes.addressof(src2), wr_ptr(), ctypes.addressof(snk_b),
                                total, 0, chunk)
    assert rc == fs.OK and committed == total
    np.testing.assert_array_equal(a, b)
    x = pool.numpy().reshape(nseg, n)
    if out_kind == fs.OUT_POWER:
        assert rel_l2(a.view(np.float32).reshape(nseg, n), oracle.power(x)) <= tol_power(n)
    else:
        assert rel_l2(a.view(np.complex64).reshape(nseg, n), oracle.fft(x)) <= tol_fp32(n)


def test_stream_view_failure_resume_and_tail():
    n, chunk, nseg = 1 << 12, 16, 70
    total = nseg * n * 8
    pool = torch.empty(nseg * n, dtype=torch.complex64, pin_memory=True)
    siggen.fill_pointer(siggen.KIND_UNIFORM, 22, 0, nseg * n, pool.data_ptr())
    plan = fs.Plan(n, chunk, fs.FORWARD)
    ref = plan.exec(pool.cuda().view(nseg, n)[:chunk], nseg=chunk)  # the first chunk, resident
    out = np.zeros(nseg * n * 8, dtype=np.uint8)
    # the source fails on its third call: two chunks are complete, E_IO, and
    # the committed offset is where a later call resumes
    src, snk = siggen.pool_source(pool.data_ptr(), total, total, fail_at_call=2), siggen.sink(out)
    rc, committed = plan.stream_view(siggen.view_fn_ptr(), ctypes.addressof(src), wr_ptr(),
                                     ctypes.addressof(snk), total, 0, chunk)
    assert rc == fs.E_IO and committed == 2 * chunk * n * 8
    src, snk = siggen.pool_source(pool.data_ptr(), total, total), siggen.sink(out)
    rc, committed = plan.stream_view(siggen.view_fn_ptr(), ctypes.addressof(src), wr_ptr(),
                                     ctypes.addressof(snk), total, committed, chunk)
    assert rc == fs.OK and committed == total
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.view(np.complex64)[:chunk * n], ref.cpu().numpy().ravel())
    full = fs.Plan(n, nseg, fs.FORWARD).exec(pool.cuda().view(nseg, n)).cpu().numpy().ravel()
    np.testing.assert_array_equal(out.view(np.complex64), full)
    # a signal that ends inside a segment: E_PARTIAL, or zero-padded with the flag
    short = total - 3 * 8
    scratch = np.zeros_like(out)
    src, snk = siggen.pool_source(pool.data_ptr(), total, short), siggen.sink(scratch)
    rc, committed = plan.stream_view(siggen.view_fn_ptr(), ctypes.addressof(src), wr_ptr(),
                                     ctypes.addressof(snk), short, 0, chunk)
    assert rc == fs.E_PARTIAL and committed == (nseg - 1) * n * 8
    padded = fs.Plan(n, chunk, fs.FORWARD, flags=fs.FLAG_ZERO_PAD)
    out2 = np.zeros_like(out)
    src, snk = siggen.pool_source(pool.data_ptr(), total, short), siggen.sink(out2)
    rc, committed = padded.stream_view(siggen.view_fn_ptr(), ctypes.addressof(src), wr_ptr(),
                                       ctypes.addressof(snk), short, 0, chunk)
    assert rc == fs.OK
    last = pool.numpy()[(nseg - 1) * n:].copy()
    last[-3:] = 0
    want = oracle.fft(last.reshape(1, n))
    assert rel_l2(out2.view(np.complex64)[(nseg - 1) * n:].reshape(1, n), want) <= tol_fp32(n)
    # frame plans stream through the copying reader only
    fp = fs.FramePlan(n, n // 2, 4)
    assert lib_status(fp) == fs.E_UNSUPPORTED


def lib_status(plan):
    committed = ctypes.c_int64(0)
    return fs.lib().fftseg_stream_view(plan._h, ctypes.c_void_p(siggen.view_fn_ptr()), None,
                                       ctypes.c_void_p(wr_ptr()), None, 1 << 20, 0, 0, ctypes.byref(committed))
