"""Parity at the workloads' full sizes, in the launch configurations bench.py
times, on sampled segments the FP64 oracle computes one by one.

- 4096 x 1024 forward (uniform, seed 0): the whole output against the oracle.
- 16384 x 65536 forward then inverse (tones + noise, seed 1): one plan of the
  full batch, as the bench runs it; the first, last and six seeded segments of
  the spectrum against the oracle, and the round trip over every segment.
- 2^29 samples (4 GiB) at n = 2^12, 2^16, 2^20, 2^24, uniform (seed 3) and
  tones + noise (seed 4), FP32 and the two tensor-core precisions: sampled
  segments against the oracle, each within its bound.
- The 2^20-point |X|^2 stream (tones + noise, seed 2) in chunks of 64
  segments, as the bench streams it: sampled segments against the oracle.

Each segment is transformed on its own (Sec. III), so a sampled segment's
oracle result is exactly what the full batch must hold at that offset.
"""
import ctypes

import numpy as np
import pytest

import oracle
import siggen
from tests._util import TOL_TC, rel_l2, tol_fp32, tol_power

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()


def pinned_signal(kind, seed, count):
    h = torch.empty(count, dtype=torch.complex64, pin_memory=True)
    siggen.fill_pointer(kind, seed, 0, count, h.data_ptr())
    return h


def sample_rows(nseg, k, seed):
    rng = np.random.default_rng(seed)
    rows = {0, nseg - 1} | set(int(r) for r in rng.integers(0, nseg, size=k))
    return sorted(rows)


def test_c1_4096x1024_forward_whole_output():
    n, B = 1024, 4096
    x = siggen.uniform(0, B * n).reshape(B, n)
    plan = fs.Plan(n, B, fs.FORWARD)
    y = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    err = rel_l2(y.cpu().numpy(), oracle.fft(x, oracle.FORWARD, oracle.NORM_NONE))
    assert err <= tol_fp32(n), err


def test_c2_16384x65536_forward_inverse():
    n, B = 1 << 16, 16384
    h = pinned_signal(siggen.KIND_TONES, 1, B * n)
    x = h.cuda().view(B, n)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    fwd = fs.Plan(n, B, fs.FORWARD, fs.NORM_NONE)
    inv = fs.Plan(n, B, fs.INVERSE, fs.NORM_BACKWARD)
    fwd.exec(x, out=y)
    inv.exec(y, out=z)
    torch.cuda.synchronize()
    fwd.check()
    inv.check()
    rows = sample_rows(B, 6, 21)
    xs = h.view(B, n)[rows].numpy()
    ref = oracle.fft(xs, oracle.FORWARD, oracle.NORM_NONE)
    got = y[rows].cpu().numpy()
    for i, r in enumerate(rows):
        assert rel_l2(got[i], ref[i]) <= tol_fp32(n), (r, rel_l2(got[i], ref[i]))
    # the inverse of the sampled spectra against the oracle's inverse of the same spectra
    ref_inv = oracle.fft(got, oracle.INVERSE, oracle.NORM_BACKWARD)
    assert rel_l2(z[rows].cpu().numpy(), ref_inv) <= tol_fp32(n)
    # round trip over all 2^30 samples, on the device
    rt = float(torch.linalg.vector_norm((z - x).flatten()) / torch.linalg.vector_norm(x.flatten()))
    assert rt <= 2 * tol_fp32(n), rt


C4_SIZES = [12, 16, 20, 24]
C4_PRECS = [fs.PREC_FP32, fs.PREC_TC_FP16, fs.PREC_TC_BF16]


@pytest.fixture(scope="module")
def c4_signals():
    count = 1 << 29
    return {"uniform": pinned_signal(siggen.KIND_UNIFORM, 3, count),
            "tones": pinned_signal(siggen.KIND_TONES, 4, count)}


@pytest.mark.parametrize("family", ["uniform", "tones"])
@pytest.mark.parametrize("log_n", C4_SIZES)
def test_c4_4gib_batches_fp32_and_tensor_core(c4_signals, family, log_n):
    n = 1 << log_n
    B = (1 << 29) // n
    h = c4_signals[family]
    x = h.cuda().view(B, n)
    y = torch.empty_like(x)
    rows = sample_rows(B, {12: 4, 16: 3, 20: 1, 24: 0}[log_n], 40 + log_n)
    ref = oracle.fft(h.view(B, n)[rows].numpy(), oracle.FORWARD, oracle.NORM_NONE)
    for prec in C4_PRECS:
        plan = fs.Plan(n, B, fs.FORWARD, precision=prec)
        plan.exec(x, out=y)
        torch.cuda.synchronize()
        plan.check()
        got = y[rows].cpu().numpy()
        bound = tol_fp32(n) if prec == fs.PREC_FP32 else TOL_TC
        for i, r in enumerate(rows):
            err = rel_l2(got[i], ref[i])
            assert err <= bound, (family, n, prec, r, err)
        del plan


def test_c3_stream_2p20_power_in_64_segment_chunks():
    n, chunk, nseg = 1 << 20, 64, 128
    total = nseg * n * 8
    plan = fs.Plan(n, chunk, fs.FORWARD, out_kind=fs.OUT_POWER)
    out = np.zeros(nseg * n, dtype=np.float32)
    src = siggen.source(siggen.KIND_TONES, 2, total)
    snk = siggen.sink(out.view(np.uint8))
    rc, committed = plan.stream(siggen.read_fn_ptr(), ctypes.addressof(src), siggen.write_fn_ptr(),
                                ctypes.addressof(snk), total, 0, chunk)
    assert rc == fs.OK and committed == total
    out = out.reshape(nseg, n)
    for r in (0, 63, 64, nseg - 1):
        xs = siggen.tones(2, n, t0=r * n).reshape(1, n)
        ref = oracle.power(xs, oracle.FORWARD, oracle.NORM_NONE)[0]
        err = rel_l2(out[r], ref)
        assert err <= tol_power(n), (r, err)
