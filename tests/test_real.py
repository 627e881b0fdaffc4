"""Real-signal segments (FFTSEG_FLAG_REAL) against the FP64 oracle.

The paper's records are real single-precision samples (Sec. III: a 1024-point
record is 4096 bytes).  A forward real plan writes the n/2 + 1 bins of each
segment's DFT; an inverse plan goes back from those bins.  Sizes span the
block, cluster and four-step paths of the inner n/2-point transform, batches
span several chunks of the intermediate with a ragged last chunk.
"""
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


def real_signal(seed, nseg, n):
    # the real and imaginary parts of a tones + noise signal, as 2*nseg*n/2 reals
    return siggen.tones(seed, nseg * n // 2).view(np.float32).reshape(nseg, n)


@pytest.fixture(autouse=True)
def small_chunks(monkeypatch):
    # 32 MiB chunks of the n/2-point intermediate (the default is 512 MiB), so
    # that modest batches span several chunks
    monkeypatch.setenv("FFTSEG_REAL_CHUNK_MB", "32")


def nseg_for(n):
    # more than one 32 MiB chunk of the n/2-point intermediate, plus a ragged tail
    return max(3, (48 << 20) // (4 * n) + 1) if n <= (1 << 20) else 3


@pytest.mark.parametrize("log_n", [2, 3, 4, 5, 8, 10, 12, 13, 14, 16, 17, 20])
@pytest.mark.parametrize("norm", [fs.NORM_NONE, fs.NORM_ORTHO])
def test_r2c_matches_oracle(log_n, norm):
    n = 1 << log_n
    B = nseg_for(n)
    x = real_signal(100 + log_n, B, n)
    plan = fs.Plan(n, B, FWD, norm, flags=fs.FLAG_REAL)
    assert plan.info()["path"] == "real"
    buf, got = guard(torch.empty(B, n // 2 + 1, dtype=torch.complex64, device="cuda"))
    plan.exec(torch.from_numpy(x).cuda(), out=got)
    torch.cuda.synchronize()
    plan.check()
    check_guard(buf)  # nothing past the n/2 + 1 bins of the last segment
    got = got.cpu().numpy().astype(np.complex128)
    sample = np.r_[0:2, B // 2, B - 1]
    ref = oracle.rfft(x[sample], norm)
    assert rel_l2(got[sample], ref) <= tol_fp32(n)
    # real bins are real
    assert np.all(got[:, 0].imag == 0) and np.all(got[:, n // 2].imag == 0)


@pytest.mark.parametrize("log_n,B", [(10, 4096), (13, 33)])
def test_back_to_back_real_round_trips(log_n, B):
    # the fused forward kernel may start while the previous kernel runs
    # (programmatic launch, its first tiles prefetched into L2 before it
    # waits): four round trips on one stream with no host synchronisation,
    # each launch reading the previous one's output, give exactly what the
    # same calls give one at a time, and the samples back
    n = 1 << log_n
    x = real_signal(1300 + log_n, B, n)
    fwd = fs.Plan(n, B, FWD, flags=fs.FLAG_REAL)
    inv = fs.Plan(n, B, INV, fs.NORM_BACKWARD, flags=fs.FLAG_REAL)
    xd = torch.from_numpy(x).cuda()
    bins = torch.empty(B, n // 2 + 1, dtype=torch.complex64, device="cuda")
    cur = xd.clone()
    for _ in range(4):
        fwd.exec(cur, out=bins)
        inv.exec(bins, out=cur)
    torch.cuda.synchronize()
    ref = xd.clone()
    for _ in range(4):
        b = fwd.exec(ref)
        torch.cuda.synchronize()
        ref = inv.exec(b)
        torch.cuda.synchronize()
    assert torch.equal(cur, ref)
    assert rel_l2(cur.cpu().numpy(), x) <= 8 * tol_fp32(n)


@pytest.mark.parametrize("log_n", [2, 4, 9, 12, 15, 16, 18])
def test_r2c_power(log_n):
    n = 1 << log_n
    B = 5
    x = real_signal(300 + log_n, B, n)
    plan = fs.Plan(n, B, FWD, out_kind=fs.OUT_POWER, flags=fs.FLAG_REAL)
    got = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    X = oracle.rfft(x)
    assert rel_l2(got.cpu().numpy(), X.real ** 2 + X.imag ** 2) <= 2 * tol_fp32(n)


# forward plans whose n/2-point transform runs on the cluster kernel split the
# spectrum in that kernel's epilogue (bins k and n/2 - k sit in different CTAs
# of the cluster): every cluster shape, both outputs, batches smaller than the
# grid's clusters and ragged ones, every segment compared
@pytest.mark.parametrize("log_n,cflag", [(14, 0), (15, 0), (16, 0), (17, 3), (17, 4), (18, 4)])
@pytest.mark.parametrize("out_kind,norm", [(fs.OUT_COMPLEX, fs.NORM_NONE), (fs.OUT_COMPLEX, fs.NORM_ORTHO),
                                           (fs.OUT_POWER, fs.NORM_NONE)])
def test_r2c_cluster_split(log_n, cflag, out_kind, norm):
    n = 1 << log_n
    B = 37
    x = real_signal(900 + log_n + cflag, B, n)
    flags = fs.FLAG_REAL | (fs.FLAG_CLUSTER_LOG2(cflag) if cflag else 0)
    plan = fs.Plan(n, B, FWD, norm, out_kind=out_kind, flags=flags)
    info = plan.info()
    assert info["launches_per_exec"] == 1 and info["work_bytes"] == 0, info
    power = out_kind == fs.OUT_POWER
    X = oracle.rfft(x, norm)
    ref = X.real ** 2 + X.imag ** 2 if power else X
    d = torch.from_numpy(x).cuda()
    for nseg in (B, 1, 5):
        dt = torch.float32 if power else torch.complex64
        buf, got = guard(torch.empty(nseg, n // 2 + 1, dtype=dt, device="cuda"))
        plan.exec(d, out=got, nseg=nseg)
        torch.cuda.synchronize()
        plan.check()
        check_guard(buf)
        g = got.cpu().numpy()
        assert rel_l2(g, ref[:nseg]) <= (2 if power else 1) * tol_fp32(n), (nseg, rel_l2(g, ref[:nseg]))
        if not power:
            assert np.all(g[:, 0].imag == 0) and np.all(g[:, n // 2].imag == 0)


# inverse plans whose n/2-point transform runs on the cluster kernel (up to
# n/2 = 2^14, batches of up to 64 MiB of samples) join the bins in its column
# pass (each point also reads its mirror bin X[n/2 - m]): batches smaller
# than the grid and ragged, every segment; larger batches run chunked
@pytest.mark.parametrize("log_n,cflag", [(14, 0), (15, 0)])
@pytest.mark.parametrize("norm", [fs.NORM_NONE, fs.NORM_BACKWARD, fs.NORM_ORTHO])
def test_c2r_cluster_join(log_n, cflag, norm):
    n = 1 << log_n
    B = 37
    X = siggen.tones(980 + log_n + cflag, B * (n // 2 + 1)).reshape(B, n // 2 + 1)
    flags = fs.FLAG_REAL | (fs.FLAG_CLUSTER_LOG2(cflag) if cflag else 0)
    plan = fs.Plan(n, B, INV, norm, flags=flags)
    info = plan.info()
    assert info["launches_per_exec"] == 1 and info["work_bytes"] == 0, info
    big = fs.Plan(n, (128 << 20) // (4 * n), INV, norm, flags=flags).info()
    assert big["launches_per_exec"] > 1 and big["work_bytes"] > 0, big
    ref = oracle.irfft(X, n, norm)
    d = torch.from_numpy(X).cuda()
    for nseg in (B, 1, 5):
        buf, got = guard(torch.empty(nseg, n, dtype=torch.float32, device="cuda"))
        plan.exec(d, out=got, nseg=nseg)
        torch.cuda.synchronize()
        plan.check()
        check_guard(buf)
        assert rel_l2(got.cpu().numpy(), ref[:nseg]) <= tol_fp32(n), (nseg, rel_l2(got.cpu().numpy(), ref[:nseg]))


@pytest.mark.parametrize("log_n", [2, 3, 6, 12, 13, 16, 20])
@pytest.mark.parametrize("norm", [fs.NORM_NONE, fs.NORM_BACKWARD, fs.NORM_ORTHO])
def test_c2r_matches_oracle(log_n, norm):
    n = 1 << log_n
    B = nseg_for(n)
    X = oracle.rfft(real_signal(500 + log_n, B, n)).astype(np.complex64)
    X[:, 0] += 0.5j  # the imaginary parts of the real bins are ignored
    X[:, n // 2] -= 0.25j
    plan = fs.Plan(n, B, INV, norm, flags=fs.FLAG_REAL)
    got = plan.exec(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    plan.check()
    assert got.shape == (B, n) and got.dtype == torch.float32
    got = got.cpu().numpy()
    sample = np.r_[0:2, B // 2, B - 1]
    ref = oracle.irfft(X[sample], n, norm)
    assert rel_l2(got[sample], ref) <= tol_fp32(n)


@pytest.mark.parametrize("log_n", [2, 10, 16, 17])
def test_round_trip(log_n):
    n = 1 << log_n
    B = 7
    x = real_signal(700 + log_n, B, n)
    fwd = fs.Plan(n, B, FWD, flags=fs.FLAG_REAL)
    inv = fs.Plan(n, B, INV, fs.NORM_BACKWARD, flags=fs.FLAG_REAL)
    y = inv.exec(fwd.exec(torch.from_numpy(x).cuda()))
    torch.cuda.synchronize()
    assert rel_l2(y.cpu().numpy(), x) <= 2 * tol_fp32(n)


def test_real_plan_rejections():
    with pytest.raises(fs.FFTSegError):
        fs.Plan(2, 1, FWD, flags=fs.FLAG_REAL)  # n >= 4
    with pytest.raises(fs.FFTSegError):
        fs.Plan(1 << 12, 1, FWD, precision=fs.PREC_TC_FP16, flags=fs.FLAG_REAL)  # FP32 only
    with pytest.raises(fs.FFTSegError):
        fs.Plan(1 << 12, 1, INV, out_kind=fs.OUT_POWER, flags=fs.FLAG_REAL)
    plan = fs.Plan(1 << 12, 2, FWD, flags=fs.FLAG_REAL)
    buf = torch.zeros(2 << 12, dtype=torch.float32, device="cuda")
    with pytest.raises(fs.FFTSegError):
        plan.exec_ptr(buf.data_ptr(), buf.data_ptr())  # out of place only
    with pytest.raises(fs.FFTSegError):
        plan.exec_host(torch.zeros(2 << 12), torch.zeros(2 << 12))


@pytest.mark.parametrize("direction", [FWD, INV])
def test_default_chunks(monkeypatch, direction):
    # the default 512 MiB chunks: 2^19-point segments (2 MiB of intermediate
    # each), 300 of them span two chunks, the second one ragged
    monkeypatch.delenv("FFTSEG_REAL_CHUNK_MB")
    n, B = 1 << 19, 300
    plan = fs.Plan(n, B, direction, fs.NORM_NONE if direction == FWD else fs.NORM_BACKWARD, flags=fs.FLAG_REAL)
    info = plan.info()
    assert info["work_segs"] == 256 and info["launches_per_exec"] == 4, info
    x = real_signal(950 + direction, B, n)
    sample = np.r_[0, 255, 256, B - 1]
    if direction == FWD:
        got = plan.exec(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        plan.check()
        ref = oracle.rfft(x[sample])
        assert rel_l2(got.cpu().numpy()[sample], ref) <= tol_fp32(n)
    else:
        X = siggen.tones(960, B * (n // 2 + 1)).reshape(B, n // 2 + 1)  # any bins (imaginary parts of the real ones ignored)
        got = plan.exec(torch.from_numpy(X).cuda())
        torch.cuda.synchronize()
        plan.check()
        ref = oracle.irfft(X[sample], n, fs.NORM_BACKWARD)
        assert rel_l2(got.cpu().numpy()[sample], ref) <= tol_fp32(n)
