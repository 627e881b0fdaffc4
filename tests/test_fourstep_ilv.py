"""n = 2^21..2^24 on the interleaved four-step, against the FP64 oracle.

n = R * M with M = 2^16: the outer pass forms the R decimated-in-frequency
sequences Y_t[j] = w_n^{j t} sum_{t'} x[j + M t'] w_R^{t' t} (stored
interleaved), and the lane-line kernel transforms them 32 at a time into
X[t + R k] = DFT_M(Y_t)[k].  Sizes span several chunks of the workspace with a
ragged last chunk; every sampled segment is compared, and nothing may be
written past the output.
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


@pytest.fixture(autouse=True)
def small_workspace(monkeypatch):
    # 512 MiB workspace chunks (the default is 1 GiB), so that modest batches
    # span several of them
    monkeypatch.setenv("FFTSEG_ILV_WORK_MB", "512")


def run(plan, d, nseg=None):
    buf, y = guard(torch.empty(d.shape, dtype=torch.complex64, device="cuda"))
    plan.exec(d, out=y, nseg=nseg)
    torch.cuda.synchronize()
    plan.check()
    check_guard(buf)
    return y


@pytest.mark.parametrize("log_n,B", [(21, 35), (22, 17), (23, 9), (24, 5)])
@pytest.mark.parametrize("direction,norm", [(FWD, fs.NORM_NONE), (INV, fs.NORM_BACKWARD), (FWD, fs.NORM_ORTHO)])
def test_interleaved_fourstep_matches_oracle(log_n, B, direction, norm):
    n = 1 << log_n
    x = siggen.tones(1700 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, direction, norm)
    info = plan.info()
    assert info["path"] == "four-step" and info["n1"] == n >> 16 and info["n2"] == 1 << 16, info
    chunk = info["work_segs"]
    assert B > chunk and B % chunk, info  # several workspace chunks, the last one ragged
    assert info["launches_per_exec"] == 2 * -(-B // chunk)
    d = torch.from_numpy(x).cuda()
    got = run(plan, d).cpu().numpy()
    sample = np.unique(np.r_[0, chunk - 1, chunk, B // 2, B - 1])
    assert rel_l2(got[sample], oracle.fft(x[sample], direction, norm)) <= tol_fp32(n)
    np.testing.assert_array_equal(run(plan, d).cpu().numpy(), got)  # the dynamic schedule does not change bits


@pytest.mark.parametrize("log_n", [21, 24])
def test_interleaved_fourstep_in_place_and_partial(log_n):
    n = 1 << log_n
    B = 6 if log_n == 24 else 40
    x = siggen.uniform(1750 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, FWD)
    d = torch.from_numpy(x).cuda()
    ref = run(plan, d).cpu().numpy()
    plan.exec(d, out=d)  # in place, chunk after chunk
    torch.cuda.synchronize()
    plan.check()
    np.testing.assert_array_equal(d.cpu().numpy(), ref)
    # a partial batch leaves the rest of the output alone
    d = torch.from_numpy(x).cuda()
    out = torch.full((B, n), complex(3.0, -3.0), dtype=torch.complex64, device="cuda")
    k = 3 if log_n == 24 else 33
    plan.exec(d, out=out, nseg=k)
    torch.cuda.synchronize()
    plan.check()
    o = out.cpu().numpy()
    np.testing.assert_array_equal(o[:k], ref[:k])
    assert np.all(o[k:] == np.complex64(complex(3.0, -3.0)))


def test_interleaved_fourstep_impulses():
    # x = delta[j - j0] => X[k] = w_n^{j0 k} at every k, for an impulse in each
    # of the outer pass's rows and in the last column
    n = 1 << 22
    j0s = [0, 1, 65535, 65536 * 37 + 12345, n - 1]
    x = np.zeros((len(j0s), n), dtype=np.complex64)
    for s, j0 in enumerate(j0s):
        x[s, j0] = 1.0
    plan = fs.Plan(n, len(j0s), FWD)
    got = run(plan, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
    k = np.arange(n, dtype=np.int64)
    for s, j0 in enumerate(j0s):
        ref = np.exp(-2j * np.pi * ((j0 * k) % n) / n)
        assert rel_l2(got[s], ref) <= tol_fp32(n), j0


@pytest.mark.parametrize("log_n,B", [(21, 35), (24, 5)])
def test_interleaved_fourstep_power(log_n, B):
    # |X|^2 at X[t + R k]: the row pass's float boxes of 32 transforms
    n = 1 << log_n
    x = siggen.tones(1780 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, FWD, fs.NORM_ORTHO, out_kind=fs.OUT_POWER)
    assert plan.info()["n1"] == n >> 16, plan.info()
    buf, y = guard(torch.empty(B, n, dtype=torch.float32, device="cuda"))
    plan.exec(torch.from_numpy(x).cuda(), out=y)
    torch.cuda.synchronize()
    plan.check()
    check_guard(buf)
    chunk = plan.info()["work_segs"]
    sample = np.unique(np.r_[0, chunk - 1, chunk, B - 1])
    X = oracle.fft(x[sample], FWD, fs.NORM_ORTHO)
    assert rel_l2(y.cpu().numpy()[sample], X.real ** 2 + X.imag ** 2) <= 2 * tol_fp32(n)
