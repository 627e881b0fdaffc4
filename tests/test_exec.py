"""GPU parity: fftseg_exec against the FP64 oracle on the same seeded inputs.

Tolerance per result: relative L2 <= 2e-6*log2(n) (FP32 path).  Batches are
ragged (segment counts that do not fill the last CTA / workspace chunk) and
span many tiles.
"""
import math

import numpy as np
import pytest

import oracle
import siggen
from tests._util import check_guard, guard, rel_l2, tol_fp32, tol_power

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402

FWD, INV = fs.FORWARD, fs.INVERSE


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def nseg_for(n, target=1 << 20):
    # several tiles plus a ragged remainder
    return max(3, target // n) + 1


def run(plan, x_np, nseg=None):
    x = torch.from_numpy(x_np).cuda()
    dt = torch.float32 if plan.out_kind == fs.OUT_POWER else torch.complex64
    buf, y = guard(torch.empty(x.shape, dtype=dt, device="cuda"))  # canaries past the output's end
    plan.exec(x, out=y, nseg=nseg)
    torch.cuda.synchronize()
    plan.check()  # no kernel gave up a bounded wait
    check_guard(buf)
    return y.cpu().numpy()


@pytest.mark.parametrize("log_n", list(range(1, 18)))
@pytest.mark.parametrize("direction,norm", [(FWD, fs.NORM_NONE), (INV, fs.NORM_BACKWARD)])
def test_single_pass_matches_oracle(log_n, direction, norm):
    n = 1 << log_n
    B = nseg_for(n)
    x = siggen.uniform(100 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, direction, norm)
    got = run(plan, x)
    ref = oracle.fft(x, direction, norm)
    err = rel_l2(got, ref)
    assert err <= tol_fp32(n), (n, plan.info(), err)


@pytest.mark.parametrize("log_n", [8, 9, 12, 13, 16, 17])
@pytest.mark.parametrize("direction", [FWD, INV])
def test_two_pass_forced_matches_oracle(log_n, direction):
    n = 1 << log_n
    B = nseg_for(n)
    x = siggen.tones(200 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, direction, fs.NORM_NONE, flags=fs.FLAG_FORCE_TWOPASS)
    assert plan.info()["path"] == "two-pass"
    got = run(plan, x)
    ref = oracle.fft(x, direction)
    assert rel_l2(got, ref) <= tol_fp32(n)


@pytest.mark.parametrize("log_n,B", [(14, 67), (15, 33), (16, 37), (17, 9), (18, 9), (19, 5), (20, 5), (21, 3),
                                     (22, 2)])
@pytest.mark.parametrize("direction,norm", [(FWD, fs.NORM_NONE), (INV, fs.NORM_BACKWARD)])
@pytest.mark.parametrize("variant", [0, fs.FLAG_FOURSTEP_PRODUCER, fs.FLAG_FOURSTEP_TILES])
def test_persistent_fourstep_matches_oracle(log_n, B, direction, norm, variant):
    # batches that span several chunks of the ring and end in a partial chunk;
    # the default kernel for the length (lane-line at 2^17..2^20, warp-line at
    # 2^16, CTA tiles elsewhere), the producer/consumer kernel and the CTA-tile kernel
    n = 1 << log_n
    x = siggen.tones(800 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, direction, norm, flags=fs.FLAG_FOURSTEP_L2 | variant)
    assert plan.info()["path"] == "four-step"
    got = run(plan, x)
    assert rel_l2(got, oracle.fft(x, direction, norm)) <= tol_fp32(n)
    np.testing.assert_array_equal(run(plan, x), got)  # the dynamic schedule does not change bits


@pytest.mark.parametrize("variant", [0, fs.FLAG_FOURSTEP_PRODUCER])
def test_persistent_fourstep_reuses_its_ring_many_times(variant):
    # 2^14-point segments, 128 per chunk: 1500 segments cycle the 3-chunk ring
    # about four times, so every column tile waits on the release of a row tile
    n, B = 1 << 14, 1500
    x = siggen.uniform(877, B * n).reshape(B, n)
    plan = fs.Plan(n, B, FWD, flags=fs.FLAG_FOURSTEP_L2 | variant)
    assert plan.info()["work_segs"] * 3 * 3 < B
    got = run(plan, x)
    sample = np.r_[0:3, 700:703, B - 3:B]
    assert rel_l2(got[sample], oracle.fft(x[sample])) <= tol_fp32(n)
    np.testing.assert_array_equal(run(plan, x), got)


@pytest.mark.parametrize("direction,norm", [(FWD, fs.NORM_NONE), (INV, fs.NORM_BACKWARD)])
def test_warp_line_fourstep_65536_cycles_ring_in_place(direction, norm):
    # n = 256 x 256 on the warp-local-line kernel: 32 segments per chunk, so 230
    # segments cycle the 3-chunk ring more than twice and end in a partial chunk
    n, B = 1 << 16, 230
    x = siggen.tones(881, B * n).reshape(B, n)
    plan = fs.Plan(n, B, direction, norm, flags=fs.FLAG_FOURSTEP_L2 | fs.FLAG_FOURSTEP_WARP_LINES)
    assert plan.info()["path"] == "four-step"
    got = run(plan, x)
    sample = np.r_[0:2, 95:98, B - 2:B]
    assert rel_l2(got[sample], oracle.fft(x[sample], direction, norm)) <= tol_fp32(n)
    np.testing.assert_array_equal(run(plan, x), got)  # the static schedule is deterministic
    d = torch.from_numpy(x).cuda()
    plan.exec(d, out=d)  # in place
    torch.cuda.synchronize()
    plan.check()
    np.testing.assert_array_equal(d.cpu().numpy(), got)


def test_persistent_fourstep_2p24_power():
    n = 1 << 24
    x = siggen.uniform(824, 2 * n).reshape(2, n)
    plan = fs.Plan(n, 2, FWD, out_kind=fs.OUT_POWER, flags=fs.FLAG_FOURSTEP_L2)
    got = run(plan, x)
    assert rel_l2(got, oracle.power(x)) <= 2 * tol_fp32(n)


@pytest.mark.parametrize("log_n,B", [(18, 9), (19, 5), (20, 5), (21, 2), (22, 1)])
def test_two_pass_large_matches_oracle(log_n, B):
    n = 1 << log_n
    x = siggen.tones(300 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, FWD, flags=fs.FLAG_FORCE_TWOPASS)
    info = plan.info()
    assert info["path"] == "two-pass"
    got = run(plan, x)
    ref = oracle.fft(x, FWD)
    assert rel_l2(got, ref) <= tol_fp32(n), info


def test_default_2p24_matches_oracle():
    n = 1 << 24
    x = siggen.uniform(324, n).reshape(1, n)
    plan = fs.Plan(n, 1, INV, fs.NORM_BACKWARD)
    got = run(plan, x)
    ref = oracle.fft(x, INV, fs.NORM_BACKWARD)
    assert rel_l2(got, ref) <= tol_fp32(n)


@pytest.mark.parametrize("log_n", [24, 20, 16])
def test_impulse_closed_form_at_large_n(log_n):
    # x = delta[j - j0]  =>  X[k] = exp(-2 pi i j0 k / n), checked at every k
    n = 1 << log_n
    j0 = 12345 % n
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    x[j0] = 1.0
    plan = fs.Plan(n, 1, FWD)
    got = plan.exec(x).cpu().numpy().astype(np.complex128)
    k = np.arange(n, dtype=np.int64)
    ref = np.exp(-2j * np.pi * ((j0 * k) % n) / n)
    assert rel_l2(got, ref) <= tol_fp32(n)


@pytest.mark.parametrize("log_n", [10, 16, 20])
def test_power_output(log_n):
    n = 1 << log_n
    B = max(2, (1 << 21) // n) + 1
    x = siggen.tones(400 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, FWD, out_kind=fs.OUT_POWER)
    got = run(plan, x)
    assert got.dtype == np.float32
    ref = oracle.power(x, FWD)
    assert rel_l2(got, ref) <= tol_power(n)


@pytest.mark.parametrize("log_n", [6, 10, 14, 16, 18])
def test_ortho_and_in_place(log_n):
    n = 1 << log_n
    B = nseg_for(n, 1 << 19)
    x = siggen.uniform(500 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, FWD, fs.NORM_ORTHO)
    xd = torch.from_numpy(x).cuda()
    plan.exec_ptr(xd.data_ptr(), xd.data_ptr())  # in place
    got = xd.cpu().numpy()
    assert rel_l2(got, oracle.fft(x, FWD, fs.NORM_ORTHO)) <= tol_fp32(n)
    out_of_place = run(plan, x)
    np.testing.assert_array_equal(out_of_place, got)  # same kernels, same bits


@pytest.mark.parametrize("log_n", [10, 16, 20])
def test_partial_batch_and_empty(log_n):
    n = 1 << log_n
    B = 7
    x = siggen.uniform(600 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, FWD)
    xd = torch.from_numpy(x).cuda()
    out = torch.full((B, n), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    plan.exec(xd, out=out, nseg=3)
    got = out.cpu().numpy()
    assert rel_l2(got[:3], oracle.fft(x[:3], FWD)) <= tol_fp32(n)
    assert np.all(got[3:] == np.complex64(complex(7.0, -7.0)))  # nothing past nseg is written
    plan.exec(xd, out=out, nseg=0)
    with pytest.raises(fs.FFTSegError):
        plan.exec(xd, out=out, nseg=B + 1)


def test_round_trip_and_determinism():
    n, B = 1 << 16, 33
    x = siggen.tones(700, B * n).reshape(B, n)
    xd = torch.from_numpy(x).cuda()
    fwd = fs.Plan(n, B, FWD)
    inv = fs.Plan(n, B, INV, fs.NORM_BACKWARD)
    X1 = fwd.exec(xd)
    X2 = fwd.exec(xd)
    assert torch.equal(X1, X2)
    back = inv.exec(X1).cpu().numpy()
    assert rel_l2(back, x) <= 2 * tol_fp32(n)


@pytest.mark.parametrize("n,B", [(1 << 10, 4096), (1 << 6, 3000), (1 << 12, 37), (1000, 4099), (360, 777)])
def test_back_to_back_dependent_small_batches(n, B):
    # the single-pass kernels' launches (block and mixed-radix) may start
    # while the previous one runs (programmatic launch; each block prefetches
    # its first tiles into L2 before it waits): a chain of eight launches on
    # one stream with no host synchronisation, each reading the previous
    # one's output, in place and out of place, forward and inverse, must give
    # exactly what the same launches give one at a time
    x = siggen.tones(720 + n % 97, B * n).reshape(B, n)
    xd = torch.from_numpy(x).cuda()
    fwd = fs.Plan(n, B, FWD)
    inv = fs.Plan(n, B, INV, fs.NORM_BACKWARD)
    assert fwd.info()["path"] == ("block" if n & (n - 1) == 0 else "mixed-radix")
    plans = [fwd, inv, fwd, inv, fwd, inv, fwd, fwd]
    bufs = [xd.clone(), torch.empty_like(xd)]
    cur = 0
    for k, p in enumerate(plans):  # even k out of place, odd k in place
        if k % 2 == 0:
            p.exec_ptr(bufs[cur].data_ptr(), bufs[1 - cur].data_ptr())
            cur = 1 - cur
        else:
            p.exec_ptr(bufs[cur].data_ptr(), bufs[cur].data_ptr())
    torch.cuda.synchronize()
    ref = xd.clone()
    for k, p in enumerate(plans):
        ref = p.exec(ref)
        torch.cuda.synchronize()
    assert torch.equal(bufs[cur], ref)
    # three round trips, then two unscaled forward transforms: n x[(-j) mod n]
    xr = n * np.roll(x[:, ::-1], 1, axis=1)
    assert rel_l2(bufs[cur].cpu().numpy(), xr) <= 8 * tol_fp32(n)


def test_misaligned_pointer_rejected():
    n = 1024
    plan = fs.Plan(n, 1, FWD)
    x = torch.zeros(n + 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(fs.FFTSegError) as ei:
        plan.exec_ptr(x.data_ptr() + 8, x.data_ptr())
    assert ei.value.status == fs.E_INVALID


def test_launch_counter_counts_kernels():
    n, B = 1 << 20, 9
    plan = fs.Plan(n, B, FWD)
    x = torch.zeros(B, n, dtype=torch.complex64, device="cuda")
    before = fs.launch_count()
    plan.exec(x)
    assert fs.launch_count() - before == plan.info()["launches_per_exec"]


def test_default_schedules():
    # the plan picks these schedules by default (the measured best on GB300):
    # (n, output) -> (path, n1, n2, launches per exec of one segment)
    P = fs.OUT_POWER
    expect = {
        (1 << 4, 0): ("block", 16, 1, 1), (1 << 12, 0): ("block", 4096, 1, 1),
        (1 << 13, 0): ("cluster", 64, 128, 1), (1 << 15, 0): ("cluster", 256, 128, 1),
        (1 << 16, 0): ("four-step", 256, 256, 1), (1 << 16, P): ("four-step", 256, 256, 1),
        (1 << 20, 0): ("four-step", 1024, 1024, 1), (1 << 20, P): ("four-step", 1024, 1024, 1),
        (1 << 21, 0): ("four-step", 32, 65536, 2), (1 << 24, 0): ("four-step", 256, 65536, 2),
        (1 << 24, P): ("four-step", 256, 65536, 2), (1000, 0): ("mixed-radix", 1000, 1, 1),
    }
    for (n, kind), (path, n1, n2, launches) in expect.items():
        plan = fs.Plan(n, 1, FWD, out_kind=P if kind else fs.OUT_COMPLEX)
        info = plan.info()
        assert (info["path"], info["n1"], info["n2"], info["launches_per_exec"]) == (path, n1, n2, launches), (n, kind, info)
