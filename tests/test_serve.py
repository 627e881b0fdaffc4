"""The continuous-batching server (fftsrv_*): results are the same alone and
in any mix (bit for bit: every job runs the same tile code either way),
match the FP64 oracle, admission respects the HBM budget, polls time out
instead of blocking, and destroy drains the queue."""
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


def make_jobs(seed=0):
    rng = np.random.default_rng(seed)
    specs = []
    for i, e in enumerate([8, 9, 12, 10, 13, 8, 16, 11, 17, 14, 9, 12]):
        nseg = int(rng.integers(1, 40)) if e <= 12 else int(rng.integers(1, 6))
        direction = fs.FORWARD if i % 2 == 0 else fs.INVERSE
        norm = fs.NORM_BACKWARD if direction == fs.INVERSE else fs.NORM_NONE
        specs.append((1 << e, nseg, direction, norm, 5000 + i))
    jobs = []
    for n, nseg, direction, norm, seed_i in specs:
        x = torch.from_numpy(siggen.uniform(seed_i, nseg * n).reshape(nseg, n)).cuda()
        jobs.append(dict(n=n, nseg=nseg, direction=direction, norm=norm, x=x))
    return jobs


def run_server(jobs, budget=1 << 33, max_inflight=64):
    srv = fs.Server(hbm_budget_bytes=budget, max_inflight_jobs=max_inflight)
    outs, ids = [], []
    for j in jobs:
        y = torch.full_like(j["x"], complex(9.0, 9.0))
        outs.append(y)
        ids.append(srv.submit(j["x"], y, j["n"], j["nseg"], j["direction"], j["norm"]))
    for jid in ids:
        done, status = srv.poll(jid, timeout_us=30_000_000)
        assert done and status == fs.OK
    stats = srv.stats()
    srv.destroy()
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], stats


def test_alone_equals_mix_and_oracle():
    jobs = make_jobs()
    alone = [run_server([j])[0][0] for j in jobs]
    mixed, stats = run_server(jobs)
    assert stats["submitted"] == len(jobs) and stats["completed"] == len(jobs)
    for j, a, m in zip(jobs, alone, mixed):
        np.testing.assert_array_equal(a, m)  # bit for bit, alone and in the mix
        ref = oracle.fft(j["x"].cpu().numpy(), j["direction"], j["norm"])
        assert rel_l2(m, ref) <= tol_fp32(j["n"]), j["n"]


def test_small_jobs_match_plan_path_bitwise():
    jobs = [j for j in make_jobs(1) if j["n"] <= 4096]
    mixed, _ = run_server(jobs)
    for j, m in zip(jobs, mixed):
        plan = fs.Plan(j["n"], j["nseg"], j["direction"], j["norm"])
        np.testing.assert_array_equal(m, plan.exec(j["x"]).cpu().numpy())


def test_budget_is_respected_and_big_jobs_are_split():
    n, nseg = 1 << 16, 24  # 12 MiB in + 12 MiB out: larger than the 4 MiB budget
    x = torch.from_numpy(siggen.tones(77, nseg * n).reshape(nseg, n)).cuda()
    small = make_jobs(2)[:4]
    jobs = small + [dict(n=n, nseg=nseg, direction=fs.FORWARD, norm=fs.NORM_NONE, x=x)]
    budget = 4 << 20
    outs, stats = run_server(jobs, budget=budget, max_inflight=3)
    assert 0 < stats["peak_admitted_bytes"] <= budget
    assert rel_l2(outs[-1], oracle.fft(x.cpu().numpy())) <= tol_fp32(n)


def test_poll_times_out_instead_of_blocking():
    srv = fs.Server(hbm_budget_bytes=1 << 33, max_inflight_jobs=8)
    n, nseg = 1 << 20, 64
    x = torch.zeros(nseg, n, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    ids = [srv.submit(x, y, n, nseg) for _ in range(4)]
    done, st = srv.poll(ids[-1], timeout_us=1)  # 512 MiB x 4 cannot be done in 1 us
    assert not done, (st, fs.last_error(), srv.stats())
    for jid in ids:
        assert srv.poll(jid, timeout_us=60_000_000) == (True, fs.OK)
    with pytest.raises(fs.FFTSegError):
        srv.poll(ids[0])  # a finished job is reported once
    srv.destroy()


def test_poll_latency_is_the_jobs_own():
    # a job polled long after it completed still reports its own time in the
    # server (submit to completion), not the time until the poll
    import time
    srv = fs.Server(hbm_budget_bytes=1 << 33, max_inflight_jobs=8)
    n, nseg = 1 << 16, 256
    x = torch.zeros(nseg, n, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    t0 = time.perf_counter()
    a = srv.submit(x, y, n, nseg)
    b = srv.submit(x, y, 256, 4)
    done, st, lat_a = srv.poll_latency(a, timeout_us=30_000_000)
    t_a = time.perf_counter() - t0
    assert done and st == fs.OK and 0 < lat_a <= t_a
    time.sleep(0.2)
    done, st, lat_b = srv.poll_latency(b, timeout_us=30_000_000)
    assert done and st == fs.OK and 0 < lat_b < 0.2 < time.perf_counter() - t0
    with pytest.raises(fs.FFTSegError):
        srv.poll_latency(a)  # reported once, as by poll
    srv.destroy()


def test_destroy_drains_queue():
    jobs = make_jobs(3)
    srv = fs.Server(hbm_budget_bytes=1 << 30, max_inflight_jobs=2)
    outs = []
    for j in jobs:
        y = torch.empty_like(j["x"])
        outs.append(y)
        srv.submit(j["x"], y, j["n"], j["nseg"], j["direction"], j["norm"])
    srv.destroy()  # waits for every queued job
    torch.cuda.synchronize()
    for j, y in zip(jobs, outs):
        ref = oracle.fft(j["x"].cpu().numpy(), j["direction"], j["norm"])
        assert rel_l2(y.cpu().numpy(), ref) <= tol_fp32(j["n"])


def test_submit_rejects_bad_jobs():
    srv = fs.Server(hbm_budget_bytes=1 << 20, max_inflight_jobs=1)
    x = torch.zeros(1 << 17, dtype=torch.complex64, device="cuda")
    with pytest.raises(fs.FFTSegError) as ei:
        srv.submit(x, x, 1000, 1)
    assert ei.value.status == fs.E_UNSUPPORTED
    with pytest.raises(fs.FFTSegError):
        srv.submit(x, torch.empty_like(x), 1 << 17, 1)  # 2 MiB (in + out) for one segment: over budget
    jid = srv.submit(x, x, 1 << 16, 1)  # in place: 512 KiB fits
    assert srv.poll(jid, timeout_us=10_000_000) == (True, fs.OK)
    srv.destroy()
