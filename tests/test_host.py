"""fftseg_exec_host: a batch in host memory through a chain of plans.

Every segment is transformed on its own (Sec. III), so the chunked, overlapped
host pipeline must give exactly the bits of the resident fftseg_exec of the
same plans, for any chunk size, pinned or pageable host memory, in place or
not; the forward result is also checked against the FP64 oracle.
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


def host_signal(n, nseg, seed, pinned=True):
    x = siggen.tones(seed, nseg * n).reshape(nseg, n)
    t = torch.from_numpy(x)
    return t.pin_memory() if pinned else t.clone()


def resident(plans, h):
    """The same chain through fftseg_exec on the device."""
    x = h.cuda()
    for p in plans:
        x = p.exec(x)
    torch.cuda.synchronize()
    return x.cpu()


@pytest.mark.parametrize("log_n,nseg,chunk", [(10, 37, 8), (12, 20, 7), (16, 9, 4), (17, 5, 2), (13, 11, 0)])
@pytest.mark.parametrize("pinned", [True, False])
def test_forward_equals_resident_and_oracle(log_n, nseg, chunk, pinned):
    n = 1 << log_n
    h = host_signal(n, nseg, 100 + log_n, pinned)
    plan = fs.Plan(n, max(nseg, 8), fs.FORWARD)
    out = torch.empty_like(h)
    plan.exec_host(h, out, nseg, chunk)
    ref = resident([plan], h)
    assert torch.equal(out, ref), "host pipeline differs from the resident exec"
    err = rel_l2(out.numpy(), oracle.fft(h.numpy(), oracle.FORWARD, oracle.NORM_NONE))
    assert err <= tol_fp32(n), err


@pytest.mark.parametrize("log_n,nseg,chunk", [(16, 13, 4), (14, 33, 16), (20, 3, 1)])
def test_round_trip_chain(log_n, nseg, chunk):
    n = 1 << log_n
    h = host_signal(n, nseg, 7 + log_n)
    fwd = fs.Plan(n, chunk, fs.FORWARD)
    inv = fs.Plan(n, chunk, fs.INVERSE, fs.NORM_BACKWARD)
    out = torch.empty_like(h)
    fs.exec_host([fwd, inv], h, out, nseg, chunk)
    # the same kernels on the whole batch at once (a plan's batch does not change a segment's bits)
    ref = resident([fs.Plan(n, nseg, fs.FORWARD), fs.Plan(n, nseg, fs.INVERSE, fs.NORM_BACKWARD)], h)
    assert torch.equal(out, ref)
    assert rel_l2(out.numpy(), h.numpy()) <= 2 * tol_fp32(n)


def test_power_output_in_place():
    n, nseg = 4096, 19
    h = host_signal(n, nseg, 5)
    ref = resident([fs.Plan(n, nseg, fs.FORWARD, out_kind=fs.OUT_POWER)], h)
    plan = fs.Plan(n, 6, fs.FORWARD, out_kind=fs.OUT_POWER)
    buf = h.clone().pin_memory()
    plan.exec_host(buf, buf, nseg, 5)  # power rows land in the first half of the same buffer
    got = buf.view(torch.float32).view(-1)[: nseg * n].view(nseg, n)
    assert torch.equal(got, ref)


def test_in_place_complex_and_staging_regrow():
    n, nseg = 1024, 50
    h = host_signal(n, nseg, 9)
    plan = fs.Plan(n, 32, fs.FORWARD)
    ref = resident([fs.Plan(n, nseg, fs.FORWARD)], h)
    a = h.clone().pin_memory()
    plan.exec_host(a, a, nseg, 3)    # small staging first
    assert torch.equal(a, ref)
    b = h.clone().pin_memory()
    plan.exec_host(b, b, nseg, 32)   # a larger chunk regrows it
    assert torch.equal(b, ref)


def test_zero_segments_is_a_no_op():
    plan = fs.Plan(1024, 4, fs.FORWARD)
    h = torch.zeros(4, 1024, dtype=torch.complex64)
    plan.exec_host(h, h, 0)


def test_rejections():
    n = 1024
    a = fs.Plan(n, 8, fs.FORWARD)
    b = fs.Plan(2 * n, 8, fs.FORWARD)
    pw = fs.Plan(n, 8, fs.FORWARD, out_kind=fs.OUT_POWER)
    h = torch.zeros(8, n, dtype=torch.complex64)
    cases = [
        lambda: fs.exec_host([], h, h, 8),                      # no plans
        lambda: fs.exec_host([a, b], h, h, 8),                  # lengths differ
        lambda: fs.exec_host([pw, a], h, h, 8),                 # power output before the last plan
        lambda: fs.exec_host([a], h, h, 8, chunk_segments=9),  # chunk above the batch
        lambda: fs.exec_host([a], h, h, -1),                    # negative count
        lambda: fs.exec_host([a], 0, h, 8),                     # NULL input
    ]
    for f in cases:
        with pytest.raises(fs.FFTSegError) as ei:
            f()
        assert ei.value.status == fs.E_INVALID
