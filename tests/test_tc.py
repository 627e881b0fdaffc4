"""GPU parity of the tensor-core radix-16 form (split hi+lo FP16 / BF16 operands,
FP32 accumulation) against the FP64 oracle: relative L2 <= 1e-4 per result,
for the sizes 16^1..16^6, both directions, uniform and tone+noise inputs."""
import functools

import numpy as np
import pytest

import oracle
import siggen
from tests._util import TOL_TC, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402

PRECS = [fs.PREC_TC_FP16, fs.PREC_TC_BF16]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def case(log_n, nseg, family, direction):
    n = 1 << log_n
    gen = siggen.uniform if family == "uniform" else siggen.tones
    x = gen(1000 + 10 * log_n + (family == "tones"), nseg * n).reshape(nseg, n)
    norm = fs.NORM_BACKWARD if direction == fs.INVERSE else fs.NORM_NONE
    return x, oracle.fft(x, direction, norm), norm


def run_tc(prec, log_n, nseg, family, direction):
    x, ref, norm = case(log_n, nseg, family, direction)
    plan = fs.Plan(1 << log_n, nseg, direction, norm, precision=prec)
    y = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    return rel_l2(y.cpu().numpy(), ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("log_n,nseg", [(4, 300), (8, 70), (12, 33), (16, 9), (20, 2)])
@pytest.mark.parametrize("family", ["uniform", "tones"])
@pytest.mark.parametrize("direction", [fs.FORWARD, fs.INVERSE])
def test_tc_matches_oracle(prec, log_n, nseg, family, direction):
    err = run_tc(prec, log_n, nseg, family, direction)
    assert err <= TOL_TC, (prec, log_n, family, direction, err)


@pytest.mark.parametrize("prec", PRECS)
def test_tc_2p24(prec):
    err = run_tc(prec, 24, 1, "tones", fs.FORWARD)
    assert err <= TOL_TC, err


def test_tc_fp16_is_close_to_fp32_accuracy():
    # hi+lo FP16 keeps about 22 bits: far inside the bound, near the FP32 path
    err16 = run_tc(fs.PREC_TC_FP16, 16, 9, "tones", fs.FORWARD)
    err32 = run_tc(fs.PREC_FP32, 16, 9, "tones", fs.FORWARD)
    assert err16 < 10 * max(err32, 1e-7), (err16, err32)


@pytest.mark.parametrize("n,flags", [(1024, 0), (1 << 14, 0), (1 << 16, fs.FLAG_FORCE_TWOPASS)])
def test_tc_rejects_unbuilt_shapes(n, flags):
    with pytest.raises(fs.FFTSegError) as ei:
        fs.Plan(n, 1, fs.FORWARD, precision=fs.PREC_TC_BF16, flags=flags)
    assert ei.value.status == fs.E_UNSUPPORTED
