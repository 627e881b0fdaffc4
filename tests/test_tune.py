"""The autotuner: every schedule it may pick computes the same DFT (checked
against the FP64 oracle), its choice is one of the built schedules, and the
FFTSEG_TUNE_CACHE file is read back and appended to."""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle
import siggen
from tests._util import rel_l2, tol_fp32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PATH_MASK = fs.FLAG_FORCE_TWOPASS | fs.FLAG_FOURSTEP_L2 | fs.FLAG_FOURSTEP_PRODUCER | fs.FLAG_CLUSTER_LOG2(0xF)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1407_6915_gb300 import build
    build.build()


@pytest.mark.parametrize("log_n", [13, 14, 16, 17, 20])
def test_autotuned_plan_matches_oracle(log_n):
    n = 1 << log_n
    B = max(3, (1 << 21) // n) + 1
    flags, ms = fs.autotune(n, B)
    assert flags & ~PATH_MASK == 0 and ms > 0, (flags, ms)
    x = siggen.tones(300 + log_n, B * n).reshape(B, n)
    plan = fs.Plan(n, B, fs.FORWARD, flags=fs.FLAG_AUTOTUNE)
    y = plan.exec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    plan.check()
    err = rel_l2(y.cpu().numpy(), oracle.fft(x, oracle.FORWARD, oracle.NORM_NONE))
    assert err <= tol_fp32(n), (flags, plan.info(), err)


def test_single_schedule_sizes_are_not_timed():
    before = fs.launch_count()
    assert fs.autotune(1024, 100) == (0, -1.0)
    assert fs.autotune(1 << 16, 8, precision=fs.PREC_TC_FP16) == (0, -1.0)
    assert fs.launch_count() == before


def run_child(code, cache):
    env = dict(os.environ, FFTSEG_TUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    return r.stdout


def test_cache_file_is_read_and_appended(tmp_path):
    cache = tmp_path / "tune.txt"
    props = torch.cuda.get_device_properties(0)
    name = props.name.replace(" ", "_")
    # a stored choice (8-CTA clusters for 2^16 at 512 segments) is used without timing
    cache.write_text("%s %d 16 0 0 512 300 1.250000\n" % (name, props.multi_processor_count))
    out = run_child("""
        import paper_1407_6915_gb300 as fs
        b = fs.launch_count()
        print(fs.autotune(1 << 16, 4096), fs.launch_count() - b)
    """, cache)
    assert out.split() == ["(768,", "1.25)", "0"]
    # a new choice is timed and appended
    out = run_child("""
        import paper_1407_6915_gb300 as fs
        print(fs.autotune(1 << 14, 64))
    """, cache)
    lines = cache.read_text().splitlines()
    assert len(lines) == 2 and lines[1].split()[2:6] == ["14", "0", "0", "64"], lines
