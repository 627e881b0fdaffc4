"""The command-line job (python -m paper_1407_6915_gb300): argument handling,
the plan it asks for, and its one-process and two-rank (gloo) runs on the CPU
with a stand-in plan that keeps the library's positional contract (the GPU
side of a run is fftseg_stream_file, covered by tests/test_file.py)."""
import datetime
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import paper_1407_6915_gb300 as fs  # noqa: E402
from paper_1407_6915_gb300 import __main__ as cli  # noqa: E402


class FakePlan:
    """fftseg_stream_file's positional contract for segments (complex64 n
    points -> n points at the same offsets) or frames (frame f -> offset
    f*n*8); the 'transform' negates the samples."""

    def __init__(self, kind, kw):
        self.kind, self.kw = kind, kw
        self.n = kw["n"]
        if kind == "frames":
            self.hop = kw["hop"]

    def segment_bytes(self):
        return self.n * 8, self.n * 8

    def stream_file(self, in_path, out_path, start_offset=0, end_offset=0, chunk_segments=0, direct=True,
                    keep_output=False):
        x = np.fromfile(in_path, dtype=np.complex64)
        end = x.size if end_offset == 0 else end_offset // 8
        mode = "r+b" if (keep_output or start_offset) and os.path.exists(out_path) else "wb"
        with open(out_path, mode) as f:
            if self.kind == "frames":
                f0 = start_offset // (self.hop * 8)
                nf = 0 if end - start_offset // 8 < self.n else (end - start_offset // 8 - self.n) // self.hop + 1
                for k in range(nf):
                    s = (f0 + k) * self.hop
                    f.seek((f0 + k) * self.n * 8)
                    f.write((-x[s: s + self.n]).tobytes())
                return fs.OK, (f0 + nf) * self.hop * 8
            s0, s1 = start_offset // 8, end - end % self.n
            f.seek(start_offset)
            f.write((-x[s0:s1]).tobytes())
            return (fs.OK if end % self.n == 0 else fs.E_PARTIAL), s1 * 8

    def stream_phases(self):
        return {"read_ms": 1.0, "wall_ms": 2.0}


def test_plan_spec():
    kind, kw, chunk = cli.plan_spec(cli.parse(["a", "b", "--n", "1024"]), 1 << 30)
    assert kind == "segments" and kw["direction"] == fs.FORWARD and kw["flags"] == 0 and chunk == 32768
    kind, kw, chunk = cli.plan_spec(cli.parse(["a", "b", "--n", "4096", "--real", "--power", "--chunk", "100"]),
                                    4096 * 4 * 10)
    assert kw["flags"] == fs.FLAG_REAL and kw["out_kind"] == fs.OUT_POWER and chunk == 10  # at most the file's
    kind, kw, chunk = cli.plan_spec(cli.parse(["a", "b", "--n", "1024", "--inverse", "--norm", "backward"]),
                                    8 << 20)
    assert kw["direction"] == fs.INVERSE and kw["norm"] == fs.NORM_BACKWARD and chunk == 1024
    kind, kw, chunk = cli.plan_spec(cli.parse(["a", "b", "--n", "1024", "--frames", "256", "--window", "rect"]),
                                    (99 * 256 + 1024) * 8)
    assert kind == "frames" and kw["hop"] == 256 and kw["window"] == fs.WINDOW_RECT and chunk == 100
    for bad in (["a", "b"], ["a", "b", "--n", "8", "--frames", "4", "--inverse"],
                ["a", "b", "--n", "8", "--real", "--frames", "4"], ["a", "b", "--n", "8", "--real", "--inverse",
                                                                    "--power"]):
        with pytest.raises(SystemExit):
            cli.parse(bad)


def test_one_process_run(tmp_path, capsys):
    n = 64
    x = (np.arange(10 * n + 5) * (1 - 2j)).astype(np.complex64)  # ten segments and a partial one
    x.tofile(tmp_path / "in.c64")
    rc = cli.main([str(tmp_path / "in.c64"), str(tmp_path / "out.c64"), "--n", str(n), "--chunk", "3"],
                  plan_factory=FakePlan)
    line = json.loads(capsys.readouterr().out.strip())
    assert rc == 1 and line["status"] == "partial" and line["committed_offset"] == 10 * n * 8
    assert line["chunk_segments"] == 3 and line["phases_ms"]["wall_ms"] == 2.0
    np.testing.assert_array_equal(np.fromfile(tmp_path / "out.c64", dtype=np.complex64), -x[: 10 * n])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, argv, results):
    # host-only ranks (gloo, a fake plan): no GPU is touched, also on a machine with fewer GPUs than ranks
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    results[rank] = cli.main(argv, plan_factory=FakePlan)


@pytest.mark.parametrize("frames", [False, True])
def test_two_ranks_with_gloo(tmp_path, frames):
    import torch.multiprocessing as mp
    n, hop = 64, 40
    x = (np.arange(23 * n) * (0.5 + 1j)).astype(np.complex64)
    x.tofile(tmp_path / "in.c64")
    argv = [str(tmp_path / "in.c64"), str(tmp_path / "out.c64"), "--n", str(n), "--chunk", "4"]
    if frames:
        argv += ["--frames", str(hop)]
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank, args=(2, _free_port(), argv, results), nprocs=2, join=True)
        results = dict(results)
    assert results == {0: 0, 1: 0}
    got = np.fromfile(tmp_path / "out.c64", dtype=np.complex64)
    if frames:
        F = (x.size - n) // hop + 1
        ref = -np.concatenate([x[f * hop: f * hop + n] for f in range(F)])
    else:
        ref = -x
    np.testing.assert_array_equal(got, ref)
