"""The multi-process host logic, on CPU with gloo (world size 2).

Segments are independent (paper Sec. III), so ranks take contiguous segment
ranges and write their results in place: no collective on the data path, only
barriers; the bench reduces its time with a max over ranks.  A stand-in plan
(this file's FilePlan: the same positional contract as fftseg_stream_file,
with a byte-level transformation instead of the GPU transform) exercises the
sharded file stream without a GPU.
"""
import datetime
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1407_6915_gb300.shard import segment_range, stream_file_sharded  # noqa: E402

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("nseg,world", [(0, 1), (1, 2), (7, 2), (8, 3), (16384, 8), (5, 8)])
def test_segment_ranges_partition_the_signal(nseg, world):
    ranges = [segment_range(nseg, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == nseg
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0  # contiguous, in rank order
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


class FilePlan:
    """Positional contract of fftseg_stream_file for complex output: input
    bytes [start, end) of whole n-point segments -> output at the same byte
    offsets; the 'transform' negates every sample (enough to see where each
    segment's result lands)."""

    def __init__(self, n):
        self.n = n

    def segment_bytes(self):
        return self.n * 8, self.n * 8

    def stream_file(self, in_path, out_path, start_offset=0, end_offset=0, chunk_segments=0, direct=True,
                    keep_output=False):
        assert keep_output and start_offset % (self.n * 8) == 0
        if end_offset == 0:  # the end of the file
            end_offset = os.path.getsize(in_path)
        with open(in_path, "rb") as f:
            f.seek(start_offset)
            x = np.frombuffer(f.read(end_offset - start_offset), dtype=np.complex64)
        with open(out_path, "r+b") as f:
            f.seek(start_offset)
            f.write((-x).tobytes())
        return 0, end_offset


class FrameFilePlan:
    """The same for a frame plan: frame f (samples [f*hop, f*hop + n)) goes,
    negated, to output offset f*n*8; the input range [start, end) holds the
    frames that lie wholly inside it."""

    def __init__(self, n, hop):
        self.n, self.hop = n, hop

    def stream_file(self, in_path, out_path, start_offset=0, end_offset=0, chunk_segments=0, direct=True,
                    keep_output=False):
        assert keep_output and start_offset % (self.hop * 8) == 0
        if end_offset == 0:
            end_offset = os.path.getsize(in_path)
        x = np.fromfile(in_path, dtype=np.complex64)[start_offset // 8: end_offset // 8]
        f0 = start_offset // (self.hop * 8)
        nf = 0 if x.size < self.n else (x.size - self.n) // self.hop + 1
        with open(out_path, "r+b") as f:
            for k in range(nf):
                f.seek((f0 + k) * self.n * 8)
                f.write((-x[k * self.hop: k * self.hop + self.n]).tobytes())
        return 0, (f0 + nf) * self.hop * 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, in_path, out_path, n, results, hop=None):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        plan = FilePlan(n) if hop is None else FrameFilePlan(n, hop)
        rc, committed = stream_file_sharded(plan, in_path, out_path, rank, world, dist.barrier)
        import bench
        slowest = bench.max_over_ranks(1.5 + rank)
        results[rank] = (rc, committed, slowest)
    finally:
        dist.destroy_process_group()


def test_sharded_file_stream_and_max_over_ranks_with_gloo(tmp_path):
    import torch.multiprocessing as mp
    n, nseg, world = 64, 13, 2
    x = (np.arange(nseg * n) + 1j * np.arange(nseg * n)[::-1]).astype(np.complex64)
    src, dst = tmp_path / "signal.c64", tmp_path / "out.c64"
    x.tofile(src)
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), str(src), str(dst), n, results), nprocs=world, join=True)
        results = dict(results)
    # every segment's result at its position, written by exactly its rank
    np.testing.assert_array_equal(np.fromfile(dst, dtype=np.complex64), -x)
    for r in range(world):
        rc, committed, slowest = results[r]
        assert rc == 0 and committed == segment_range(nseg, r, world)[1] * n * 8
        assert slowest == 1.5 + world - 1  # the max over ranks, on every rank


def test_sharded_frames_with_gloo(tmp_path):
    # frames split over ranks by frame ranges: each rank reads from its first
    # frame's start to its last frame's end (the overlap read by both sides)
    import torch.multiprocessing as mp
    n, hop, world = 64, 24, 2
    F = 37
    x = (np.arange((F - 1) * hop + n + 5) * (1 + 0.5j)).astype(np.complex64)  # 5 samples start no frame
    src, dst = tmp_path / "signal.c64", tmp_path / "frames.c64"
    x.tofile(src)
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), str(src), str(dst), n, results, hop), nprocs=world, join=True)
        results = dict(results)
    ref = -np.stack([x[f * hop: f * hop + n] for f in range(F)]).ravel()
    np.testing.assert_array_equal(np.fromfile(dst, dtype=np.complex64), ref)
    for r in range(world):
        rc, committed, _ = results[r]
        assert rc == 0 and committed == segment_range(F, r, world)[1] * hop * 8
