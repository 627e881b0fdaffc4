"""Segments over several processes (one per GPU): each rank takes a contiguous
range of the signal's segments and writes its results at their positions in
the shared output, so the positional merge of the paper's pipeline (Sec. III:
outputs named by position, merged in order) needs no merge step and the data
path has no collective.  Only barriers order the ranks: rank 0 creates the
output before anyone writes, and everyone finishes before anyone reads.
"""
import os


def segment_range(nseg: int, rank: int, world: int):
    """Contiguous [first, last) segments of rank `rank` out of `world`: the
    first nseg % world ranks take one segment more."""
    if world < 1 or not 0 <= rank < world or nseg < 0:
        raise ValueError("bad segment_range(%r, %r, %r)" % (nseg, rank, world))
    base, extra = divmod(nseg, world)
    first = rank * base + min(rank, extra)
    return first, first + base + (1 if rank < extra else 0)


def _units(plan, size):
    """Units a file of `size` bytes holds for `plan`, and the input byte range
    [start(u0), end(u1)) of units u0..u1-1: segments of a segment plan, or
    frames of a frame plan (frame f spans samples [f*hop, f*hop + n), so a
    range of frames ends at its last frame's last sample)."""
    hop = getattr(plan, "hop", None)
    if hop is not None:
        nframes = 0 if size // 8 < plan.n else (size // 8 - plan.n) // hop + 1
        return nframes, (lambda u: u * hop * 8), (lambda u: ((u - 1) * hop + plan.n) * 8)
    seg = plan.segment_bytes()[0]
    return size // seg, (lambda u: u * seg), (lambda u: u * seg)


def stream_file_sharded(plan, in_path, out_path, rank: int, world: int, barrier, chunk_segments=0,
                        direct=True):
    """This rank's share of fftseg_stream_file over the whole signal file:
    units (segments, or frames of a frame plan) segment_range(units in the
    file, rank, world), results written in place in out_path.  The last rank
    reads to the end of the file, so a partial last segment is reported
    (E_PARTIAL) or zero-padded as the plan's flags say, as in the
    single-process stream.  `barrier()` synchronises the ranks (e.g.
    torch.distributed.barrier).  Returns (status, committed input offset)."""
    size = os.path.getsize(in_path)
    nunits, start, end_of = _units(plan, size)
    first, last = segment_range(nunits, rank, world)
    is_last = rank == world - 1
    end = 0 if is_last else end_of(last)  # 0: the end of the file
    if rank == 0:  # create (or empty) the output once, before any rank writes
        with open(out_path, "wb"):
            pass
    barrier()
    if last > first or (is_last and size > end_of(nunits)):
        rc, committed = plan.stream_file(in_path, out_path, start_offset=start(first), end_offset=end,
                                         chunk_segments=chunk_segments, direct=direct, keep_output=True)
    else:
        rc, committed = 0, start(first)
    barrier()
    return rc, committed
