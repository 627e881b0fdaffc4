"""Transform a signal file segment by segment, results in positional order:
the paper's job (Sec. III) as one command.

    python -m paper_1407_6915_gb300 IN OUT --n 1024 [--inverse] [--norm backward]
        [--power] [--real | --frames HOP [--window rect]] [--chunk SEGMENTS]
        [--start OFFSET] [--no-direct]

One process streams the whole file through one GPU (fftseg_stream_file).
Under torchrun, every rank takes a contiguous range of segments (or frames)
on its own GPU and writes its results in place in the shared output; only
barriers cross ranks.  Prints one JSON line per rank (status, committed
offset, phase split) and exits non-zero unless every segment was written.
"""
import argparse
import json
import os
import sys

import paper_1407_6915_gb300 as fs
from paper_1407_6915_gb300.shard import stream_file_sharded

NORMS = {"none": fs.NORM_NONE, "backward": fs.NORM_BACKWARD, "ortho": fs.NORM_ORTHO}
STATUS = {fs.OK: "ok", fs.E_IO: "io_error", fs.E_PARTIAL: "partial"}


def parse(argv):
    ap = argparse.ArgumentParser(prog="python -m paper_1407_6915_gb300", description=__doc__.split("\n\n")[0])
    ap.add_argument("input", help="signal file: complex64 samples (float32 with --real forward)")
    ap.add_argument("output", help="result file, written at each segment's output offset")
    ap.add_argument("--n", type=int, required=True, help="points per segment (or frame)")
    ap.add_argument("--inverse", action="store_true", help="inverse transform (default forward)")
    ap.add_argument("--norm", choices=sorted(NORMS), default="none")
    ap.add_argument("--power", action="store_true", help="write float32 |X|^2 instead of complex64")
    kind = ap.add_mutually_exclusive_group()
    kind.add_argument("--real", action="store_true", help="real float32 samples <-> n/2 + 1 bins")
    kind.add_argument("--frames", type=int, metavar="HOP", help="overlapping frames at this hop (forward)")
    ap.add_argument("--window", choices=["hann", "rect"], default="hann", help="frame window")
    ap.add_argument("--chunk", type=int, default=0,
                    help="segments per chunk (default: about 256 MiB of input, at most the file's)")
    ap.add_argument("--start", type=int, default=0, help="input byte offset to resume from (one process)")
    ap.add_argument("--no-direct", action="store_true", help="buffered I/O instead of O_DIRECT")
    args = ap.parse_args(argv)
    if args.frames is not None and args.inverse:
        ap.error("frames are forward transforms")
    if args.power and args.inverse and args.real:
        ap.error("an inverse real plan writes samples, not a power spectrum")
    return args


def plan_spec(args, file_bytes):
    """(kind, keyword arguments, chunk) of the plan the arguments ask for."""
    direction = fs.INVERSE if args.inverse else fs.FORWARD
    out_kind = fs.OUT_POWER if args.power else fs.OUT_COMPLEX
    norm = NORMS[args.norm]
    n = args.n
    if args.frames is not None:
        unit = args.frames * 8
        units = 0 if file_bytes // 8 < n else (file_bytes // 8 - n) // args.frames + 1
    elif args.real:
        unit = n * 4 if direction == fs.FORWARD else (n // 2 + 1) * 8
        units = file_bytes // unit
    else:
        unit = n * 8
        units = file_bytes // unit
    chunk = args.chunk or max(1, (256 << 20) // unit)
    chunk = max(1, min(chunk, max(units, 1)))
    if args.frames is not None:
        window = fs.WINDOW_HANN if args.window == "hann" else fs.WINDOW_RECT
        return "frames", dict(n=n, hop=args.frames, batch=chunk, window=window, norm=norm,
                              out_kind=out_kind), chunk
    flags = fs.FLAG_REAL if args.real else 0
    return "segments", dict(n=n, batch=chunk, direction=direction, norm=norm, out_kind=out_kind,
                            flags=flags), chunk


def make_plan(kind, kw):
    return fs.FramePlan(**kw) if kind == "frames" else fs.Plan(**kw)


def main(argv=None, plan_factory=make_plan):
    args = parse(sys.argv[1:] if argv is None else argv)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.start:
        raise SystemExit("--start resumes a one-process run; ranks take their own ranges")
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    try:
        kind, kw, chunk = plan_spec(args, os.path.getsize(args.input))
        plan = plan_factory(kind, kw)
        direct = not args.no_direct
        if world > 1:
            rc, committed = stream_file_sharded(plan, args.input, args.output, rank, world, dist.barrier,
                                                chunk_segments=chunk, direct=direct)
        else:
            rc, committed = plan.stream_file(args.input, args.output, start_offset=args.start,
                                             chunk_segments=chunk, direct=direct)
        line = {"rank": rank, "world": world, "status": STATUS.get(rc, rc), "committed_offset": committed,
                "plan": kind, "n": args.n, "chunk_segments": chunk}
        phases = getattr(plan, "stream_phases", None)
        if phases is not None:
            line["phases_ms"] = {k: round(v, 3) for k, v in phases().items()}
        print(json.dumps(line), flush=True)
        return 0 if rc == fs.OK else 1
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
