"""Benchmark of the segmented FFT on one or more GB300s (one process per GPU).

Default workload: a resident 2^30-sample complex64 signal (8 GiB) cut into
16384 segments of 65536 points; one step = forward transform (no scaling)
then inverse transform (1/n) of every segment, i.e. two batched transforms.
The signal is 32 off-bin complex tones (amplitudes log-uniform 1e-3..1) plus
complex Gaussian noise (sigma 0.1), seed 1, synthesised on the host.

Metric: GFLOP/s by the 5*n*log2(n) convention per transformed segment,
whole job (all GPUs).  Every buffer is 8 GiB, far larger than L2, so no L2
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the FP64 CPU oracle (the reference arm of this
build: the paper has no code) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 1 << 16
SEGMENTS = 16384
SEED = 1
METRIC = "segment-FFT GFLOP/s and % HBM roofline, FP32 vs TC split; serve p50/p99 ms"
UNIT = "GFLOP/s"
WORKLOAD = "resident 8 GiB complex64 signal, 16384 segments x 65536 points, forward then inverse (1/n)"


def workload_name(segments, n=N):
    if segments == SEGMENTS and n == N:
        return WORKLOAD
    return ("resident %g GiB complex64 signal, %d segments x %d points, forward then inverse (1/n)"
            % (segments * n * 8 / 2**30, segments, n))


def kernel_name(path, n, flags):
    """The kernel a complex FP32 plan runs (for the roofline record)."""
    import paper_1407_6915_gb300 as fs
    if path == "cluster":
        return "k_cluster: one thread-block cluster per segment, all-to-all over distributed shared memory"
    if path != "four-step":
        return path
    if flags & (fs.FLAG_FOURSTEP_PRODUCER | fs.FLAG_FOURSTEP_TILES):
        return "k_fourstep: persistent four-step over CTA tiles, intermediate kept in L2"
    if n == 1 << 16 and flags & fs.FLAG_FOURSTEP_WARP_LINES:
        return "k_fourstep_hw: persistent four-step, warp-local lines, intermediate kept in L2"
    if (1 << 16) <= n <= (1 << 20):
        return "k_fourstep_wl: persistent four-step, lane-local lines of 32 points per lane, intermediate kept in L2"
    if (1 << 21) <= n <= (1 << 24) and not flags & fs.FLAG_FOURSTEP_WARP_LINES:
        return ("k_outer + k_fourstep_wl: outer radix-R pass, then the lane-line kernel over units of 32 "
                "interleaved 2^16-point transforms (two HBM passes, two launches per workspace chunk)")
    return "k_fourstep: persistent four-step over CTA tiles, intermediate kept in L2"


def vendor_context(n, segments):
    """Context only: the vendor FFT library (through torch.fft) on the same GPU and
    shape, forward, out of place.  It is not part of fftseg and not a baseline."""
    import torch
    x = torch.zeros(segments, n, dtype=torch.complex64, device="cuda")
    for _ in range(3):
        y = torch.fft.fft(x, dim=-1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        y = torch.fft.fft(x, dim=-1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 5
    del x, y
    torch.cuda.empty_cache()
    return {"what": "vendor FFT library via torch.fft on the same GPU and shape (context only)",
            "n": n, "segments": segments, "ms_per_transform": round(ms, 4),
            "gbs_16B_per_point": round(16.0 * n * segments / (ms / 1e3) / 1e9, 1)}


def flops_per_transform(n, segments):
    return 5.0 * n * math.log2(n) * segments


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        rows = []
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"unavailable": "nvidia-smi gave no samples"}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(seconds_target=12.0):
    """The FP64 oracle as it stands, timed on this host's cores on a sample of
    the workload: with every core, and with one core on a smaller sample."""
    import numpy as np
    import oracle
    import siggen
    cores = os.cpu_count() or 1

    def timed(seg, threads, target):
        x = siggen.tones(SEED, seg * N).reshape(seg, N)
        t0 = time.perf_counter()
        X = oracle.fft(x, oracle.FORWARD, oracle.NORM_NONE, nthreads=threads)
        oracle.fft(X.astype(np.complex64), oracle.INVERSE, oracle.NORM_BACKWARD, nthreads=threads)
        dt = time.perf_counter() - t0
        reps = min(64, max(1, int(target / max(dt, 1e-3))))
        t0 = time.perf_counter()
        for _ in range(reps):
            X = oracle.fft(x, oracle.FORWARD, oracle.NORM_NONE, nthreads=threads)
            oracle.fft(X.astype(np.complex64), oracle.INVERSE, oracle.NORM_BACKWARD, nthreads=threads)
        dt = time.perf_counter() - t0
        return 2 * flops_per_transform(N, seg * reps) / dt / 1e9, reps, dt

    seg = max(cores, 8)
    value, reps, dt = timed(seg, cores, seconds_target)
    v1, reps1, dt1 = timed(2, 1, seconds_target / 3)
    return {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of the 16384 segments, forward+inverse, %d repetitions, %.1f s wall"
                      % (seg, reps, dt),
            "single_core": {"value": round(v1, 3), "unit": UNIT, "cores": 1,
                            "sample": "2 segments, forward+inverse, %d repetitions, %.1f s wall" % (reps1, dt1)}}


def c1_bench(peak, pairs=16):
    """C1, the paper's record size: 4096 segments x 1024 points (32 MiB)
    forward, uniform input (seed 0), timed over `pairs` rotating input/output
    buffer pairs (together larger than 4x L2), so every launch reads and
    writes HBM.  Kernel time from CUDA events; the host time of the
    fftseg_exec call (launch only, no synchronisation) beside it."""
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen
    n, B = 1024, 4096
    x0 = torch.from_numpy(siggen.uniform(0, B * n).reshape(B, n)).cuda()
    ins = [x0.clone() for _ in range(pairs)]
    outs = [torch.empty_like(x0) for _ in range(pairs)]
    plan = fs.Plan(n, B, fs.FORWARD)
    stream = torch.cuda.current_stream()
    for i in range(pairs):
        plan.exec_ptr(ins[i].data_ptr(), outs[i].data_ptr(), B, stream)
    torch.cuda.synchronize()
    plan.check()
    reps = 8 * pairs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    host = 0.0
    e0.record(stream)
    for k in range(reps):
        i = k % pairs
        t0 = time.perf_counter()
        plan.exec_ptr(ins[i].data_ptr(), outs[i].data_ptr(), B, stream)
        host += time.perf_counter() - t0
    e1.record(stream)
    torch.cuda.synchronize()
    plan.check()
    ms = e0.elapsed_time(e1) / reps
    gbs = 16.0 * n * B / (ms / 1e3) / 1e9
    ok = bool(torch.equal(outs[0], outs[pairs - 1]))  # same input, same bits
    return {"workload": "4096 segments x 1024 points complex64, forward, uniform[-1,1) seed 0",
            "path": plan.info()["path"], "ms": round(ms, 5),
            "gflops": round(flops_per_transform(n, B) / (ms / 1e3) / 1e9, 1),
            "gbs_algorithmic": round(gbs, 1), "hbm_frac": round(gbs / peak, 4),
            "api_us_per_call": round(host / reps * 1e6, 2),
            "l2": "%d rotating buffer pairs, %d MiB in all (L2 is about 126 MiB)" % (pairs, pairs * 64),
            "outputs_equal_across_buffers": ok}


# the translation unit that instantiates each path's kernel
KERNEL_TU = {"four-step": ("k_fourstep.cu", "k_fourstep_wl.cu"), "cluster": ("k_cluster.cu",),
             "block": ("k_lines.cu",)}


def kernel_rev(path="four-step"):
    """Hash of the device code of a path's kernel (its translation units and
    every header they include, transitively): a DRAM-traffic figure only
    applies to the kernel sources it was taken on."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1407_6915_gb300", "csrc")
    seen, todo = set(), list(KERNEL_TU.get(path, ()))
    while todo:
        name = todo.pop()
        if name in seen or not os.path.exists(os.path.join(csrc, name)):
            continue
        seen.add(name)
        with open(os.path.join(csrc, name)) as f:
            todo += re.findall(r'^#include "([^"]+)"', f.read(), re.M)
    h = hashlib.sha1()
    for name in sorted(seen):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:12]


def measured_traffic(key):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from the committed ncu
    summary (profiles/dram_traffic.txt: `<path>:<n> <bytes per launch> <kernel rev>`),
    or None when it was taken on other kernel sources."""
    try:
        rev = kernel_rev(key.split(":")[0])
        with open(os.path.join(ROOT, "profiles", "dram_traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 3 and parts[0] == key and parts[2] == rev:
                    return float(parts[1])
    except OSError:
        pass
    return None


def link_peaks(dev, gib=1, reps=3):
    """Measured pinned host<->device copy rates (GB/s): each direction alone
    and both at once on two streams (each way), best of `reps`."""
    import torch
    n = gib << 27
    h1 = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    h2 = torch.empty(n, dtype=torch.complex64, pin_memory=True)
    h1.zero_()
    d1 = torch.empty(n, dtype=torch.complex64, device=dev)
    d2 = torch.zeros(n, dtype=torch.complex64, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    nb = n * 8
    best = {"h2d": 0.0, "d2h": 0.0, "concurrent_each_way": 0.0}
    for _ in range(reps):
        for key, fn in (("h2d", lambda: d1.copy_(h1, non_blocking=True)),
                        ("d2h", lambda: h2.copy_(d2, non_blocking=True))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best[key] = max(best[key], nb / (time.perf_counter() - t0) / 1e9)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s1):
            d1.copy_(h1, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        best["concurrent_each_way"] = max(best["concurrent_each_way"], nb / (time.perf_counter() - t0) / 1e9)
    del h1, h2, d1, d2
    return {k: round(v, 1) for k, v in best.items()}


def stream_bench(link, h_signal=None):
    """C3, the out-of-core stream at its configured size: 128 GiB of complex64
    signal in 2^20-point segments through fftseg_stream with |X|^2 output, in
    chunks of 64 segments (512 MiB).

    The tones + noise generator (seed 2) runs at about 1 GB/s on the box's
    host cores, two orders of magnitude below the host link, so a stream fed
    by it measures the generator.  The full-size run therefore reads a
    host-resident source: 2 GiB of the seed-2 signal generated once into
    pinned memory and read cyclically by the reader callback (several copy
    threads), as a signal already in host memory would be.  The generator's
    own rate and a generator-fed stream of 2 GiB are reported beside it; a
    host-resident batch through fftseg_exec_host shows the same pipeline
    without callbacks."""
    import ctypes
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen
    n = 1 << 20
    chunk = 64
    nseg = 16384  # 128 GiB
    pool_segs = 256  # 2 GiB
    total = nseg * n * 8
    cores = os.cpu_count() or 1
    plan = fs.Plan(n, chunk, fs.FORWARD, out_kind=fs.OUT_POWER)
    pool = torch.empty(pool_segs * n, dtype=torch.complex64, pin_memory=True)
    t0 = time.perf_counter()
    siggen.fill_pointer(siggen.KIND_TONES, 2, 0, pool_segs * n, pool.data_ptr(), nthreads=cores)
    gen_s = time.perf_counter() - t0
    out = {"n": n, "segments": nseg, "chunk_segments": chunk, "input_bytes": total,
           "generator": {"what": "tones + noise, seed 2, into pinned memory", "bytes": pool_segs * n * 8,
                         "s": round(gen_s, 3), "gbs": round(pool_segs * n * 8 / gen_s / 1e9, 3), "threads": cores}}
    # full size, host-resident source lent in place (fftseg_stream_view): each
    # chunk goes to the GPU straight from the pool
    snk = siggen.sink(None)  # counts the bytes, keeps nothing

    def full_run(lend):
        src = siggen.pool_source(pool.data_ptr(), pool_segs * n * 8, total, nthreads=min(cores, 16))
        go = plan.stream_view if lend else plan.stream
        fn = siggen.view_fn_ptr() if lend else siggen.read_fn_ptr()
        go(fn, ctypes.addressof(src), siggen.write_fn_ptr(), ctypes.addressof(snk), 1 << 32, 0, chunk)  # warm-up
        t0 = time.perf_counter()
        rc, committed = go(fn, ctypes.addressof(src), siggen.write_fn_ptr(), ctypes.addressof(snk), total, 0, chunk)
        wall = time.perf_counter() - t0
        ph = plan.stream_phases()
        h2d_gbs, d2h_gbs = total / wall / 1e9, total / 2 / wall / 1e9
        return {"status": rc, "committed_bytes": int(committed), "wall_s": round(wall, 3),
                "gflops": round(flops_per_transform(n, nseg) / wall / 1e9, 1),
                "h2d_gbs": round(h2d_gbs, 2), "d2h_gbs": round(d2h_gbs, 2),
                "link_frac": round(max(h2d_gbs / link["h2d"], d2h_gbs / link["d2h"]), 4),
                "phases_ms": {k: round(v, 1) for k, v in ph.items()},
                "bound": "reader" if ph["read_ms"] > 0.8 * ph["wall_ms"] else "pipeline"}

    out["source"] = "2 GiB pinned pool of the seed-2 signal, read cyclically"
    out.update(full_run(True))
    out["call"] = "fftseg_stream_view (the pool lent in place)"
    out["copying_reader"] = dict(full_run(False), call="fftseg_stream, the reader copying from the pool "
                                 "(%d threads)" % min(cores, 16))
    # a generator-fed sample (2 GiB)
    gseg = 256
    gsrc = siggen.source(siggen.KIND_TONES, 2, gseg * n * 8)
    t0 = time.perf_counter()
    grc, _ = plan.stream(siggen.read_fn_ptr(), ctypes.addressof(gsrc), siggen.write_fn_ptr(),
                         ctypes.addressof(snk), gseg * n * 8, 0, chunk)
    gwall = time.perf_counter() - t0
    gph = plan.stream_phases()
    out["generator_fed_sample"] = {"segments": gseg, "status": grc, "wall_s": round(gwall, 3),
                                   "h2d_gbs": round(gseg * n * 8 / gwall / 1e9, 2),
                                   "bound": "generator" if gph["read_ms"] > 0.8 * gph["wall_ms"] else "pipeline",
                                   "full_128gib_s_at_this_rate": round(gwall * nseg / gseg, 1)}
    plan.destroy()
    del pool
    if h_signal is not None:
        hn = min(h_signal.numel() // n, 512)
        hp = fs.Plan(n, chunk, fs.FORWARD, out_kind=fs.OUT_POWER)
        h_pow = torch.empty(hn * n, dtype=torch.float32, pin_memory=True)
        for _ in range(3):  # staging, first touch, link ramp-up
            fs.exec_host([hp], h_signal.data_ptr(), h_pow.data_ptr(), hn, chunk)
        t0 = time.perf_counter()
        fs.exec_host([hp], h_signal.data_ptr(), h_pow.data_ptr(), hn, chunk)
        dt = time.perf_counter() - t0
        in_gbs = hn * n * 8 / dt / 1e9
        out["host_resident"] = {"call": "fftseg_exec_host, |X|^2 out", "segments": hn,
                                "input_bytes": hn * n * 8, "s": round(dt, 4),
                                "gflops": round(flops_per_transform(n, hn) / dt / 1e9, 1),
                                "h2d_gbs": round(in_gbs, 1), "d2h_gbs": round(in_gbs / 2, 1),
                                "link_frac": round(max(in_gbs / link["h2d"], in_gbs / 2 / link["d2h"]), 4)}
        hp.destroy()
        del h_pow
    return out


def extra(fn, *args):
    """One extra measurement for the JSON line.  A failure is recorded in its
    place, with the exception, and does not take the main line with it."""
    import torch
    try:
        return fn(*args)
    except Exception as e:  # noqa: BLE001 - reported in the line, not hidden
        if torch.cuda.is_available():
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        return {"error": "%s: %s" % (type(e).__name__, e)}


def tc_split(peak):
    """FP32 versus tensor-core (split hi+lo FP16 / BF16) on the same GPU: time of one
    4 GiB batch (uniform input) and the round-trip error of each precision (forward,
    then the inverse of the same precision with 1/n, against the input; parity with
    the FP64 oracle is the tests' job), for both input families (uniform seed 3,
    tones + noise seed 4: one 2^29-sample signal each, cut into segments of every
    size)."""
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen
    out = []
    count = 1 << 29
    fam = {}
    for name, kind, seed in (("uniform", siggen.KIND_UNIFORM, 3), ("tones", siggen.KIND_TONES, 4)):
        h = torch.empty(count, dtype=torch.complex64, pin_memory=True)
        siggen.fill_pointer(kind, seed, 0, count, h.data_ptr())
        fam[name] = (h, h.cuda())
    for log_n in (12, 16, 20, 24):
        n = 1 << log_n
        B = count // n
        y = torch.empty(B, n, dtype=torch.complex64, device="cuda")
        z = torch.empty(B, n, dtype=torch.complex64, device="cuda")
        row = {"n": n, "segments": B}
        for name, prec in (("fp32", fs.PREC_FP32), ("tc_fp16", fs.PREC_TC_FP16), ("tc_bf16", fs.PREC_TC_BF16)):
            plan = fs.Plan(n, B, fs.FORWARD, precision=prec)
            inv = fs.Plan(n, B, fs.INVERSE, fs.NORM_BACKWARD, precision=prec)
            errs = {}
            for f, (_, d) in fam.items():
                plan.exec(d.view(B, n), out=y)
                inv.exec(y, out=z)
                torch.cuda.synchronize()
                inv.check()
                errs[f] = float(torch.linalg.vector_norm(z.view(-1) - d) / torch.linalg.vector_norm(d))
            del inv
            x = fam["uniform"][1].view(B, n)
            for _ in range(3):
                plan.exec(x, out=y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            reps = 5
            for _ in range(reps):
                plan.exec(x, out=y)
            e1.record()
            torch.cuda.synchronize()
            plan.check()
            ms = e0.elapsed_time(e1) / reps
            gbs = 16.0 * n * B / (ms / 1e3) / 1e9
            row[name] = {"ms": round(ms, 4), "gflops": round(flops_per_transform(n, B) / (ms / 1e3) / 1e9, 1),
                         "hbm_frac": round(gbs / peak, 4), "round_trip_rel_l2_uniform": errs["uniform"],
                         "round_trip_rel_l2_tones": errs["tones"], "path": plan.info()["path"]}
            del plan
        out.append(row)
        del y, z
        torch.cuda.empty_cache()
    del fam
    torch.cuda.empty_cache()
    return {"batch_bytes": 1 << 32, "timed_input": "uniform[-1,1), seed 3",
            "round_trip": "forward then inverse (1/n) in the same precision, rel-L2 against the input "
                          "over every segment (parity with the oracle: tests/test_tc.py)",
            "round_trip_inputs": "uniform seed 3; 32 tones + noise seed 4",
            "bound_fp32_per_transform": "2e-6*log2(n)", "bound_tc_per_transform": 1e-4,
            "role": "accuracy option: the tensor-core forms meet 1e-4 but are slower than FP32 at every size "
                    "(their operands make a shared-memory round trip per stage on a path whose shared-memory "
                    "pipe is already the limit)",
            "sizes": out}


def real_bench(peak, sizes=None):
    """Real-signal segments (FLAG_REAL): 4 GiB of float32 samples cut into
    n-point segments (n = 1024, the paper's record size, and 65536), to the
    n/2 + 1 bins of each segment (forward) and back (inverse, timed on the
    forward's bins).  Algorithmic bytes per segment: 4n and 8 (n/2 + 1).
    `sizes`: other (n, segments) pairs (profiler captures)."""
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen
    rows = []
    for n, B in sizes or [(n, (1 << 30) // n) for n in (1024, 65536)]:
        h = torch.empty(B * n // 2, dtype=torch.complex64, pin_memory=True)
        siggen.fill_pointer(siggen.KIND_TONES, 6, 0, B * n // 2, h.data_ptr())
        x = h.cuda().view(torch.float32).view(B, n)
        plan = fs.Plan(n, B, fs.FORWARD, flags=fs.FLAG_REAL)
        y = torch.empty(B, n // 2 + 1, dtype=torch.complex64, device="cuda")
        for _ in range(3):
            plan.exec(x, out=y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            plan.exec(x, out=y)
        e1.record()
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1) / 5
        algo = B * (4.0 * n + 8.0 * (n // 2 + 1))
        # round trip through the inverse real plan (1/n) against the samples,
        # and the inverse plan's own time (the same bytes the other way)
        inv = fs.Plan(n, B, fs.INVERSE, fs.NORM_BACKWARD, flags=fs.FLAG_REAL)
        xr = inv.exec(y)
        for _ in range(2):
            inv.exec(y, out=xr)
        e0.record()
        for _ in range(5):
            inv.exec(y, out=xr)
        e1.record()
        torch.cuda.synchronize()
        inv.check()
        inv_ms = e0.elapsed_time(e1) / 5
        xr = inv.exec(y)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(xr - x) / torch.linalg.vector_norm(x))
        rows.append({"n": n, "segments": B, "ms": round(ms, 4),
                     "gflops_real_convention": round(2.5 * n * math.log2(n) * B / (ms / 1e3) / 1e9, 1),
                     "gbs_algorithmic": round(algo / (ms / 1e3) / 1e9, 1),
                     "hbm_frac": round(algo / (ms / 1e3) / 1e9 / peak, 4),
                     "launches_per_exec": plan.info()["launches_per_exec"],
                     "inverse_ms": round(inv_ms, 4),
                     "inverse_hbm_frac": round(algo / (inv_ms / 1e3) / 1e9 / peak, 4),
                     "inverse_launches_per_exec": inv.info()["launches_per_exec"],
                     "round_trip_rel_l2": err})
        del x, y, h, plan, inv, xr
        torch.cuda.empty_cache()
    return {"what": "real float32 segments -> n/2 + 1 complex bins (forward), tones + noise seed 6",
            "flops_convention": "2.5 n log2 n per real segment", "sizes": rows}


def frames_bench(peak):
    """Overlapping segments (FramePlan): a 2^29-sample complex64 signal (4 GiB),
    periodic Hann window, hop n/2, at n = 1024 and 65536.  Algorithmic bytes per
    frame: 8 hop read (each sample once, overlaps re-read from L2) + 8 n written."""
    import numpy as np
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen
    count = 1 << 29
    h = torch.empty(count, dtype=torch.complex64, pin_memory=True)
    siggen.fill_pointer(siggen.KIND_TONES, 7, 0, count, h.data_ptr())
    x = h.cuda()
    rows = []
    for n in (1024, 65536):
        hop = n // 2
        plan = fs.FramePlan(n, hop, (count - n) // hop + 1, fs.WINDOW_HANN)
        F = plan.frames_in(count)
        y = torch.empty(F, n, dtype=torch.complex64, device="cuda")
        for _ in range(3):
            plan.exec(x, out=y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            plan.exec(x, out=y)
        e1.record()
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1) / 5
        algo = F * (8.0 * hop + 8.0 * n)
        # the first two frames against the library's n-point segment plan on
        # the same frames windowed here (periodic Hann, evaluated in double,
        # rounded once); parity with the oracle is the tests' job
        w = torch.from_numpy((0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / n)).astype(np.float32)).cuda()
        fr = torch.stack([x[f * hop: f * hop + n] for f in range(2)]) * w
        ys = fs.Plan(n, 2, fs.FORWARD).exec(fr.contiguous())
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(y[:2] - ys) / torch.linalg.vector_norm(ys))
        rows.append({"n": n, "hop": hop, "frames": F, "ms": round(ms, 4),
                     "gflops": round(5.0 * n * math.log2(n) * F / (ms / 1e3) / 1e9, 1),
                     "gbs_algorithmic": round(algo / (ms / 1e3) / 1e9, 1),
                     "hbm_frac": round(algo / (ms / 1e3) / 1e9 / peak, 4),
                     "rel_l2_vs_segment_plan_first_2_frames": err})
        del y, plan
        torch.cuda.empty_cache()
    del x, h
    torch.cuda.empty_cache()
    return {"what": "short-time FFT: Hann-windowed frames of a tones + noise signal (seed 7), hop n/2",
            "sizes": rows}


def file_bench():
    """File-backed streaming (fftseg_stream_file): a tones + noise signal file
    (seed 8; up to 2 GiB, a quarter of the free space at most) in the temporary
    directory, 2^20-point segments to |X|^2, O_DIRECT where the file system
    allows it.  The phase split is the analog of the paper's I/O versus FFT
    breakdown (Sec. IV, Figs. 4-5)."""
    import shutil
    import tempfile
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen
    tmp = tempfile.gettempdir()
    n = 1 << 20
    seg = n * 8
    segs = int(min(2 << 30, shutil.disk_usage(tmp).free // 4) // seg)
    if segs < 8:
        return {"unavailable": "less than 8 segments of free space in %s" % tmp}
    fstype = "unknown"
    try:
        best = ""
        with open("/proc/mounts") as f:
            for line in f:
                parts = line.split()
                if len(parts) > 2 and tmp.startswith(parts[1]) and len(parts[1]) > len(best):
                    best, fstype = parts[1], parts[2]
    except OSError:
        pass
    src = os.path.join(tmp, "fftseg_bench_signal.c64")
    dst = os.path.join(tmp, "fftseg_bench_power.f32")
    try:
        h = torch.empty(segs * n, dtype=torch.complex64, pin_memory=True)
        siggen.fill_pointer(siggen.KIND_TONES, 8, 0, segs * n, h.data_ptr())
        h.numpy().tofile(src)
        del h
        plan = fs.Plan(n, 64, fs.FORWARD, out_kind=fs.OUT_POWER)
        t0 = time.perf_counter()
        rc, committed = plan.stream_file(src, dst, chunk_segments=64, direct=True)
        wall = time.perf_counter() - t0
        ph = plan.stream_phases()
        io = ph["read_ms"] + ph["write_ms"]
        return {"file_bytes": segs * seg, "segments": segs, "n": n, "out": "float32 |X|^2", "status": rc,
                "file_system": fstype, "dir": tmp, "s": round(wall, 3),
                "in_gbs": round(segs * seg / wall / 1e9, 2),
                "phases_ms": {k: round(v, 1) for k, v in ph.items()},
                "share_of_wall": {"file_read": round(ph["read_ms"] / ph["wall_ms"], 3),
                                  "file_write": round(ph["write_ms"] / ph["wall_ms"], 3),
                                  "fft": round(ph["fft_ms"] / ph["wall_ms"], 3),
                                  "h2d_d2h": round((ph["h2d_ms"] + ph["d2h_ms"]) / ph["wall_ms"], 3)},
                "io_share": round(io / (io + ph["fft_ms"]), 3)}
    finally:
        for f in (src, dst):
            try:
                os.remove(f)
            except OSError:
                pass


def bluestein_bench(peak):
    """Lengths that are not powers of two, 2^29 complex64 samples (4 GiB)
    each, forward: n = 1000 and 3000 on the mixed-radix path (the default for
    lengths 2^a 3^b 5^c 7^d <= 4096), n = 1000 through Bluestein (M = 2048)
    for comparison, and the primes 10007 and 40009 through Bluestein
    (M = 32768 and 131072).  Algorithmic bytes: 16 per point, as for every
    length."""
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen
    rows = []
    for n, flags in ((1000, 0), (3000, 0), (1000, fs.FLAG_BLUESTEIN), (10007, 0), (40009, 0)):
        B = (1 << 29) // n
        x = torch.from_numpy(siggen.uniform(9, B * n)).cuda().view(B, n)
        plan = fs.Plan(n, B, fs.FORWARD, flags=flags)
        y = torch.empty_like(x)
        for _ in range(2):
            plan.exec(x, out=y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            plan.exec(x, out=y)
        e1.record()
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1) / 3
        # round trip through the inverse plan (1/n) against the input; parity
        # with the oracle's direct DFT is the tests' job
        inv = fs.Plan(n, B, fs.INVERSE, fs.NORM_BACKWARD, flags=flags)
        z = inv.exec(y)
        torch.cuda.synchronize()
        inv.check()
        err = float(torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x))
        del inv, z
        algo = 16.0 * n * B
        info = plan.info()
        rows.append({"n": n, "path": info["path"], "M": int(info["n1"]) if info["path"] == "bluestein" else None,
                     "segments": B, "ms": round(ms, 4),
                     "gflops": round(5.0 * n * math.log2(n) * B / (ms / 1e3) / 1e9, 1),
                     "gbs_algorithmic": round(algo / (ms / 1e3) / 1e9, 1),
                     "hbm_frac": round(algo / (ms / 1e3) / 1e9 / peak, 4),
                     "launches_per_exec": plan.info()["launches_per_exec"], "round_trip_rel_l2": err})
        del x, y, plan
        torch.cuda.empty_cache()
    return {"what": "lengths that are not powers of two, uniform[-1,1) seed 9, forward", "sizes": rows}


def tune_table():
    """The autotuner's choice per length (FP32, complex output, a 256 MiB batch)
    beside the library's default schedule."""
    import torch
    import paper_1407_6915_gb300 as fs
    rows = []
    x = torch.zeros(1 << 25, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    for log_n in range(13, 25):
        n = 1 << log_n
        B = max(1, (1 << 25) // n)
        flags, ms = fs.autotune(n, B)
        plan = fs.Plan(n, B, fs.FORWARD)
        default = plan.info()["path"]
        # the default schedule, timed the way the tuner times its candidates
        for _ in range(3):
            plan.exec(x.view(B, n), out=y.view(B, n))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            plan.exec(x.view(B, n), out=y.view(B, n))
        e1.record()
        torch.cuda.synchronize()
        plan.check()
        dms = e0.elapsed_time(e1) / 10
        plan.destroy()
        plan = fs.Plan(n, 1, fs.FORWARD, flags=flags)
        rows.append({"n": n, "tuned_flags": hex(flags), "tuned_path": plan.info()["path"],
                     "tuned_ms_per_256mib": round(ms, 4), "default_path": default,
                     "default_ms_per_256mib": round(dms, 4),
                     "default_over_tuned": round(dms / ms, 3) if ms > 0 else None})
        plan.destroy()
    return rows


def serve_bench(peak, njobs=600, seed=5):
    """Poisson arrivals at 0.3/0.7/0.95 of the measured saturated throughput through the
    continuous-batching server (32 GB budget); p50/p99 submit-to-completion latency."""
    import numpy as np
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen
    rng = np.random.default_rng(seed)
    cap = 1 << 28  # samples per job at most (2 GiB of input), so a bounded pool holds the jobs in flight
    jobs = []
    for _ in range(njobs):
        e = int(rng.integers(8, 23))
        n = 1 << e
        nseg = max(1, int(2.0 ** rng.uniform(0, 12)))
        nseg = max(1, min(nseg, cap // n))
        direction = fs.FORWARD if rng.random() < 0.5 else fs.INVERSE
        norm = fs.NORM_BACKWARD if direction == fs.INVERSE else fs.NORM_NONE
        jobs.append((n, nseg, direction, norm))
    x = torch.empty(cap, dtype=torch.complex64, device="cuda")
    h = torch.empty(cap, dtype=torch.complex64, pin_memory=True)
    siggen.fill_pointer(siggen.KIND_UNIFORM, seed, 0, cap, h.data_ptr())
    x.copy_(h)
    ring_elems = 34 << 27  # 34 GiB of complex64 outputs, used round-robin
    ring = torch.empty(ring_elems, dtype=torch.complex64, device="cuda")
    budget = 32 << 30

    # one server for every run, as in service: its resident plans (one per
    # length, direction, norm and lane) are made during the warm-up run
    srv = fs.Server(hbm_budget_bytes=budget, max_inflight_jobs=256)

    def run(arrivals, subset=None):
        # submit at the arrival times from this thread; each job's latency is
        # the server's own submit-to-completion time, read once all are in
        launches0 = srv.stats()["launches"]
        lat = [None] * len(jobs)
        pos = 0
        ids = []
        t0 = time.perf_counter()
        for i, (n, nseg, direction, norm) in enumerate(jobs):
            if subset is not None and i not in subset:
                continue
            if arrivals is not None:
                wait = t0 + arrivals[i] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
            sz = n * nseg
            if pos + sz > ring_elems:
                pos = 0
            out_ptr = ring.data_ptr() + 8 * pos
            pos += sz
            ids.append((i, srv.submit(x.data_ptr(), out_ptr, n, nseg, direction, norm)))
        for i, jid in ids:
            done, st, secs = srv.poll_latency(jid, timeout_us=120_000_000)
            lat[i] = secs if (done and st == fs.OK) else None
        wall = time.perf_counter() - t0
        stats = srv.stats()
        stats["launches"] -= launches0
        return lat, wall, stats

    samples = sum(n * nseg for n, nseg, _, _ in jobs)
    flops = sum(5.0 * n * math.log2(n) * nseg for n, nseg, _, _ in jobs)
    run(None)  # warm-up: plans, graphs, first-touch
    _, wall_sat, _ = run(None)
    sat_rate = samples / wall_sat  # samples/s, everything queued at once
    loads = []
    for load in (0.3, 0.7, 0.95):
        lam = load * sat_rate / (samples / len(jobs))  # jobs/s
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(jobs)))
        lat, wall, stats = run(arrivals)
        ok = [v for v in lat if v is not None]
        loads.append({"offered_load": load, "offered_jobs_per_s": round(lam, 1),
                      "p50_ms": round(1e3 * float(np.percentile(ok, 50)), 3),
                      "p99_ms": round(1e3 * float(np.percentile(ok, 99)), 3),
                      "throughput_gflops": round(flops / wall / 1e9, 1),
                      "hbm_frac": round(16.0 * samples / wall / 1e9 / peak, 4),
                      "jobs_ok": len(ok), "launches": stats["launches"],
                      "peak_admitted_bytes": stats["peak_admitted_bytes"]})
    # where the saturated time goes: each length class's jobs run alone (queued at once)
    classes = (("n <= 4096 (ragged kernel)", 1 << 8, 1 << 12), ("2^13..2^16", 1 << 13, 1 << 16),
               ("2^17..2^20", 1 << 17, 1 << 20), ("2^21..2^22", 1 << 21, 1 << 22))
    per_class = []
    for name, lo, hi in classes:
        sub = {i for i, (n, _, _, _) in enumerate(jobs) if lo <= n <= hi}
        if not sub:
            continue
        cs = sum(jobs[i][0] * jobs[i][1] for i in sub)
        _, wall_c, _ = run(None, sub)
        per_class.append({"class": name, "jobs": len(sub), "sample_share": round(cs / samples, 4),
                          "alone_s": round(wall_c, 4), "share_of_saturated_time": round(wall_c / wall_sat, 4),
                          "hbm_frac_alone": round(16.0 * cs / wall_c / 1e9 / peak, 4)})
    srv.destroy()
    del ring, x
    torch.cuda.empty_cache()
    return {"jobs": njobs, "budget_bytes": budget, "per_length_class": per_class,
            "server": "one server for all runs; its resident plans made in the warm-up run",
            "latency": "submit-to-completion by the server's host clock (fftsrv_poll_latency); jobs submitted "
                       "from one thread at their arrival times",
            "job_recipe": "n = 2^e, e uniform in 8..22; segments 2^U(0,12) capped at 2^28 samples per job; "
                          "50/50 forward / inverse(1/n); uniform[-1,1) input",
            "saturated_gflops": round(flops / wall_sat / 1e9, 1),
            "saturated_hbm_frac": round(16.0 * samples / wall_sat / 1e9 / peak, 4), "loads": loads}


def max_over_ranks(value, device=None):
    """The largest of every rank's value, on every rank (the job's time is its
    slowest rank's); the value itself in a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    import siggen
    cores = os.cpu_count() or 1
    seg = 2 * cores  # a bounded sample per step on every core: a few seconds of CPU work
    x = siggen.tones(SEED, seg * N).reshape(seg, N)
    for _ in range(args.warmup):
        X = oracle.fft(x, oracle.FORWARD, oracle.NORM_NONE, nthreads=cores)
        oracle.fft(X.astype(np.complex64), oracle.INVERSE, oracle.NORM_BACKWARD, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        X = oracle.fft(x, oracle.FORWARD, oracle.NORM_NONE, nthreads=cores)
        oracle.fft(X.astype(np.complex64), oracle.INVERSE, oracle.NORM_BACKWARD, nthreads=cores)
    dt = time.perf_counter() - t0
    value = 2 * flops_per_transform(N, seg) * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "segments": SEGMENTS,
                       "sample_per_step": seg, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d segments forward+inverse per step" % seg},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_1407_6915_gb300 as fs
    import siggen

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    n = args.n
    S = args.segments if args.segments else (SEGMENTS if n == n else max(1, (1 << 30) // n))
    pflags = args.flags

    # ---- inputs: synthesised on the host straight into pinned memory
    h_in = torch.empty(S * n, dtype=torch.complex64, pin_memory=True)
    siggen.fill_pointer(siggen.KIND_TONES, SEED, 0, S * n, h_in.data_ptr())
    h_out = torch.empty(S * n, dtype=torch.complex64, pin_memory=True)
    x = h_in.to(dev).view(S, n)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    fwd = fs.Plan(n, S, fs.FORWARD, fs.NORM_NONE, flags=pflags)
    inv = fs.Plan(n, S, fs.INVERSE, fs.NORM_BACKWARD, flags=pflags)

    def step():
        fwd.exec_ptr(x.data_ptr(), y.data_ptr(), S, stream)
        inv.exec_ptr(y.data_ptr(), z.data_ptr(), S, stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    fwd.check()
    inv.check()

    # ---- timed region: K steps, events around every launch for the roofline
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = fs.launch_count()
    with Clocks(local) as clk:
        barrier()
        e_start.record(stream)
        for i in range(args.steps):
            a, b, c = evs[i]
            a.record(stream)
            fwd.exec_ptr(x.data_ptr(), y.data_ptr(), S, stream)
            b.record(stream)
            inv.exec_ptr(y.data_ptr(), z.data_ptr(), S, stream)
            c.record(stream)
        e_end.record(stream)
        barrier()
    launches = fs.launch_count() - launches0
    ms = e_start.elapsed_time(e_end)
    kernel_ms = [a.elapsed_time(b) for a, b, _ in evs] + [b.elapsed_time(c) for _, b, c in evs]
    ms = max_over_ranks(ms, dev)
    ms_per_step = ms / args.steps
    flops_step = 2 * flops_per_transform(n, S)
    value = world * flops_step / (ms_per_step / 1e3) / 1e9

    # round-trip check of this very run (inverse(forward(x)) == x up to rounding)
    err = float(torch.linalg.vector_norm((z - x).flatten()) / torch.linalg.vector_norm(x.flatten()))

    # ---- roofline of the dominant kernel: algorithmic bytes per launch / mean launch time
    peak, peak_kind = peaks()
    per_launch_ms = statistics.mean(kernel_ms)
    algo_bytes = 16.0 * n * S
    achieved = algo_bytes / (per_launch_ms / 1e3) / 1e9
    traffic = measured_traffic("%s:%d" % (fwd.info()["path"], n))

    # ---- end to end through the public API with host buffers: fftseg_exec_host
    # runs the forward + inverse chain over the pinned host signal in chunks,
    # copies in both directions overlapped with the transforms
    # (untimed warm-up calls: the first host transfers after an idle spell run
    # several times slower while the host link ramps up)
    e2e, link = None, None
    if not args.no_e2e:
        e2e_steps = min(max(args.steps, 10), 20)  # isolated slow host transfers weigh less over more steps
        e2e_warm = max(args.warmup, 6)  # the first host transfers after an idle spell ramp up slowly
        for _ in range(e2e_warm):
            fs.exec_host([fwd, inv], h_in.data_ptr(), h_out.data_ptr(), S)
        barrier()
        t0 = time.perf_counter()
        e2e_step_ms = []
        for _ in range(e2e_steps):
            t1 = time.perf_counter()
            fs.exec_host([fwd, inv], h_in.data_ptr(), h_out.data_ptr(), S)  # synchronous
            e2e_step_ms.append(round((time.perf_counter() - t1) * 1e3, 2))
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e_value = world * flops_step / e2e_s / 1e9
        link = link_peaks(dev)
        k = min(S, 4)
        e2e_err = float(torch.linalg.vector_norm((h_out[: k * n] - h_in[: k * n])) / torch.linalg.vector_norm(h_in[: k * n]))
        e2e = {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(x.numel() * 8),
               "d2h_bytes_per_step": int(z.numel() * 8), "ms_per_step": round(e2e_s * 1e3, 2),
               "step_ms": e2e_step_ms, "median_step_ms": round(statistics.median(e2e_step_ms), 2),
               "warmup_calls": e2e_warm, "call": "fftseg_exec_host([forward, inverse]) on pinned host buffers",
               "link_gbs_each_way": round(x.numel() * 8 / e2e_s / 1e9, 1),
               "link_peaks_gbs": link,
               "link_frac": round(x.numel() * 8 / e2e_s / 1e9 / link["concurrent_each_way"], 4),
               "round_trip_rel_l2_first_%d_segments" % k: e2e_err}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(S, n), "n": n, "segments": S, "path": fwd.info()["path"],
                           "signal": "32 off-bin tones (log-uniform 1e-3..1) + complex Gaussian noise sigma 0.1, seed 1",
                           "l2": "inputs larger than L2 (%g GiB per buffer), no flush needed" % (S * n * 8 / 2**30),
                           "replicas": "one independent replica per GPU (no collective on the data path)"},
                "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved / peak, 4), "traffic": traffic,
                             "peak_kind": peak_kind,
                             "kernel": kernel_name(fwd.info()["path"], n, pflags) +
                             ("" if fwd.info()["launches_per_exec"] > 1 else " (one launch per transform, one HBM pass)"),
                             "algorithmic_bytes_per_launch": algo_bytes,
                             "mean_launch_ms": round(per_launch_ms, 4)},
                "gpu_launches": int(launches),
                "clocks": clk.summary(),
                "round_trip_rel_l2": err}
        if e2e is not None:
            line["e2e"] = e2e
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        if world == 1 and not args.no_extras:
            del x, y, z
            torch.cuda.empty_cache()
            line["vendor_fft_context"] = extra(vendor_context, n, S)
            line["c1"] = extra(c1_bench, peak)
            line["stream"] = extra(stream_bench, link or link_peaks(dev), h_in)
            line["tc_split"] = extra(tc_split, peak)
            line["real"] = extra(real_bench, peak)
            line["frames"] = extra(frames_bench, peak)
            line["file"] = extra(file_bench)
            line["bluestein"] = extra(bluestein_bench, peak)
            line["autotune"] = extra(tune_table)
            line["serve"] = extra(serve_bench, peak)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the tensor-core split and the serving run")
    ap.add_argument("--segments", type=int, default=0,
                    help="segments per transform (default 16384 at n = 65536, else 2^30 / n; "
                         "smaller only for profiler captures)")
    ap.add_argument("--n", type=int, default=N,
                    help="points per segment (default 65536, the benchmarked workload; other lengths only for "
                         "profiler captures of their kernels)")
    ap.add_argument("--flags", type=lambda v: int(v, 0), default=0, help="plan flags (profiler captures)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiler captures)")
    ap.add_argument("--only", choices=["real", "serve"], default=None,
                    help="run one extra measurement alone, at --n and --segments when given (profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch
        torch.cuda.set_device(0)
        peak, _ = peaks()
        if args.only == "real":
            sizes = [(args.n, args.segments or (1 << 30) // args.n)] if args.segments else None
            res = real_bench(peak, sizes)
        else:
            res = serve_bench(peak)
        print(json.dumps({"only": args.only, args.only: res}), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
