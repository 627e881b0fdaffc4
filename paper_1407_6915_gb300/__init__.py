"""fftseg: batched forward/inverse complex FFTs over fixed-length segments of a
very large signal, on one GB300 (sm_103a).

Thin ctypes binding of the C ABI in include/fftseg.h: it marshals arguments
(torch tensors -> device pointers, torch streams -> cudaStream_t) and does no
arithmetic.  Every transform runs in libfftseg.so's CUDA kernels; if that
library is missing or cannot load, importing the binding's entry points raises
(there is no CPU fallback).

Paper: Tsiomenko & Rees, "Accelerating Fast Fourier Transforms Using Hadoop
and CUDA", Sec. III (segments as <offset, FFT segment> records, batched plan
over a block, outputs in positional order).
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfftseg.so")

FORWARD, INVERSE = -1, 1
NORM_NONE, NORM_BACKWARD, NORM_ORTHO = 0, 1, 2
PREC_FP32, PREC_TC_FP16, PREC_TC_BF16 = 0, 1, 2
OUT_COMPLEX, OUT_POWER = 0, 1
FLAG_ZERO_PAD, FLAG_FORCE_TWOPASS, FLAG_FOURSTEP_L2, FLAG_FOURSTEP_PRODUCER = 0x1, 0x2, 0x4, 0x8
FLAG_AUTOTUNE = 0x10
FLAG_REAL = 0x20
FLAG_FOURSTEP_WARP_LINES, FLAG_FOURSTEP_TILES = 0x40, 0x80
FLAG_TEST_STALL = 0x1000
FLAG_BLUESTEIN = 0x2000
FILE_DIRECT, FILE_KEEP = 0x1, 0x2


WINDOW_RECT, WINDOW_HANN = 0, 1
PATH_NAMES = {0: "block", 1: "cluster", 2: "two-pass", 3: "tensor-core", 4: "four-step", 5: "real",
              6: "frames", 7: "bluestein", 8: "mixed-radix"}

OK, E_INVALID, E_NOMEM, E_CUDA, E_IO, E_PARTIAL, E_TIMEOUT, E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7


def FLAG_CLUSTER_LOG2(c):
    """Plan flag: single-pass cluster of 2^c CTAs (0 = the library's choice)."""
    return (int(c) & 0xF) << 8


STATUS_NAMES = {0: "OK", -1: "E_INVALID", -2: "E_NOMEM", -3: "E_CUDA", -4: "E_IO", -5: "E_PARTIAL",
                -6: "E_TIMEOUT", -7: "E_UNSUPPORTED"}

READ_FN = ctypes.CFUNCTYPE(ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64)
VIEW_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                           ctypes.POINTER(ctypes.c_int64))
WRITE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64)


class FFTSegError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%s)" % (message, STATUS_NAMES.get(status, status)))
        self.status = status


class SrvConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight_jobs", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class SrvJob(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("nseg", ctypes.c_int64), ("direction", ctypes.c_int), ("norm", ctypes.c_int)]


_lib = None

_SIGS = {
    "fftseg_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint]),
    "fftseg_plan_create_frames": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_uint]),
    "fftseg_exec": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fftseg_exec_n": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p]),
    "fftseg_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int64)]),
    "fftseg_stream_view": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "fftseg_stream_phases": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "fftseg_stream_file": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_uint,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "fftseg_autotune": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_double)]),
    "fftseg_exec_host": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]),
    "fftseg_exec_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "fftseg_noalloc_check": (ctypes.c_int, []),
    "fftseg_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fftseg_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "fftseg_plan_check": (ctypes.c_int, [ctypes.c_void_p]),
    "fftseg_last_error": (ctypes.c_char_p, []),
    "fftseg_launch_count": (ctypes.c_int64, []),
    "fftsrv_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(SrvConfig)]),
    "fftsrv_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SrvJob), ctypes.POINTER(ctypes.c_uint64)]),
    "fftsrv_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]),
    "fftsrv_poll_latency": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double)]),
    "fftsrv_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "fftsrv_destroy": (ctypes.c_int, [ctypes.c_void_p]),
}


def lib():
    """The loaded libfftseg.so.  Raises if it is absent: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfftseg.so is not built (run __graft_entry__.build()); "
                               "fftseg has no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().fftseg_last_error().decode(errors="replace")


def launch_count() -> int:
    return int(lib().fftseg_launch_count())


def check(status, what="fftseg"):
    if status != OK:
        raise FFTSegError(status, "%s: %s" % (what, last_error()))
    return status


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    return t if isinstance(t, int) else t.data_ptr()


def autotune(n, batch, precision=None, out_kind=None):
    """fftseg_autotune: (schedule flags, ms per exec) of the fastest schedule for n."""
    precision = PREC_FP32 if precision is None else precision
    out_kind = OUT_COMPLEX if out_kind is None else out_kind
    flags, ms = ctypes.c_uint(0), ctypes.c_double(0.0)
    check(lib().fftseg_autotune(int(n), int(batch), precision, out_kind, ctypes.byref(flags), ctypes.byref(ms)),
          "fftseg_autotune")
    return flags.value, ms.value


def exec_host(plans, h_in, h_out, nseg, chunk_segments=0) -> None:
    """fftseg_exec_host: nseg segments in host memory (tensors or addresses)
    through the plans in order; synchronous."""
    plans = list(plans) if isinstance(plans, (list, tuple)) else [plans]
    arr = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    check(lib().fftseg_exec_host(arr, len(plans), _ptr(h_in), _ptr(h_out), int(nseg), int(chunk_segments)),
          "fftseg_exec_host")


def segment_offset(s: int, n: int, sample_bytes: int = 8) -> int:
    """Byte offset of segment s (Sec. III: offset = bytes from the start of the file)."""
    return s * n * sample_bytes


def segment_count(total_bytes: int, n: int, sample_bytes: int = 8):
    """(complete segments, bytes left over) in a signal of total_bytes."""
    seg = n * sample_bytes
    return total_bytes // seg, total_bytes % seg


class Plan:
    """A batched plan over `batch` segments of n points (fftseg_plan_create)."""

    def __init__(self, n, batch, direction=FORWARD, norm=NORM_NONE, precision=PREC_FP32,
                 out_kind=OUT_COMPLEX, flags=0):
        self._h = ctypes.c_void_p()
        self.n, self.batch, self.direction, self.norm = int(n), int(batch), direction, norm
        self.precision, self.out_kind, self.flags = precision, out_kind, flags
        check(lib().fftseg_plan_create(ctypes.byref(self._h), self.n, self.batch, direction, norm,
                                       precision, out_kind, flags), "fftseg_plan_create")

    @property
    def handle(self):
        return self._h.value

    def segment_bytes(self):
        """(input, output) bytes of one segment as fftseg_stream counts them:
        complex64 n points in, n complex64 or float32 |X|^2 out; real-signal
        plans take 4n bytes of samples (forward) or n/2 + 1 bins (inverse)."""
        pw = 4 if self.out_kind == OUT_POWER else 8
        if self.flags & FLAG_REAL:
            bins = (self.n // 2 + 1) * 8
            if self.direction == FORWARD:
                return self.n * 4, (self.n // 2 + 1) * pw
            return bins, self.n * 4
        return self.n * 8, self.n * pw

    def info(self) -> dict:
        a = (ctypes.c_int64 * 6)()
        check(lib().fftseg_plan_info(self._h, a), "fftseg_plan_info")
        return {"path": PATH_NAMES.get(a[0], a[0]), "n1": a[1], "n2": a[2], "work_bytes": a[3],
                "work_segs": a[4], "launches_per_exec": a[5]}

    def exec_ptr(self, d_in: int, d_out: int, nseg: int = None, stream=None) -> None:
        """Raw-pointer form of fftseg_exec_n (asynchronous on `stream`)."""
        nseg = self.batch if nseg is None else nseg
        check(lib().fftseg_exec_n(self._h, d_in, d_out, nseg, _stream_handle(stream)), "fftseg_exec")

    def exec_host(self, h_in, h_out, nseg=None, chunk_segments=0) -> None:
        """fftseg_exec_host with this plan alone (host tensors or addresses)."""
        exec_host([self], h_in, h_out, self.batch if nseg is None else nseg, chunk_segments)

    def exec(self, x, out=None, nseg=None, stream=None):
        """Transform the first nseg segments of the device tensor x; returns `out`
        (allocated if None).  Complex plans: x complex64 [.., n].  Real-signal
        plans (FLAG_REAL): forward x float32 [.., n] -> complex64 (or float32
        power) [.., n/2 + 1]; inverse x complex64 [.., n/2 + 1] -> float32 [.., n]."""
        import torch
        if not (x.is_cuda and x.is_contiguous()):
            raise ValueError("fftseg.Plan.exec wants a contiguous CUDA tensor")
        real = bool(self.flags & FLAG_REAL)
        if real and self.direction == FORWARD:
            want, seg_in, seg_out = torch.float32, self.n, self.n // 2 + 1
            out_dt = torch.float32 if self.out_kind == OUT_POWER else torch.complex64
        elif real:
            want, seg_in, seg_out, out_dt = torch.complex64, self.n // 2 + 1, self.n, torch.float32
        else:
            want, seg_in, seg_out = torch.complex64, self.n, self.n
            out_dt = torch.float32 if self.out_kind == OUT_POWER else torch.complex64
        if x.dtype != want:
            raise ValueError("fftseg.Plan.exec wants %s input for this plan" % want)
        nseg = (x.numel() // seg_in) if nseg is None else nseg
        if out is None:
            shape = tuple(x.shape[:-1]) + (seg_out,) if x.dim() > 1 else (x.numel() // seg_in * seg_out,)
            out = torch.empty(shape, dtype=out_dt, device=x.device)
        self.exec_ptr(x.data_ptr(), out.data_ptr(), nseg, stream)
        return out

    def stream(self, reader, rctx, writer, wctx, total_bytes, start_offset=0, chunk_segments=0):
        """fftseg_stream.  reader/writer: C function pointers (int) with their
        context pointers, or Python callables (ctx ignored).  Returns
        (status, committed_offset) and does not raise on E_IO/E_PARTIAL."""
        keep = []

        def as_fn(f, proto):
            if isinstance(f, int):
                return ctypes.c_void_p(f)
            cb = proto(f)
            keep.append(cb)
            return ctypes.cast(cb, ctypes.c_void_p)

        committed = ctypes.c_int64(0)
        rc = lib().fftseg_stream(self._h, as_fn(reader, READ_FN), rctx, as_fn(writer, WRITE_FN), wctx,
                                 int(total_bytes), int(start_offset), int(chunk_segments),
                                 ctypes.byref(committed))
        if rc not in (OK, E_IO, E_PARTIAL):
            check(rc, "fftseg_stream")
        return rc, committed.value

    def stream_view(self, view, vctx, writer, wctx, total_bytes, start_offset=0, chunk_segments=0):
        """fftseg_stream_view: `view` lends the signal's host memory (a C
        function pointer (int) with its context, or a Python callable
        (ctx, offset, nbytes) -> (address, nbytes) or None).  Returns
        (status, committed_offset) and does not raise on E_IO/E_PARTIAL."""
        keep = []
        if isinstance(view, int):
            vfn = ctypes.c_void_p(view)
        else:
            def shim(ctx, off, nbytes, got):
                r = view(ctx, off, nbytes)
                if r is None:
                    return None
                got[0] = int(r[1])
                return int(r[0])
            cb = VIEW_FN(shim)
            keep.append(cb)
            vfn = ctypes.cast(cb, ctypes.c_void_p)
        if isinstance(writer, int):
            wfn = ctypes.c_void_p(writer)
        else:
            wcb = WRITE_FN(writer)
            keep.append(wcb)
            wfn = ctypes.cast(wcb, ctypes.c_void_p)
        committed = ctypes.c_int64(0)
        rc = lib().fftseg_stream_view(self._h, vfn, vctx, wfn, wctx, int(total_bytes), int(start_offset),
                                      int(chunk_segments), ctypes.byref(committed))
        if rc not in (OK, E_IO, E_PARTIAL):
            check(rc, "fftseg_stream_view")
        return rc, committed.value

    def stream_file(self, in_path, out_path, start_offset=0, chunk_segments=0, direct=True, end_offset=0,
                    keep_output=False):
        """fftseg_stream_file: the input byte range [start_offset, end_offset)
        (0: to the end) of the signal file through the plan into out_path, in
        positional order.  Returns (status, committed_offset) and does not raise
        on E_IO/E_PARTIAL."""
        committed = ctypes.c_int64(0)
        flags = (FILE_DIRECT if direct else 0) | (FILE_KEEP if keep_output else 0)
        rc = lib().fftseg_stream_file(self._h, os.fsencode(in_path), os.fsencode(out_path), int(start_offset),
                                      int(end_offset), int(chunk_segments), flags, ctypes.byref(committed))
        if rc not in (OK, E_IO, E_PARTIAL):
            check(rc, "fftseg_stream_file")
        return rc, committed.value

    def check(self) -> None:
        """Synchronise and raise if a kernel of this plan gave up a bounded wait."""
        check(lib().fftseg_plan_check(self._h), "fftseg_plan_check")

    def stream_phases(self) -> dict:
        a = (ctypes.c_double * 6)()
        check(lib().fftseg_stream_phases(self._h, a), "fftseg_stream_phases")
        return dict(zip(("read_ms", "h2d_ms", "fft_ms", "d2h_ms", "write_ms", "wall_ms"), list(a)))

    def destroy(self):
        if self._h and self._h.value:
            lib().fftseg_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class FramePlan(Plan):
    """Overlapping segments, a short-time FFT (fftseg_plan_create_frames): frame
    f of the signal holds samples [f*hop, f*hop + n), multiplied by the window,
    and is transformed forward like a segment of a complex plan."""

    def __init__(self, n, hop, batch, window=WINDOW_HANN, norm=NORM_NONE, out_kind=OUT_COMPLEX, flags=0):
        self._h = ctypes.c_void_p()
        self.n, self.batch, self.direction, self.norm = int(n), int(batch), FORWARD, norm
        self.precision, self.out_kind, self.flags = PREC_FP32, out_kind, flags
        self.hop, self.window = int(hop), window
        check(lib().fftseg_plan_create_frames(ctypes.byref(self._h), self.n, self.hop, window, self.batch, norm,
                                              out_kind, flags), "fftseg_plan_create_frames")

    def frames_in(self, samples: int) -> int:
        """Whole frames in a signal of `samples` samples."""
        return 0 if samples < self.n else (samples - self.n) // self.hop + 1

    def exec(self, x, out=None, nseg=None, stream=None):
        """Frames of the complex64 device signal x (contiguous): the first
        nseg frames (default: every whole frame, at most batch) -> out
        [nframes][n] (complex64, or float32 |X|^2)."""
        import torch
        if not (x.is_cuda and x.is_contiguous() and x.dtype == torch.complex64):
            raise ValueError("fftseg.FramePlan.exec wants a contiguous complex64 CUDA tensor")
        avail = self.frames_in(x.numel())
        nf = min(avail, self.batch) if nseg is None else int(nseg)
        if nf > avail:
            raise ValueError("the signal holds %d whole frames, %d asked" % (avail, nf))
        if out is None:
            dt = torch.float32 if self.out_kind == OUT_POWER else torch.complex64
            out = torch.empty((nf, self.n), dtype=dt, device=x.device)
        self.exec_ptr(x.data_ptr(), out.data_ptr(), nf, stream)
        return out


class Server:
    """Continuous-batching server (fftsrv_*)."""

    def __init__(self, hbm_budget_bytes=32 << 30, max_inflight_jobs=64, stream=None):
        self._h = ctypes.c_void_p()
        cfg = SrvConfig(hbm_budget_bytes=int(hbm_budget_bytes), max_inflight_jobs=int(max_inflight_jobs),
                        stream=(None if stream is None else _stream_handle(stream)))
        check(lib().fftsrv_create(ctypes.byref(self._h), ctypes.byref(cfg)), "fftsrv_create")

    def submit(self, d_in, d_out, n, nseg, direction=FORWARD, norm=NORM_NONE) -> int:
        job = SrvJob(d_in=_ptr(d_in), d_out=_ptr(d_out), n=int(n), nseg=int(nseg), direction=direction,
                     norm=norm)
        jid = ctypes.c_uint64()
        check(lib().fftsrv_submit(self._h, ctypes.byref(job), ctypes.byref(jid)), "fftsrv_submit")
        return jid.value

    def poll(self, job_id, timeout_us=0):
        """(done, job_status): done False while the job is queued or running."""
        st = ctypes.c_int(0)
        rc = lib().fftsrv_poll(self._h, job_id, int(timeout_us), ctypes.byref(st))
        if rc == E_TIMEOUT:
            return False, None
        check(rc, "fftsrv_poll")
        return True, st.value

    def poll_latency(self, job_id, timeout_us=0):
        """(done, job_status, latency_s): the job's submit-to-completion time
        as the server's host clock saw it (None while queued or running)."""
        st, lat = ctypes.c_int(0), ctypes.c_double(0.0)
        rc = lib().fftsrv_poll_latency(self._h, job_id, int(timeout_us), ctypes.byref(st), ctypes.byref(lat))
        if rc == E_TIMEOUT:
            return False, None, None
        check(rc, "fftsrv_poll_latency")
        return True, st.value, lat.value * 1e-6

    def stats(self) -> dict:
        a = (ctypes.c_int64 * 5)()
        check(lib().fftsrv_stats(self._h, a), "fftsrv_stats")
        return dict(zip(("submitted", "completed", "launches", "peak_admitted_bytes", "queue_depth"), list(a)))

    def destroy(self):
        if self._h and self._h.value:
            rc = lib().fftsrv_destroy(self._h)
            self._h = ctypes.c_void_p()
            check(rc, "fftsrv_destroy")

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
