"""Seeded synthetic signals (and reader/writer callbacks) for tests and benchmarks.

Holds no transform arithmetic.  Every complex64 sample is a pure function of
(seed, global sample index t), so a segment at byte offset b (paper Sec. III,
<offset, FFT segment> records) is regenerated from t = b / 8.  Both the CUDA
path's tests and the FP64 oracle take their inputs from here.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "siggen.c")
LIB = os.path.join(HERE, "libsiggen.so")

KIND_UNIFORM = 0
KIND_TONES = 1
KIND_POOL = 2
DEFAULT_TONES = 32
DEFAULT_SIGMA = 0.1


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                    "-o", tmp, SRC, "-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


class Source(ctypes.Structure):
    """Reader context (mirrors siggen_source in siggen.c)."""
    _fields_ = [("kind", ctypes.c_int32), ("ntones", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("sigma", ctypes.c_double), ("total_bytes", ctypes.c_int64),
                ("nthreads", ctypes.c_int32), ("fail_at_call", ctypes.c_int32),
                ("calls", ctypes.c_int64), ("pool", ctypes.c_void_p), ("pool_bytes", ctypes.c_int64)]


class Sink(ctypes.Structure):
    """Writer context (mirrors siggen_sink in siggen.c)."""
    _fields_ = [("base", ctypes.c_void_p), ("capacity", ctypes.c_int64),
                ("fail_at_call", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("calls", ctypes.c_int64), ("bytes_written", ctypes.c_int64),
                ("last_offset", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.siggen_uniform_c64.restype = ctypes.c_int
        L.siggen_uniform_c64.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_int]
        L.siggen_tones_c64.restype = ctypes.c_int
        L.siggen_tones_c64.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int]
        L.siggen_tone_params.restype = ctypes.c_int
        L.siggen_tone_params.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]
        L.siggen_read.restype = ctypes.c_int64
        L.siggen_read.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
        L.siggen_view.restype = ctypes.c_void_p
        L.siggen_view.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.siggen_write.restype = ctypes.c_int
        L.siggen_write.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64]
        _lib = L
    return _lib


def _threads(nthreads):
    return int(nthreads or max(1, os.cpu_count() or 1))


def uniform(seed: int, count: int, t0: int = 0, out=None, nthreads: int = None) -> np.ndarray:
    """complex64 samples t0 .. t0+count-1, re/im i.i.d. uniform on [-1, 1)."""
    if out is None:
        out = np.empty(count, dtype=np.complex64)
    assert out.dtype == np.complex64 and out.flags.c_contiguous and out.size == count
    if lib().siggen_uniform_c64(seed, t0, count, out.ctypes.data, _threads(nthreads)) != 0:
        raise ValueError("siggen_uniform_c64 rejected its arguments")
    return out


def tones(seed: int, count: int, t0: int = 0, ntones: int = DEFAULT_TONES,
          sigma: float = DEFAULT_SIGMA, out=None, nthreads: int = None) -> np.ndarray:
    """complex64 samples of `ntones` off-bin complex tones plus complex Gaussian noise."""
    if out is None:
        out = np.empty(count, dtype=np.complex64)
    assert out.dtype == np.complex64 and out.flags.c_contiguous and out.size == count
    if lib().siggen_tones_c64(seed, t0, count, out.ctypes.data, ntones, sigma,
                              _threads(nthreads)) != 0:
        raise ValueError("siggen_tones_c64 rejected its arguments")
    return out


def generate(kind: int, seed: int, count: int, t0: int = 0, out=None, nthreads: int = None,
             ntones: int = DEFAULT_TONES, sigma: float = DEFAULT_SIGMA) -> np.ndarray:
    if kind == KIND_UNIFORM:
        return uniform(seed, count, t0, out, nthreads)
    return tones(seed, count, t0, ntones, sigma, out, nthreads)


def fill_pointer(kind: int, seed: int, t0: int, count: int, ptr: int, nthreads: int = None,
                 ntones: int = DEFAULT_TONES, sigma: float = DEFAULT_SIGMA) -> None:
    """Generate straight into host memory at address ``ptr`` (e.g. a pinned tensor)."""
    L = lib()
    if kind == KIND_UNIFORM:
        rc = L.siggen_uniform_c64(seed, t0, count, ptr, _threads(nthreads))
    else:
        rc = L.siggen_tones_c64(seed, t0, count, ptr, ntones, sigma, _threads(nthreads))
    if rc != 0:
        raise ValueError("siggen rejected its arguments")


def tone_params(seed: int, ntones: int = DEFAULT_TONES):
    F = np.empty(ntones, dtype=np.uint64)
    Phi = np.empty(ntones, dtype=np.uint64)
    a = np.empty(ntones, dtype=np.float64)
    if lib().siggen_tone_params(seed, ntones, F.ctypes.data, Phi.ctypes.data, a.ctypes.data) != 0:
        raise ValueError("bad tone count")
    return F, Phi, a


def source(kind: int, seed: int, total_bytes: int, nthreads: int = None,
           ntones: int = DEFAULT_TONES, sigma: float = DEFAULT_SIGMA, fail_at_call: int = -1) -> Source:
    return Source(kind=kind, ntones=ntones, seed=seed, sigma=sigma, total_bytes=total_bytes,
                  nthreads=_threads(nthreads), fail_at_call=fail_at_call, calls=0, pool=None, pool_bytes=0)


def pool_source(pool_ptr: int, pool_bytes: int, total_bytes: int, nthreads: int = None,
                fail_at_call: int = -1) -> Source:
    """A reader context over a pre-generated host buffer (pool_bytes, a multiple
    of 8), read cyclically: byte offset b of the signal is pool[b mod pool_bytes]."""
    return Source(kind=KIND_POOL, ntones=0, seed=0, sigma=0.0, total_bytes=total_bytes,
                  nthreads=_threads(nthreads), fail_at_call=fail_at_call, calls=0, pool=pool_ptr,
                  pool_bytes=pool_bytes)


def sink(buf=None, fail_at_call: int = -1) -> Sink:
    """A writer context; ``buf`` (a writable numpy array or None) receives output at its offsets."""
    if buf is None:
        return Sink(base=None, capacity=0, fail_at_call=fail_at_call, pad=0, calls=0,
                    bytes_written=0, last_offset=-1)
    return Sink(base=buf.ctypes.data, capacity=buf.nbytes, fail_at_call=fail_at_call, pad=0,
                calls=0, bytes_written=0, last_offset=-1)


def view_fn_ptr() -> int:
    """siggen_view: the lending source of fftseg_stream_view over a pool source."""
    return ctypes.cast(lib().siggen_view, ctypes.c_void_p).value


def read_fn_ptr() -> int:
    return ctypes.cast(lib().siggen_read, ctypes.c_void_p).value


def write_fn_ptr() -> int:
    return ctypes.cast(lib().siggen_write, ctypes.c_void_p).value
