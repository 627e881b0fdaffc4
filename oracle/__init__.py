"""FP64 CPU oracle for the segmented DFT (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
may import this package.  The product library never calls it and there is no
CPU fallback built on it.

What it computes (paper Sec. III, segments as <offset, FFT segment> records;
Sec. I, Cooley-Tukey = the DFT): for each segment s of length n,

    X_s[k] = scale * sum_j x_s[j] * exp(sigma * 2 pi i j k / n)

with sigma = -1 forward / +1 inverse and scale 1 (NONE), 1/n on the inverse
(BACKWARD) or 1/sqrt(n) (ORTHO).  The arithmetic is the recursive radix-2
FFT in oracle.c, in double precision.  The power output is |X|^2 in double.
"""
import ctypes
import os

import numpy as np

from . import build as _build

FORWARD = -1
INVERSE = +1
NORM_NONE = 0
NORM_BACKWARD = 1
NORM_ORTHO = 2

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        for name, ptr_t in (("oracle_fft_c64", ctypes.c_void_p), ("oracle_fft_c128", ctypes.c_void_p)):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [ptr_t, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                           ctypes.c_int, ctypes.c_int, ctypes.c_int]
        fn = lib.oracle_dft_c64
        fn.restype = ctypes.c_int
        fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def fft(x, direction: int = FORWARD, norm: int = NORM_NONE, nthreads: int = None) -> np.ndarray:
    """Segment-wise DFT of ``x`` along its last axis (length n, a power of two).

    ``x`` may be complex64 (the library's sample type; widened to double
    inside) or complex128 (exact inputs for pinning).  Returns complex128 of
    the same shape.
    """
    lib = _load()
    x = np.asarray(x)
    if x.dtype not in (np.complex64, np.complex128):
        raise TypeError("oracle.fft wants complex64 or complex128 input")
    if x.ndim == 0:
        raise ValueError("oracle.fft wants at least one axis")
    n = x.shape[-1]
    nseg = int(np.prod(x.shape[:-1], dtype=np.int64)) if x.ndim > 1 else 1
    xc = np.ascontiguousarray(x)
    out = np.empty(x.shape, dtype=np.complex128)
    if nseg == 0 or n == 0:
        return out
    fn = lib.oracle_fft_c64 if xc.dtype == np.complex64 else lib.oracle_fft_c128
    rc = fn(xc.ctypes.data, out.ctypes.data, n, nseg, int(direction), int(norm),
            int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("oracle rejected the arguments (status %d): n=%d must be a power of two" % (rc, n))
    return out


def power(x, direction: int = FORWARD, norm: int = NORM_NONE, nthreads: int = None) -> np.ndarray:
    """|X|^2 of the segment-wise DFT, in double."""
    X = fft(x, direction, norm, nthreads)
    return X.real * X.real + X.imag * X.imag


def rfft(x, norm: int = NORM_NONE, nthreads: int = None) -> np.ndarray:
    """DFT of real segments, bins k = 0..n/2 (the paper's records are real
    single-precision samples, Sec. III).

    The definition written out: the complex DFT of the real samples (imaginary
    part zero), forward, with the plan's scale (1, or 1/sqrt(n) for ORTHO),
    keeping the first n/2 + 1 bins; the rest follow by X[n-k] = conj(X[k]).
    ``x`` is float32 or float64, last axis of length n."""
    x = np.asarray(x)
    if x.dtype not in (np.float32, np.float64):
        raise TypeError("oracle.rfft wants float32 or float64 input")
    X = fft(x.astype(np.complex128), FORWARD, norm, nthreads)
    return X[..., : x.shape[-1] // 2 + 1]


def irfft(X, n: int, norm: int = NORM_NONE, nthreads: int = None) -> np.ndarray:
    """Real signal of length n from the bins X[0..n/2] of its DFT.

    The definition written out: the Hermitian extension Xf[k] = X[k] for
    k <= n/2 and Xf[k] = conj(X[n-k]) above, with the imaginary parts of X[0]
    and X[n/2] dropped (real bins of a real signal), through the inverse DFT
    with the plan's scale (1, 1/n for BACKWARD, 1/sqrt(n) for ORTHO); the
    result is real, its real part is returned."""
    X = np.asarray(X, dtype=np.complex128)
    if X.shape[-1] != n // 2 + 1:
        raise ValueError("oracle.irfft wants n/2 + 1 bins")
    Xf = np.empty(X.shape[:-1] + (n,), dtype=np.complex128)
    Xf[..., : n // 2 + 1] = X
    Xf[..., 0] = X[..., 0].real
    Xf[..., n // 2] = X[..., n // 2].real
    Xf[..., n // 2 + 1:] = np.conj(X[..., 1: n // 2][..., ::-1])
    return fft(Xf, INVERSE, norm, nthreads).real


WINDOW_RECT, WINDOW_HANN = 0, 1


def window(n: int, kind: int) -> np.ndarray:
    """The frame window in double: 1 (rectangular) or the periodic Hann window
    w[j] = (1 - cos(2 pi j / n)) / 2."""
    if kind == WINDOW_RECT:
        return np.ones(n)
    if kind == WINDOW_HANN:
        return 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / n)
    raise ValueError("unknown window %r" % kind)


def frames_fft(x, n: int, hop: int, nframes: int, kind: int = WINDOW_HANN, norm: int = NORM_NONE,
               nthreads: int = None) -> np.ndarray:
    """Overlapping segments, the definition written out: frame f holds samples
    x[f*hop .. f*hop + n - 1] (x complex, one signal), times the window, then
    the forward DFT with the plan's scale.  Returns [nframes][n] complex128."""
    x = np.asarray(x)
    idx = np.arange(nframes)[:, None] * hop + np.arange(n)[None, :]
    fr = x.astype(np.complex128)[idx] * window(n, kind)[None, :]
    return fft(fr, FORWARD, norm, nthreads)


def dft(x, direction: int = FORWARD, norm: int = NORM_NONE, bins=None, nthreads: int = None) -> np.ndarray:
    """Direct DFT of complex64 segments of any length n (last axis), the
    definition written out with the exponent index (j*k mod n) reduced exactly:
    X[k] = scale * sum_j x[j] exp(sigma 2 pi i j k / n).  `bins`: compute only
    these k (all n when None).  Returns complex128 [.., nbins]."""
    lib = _load()
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex64))
    n = x.shape[-1]
    nseg = int(np.prod(x.shape[:-1], dtype=np.int64)) if x.ndim > 1 else 1
    b = None if bins is None else np.ascontiguousarray(np.asarray(bins, dtype=np.int64))
    nb = n if b is None else b.size
    out = np.empty(x.shape[:-1] + (nb,), dtype=np.complex128)
    if nseg == 0 or n == 0 or nb == 0:
        return out
    rc = lib.oracle_dft_c64(x.ctypes.data, out.ctypes.data, n, nseg, int(direction), int(norm),
                            None if b is None else b.ctypes.data, int(nb), int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError("oracle rejected the arguments (status %d)" % rc)
    return out
