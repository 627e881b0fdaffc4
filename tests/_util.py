"""Shared helpers for the GPU parity tests (no transform arithmetic here)."""
import math

import numpy as np


def _as_rows(a):
    a = np.asarray(a)
    if a.ndim == 0:
        return a.reshape(1, 1)
    if a.ndim == 1:
        return a.reshape(1, -1)
    return a.reshape(a.shape[0], -1)


def rel_l2_global(got, ref) -> float:
    """||got - ref||_2 / ||ref||_2 over the whole result (all segments)."""
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) else np.float64)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((got - ref).ravel()) / (den if den > 0 else 1.0))


def seg_rel_l2(got, ref) -> float:
    """Worst single segment: max over rows s (the leading axis) of
    ||got[s] - ref[s]|| / ||ref[s]||.  A row whose reference is all zero is
    measured against the RMS row norm of the reference instead, so it must come
    out (close to) zero as well."""
    g = _as_rows(np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) else np.float64))
    r = _as_rows(ref)
    if g.shape != r.shape:
        raise ValueError("shape mismatch: %s vs %s" % (g.shape, r.shape))
    if g.size == 0:
        return 0.0
    num = np.linalg.norm(g - r, axis=1)
    den = np.linalg.norm(r, axis=1)
    rms = float(np.sqrt(np.mean(den ** 2)))
    den = np.where(den > 0, den, rms if rms > 0 else 1.0)
    return float(np.max(num / den))


def rel_l2(got, ref) -> float:
    """The error a parity test asserts: the larger of the whole-result relative
    L2 error and the worst single segment's (segments = rows of the leading
    axis), so that one bad segment cannot hide in a large batch."""
    return max(rel_l2_global(got, ref), seg_rel_l2(got, ref))


def tol_fp32(n: int) -> float:
    """FP32 path bound: relative L2 error <= 2e-6 * log2(n) per result."""
    return 2e-6 * max(1.0, math.log2(n))


def tol_power(n: int) -> float:
    """|X|^2 doubles the relative error to first order."""
    return 2.0 * tol_fp32(n)


TOL_TC = 1e-4  # tensor-core radix-16 path, per result


def guard(t, words: int = 64, value: int = 0x7FC0DEAD):
    """A guard band for an output buffer: returns (buffer, view) where view is
    the first t.numel() elements of a larger buffer whose tail of `words`
    32-bit words holds a canary, for check_guard."""
    import torch
    flat = t.reshape(-1)
    bytes_ = flat.numel() * flat.element_size()
    assert bytes_ % 4 == 0
    buf = torch.empty(bytes_ // 4 + words, dtype=torch.int32, device=t.device)
    buf[bytes_ // 4:] = value
    view = buf[:bytes_ // 4].view(t.dtype).reshape(t.shape)
    return buf, view


def check_guard(buf, words: int = 64, value: int = 0x7FC0DEAD):
    """Asserts that nothing wrote past the end of the guarded output."""
    tail = buf[buf.numel() - words:].cpu()
    assert bool((tail == value).all()), "a kernel wrote past the end of its output buffer"
