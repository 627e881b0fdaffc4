"""Shared helpers for the GPU parity tests (no transform arithmetic here)."""
import math

import numpy as np


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) else np.float64)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((got - ref).ravel()) / (den if den > 0 else 1.0))


def tol_fp32(n: int) -> float:
    """FP32 path bound: relative L2 error <= 2e-6 * log2(n) per result."""
    return 2e-6 * max(1.0, math.log2(n))


def tol_power(n: int) -> float:
    """|X|^2 doubles the relative error to first order."""
    return 2.0 * tol_fp32(n)


TOL_TC = 1e-4  # tensor-core radix-16 path, per result
