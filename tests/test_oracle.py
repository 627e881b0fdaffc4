"""Pins of the FP64 oracle against facts fixed by the mathematics, not by itself.

The paper (Sec. I, Sec. III) fixes the operation as the Cooley-Tukey FFT of
each fixed-length segment, i.e. exactly the DFT of each segment; it prints no
worked transform.  Each pin below would fail for a plausible mistake in
oracle.c (wrong twiddle sign or index, dropped scale, swapped halves, wrong
stride): see test_planted_mistakes_are_caught.
"""
import os
import re
import shutil
import subprocess
import ctypes

import numpy as np
import pytest

import oracle

FWD, INV = oracle.FORWARD, oracle.INVERSE
NONE, BACK, ORTHO = oracle.NORM_NONE, oracle.NORM_BACKWARD, oracle.NORM_ORTHO


def rel_l2(a, b):
    b = np.asarray(b)
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def brute_dft(x, sigma, scale):
    """O(n^2) DFT with the phase index reduced exactly: (j*k mod n)."""
    n = x.shape[-1]
    j = np.arange(n, dtype=np.int64)
    jk = np.outer(j, j) % n
    W = np.exp(sigma * 2j * np.pi * jk / n)
    return scale * (x @ W)


def rand_c128(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256])
@pytest.mark.parametrize("direction,norm", [(FWD, NONE), (INV, NONE), (INV, BACK), (FWD, BACK),
                                            (FWD, ORTHO), (INV, ORTHO)])
def test_matches_brute_force_dft(n, direction, norm):
    rng = np.random.default_rng(1000 + n)
    x = rand_c128(rng, (3, n))
    if norm == BACK:
        scale = 1.0 / n if direction == INV else 1.0
    elif norm == ORTHO:
        scale = 1.0 / np.sqrt(n)
    else:
        scale = 1.0
    ref = brute_dft(x, direction, scale)
    got = oracle.fft(x, direction, norm)
    assert rel_l2(got, ref) < 1e-13


def test_textbook_length4():
    # DFT of [1, 2, 3, 4]: X = [10, -2+2i, -2, -2-2i] (forward, exponent -)
    got = oracle.fft(np.array([1, 2, 3, 4], dtype=np.complex128), FWD)
    np.testing.assert_allclose(got, [10, -2 + 2j, -2, -2 - 2j], atol=1e-14)
    got = oracle.fft(np.array([1, 2, 3, 4], dtype=np.complex128), INV)
    np.testing.assert_allclose(got, [10, -2 - 2j, -2, -2 + 2j], atol=1e-14)


@pytest.mark.parametrize("n", [2, 16, 1024, 4096, 1 << 14])
@pytest.mark.parametrize("direction", [FWD, INV])
def test_impulse_closed_form(n, direction):
    # x = delta[j - j0]  =>  X[k] = exp(sigma 2 pi i j0 k / n), for every k
    k = np.arange(n, dtype=np.int64)
    for j0 in sorted({0, 1, n // 2, n - 1, (n * 3) // 7}):
        x = np.zeros(n, dtype=np.complex128)
        x[j0] = 1.0
        ref = np.exp(direction * 2j * np.pi * ((j0 * k) % n) / n)
        got = oracle.fft(x, direction)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.log2(max(n, 2))


@pytest.mark.parametrize("n", [4, 256, 8192])
def test_pure_tone_closed_form(n):
    j = np.arange(n, dtype=np.int64)
    for m in sorted({0, 1, n // 4, n - 1}):
        x = np.exp(2j * np.pi * ((m * j) % n) / n)
        fwd = oracle.fft(x, FWD)
        ref = np.zeros(n, dtype=np.complex128)
        ref[m] = n
        assert np.max(np.abs(fwd - ref)) < 1e-9 * n
        inv = oracle.fft(x, INV)
        ref = np.zeros(n, dtype=np.complex128)
        ref[(-m) % n] = n
        assert np.max(np.abs(inv - ref)) < 1e-9 * n
    const = np.full(n, 2.5 - 1j)
    got = oracle.fft(const, FWD)
    ref = np.zeros(n, dtype=np.complex128)
    ref[0] = n * (2.5 - 1j)
    assert np.max(np.abs(got - ref)) < 1e-10 * n


@pytest.mark.parametrize("n", [8, 1024, 1 << 16])
def test_parseval(n):
    rng = np.random.default_rng(7)
    x = rand_c128(rng, (2, n))
    X = oracle.fft(x, FWD)
    lhs = np.sum(np.abs(X) ** 2, axis=-1)
    rhs = n * np.sum(np.abs(x) ** 2, axis=-1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12)
    Xo = oracle.fft(x, FWD, ORTHO)
    np.testing.assert_allclose(np.sum(np.abs(Xo) ** 2, axis=-1), np.sum(np.abs(x) ** 2, axis=-1),
                               rtol=1e-12)


def test_linearity():
    rng = np.random.default_rng(8)
    n = 512
    x, y = rand_c128(rng, n), rand_c128(rng, n)
    a, b = 0.75 - 1.25j, -2.0 + 0.5j
    lhs = oracle.fft(a * x + b * y, FWD)
    rhs = a * oracle.fft(x, FWD) + b * oracle.fft(y, FWD)
    assert rel_l2(lhs, rhs) < 1e-14


@pytest.mark.parametrize("n", [2, 64, 4096, 1 << 15])
def test_round_trip(n):
    rng = np.random.default_rng(9)
    x = rand_c128(rng, (2, n))
    back = oracle.fft(oracle.fft(x, FWD, NONE), INV, BACK)
    assert rel_l2(back, x) < 1e-14
    back = oracle.fft(oracle.fft(x, FWD, ORTHO), INV, ORTHO)
    assert rel_l2(back, x) < 1e-14


def test_shift_theorem():
    rng = np.random.default_rng(10)
    n, m = 1024, 37
    x = rand_c128(rng, n)
    xs = np.roll(x, m)  # xs[j] = x[(j - m) mod n]
    k = np.arange(n)
    ref = oracle.fft(x, FWD) * np.exp(-2j * np.pi * ((m * k) % n) / n)
    assert rel_l2(oracle.fft(xs, FWD), ref) < 1e-13


def test_conjugate_symmetry_real_input():
    rng = np.random.default_rng(11)
    n = 2048
    x = rng.standard_normal(n).astype(np.complex128)
    X = oracle.fft(x, FWD)
    k = np.arange(1, n)
    assert np.max(np.abs(X[n - k] - np.conj(X[k]))) < 1e-11
    assert abs(X[0].imag) < 1e-11 and abs(X[n // 2].imag) < 1e-11


@pytest.mark.parametrize("n", [2, 1024, 1 << 16])
def test_numpy_library_cross_check(n):
    # numpy's pocketfft is a library routine used here only as a check
    rng = np.random.default_rng(12)
    x = rand_c128(rng, (2, n)).astype(np.complex64)
    assert rel_l2(oracle.fft(x, FWD), np.fft.fft(x.astype(np.complex128))) < 1e-12
    assert rel_l2(oracle.fft(x, INV, BACK), np.fft.ifft(x.astype(np.complex128))) < 1e-12
    assert rel_l2(oracle.fft(x, FWD, ORTHO), np.fft.fft(x.astype(np.complex128), norm="ortho")) < 1e-12


def test_segments_are_independent_and_in_offset_order():
    # Sec. III: the file is a sequence of <offset, FFT segment> records; each
    # segment is transformed on its own and outputs keep positional order.
    rng = np.random.default_rng(13)
    n, B = 256, 9
    sig = rand_c128(rng, n * B)
    batch = oracle.fft(sig.reshape(B, n), FWD)
    for s in range(B):
        offset_bytes = s * n * 16  # complex128 here
        seg = sig.view(np.uint8)[offset_bytes:offset_bytes + n * 16].view(np.complex128)
        np.testing.assert_array_equal(batch[s], oracle.fft(seg, FWD))


def test_complex64_input_is_widened_exactly():
    rng = np.random.default_rng(14)
    x32 = rand_c128(rng, 128).astype(np.complex64)
    np.testing.assert_array_equal(oracle.fft(x32, FWD), oracle.fft(x32.astype(np.complex128), FWD))


def test_thread_count_does_not_change_results():
    rng = np.random.default_rng(15)
    x = rand_c128(rng, (13, 512)).astype(np.complex64)
    a = oracle.fft(x, FWD, nthreads=1)
    b = oracle.fft(x, FWD, nthreads=5)
    np.testing.assert_array_equal(a, b)


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.zeros(12, dtype=np.complex64))


def test_power_is_squared_magnitude():
    rng = np.random.default_rng(16)
    x = rand_c128(rng, (2, 64)).astype(np.complex64)
    X = oracle.fft(x, FWD)
    np.testing.assert_allclose(oracle.power(x), np.abs(X) ** 2, rtol=1e-14)


# ------------------------------------------------------------------------
# Planted mistakes: each mutation of oracle.c must be caught by the pins.

MUTATIONS = {
    "twiddle_sign": ("const double wi = (double)sigma * sin(a);", "const double wi = -(double)sigma * sin(a);"),
    "twiddle_index": ("const double a = kTwoPi * (double)k / (double)n;",
                      "const double a = kTwoPi * (double)(k + 1) / (double)n;"),
    "dropped_scale": ("return sigma > 0 ? 1.0 / (double)n : 1.0;", "return 1.0;"),
    "swapped_halves": ("fft_rec(x, 2 * stride, X, h, sigma);", "fft_rec(x + 2 * stride, 2 * stride, X, h, sigma);"),
    "butterfly_sign": ("X[2 * (k + h)] = er - tr;", "X[2 * (k + h)] = er + tr;"),
}


def _build_mutant(tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) >= 1, name
    src = src.replace(old, new, 1)
    if name == "swapped_halves":
        src = src.replace("fft_rec(x + 2 * stride, 2 * stride, X + 2 * h, h, sigma);",
                          "fft_rec(x, 2 * stride, X + 2 * h, h, sigma);", 1)
    c = tmp_path / ("m_%s.c" % name)
    c.write_text(src)
    so = tmp_path / ("m_%s.so" % name)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-pthread", "-o", str(so), str(c), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    fn = lib.oracle_fft_c128
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int]
    return fn


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(tmp_path, name):
    fn = _build_mutant(tmp_path, name)
    rng = np.random.default_rng(17)
    n = 64
    x = np.ascontiguousarray(rand_c128(rng, n))
    caught = False
    for direction, norm in ((FWD, NONE), (INV, BACK)):
        out = np.empty(n, dtype=np.complex128)
        assert fn(x.ctypes.data, out.ctypes.data, n, 1, direction, norm, 1) == 0
        scale = 1.0 / n if (direction == INV and norm == BACK) else 1.0
        if rel_l2(out, brute_dft(x, direction, scale)) > 1e-6:
            caught = True
    assert caught, "mutation %s survived the brute-force pin" % name


# ---- real-signal segments (rfft / irfft): pinned against the complex DFT's
# symmetry, a library cross-check and the round trip

@pytest.mark.parametrize("n", [4, 8, 16, 256, 4096])
def test_rfft_is_the_half_spectrum_of_the_brute_force_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n))
    X = oracle.rfft(x)
    ref = brute_dft(x.astype(np.complex128), -1, 1.0)[:, : n // 2 + 1]
    assert rel_l2(X, ref) < 1e-12
    assert np.all(np.abs(X[:, 0].imag) < 1e-9) and np.all(np.abs(X[:, n // 2].imag) < 1e-9)


@pytest.mark.parametrize("n", [4, 64, 1 << 14])
@pytest.mark.parametrize("norm,np_norm", [(NONE, "backward"), (ORTHO, "ortho")])
def test_rfft_irfft_match_numpy(n, norm, np_norm):
    rng = np.random.default_rng(7 + n)
    x = rng.standard_normal((2, n))
    assert rel_l2(oracle.rfft(x, norm), np.fft.rfft(x, norm=np_norm)) < 1e-12
    X = np.fft.rfft(x) + 1j * 0.25  # the imaginary parts of X[0], X[n/2] must be ignored
    want = np.fft.irfft(X, n, norm="forward" if norm == NONE else "ortho")
    assert rel_l2(oracle.irfft(X, n, norm), want) < 1e-12


@pytest.mark.parametrize("n", [4, 32, 1 << 12])
def test_irfft_inverts_rfft(n):
    x = np.random.default_rng(n).standard_normal((4, n))
    assert rel_l2(oracle.irfft(oracle.rfft(x), n, BACK), x) < 1e-12
    assert rel_l2(oracle.irfft(oracle.rfft(x, ORTHO), n, ORTHO), x) < 1e-12


# ---- overlapping segments (frames_fft): pinned by reduction to the pinned
# segment DFT, closed forms of the Hann window, and brute force

def test_frames_with_hop_n_and_no_window_are_segments():
    n, F = 64, 5
    x = rand_c128(np.random.default_rng(3), F * n)
    got = oracle.frames_fft(x, n, n, F, oracle.WINDOW_RECT)
    assert rel_l2(got, oracle.fft(x.reshape(F, n))) < 1e-14


@pytest.mark.parametrize("n,hop", [(16, 8), (64, 17), (256, 64)])
def test_hann_frames_of_an_on_bin_tone(n, hop):
    # x[t] = exp(2 pi i m t / n): frame f is the tone times the window, with
    # phase exp(2 pi i m f hop / n); the periodic Hann window's DFT is
    # n/2 at 0 and -n/4 at +-1, so X_f = phase * (n/2, -n/4, -n/4 at m, m+-1)
    m, F = 5, 4
    t = np.arange((F - 1) * hop + n)
    x = np.exp(2j * np.pi * ((m * t) % n) / n)
    got = oracle.frames_fft(x, n, hop, F, oracle.WINDOW_HANN)
    want = np.zeros((F, n), dtype=np.complex128)
    for f in range(F):
        ph = np.exp(2j * np.pi * ((m * f * hop) % n) / n)
        want[f, m] = ph * n / 2
        want[f, (m + 1) % n] = -ph * n / 4
        want[f, (m - 1) % n] = -ph * n / 4
    assert np.max(np.abs(got - want)) < 1e-9 * n


@pytest.mark.parametrize("n,hop,kind", [(8, 3, 0), (16, 5, 1), (32, 32, 1), (16, 20, 0)])
def test_frames_brute_force(n, hop, kind):
    F = 4
    x = rand_c128(np.random.default_rng(n + hop), (F - 1) * hop + n)
    w = np.ones(n) if kind == 0 else np.array([0.5 - 0.5 * np.cos(2 * np.pi * j / n) for j in range(n)])
    want = np.stack([brute_dft(x[f * hop: f * hop + n] * w, -1, 1.0) for f in range(F)])
    assert rel_l2(oracle.frames_fft(x, n, hop, F, kind), want) < 1e-12
    assert rel_l2(oracle.frames_fft(x, n, hop, F, kind, ORTHO), want / np.sqrt(n)) < 1e-12


# ---- the direct DFT (any length): pinned against the radix-2 oracle where
# both apply, numpy elsewhere, and the impulse closed form

@pytest.mark.parametrize("n", [1, 2, 8, 64, 512])
def test_direct_dft_equals_radix2_at_powers_of_two(n):
    x = rand_c128(np.random.default_rng(n), (3, n)).astype(np.complex64)
    for sigma, norm in ((FWD, NONE), (INV, BACK), (FWD, ORTHO)):
        assert rel_l2(oracle.dft(x, sigma, norm), oracle.fft(x, sigma, norm)) < 1e-13


@pytest.mark.parametrize("n", [3, 5, 6, 7, 12, 100, 1000, 1001, 4093])
def test_direct_dft_matches_numpy(n):
    x = rand_c128(np.random.default_rng(n), (2, n)).astype(np.complex64)
    xc = x.astype(np.complex128)
    assert rel_l2(oracle.dft(x), np.fft.fft(xc)) < 1e-12
    assert rel_l2(oracle.dft(x, INV, BACK), np.fft.ifft(xc)) < 1e-12


@pytest.mark.parametrize("n,j0", [(12, 5), (1001, 700)])
def test_direct_dft_impulse_and_bins(n, j0):
    x = np.zeros(n, dtype=np.complex64)
    x[j0] = 1
    k = np.arange(n)
    want = np.exp(-2j * np.pi * ((j0 * k) % n) / n)
    assert np.max(np.abs(oracle.dft(x) - want)) < 1e-12
    sel = np.array([0, n - 1, 7 % n, n // 2])
    assert np.max(np.abs(oracle.dft(x, bins=sel) - want[sel])) < 1e-12
