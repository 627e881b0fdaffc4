"""The seeded input generators: determinism, offset regeneration, definition."""
import numpy as np

import siggen


def test_uniform_range_and_grid():
    x = siggen.uniform(0, 1 << 16)
    parts = np.concatenate([x.real, x.imag]).astype(np.float64)
    assert parts.min() >= -1.0 and parts.max() < 1.0
    # values lie on the 2^-23 grid (24-bit integers), exact in float32
    k = (parts + 1.0) * 2.0 ** 23
    np.testing.assert_array_equal(k, np.round(k))
    assert abs(parts.mean()) < 0.01 and abs(parts.var() - 1.0 / 3.0) < 0.01


def test_segments_regenerate_from_their_offset():
    # Sec. III: a segment is identified by its byte offset; the generator must
    # give the same samples whether produced in one piece or from the offset.
    n = 1024
    whole = siggen.uniform(3, 8 * n)
    seg5 = siggen.uniform(3, n, t0=5 * n)
    np.testing.assert_array_equal(whole[5 * n:6 * n], seg5)
    whole = siggen.tones(4, 8 * n)
    for t0, cnt in ((5 * n, n), (77, 300), (1, 63)):
        np.testing.assert_array_equal(whole[t0:t0 + cnt], siggen.tones(4, cnt, t0=t0))


def test_thread_count_independent():
    a = siggen.tones(1, 100_000, t0=123, nthreads=1)
    b = siggen.tones(1, 100_000, t0=123, nthreads=7)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(siggen.uniform(2, 50_000, nthreads=1), siggen.uniform(2, 50_000, nthreads=6))


def test_seeds_differ():
    assert not np.array_equal(siggen.uniform(0, 64), siggen.uniform(1, 64))
    assert not np.array_equal(siggen.tones(0, 64), siggen.tones(1, 64))


def test_tones_follow_their_definition():
    seed, ntones = 1, 32
    F, Phi, a = siggen.tone_params(seed, ntones)
    assert np.all(a >= 1e-3 - 1e-15) and np.all(a <= 1.0)
    t = np.arange(5000, 5000 + 256, dtype=np.uint64)
    x = siggen.tones(seed, t.size, t0=int(t[0]), ntones=ntones, sigma=0.0)
    ref = np.zeros(t.size, dtype=np.complex128)
    for k in range(ntones):
        theta = (F[k] * t + Phi[k])  # uint64 arithmetic wraps mod 2^64
        frac = (theta >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        ref += a[k] * np.exp(2j * np.pi * frac)
    assert np.max(np.abs(x - ref)) < 1e-5 * np.max(np.abs(ref))


def _mix64(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def test_tones_and_noise_to_float32_rounding():
    # the whole sample against its definition evaluated independently in numpy
    # (SplitMix64 counters, exact integer phases, Box-Muller), rounded once to
    # float32: at most one float32 ulp apart (the two double evaluations
    # differ only in their last bits)
    seed, ntones, sigma = 2, 32, 0.1
    G = np.uint64(0x9E3779B97F4A7C15)
    key = lambda stream: _mix64(_mix64(np.uint64(seed)) + np.uint64(stream) * G)
    F, Phi, a = siggen.tone_params(seed, ntones)
    t = np.arange(123_456, 123_456 + 700, dtype=np.uint64)
    with np.errstate(over="ignore"):
        u1 = ((_mix64(key(2) + (t + np.uint64(1)) * G) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = (_mix64(key(3) + (t + np.uint64(1)) * G) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        ref = sigma * np.sqrt(-2.0 * np.log(u1)) * np.exp(2j * np.pi * u2)
        for k in range(ntones):
            frac = ((F[k] * t + Phi[k]) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
            ref = ref + a[k] * np.exp(2j * np.pi * frac)
    x = siggen.tones(seed, t.size, t0=int(t[0]), ntones=ntones, sigma=sigma)
    for part in ("real", "imag"):
        got = getattr(x, part).astype(np.float64)
        want = getattr(ref, part)
        ulp = np.spacing(np.abs(want).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got - want) <= ulp + 1e-15), part


def test_pool_source_reads_cyclically():
    import ctypes
    L = siggen.lib()
    pool = siggen.uniform(4, 5000)
    src = siggen.pool_source(pool.ctypes.data, pool.nbytes, total_bytes=3 * pool.nbytes, nthreads=3)
    buf = np.empty(7000, dtype=np.complex64)
    assert L.siggen_read(ctypes.byref(src), 4000 * 8, buf.ctypes.data, buf.nbytes) == buf.nbytes
    want = np.concatenate([pool, pool, pool])[4000:11000]
    np.testing.assert_array_equal(buf, want)


def test_noise_statistics():
    x = siggen.tones(9, 1 << 18, ntones=0, sigma=0.1).astype(np.complex128)
    assert abs(np.std(x.real) - 0.1) < 0.002 and abs(np.std(x.imag) - 0.1) < 0.002
    assert abs(np.mean(x.real)) < 0.002 and abs(np.corrcoef(x.real, x.imag)[0, 1]) < 0.01


def test_reader_and_writer_callbacks():
    import ctypes
    L = siggen.lib()
    n = 256
    src = siggen.source(siggen.KIND_TONES, 5, total_bytes=10 * n * 8)
    buf = np.empty(3 * n, dtype=np.complex64)
    got = L.siggen_read(ctypes.byref(src), 2 * n * 8, buf.ctypes.data, buf.nbytes)
    assert got == buf.nbytes
    np.testing.assert_array_equal(buf, siggen.tones(5, 3 * n, t0=2 * n))
    # short read at the end of the signal
    got = L.siggen_read(ctypes.byref(src), 9 * n * 8, buf.ctypes.data, buf.nbytes)
    assert got == n * 8
    out = np.zeros(4 * n, dtype=np.complex64)
    snk = siggen.sink(out)
    assert L.siggen_write(ctypes.byref(snk), n * 8, buf.ctypes.data, n * 8) == 0
    np.testing.assert_array_equal(out[n:2 * n], buf[:n])
    assert snk.bytes_written == n * 8 and snk.last_offset == n * 8
    bad = siggen.source(siggen.KIND_UNIFORM, 5, total_bytes=10 * n * 8, fail_at_call=0)
    assert L.siggen_read(ctypes.byref(bad), 0, buf.ctypes.data, buf.nbytes) == -1
