"""The lane-line four-step kernel's shared-memory addressing, checked on the
CPU (no GPU): for every line length (256, 512, 1024) and tile size (4096 and
8192 points) the address formulas of fourstep_wl.cuh, restated here, must
- land the TMA tile (swizzled rows of 32, 64 or 128 bytes) in the buffer,
- give every half-warp 16 distinct 8-byte bank slots in each phase (the
  stage-1 reads, both sides of the exchange, the stage-2 reads and the
  staged output), i.e. no bank conflicts,
- make the exchange a bijection of the line's own slots, and
- carry the data so that two Stockham stages (radix 32, then radix L/32)
  produce the line's DFT in the bins the kernel stores (checked against
  numpy's FFT on random lines).
This pins the layout's design; the GPU parity tests pin the kernel."""
import numpy as np
import pytest


def tile_offset(i, c, L, W):
    """Byte offset of element (row i, column c) of a tile as TMA lands it."""
    PW = min(W, 16)
    ROWB = PW * 8
    p, cc = divmod(c, PW)
    s = {128: 0, 64: 1, 32: 2}[ROWB]
    M = ROWB // 16 - 1
    return p * L * ROWB + i * ROWB + 16 * ((cc >> 1) ^ ((i >> s) & M)) + 8 * (cc & 1)


@pytest.mark.parametrize("log_l,log_e", [(8, 13), (9, 13), (10, 13), (8, 12), (9, 12), (10, 12)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_lane_line_tile_addressing(log_l, log_e, sign):
    L, E = 1 << log_l, 1 << log_e
    W, P = E // L, L // 32
    Q = 32 // P
    PW = min(W, 16)
    ROWB = PW * 8
    s = {128: 0, 64: 1, 32: 2}[ROWB]
    M = ROWB // 16 - 1

    def K(x):
        return ROWB * x + 16 * ((x >> s) & M)

    rng = np.random.default_rng(log_l * 10 + log_e)
    X = rng.standard_normal((W, L)) + 1j * rng.standard_normal((W, L))
    mem = np.full(E, np.nan + 0j)  # 8-byte slots of one tile buffer
    landed = set()
    for c in range(W):
        for i in range(L):
            o = tile_offset(i, c, L, W)
            assert o % 8 == 0 and 0 <= o < E * 8
            landed.add(o)
            mem[o // 8] = X[c, i]
    assert len(landed) == E

    TC, G = E // 32, 2 * P
    thr = []
    for t in range(TC):
        g, u = divmod(t, G)
        thr.append((2 * g + ((u >> 3) & 1), (u & 7) | ((u >> 4) << 3)))
    assert sorted(thr) == sorted((c, j) for c in range(W) for j in range(P))

    def bases(c, j):
        j7, ch, h = j & 7, (c % PW) >> 1, c & 1
        pb = (c // PW) * L * ROWB
        sw = 16 * (ch ^ ((j7 >> s) & M)) + 8 * h
        return pb + ROWB * j + sw, pb + 32 * ROWB * j + ROWB * j7 + sw

    def no_conflicts(addr):
        for h0 in range(0, TC, 16):
            assert len({(addr(t) % 128) // 8 for t in range(h0, h0 + 16)}) == 16

    for r in range(32):
        no_conflicts(lambda t: bases(*thr[t])[0] + ROWB * P * r)
    V = {}
    for t, (c, j) in enumerate(thr):
        rb, _ = bases(c, j)
        v = np.array([mem[(rb + ROWB * P * r) // 8] for r in range(32)])
        np.testing.assert_array_equal(v, X[c, j + P * np.arange(32)])
        V[t] = np.fft.fft(v) if sign < 0 else np.fft.ifft(v) * 32
    for r in range(32):
        no_conflicts(lambda t: (bases(*thr[t])[1] ^ K(r & 7)) + 8 * ROWB * (r >> 3))
    written = set()
    for t, (c, j) in enumerate(thr):
        _, wb = bases(c, j)
        for r in range(32):
            o = (wb ^ K(r & 7)) + 8 * ROWB * (r >> 3)
            assert 0 <= o < E * 8 and o not in written
            written.add(o)
            mem[o // 8] = V[t][r]
    assert written == landed
    for e in range(Q):
        for r in range(P):
            no_conflicts(lambda t: (bases(*thr[t])[0] ^ K(r & 7)) + ROWB * (P * e + 32 * r))
            no_conflicts(lambda t: bases(*thr[t])[0] + ROWB * (P * e + 32 * r))
    ref = np.fft.fft(X, axis=1) if sign < 0 else np.fft.ifft(X, axis=1) * L
    for t, (c, j) in enumerate(thr):
        rb, _ = bases(c, j)
        for e in range(Q):
            b = j + P * e
            seg = np.array([mem[((rb ^ K(r & 7)) + ROWB * (P * e + 32 * r)) // 8] for r in range(P)])
            seg = seg * np.exp(sign * 2j * np.pi * b * np.arange(P) / L)
            out = np.fft.fft(seg) if sign < 0 else np.fft.ifft(seg) * P
            for r in range(P):
                k = b + 32 * r
                assert abs(out[r] - ref[c, k]) < 1e-9 * L
                assert rb + ROWB * (P * e + 32 * r) == tile_offset(k, c, L, W)  # the staged bin's place


@pytest.mark.parametrize("log_n1,log_n2", [(8, 8), (9, 8), (9, 9), (10, 9), (10, 10)])
def test_frame_window_from_row_and_column_factors(log_n1, log_n2):
    """The lane-line kernel's periodic Hann window on a frame of n = N1 N2
    points, restated: lane j of a column line holds rows j1 = j + P r
    (P = N1 / 32, r < 32); its row factor is the table's (cos, sin)(2 pi j / N1)
    times exp(2 pi i (r mod 16) / 32), negated for r >= 16, and the window is
    1/2 - 1/2 Re(row factor x column factor (cos, sin)(2 pi j2 / n)).  It must
    equal (1 - cos(2 pi (j1 N2 + j2) / n)) / 2 at every point."""
    n1, n2 = 1 << log_n1, 1 << log_n2
    n, P = n1 * n2, n1 // 32
    j = np.arange(P)[:, None, None]
    r = np.arange(32)[None, :, None]
    j2 = np.arange(n2)[None, None, :]
    r0 = np.exp(2j * np.pi * j / n1)
    rr = r0 * np.exp(2j * np.pi * (r % 16) / 32) * np.where(r >= 16, -1, 1)
    wcol = np.exp(2j * np.pi * j2 / n)
    got = 0.5 - 0.5 * (rr * wcol).real
    j1 = j + P * r
    ref = 0.5 - 0.5 * np.cos(2 * np.pi * (j1 * n2 + j2) / n)
    np.testing.assert_allclose(got, ref, atol=1e-12)
