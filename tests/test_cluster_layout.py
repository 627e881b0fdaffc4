"""Host emulation of the cluster kernel's index maps and of the forms built on
it (no GPU): the real-signal split and join and the two Bluestein passes.

A segment of N = N1 N2 points is transformed by C = 2^LOG_C CTAs: CTA r takes
the column slab j2 in [r WA, (r + 1) WA) (point m = i N2 + r WA + c, i < N1) in
the column pass and rows k1 in [r WB, (r + 1) WB) in the row pass (bin
k = k1 + N1 k2).  Real-signal forward kernels deal the rows in mirror pairs
instead (rf_row / rf_place), so that bin k and bin N - k meet in one CTA.  This
test restates those maps and the formulas of the epilogues and column-pass
gathers, runs them with numpy FFTs in place of the stages, and checks the
results against numpy's rfft / irfft / fft.  The GPU parity tests pin
the kernels themselves.
"""
import numpy as np
import pytest

# (LOG_N1, LOG_N2, LOG_C) of every cluster shape the library instantiates
SHAPES = [(6, 7, 1), (7, 7, 2), (8, 7, 3), (8, 8, 3), (8, 8, 4), (8, 9, 4)]


def rf_row(N1, WB, d, c):
    H = WB // 2
    if c < H:
        return d * H + c
    m = d * H + c - H
    return N1 // 2 if m == 0 else N1 - m


def rf_place(N1, WB, k1):
    H = WB // 2
    hb = int(k1 >= N1 // 2)
    m = (N1 - k1 if hb else k1) & (N1 // 2 - 1)
    return m // H, hb * H + (m & (H - 1))


@pytest.mark.parametrize("l1,l2,lc", SHAPES)
def test_column_slabs_and_row_bins_cover_the_segment(l1, l2, lc):
    N1, N2, C = 1 << l1, 1 << l2, 1 << lc
    N = N1 * N2
    WA, WB = N2 // C, N1 // C
    pts = [i * N2 + r * WA + c for r in range(C) for i in range(N1) for c in range(WA)]
    assert sorted(pts) == list(range(N))
    bins = [r * WB + c + k2 * N1 for r in range(C) for c in range(WB) for k2 in range(N2)]
    assert sorted(bins) == list(range(N))


@pytest.mark.parametrize("l1,l2,lc", SHAPES)
def test_mirror_rows_meet_in_one_cta(l1, l2, lc):
    N1, C = 1 << l1, 1 << lc
    WB = N1 // C
    H = WB // 2
    rows = {}
    for d in range(C):
        for c in range(WB):
            k1 = rf_row(N1, WB, d, c)
            assert rf_place(N1, WB, k1) == (d, c)
            rows[k1] = (d, c)
            # the partner row sits in the same CTA, the other half
            if k1 not in (0, N1 // 2):
                assert rows.get(N1 - k1, rf_place(N1, WB, N1 - k1)) == (d, c ^ H)
    assert sorted(rows) == list(range(N1))
    assert rows[0] == (0, 0) and rows[N1 // 2] == (0, H)


@pytest.mark.parametrize("l1,l2,lc", [(6, 7, 1), (7, 7, 2), (8, 7, 3)])
def test_real_split_in_mirror_pairs(l1, l2, lc):
    # forward: z[j] = x[2j] + i x[2j+1], Z = DFT_N(z); each CTA's rows pair up
    # (k1, N1 - k1): bin k = k1 + N1 k2 with N - k = (N1 - k1) + N1 (N2 - 1 - k2)
    # (row 0: column N2 - k2 mod N2), X[k] = P + Q, X[N - k] = conj(P - Q)
    N1, N2, C = 1 << l1, 1 << l2, 1 << lc
    N = N1 * N2
    WB = N1 // C
    rng = np.random.default_rng(l1 * 100 + l2 * 10 + lc)
    x = rng.standard_normal(2 * N)
    Z = np.fft.fft(x[0::2] + 1j * x[1::2])
    X = np.full(N + 1, np.nan + 0j)
    for d in range(C):
        for c in range(WB):
            k1 = rf_row(N1, WB, d, c)
            for k2 in range(N2):
                if k1 == 0:
                    if k2 > N2 // 2:
                        continue  # formed with its partner N2 - k2
                    k, p1, p2 = 0, 0, (N2 - k2) % N2
                elif k1 == N1 // 2:
                    if k2 >= N2 // 2:
                        continue
                    k, p1, p2 = k1, k1, N2 - 1 - k2
                else:
                    if k1 > N1 // 2:
                        continue  # the first row of the pair forms both bins
                    k, p1, p2 = k1, N1 - k1, N2 - 1 - k2
                k += N1 * k2
                A, B = Z[k], np.conj(Z[p1 + N1 * p2])
                w = np.exp(-2j * np.pi * k / (2 * N))
                P, Q = (A + B) / 2, -1j * w * (A - B) / 2
                X[k], X[N - k] = P + Q, np.conj(P - Q)
    assert not np.isnan(X).any()
    np.testing.assert_allclose(X, np.fft.rfft(x), atol=1e-9 * np.abs(X).max())


@pytest.mark.parametrize("N", [1 << 13, 1 << 14])
def test_real_join_in_the_column_gather(N):
    # inverse: Z[m] = (A + B) + i conj(w_{2N}^m) (A - B), A = X[m],
    # B = conj(X[N - m]) (X[N] at m = 0; imaginary parts of X[0], X[N]
    # ignored); the unscaled inverse DFT_N of Z is x[2j] + i x[2j + 1], x the
    # unscaled inverse real DFT of length 2N of the bins
    rng = np.random.default_rng(N)
    X = rng.standard_normal(N + 1) + 1j * rng.standard_normal(N + 1)
    Xr = X.copy()
    Xr[0] = Xr[0].real
    Xr[N] = Xr[N].real
    m = np.arange(N)
    A = X[m].copy()
    A[0] = A[0].real
    Bm = X[N - m].copy()
    Bm[0] = Bm[0].real  # X[N] at m = 0
    B = np.conj(Bm)
    cw = np.conj(np.exp(-2j * np.pi * m / (2 * N)))
    Zm = (A + B) + 1j * cw * (A - B)
    z = np.fft.ifft(Zm) * N  # the kernel's unscaled inverse transform
    x = np.fft.irfft(Xr, 2 * N) * (2 * N)  # unscaled real inverse
    np.testing.assert_allclose(z.real, x[0::2], atol=1e-9 * np.abs(x).max())
    np.testing.assert_allclose(z.imag, x[1::2], atol=1e-9 * np.abs(x).max())


@pytest.mark.parametrize("n,sign", [(4099, -1), (9001, 1), (20011, -1)])
def test_bluestein_two_cluster_passes(n, sign):
    # forward pass (BF): point m = i N2 + r WA + c of row s is x[m] w[m] for
    # m < n, else 0; inverse pass (BL): its input times B as the column pass
    # reads it, bin k = r WB + c + k2 N1 of the result times scale w[k],
    # kept for k < n.  The shape is the cluster shape of M.
    M = 1 << int(np.ceil(np.log2(2 * n - 1)))
    l = int(np.log2(M))
    l1, l2, lc = {13: (6, 7, 1), 14: (7, 7, 2), 15: (8, 7, 3), 16: (8, 8, 4)}[l]
    N1, N2, C = 1 << l1, 1 << l2, 1 << lc
    WA, WB = N2 // C, N1 // C
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    mm = np.arange(n)
    w = np.exp(sign * 1j * np.pi * ((mm * mm) % (2 * n)) / n)
    b = np.zeros(M, dtype=complex)
    b[:n] = np.conj(w)
    b[M - n + 1:] = np.conj(w[1:][::-1])
    Bh = np.fft.fft(b) / M
    a = np.zeros(M, dtype=complex)
    for r in range(C):  # the forward pass's gather
        for i in range(N1):
            for c in range(WA):
                m = i * N2 + r * WA + c
                a[m] = x[m] * w[m] if m < n else 0
    Y = np.fft.fft(a) * Bh  # the inverse pass's input times B
    y = np.fft.ifft(Y) * M  # unscaled inverse transform
    out = np.full(n, np.nan + 0j)
    for r in range(C):  # the inverse pass's epilogue
        for c in range(WB):
            for k2 in range(N2):
                k = r * WB + c + k2 * N1
                if k < n:
                    out[k] = y[k] * w[k]
    assert not np.isnan(out).any()
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * n  # the length-n DFT
    np.testing.assert_allclose(out, ref, atol=1e-8 * np.abs(ref).max())
