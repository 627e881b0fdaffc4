"""Host emulation of the interleaved four-step's data layouts (no GPU).

For n = R * M (M = N1 N2) the library runs an outer radix-R pass that forms
Y_t[j] = w_n^{j t} DFT_R(x[j + M t'])[t] and stores it unit by unit: unit
b = t div 32 of segment s holds its 32 transforms column after column, point
j = j1 N2 + j2 of transform 32 b + c at ((b N2 + j2) N1 + j1) 32 + c of the
segment.  A lane-line pass then takes, per unit, column tile j2 (one
contiguous N1 x 32 block), keeps the ring as [k1][j2][transform], and row
tile k1 writes X[t + R (k1 + N1 k2)] as row k2, element R k1 + t.  This test
walks exactly those index maps with numpy DFTs at small sizes (N1 = N2 = 8)
and checks the result against numpy's FFT of the whole segment.
"""
import numpy as np
import pytest


def emulate(x, R, N1, N2):
    M = N1 * N2
    n = R * M
    G = R // 32
    nseg = x.shape[0]
    # outer pass: Y[s][((b N2 + j2) N1 + j1) 32 + c] for t = 32 b + c, j = j1 N2 + j2
    Y = np.full((nseg, n), np.nan + 0j)
    t = np.arange(R)
    for j in range(M):
        j1, j2 = divmod(j, N2)
        col = x[:, j + M * t]                              # [s][t']
        d = np.fft.fft(col, axis=1)                        # DFT_R over t'
        Y[:, ((t // 32 * N2 + j2) * N1 + j1) * 32 + t % 32] = d * np.exp(-2j * np.pi * j * t / n)
    assert not np.isnan(Y).any()
    X = np.full((nseg, n), np.nan + 0j)
    for s in range(nseg):
        for b in range(G):
            ring = np.empty((N1, N2, 32), dtype=np.complex128)   # [k1][j2][c]
            for j2 in range(N2):                                 # column tile j2 of unit s G + b
                # one contiguous block [j1][c] at ((b N2 + j2) N1) 32
                tile = Y[s].reshape(G * N2, N1, 32)[b * N2 + j2]  # [j1][c]
                colft = np.fft.fft(tile, axis=0)                  # over j1 -> k1
                k1 = np.arange(N1)[:, None]
                ring[:, j2, :] = colft * np.exp(-2j * np.pi * j2 * k1 / M)
            out = X[s].reshape(N2, N1 * R)                         # [k2][R k1 + t]
            for k1 in range(N1):                                  # row tile k1
                rowft = np.fft.fft(ring[k1], axis=0)              # over j2 -> k2, [k2][c]
                out[:, R * k1 + 32 * b: R * k1 + 32 * b + 32] = rowft
    return X


@pytest.mark.parametrize("R", [32, 64])
def test_interleaved_layouts_give_the_dft(R):
    rng = np.random.default_rng(R)
    N1 = N2 = 8
    n = R * N1 * N2
    x = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    X = emulate(x, R, N1, N2)
    assert not np.isnan(X).any()  # every output written
    np.testing.assert_allclose(X, np.fft.fft(x, axis=1), rtol=0, atol=1e-9 * np.sqrt(n))
