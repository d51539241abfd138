"""Pins of the oracle's circulant embedding and BTTB product (Sections II.B, V.A-B).

The FFT-based product must equal the plain O(N^2) Toeplitz sum exactly (up
to rounding) on tiny and non-cubic grids; a non-symmetric random defining
tensor makes any index reversal or axis swap visible.
"""
import numpy as np
import pytest

from oracle import embed as E
from oracle import kernel as K
from oracle import matvec as M

K0 = K.wavenumber(298e6)


def _rand(shape, rng):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n", [(3, 4, 5), (4, 4, 4), (2, 3, 2), (5, 3, 4)])
def test_fft_product_equals_toeplitz_sum_random_tensor(n):
    rng = np.random.default_rng(7)
    n1, n2, n3 = n
    T = _rand((6, 2 * n1 - 1, 2 * n2 - 1, 2 * n3 - 1), rng)
    J = _rand((2, 3, n1, n2, n3), rng)
    Ghat = E.green_spectra(T, n1, n2, n3)
    y_fft = M.matvec_fft(Ghat, J)
    y_bf = M.matvec_bruteforce(T, J)
    assert np.linalg.norm(y_fft - y_bf) <= 1e-12 * np.linalg.norm(y_bf)


@pytest.mark.parametrize("n", [(3, 4, 5), (6, 6, 6)])
def test_fft_product_equals_toeplitz_sum_green_kernel(n):
    rng = np.random.default_rng(3)
    n1, n2, n3 = n
    T = K.toeplitz_tensor(n1, n2, n3, 5e-3, K0)
    J = _rand((3, n1, n2, n3), rng)
    y_fft = M.matvec_fft(E.green_spectra(T, n1, n2, n3), J)
    y_bf = M.matvec_bruteforce(T, J)
    assert np.linalg.norm(y_fft - y_bf) <= 1e-12 * np.linalg.norm(y_bf)


def test_dense_operator_matches_bruteforce_and_is_complex_symmetric():
    rng = np.random.default_rng(1)
    n1, n2, n3 = 3, 2, 4
    T = K.toeplitz_tensor(n1, n2, n3, 5e-3, K0)
    G = M.dense_operator(T, n1, n2, n3)
    J = _rand((3, n1, n2, n3), rng)
    assert np.allclose(G @ J.ravel(), M.matvec_bruteforce(T, J).ravel(), rtol=0, atol=1e-14)
    assert np.allclose(G, G.T, rtol=0, atol=0)


def test_embedding_layout():
    n1, n2, n3 = 3, 4, 2
    T = np.arange(6 * 5 * 7 * 3, dtype=np.float64).reshape(6, 5, 7, 3) + 1.0
    C = E.circulant_embed(T.astype(np.complex128), n1, n2, n3)
    assert C.shape == (6, 6, 8, 4)
    # offset (i,j,k) lives at (i mod P)
    for (i, j, k) in [(0, 0, 0), (-2, 3, 1), (2, -3, -1), (-1, -1, -1)]:
        assert C[2, i % 6, j % 8, k % 4] == T[2, i + 2, j + 3, k + 1]
    # the wrap-around planes at index n are zero
    assert np.all(C[:, 3] == 0) and np.all(C[:, :, 4] == 0) and np.all(C[:, :, :, 2] == 0)


def test_spectrum_parity_of_green_components():
    """DFT of an even / odd circulant sequence is even / odd: Chat[P - k] = s Chat[k]."""
    n = 4
    T = K.toeplitz_tensor(n, n, n, 5e-3, K0)
    Ghat = E.green_spectra(T, n, n, n)
    P = 2 * n
    rev = (-np.arange(P)) % P
    for c, (a, b) in enumerate(K.COMPONENTS):
        for axis in range(3):
            s = (-1) ** ((a == axis) + (b == axis))
            flipped = np.take(Ghat[c], rev, axis=axis)
            assert np.allclose(flipped, s * Ghat[c], rtol=0, atol=1e-12 * np.abs(Ghat[c]).max())


def test_paper_memory_figure_pins_padded_size():
    """Section VI.A: 270 x 141 x 902 voxels, 60 unique PWL N components and 30 K
    components of the circulant forms take 245.6 and 122.8 GB (complex128), which
    holds for padded edges P_q = 2 n_q (tests/golden/paper_memory.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_memory.txt")
    rows = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            key, val = line.split("=")
            rows[key.strip()] = float(val)
    P = E.padded_shape(270, 141, 902)
    per_component = np.prod(P) * 16 / 2 ** 30
    assert abs(60 * per_component - rows["N_GB"]) < 0.05
    assert abs(30 * per_component - rows["K_GB"]) < 0.05


def test_system_operator_definition():
    rng = np.random.default_rng(2)
    n1, n2, n3 = 3, 3, 3
    T = K.toeplitz_tensor(n1, n2, n3, 5e-3, K0)
    G = M.dense_operator(T, n1, n2, n3)
    chi = _rand((n1, n2, n3), rng)
    w = _rand((3, n1, n2, n3), rng)
    Aw = M.apply_system(E.green_spectra(T, n1, n2, n3), chi, w)
    dense = w.ravel() - np.tile(chi.ravel(), 3) * (G @ w.ravel())
    assert np.allclose(Aw.ravel(), dense, rtol=0, atol=1e-12)


def test_matvec_at_sampled_voxels_equals_bruteforce():
    """The product at chosen voxels (kernel formed per output voxel) equals the
    brute-force BTTB product there: every voxel of two non-cubic grids, both
    self-term readings, a batch of two right-hand sides."""
    rng = np.random.default_rng(7)
    for n1, n2, n3 in ((3, 4, 5), (5, 2, 3)):
        J = _rand((2, 3, n1, n2, n3), rng)
        for mode in ("full", "pv"):
            T = K.toeplitz_tensor(n1, n2, n3, 5e-3, K0, mode)
            ref = M.matvec_bruteforce(T, J)
            vox = [(a, b, c) for a in range(n1) for b in range(n2) for c in range(n3)]
            got = M.matvec_at(J, 5e-3, K0, vox, mode)
            assert got.shape == (2, len(vox), 3)
            want = np.stack([ref[:, :, a, b, c] for a, b, c in vox], axis=1)
            assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
