"""Pins of the factor-wise embedding and DFT (Section V.A) against what the
mathematics fixes: with full ranks it reproduces the spectrum of the whole
embedded tensor exactly; the unfolding singular values of the spectrum are
those of the Toeplitz tensor scaled by sqrt(P1 P2 P3) (Parseval), so the
HOSVD ranks agree; and the truncated model meets eq. (12)'s bound on the
spectrum."""
import math

import numpy as np
import pytest

from oracle import embed as E
from oracle import factorwise as FW
from oracle import hosvd as H
from oracle import kernel as K

H_VOX, F = 5e-3, 298e6


@pytest.mark.parametrize("n", [(3, 4, 5), (6, 5, 7)])
def test_full_rank_reproduces_the_spectrum(n):
    T = K.toeplitz_tensor(*n, H_VOX, K.wavenumber(F))
    Ghat = E.green_spectra(T, *n)
    for c in (0, 1, 5):
        core, Uhat, _ = FW.factorwise_tucker(T[c], 1e-15)
        A = H.tucker_full(core, Uhat)
        assert np.linalg.norm(A - Ghat[c]) <= 1e-12 * np.linalg.norm(Ghat[c])


def test_singular_values_scale_and_ranks_agree():
    n = (6, 5, 7)
    P = [2 * v for v in n]
    T = K.toeplitz_tensor(*n, H_VOX, K.wavenumber(F))
    Ghat = E.green_spectra(T, *n)
    scale = math.sqrt(P[0] * P[1] * P[2])
    for c in range(6):
        for q in range(3):
            sT = np.linalg.svd(H.unfold(T[c], q), compute_uv=False)
            sC = np.linalg.svd(H.unfold(Ghat[c], q), compute_uv=False)[: sT.size]
            assert np.allclose(sC, scale * sT, rtol=0, atol=1e-10 * scale * sT[0])
        for tol in (1e-3, 1e-6):
            _, U_fw, _ = FW.factorwise_tucker(T[c], tol)
            _, U_c, _ = H.hosvd(Ghat[c], tol)
            assert [u.shape[1] for u in U_fw] == [u.shape[1] for u in U_c]


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_truncated_model_meets_the_bound_on_the_spectrum(tol):
    n = (6, 5, 7)
    T = K.toeplitz_tensor(*n, H_VOX, K.wavenumber(F))
    Ghat = E.green_spectra(T, *n)
    for c in range(6):
        core, Uhat, _ = FW.factorwise_tucker(T[c], tol)
        err = np.linalg.norm(H.tucker_full(core, Uhat) - Ghat[c])
        assert err <= tol * np.linalg.norm(Ghat[c]) * (1 + 1e-9)


def test_a_misplaced_embedding_row_is_caught():
    """A plausible indexing slip (negative offsets shifted by one row) breaks the
    exactness pin, so the pin above does test the embedding."""
    n = (3, 4, 5)
    T = K.toeplitz_tensor(*n, H_VOX, K.wavenumber(F))
    Ghat = E.green_spectra(T, *n)
    core, U, _ = H.hosvd(T[0], 1e-15)

    def wrong(Uq, m):
        out = np.zeros((2 * m, Uq.shape[1]), dtype=np.complex128)
        out[np.arange(-(m - 1), m) % (2 * m - 1)] = Uq
        return np.fft.fft(out, axis=0)

    A = H.tucker_full(core, [wrong(U[q], n[q]) for q in range(3)])
    assert np.linalg.norm(A - Ghat[0]) > 1e-3 * np.linalg.norm(Ghat[0])
