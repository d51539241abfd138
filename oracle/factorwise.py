"""Circulant embedding and DFT applied to the Tucker factors (Section V.A), FP64.

Test infrastructure: see the package docstring.

The embedding and the 3-D DFT act on each mode separately.  With E_q the
P_q x (2 n_q - 1) matrix that puts offset i in row i mod P_q (row n_q stays
zero) and F_q the P_q-point DFT matrix,
    C = T x1 E1 x2 E2 x3 E3,      C^ = C x1 F1 x2 F2 x3 F3,
so a Tucker model T ~ G x1 U1 x2 U2 x3 U3 of the Toeplitz defining tensor
gives C^ ~ G x1 (F1 E1 U1) x2 (F2 E2 U2) x3 (F3 E3 U3): one DFT per factor
column instead of one 3-D DFT of the P1 x P2 x P3 tensor.  F_q E_q has
orthogonal columns of norm sqrt(P_q), so the unfolding singular values of C^
are those of T times sqrt(P1 P2 P3), and truncation at a tolerance relative
to the tensor's own norm keeps the same ranks.
"""
from __future__ import annotations

import numpy as np

from .hosvd import hosvd


def embed_rows(U: np.ndarray, n: int) -> np.ndarray:
    """E U: row i + n - 1 of U (offset i, |i| < n) moves to row i mod 2n; row n is zero."""
    P = 2 * n
    out = np.zeros((P, U.shape[1]), dtype=np.complex128)
    out[np.arange(-(n - 1), n) % P] = U
    return out


def factor_spectrum(U: np.ndarray, n: int) -> np.ndarray:
    """F E U: the unnormalised forward DFT of every embedded factor column."""
    return np.fft.fft(embed_rows(U, n), axis=0)


def factorwise_tucker(T: np.ndarray, tol: float, rule: str = "tail"):
    """HOSVD (Algorithm 1) of one Toeplitz defining tensor [2n1-1, 2n2-1, 2n3-1],
    then the embedding and DFT of its factors.  Returns (core, [U1^, U2^, U3^],
    sigmas of T's unfoldings); tucker_full(core, U^) approximates the spectrum."""
    core, U, sigmas = hosvd(T, tol, rule)
    Uhat = [factor_spectrum(U[q], (T.shape[q] + 1) // 2) for q in range(3)]
    return core, Uhat, sigmas
