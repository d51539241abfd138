"""Circulant embedding and DFT of the defining tensors (Sections II.B, V.A), FP64.

Test infrastructure: see the package docstring.

A BTTB matrix with defining tensor T[i, j, k], |i| < n1, |j| < n2, |k| < n3,
is the top-left block of a block-circulant matrix of size P1 P2 P3 with
P_q = 2 n_q, whose generating tensor C holds T at indices taken modulo P_q.
The wrap-around entries with an index equal to n_q are never reached by a
product on the n1 x n2 x n3 grid; the paper does not say what they hold, and
they are set to zero here (they change the spectrum, and so the Tucker ranks,
but not the cropped product).
"""
from __future__ import annotations

import numpy as np


def padded_shape(n1: int, n2: int, n3: int):
    return (2 * n1, 2 * n2, 2 * n3)


def circulant_embed(T: np.ndarray, n1: int, n2: int, n3: int) -> np.ndarray:
    """C[i mod P1, j mod P2, k mod P3] = T[i, j, k]; entries with an index n_q are 0.

    ``T`` has shape [..., 2 n1 - 1, 2 n2 - 1, 2 n3 - 1] (offset + n - 1 indexing).
    """
    P1, P2, P3 = padded_shape(n1, n2, n3)
    lead = T.shape[:-3]
    C = np.zeros(lead + (P1, P2, P3), dtype=np.complex128)
    i = np.arange(-(n1 - 1), n1) % P1
    j = np.arange(-(n2 - 1), n2) % P2
    k = np.arange(-(n3 - 1), n3) % P3
    C[..., i[:, None, None], j[None, :, None], k[None, None, :]] = T
    return C


def spectrum(C: np.ndarray) -> np.ndarray:
    """Unnormalised forward 3-D DFT over the last three axes (exp(-2 pi i kappa x / P))."""
    return np.fft.fftn(C, axes=(-3, -2, -1))


def green_spectra(T: np.ndarray, n1: int, n2: int, n3: int) -> np.ndarray:
    """Embedding followed by the DFT: the six FFT'd circulant components."""
    return spectrum(circulant_embed(T, n1, n2, n3))
