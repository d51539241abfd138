"""BTTB matrix-vector product of the J-block operator, FP64.

Test infrastructure: see the package docstring.

The product of Section II.B: (G J)_a[m] = sum_b sum_{m'} T_ab[m - m'] J_b[m']
over the n1 x n2 x n3 grid, for the symmetric dyad T_ab (six unique
components).  It is computed two ways:
  * ``matvec_bruteforce``  - the definition itself, O(N^2), for tiny grids;
  * ``matvec_fft``         - zero-pad to (2 n1, 2 n2, 2 n3), 3-D DFT, multiply
                             voxel by voxel with the FFT'd circulant components,
                             inverse DFT, crop (Section V.B, the "traditional"
                             FFT-based product);
  * ``matvec_at``          - the definition evaluated only at chosen output
                             voxels, with the kernel formed on the fly, for
                             grids too large for the other two.
The system operator of the J-block of eq. (4), rescaled to w = j / c_e, is
  A w = w - chi * (G w),   right-hand side  chi * e_inc.
"""
from __future__ import annotations

import numpy as np

from .kernel import COMPONENTS, component_index, dyadic, self_term


def _as_batch(J):
    J = np.asarray(J)
    return (J[None], True) if J.ndim == 4 else (J, False)


def matvec_bruteforce(T: np.ndarray, J: np.ndarray) -> np.ndarray:
    """Plain BTTB product from the defining tensors T [6, 2n1-1, 2n2-1, 2n3-1]."""
    Jb, single = _as_batch(J)
    B, _, n1, n2, n3 = Jb.shape
    Y = np.zeros(Jb.shape, dtype=np.complex128)
    for m1 in range(n1):
        for m2 in range(n2):
            for m3 in range(n3):
                # entry at m' is T[m - m'], i.e. the offset window reversed
                W = T[:, m1:m1 + n1, m2:m2 + n2, m3:m3 + n3][:, ::-1, ::-1, ::-1]
                for a in range(3):
                    acc = np.zeros(B, dtype=np.complex128)
                    for b in range(3):
                        acc += np.sum(W[component_index(a, b)] * Jb[:, b], axis=(1, 2, 3))
                    Y[:, a, m1, m2, m3] = acc
    return Y[0] if single else Y


def pad(J: np.ndarray, P) -> np.ndarray:
    out = np.zeros(J.shape[:-3] + tuple(P), dtype=np.complex128)
    n1, n2, n3 = J.shape[-3:]
    out[..., :n1, :n2, :n3] = J
    return out


def product(Ghat, Jhat):
    """Yhat_a = sum_b Ghat_ab * Jhat_b with Ghat given as its six unique components."""
    Yhat = np.zeros_like(Jhat)
    for a in range(3):
        for b in range(3):
            Yhat[..., a, :, :, :] += Ghat[component_index(a, b)] * Jhat[..., b, :, :, :]
    return Yhat


def matvec_fft(Ghat: np.ndarray, J: np.ndarray) -> np.ndarray:
    """FFT-based product with the six spectra Ghat [6, P1, P2, P3] (exact or rebuilt)."""
    Jb, single = _as_batch(J)
    n1, n2, n3 = Jb.shape[-3:]
    P = Ghat.shape[-3:]
    Jhat = np.fft.fftn(pad(Jb, P), axes=(-3, -2, -1))
    Y = np.fft.ifftn(product(Ghat, Jhat), axes=(-3, -2, -1))[..., :n1, :n2, :n3]
    return Y[0] if single else Y


def apply_system(Ghat: np.ndarray, chi: np.ndarray, w: np.ndarray) -> np.ndarray:
    """A w = w - chi * (G w): J-block of eq. (4) with mu_r = 1, w = j / c_e."""
    return w - chi * matvec_fft(Ghat, w)


def system_rhs(chi: np.ndarray, einc: np.ndarray) -> np.ndarray:
    """Right-hand side chi * e_inc of the rescaled J-block equation."""
    return chi * einc


def total_field(Ghat: np.ndarray, einc: np.ndarray, w: np.ndarray) -> np.ndarray:
    """E = e_inc + G w."""
    return einc + matvec_fft(Ghat, w)


def dense_operator(T: np.ndarray, n1: int, n2: int, n3: int) -> np.ndarray:
    """The 3N x 3N BTTB matrix G (N = n1 n2 n3) in [a][m] ordering, for tiny grids."""
    N = n1 * n2 * n3
    G = np.zeros((3 * N, 3 * N), dtype=np.complex128)
    m = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3),
                             indexing="ij"), axis=-1).reshape(N, 3)
    d = m[:, None, :] - m[None, :, :]              # m - m'
    idx = (d[..., 0] + n1 - 1, d[..., 1] + n2 - 1, d[..., 2] + n3 - 1)
    for a in range(3):
        for b in range(3):
            G[a * N:(a + 1) * N, b * N:(b + 1) * N] = T[component_index(a, b)][idx]
    return G


def matvec_at(J: np.ndarray, h: float, k0: float, voxels, self_mode: str = "full") -> np.ndarray:
    """(G J)_a[m] = sum_b sum_{m'} T_ab[m - m'] J_b[m'] at the output voxels m in
    ``voxels`` (index triples), for every right-hand side of J [B, 3, n1, n2, n3]
    (or [3, n1, n2, n3]).  T_ab[r] is h^3 times the dyadic kernel at offset r h,
    and the self term at r = 0 (the entries of kernel.toeplitz_tensor), formed
    here only for the offsets one output voxel needs.  Returns [B, S, 3]
    (or [S, 3])."""
    Jb, single = _as_batch(J)
    n1, n2, n3 = Jb.shape[-3:]
    i, j, k = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    out = np.zeros((Jb.shape[0], len(voxels), 3), dtype=np.complex128)
    for s_, m in enumerate(voxels):
        m = tuple(int(v) for v in m)
        R = np.stack([(m[0] - i) * h, (m[1] - j) * h, (m[2] - k) * h], axis=-1)
        R[m] = (1.0, 0.0, 0.0)                 # placeholder for the zero offset
        T = dyadic(R, k0) * h ** 3
        st = self_term(h, k0, self_mode)
        for c, (a, b) in enumerate(COMPONENTS):
            T[(c,) + m] = st if a == b else 0.0
        for a in range(3):
            for b in range(3):
                Tab = T[component_index(a, b)].ravel()
                out[:, s_, a] += Jb[:, b].reshape(Jb.shape[0], -1) @ Tab
    return out[0] if single else out
