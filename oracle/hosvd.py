"""Truncated HOSVD (Algorithm 1) and the Tucker model (eqs. (13)-(14)), FP64.

Test infrastructure: see the package docstring.

Definitions followed:
  * Frobenius norm, Definition A.2.
  * n-mode product, Definition A.3: (A x_q M)[.., i, ..] = sum_t A[.., t, ..] M[i, t].
  * mode-q unfolding (Fig. 2): rows indexed by the q-th index, columns by the
    other two (their order does not change the left singular vectors).
  * Algorithm 1: SVD of each unfolding, truncation to rank r_q, factors U^q =
    the first r_q left singular vectors, core = A x1 U1^* x2 U2^* x3 U3^*
    (^* the conjugate transpose, Table I).
  * eq. (13)/(14): A~ = core x1 U1 x2 U2 x3 U3.

The truncation rule printed with Algorithm 1 is garbled ("sigma_{r_i} <
eps / sqrt(3) sigma_max").  Two readings are provided:
  * ``rule='tail'`` (default): the smallest r_q whose discarded tail obeys
    sqrt(sum_{j > r_q} sigma_j^2) <= (eps / sqrt(3)) ||A||_F.  Summed over the
    three modes this guarantees ||A - A~||_F <= eps ||A||_F, the prescribed
    accuracy of eq. (12) taken relative to the component's own norm.
  * ``rule='sigma_max'``: keep every sigma_j >= (eps / sqrt(3)) sigma_max.
A tail (or singular value) exactly at the threshold is discarded under
'tail' and kept under 'sigma_max'.  The rank is at least 1.
"""
from __future__ import annotations

import math

import numpy as np


def frobenius(A: np.ndarray) -> float:
    """Definition A.2."""
    return float(np.sqrt(np.sum(np.abs(A) ** 2)))


def unfold(A: np.ndarray, q: int) -> np.ndarray:
    """Mode-q unfolding A^(q) in C^{n_q x (product of the other two)}."""
    return np.moveaxis(A, q, 0).reshape(A.shape[q], -1)


def mode_product(A: np.ndarray, M: np.ndarray, q: int) -> np.ndarray:
    """Definition A.3: B = A x_q M, B[.., i, ..] = sum_t A[.., t, ..] M[i, t]."""
    return np.moveaxis(np.tensordot(M, A, axes=(1, q)), 0, q)


def truncation_rank(s: np.ndarray, tol: float, norm_A: float, rule: str = "tail") -> int:
    """Rank kept from the singular values ``s`` (descending) of one unfolding."""
    s = np.asarray(s, dtype=np.float64)
    if s.size == 0 or s[0] == 0.0:
        return 1
    if rule == "tail":
        bound = (tol / math.sqrt(3.0)) * norm_A
        tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])   # tail[r] = sqrt(sum_{j >= r} s_j^2)
        for r in range(1, s.size + 1):
            t = tail[r] if r < s.size else 0.0
            if t <= bound:
                return r
        return s.size
    if rule == "sigma_max":
        thr = (tol / math.sqrt(3.0)) * s[0]
        return max(1, int(np.count_nonzero(s >= thr)))
    raise ValueError(rule)


def hosvd(A: np.ndarray, tol: float, rule: str = "tail"):
    """Algorithm 1 on a 3-way tensor.  Returns (core, [U1, U2, U3], [s1, s2, s3])."""
    norm_A = frobenius(A)
    factors, sigmas = [], []
    for q in range(3):
        U, s, _ = np.linalg.svd(unfold(A, q), full_matrices=False)
        r = truncation_rank(s, tol, norm_A, rule)
        factors.append(U[:, :r].copy())
        sigmas.append(s)
    core = A
    for q in range(3):
        core = mode_product(core, factors[q].conj().T, q)
    return core, factors, sigmas


def tucker_full(core: np.ndarray, factors) -> np.ndarray:
    """eq. (14): A~ = core x1 U1 x2 U2 x3 U3."""
    A = core
    for q in range(3):
        A = mode_product(A, factors[q], q)
    return A


def compress_components(Ghat: np.ndarray, tol: float, rule: str = "tail"):
    """HOSVD of each of the six FFT'd components ("each component", Section V.B)."""
    return [hosvd(Ghat[c], tol, rule) for c in range(Ghat.shape[0])]


def rebuild_components(compressed) -> np.ndarray:
    """The six rebuilt spectra A~_c as one array [6, P1, P2, P3]."""
    return np.stack([tucker_full(core, U) for core, U, _ in compressed])
