"""Tucker+CP (Algorithm 2, eq. (17)), FP64.

Test infrastructure: see the package docstring.

Steps of Algorithm 2, in its order:
  * HOSVD of the tensor (Algorithm 1, ``hosvd.py``): A ~ G x1 U1 x2 U2 x3 U3.
  * A CP model of the core with r terms, G ~ sum_l V1[:, l] o V2[:, l] o V3[:, l]
    (o the outer product), fitted by alternating least squares, the method
    the paper names for this step.
  * Tucker+CP factors W^q = U^q V^q.
  * eq. (17): A~ = sum_l W1[:, l] o W2[:, l] o W3[:, l].

Readings where the paper is silent:
  * The rank r is given by the caller (the paper leaves the CP algorithm and
    its rank open; its Table II only names r).
  * ALS: a sweep updates V1, V2, V3 in turn, each as the linear least-squares
    problem with the other two fixed, on the mode-q unfolding of ``hosvd.py``
    and the Khatri-Rao product of the other two factors (numpy.linalg.lstsq).
    Sweeps stop when the relative error ||G - CP||_F / ||G||_F changes by less
    than ``tol`` between sweeps, or after ``max_iter`` sweeps.
  * Start: seeded complex normal factors (numpy default_rng(seed)).
"""
from __future__ import annotations

import numpy as np

from .hosvd import frobenius, hosvd, unfold


def cp_full(V) -> np.ndarray:
    """sum_l V1[:, l] o V2[:, l] o V3[:, l] as a dense 3-way array."""
    V1, V2, V3 = V
    return np.einsum("al,bl,cl->abc", V1, V2, V3)


def khatri_rao(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Column-wise Kronecker product: row x * len(Y) + y, column l = X[x, l] Y[y, l]."""
    return (X[:, None, :] * Y[None, :, :]).reshape(X.shape[0] * Y.shape[0], X.shape[1])


def _others(q: int):
    """The two modes other than q, in the column order of ``unfold(., q)``."""
    return [p for p in range(3) if p != q]


def cp_als(G: np.ndarray, r: int, tol: float = 1e-10, max_iter: int = 500, seed: int = 0):
    """CP model of ``G`` with ``r`` terms by ALS.

    Returns ([V1, V2, V3], history) where history[i] is the relative error
    ||G - CP||_F / ||G||_F after sweep i.
    """
    rng = np.random.default_rng(seed)
    V = [rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)) for n in G.shape]
    norm_G = frobenius(G)
    history = []
    for _ in range(max_iter):
        for q in range(3):
            x, y = _others(q)
            # G_(q) = V_q KR^T  =>  V_q^T = argmin ||KR X - G_(q)^T||
            KR = khatri_rao(V[x], V[y])
            Vt, *_ = np.linalg.lstsq(KR, unfold(G, q).T, rcond=None)
            V[q] = Vt.T
        err = frobenius(G - cp_full(V)) / norm_G
        history.append(err)
        if len(history) > 1 and abs(history[-2] - history[-1]) < tol:
            break
    return V, history


def tucker_cp(A: np.ndarray, tol_svd: float, r: int, rule: str = "tail", tol: float = 1e-10,
              max_iter: int = 500, seed: int = 0):
    """Algorithm 2 on a 3-way tensor.  Returns ([W1, W2, W3], core, [U1, U2, U3], history)."""
    core, U, _ = hosvd(A, tol_svd, rule)
    V, history = cp_als(core, r, tol, max_iter, seed)
    W = [U[q] @ V[q] for q in range(3)]
    return W, core, U, history


def cp_components(compressed, r: int, tol: float = 1e-10, max_iter: int = 500, seed: int = 0):
    """The CP step of Algorithm 2 on each of the six HOSVD cores ``compressed``
    (from ``hosvd.compress_components``): list of ([W1, W2, W3], history)."""
    out = []
    for c, (core, U, _) in enumerate(compressed):
        V, history = cp_als(core, r, tol, max_iter, seed + c)
        out.append(([U[q] @ V[q] for q in range(3)], history))
    return out


def rebuild_cp(W_list) -> np.ndarray:
    """eq. (17) for each component: [6, P1, P2, P3] from the Tucker+CP factors."""
    return np.stack([cp_full(W) for W in W_list])
