"""Pins of the Tucker+CP oracle (Algorithm 2, eq. (17)) against what the
mathematics fixes, independent of the oracle's own formulas:

  * a tensor built from r planted rank-one terms is recovered exactly (the
    CP model of a generic rank-r tensor is unique, so ALS reaches zero error);
  * every ALS sweep solves least-squares problems, so the error never grows;
  * with a trailing mode of size 1 the tensor is a matrix, and the best
    rank-r CP model is the truncated SVD (Eckart-Young): ALS reaches its
    error sqrt(sum_{j >= r} sigma_j^2);
  * step 4 of Algorithm 2: sum_l (U1 V1)_l o (U2 V2)_l o (U3 V3)_l equals the
    Tucker model of the CP core, for any factors;
  * the HOSVD factors have orthonormal columns, so the Tucker+CP error against
    the Tucker model equals the CP error on the core (an isometry), on a
    Green's component.
"""
import numpy as np
import pytest

from oracle import cp as CP
from oracle import embed as E
from oracle import hosvd as H
from oracle import kernel as K


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_planted_rank_is_recovered():
    rng = np.random.default_rng(7)
    V = [crandn(rng, n, 3) for n in (6, 7, 8)]
    G = CP.cp_full(V)
    W, hist = CP.cp_als(G, 3, tol=1e-15, max_iter=3000, seed=1)
    assert hist[-1] < 1e-9
    assert np.linalg.norm(CP.cp_full(W) - G) <= 1e-9 * np.linalg.norm(G)


def test_als_error_never_grows():
    rng = np.random.default_rng(3)
    G = crandn(rng, 7, 6, 5)
    _, hist = CP.cp_als(G, 4, tol=0.0, max_iter=60, seed=2)
    assert len(hist) == 60
    assert all(b <= a * (1 + 1e-12) + 1e-15 for a, b in zip(hist, hist[1:]))


@pytest.mark.parametrize("r", [1, 2, 4])
def test_matrix_case_reaches_eckart_young(r):
    rng = np.random.default_rng(11)
    M = crandn(rng, 9, 7)
    s = np.linalg.svd(M, compute_uv=False)
    best = np.sqrt(np.sum(s[r:] ** 2)) / np.linalg.norm(M)
    _, hist = CP.cp_als(M[:, :, None], r, tol=1e-16, max_iter=4000, seed=5)
    assert abs(hist[-1] - best) <= 1e-8
    assert hist[-1] >= best * (1 - 1e-10)       # never better than the optimum


def test_rank_one_is_exact():
    rng = np.random.default_rng(5)
    V = [crandn(rng, n, 1) for n in (4, 5, 3)]
    G = CP.cp_full(V)
    _, hist = CP.cp_als(G, 1, tol=1e-15, max_iter=200, seed=9)
    assert hist[-1] < 1e-12


def test_step_four_identity():
    rng = np.random.default_rng(13)
    U = [crandn(rng, p, n) for p, n in ((10, 4), (9, 5), (8, 3))]
    V = [crandn(rng, n, 6) for n in (4, 5, 3)]
    W = [U[q] @ V[q] for q in range(3)]
    lhs = CP.cp_full(W)
    rhs = H.tucker_full(CP.cp_full(V), U)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)


def test_tucker_cp_error_equals_core_error_on_a_green_component():
    n = (6, 5, 7)
    h, f = 5e-3, 298e6
    Ghat = E.green_spectra(K.toeplitz_tensor(*n, h, K.wavenumber(f)), *n)
    A = Ghat[1]                                   # xy
    W, core, U, hist = CP.tucker_cp(A, 1e-6, 8, max_iter=300, seed=4)
    At = H.tucker_full(core, U)
    Acp = CP.cp_full(W)
    V_err = hist[-1] * np.linalg.norm(core)
    assert abs(np.linalg.norm(At - Acp) - V_err) <= 1e-10 * np.linalg.norm(core)
    # triangle inequality against the uncompressed spectrum
    assert np.linalg.norm(A - Acp) <= np.linalg.norm(A - At) + V_err + 1e-12 * np.linalg.norm(A)
