"""Pins of the oracle's truncated HOSVD (Algorithm 1, eqs. (12)-(16)).

Checked against: orthonormality, exact recovery at full rank, the
De Lathauwer truncation bound that underlies eq. (16), recovery of a known
multilinear rank, reduction to the truncated matrix SVD when one mode has
size 1, and the prescribed accuracy of eq. (12) on the Green's spectra.
"""
import math

import numpy as np
import pytest

from oracle import embed as E
from oracle import hosvd as H
from oracle import kernel as K

K0 = K.wavenumber(298e6)


def _rand(shape, rng):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _orth(n, r, rng):
    q, _ = np.linalg.qr(_rand((n, r), rng))
    return q


def test_factors_orthonormal_and_full_rank_exact():
    rng = np.random.default_rng(0)
    A = _rand((5, 6, 7), rng)
    core, U, _ = H.hosvd(A, tol=0.0)
    assert core.shape == (5, 6, 7)
    for u in U:
        assert np.allclose(u.conj().T @ u, np.eye(u.shape[1]), atol=1e-13)
    assert np.linalg.norm(H.tucker_full(core, U) - A) <= 1e-13 * np.linalg.norm(A)


def test_known_multilinear_rank_is_recovered():
    rng = np.random.default_rng(1)
    ranks = (3, 2, 4)
    G = _rand(ranks, rng)
    U = [_orth(n, r, rng) for n, r in zip((9, 8, 10), ranks)]
    # independent construction of the tensor: one einsum with the three factors
    A = np.einsum("abc,ia,jb,kc->ijk", G, U[0], U[1], U[2])
    A = A + 1e-10 * _rand(A.shape, rng)
    core, F, _ = H.hosvd(A, tol=1e-6)
    assert tuple(core.shape) == ranks
    assert np.linalg.norm(H.tucker_full(core, F) - A) <= 1e-9 * np.linalg.norm(A)


def test_single_slice_reduces_to_truncated_svd():
    rng = np.random.default_rng(2)
    M = _rand((12, 9), rng) @ np.diag(np.logspace(0, -8, 9)) @ _orth(9, 9, rng).conj().T
    A = M[:, :, None]
    core, F, _ = H.hosvd(A, tol=1e-4, rule="sigma_max")
    u, s, vh = np.linalg.svd(M, full_matrices=False)
    r = core.shape[0]
    assert core.shape[1] == r and core.shape[2] == 1
    ref = (u[:, :r] * s[:r]) @ vh[:r]
    assert np.linalg.norm(H.tucker_full(core, F)[:, :, 0] - ref) <= 1e-12 * np.linalg.norm(M)
    assert r == int(np.count_nonzero(s >= 1e-4 / math.sqrt(3) * s[0]))


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_truncation_bound(tol):
    rng = np.random.default_rng(3)
    # graded tensor so that truncation really happens
    A = np.einsum("abc,ia,jb,kc->ijk", _rand((8, 8, 8), rng) * np.logspace(0, -6, 8)[:, None, None],
                  _orth(10, 8, rng), _orth(11, 8, rng), _orth(12, 8, rng))
    core, U, sig = H.hosvd(A, tol=tol)
    err2 = np.linalg.norm(H.tucker_full(core, U) - A) ** 2
    discarded = sum(np.sum(s[u.shape[1]:] ** 2) for s, u in zip(sig, U))
    assert err2 <= discarded * (1 + 1e-10) + (1e-13 * np.linalg.norm(A)) ** 2
    assert math.sqrt(err2) <= tol * np.linalg.norm(A) * (1 + 1e-10)


@pytest.mark.parametrize("n,tol", [(4, 1e-8), (6, 1e-6), (8, 1e-8)])
def test_green_spectra_meet_prescribed_accuracy(n, tol):
    T = K.toeplitz_tensor(n, n, n, 5e-3, K0)
    Ghat = E.green_spectra(T, n, n, n)
    comp = H.compress_components(Ghat, tol)
    Gt = H.rebuild_components(comp)
    for c in range(6):
        assert np.linalg.norm(Gt[c] - Ghat[c]) <= tol * np.linalg.norm(Ghat[c])
        assert all(u.shape[1] <= 2 * n for u in comp[c][1])


def test_error_falls_with_tolerance():
    """Section VI.C: the HOSVD error decreases (roughly linearly) with the tolerance."""
    n = 16
    Ghat = E.green_spectra(K.toeplitz_tensor(n, n, n, 5e-3, K0), n, n, n)
    errs = []
    for tol in (1e-2, 1e-4, 1e-6, 1e-8):
        core, U, _ = H.hosvd(Ghat[0], tol)
        errs.append(np.linalg.norm(H.tucker_full(core, U) - Ghat[0]) / np.linalg.norm(Ghat[0]))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert all(e <= t for e, t in zip(errs, (1e-2, 1e-4, 1e-6, 1e-8)))


def test_rank_rules():
    s = np.array([10.0, 1.0, 1e-3, 1e-6, 1e-9])
    nrm = float(np.sqrt(np.sum(s ** 2)))
    # sigma_max rule: keep s >= tol/sqrt(3) * s_max
    assert H.truncation_rank(s, 1e-4 * math.sqrt(3), nrm, "sigma_max") == 3
    # tail rule: smallest r with sqrt(sum_{j>r} s^2) <= tol/sqrt(3) ||A||
    r = H.truncation_rank(s, 1e-5, nrm, "tail")
    tails = [math.sqrt(np.sum(s[k:] ** 2)) for k in range(1, 6)] + [0.0]
    bound = 1e-5 / math.sqrt(3) * nrm
    assert r == min(k for k in range(1, 6) if (tails[k - 1] if k < 5 else 0.0) <= bound)
    assert H.truncation_rank(np.zeros(4), 1e-6, 0.0) == 1


def test_mode_product_definition_a3():
    """Definition A.3 on a case small enough to write out by hand."""
    A = np.arange(8, dtype=np.complex128).reshape(2, 2, 2)
    M = np.array([[1.0, 2.0]], dtype=np.complex128)            # 1 x 2
    B = H.mode_product(A, M, 1)                                 # sums over the 2nd index
    assert B.shape == (2, 1, 2)
    assert B[1, 0, 1] == A[1, 0, 1] * 1 + A[1, 1, 1] * 2        # 5 + 2*7
    assert B[1, 0, 1] == 19
