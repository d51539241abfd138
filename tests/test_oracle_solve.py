"""Pins of the oracle's GMRES solve, adjoint and contrast gradient.

Checked against dense direct solves on tiny grids, the adjoint identity,
and FP64 central finite differences of the misfit.
"""
import numpy as np
import pytest

import workloads
from oracle import adjoint as AD
from oracle import embed as E
from oracle import gmres as GM
from oracle import kernel as K
from oracle import matvec as M

K0 = K.wavenumber(298e6)


def _rand(shape, rng):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _tiny(n=4, seed=5):
    wl = workloads.make("tiny", n, seed=seed, incident="plane")
    T = K.toeplitz_tensor(n, n, n, wl.h, K0)
    return wl, T, E.green_spectra(T, n, n, n), M.dense_operator(T, n, n, n)


def test_gmres_random_system():
    rng = np.random.default_rng(0)
    A = np.eye(60) * 4 + _rand((60, 60), rng) * 0.2
    b = _rand(60, rng)
    x, info = GM.gmres(lambda v: A @ v, b, tol=1e-13, restart=7, max_outer=200)
    assert info["converged"]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(x)


def test_gmres_zero_rhs():
    x, info = GM.gmres(lambda v: v, np.zeros(5, dtype=complex))
    assert info["converged"] and not np.any(x)


@pytest.mark.parametrize("restart", [50, 6])
def test_vie_solve_matches_dense(restart):
    wl, T, Ghat, G = _tiny()
    chi, e = wl.chi, wl.einc[0]
    w, info = GM.gmres(lambda v: M.apply_system(Ghat, chi, v), M.system_rhs(chi, e),
                       tol=1e-12, restart=restart, max_outer=400)
    assert info["converged"]
    N = chi.size
    A = np.eye(3 * N) - np.tile(chi.ravel(), 3)[:, None] * G
    w_ref = np.linalg.solve(A, (chi * e).ravel())
    assert np.linalg.norm(w.ravel() - w_ref) <= 1e-9 * np.linalg.norm(w_ref)


def test_adjoint_identity():
    rng = np.random.default_rng(4)
    n1, n2, n3 = 3, 4, 5
    Ghat = E.green_spectra(K.toeplitz_tensor(n1, n2, n3, 5e-3, K0), n1, n2, n3)
    x = _rand((3, n1, n2, n3), rng)
    y = _rand((3, n1, n2, n3), rng)
    lhs = np.vdot(M.matvec_fft(Ghat, x), y)
    rhs = np.vdot(x, AD.adjoint_matvec(Ghat, y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # complex symmetry y^T G x = x^T G y
    assert abs(np.sum(y * M.matvec_fft(Ghat, x)) - np.sum(x * M.matvec_fft(Ghat, y))) <= 1e-12 * abs(lhs)


def test_gradient_matches_dense_closed_form_and_finite_differences():
    wl, T, Ghat, G = _tiny(n=4, seed=9)
    rng = np.random.default_rng(11)
    chi, e = wl.chi, wl.einc[0]
    E_target = e + 0.3 * _rand(e.shape, rng)
    L, grad, finfo, ainfo = AD.gradient(Ghat, chi, e, E_target)
    L_d, grad_d = AD.dense_gradient(G, chi, e, E_target)
    assert abs(L - L_d) <= 1e-10 * abs(L_d)
    assert np.linalg.norm(grad - grad_d) <= 1e-8 * np.linalg.norm(grad_d)
    step = 1e-4
    for v in rng.choice(np.flatnonzero(wl.mask.ravel()), size=4, replace=False):
        idx = np.unravel_index(v, chi.shape)
        for part, unit in (("re", 1.0), ("im", 1j)):
            cp, cm = chi.copy(), chi.copy()
            cp[idx] += unit * step
            cm[idx] -= unit * step
            fd = (AD.loss_of_chi(Ghat, cp, e, E_target) - AD.loss_of_chi(Ghat, cm, e, E_target)) / (2 * step)
            an = grad[idx].real if part == "re" else grad[idx].imag
            assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-6 * np.abs(grad).max())


def _dense_fields(G, chi, einc, E_target):
    """w, E and the adjoint state lam of the dense system (numpy.linalg.solve only)."""
    N = chi.size
    chi3 = np.tile(chi.ravel(), 3)
    A = np.eye(3 * N) - chi3[:, None] * G
    e = einc.reshape(3 * N)
    w = np.linalg.solve(A, chi3 * e)
    E = e + G @ w
    lam = np.linalg.solve(A.conj().T, G.conj().T @ (E - E_target.reshape(3 * N)))
    return E, lam


def test_contrast_gradient_matches_finite_differences_of_the_dense_misfit():
    """contrast_gradient(lam, E) is dL/dRe chi + i dL/dIm chi (the adjoint-state
    gradient of the misfit, motivated in Section VII), for two incident fields
    whose gradients add: checked at every voxel of a 3x3x4 grid against central
    finite differences of the misfit computed with dense direct solves."""
    n1, n2, n3 = 3, 3, 4
    h = 5e-3
    rng = np.random.default_rng(21)
    T = K.toeplitz_tensor(n1, n2, n3, h, K0)
    G = M.dense_operator(T, n1, n2, n3)
    chi = rng.uniform(0.5, 2.0, (n1, n2, n3)) - 1j * rng.uniform(0.2, 1.0, (n1, n2, n3))
    einc = _rand((2, 3, n1, n2, n3), rng)
    E_t = _rand((2, 3, n1, n2, n3), rng)

    def loss(c):
        total = 0.0
        for b in range(2):
            E, _ = _dense_fields(G, c, einc[b], E_t[b])
            total += AD.misfit(E, E_t[b].reshape(-1))
        return total

    lam = np.zeros_like(einc)
    Ef = np.zeros_like(einc)
    for b in range(2):
        E, l_ = _dense_fields(G, chi, einc[b], E_t[b])
        Ef[b] = E.reshape(3, n1, n2, n3)
        lam[b] = l_.reshape(3, n1, n2, n3)
    g = AD.contrast_gradient(lam, Ef)
    assert g.shape == chi.shape
    step = 1e-6
    fd = np.zeros(chi.shape, dtype=np.complex128)
    for idx in np.ndindex(chi.shape):
        for unit in (1.0, 1j):
            cp, cm = chi.copy(), chi.copy()
            cp[idx] += unit * step
            cm[idx] -= unit * step
            d = (loss(cp) - loss(cm)) / (2 * step)
            fd[idx] += d if unit == 1.0 else 1j * d
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)
    # the single-field closed form of the dense reference agrees as well
    _, gd = AD.dense_gradient(G, chi, einc[0], E_t[0])
    assert np.linalg.norm(AD.contrast_gradient(lam[0], Ef[0]) - gd) <= 1e-10 * np.linalg.norm(gd)
