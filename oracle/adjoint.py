"""Adjoint operator and the contrast gradient of a field misfit, FP64.

Test infrastructure: see the package docstring.

The paper only motivates inverse problems (Section VII); these are the
plain definitions for the rescaled J-block system A(chi) w = chi e_inc with
A = I - M_chi G and total field E = e_inc + G w.

  * G is complex symmetric (T_ab = T_ba and T(-R) = T(R)), so
    G^H y = conj(G conj(y)), and A^H = I - G^H M_conj(chi).
  * Loss L = sum_{v,a} |E_va - E^t_va|^2.  With r = E - E^t, dE = G dw and
    A dw = dchi * E, so dL = 2 Re <lambda, dchi * E> where A^H lambda = G^H r.
    Hence dL/dRe chi_v = 2 Re s_v, dL/dIm chi_v = -2 Im s_v, with
    s_v = sum_a conj(lambda_va) E_va; as one complex number (PyTorch's
    convention for a real loss) grad_v = 2 sum_a lambda_va conj(E_va).
"""
from __future__ import annotations

import numpy as np

from . import gmres as _gmres
from .matvec import matvec_fft, system_rhs


def adjoint_matvec(Ghat, y):
    """G^H y = conj(G conj(y))."""
    return np.conj(matvec_fft(Ghat, np.conj(y)))


def apply_system_adjoint(Ghat, chi, lam):
    """A^H lam = lam - G^H (conj(chi) * lam)."""
    return lam - adjoint_matvec(Ghat, np.conj(chi) * lam)


def forward(Ghat, chi, einc, tol=1e-12, restart=50, max_outer=400):
    """Solve A w = chi e_inc by GMRES; return (w, E, info)."""
    b = system_rhs(chi, einc)
    w, info = _gmres.gmres(lambda v: v - chi * matvec_fft(Ghat, v), b, tol=tol,
                           restart=restart, max_outer=max_outer)
    return w, einc + matvec_fft(Ghat, w), info


def misfit(E, E_target) -> float:
    return float(np.sum(np.abs(E - E_target) ** 2))


def gradient(Ghat, chi, einc, E_target, tol=1e-12, restart=50, max_outer=400):
    """(loss, complex gradient [n1,n2,n3], forward info, adjoint info)."""
    w, E, finfo = forward(Ghat, chi, einc, tol, restart, max_outer)
    r = E - E_target
    rhs = adjoint_matvec(Ghat, r)
    lam, ainfo = _gmres.gmres(lambda v: apply_system_adjoint(Ghat, chi, v), rhs,
                              tol=tol, restart=restart, max_outer=max_outer)
    grad = 2.0 * np.sum(lam * np.conj(E), axis=-4)
    if grad.ndim == 4:          # batch of incident fields: gradients add
        grad = grad.sum(axis=0)
    return misfit(E, E_target), grad, finfo, ainfo


def contrast_gradient(lam, E, scale=2.0):
    """scale * sum over RHS and components of lam * conj(E) (per voxel)."""
    g = scale * np.sum(lam * np.conj(E), axis=-4)
    return g.sum(axis=0) if g.ndim == 4 else g


def loss_of_chi(Ghat, chi, einc, E_target, tol=1e-12):
    _, E, _ = forward(Ghat, chi, einc, tol)
    return misfit(E, E_target)


def dense_gradient(G, chi, einc, E_target):
    """Closed-form gradient with the dense 3N x 3N operator G (tiny grids)."""
    N = chi.size
    chi3 = np.tile(chi.ravel(), 3)
    A = np.eye(3 * N) - chi3[:, None] * G
    e = einc.reshape(3 * N)
    w = np.linalg.solve(A, chi3 * e)
    E = e + G @ w
    r = E - E_target.reshape(3 * N)
    lam = np.linalg.solve(A.conj().T, G.conj().T @ r)
    s = np.conj(lam) * E
    grad = 2.0 * np.conj(s.reshape(3, N).sum(axis=0))
    return misfit(E, E_target.reshape(3 * N)), grad.reshape(chi.shape)
