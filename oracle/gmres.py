"""Restarted GMRES (Section VI.C: inner 50 / outer 200 iterations), FP64.

Test infrastructure: see the package docstring.

Saad-Schultz GMRES(m): Arnoldi with modified Gram-Schmidt, the least-squares
problem on the Hessenberg matrix solved by Givens rotations, x0 = 0 unless
given, no preconditioner, stop when ||b - A x||_2 / ||b||_2 <= tol.  The
paper names the method and its settings only; any stable Arnoldi variant
gives the same solution, not the same iterates.
"""
from __future__ import annotations

import numpy as np


def _dot(u, v):
    return np.vdot(u, v)        # conj(u) . v


def gmres(apply_A, b, tol=1e-5, restart=50, max_outer=200, x0=None):
    """Solve A x = b.  Returns (x, info) with info = dict(iters, matvecs, relres, converged)."""
    shape = b.shape
    bv = b.ravel().astype(np.complex128)
    x = np.zeros_like(bv) if x0 is None else np.asarray(x0, dtype=np.complex128).ravel().copy()
    bnorm = np.linalg.norm(bv)
    info = {"iters": 0, "matvecs": 0, "relres": [], "converged": False}
    if bnorm == 0.0:
        info["converged"] = True
        return x.reshape(shape), info

    def A(v):
        info["matvecs"] += 1
        return apply_A(v.reshape(shape)).ravel()

    for _outer in range(max_outer):
        r = bv - A(x) if np.any(x) else bv.copy()
        beta = np.linalg.norm(r)
        info["relres"].append(beta / bnorm)
        if beta / bnorm <= tol:
            info["converged"] = True
            return x.reshape(shape), info
        m = restart
        V = np.zeros((m + 1, bv.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            w = A(V[k])
            for i in range(k + 1):                      # modified Gram-Schmidt
                H[i, k] = _dot(V[i], w)
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):                          # apply earlier rotations
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -np.conj(sn[i]) * H[i, k] + np.conj(cs[i]) * H[i + 1, k]
                H[i, k] = t
            # new rotation zeroing H[k+1, k]
            a, bb = H[k, k], H[k + 1, k]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if den == 0.0:
                cs[k], sn[k] = 1.0, 0.0
            else:
                cs[k] = np.conj(a) / den
                sn[k] = np.conj(bb) / den
            H[k, k] = cs[k] * a + sn[k] * bb
            H[k + 1, k] = 0.0
            g[k + 1] = -np.conj(sn[k]) * g[k]
            g[k] = cs[k] * g[k]
            info["iters"] += 1
            k_done = k + 1
            if abs(g[k + 1]) / bnorm <= tol or H[k, k] == 0.0:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + V[:k_done].T @ y
    r = bv - A(x)
    info["relres"].append(np.linalg.norm(r) / bnorm)
    info["converged"] = info["relres"][-1] <= tol
    return x.reshape(shape), info
