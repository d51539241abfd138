"""GPU parity of the length-512 FFT kernels (256-voxel grid edges, P = 512)
against the FP64 CPU oracle.

The x / y line stages and the fused z stage of that length are three-pass
radix-8 kernels of their own.  Thin grids put the 256-voxel edge on one axis
at a time (x stage, y stage with a ragged 9-column tile, fused z stage on the
Tucker and stored paths), and one grid on two axes; the system operator with
the contrast (prologue / epilogue flags of the line kernels) and a small
refined solve (the per-right-hand-side scale factors of the Krylov basis) run
through the same kernels.  Tolerance: the FP32 matvec gate of 1e-5 relative
L2 against the oracle's own HOSVD of the same spectra (1e-5 + 4 tol against
the exact spectra on the stored path).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import adjoint as AD
from oracle import embed as E
from oracle import hosvd as H
from oracle import kernel as K
from oracle import matvec as M

vie = pytest.importorskip("paper_1811_00484_gb300")
pytestmark = pytest.mark.gpu

F = 298e6
HVOX = 5e-3
K0 = K.wavenumber(F)
TOL = 1e-6


def dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rand_field(n, B=1, seed=0):
    rng = np.random.default_rng(seed)
    shape = (B, 3) + tuple(n)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


_cache = {}


def setup_case(n):
    if n not in _cache:
        Ghat = E.green_spectra(K.toeplitz_tensor(*n, HVOX, K0), *n)
        rebuilt = H.rebuild_components(H.compress_components(Ghat, TOL))
        op = vie.Operator(n, HVOX, F, TOL, store_uncompressed=True)
        _cache[n] = (Ghat, rebuilt, op)
    return _cache[n]


@pytest.mark.parametrize("n", [(256, 3, 5), (5, 256, 9), (3, 4, 256), (256, 5, 256)])
def test_length512_matvec_paths_and_adjoint(n):
    Ghat, rebuilt, op = setup_case(n)
    J = rand_field(n, B=3, seed=21)
    assert rel(host(op.matvec(dev(J))), M.matvec_fft(rebuilt, J)) <= 1e-5
    exact = M.matvec_fft(Ghat, J)
    assert rel(host(op.matvec(dev(J), path="uncompressed")), exact) <= 1e-5
    y = rand_field(n, B=1, seed=22)
    assert rel(host(op.matvec_adjoint(dev(y))), AD.adjoint_matvec(rebuilt, y)) <= 1e-5
    # FP64 path of the same grid (refinement residuals) for reference
    assert rel(host(op.matvec(dev(J, torch.complex128))), M.matvec_fft(rebuilt, J)) <= 1e-11


@pytest.mark.parametrize("n", [(256, 4, 6), (6, 4, 256)])
def test_length512_system_operator(n):
    Ghat, rebuilt, op = setup_case(n)
    wl = workloads.make("t512", n, seed=23, incident="plane")
    w = rand_field(n, B=2, seed=24)
    got = host(op.apply_system(dev(wl.chi), dev(w)))
    assert rel(got, M.apply_system(rebuilt, wl.chi, w)) <= 1e-5
    goth = host(op.apply_system(dev(wl.chi), dev(w), adjoint=True))
    assert rel(goth, AD.apply_system_adjoint(rebuilt, wl.chi, w)) <= 1e-5


def test_length512_refined_solve():
    n = (256, 4, 6)
    Ghat, rebuilt, op = setup_case(n)
    wl = workloads.make("t512s", n, seed=25, incident="plane")
    chi = dev(wl.chi, torch.complex128)
    einc = dev(np.concatenate([wl.einc, 0.5 * wl.einc], axis=0), torch.complex128)
    w, info = op.solve(chi, einc, tol=1e-9)
    assert info["converged"]
    wn = host(w)
    for b in range(2):
        e = wl.einc[0] * (1.0 if b == 0 else 0.5)
        rhs = M.system_rhs(wl.chi, e)
        r = rhs - M.apply_system(rebuilt, wl.chi, wn[b])
        assert np.linalg.norm(r) <= 2e-9 * np.linalg.norm(rhs)
