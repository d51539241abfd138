"""GPU parity of the Tucker+CP path (Algorithm 2, eq. (17)).

ALS from different starts reaches different (equally valid) CP models, so the
oracle does not rerun ALS and compare factors.  It checks what is unique:
  * the matvec and adjoint matvec with VIE_PATH_TUCKER_CP equal the oracle's
    FFT matvec with spectra rebuilt by eq. (17) from the exported factors
    W^q (FP32 gate 1e-5 relative L2);
  * the reported relative core error equals ||A~_Tucker - A~_CP||_F / ||core||_F
    computed from the exported Tucker and Tucker+CP factors (the U^q are
    orthonormal, so the two agree), to 1e-9;
  * a solve on the CP path meets its FP64 target against the Tucker operator.
Tolerances as in test_gpu_matvec.py.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as AD
from oracle import cp as CP
from oracle import hosvd as H
from oracle import matvec as M

vie = pytest.importorskip("paper_1811_00484_gb300")
pytestmark = pytest.mark.gpu

F = 298e6
HVOX = 5e-3


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


@pytest.mark.parametrize("n,tol,R", [((16, 16, 16), 1e-6, 8), ((16, 18, 32), 1e-4, 13),
                                     ((20, 9, 32), 1e-6, 32), ((6, 10, 48), 1e-6, 5)])
def test_cp_matvec_and_adjoint_equal_eq17_of_the_exported_factors(n, tol, R):
    op = vie.Operator(n, HVOX, F, tol)
    errs = op.tucker_cp(R, tol=1e-10, max_iter=200, seed=3)
    info = op.info()
    assert info["cp_rank"] == R and all(s >= 1 for s in info["cp_sweeps"])
    assert all(0.0 <= e < 1.0 for e in errs)
    W = [op.cp_export(c)[0] for c in range(6)]
    spectra = CP.rebuild_cp(W)
    J = rand_field(n, B=2, seed=21)
    y = host(op.matvec(dev(J), path="tucker_cp"))
    assert rel(y, M.matvec_fft(spectra, J)) <= 1e-5
    x = host(op.matvec_adjoint(dev(J[:1]), path="tucker_cp"))
    assert rel(x, AD.adjoint_matvec(spectra, J[:1])) <= 1e-5
    # the Tucker path of the same operator is untouched
    core, U, _ = op.export(0)
    tucker = np.stack([H.tucker_full(*op.export(c)[:2]) for c in range(6)])
    assert rel(host(op.matvec(dev(J))), M.matvec_fft(tucker, J)) <= 1e-5
    op.close()


def test_reported_cp_error_is_the_tucker_to_cp_distance():
    n = (16, 16, 16)
    op = vie.Operator(n, HVOX, F, 1e-6)
    errs = op.tucker_cp(6, tol=1e-12, max_iter=100, seed=1)
    for c in range(6):
        core, U, _ = op.export(c)
        W, err, sweeps = op.cp_export(c)
        assert err == errs[c] and 1 <= sweeps <= 100
        d = np.linalg.norm(H.tucker_full(core, U) - CP.cp_full(W)) / np.linalg.norm(core)
        assert abs(d - err) <= 1e-9 * max(err, 1e-3)
    op.close()


def test_cp_error_falls_with_rank_and_solve_meets_target():
    import workloads
    wl = workloads.make("solve", 16, seed=0, B=1, tol_svd=1e-6, incident="plane")
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd)
    e_lo = max(op.tucker_cp(2, tol=1e-12, max_iter=300, seed=2))
    e_hi = max(op.tucker_cp(24, tol=1e-12, max_iter=300, seed=2))
    assert e_hi < e_lo
    chi = dev(wl.chi, torch.complex128)
    einc = dev(wl.einc, torch.complex128)
    w, info = op.solve(chi, einc, tol=1e-8, path="tucker_cp")
    assert info["converged"]
    b = chi[None, None] * einc
    r = b - op.apply_system(chi, w)                # FP64, Tucker operator
    assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b)) <= 1e-8
    # a new model replaces the buffers the cached solver graphs read
    op.tucker_cp(16, tol=1e-12, max_iter=300, seed=5)
    w2, info2 = op.solve(chi, einc, tol=1e-8, path="tucker_cp")
    assert info2["converged"]
    r = b - op.apply_system(chi, w2)
    assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b)) <= 1e-8
    op.close()


def test_cp_path_errors():
    n = (16, 16, 16)
    op = vie.Operator(n, HVOX, F, 1e-6)
    J = dev(rand_field(n))
    with pytest.raises(vie.VieError):
        op.matvec(J, path="tucker_cp")             # no model yet
    for bad in (0, 33):
        with pytest.raises(vie.VieError):
            op.tucker_cp(bad)
    op.tucker_cp(4, max_iter=20)
    with pytest.raises(vie.VieError):
        op.matvec(dev(rand_field(n), torch.complex128), path="tucker_cp")   # FP32 model only
    op.close()
