"""Several grids through one launch per stage (vie_matvec_multi) and the autotuner.

The multi-grid kernels run the same device bodies as the per-operator ones,
so their outputs must agree with vie_matvec to rounding (1e-6 relative) and
with the oracle to the matvec gate (1e-5).  The autotuner only changes CTA
sizes: results after tuning agree with those before to 1e-6.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import embed as E
from oracle import hosvd as H
from oracle import kernel as K
from oracle import matvec as M

vie = pytest.importorskip("paper_1811_00484_gb300")
pytestmark = pytest.mark.gpu


def field(n, B, seed):
    rng = np.random.default_rng(seed)
    shape = (B, 3) + tuple(n)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()


def rel_t(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_multi_grid_matvec_matches_single_and_oracle():
    ns = [(16, 16, 16), (32, 32, 32), (48, 16, 32)]
    Bs = [1, 2, 3]
    ops = [vie.Operator(n, 5e-3, 298e6, 1e-6) for n in ns]
    Jh = [field(n, B, 20 + i) for i, (n, B) in enumerate(zip(ns, Bs))]
    Js = [dev(J) for J in Jh]
    Ys = vie.matvec_multi(ops, Js)
    for op, J, Y in zip(ops, Js, Ys):
        assert rel_t(Y, op.matvec(J)) <= 1e-6
    # the persistent launch and the launch per stage run the same device bodies
    Ys2 = vie.matvec_multi(ops, Js, mode="staged")
    for Y, Y2 in zip(Ys, Ys2):
        assert torch.equal(Y, Y2)
    k0 = K.wavenumber(298e6)
    n = ns[2]
    Gt = H.rebuild_components(H.compress_components(E.green_spectra(K.toeplitz_tensor(*n, 5e-3, k0), *n), 1e-6))
    ref = M.matvec_fft(Gt, Jh[2])
    y = Ys[2].cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y - ref) <= 1e-5 * np.linalg.norm(ref)
    for op in ops:
        op.close()


def test_mixed_size_batch_48_64_80():
    """The mixed-size batch: 48^3, 64^3, 80^3 grids with four ring-dipole fields each."""
    wls = workloads.mixed_grids()
    ops = [vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd) for wl in wls]
    Js = []
    for op, wl in zip(ops, wls):
        einc = op.incident_dipole(wl.dipoles)
        Js.append((torch.from_numpy(wl.chi.astype(np.complex64)).cuda()[None, None] * einc).contiguous())
    Ys = vie.matvec_multi(ops, Js)
    for op, J, Y in zip(ops, Js, Ys):
        assert Y.shape == J.shape and J.shape[0] == 4
        assert rel_t(Y, op.matvec(J)) <= 1e-6
    # the 48^3 grid against the oracle (exact operator; HOSVD at 1e-6)
    wl = wls[0]
    k0 = K.wavenumber(wl.freq_hz)
    ref = M.matvec_fft(E.green_spectra(K.toeplitz_tensor(*wl.n, wl.h, k0), *wl.n),
                       Js[0].cpu().numpy().astype(np.complex128))
    y = Ys[0].cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y - ref) <= (1e-5 + 4 * wl.tol_svd) * np.linalg.norm(ref)
    for op in ops:
        op.close()


def test_multi_falls_back_for_other_edge_lengths():
    ns = [(6, 10, 20), (16, 16, 16)]
    ops = [vie.Operator(n, 5e-3, 298e6, 1e-6) for n in ns]
    Js = [dev(field(n, 2, 30 + i)) for i, n in enumerate(ns)]
    Ys = vie.matvec_multi(ops, Js)
    for op, J, Y in zip(ops, Js, Ys):
        assert rel_t(Y, op.matvec(J)) <= 1e-6
    # the persistent launch and the launch per stage run the same device bodies
    Ys2 = vie.matvec_multi(ops, Js, mode="staged")
    for Y, Y2 in zip(Ys, Ys2):
        assert torch.equal(Y, Y2)
    for op in ops:
        op.close()


@pytest.mark.parametrize("n", [(32, 32, 32), (16, 24, 256)])
def test_autotune_keeps_results(n):
    """The autotuner's choices (line-stage CTA sizes; the tcgen05 rebuild's k3
    columns per CTA and CTAs per component, several range counts to choose
    from at P3 = 512) change the speed only: the FP32 matvec agrees before and
    after to FP32 rounding."""
    op = vie.Operator(n, 5e-3, 298e6, 1e-6, rebuild="tcgen05")
    assert op.info()["rebuild_kernel"] == "tcgen05"
    J = dev(field(n, 2, 40))
    before = op.matvec(J)
    threads = op.autotune(2)
    info = op.info()
    assert all(t in (64, 128, 256) for t in threads)
    assert info["tuned_batch"] == 2
    nc, ctas = info["rebuild_tiles"]
    assert (n[2] // nc) * nc == n[2] and nc % 16 == 0 and nc <= 128 and ctas >= 1
    assert rel_t(op.matvec(J), before) <= 1e-6
    op.close()


def test_solve_multi_mixed_grids_equals_separate_solves():
    """The mixed-grid batch (48^3, 64^3, 80^3, four dipole right-hand sides each) solved
    concurrently gives exactly the results of separate solves."""
    ops, chis, rhss = [], [], []
    for wl in workloads.mixed_grids():
        op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd)
        ops.append(op)
        chis.append(torch.from_numpy(wl.chi.astype(np.complex64)).cuda())
        rhss.append(op.incident_dipole(wl.dipoles, dtype=torch.complex64))
    results = vie.solve_multi(ops, chis, rhss, tol=1e-6)
    for op, chi, rhs, (w, info) in zip(ops, chis, rhss, results):
        assert info["converged"], info
        w1, info1 = op.solve(chi, rhs, tol=1e-6)
        assert info1["iterations"] == info["iterations"]
        assert torch.equal(w, w1)
        b = (chi[None, None] * rhs).to(torch.complex128)
        r = b - op.apply_system(chi.to(torch.complex128), w.to(torch.complex128))
        rel = torch.linalg.vector_norm(r.reshape(r.shape[0], -1), dim=1) / \
            torch.linalg.vector_norm(b.reshape(b.shape[0], -1), dim=1)
        assert float(rel.max()) <= 1.5e-6
    for op in ops:
        op.close()
