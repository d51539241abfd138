"""GPU parity of the GMRES solve, its adjoint and the contrast gradient.

Reference solutions are the oracle's: dense direct solves on tiny grids and
GMRES to 1e-12 with the oracle's own HOSVD (same tolerance) elsewhere.
Residuals of GPU solutions are evaluated with the oracle's FP64 operator.
Tolerances: a solve to relative residual tol has relative error up to
kappa * tol; tests either check the residual (<= tol, small slack for the
Tucker difference between the two HOSVD routes) or solve to 1e-10 and bound
the error by 1e-7.  Tight targets use complex128 inputs and outputs: a
complex64 solution is rounded to FP32 on output, which alone leaves a
relative residual of a few 1e-8 (bounded here by 5e-7).
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import adjoint as AD
from oracle import embed as E
from oracle import gmres as GM
from oracle import hosvd as H
from oracle import kernel as K
from oracle import matvec as M

vie = pytest.importorskip("paper_1811_00484_gb300")
pytestmark = pytest.mark.gpu
C128 = torch.complex128


def dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


_cache = {}


def case(n, tol_svd=1e-8, seed=5, incident="plane"):
    key = (n, tol_svd, seed, incident)
    if key not in _cache:
        wl = workloads.make("solve", n, seed=seed, tol_svd=tol_svd, incident=incident,
                            dipoles=workloads.ring_dipoles(3) if incident == "dipole" else None)
        k0 = K.wavenumber(wl.freq_hz)
        T = K.toeplitz_tensor(*wl.n, wl.h, k0)
        Ghat = E.green_spectra(T, *wl.n)
        Gt = H.rebuild_components(H.compress_components(Ghat, tol_svd))
        op = vie.Operator(wl.n, wl.h, wl.freq_hz, tol_svd, store_uncompressed=True)
        _cache[key] = (wl, T, Ghat, Gt, op)
    return _cache[key]


def residual(Ghat, chi, einc, w):
    b = M.system_rhs(chi, einc)
    return float(np.linalg.norm(b - M.apply_system(Ghat, chi, w)) / np.linalg.norm(b))


def test_tiny_solve_matches_dense_direct_solve():
    wl, T, Ghat, Gt, op = case((4, 5, 6), tol_svd=1e-10)
    n1, n2, n3 = wl.n
    G = M.dense_operator(T, n1, n2, n3)
    N = n1 * n2 * n3
    A = np.eye(3 * N) - np.tile(wl.chi.ravel(), 3)[:, None] * G
    w_ref = np.linalg.solve(A, (wl.chi * wl.einc[0]).ravel()).reshape(wl.einc[0].shape)
    for dt, bound in ((torch.complex64, 1e-6), (torch.complex128, 1e-8)):
        w, info = op.solve(dev(wl.chi, dt), dev(wl.einc, dt), tol=1e-11)
        assert info["converged"], info
        assert rel(host(w)[0], w_ref) <= bound


@pytest.mark.parametrize("use_graph", [True, False])
def test_refined_solve_n16_against_oracle_gmres(use_graph):
    wl, T, Ghat, Gt, op = case((16, 16, 16), tol_svd=1e-8, seed=1)
    w, info = op.solve(dev(wl.chi, C128), dev(wl.einc, C128), tol=1e-10, use_graph=use_graph)
    assert info["converged"] and info["relres"] <= 1e-10, info
    wg = host(w)
    w32, _ = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-8, use_graph=use_graph)
    assert residual(Gt, wl.chi, wl.einc, host(w32)) <= 5e-7
    w_ref, oinfo = GM.gmres(lambda v: M.apply_system(Gt, wl.chi, v), M.system_rhs(wl.chi, wl.einc),
                            tol=1e-12, restart=50, max_outer=400)
    assert oinfo["converged"]
    assert residual(Gt, wl.chi, wl.einc, wg) <= 2e-10
    assert rel(wg, w_ref) <= 1e-7


def test_odd_voxel_count_solve():
    """All-odd grid: 3 n1 n2 n3 is odd, so the Gram-Schmidt kernels use 8-byte loads."""
    wl, T, Ghat, Gt, op = case((5, 7, 9), tol_svd=1e-8, seed=4)
    assert (3 * 5 * 7 * 9) % 2 == 1
    w, info = op.solve(dev(wl.chi, C128), dev(wl.einc, C128), tol=1e-10)
    assert info["converged"] and info["relres"] <= 1e-10, info
    assert residual(Gt, wl.chi, wl.einc, host(w)) <= 2e-10
    w32, info32 = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-6, use_graph=False)
    assert info32["converged"]
    assert residual(Gt, wl.chi, wl.einc, host(w32)) <= 2e-6


def test_graph_and_direct_launches_agree():
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=3)
    w1, i1 = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-9, use_graph=True)
    w2, i2 = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-9, use_graph=False)
    assert i1["iterations"] == i2["iterations"]
    assert torch.equal(w1, w2)


def test_two_pass_gram_schmidt_solve():
    """orth=2: classical Gram-Schmidt with the DGKS-conditional second pass."""
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=3)
    w, info = op.solve(dev(wl.chi, C128), dev(wl.einc, C128), tol=1e-10, orth=2)
    assert info["converged"]
    assert residual(Gt, wl.chi, wl.einc, host(w)) <= 2e-10


def test_fp32_only_solve():
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=3)
    w, info = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-5, refine=False)
    assert info["converged"], info
    assert residual(Gt, wl.chi, wl.einc, host(w)) <= 1e-5


def test_uncompressed_path_solve():
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=3)
    w, info = op.solve(dev(wl.chi, C128), dev(wl.einc, C128), tol=1e-9, path="uncompressed")
    assert info["converged"]
    assert residual(Ghat, wl.chi, wl.einc, host(w)) <= 1e-9


def test_batched_dipole_solves_equal_single_solves():
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=4, incident="dipole")
    einc = op.incident_dipole(wl.dipoles, dtype=C128)
    ref = K.dipole_incident(*wl.n, wl.h, K.wavenumber(wl.freq_hz), wl.dipoles)
    assert rel(host(einc), ref) <= 1e-12
    chi = dev(wl.chi, C128)
    wb, ib = op.solve(chi, einc, tol=1e-9)
    assert ib["converged"]
    for b in range(einc.shape[0]):
        assert residual(Gt, wl.chi, ref[b], host(wb)[b]) <= 2e-9
        w1, _ = op.solve(chi, einc[b:b + 1].contiguous(), tol=1e-9)
        assert rel(host(w1)[0], host(wb)[b]) <= 1e-6


def test_adjoint_solve():
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=3)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(wl.einc.shape) + 1j * rng.standard_normal(wl.einc.shape)
    lam, info = op.solve(dev(wl.chi, C128), dev(b, C128), incident=False, adjoint=True, tol=1e-10)
    assert info["converged"]
    lh = host(lam)
    r = b - AD.apply_system_adjoint(Gt, wl.chi, lh)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 2e-10


def test_initial_guess_is_used():
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=3)
    w, info = op.solve(dev(wl.chi, torch.complex128), dev(wl.einc, torch.complex128), tol=1e-10)
    w2, info2 = op.solve(dev(wl.chi, torch.complex128), dev(wl.einc, torch.complex128), tol=1e-10,
                         x0=w)
    assert info2["converged"] and info2["iterations"] == 0 and info2["refine_steps"] == 0


def test_no_convergence_is_reported():
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=3)
    w, info = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-12, max_refine=1, max_outer=1, restart=2,
                       raise_on_failure=False)
    assert info["status"] == 4 and not info["converged"]
    assert info["relres"] > 1e-12 and len(info["history"]) == 2
    with pytest.raises(vie.VieError):
        op.solve(dev(wl.chi), dev(wl.einc), tol=1e-12, max_refine=1, max_outer=1, restart=2)


@pytest.mark.parametrize("where", ["chi", "einc"])
def test_non_finite_input_is_reported(where):
    """A NaN placed in the contrast or the incident field on the host makes the
    first FP64 residual non-finite: the solve stops with VIE_ERR_NUMERIC."""
    wl, T, Ghat, Gt, op = case((8, 6, 10), tol_svd=1e-8, seed=3)
    chi, einc = wl.chi.copy(), wl.einc.copy()
    if where == "chi":
        chi[4, 3, 5] = np.nan
    else:
        einc[0, 1, 2, 2, 2] = np.nan
    with pytest.raises(vie.VieError) as e:
        op.solve(dev(chi), dev(einc), tol=1e-8)
    assert e.value.status == 5 and "non-finite" in str(e.value)
    # the operator is still usable afterwards
    w, info = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-6)
    assert info["converged"]


def test_bounded_device_wait_gives_up_and_reports_timeout():
    """The shared-memory barrier wait of the TMA-fed kernels, run alone: it
    completes when the arrival is made, and gives up after its limit (reported
    as VIE_ERR_TIMEOUT) when nothing arrives; the context stays usable."""
    import ctypes
    import time
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert vie.lib.vie_selftest_bounded_wait(1, 0.05, stream) == 0
    t0 = time.perf_counter()
    assert vie.lib.vie_selftest_bounded_wait(0, 0.05, stream) == 6
    assert time.perf_counter() - t0 < 5.0
    assert "gave up" in vie.lib.vie_last_error().decode()
    assert vie.lib.vie_selftest_bounded_wait(0, 0.0, stream) == 1
    # the grid barrier of the persistent multi-grid matvec: met, and not met
    assert vie.lib.vie_selftest_bounded_wait(3, 0.05, stream) == 0
    t0 = time.perf_counter()
    assert vie.lib.vie_selftest_bounded_wait(2, 0.05, stream) == 6
    assert time.perf_counter() - t0 < 5.0
    x = torch.ones(8, device="cuda")
    assert float((x * 2).sum()) == 16.0


def test_autograd_gradient_matches_oracle_and_finite_differences():
    wl, T, Ghat, Gt, op = case((6, 6, 6), tol_svd=1e-10, seed=9)
    rng = np.random.default_rng(3)
    E_t = wl.einc + 0.2 * (rng.standard_normal(wl.einc.shape) + 1j * rng.standard_normal(wl.einc.shape))
    chi = dev(wl.chi, torch.complex128).requires_grad_(True)
    einc = dev(wl.einc, torch.complex128)
    Et = dev(E_t, torch.complex128)
    opts = dict(tol=1e-12, max_refine=30)
    Ef = vie.solve_fields(op, chi, einc, **opts)
    loss = torch.sum(torch.abs(Ef - Et) ** 2)
    loss.backward()
    g = chi.grad.detach().cpu().numpy()
    L_o, g_o, _, _ = AD.gradient(Gt, wl.chi, wl.einc, E_t)
    assert abs(loss.item() - L_o) <= 1e-9 * L_o
    assert rel(g, g_o) <= 1e-7
    step = 1e-4
    for v in rng.choice(np.flatnonzero(wl.mask.ravel()), size=3, replace=False):
        idx = np.unravel_index(v, wl.chi.shape)
        for unit, part in ((1.0, "re"), (1j, "im")):
            vals = []
            for sgn in (1, -1):
                c = wl.chi.copy()
                c[idx] += sgn * unit * step
                with torch.no_grad():
                    Ee = vie.solve_fields(op, dev(c, torch.complex128), einc, **opts)
                    vals.append(torch.sum(torch.abs(Ee - Et) ** 2).item())
            fd = (vals[0] - vals[1]) / (2 * step)
            an = g[idx].real if part == "re" else g[idx].imag
            assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-3 * np.abs(g).max())


def test_full_size_n64_plane_wave_solve():
    """The 64^3 solve workload: GMRES(50) to 1e-6 with FP64 refinement (Tucker at 1e-6)."""
    wl = workloads.solve_n64()
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd)
    w, info = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-6)
    assert info["converged"], info
    k0 = K.wavenumber(wl.freq_hz)
    Ghat = E.green_spectra(K.toeplitz_tensor(*wl.n, wl.h, k0), *wl.n)
    Gt = H.rebuild_components(H.compress_components(Ghat, wl.tol_svd))
    wg = host(w)
    assert residual(Gt, wl.chi, wl.einc, wg) <= 1.5e-6
    assert info["refine_steps"] >= 1
    op.close()


def test_chunked_rebuild_n128_solve():
    """128^3: the per-matvec rebuild scratch holds only part of the k1 range, so both the
    chunked rebuild and the solver's prefetch of the first chunk run.  The FP32 matvec is
    checked against the FP64 operator (shared-memory FFTs, rebuild inside each CTA, no
    scratch), and the solve's residual is that FP64 operator's."""
    n = (128, 128, 128)
    wl = workloads.make("chunked", n, seed=6, tol_svd=1e-6, incident="plane")
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd)
    info = op.info()
    H = [p // 2 + 1 for p in (256, 256, 256)]
    full = H[0] * H[1] * 6 * H[2] * 8
    assert 0 < info["rebuild_scratch_bytes"] < full
    J = dev(wl.J[:1])
    y32 = op.matvec(J).to(torch.complex128)
    y64 = op.matvec(J.to(torch.complex128))
    assert rel(host(y32), host(y64)) <= 2e-6
    chi, einc = dev(wl.chi), dev(wl.einc)
    w, sinfo = op.solve(chi, einc, tol=1e-5)
    assert sinfo["converged"], sinfo
    b = chi.to(torch.complex128)[None, None] * einc.to(torch.complex128)
    r = b - op.apply_system(chi.to(torch.complex128), w.to(torch.complex128))
    assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b)) <= 1e-5
    op.close()
