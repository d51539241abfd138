"""Parity at the workloads' full sizes, in the launch shapes the benchmark uses.

The oracle cannot run whole operators at these sizes, so it computes sampled
outputs one by one: the BTTB sum at a sampled voxel m is
  (G J)_a[m] = sum_b sum_{m'} T_ab(m - m') J_b[m'],
with T from oracle.kernel (dyadic kernel times h^3, self term at m' = m).
Properties that hold at any size cover the rest (residuals of the GPU's own
FP64 operator, finite differences of the loss).
Tolerances: sampled matvec outputs are compared relative to the RMS of the
whole output, against the exact (uncompressed) oracle sum: 1e-5 (the FP32
matvec gate) plus four times the HOSVD tolerance, because the truncation
error is not spread evenly over the voxels.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import adjoint as AD
from oracle import embed as E
from oracle import kernel as K
from oracle import matvec as M

vie = pytest.importorskip("paper_1811_00484_gb300")
pytestmark = pytest.mark.gpu
C128 = torch.complex128


def dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def sampled_product(n, h, k0, J, voxels):
    """Oracle BTTB product at the listed voxels, for every right-hand side of J
    ([B, nsample, 3])."""
    return M.matvec_at(J, h, k0, voxels)


def pick_voxels(n, count, seed):
    rng = np.random.default_rng(seed)
    vox = [tuple(int(rng.integers(0, v)) for v in n) for _ in range(count - 2)]
    return vox + [(0, 0, 0), tuple(v - 1 for v in n)]


def test_ring_dipoles_n96_batch16():
    wl = workloads.dipoles_n96()
    n, h = wl.n, wl.h
    k0 = K.wavenumber(wl.freq_hz)
    op = vie.Operator(n, h, wl.freq_hz, wl.tol_svd)
    B = wl.dipoles.shape[0]
    assert B == 16
    # incident fields at sampled voxels
    einc = op.incident_dipole(wl.dipoles, dtype=C128)
    vox = pick_voxels(n, 6, 1)
    x = (np.arange(n[0]) + 0.5 - 0.5 * n[0]) * h
    pts = np.array([[x[i], x[j], x[k]] for i, j, k in vox])
    e_h = host(einc)
    for b in range(B):
        ref = K.dipole_field(pts, wl.dipoles[b], k0)            # [3, nsample]
        got = np.stack([e_h[b, :, i, j, k] for i, j, k in vox], axis=1)
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    # batched FP32 matvec (the bench's launch shape for batched RHS) at sampled voxels
    J = wl.J[:1].repeat(B, axis=0) * np.arange(1, B + 1)[:, None, None, None, None]
    Y = host(op.matvec(dev(J)))
    ref = sampled_product(n, h, k0, J, vox)
    got = np.stack([Y[:, :, i, j, k] for i, j, k in vox], axis=1)
    scale = np.sqrt(np.mean(np.abs(Y) ** 2, axis=(1, 2, 3, 4)))[:, None, None]
    assert np.max(np.abs(got - ref) / scale) <= 1e-5 + 4 * wl.tol_svd
    # one batched solve of the 16 dipole fields to 1e-6 (FP64 refinement)
    chi = dev(wl.chi, C128)
    w, info = op.solve(chi, einc, tol=1e-6)
    assert info["converged"], info
    b = chi[None, None] * einc
    r = b - op.apply_system(chi, w)
    rel = torch.linalg.vector_norm(r.reshape(B, -1), dim=1) / torch.linalg.vector_norm(b.reshape(B, -1), dim=1)
    assert float(rel.max()) <= 1e-6
    # the FP64 operator that certified the residual, against the oracle at sampled voxels
    Gw = host(op.matvec(w))
    refw = sampled_product(n, h, k0, host(w)[:2], vox[:3])
    gotw = np.stack([Gw[:2, :, i, j, k] for i, j, k in vox[:3]], axis=1)
    scale = np.sqrt(np.mean(np.abs(Gw[:2]) ** 2, axis=(1, 2, 3, 4)))[:, None, None]
    # exact operator vs the Tucker one at 1e-6: pointwise the truncation error
    # can exceed a few times the Frobenius tolerance; same allowance as above
    assert np.max(np.abs(gotw - refw) / scale) <= 1e-5 + 4 * wl.tol_svd
    op.close()


def spread_voxels(n, count, seed):
    """Corners, the centre, voxels on the mid-planes and next to them, then
    uniformly drawn interior voxels, `count` in all."""
    n1, n2, n3 = n
    fixed = [(0, 0, 0), (n1 - 1, n2 - 1, n3 - 1), (n1 // 2, n2 // 2, n3 // 2),
             (n1 // 2 - 1, n2 // 2 - 1, n3 // 2 - 1), (n1 // 2, 0, n3 - 1), (0, n2 // 2, n3 // 2),
             (n1 - 1, n2 // 2, 0), (n1 // 2, n2 - 1, n3 // 2), (n1 // 4, 3 * n2 // 4, n3 // 2),
             (3 * n1 // 4, n2 // 4, n3 - 1), (n1 - 1, 0, n3 // 2), (n1 // 2 + 1, n2 // 2 + 1, 1)]
    rng = np.random.default_rng(seed)
    rand = [tuple(int(rng.integers(0, v)) for v in n) for _ in range(count - len(fixed))]
    return fixed + rand


def test_headline_n256_ring_dipoles():
    """The memory headline workload at its bench launch shape: 256^3 voxels (512^3
    padded), 8 ring dipoles in one batch, HOSVD 1e-6, both paths.

    The chain of checks: the FP64 matvec on the stored spectra against the oracle at
    32 sampled voxels (FP64 rounding only: 1e-10 of the output's RMS); the FP32
    matvecs of both paths against the FP64 ones over the whole field (relative L2,
    the FP32 gate 1e-5: with the dipoles' dynamic range the FP32 rounding is spread
    over the field as an absolute error, so it is not compared voxel by voxel); the
    FP64 Tucker operator against the stored one (relative L2, the HOSVD
    truncation); the refined solve to 1e-5, its residual with the GPU's FP64 Tucker
    operator and with the FP64 operator on the stored spectra, and that operator
    applied to the solution against the oracle at sampled voxels."""
    wl = workloads.memory_n256()
    n, h = wl.n, wl.h
    k0 = K.wavenumber(wl.freq_hz)
    op = vie.Operator(n, h, wl.freq_hz, wl.tol_svd, store_uncompressed=True)
    info = op.info()
    assert info["uncompressed_bytes"] == 6 * 512 ** 3 * 8
    assert info["tucker_bytes"] * 1000 < info["uncompressed_bytes"]
    B = wl.dipoles.shape[0]
    assert B == 8
    einc = op.incident_dipole(wl.dipoles)                      # c64, the bench's input
    e_h = host(einc)
    vox = spread_voxels(n, 32, 3)
    x = (np.arange(n[0]) + 0.5 - 0.5 * n[0]) * h
    pts = np.array([[x[i], x[j], x[k]] for i, j, k in vox[:8]])
    for b in range(B):
        ref = K.dipole_field(pts, wl.dipoles[b], k0)
        got = np.stack([e_h[b, :, i, j, k] for i, j, k in vox[:8]], axis=1)
        assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref))
    ref = sampled_product(n, h, k0, e_h, vox)                  # [B, 32, 3]
    del e_h
    Y32 = {p: op.matvec(einc, path=p) for p in ("tucker", "uncompressed")}
    err32 = {p: 0.0 for p in Y32}
    nrm, dtu = 0.0, 0.0
    for b0 in range(0, B, 2):                                  # FP64 two right-hand sides at a time
        e64 = einc[b0:b0 + 2].to(C128)
        Yu = op.matvec(e64, path="uncompressed")
        Yt = op.matvec(e64)
        Yh = host(Yu)
        got = np.stack([Yh[:, :, i, j, k] for i, j, k in vox], axis=1)
        scale = np.sqrt(np.mean(np.abs(Yh) ** 2, axis=(1, 2, 3, 4)))[:, None, None]
        assert np.max(np.abs(got - ref[b0:b0 + 2]) / scale) <= 1e-10
        nrm += float(torch.linalg.vector_norm(Yu)) ** 2
        dtu += float(torch.linalg.vector_norm(Yt - Yu)) ** 2
        for p, Y64 in (("tucker", Yt), ("uncompressed", Yu)):
            err32[p] += float(torch.linalg.vector_norm(Y32[p][b0:b0 + 2].to(C128) - Y64)) ** 2
        del Yu, Yt, e64, Yh
    for p in err32:
        assert (err32[p] / nrm) ** 0.5 <= 1e-5, (p, (err32[p] / nrm) ** 0.5)
    assert (dtu / nrm) ** 0.5 <= 1e-5
    del Y32
    torch.cuda.empty_cache()
    chi = dev(wl.chi)
    w, sinfo = op.solve(chi, einc, tol=1e-5)
    assert sinfo["converged"] and sinfo["relres"] <= 1e-5, sinfo
    # residual of each right-hand side with the FP64 operators, one at a time
    chi64 = chi.to(C128)
    for b in range(B):
        wb = w[b:b + 1].to(C128)
        bb = chi64[None, None] * einc[b:b + 1].to(C128)
        nb = torch.linalg.vector_norm(bb)
        r_t = bb - op.apply_system(chi64, wb)
        r_u = bb - op.apply_system(chi64, wb, path="uncompressed")
        assert float(torch.linalg.vector_norm(r_t) / nb) <= 1.01e-5
        assert float(torch.linalg.vector_norm(r_u) / nb) <= 1.5e-5
    # the FP64 operator on the stored spectra, applied to the solution, against the oracle
    w2 = w[:2].to(C128)
    Gw = host(op.matvec(w2, path="uncompressed"))
    refw = sampled_product(n, h, k0, host(w2), vox[:6])
    gotw = np.stack([Gw[:, :, i, j, k] for i, j, k in vox[:6]], axis=1)
    scale = np.sqrt(np.mean(np.abs(Gw) ** 2, axis=(1, 2, 3, 4)))[:, None, None]
    assert np.max(np.abs(gotw - refw) / scale) <= 1e-10
    op.close()


def test_gradient_n64_against_finite_differences():
    """Adjoint gradient through the solve vs FP64 central differences (step 1e-4)."""
    wl = workloads.gradient_n64()
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd)
    opts = dict(tol=1e-12, max_refine=40)
    einc = dev(wl.einc, C128)
    with torch.no_grad():
        E_t = vie.solve_fields(op, dev(wl.extras["chi_target"], C128), einc, **opts)
    chi = dev(wl.chi, C128).requires_grad_(True)
    loss = torch.sum(torch.abs(vie.solve_fields(op, chi, einc, **opts) - E_t) ** 2)
    loss.backward()
    g = chi.grad.detach().cpu().numpy()
    step = 1e-4
    an, fd = [], []
    for v in wl.extras["probe_voxels"]:
        idx = np.unravel_index(int(v), wl.chi.shape)
        for unit in (1.0, 1j):
            vals = []
            for sgn in (1, -1):
                c = wl.chi.copy()
                c[idx] += sgn * unit * step
                with torch.no_grad():
                    Ee = vie.solve_fields(op, dev(c, C128), einc, **opts)
                    vals.append(torch.sum(torch.abs(Ee - E_t) ** 2).item())
            fd.append((vals[0] - vals[1]) / (2 * step))
            an.append(g[idx].real if unit == 1.0 else g[idx].imag)
    an, fd = np.array(an), np.array(fd)
    assert np.linalg.norm(an - fd) <= 1e-4 * np.linalg.norm(fd)
    assert np.all(np.abs(an - fd) <= 1e-3 * np.abs(fd) + 1e-4 * np.linalg.norm(fd) / np.sqrt(fd.size))
    op.close()


@pytest.mark.parametrize("n", [16, 24])
def test_gradient_against_oracle_adjoint_gradient(n):
    """The gradient workload's recipe at 16^3 and 24^3, target field from the oracle's
    solve: GPU adjoint gradient vs the oracle's (the oracle's 64^3 solves to 1e-12
    are beyond a test's CPU budget; at 64^3 the gradient is pinned by finite
    differences above)."""
    wl = workloads.gradient_n64(n=n)
    k0 = K.wavenumber(wl.freq_hz)
    Ghat = E.green_spectra(K.toeplitz_tensor(*wl.n, wl.h, k0), *wl.n)
    _, E_t, _ = AD.forward(Ghat, wl.extras["chi_target"], wl.einc, tol=1e-12)
    L_o, g_o, _, _ = AD.gradient(Ghat, wl.chi, wl.einc, E_t)
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, 1e-10)
    chi = dev(wl.chi, C128).requires_grad_(True)
    Ef = vie.solve_fields(op, chi, dev(wl.einc, C128), tol=1e-12, max_refine=40)
    loss = torch.sum(torch.abs(Ef - dev(E_t, C128)) ** 2)
    loss.backward()
    g = chi.grad.detach().cpu().numpy()
    assert abs(loss.item() - L_o) <= 1e-6 * L_o
    assert np.linalg.norm(g - g_o) <= 1e-5 * np.linalg.norm(g_o)
    op.close()


def test_solve_error_against_oracle_solution_n32():
    """Solution error, not only the residual: the plane-wave solve recipe at 32^3
    (HOSVD 1e-6) against the oracle's GMRES solution to 1e-12 with its own HOSVD
    of the same spectra.  The FP64-output solve to 1e-10 sets the effective
    condition kappa = error / residual; the bench-style solve (c64 in and out, to
    1e-6) must then sit within 3 kappa tol plus the c64 rounding of the output."""
    from oracle import gmres as GM
    from oracle import hosvd as H
    wl = workloads.make("solve n=32", 32, seed=1, tol_svd=1e-6, incident="plane")
    k0 = K.wavenumber(wl.freq_hz)
    Ghat = E.green_spectra(K.toeplitz_tensor(*wl.n, wl.h, k0), *wl.n)
    Gt = H.rebuild_components(H.compress_components(Ghat, wl.tol_svd))
    b = M.system_rhs(wl.chi, wl.einc)
    w_ref, oinfo = GM.gmres(lambda v: M.apply_system(Gt, wl.chi, v), b, tol=1e-12, restart=50,
                            max_outer=400)
    assert oinfo["converged"]
    op = vie.Operator(wl.n, wl.h, wl.freq_hz, wl.tol_svd)
    w64, i64 = op.solve(dev(wl.chi, C128), dev(wl.einc, C128), tol=1e-10)
    assert i64["converged"]
    err64 = np.linalg.norm(host(w64) - w_ref) / np.linalg.norm(w_ref)
    assert err64 <= 1e-7
    kappa = max(1.0, err64 / 1e-10)
    w32, i32 = op.solve(dev(wl.chi), dev(wl.einc), tol=1e-6)
    assert i32["converged"]
    err32 = np.linalg.norm(host(w32) - w_ref) / np.linalg.norm(w_ref)
    assert err32 <= 3 * kappa * 1e-6 + 1e-7, (err32, kappa)
    op.close()
