"""Pins of the oracle's Green's kernel (eqs. (5)-(6)) and self term.

The closed form in oracle.kernel.dyadic is checked against things that do not
share its derivation: symbolic differentiation of g, central finite
differences, the far-field limit, symmetry, and a sphere quadrature of the
dyadic itself for the self term.
"""
import math

import numpy as np
import pytest

from oracle import kernel as K

K0 = K.wavenumber(298e6)


def test_wavenumber_298mhz():
    # k0 = 2 pi f / c at the 7 T frequency of Section VI.C
    assert abs(K0 - 6.2456182) < 1e-6


def _hessian_fd(R, k0, step):
    g = lambda x: K.green(np.linalg.norm(x), k0)
    H = np.zeros((3, 3), dtype=np.complex128)
    e = np.eye(3) * step
    for a in range(3):
        for b in range(3):
            if a == b:
                H[a, a] = (g(R + e[a]) - 2 * g(R) + g(R - e[a])) / step ** 2
            else:
                H[a, b] = (g(R + e[a] + e[b]) - g(R + e[a] - e[b])
                           - g(R - e[a] + e[b]) + g(R - e[a] - e[b])) / (4 * step ** 2)
    return H


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dyadic_matches_finite_difference_hessian(seed):
    rng = np.random.default_rng(seed)
    R = rng.uniform(-0.2, 0.2, size=3) + np.array([0.01, 0.0, 0.0])
    r = np.linalg.norm(R)
    H = _hessian_fd(R, K0, 1e-4 * r)
    G = K.dyadic(R, K0)
    ref = K0 ** 2 * K.green(r, K0) * np.eye(3) + H
    for c, (a, b) in enumerate(K.COMPONENTS):
        assert abs(G[c] - ref[a, b]) <= 2e-6 * np.max(np.abs(ref))


def test_dyadic_matches_symbolic_derivative():
    sp = pytest.importorskip("sympy")
    x, y, z, k = sp.symbols("x y z k", real=True)
    r = sp.sqrt(x * x + y * y + z * z)
    g = sp.exp(-sp.I * k * r) / (4 * sp.pi * r)
    X = (x, y, z)
    pts = [(0.013, -0.021, 0.034), (0.2, 0.05, -0.11), (-0.004, 0.003, 0.0017)]
    for p in pts:
        G = K.dyadic(np.array(p), K0)
        for c, (a, b) in enumerate(K.COMPONENTS):
            expr = sp.diff(g, X[a], X[b]) + (k * k * g if a == b else 0)
            val = complex(expr.subs({x: p[0], y: p[1], z: p[2], k: K0}).evalf(30))
            assert abs(G[c] - val) <= 1e-12 * abs(val) + 1e-14


def test_far_field_is_transverse():
    # r -> infinity: G -> k0^2 g (I - Rhat Rhat)
    d = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    for r in (1e3, 1e4):
        G = K.dyadic(d * r, K0)
        g = K.green(r, K0)
        for c, (a, b) in enumerate(K.COMPONENTS):
            far = K0 ** 2 * g * ((a == b) - d[a] * d[b])
            assert abs(G[c] - far) <= 5.0 / (K0 * r) * abs(K0 ** 2 * g)


def test_toeplitz_parities():
    n1, n2, n3 = 3, 4, 5
    T = K.toeplitz_tensor(n1, n2, n3, 5e-3, K0)
    assert T.shape == (6, 5, 7, 9)
    full = T[:, ::-1, ::-1, ::-1]
    assert np.allclose(T, full, rtol=0, atol=0)          # T(-R) = T(R)
    # one-axis flips: component ab changes sign once per odd index among a, b
    for axis in range(3):
        flip = np.flip(T, axis=1 + axis)
        for c, (a, b) in enumerate(K.COMPONENTS):
            s = (-1) ** ((a == axis) + (b == axis))
            assert np.allclose(flip[c], s * T[c], rtol=1e-15, atol=0)


def test_toeplitz_scaled_by_voxel_volume():
    h = 5e-3
    T = K.toeplitz_tensor(2, 2, 2, h, K0)
    R = np.array([h, -h, 0.0])
    G = K.dyadic(R, K0)
    assert np.allclose(T[:, 2, 0, 1], G * h ** 3, rtol=1e-15)
    # the zero offset holds the self term on the diagonal only
    s = K.self_term(h, K0)
    assert np.allclose(T[[0, 3, 5], 1, 1, 1], s)
    assert np.all(T[[1, 2, 4], 1, 1, 1] == 0)


def test_self_term_quasi_static_limit():
    # Lorentz depolarisation of a sphere: -1/3 as k0 -> 0
    assert abs(K.self_term(5e-3, 1e-9) + 1.0 / 3.0) < 1e-12
    assert abs(K.self_term(5e-3, 1e-9, mode="pv")) < 1e-12


@pytest.mark.parametrize("k0", [K0, 40.0, 300.0])
def test_self_term_from_sphere_quadrature(k0):
    """Principal value of the dyadic over the sphere, plus the -1/3 delta part.

    Angular Gauss-Legendre x trapezoid rules integrate Rhat Rhat exactly, so
    the 1/r^3 part cancels shell by shell; the radial rule then integrates
    the remaining smooth part.
    """
    h = 5e-3
    a = K.equivalent_sphere_radius(h)
    xr, wr = np.polynomial.legendre.leggauss(40)
    rr = 0.5 * a * (xr + 1.0)
    wr = 0.5 * a * wr
    mu, wmu = np.polynomial.legendre.leggauss(8)
    nphi = 8
    phi = 2 * math.pi * np.arange(nphi) / nphi
    acc = np.zeros(6, dtype=np.complex128)
    for r, w_r in zip(rr, wr):
        for m, w_m in zip(mu, wmu):
            st = math.sqrt(1 - m * m)
            dirs = np.stack([st * np.cos(phi), st * np.sin(phi), np.full(nphi, m)], axis=1)
            vals = K.dyadic(dirs * r, k0)
            acc += w_r * w_m * (2 * math.pi / nphi) * r * r * vals.sum(axis=1)
    s_full = K.self_term(h, k0, "full")
    s_pv = K.self_term(h, k0, "pv")
    for c, (p, q) in enumerate(K.COMPONENTS):
        want = s_pv if p == q else 0.0
        assert abs(acc[c] - want) <= 1e-10
    assert abs((s_pv - 1.0 / 3.0) - s_full) < 1e-15


def test_dipole_field_is_zz_column():
    src = np.array([0.15, 0.0, 0.0])
    p = np.array([0.01, 0.02, -0.03])
    e = K.dipole_field(p[None], src, K0)[:, 0]
    G = K.dyadic(p - src, K0)
    assert np.allclose(e, [G[2], G[4], G[5]])


@pytest.mark.parametrize("n", [(3, 4, 5), (4, 3, 2)])
def test_dipole_incident_at_hand_placed_voxel_centres(n):
    """dipole_incident samples dipole_field at the voxel centres (i + 1/2 - n/2) h,
    box centre at the origin: written out here by hand for odd and even edges."""
    h = 0.01
    centres = {2: (-0.005, 0.005), 3: (-0.01, 0.0, 0.01), 4: (-0.015, -0.005, 0.005, 0.015),
               5: (-0.02, -0.01, 0.0, 0.01, 0.02)}
    src = np.array([[0.003, -0.021, 0.0071], [-0.05, 0.04, 0.1]])
    e = K.dipole_incident(*n, h, K0, src)
    assert e.shape == (2, 3) + n
    for b in range(2):
        for i, x in enumerate(centres[n[0]]):
            for j, y in enumerate(centres[n[1]]):
                for k, z in enumerate(centres[n[2]]):
                    ref = K.dipole_field(np.array([x, y, z]), src[b], K0)
                    assert np.allclose(e[b, :, i, j, k], ref, rtol=1e-13, atol=0.0)


def test_dipole_incident_mirror_symmetry_about_the_box_centre():
    """A z-dipole at the origin of an even grid: e_z is even and e_x odd under
    x -> -x, which holds only if the voxel centres are symmetric about the box
    centre (a shift of the centres by h/2 breaks it)."""
    n = 4
    e = K.dipole_incident(n, n, n, 0.01, K0, np.zeros((1, 3)))[0]
    assert np.allclose(e[2], e[2][::-1], rtol=1e-13, atol=0.0)
    assert np.allclose(e[0], -e[0][::-1], rtol=1e-13, atol=0.0)
    assert np.allclose(e[2], e[2][:, :, ::-1], rtol=1e-13, atol=0.0)
