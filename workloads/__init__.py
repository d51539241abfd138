"""Seeded synthetic inputs for the Tucker-compressed FFT-VIE solve.

This module is shared by the FP64 CPU oracle, the tests and the benchmark.
It only *draws and lays out inputs*: voxel grids, the tissue contrast chi,
random currents, the x-polarised plane wave and dipole positions.  It holds
none of the method's arithmetic (no Green's kernel, no circulant embedding,
no FFT, no compression, no solver), so the oracle and the CUDA library stay
independent of each other.

Layouts (C order, z fastest), matching the library's boundary:
  currents J      complex  [B][3][n1][n2][n3]
  contrast chi    complex  [n1][n2][n3]
  incident field  complex  [B][3][n1][n2][n3]

Draw order for every workload (one ``numpy.random.default_rng(seed)``):
  J real part, J imaginary part (standard normal, shape [B,3,n1,n2,n3]),
  eps_r ~ U[40, 80] (n1*n2*n3), sigma ~ U[0.3, 1.0] S/m (n1*n2*n3),
  then the workload-specific extras.
The tissue is a centred ellipsoid with semi-axes 0.4/0.45/0.5 in
box-normalised coordinates u = x / (L/2), i.e. 0.2 L, 0.225 L and 0.25 L.
The paper's scatterers (a licensed voxel head model, Section VI.C; a
homogeneous sphere, Section VI.D) are replaced by this seeded ellipsoid with
voxel-wise random brain-like permittivity and conductivity at 298 MHz.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Physical constants used to form the contrast and the plane wave.
SPEED_OF_LIGHT = 299_792_458.0          # m/s
VACUUM_PERMITTIVITY = 8.8541878128e-12  # F/m
FREQ_7T_HZ = 298e6                      # 7 T proton Larmor frequency (Section VI.C)
VOXEL_H = 5e-3                          # 5 mm voxels in every workload

HEAD_SEMI_AXES = (0.4, 0.45, 0.5)       # box-normalised semi-axes of the ellipsoid


@dataclass
class Workload:
    """One synthetic problem: grid, contrast, currents and incident fields."""
    name: str
    n: tuple                      # (n1, n2, n3)
    h: float
    freq_hz: float
    tol_svd: float
    seed: int
    J: np.ndarray                 # complex128 [B,3,n1,n2,n3]
    eps_r: np.ndarray             # float64 [n1,n2,n3] (inside-mask values meaningful)
    sigma: np.ndarray             # float64 [n1,n2,n3]
    mask: np.ndarray              # bool [n1,n2,n3]
    chi: np.ndarray               # complex128 [n1,n2,n3]
    einc: np.ndarray | None = None          # complex128 [B,3,n1,n2,n3] (plane wave)
    dipoles: np.ndarray | None = None       # float64 [B,3] source points (z-directed)
    extras: dict = field(default_factory=dict)


def omega(freq_hz: float) -> float:
    return 2.0 * math.pi * freq_hz


def voxel_centres(n: int, h: float) -> np.ndarray:
    """Centres x_i = (i + 1/2 - n/2) h, so the box centre is the origin."""
    return (np.arange(n, dtype=np.float64) + 0.5 - 0.5 * n) * h


def ellipsoid_mask(n1: int, n2: int, n3: int, semi=HEAD_SEMI_AXES,
                   centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Voxels whose centre lies in the ellipsoid (box-normalised coordinates)."""
    u = (np.arange(n1) + 0.5 - 0.5 * n1) / (0.5 * n1)
    v = (np.arange(n2) + 0.5 - 0.5 * n2) / (0.5 * n2)
    w = (np.arange(n3) + 0.5 - 0.5 * n3) / (0.5 * n3)
    U, V, W = np.meshgrid(u, v, w, indexing="ij")
    q = ((U - centre[0]) / semi[0]) ** 2 + ((V - centre[1]) / semi[1]) ** 2 \
        + ((W - centre[2]) / semi[2]) ** 2
    return q <= 1.0


def contrast_from_tissue(eps_r, sigma, mask, freq_hz):
    """chi = eps_r - 1 - i sigma / (omega eps0) inside the tissue, 0 outside.

    The minus sign matches the exp(-i k0 r) Green's function of eq. (6)
    (a passive medium under that time convention).
    """
    chi = (eps_r - 1.0) - 1j * sigma / (omega(freq_hz) * VACUUM_PERMITTIVITY)
    return np.where(mask, chi, 0.0 + 0.0j)


def draw_base(rng, B, n1, n2, n3):
    """J (re, then im), eps_r, sigma in the fixed draw order."""
    shape = (B, 3, n1, n2, n3)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    J = re + 1j * im
    eps_r = rng.uniform(40.0, 80.0, size=n1 * n2 * n3).reshape(n1, n2, n3)
    sigma = rng.uniform(0.3, 1.0, size=n1 * n2 * n3).reshape(n1, n2, n3)
    return J, eps_r, sigma


def plane_wave_x(n1, n2, n3, h, freq_hz, B=1):
    """x-polarised plane wave e_inc = x_hat exp(-i k0 z), z from the box centre."""
    k0 = omega(freq_hz) / SPEED_OF_LIGHT
    z = voxel_centres(n3, h)
    e = np.zeros((B, 3, n1, n2, n3), dtype=np.complex128)
    e[:, 0] = np.exp(-1j * k0 * z)[None, None, None, :]
    return e


def ring_dipoles(count, radius=0.15, z=0.0):
    """Source points of z-directed dipoles at equispaced azimuths 2 pi m / count."""
    phi = 2.0 * math.pi * np.arange(count) / count
    return np.stack([radius * np.cos(phi), radius * np.sin(phi),
                     np.full(count, z)], axis=1)


def make(name, n, seed, B=1, tol_svd=1e-6, h=VOXEL_H, freq_hz=FREQ_7T_HZ,
         incident="none", dipoles=None):
    """Generic workload: draws J, eps_r, sigma in the fixed order."""
    if isinstance(n, int):
        n = (n, n, n)
    n1, n2, n3 = n
    rng = np.random.default_rng(seed)
    J, eps_r, sigma = draw_base(rng, B, n1, n2, n3)
    mask = ellipsoid_mask(n1, n2, n3)
    chi = contrast_from_tissue(eps_r, sigma, mask, freq_hz)
    wl = Workload(name=name, n=n, h=h, freq_hz=freq_hz, tol_svd=tol_svd, seed=seed,
                  J=J, eps_r=eps_r, sigma=sigma, mask=mask, chi=chi)
    if incident == "plane":
        wl.einc = plane_wave_x(n1, n2, n3, h, freq_hz, B=B)
    elif incident == "dipole":
        wl.dipoles = np.asarray(dipoles, dtype=np.float64)
    wl.extras["rng"] = rng
    return wl


# --- the five workloads -----------------------------------------------------

def matvec_n16():
    """Plain operator matvec at n=16 (32^3 padded), HOSVD tol 1e-8, seed 0."""
    return make("matvec n=16, tol 1e-8", 16, seed=0, tol_svd=1e-8)


def solve_n64(B=1):
    """Full solve at n=64 (128^3 padded), tol 1e-6, seed 1, x-polarised plane wave."""
    return make("solve n=64 plane wave, tol 1e-6", 64, seed=1, B=B, tol_svd=1e-6,
                incident="plane")


def dipoles_n96(count=16):
    """Batched RHS at n=96 (192^3 padded): z-dipoles on a 0.15 m ring, seed 1."""
    return make("16 ring dipoles n=96, tol 1e-6", 96, seed=1, B=1, tol_svd=1e-6,
                incident="dipole", dipoles=ring_dipoles(count))


def mixed_grids():
    """Mixed-size batch: n = 48, 64, 80, four ring dipoles each (seeds 10, 11, 12)."""
    out = []
    for n, seed in ((48, 10), (64, 11), (80, 12)):
        out.append(make(f"mixed n={n}", n, seed=seed, B=1, tol_svd=1e-6,
                        incident="dipole", dipoles=ring_dipoles(4)))
    return out


def gradient_n64(n=64, seed=2, n_probe=20):
    """Differentiable solve: target contrast with sigma raised 10% in a sub-ellipsoid.

    Extra draws after the base ones: the sub-ellipsoid centre (uniform in the
    head scaled by 0.5, box-normalised), its semi-axes (U[0.15, 0.3] times the
    head's), then ``n_probe`` voxel indices drawn uniformly from the tissue.
    """
    wl = make(f"gradient n={n}", n, seed=seed, B=1, tol_svd=1e-6, incident="plane")
    rng = wl.extras["rng"]
    n1, n2, n3 = wl.n
    while True:
        c = rng.uniform(-1.0, 1.0, size=3) * 0.5 * np.asarray(HEAD_SEMI_AXES)
        if np.sum((c / np.asarray(HEAD_SEMI_AXES)) ** 2) <= 0.25:
            break
    semi = rng.uniform(0.15, 0.3, size=3) * np.asarray(HEAD_SEMI_AXES)
    sub = ellipsoid_mask(n1, n2, n3, semi=tuple(semi), centre=tuple(c)) & wl.mask
    sigma_t = np.where(sub, wl.sigma * 1.1, wl.sigma)
    wl.extras["chi_target"] = contrast_from_tissue(wl.eps_r, sigma_t, wl.mask, wl.freq_hz)
    wl.extras["sub_mask"] = sub
    support = np.flatnonzero(wl.mask.ravel())
    wl.extras["probe_voxels"] = rng.choice(support, size=n_probe, replace=False)
    return wl


def memory_n256(count=8):
    """Memory headline at n=256 (512^3 padded), tol 1e-6, seed 3, 8 ring dipoles."""
    return make("8 ring dipoles n=256, tol 1e-6", 256, seed=3, B=1, tol_svd=1e-6,
                incident="dipole", dipoles=ring_dipoles(count))


def sphere(n, edge=0.3, radius=0.15, eps_r=65.0, sigma=0.6, freq_hz=FREQ_7T_HZ, tol_svd=1e-8):
    """The refinement study's scatterer (Sec. VI.D): a homogeneous sphere of radius
    0.15 m (eps_r = 65, sigma = 0.6 S/m) centred in a cube of edge 0.3 m resolved
    by n voxels per axis, lit by the x-polarised plane wave.  No random draws."""
    h = edge / n
    x = voxel_centres(n, h)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    mask = X ** 2 + Y ** 2 + Z ** 2 <= radius ** 2
    er = np.full((n, n, n), eps_r)
    sg = np.full((n, n, n), sigma)
    wl = Workload(name=f"sphere n={n}", n=(n, n, n), h=h, freq_hz=freq_hz, tol_svd=tol_svd,
                  seed=-1, J=np.zeros((1, 3, n, n, n), dtype=np.complex128), eps_r=er,
                  sigma=sg, mask=mask, chi=contrast_from_tissue(er, sg, mask, freq_hz))
    wl.einc = plane_wave_x(n, n, n, h, freq_hz)
    return wl
