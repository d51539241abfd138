"""Green's-function kernel of the J-block operator (eqs. (5)-(6)), FP64.

Test infrastructure: see the package docstring.

The operator N of eq. (5), curl curl of the vector potential, equals
(k0^2 + grad div) acting on the potential plus the identity.  On a uniform
voxel grid its off-voxel part is sampled at voxel-centre offsets R = (i,j,k) h
and scaled by the voxel volume h^3 (point collocation, a stand-in for the
paper's Galerkin entries of eq. (8)); the voxel's own entry is the exact
field of a uniform unit source in the equivalent sphere of radius
a = h (3 / 4 pi)^(1/3).
"""
from __future__ import annotations

import math

import numpy as np

SPEED_OF_LIGHT = 299_792_458.0

# The six unique components of the symmetric dyadic kernel, in this order.
COMPONENTS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
COMPONENT_NAMES = ("xx", "xy", "xz", "yy", "yz", "zz")


def component_index(a: int, b: int) -> int:
    """Index into COMPONENTS of the (a, b) entry of the symmetric dyad."""
    return COMPONENTS.index((min(a, b), max(a, b)))


def wavenumber(freq_hz: float) -> float:
    """k0 = omega / c = 2 pi f / c."""
    return 2.0 * math.pi * freq_hz / SPEED_OF_LIGHT


def green(r, k0):
    """Free-space Green's function of eq. (6): g = exp(-i k0 r) / (4 pi r)."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-1j * k0 * r) / (4.0 * math.pi * r)


def dyadic(R, k0):
    """(k0^2 delta_ab + d_a d_b) g(|R|) for nonzero offsets R (shape [..., 3]).

    Differentiating g twice gives, with r = |R| and Rhat = R / r,
      g [ (k0^2 - i k0/r - 1/r^2) delta_ab + (-k0^2 + 3 i k0/r + 3/r^2) Rhat_a Rhat_b ].
    Returns an array [6, ...] in COMPONENTS order.
    """
    R = np.asarray(R, dtype=np.float64)
    r = np.sqrt(np.sum(R * R, axis=-1))
    Rh = R / r[..., None]
    g = green(r, k0)
    diag = k0 * k0 - 1j * k0 / r - 1.0 / (r * r)
    dyad = -k0 * k0 + 3j * k0 / r + 3.0 / (r * r)
    out = np.empty((6,) + r.shape, dtype=np.complex128)
    for c, (a, b) in enumerate(COMPONENTS):
        out[c] = g * ((diag if a == b else 0.0) + dyad * Rh[..., a] * Rh[..., b])
    return out


def equivalent_sphere_radius(h: float) -> float:
    """Radius of the sphere with the voxel's volume h^3."""
    return h * (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)


def self_term(h: float, k0: float, mode: str = "full") -> complex:
    """Diagonal entry of the voxel's own interaction (the paper is silent on it).

    Reading: the field at the centre of a sphere of radius a carrying a
    uniform unit source.  With Phi = int_sphere g dV = k0^-2 [(1 + i k0 a)
    exp(-i k0 a) - 1] and grad grad Phi = (1/3) lap Phi I = (1/3)(-k0^2 Phi - 1) I,
      (k0^2 + grad grad) Phi = (2/3) k0^2 Phi - 1/3
                             = (2/3)(1 + i k0 a) exp(-i k0 a) - 1.
    ``mode='full'`` keeps the -1/3 depolarisation part (default); ``'pv'``
    drops it (principal value only).  Not scaled by h^3.
    """
    a = equivalent_sphere_radius(h)
    full = (2.0 / 3.0) * (1.0 + 1j * k0 * a) * np.exp(-1j * k0 * a) - 1.0
    if mode == "full":
        return complex(full)
    if mode == "pv":
        return complex(full + 1.0 / 3.0)
    raise ValueError(mode)


def toeplitz_tensor(n1: int, n2: int, n3: int, h: float, k0: float,
                    self_mode: str = "full") -> np.ndarray:
    """Defining tensors T_c[i, j, k] of the BTTB operator, offsets |i| < n1 etc.

    Returns complex128 [6, 2 n1 - 1, 2 n2 - 1, 2 n3 - 1]; entry
    [c, i + n1 - 1, j + n2 - 1, k + n3 - 1] is h^3 G_c((i, j, k) h) for a
    nonzero offset and self_term() * delta_ab at the zero offset.
    """
    i = np.arange(-(n1 - 1), n1) * h
    j = np.arange(-(n2 - 1), n2) * h
    k = np.arange(-(n3 - 1), n3) * h
    I, Jg, K = np.meshgrid(i, j, k, indexing="ij")
    R = np.stack([I, Jg, K], axis=-1)
    zero = (n1 - 1, n2 - 1, n3 - 1)
    R[zero] = (1.0, 0.0, 0.0)            # placeholder, overwritten below
    T = dyadic(R, k0) * h ** 3
    s = self_term(h, k0, self_mode)
    for c, (a, b) in enumerate(COMPONENTS):
        T[(c,) + zero] = s if a == b else 0.0
    return T


def dipole_field(points, src, k0):
    """Field of a unit z-directed point dipole at ``src``: e_a(r) = G_az(r - src).

    ``points`` has shape [..., 3]; returns [3, ...] (components x, y, z).
    The dyadic kernel is used without the voxel volume (unit moment).
    """
    R = np.asarray(points, dtype=np.float64) - np.asarray(src, dtype=np.float64)
    G = dyadic(R, k0)
    return np.stack([G[component_index(0, 2)], G[component_index(1, 2)],
                     G[component_index(2, 2)]])


def dipole_incident(n1, n2, n3, h, k0, sources):
    """Incident fields [B, 3, n1, n2, n3] of z-dipoles at ``sources`` [B, 3]."""
    x = (np.arange(n1) + 0.5 - 0.5 * n1) * h
    y = (np.arange(n2) + 0.5 - 0.5 * n2) * h
    z = (np.arange(n3) + 0.5 - 0.5 * n3) * h
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1)
    return np.stack([dipole_field(P, s, k0) for s in np.asarray(sources)])
