"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module only *draws* inputs: gauge fields, Gaussian weights and Gaussian
test vectors.  It contains none of the method's arithmetic (no Dirac operator,
no solver, no noise generator, no contraction), so both the oracle and the GPU
path may use it without sharing any of the computation they are compared on.

Layouts (canonical, also the C ABI layout):

* gauge field ``U[t, z, y, x, mu, a, b]`` complex128, ``mu = 0..3`` for the
  x, y, z, t directions; ``U[..., mu, :, :]`` is the link from site x to
  x + mu-hat.  Flattened, the site index is ``x + Lx*(y + Ly*(z + Lz*t))``.
* colour-spinor field ``psi[..., t, z, y, x, spin, colour]`` complex128.

``dims`` is always ``(Lx, Ly, Lz, Lt)``.

The paper's ensemble (SESAM/TchiL, N_f=2 Wilson, 16^3 x 32 at kappa=0.157,
Sec. II) is not available; these synthetic fields of the same lattice shapes
stand in for it.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lattice_shape",
    "haar_su3_field",
    "eps_su3_field",
    "unit_gauge_field",
    "gaussian_weights",
    "gaussian_spinors",
    "random_gauge_transform",
]


def lattice_shape(dims):
    """Array shape (Lt, Lz, Ly, Lx) of a lattice with ``dims=(Lx, Ly, Lz, Lt)``."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _haar_su3(rng, n):
    """n Haar-distributed SU(3) matrices.

    Complex Gaussian 3x3 -> QR with the phases of diag(R) moved into Q
    (Mezzadri, Notices AMS 54 (2007) 592) gives Haar U(3); dividing by the
    principal cube root of the determinant maps it to SU(3) and commutes with
    left multiplication by SU(3), so the result is Haar on SU(3).
    """
    z = rng.standard_normal((n, 3, 3, 2))
    z = (z[..., 0] + 1j * z[..., 1]) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    ph = d / np.abs(d)
    q = q * ph[:, None, :]
    det = np.linalg.det(q)
    q = q / np.exp(1j * np.angle(det) / 3.0)[:, None, None]
    return q


def haar_su3_field(dims, seed):
    """Haar-random SU(3) gauge field, drawn in [t][z][y][x][mu] order."""
    shp = lattice_shape(dims)
    n = int(np.prod(shp)) * 4
    rng = np.random.default_rng(seed)
    u = _haar_su3(rng, n)
    return u.reshape(shp + (4, 3, 3))


def _gell_mann():
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1] = -1j
    lam[1, 1, 0] = 1j
    lam[2, 0, 0] = 1
    lam[2, 1, 1] = -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2] = -1j
    lam[4, 2, 0] = 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2] = -1j
    lam[6, 2, 1] = 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3.0)
    lam[7, 2, 2] = -2 / np.sqrt(3.0)
    return lam


def eps_su3_field(dims, eps, seed):
    """Near-unit gauge field U = exp(i*eps*H), H = sum_a h_a lambda_a / 2.

    h_a ~ N(0, 1) drawn in [t][z][y][x][mu][a] order; the exponential is taken
    through the eigen-decomposition of the Hermitian traceless H.
    """
    shp = lattice_shape(dims)
    n = int(np.prod(shp)) * 4
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((n, 8))
    H = np.einsum("na,aij->nij", h, _gell_mann()) / 2.0
    w, v = np.linalg.eigh(H)
    u = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * eps * w), v.conj())
    return u.reshape(shp + (4, 3, 3))


def unit_gauge_field(dims):
    """Free field U = 1."""
    shp = lattice_shape(dims)
    u = np.zeros(shp + (4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def random_gauge_transform(dims, seed):
    """Haar SU(3) matrix g(x) per site, shape (Lt, Lz, Ly, Lx, 3, 3)."""
    shp = lattice_shape(dims)
    rng = np.random.default_rng(seed)
    return _haar_su3(rng, int(np.prod(shp))).reshape(shp + (3, 3))


def gaussian_weights(n, seed):
    """n real N(0, 1) weights (the w_t of a weighted sum of time-slice loops)."""
    return np.random.default_rng(seed).standard_normal(n)


def gaussian_spinors(dims, nrhs, seed):
    """nrhs complex Gaussian colour-spinor fields, shape (nrhs, Lt, Lz, Ly, Lx, 4, 3)."""
    shp = lattice_shape(dims)
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((nrhs,) + shp + (4, 3, 2))
    return z[..., 0] + 1j * z[..., 1]
