"""Dense 12V x 12V Wilson-Dirac matrix for tiny lattices (2^4, 4^4).

Built entry by entry from the hopping definition (one 3x3 colour block times
a 4x4 spin factor per link and direction), independently of the array
stencil in ``dirac.hop``.  Index of (site, spin, colour) = 12*site + 3*spin +
colour with site = x + Lx*(y + Ly*(z + Lz*t)).

Used as the dense reference: numpy.linalg
inversion / LU of this matrix gives G exactly (to rounding).
"""
from __future__ import annotations

import numpy as np

from .dirac import GAMMA, IDENT4


def site_index(dims, x, y, z, t):
    lx, ly, lz, lt = dims
    return x + lx * (y + ly * (z + lz * t))


def dense_hop(U, dims):
    """Dense matrix of H (antiperiodic in t)."""
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    H = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    L = (lx, ly, lz, lt)
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    c = [x, y, z, t]
                    i = site_index(dims, x, y, z, t)
                    for mu in range(4):
                        f = list(c)
                        f[mu] = (c[mu] + 1) % L[mu]
                        sign = -1.0 if (mu == 3 and c[3] == lt - 1) else 1.0
                        j = site_index(dims, *f)
                        u = U[t, z, y, x, mu]
                        # forward: row site x, column site x+mu
                        H[12 * i:12 * i + 12, 12 * j:12 * j + 12] += sign * np.kron(IDENT4 - GAMMA[mu], u)
                        # backward: row site x+mu, column site x, with U_mu(x)^+
                        H[12 * j:12 * j + 12, 12 * i:12 * i + 12] += sign * np.kron(IDENT4 + GAMMA[mu], u.conj().T)
    return H


def dense_D(U, kappa, dims):
    H = dense_hop(U, dims)
    return np.eye(H.shape[0], dtype=np.complex128) - kappa * H


def to_vec(psi):
    """Spinor array (..., Lt, Lz, Ly, Lx, 4, 3) -> (..., 12V) vector in dense index order."""
    return psi.reshape(psi.shape[:-6] + (-1,))


def from_vec(v, dims):
    lx, ly, lz, lt = dims
    return v.reshape(v.shape[:-1] + (lt, lz, ly, lx, 4, 3))
