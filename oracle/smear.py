"""Gaussian quark smearing and APE link smearing (Sec. III, smearing of the
interpolating fields), plain FP64.  Test infrastructure only.

Gaussian smearing (Sec. III): within each time slice
    q_smear = F q,   F = (1 + alpha H)^n,
    (H q)(x) = sum_{i=1,2,3} [ U_i(x) q(x + i) + U_i(x - i)^+ q(x - i) ]
(spatial hops only, colour only: every spin component is smeared alike;
periodic in space).  The paper uses alpha = 4, n = 50.  With ``normalise`` each
factor is divided by (1 + 6 alpha), which changes only the overall scale (the
free-field F(p = 0) becomes 1); the paper's F is the unnormalised one.

APE smearing of the spatial links entering H (Sec. III; the paper does not
write the formula or its parameters).  Reading used: n steps of
    U_i'(x) = P[ U_i(x) + alpha sum_{j != i, spatial} S_ij(x) ],
    S_ij(x) = U_j(x) U_i(x + j) U_j(x + i)^+ + U_j(x - j)^+ U_i(x - j) U_j(x - j + i)
with the four spatial staples, temporal links untouched, and P the projection
onto SU(3): the unitary polar factor W = V (V^+ V)^{-1/2} (from the SVD
V = A S B^+, W = A B^+), divided by the principal cube root of det W.

Pins (tests/test_oracle_smear.py): free-field plane waves are eigenvectors
with F(p) = (1 + 2 alpha sum_i cos p_i)^n; gauge covariance of both smearings;
time slices stay independent; alpha = 0 and the unit field are fixed points of
APE; P returns SU(3) matrices, leaves c W (c > 0, W in SU(3)) at W, and its
unitary factor maximises Re Tr(W^+ V) over U(3).
"""
from __future__ import annotations

import numpy as np

from .dirac import colour_mul, colour_mul_dag

# spinor axis of spatial direction i (x, y, z) in [..., Lt, Lz, Ly, Lx, 4, 3]
_SP_AXIS = (-3, -4, -5)
# gauge-array axis of spatial direction i in [Lt, Lz, Ly, Lx, 4, 3, 3]
_U_AXIS = (3, 2, 1)


def hop3(U, q):
    """(H q)(x) = sum_i U_i(x) q(x + i) + U_i(x - i)^+ q(x - i), spatial i only."""
    bshape = q.shape[:-6]
    lat = q.shape[-6:-2]
    nb = int(np.prod(bshape)) if bshape else 1
    p = np.moveaxis(q.reshape((nb,) + q.shape[-6:]), 0, 4).reshape(lat + (nb * 4, 3))
    out = np.zeros(lat + (nb * 4, 3), dtype=np.complex128)
    for i in range(3):
        ax = 3 - i
        Ui = U[..., i, :, :]
        out += colour_mul(Ui, np.roll(p, -1, axis=ax))
        out += np.roll(colour_mul_dag(Ui, p), 1, axis=ax)
    out = np.moveaxis(out.reshape(lat + (nb, 4, 3)), 4, 0).reshape(bshape + lat + (4, 3))
    return out


def gaussian_smear(U, q, alpha, n, normalise=False):
    """F q with F = (1 + alpha H)^n (divided by (1 + 6 alpha)^n if normalise)."""
    out = np.array(q, dtype=np.complex128, copy=True)
    for _ in range(n):
        out = out + alpha * hop3(U, out)
        if normalise:
            out = out / (1.0 + 6.0 * alpha)
    return out


def project_su3(V):
    """P(V): unitary polar factor of V (via SVD) divided by the cube root of its determinant."""
    A, _, Bh = np.linalg.svd(V)
    W = A @ Bh
    det = np.linalg.det(W)
    phase = np.exp(-1j * np.angle(det) / 3.0)
    return W * phase[..., None, None]


def staples(U, i):
    """Sum of the four spatial staples around U_i(x), j != i spatial."""
    S = np.zeros(U.shape[:4] + (3, 3), dtype=np.complex128)
    Ui = U[..., i, :, :]
    for j in range(3):
        if j == i:
            continue
        Uj = U[..., j, :, :]
        ai, aj = _U_AXIS[i], _U_AXIS[j]
        Ui_xj = np.roll(Ui, -1, axis=aj)          # U_i(x + j)
        Uj_xi = np.roll(Uj, -1, axis=ai)          # U_j(x + i)
        S += Uj @ Ui_xj @ np.conj(np.swapaxes(Uj_xi, -1, -2))
        Uj_mj = np.roll(Uj, 1, axis=aj)           # U_j(x - j)
        Ui_mj = np.roll(Ui, 1, axis=aj)           # U_i(x - j)
        Uj_mj_pi = np.roll(Uj_mj, -1, axis=ai)    # U_j(x - j + i)
        S += np.conj(np.swapaxes(Uj_mj, -1, -2)) @ Ui_mj @ Uj_mj_pi
    return S


def ape_smear(U, alpha, n):
    """n APE steps on the spatial links (temporal links unchanged)."""
    out = np.array(U, dtype=np.complex128, copy=True)
    for _ in range(n):
        new = out.copy()
        for i in range(3):
            new[..., i, :, :] = project_su3(out[..., i, :, :] + alpha * staples(out, i))
        out = new
    return out


__all__ = ["hop3", "gaussian_smear", "project_su3", "staples", "ape_smear"]
