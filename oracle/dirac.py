"""Wilson-Dirac operator on a 4-d periodic lattice, antiperiodic in time (FP64).

Conventions (Sec. III names the Wilson-Dirac operator M but does not write it out;
the explicit operator is the standard Wilson form):

  (D psi)(x) = psi(x) - kappa * sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                                        + (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu) ]

with every hop across the t = Lt-1 <-> 0 boundary multiplied by -1.  H is the
bracketed hopping term, D = 1 - kappa H and G = D^{-1} (Eq. loop uses G).

Arrays: spinors ``[..., Lt, Lz, Ly, Lx, 4, 3]``; gauge ``[Lt, Lz, Ly, Lx, 4, 3, 3]``.
Gamma matrices: DeGrand-Rossi (chiral) basis; the paper does not fix one.
"""
from __future__ import annotations

import numpy as np

# gamma_1..gamma_4 in the DeGrand-Rossi basis.
GAMMA = np.array(
    [
        [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
        [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
        [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
    ],
    dtype=np.complex128,
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
IDENT4 = np.eye(4, dtype=np.complex128)

# The insertions of Eq. (loop): Gamma = 1, gamma_5, gamma_mu -- in this order.
GAMMA_SET = np.stack([IDENT4, GAMMA5, GAMMA[0], GAMMA[1], GAMMA[2], GAMMA[3]])
GAMMA_NAMES = ("1", "g5", "g1", "g2", "g3", "g4")

# spinor array axis of direction mu (x, y, z, t -> Lx, Ly, Lz, Lt axes)
_SPINOR_AXIS = (-3, -4, -5, -6)


def dims_of(U):
    lt, lz, ly, lx = U.shape[:4]
    return (lx, ly, lz, lt)


def _monomial(g):
    """(perm, phase) with g[s, perm[s]] = phase[s] the only nonzero of row s, or None."""
    perm = np.argmax(np.abs(g) > 0, axis=1)
    phase = g[np.arange(4), perm]
    if np.count_nonzero(g) != 4 or not np.allclose(g, _from_monomial(perm, phase), atol=0):
        return None
    return perm, phase


def _from_monomial(perm, phase):
    m = np.zeros((4, 4), dtype=np.complex128)
    m[np.arange(4), perm] = phase
    return m


def spin_mul(g, psi):
    """(g psi)_s = sum_t g[s, t] psi_t for a 4x4 spin matrix g (psi: [..., 4, 3])."""
    mono = _monomial(g)
    if mono is None:
        return np.matmul(g, psi)
    perm, phase = mono
    return psi[..., perm, :] * phase[:, None]


def colour_mul(u, psi):
    """(u psi)_{s,a} = sum_b u[..., a, b] psi_{s,b}; u: [L..., 3, 3], psi: [L..., n, 3]."""
    return np.matmul(psi, np.swapaxes(u, -1, -2))


def colour_mul_dag(u, psi):
    """(u^+ psi)_{s,a} = sum_b conj(u[..., b, a]) psi_{s,b}."""
    return np.matmul(psi, np.conj(u))


def hop(U, psi):
    """H psi: the hopping term of the Wilson operator (antiperiodic in t).

    psi: [..., Lt, Lz, Ly, Lx, 4, 3].  Internally the batch axes are moved
    behind the lattice axes so that one 3x3 colour matrix per site multiplies
    all spin components of all batch members at once.
    """
    bshape = psi.shape[:-6]
    lat = psi.shape[-6:-2]
    nb = int(np.prod(bshape)) if bshape else 1
    p = np.moveaxis(psi.reshape((nb,) + psi.shape[-6:]), 0, 4)  # (Lt,Lz,Ly,Lx,nb,4,3)
    p = p.reshape(lat + (nb * 4, 3))
    out = np.zeros(lat + (nb, 4, 3), dtype=np.complex128)
    for mu in range(4):
        ax = 3 - mu  # lattice axis of direction mu (t, z, y, x order)
        Umu = U[..., mu, :, :]
        # forward hop: (1 - gamma_mu) U_mu(x) psi(x + mu)
        fwd = np.roll(p, -1, axis=ax)
        if mu == 3:
            fwd[-1] *= -1.0
        uf = colour_mul(Umu, fwd).reshape(lat + (nb, 4, 3))
        out += uf - spin_mul(GAMMA[mu], uf)
        # backward hop: (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu)
        ub = colour_mul_dag(Umu, p)
        bwd = np.roll(ub, 1, axis=ax)
        if mu == 3:
            bwd[0] *= -1.0
        bwd = bwd.reshape(lat + (nb, 4, 3))
        out += bwd + spin_mul(GAMMA[mu], bwd)
    out = np.moveaxis(out, 4, 0).reshape(bshape + lat + (4, 3))
    return out


def apply_D(U, kappa, psi):
    """D psi = psi - kappa H psi."""
    return psi - kappa * hop(U, psi)


def apply_Ddag(U, kappa, psi):
    """D^+ psi, using D^+ = gamma5 D gamma5 (gamma5-hermiticity, pinned by test)."""
    return spin_mul(GAMMA5, apply_D(U, kappa, spin_mul(GAMMA5, psi)))


def parity_masks(dims):
    """(even, odd) masks of shape (Lt, Lz, Ly, Lx, 1, 1); parity = (x+y+z+t) mod 2."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    par = (x + y + z + t) % 2
    even = (par == 0).astype(np.float64)[..., None, None]
    return even, 1.0 - even


def schur_apply(U, kappa, v_e, masks):
    """D_hat v_e = v_e - kappa^2 H_eo H_oe v_e on even sites (v_e zero on odd sites)."""
    even, odd = masks
    return v_e - kappa * kappa * even * hop(U, odd * hop(U, v_e))


def prepare_source(U, kappa, b, masks):
    """Schur right-hand side  b_hat_e = b_e + kappa H_eo b_o."""
    even, odd = masks
    return even * (b + kappa * hop(U, odd * b))


def reconstruct_odd(U, kappa, x_e, b, masks):
    """Full solution from the even half: x_o = b_o + kappa H_oe x_e."""
    even, odd = masks
    return even * x_e + odd * (b + kappa * hop(U, x_e))


def plaquette(U):
    """P = (1 / (18 V)) sum_{x, mu<nu} Re Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+.

    Periodic link products (no fermion boundary sign enters the gauge action).
    """
    lt, lz, ly, lx = U.shape[:4]
    axis = (3, 2, 1, 0)  # lattice axis of direction mu in a gauge array
    total = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            umu = U[..., mu, :, :]
            unu = U[..., nu, :, :]
            unu_xpmu = np.roll(unu, -1, axis=axis[mu])
            umu_xpnu = np.roll(umu, -1, axis=axis[nu])
            p = umu @ unu_xpmu @ np.conj(np.swapaxes(umu_xpnu, -1, -2)) @ np.conj(np.swapaxes(unu, -1, -2))
            total += np.trace(p, axis1=-2, axis2=-1).real.sum()
    return total / (18.0 * lt * lz * ly * lx)


def inner(a, b):
    """<a, b> = sum conj(a) b over the lattice and spin-colour indices (batched)."""
    return np.sum(np.conj(a) * b, axis=(-6, -5, -4, -3, -2, -1))


def norm2(a):
    return np.sum(np.abs(a) ** 2, axis=(-6, -5, -4, -3, -2, -1))
