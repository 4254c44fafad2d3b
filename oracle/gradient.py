"""Gradients of loops by forward and gamma5-adjoint solves (FP64).

The paper computes no gradients; these are the derivatives of its loops:

* d/dkappa sum_x Tr[Gamma G(x;x)] = Tr[Gamma G H G]  (dD/dkappa = -H).
  For fixed noise the estimator sum_d xi_d^+ Gamma G xi_d has the exact
  derivative sum_d chi_d^+ H phi_d with phi_d = G xi_d and
  chi_d = G^+ Gamma^+ xi_d = gamma5 G gamma5 Gamma^+ xi_d  (D^+ = gamma5 D gamma5).
* gauge-link gradient of S = Re sum_t w_t L_1(t) = Re sum_d xi_d^+ W G xi_d
  (W = w_{t(x)}): with phi_d = G xi_d, chi_d = gamma5 G gamma5 W xi_d,
      dS = Re kappa sum_d chi_d^+ dH phi_d.
  Reported as the complex matrix g = dS/dRe U + i dS/dIm U per link (the
  convention torch.autograd uses for complex leaves), so that
  dS = Re sum conj(g_ij) dU_ij.  For the link U_mu(x) with boundary sign s:
      g = kappa s ( X^* + Y^T ),
      X_ij = sum_{ab} chi(x)^*_{a i} (1 - gamma_mu)_{ab} phi(x+mu)_{b j},
      Y_ij = sum_{ab} chi(x+mu)^*_{a i} (1 + gamma_mu)_{ab} phi(x)_{b j}.
  The Lie derivative along T_a = i lambda_a / 2 is Re sum conj(g) (T_a U).

Dense references (exact, no noise): Tr[Gamma G H G] and the same link formula
with phi chi^+ replaced by M = G W G, on lattices small enough for a dense G.

Parity: pinned by central finite differences of the oracle's own loops
(h = 1e-5) and by full-dilution noise reproducing the dense reference
(tests/test_oracle_gradient.py).
"""
from __future__ import annotations

import numpy as np

from .dirac import GAMMA, GAMMA5, GAMMA_SET, IDENT4, hop, inner, spin_mul, dims_of
from .dense import dense_D, dense_hop
from .solver import solve

_SPINOR_AXIS = (-3, -4, -5, -6)


def _shift_fwd(psi, mu):
    """psi(x + mu) with the antiperiodic sign on the t boundary."""
    f = np.roll(psi, -1, axis=_SPINOR_AXIS[mu])
    if mu == 3:
        f[..., -1, :, :, :, :, :] *= -1.0
    return f


def weight_field(w_t, dims, srcs):
    """W xi: multiply each time slice t of srcs by w_t."""
    lt = dims[3]
    return srcs * np.asarray(w_t, dtype=np.float64).reshape((lt, 1, 1, 1, 1, 1))


def dkappa_estimator(U, kappa, srcs, gamma_index, tol=1e-12):
    """sum_d chi_d^+ H phi_d for the pieces srcs (n, Lt, Lz, Ly, Lx, 4, 3)."""
    g = GAMMA_SET[gamma_index]
    phi, _ = solve(U, kappa, srcs, tol=tol)
    y, _ = solve(U, kappa, spin_mul(GAMMA5 @ g.conj().T, srcs), tol=tol)
    chi = spin_mul(GAMMA5, y)
    return np.sum(inner(chi, hop(U, phi)))


def loop_sum_estimator(U, kappa, srcs, gamma_index, tol=1e-12):
    """sum_d xi_d^+ Gamma G xi_d = sum_x of the (undivided) loop estimator."""
    g = GAMMA_SET[gamma_index]
    phi, _ = solve(U, kappa, srcs, tol=tol)
    return np.sum(inner(srcs, spin_mul(g, phi)))


def link_grad_from_fields(U, kappa, phi, chi):
    """g_mu(x) (Lt, Lz, Ly, Lx, 4, 3, 3) from forward fields phi and adjoint fields chi (summed over n)."""
    out = np.zeros(U.shape, dtype=np.complex128)
    for mu in range(4):
        phi_f = _shift_fwd(phi, mu)
        chi_f = _shift_fwd(chi, mu)
        pm = IDENT4 - GAMMA[mu]
        pp = IDENT4 + GAMMA[mu]
        X = np.einsum("n...ai,ab,n...bj->...ij", np.conj(chi), pm, phi_f)
        Y = np.einsum("n...ai,ab,n...bj->...ij", np.conj(chi_f), pp, phi)
        out[..., mu, :, :] = kappa * (np.conj(X) + np.swapaxes(Y, -1, -2))
    return out


def link_grad_estimator(U, kappa, srcs, w_t, tol=1e-12):
    """dS/dU for S = Re sum_d xi_d^+ W G xi_d (torch complex-gradient convention)."""
    dims = dims_of(U)
    phi, _ = solve(U, kappa, srcs, tol=tol)
    y, _ = solve(U, kappa, spin_mul(GAMMA5, weight_field(w_t, dims, srcs)), tol=tol)
    chi = spin_mul(GAMMA5, y)
    return link_grad_from_fields(U, kappa, phi, chi)


def weighted_loop_estimator(U, kappa, srcs, w_t, tol=1e-12):
    """S = Re sum_d xi_d^+ W G xi_d."""
    dims = dims_of(U)
    phi, _ = solve(U, kappa, srcs, tol=tol)
    return float(np.real(np.sum(inner(weight_field(w_t, dims, srcs), phi))))


# ----------------------------------------------------------------- dense references
def dense_G(U, kappa):
    dims = dims_of(U)
    return np.linalg.inv(dense_D(U, kappa, dims))


def dense_dkappa(U, kappa, gamma_index):
    """Tr[Gamma G H G] with dense G and H."""
    dims = dims_of(U)
    G = dense_G(U, kappa)
    H = dense_hop(U, dims)
    V = G.shape[0] // 12
    Gam = np.kron(np.eye(V), np.kron(GAMMA_SET[gamma_index], np.eye(3)))
    return np.trace(Gam @ G @ H @ G)


def dense_link_grad(U, kappa, w_t):
    """dS/dU for S = Re Tr[W G] with dense G: M = G W G in place of phi chi^+."""
    dims = dims_of(U)
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    G = dense_G(U, kappa)
    wsite = np.repeat(np.asarray(w_t, dtype=np.float64), lx * ly * lz)  # site order is t-major
    W = np.repeat(wsite, 12)
    M = (G * W[None, :]) @ G
    M6 = M.reshape(lt, lz, ly, lx, 4, 3, lt, lz, ly, lx, 4, 3)
    out = np.zeros(U.shape, dtype=np.complex128)
    L = (lx, ly, lz, lt)
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    c = [x, y, z, t]
                    for mu in range(4):
                        f = list(c)
                        f[mu] = (c[mu] + 1) % L[mu]
                        s = -1.0 if (mu == 3 and t == lt - 1) else 1.0
                        fx, fy, fz, ft = f
                        # M(x+mu, x)[b j, a i] and M(x, x+mu)[b j, a i]
                        Mfx = M6[ft, fz, fy, fx, :, :, t, z, y, x]
                        Mxf = M6[t, z, y, x, :, :, ft, fz, fy, fx]
                        X = np.einsum("ab,bjai->ij", IDENT4 - GAMMA[mu], Mfx)
                        Y = np.einsum("ab,bjai->ij", IDENT4 + GAMMA[mu], Mxf)
                        out[t, z, y, x, mu] = kappa * s * (np.conj(X) + Y.T)
    return out


def dense_weighted_loop(U, kappa, w_t):
    """S = Re Tr[W G] with dense G."""
    dims = dims_of(U)
    lx, ly, lz, lt = dims
    G = dense_G(U, kappa)
    W = np.repeat(np.repeat(np.asarray(w_t, dtype=np.float64), lx * ly * lz), 12)
    return float(np.real(np.sum(W * np.diag(G))))


def su3_generators():
    """T_a = i lambda_a / 2 (anti-Hermitian generators of su(3))."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1], lam[1, 1, 0] = -1j, 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2], lam[4, 2, 0] = -1j, 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2], lam[6, 2, 1] = -1j, 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3.0)
    lam[7, 2, 2] = -2 / np.sqrt(3.0)
    return 0.5j * lam


def lie_derivative(U, grad, site_txyz, mu):
    """F^a = Re sum conj(g_ij) (T_a U)_ij for one link -> (8,) reals."""
    t, z, y, x = site_txyz
    u = U[t, z, y, x, mu]
    g = grad[t, z, y, x, mu]
    return np.array([np.real(np.sum(np.conj(g) * (T @ u))) for T in su3_generators()])
