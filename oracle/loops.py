"""Disconnected loops L(x) = Tr[Gamma G(x;x)] (Eq. loop), exact and stochastic.

* exact: G(x;x) column (beta, b) is the solution phi of D phi = e_{x,beta,b}
  at site x (point source); L_Gamma(x) = sum_{alpha,beta,a} Gamma[beta, alpha]
  G(x;x)[(alpha,a), (beta,a)].
* stochastic (Eq. loop stochastic): L(x) = (1/N_r) sum_r sum_d
  xi_d(x)^+ Gamma phi_d(x) with phi_d = D^{-1} xi_d over the dilution pieces d
  of noise vector r (the pieces of one vector are summed, not averaged).
* truncated solver method (Sec. II; Bali, Collins, Schafer, CPC 181 (2010)
  1570): L = (1/N_LP) sum_{r in LP} xi_r^+ Gamma phi_r^{LP}
           + (1/N_HP) sum_{r in HP} xi_r^+ Gamma (phi_r^{HP} - phi_r^{LP}),
  with the HP set drawn from stream 1 and phi^{LP} from the same truncated
  solver on both sets.

Per-time-slice loops are sums (not averages) over the sites of a time slice;
momentum-projected loops weight each site with e^{+i p.x} (the sink phase of
the disconnected correlator, Sec. III).
Gamma order: 1, gamma5, gamma1, gamma2, gamma3, gamma4.

Parity: pinned by the free-field momentum sum, the hopping expansion to
O(kappa^4), gauge invariance, reality and charge-conjugation properties, and
the reduction of fully (site-)diluted noise to the exact loop
(tests/test_oracle_loops.py, tests/test_oracle_tsm.py).  The TSM correction's
weight 1/N_HP and sign are pinned by single-site pieces (t+s+c and cubic
dilution on 2^3 x 4), where the LP estimate is the same truncated diagonal for
every noise vector and the TSM estimate must equal the exact loops.
"""
from __future__ import annotations

import numpy as np

from .dirac import GAMMA_SET
from .philox import diluted_sources, z2_noise, DIL_NONE
from .solver import solve


def contract(src, sol):
    """Per-site sum over the leading batch of src(x)^+ Gamma sol(x), all Gammas.

    src, sol: (n, Lt, Lz, Ly, Lx, 4, 3).  Returns (Lt, Lz, Ly, Lx, 6) complex.
    """
    return np.einsum("n...ac,gab,n...bc->...g", np.conj(src), GAMMA_SET, sol)


def per_timeslice(per_site):
    """Sum a (Lt, Lz, Ly, Lx, 6) per-site array over each time slice -> (Lt, 6)."""
    return per_site.sum(axis=(1, 2, 3))


def point_source(dims, site_txyz, spin, colour):
    """e_{x, spin, colour}: one at site (t, z, y, x), zero elsewhere."""
    lx, ly, lz, lt = dims
    e = np.zeros((lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    t, z, y, x = site_txyz
    e[t, z, y, x, spin, colour] = 1.0
    return e


def exact_propagator_diag(U, kappa, dims, sites, tol=1e-12):
    """G(x;x) as (n_sites, 4, 3, 4, 3) [alpha, a, beta, b] for the listed (t,z,y,x) sites."""
    out = np.zeros((len(sites), 4, 3, 4, 3), dtype=np.complex128)
    for i, s in enumerate(sites):
        srcs = np.stack([point_source(dims, s, beta, b) for beta in range(4) for b in range(3)])
        phi, info = solve(U, kappa, srcs, tol=tol)
        t, z, y, x = s
        # phi[(beta,b)] at site x is column (beta,b) of G(x;x)
        col = phi[:, t, z, y, x]  # (12, 4, 3) = [(beta,b), alpha, a]
        out[i] = np.transpose(col.reshape(4, 3, 4, 3), (2, 3, 0, 1))
    return out


def loops_from_G(Gxx):
    """L_Gamma = Tr[Gamma G(x;x)] from (n, 4, 3, 4, 3) diagonal blocks -> (n, 6)."""
    return np.einsum("gba,nacbc->ng", GAMMA_SET, Gxx)


def exact_loops(U, kappa, dims, sites, tol=1e-12):
    """Exact L_Gamma(x) (n_sites, 6) from 12 point-source solves per site."""
    return loops_from_G(exact_propagator_diag(U, kappa, dims, sites, tol))


def exact_loops_dense(U, kappa):
    """Exact L_Gamma(x) at every site (Lt, Lz, Ly, Lx, 6) from the dense inverse of D.

    For lattices small enough for a dense 12V x 12V inverse (4^4: 3072^2):
    G(x;x) is the 12x12 diagonal block of numpy.linalg.inv(D).
    """
    from .dense import dense_D
    from .dirac import dims_of
    dims = dims_of(U)
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    G = np.linalg.inv(dense_D(U, kappa, dims))
    blocks = np.stack([G[12 * i:12 * i + 12, 12 * i:12 * i + 12] for i in range(V)]).reshape(V, 4, 3, 4, 3)
    return loops_from_G(blocks).reshape(lt, lz, ly, lx, 6)


def stochastic_loops(U, kappa, dims, seed, noise_indices, scheme, tol=1e-10, stream=0):
    """Eq. (loop stochastic) with dilution; returns per-site (Lt,Lz,Ly,Lx,6) loops."""
    acc = None
    for r in noise_indices:
        srcs = diluted_sources(dims, seed, r, scheme, stream)
        phi, _ = solve(U, kappa, srcs, tol=tol)
        c = contract(srcs, phi)
        acc = c if acc is None else acc + c
    return acc / len(noise_indices)


def tsm_loops(U, kappa, dims, seed, n_lp, n_hp, tol_lp, tol_hp, scheme=DIL_NONE):
    """Truncated solver method estimate, per site (Lt,Lz,Ly,Lx,6).

    LP vectors are noise indices 0..n_lp-1 of stream 0; HP correction vectors
    are noise indices 0..n_hp-1 of stream 1, each solved at both tolerances.
    """
    lp = stochastic_loops(U, kappa, dims, seed, range(n_lp), scheme, tol_lp, stream=0)
    corr = None
    for r in range(n_hp):
        srcs = diluted_sources(dims, seed, r, scheme, stream=1)
        phi_hp, _ = solve(U, kappa, srcs, tol=tol_hp)
        phi_lp, _ = solve(U, kappa, srcs, tol=tol_lp)
        c = contract(srcs, phi_hp - phi_lp)
        corr = c if corr is None else corr + c
    return lp + corr / n_hp


def momentum_loops(per_site, moms):
    """Momentum-projected loops L_Gamma(p, t) = sum_{x in t} e^{+i p.x} L_Gamma(x).

    The sink-side phase of the disconnected correlator (Sec. III, Eq. for D_AB)
    and of the current insertion (Eq. 3-point).  per_site: (Lt, Lz, Ly, Lx, 6);
    moms: integer triples (n_x, n_y, n_z) with p_i = 2 pi n_i / L_i.
    Returns (n_mom, Lt, 6) complex.
    """
    lt, lz, ly, lx, ng = per_site.shape
    z, y, x = np.meshgrid(np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    out = np.zeros((len(moms), lt, ng), dtype=np.complex128)
    for m, (nx, ny, nz) in enumerate(moms):
        phase = np.exp(2j * np.pi * (nx * x / lx + ny * y / ly + nz * z / lz))
        for t in range(lt):
            out[m, t] = (phase[..., None] * per_site[t]).sum(axis=(0, 1, 2))
    return out


def disconnected_correlator(loops_p, loops_mp, l3, unbiased=True):
    """Disconnected two-point function D_AB(p, t) (Sec. III, Eq. for D_AB).

    D_AB(p, t) = 1/(L^3 Lt) sum_t' < L_A(p, t + t') L_B(-p, t') >, averaged
    over the source time t' (time-translation invariance).  loops_p /
    loops_mp: (N, Lt, 6) loops at momentum p / -p of N noise vectors (or N = 1
    exact loops).  unbiased: average over ordered pairs of distinct vectors
    r != r' (so no noise enters squared); otherwise over all N^2 pairs, which
    for N = 1 is the plain product.  Returns (Lt, 6, 6) complex [t, A, B].
    """
    n, lt, ng = loops_p.shape
    if unbiased and n < 2:
        raise ValueError("the unbiased estimator needs at least two noise vectors")
    d = np.zeros((lt, ng, ng), dtype=np.complex128)
    for t in range(lt):
        for tp in range(lt):
            for r in range(n):
                for rp in range(n):
                    if unbiased and r == rp:
                        continue
                    d[t] += np.outer(loops_p[r, (t + tp) % lt], loops_mp[rp, tp])
    pairs = n * (n - 1) if unbiased else n * n
    return d / (l3 * lt * pairs)


__all__ = ["momentum_loops", "disconnected_correlator", "contract", "per_timeslice", "point_source", "exact_propagator_diag",
           "loops_from_G", "exact_loops", "exact_loops_dense", "stochastic_loops", "tsm_loops", "z2_noise"]
