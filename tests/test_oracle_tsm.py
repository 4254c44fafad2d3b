"""Pins of the oracle's stochastic estimator and truncated solver method (Sec. II, Sec. III).

* unbiasedness: the time+spin+colour diluted estimator of the per-time-slice
  loops agrees with the exact per-time-slice loops as a z-test over noise vectors;
* TSM with LP tolerance = HP tolerance has a zero correction;
* TSM whose HP set is the LP set telescopes to the pure HP estimator.
"""
import numpy as np

from lattice_inputs import haar_su3_field
from oracle.loops import exact_loops, stochastic_loops, tsm_loops, contract, per_timeslice
from oracle.philox import DIL_TSC, DIL_NONE, diluted_sources
from oracle.solver import solve

DIMS = (2, 2, 2, 4)


def test_diluted_estimator_unbiased_per_timeslice():
    U = haar_su3_field(DIMS, 0)
    kappa = 0.125
    lx, ly, lz, lt = DIMS
    sites = [(t, z, y, x) for t in range(lt) for z in range(lz) for y in range(ly) for x in range(lx)]
    ex = exact_loops(U, kappa, DIMS, sites, tol=1e-12).reshape(lt, lz * ly * lx, 6).sum(axis=1)
    n = 24
    per = []
    for r in range(n):
        per.append(per_timeslice(stochastic_loops(U, kappa, DIMS, 5, [r], DIL_TSC, tol=1e-12)))
    per = np.array(per)  # (n, lt, 6)
    for part in (np.real, np.imag):
        d = part(per.mean(axis=0) - ex)
        e = part(per).std(axis=0, ddof=1) / np.sqrt(n)
        mask = e > 1e-12
        z = np.abs(d[mask]) / e[mask]
        assert np.all(z < 5.0), z.max()
        # where the diluted estimator has no noise it is exact
        assert np.all(np.abs(d[~mask]) < 1e-9)


def test_tsm_equal_tolerances_gives_zero_correction():
    U = haar_su3_field(DIMS, 1)
    a = tsm_loops(U, 0.12, DIMS, 3, n_lp=2, n_hp=2, tol_lp=1e-9, tol_hp=1e-9)
    b = stochastic_loops(U, 0.12, DIMS, 3, range(2), DIL_NONE, tol=1e-9)
    assert np.max(np.abs(a - b)) < 1e-14


def test_tsm_same_sets_telescopes_to_hp():
    """With the HP set equal to the LP set: LP mean + (HP - LP) mean = HP mean."""
    U = haar_su3_field(DIMS, 2)
    kappa = 0.12
    lp_tol, hp_tol = 1e-2, 1e-12
    acc_lp = 0
    acc_corr = 0
    acc_hp = 0
    for r in range(3):
        src = diluted_sources(DIMS, 7, r, DIL_NONE, stream=1)
        phi_lp, _ = solve(U, kappa, src, tol=lp_tol)
        phi_hp, _ = solve(U, kappa, src, tol=hp_tol)
        acc_lp = acc_lp + contract(src, phi_lp)
        acc_corr = acc_corr + contract(src, phi_hp - phi_lp)
        acc_hp = acc_hp + contract(src, phi_hp)
    assert np.max(np.abs((acc_lp + acc_corr) - acc_hp)) < 1e-12
    # and the LP-only estimate really is different (truncated)
    assert np.max(np.abs(acc_lp - acc_hp)) > 1e-6


def test_tsm_with_single_site_pieces_equals_exact_loops():
    """The weight and sign of the TSM correction (Sec. II; Bali et al.).

    On 2^3 x 4 with time+spin+colour and cubic dilution every piece is one
    (site, spin, colour) times a phase c with |c| = 1.  BiCGstab from x = 0 is
    equivariant under b -> c b (every Krylov vector scales by c, every scalar is
    unchanged, the relative stopping rule is scale free), so the low-precision
    estimate is the same truncated diagonal for every noise vector of either
    stream.  The LP mean over 3 vectors plus the (HP - LP) mean over 2 vectors
    must then reproduce the exact loops: a correction weighted 1/n_lp instead of
    1/n_hp, dropped, or added with the wrong sign leaves the truncation error.
    """
    from oracle.loops import exact_loops_dense
    from oracle.philox import DIL_CUBE
    U = haar_su3_field(DIMS, 0)
    kappa = 0.125
    scheme = DIL_TSC | DIL_CUBE
    exact = exact_loops_dense(U, kappa)
    tsm = tsm_loops(U, kappa, DIMS, 11, n_lp=3, n_hp=2, tol_lp=1e-2, tol_hp=1e-13, scheme=scheme)
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(tsm - exact)) < 1e-10 * scale
    # teeth: the low-precision estimate alone is visibly truncated
    lp_only = stochastic_loops(U, kappa, DIMS, 11, range(3), scheme, tol=1e-2)
    assert np.max(np.abs(lp_only - exact)) > 1e-4 * scale
