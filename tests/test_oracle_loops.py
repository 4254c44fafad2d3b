"""Pins of the oracle's loops L(x) = Tr[Gamma G(x;x)] (Eq. loop) and the noise estimator.

* free field: G(x;x) = (1/V) sum_p D(p)^{-1} in closed form (momentum sum);
* hopping expansion: Tr G(x;x) = 12 + kappa^4 c4(x) + O(kappa^6), with c4(x)
  computed here by brute-force enumeration of all closed 4-step walks;
* gauge invariance, reality / imaginarity from gamma5-hermiticity, charge
  conjugation U -> U^*, invariance under moving the antiperiodic boundary;
* the estimator of Eq. (loop stochastic) with noise on single
  (site, spin, colour) pieces reproduces the exact loop.
"""
import itertools

import numpy as np
import pytest

from lattice_inputs import haar_su3_field, unit_gauge_field, random_gauge_transform
from oracle import dirac
from oracle.loops import exact_loops, contract, point_source, exact_propagator_diag
from oracle.philox import z2_noise

DIMS = (4, 4, 4, 4)


def free_field_loops(dims, kappa):
    """(1/V) sum_p Tr[Gamma D(p)^{-1}] with antiperiodic time momenta."""
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    out = np.zeros(6, dtype=np.complex128)
    G6 = dirac.GAMMA_SET
    for nx, ny, nz, nt in itertools.product(range(lx), range(ly), range(lz), range(lt)):
        p = (2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz, (2 * nt + 1) * np.pi / lt)
        Dp = (1 - 2 * kappa * sum(np.cos(p))) * np.eye(4) + 2j * kappa * sum(dirac.GAMMA[m] * np.sin(p[m]) for m in range(4))
        Gp = np.linalg.inv(Dp)
        out += 3 * np.array([np.trace(g @ Gp) for g in G6])  # colour trace of the identity = 3
    return out / V


def test_free_field_closed_form():
    kappa = 0.125
    U = unit_gauge_field(DIMS)
    L = exact_loops(U, kappa, DIMS, [(0, 0, 0, 0), (3, 1, 2, 1)], tol=1e-13)
    ref = free_field_loops(DIMS, kappa)
    # scalar trace in closed form: 12/V sum_p M / (M^2 + 4 kappa^2 sum_mu sin^2 p_mu),
    # M = 1 - 2 kappa sum_mu cos p_mu
    lx, ly, lz, lt = DIMS
    scal = 0.0
    for n in itertools.product(range(lx), range(ly), range(lz), range(lt)):
        p = np.array([2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, (2 * n[3] + 1) * np.pi / lt])
        M = 1 - 2 * kappa * np.cos(p).sum()
        scal += 12 * M / (M * M + 4 * kappa ** 2 * (np.sin(p) ** 2).sum())
    assert abs(ref[0] - scal / (lx * ly * lz * lt)) < 1e-12
    for row in L:
        assert np.max(np.abs(row - ref)) < 1e-11
    assert np.max(np.abs(ref[1:])) < 1e-13  # gamma5 and gamma_mu loops vanish for U = 1


def _c4_by_walks(U, dims, site):
    """Coefficient of kappa^4 in Tr G(x;x): sum over closed 4-step walks from x of Tr[spin] Tr[colour]."""
    lx, ly, lz, lt = dims
    L = (lx, ly, lz, lt)
    steps = [(mu, +1) for mu in range(4)] + [(mu, -1) for mu in range(4)]
    x0 = list(site)  # (x, y, z, t)
    total = 0.0 + 0.0j
    for walk in itertools.product(steps, repeat=4):
        pos = list(x0)
        spin = np.eye(4, dtype=np.complex128)
        col = np.eye(3, dtype=np.complex128)
        sign = 1.0
        for mu, d in walk:
            if d > 0:
                u = U[pos[3], pos[2], pos[1], pos[0], mu]
                spin = spin @ (np.eye(4) - dirac.GAMMA[mu])
                col = col @ u
                if mu == 3 and pos[3] == lt - 1:
                    sign = -sign
                pos[mu] = (pos[mu] + 1) % L[mu]
            else:
                pos[mu] = (pos[mu] - 1) % L[mu]
                u = U[pos[3], pos[2], pos[1], pos[0], mu]
                spin = spin @ (np.eye(4) + dirac.GAMMA[mu])
                col = col @ u.conj().T
                if mu == 3 and pos[3] == lt - 1:
                    sign = -sign
        if pos == x0:
            total += sign * np.trace(spin) * np.trace(col)
    return total


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 6, 6, 6)])
def test_hopping_expansion_kappa4(dims):
    U = haar_su3_field(dims, 2)
    site = (1, 0, 3, 2)  # (x, y, z, t)
    c4 = _c4_by_walks(U, dims, site)
    txyz = (site[3], site[2], site[1], site[0])
    f = []
    ks = (0.02, 0.01)
    for k in ks:
        L1 = exact_loops(U, k, dims, [txyz], tol=1e-14)[0, 0]
        f.append((L1 - 12.0) / k ** 4)
    # (L - 12)/k^4 = c4 + c6 k^2 + ...; Richardson in k^2
    est = (f[1] * ks[0] ** 2 - f[0] * ks[1] ** 2) / (ks[0] ** 2 - ks[1] ** 2)
    assert abs(est - c4) < 1e-3 * max(1.0, abs(c4))
    assert abs(c4.imag) < 1e-12


def test_hopping_expansion_free_coefficients():
    """Free field: c4 = -1152 per site for L >= 6 and -768 on 4^4 (winding loops enter)."""
    for dims, expect in (((4, 4, 4, 4), -768.0), ((6, 6, 6, 6), -1152.0)):
        U = unit_gauge_field(dims)
        assert abs(_c4_by_walks(U, dims, (0, 0, 0, 0)) - expect) < 1e-9


def test_gauge_invariance_and_reality():
    U = haar_su3_field(DIMS, 5)
    kappa = 0.125
    sites = [(0, 0, 0, 0), (2, 3, 1, 0)]
    L = exact_loops(U, kappa, DIMS, sites, tol=1e-13)
    g = random_gauge_transform(DIMS, 6)
    axis = (3, 2, 1, 0)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(np.roll(g, -1, axis=axis[mu]), -1, -2))
    Lg = exact_loops(Ug, kappa, DIMS, sites, tol=1e-13)
    assert np.max(np.abs(L - Lg)) < 1e-10
    # Tr G, Tr g5 G real; Tr g_mu G imaginary (gamma5-hermiticity)
    assert np.max(np.abs(L[:, :2].imag)) < 1e-11
    assert np.max(np.abs(L[:, 2:].real)) < 1e-11
    assert np.max(np.abs(L[:, 2:].imag)) > 1e-4


def test_charge_conjugation_and_boundary_move():
    U = haar_su3_field(DIMS, 8)
    kappa = 0.125
    sites = [(1, 1, 2, 3)]
    L = exact_loops(U, kappa, DIMS, sites, tol=1e-13)
    Lc = exact_loops(np.conj(U), kappa, DIMS, sites, tol=1e-13)
    assert np.max(np.abs(Lc[:, :2] - L[:, :2])) < 1e-10
    assert np.max(np.abs(Lc[:, 2:] + L[:, 2:])) < 1e-10
    # move the antiperiodic sign from the t = Lt-1 -> 0 links to the t = 1 -> 2 links
    Um = U.copy()
    Um[DIMS[3] - 1, :, :, :, 3] *= -1.0
    Um[1, :, :, :, 3] *= -1.0
    Lm = exact_loops(Um, kappa, DIMS, sites, tol=1e-13)
    assert np.max(np.abs(Lm - L)) < 1e-10


def test_noise_on_single_components_reproduces_exact():
    """Eq. (loop stochastic) with each piece a single (x, spin, colour): |xi|^2 = 1 makes it exact."""
    U = haar_su3_field(DIMS, 9)
    kappa = 0.125
    site = (2, 1, 0, 3)
    xi = z2_noise(DIMS, 31, 0, 0)
    pieces = []
    for s in range(4):
        for c in range(3):
            pieces.append(point_source(DIMS, site, s, c) * xi[site + (s, c)])
    pieces = np.stack(pieces)
    from oracle.solver import solve
    phi, _ = solve(U, kappa, pieces, tol=1e-13)
    est = contract(pieces, phi)[site]
    exact = exact_loops(U, kappa, DIMS, [site], tol=1e-13)[0]
    assert np.max(np.abs(est - exact)) < 1e-10


def test_propagator_diag_block_layout():
    """G(x;x)[alpha,a,beta,b] equals the dense inverse's diagonal block."""
    from oracle.dense import dense_D, site_index
    dims = (2, 2, 2, 2)
    U = haar_su3_field(dims, 4)
    kappa = 0.15
    G = np.linalg.inv(dense_D(U, kappa, dims))
    t, z, y, x = (1, 0, 1, 1)
    i = site_index(dims, x, y, z, t)
    blk = exact_propagator_diag(U, kappa, dims, [(t, z, y, x)], tol=1e-13)[0].reshape(12, 12)
    assert np.max(np.abs(blk - G[12 * i:12 * i + 12, 12 * i:12 * i + 12])) < 1e-11


def test_dense_exact_loops_match_point_source_solves():
    from oracle.loops import exact_loops_dense
    U = haar_su3_field(DIMS, 0)
    full = exact_loops_dense(U, 0.125)
    sites = [(0, 0, 0, 0), (3, 2, 1, 0)]
    L = exact_loops(U, 0.125, DIMS, sites, tol=1e-13)
    for k, s in enumerate(sites):
        assert np.max(np.abs(full[s] - L[k])) < 1e-10


def test_cubic_tsc_dilution_on_2cube_lattice_is_exact():
    """On a 2^3 x Lt lattice t+s+c dilution with cubic spatial partitioning puts
    one (site, spin, colour) in each piece, so Eq. (loop stochastic) with one
    noise vector reproduces the exact loop at every site (|xi|^2 = 1)."""
    from oracle.loops import exact_loops_dense, stochastic_loops
    from oracle.philox import DIL_TSC, DIL_CUBE
    dims = (2, 2, 2, 4)
    U = haar_su3_field(dims, 12)
    kappa = 0.13
    est = stochastic_loops(U, kappa, dims, 5, [0], DIL_TSC | DIL_CUBE, tol=1e-13)
    exact = exact_loops_dense(U, kappa)
    assert np.max(np.abs(est - exact)) < 1e-10
    # even-odd alone is not site-exact on this lattice: off-diagonal noise remains
    from oracle.philox import DIL_EO
    est_eo = stochastic_loops(U, kappa, dims, 5, [0], DIL_TSC | DIL_EO, tol=1e-13)
    assert np.max(np.abs(est_eo - exact)) > 1e-6


def test_momentum_loops_plane_wave_and_translation():
    """sum_x e^{ip.x} e^{-iq.x} = L^3 delta_{p,q}; a spatial shift by a multiplies
    by e^{ip.a}; p = 0 is the time-slice sum; n_i and n_i + L_i agree."""
    from oracle.loops import momentum_loops, per_timeslice
    lx, ly, lz, lt = 4, 6, 2, 3
    z, y, x = np.meshgrid(np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    q = (1, 2, 1)
    wave = np.exp(-2j * np.pi * (q[0] * x / lx + q[1] * y / ly + q[2] * z / lz))
    ps = np.zeros((lt, lz, ly, lx, 6), dtype=np.complex128)
    ps[1, ..., 4] = wave
    moms = [(0, 0, 0), q, (1, 0, 0), (q[0] + lx, q[1] - ly, q[2])]
    m = momentum_loops(ps, moms)
    assert abs(m[1, 1, 4] - lx * ly * lz) < 1e-9
    assert abs(m[3, 1, 4] - lx * ly * lz) < 1e-9
    assert abs(m[0, 1, 4]) < 1e-9 and abs(m[2, 1, 4]) < 1e-9
    assert np.max(np.abs(np.delete(m, 1, axis=1))) == 0.0
    rng = np.random.default_rng(4)
    ps = rng.normal(size=(lt, lz, ly, lx, 6)) + 1j * rng.normal(size=(lt, lz, ly, lx, 6))
    assert np.allclose(momentum_loops(ps, [(0, 0, 0)])[0], per_timeslice(ps), atol=1e-12)
    a = (1, 2, 1)  # L'(x) = L(x - a)
    shifted = np.roll(ps, shift=(a[2], a[1], a[0]), axis=(1, 2, 3))
    p = (1, 1, 1)
    phase = np.exp(2j * np.pi * (p[0] * a[0] / lx + p[1] * a[1] / ly + p[2] * a[2] / lz))
    assert np.allclose(momentum_loops(shifted, [p])[0], phase * momentum_loops(ps, [p])[0], atol=1e-11)
    # a single site x0 gives the phase e^{ip.x0}
    d = np.zeros((lt, lz, ly, lx, 6), dtype=np.complex128)
    d[2, 1, 3, 2, 0] = 1.0
    got = momentum_loops(d, [p])[0, 2, 0]
    assert abs(got - np.exp(2j * np.pi * (p[0] * 2 / lx + p[1] * 3 / ly + p[2] * 1 / lz))) < 1e-14


def test_disconnected_correlator_identities():
    """Unbiased estimator = ((sum_r L^r)(sum_r' L^r') - sum_r L^r L^r) / (N(N-1));
    time translation invariance; N = 1 product form; zero-mean independent noise
    on top of fixed loops leaves the unbiased estimator centred on the exact D."""
    from oracle.loops import disconnected_correlator
    rng = np.random.default_rng(7)
    n, lt, l3 = 5, 6, 8
    A = rng.normal(size=(n, lt, 6)) + 1j * rng.normal(size=(n, lt, 6))
    B = rng.normal(size=(n, lt, 6)) + 1j * rng.normal(size=(n, lt, 6))
    D = disconnected_correlator(A, B, l3)
    sa, sb = A.sum(0), B.sum(0)
    ref = np.zeros((lt, 6, 6), dtype=np.complex128)
    for t in range(lt):
        sa_t = np.roll(sa, -t, axis=0)
        diag = np.einsum("rta,rtb->ab", np.roll(A, -t, axis=1), B)
        ref[t] = (np.einsum("ta,tb->ab", sa_t, sb) - diag) / (n * (n - 1))
    assert np.allclose(D, ref / (l3 * lt), atol=1e-13)
    # translating every loop in time leaves D unchanged
    assert np.allclose(disconnected_correlator(np.roll(A, 2, axis=1), np.roll(B, 2, axis=1), l3), D, atol=1e-13)
    # N = 1 (exact loops): D(t) = 1/(L^3 Lt) sum_t' L_A(t + t') L_B(t')
    D1 = disconnected_correlator(A[:1], B[:1], l3, unbiased=False)
    assert np.allclose(D1[1], np.einsum("ta,tb->ab", np.roll(A[0], -1, axis=0), B[0]) / (l3 * lt), atol=1e-13)
    with pytest.raises(ValueError):
        disconnected_correlator(A[:1], B[:1], l3)
    # unbiasedness: L^r = mu + eta^r with independent zero-mean eta
    mu_a, mu_b = A[0], B[0]
    exact = disconnected_correlator(mu_a[None], mu_b[None], l3, unbiased=False)
    reps = []
    for k in range(400):
        eta = rng.normal(size=(2, 4, lt, 6))
        reps.append(disconnected_correlator(mu_a + eta[0], mu_b + eta[1], l3))
    reps = np.array(reps)
    err = reps.std(axis=0).real / np.sqrt(len(reps))
    z = np.abs(reps.mean(axis=0).real - exact.real) / err
    assert np.mean(z ** 2) < 2.0
    biased = np.array([disconnected_correlator(mu_a + e[0], mu_a + e[0], l3, unbiased=False)
                       for e in rng.normal(size=(50, 2, 4, lt, 6))]).mean(axis=0)
    # with the same noise in both loops the r = r' terms add <eta^2> / N per source time on the
    # Gamma diagonal at t = 0: bias = Lt <eta^2> / (N L^3 Lt) = 1 / (4 * 8) here
    bias = np.mean(biased.real[0].diagonal() - disconnected_correlator(mu_a[None], mu_a[None], l3,
                                                                        unbiased=False)[0].real.diagonal())
    assert 0.02 < bias < 0.045


def _golden_free():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "free_field_loops.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    return [((int(r[0]), int(r[1]), int(r[2]), int(r[3])), float(r[4]), float(r[5])) for r in rows]


def test_free_field_golden_traces():
    """Exact loops of the free field against the stored closed-form traces (tests/golden)."""
    for dims, kappa, trace in _golden_free():
        U = unit_gauge_field(dims)
        L = exact_loops(U, kappa, dims, [(0, 0, 0, 0), (dims[3] - 1, dims[2] - 1, 0, 1)], tol=1e-13)
        for row in L:
            assert abs(row[0] - trace) < 1e-10
            assert np.max(np.abs(row[1:])) < 1e-12
