"""GPU parity of the stochastic loops and the truncated solver method
(lqcd_loops_stochastic) against the oracle."""
import numpy as np
import pytest

from lattice_inputs import eps_su3_field, haar_su3_field
from oracle import loops as olp
from oracle.philox import DIL_TSC, DIL_NONE, DIL_TS, DIL_EO, DIL_CUBE
from tests._gpu import lattice, rel_err, torch

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 8)


def _run(L, h, sp, solver, dims):
    V = int(np.prod(dims))
    ps = torch.zeros((V, 6), dtype=torch.complex128, device="cuda")
    pt = torch.zeros((dims[3], 6), dtype=torch.complex128)  # host per_t
    rc, summ = L.lqcd_loops_stochastic(h, sp, solver, ps, pt)
    lx, ly, lz, lt = dims
    return rc, summ, ps.cpu().numpy().reshape(lt, lz, ly, lx, 6), pt.numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp16"])
@pytest.mark.parametrize("scheme", [DIL_TSC, DIL_TS])
def test_plain_diluted_estimator_matches_oracle(prec, scheme):
    U = eps_su3_field(DIMS, 0.35, 1)
    kappa = 0.12
    with lattice(DIMS, U, kappa) as (L, h):
        pr = L.LQCD_PREC_FP64 if prec == "fp64" else L.LQCD_PREC_MIXED_FP16
        sp = L.stochastic_params(seed=11, n_lp=2, n_hp=0, tol_lp=1e-11, dilution=scheme, chunk=40)
        rc, summ, ps, pt = _run(L, h, sp, L.solver_params(precision=pr, rhs_block=16), DIMS)
    assert rc == 0 and summ[0]["true_rel_residual"] <= 1e-11
    ref = olp.stochastic_loops(U, kappa, DIMS, 11, [0, 1], scheme, tol=1e-13)
    assert rel_err(ps, ref) < 1e-8
    assert rel_err(pt, olp.per_timeslice(ref)) < 1e-8


def test_tsm_equal_tolerances_is_plain_estimator():
    U = haar_su3_field(DIMS, 2)
    with lattice(DIMS, U, 0.12) as (L, h):
        s = L.solver_params(precision=L.LQCD_PREC_MIXED_FP16)
        a = _run(L, h, L.stochastic_params(5, 3, 2, 1e-9, 1e-9, DIL_NONE), s, DIMS)
        b = _run(L, h, L.stochastic_params(5, 3, 0, 1e-9, 1e-9, DIL_NONE), s, DIMS)
    assert a[0] == 0 and b[0] == 0
    # the correction adds and subtracts identical solutions: zero up to rounding of the sums
    assert np.max(np.abs(a[2] - b[2])) <= 1e-13 * np.max(np.abs(b[2]))


def test_tsm_matches_oracle_within_truncation():
    """LP solves at 1e-3 differ between two correct solvers by O(1e-3) of the
    solution; the TSM estimates then agree to that order, and both agree with the
    exact loops within statistics."""
    dims = DIMS
    U = eps_su3_field(dims, 0.35, 1)
    kappa = 0.12
    with lattice(dims, U, kappa) as (L, h):
        sp = L.stochastic_params(7, 6, 3, 1e-3, 1e-10, DIL_NONE)
        rc, summ, ps, pt = _run(L, h, sp, L.solver_params(precision=L.LQCD_PREC_MIXED_FP16), dims)
    assert rc == 0
    assert summ[0]["true_rel_residual"] <= 1e-3 and summ[1]["true_rel_residual"] <= 1e-10
    assert summ[0]["iterations"] * 2 < summ[1]["iterations"]
    ref = olp.tsm_loops(U, kappa, dims, 7, 6, 3, 1e-3, 1e-10, DIL_NONE)
    scale = np.max(np.abs(olp.per_timeslice(ref)))
    assert np.max(np.abs(pt - olp.per_timeslice(ref))) < 2e-2 * scale
    # the scalar loop (real, O(12) per site) is dominated by the exact diagonal: tight relative check
    assert np.max(np.abs(pt[:, 0] - olp.per_timeslice(ref)[:, 0])) < 5e-3 * np.max(np.abs(pt[:, 0]))


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_cubic_dilution_site_exact_on_2cube_lattice(prec):
    """t+s+c + cubic dilution on 2^3 x 4 leaves one (site, spin, colour) per
    piece: one noise vector reproduces the exact loops (dense inverse)."""
    dims = (2, 2, 2, 4)
    U = haar_su3_field(dims, 12)
    kappa = 0.13
    with lattice(dims, U, kappa) as (L, h):
        pr = L.LQCD_PREC_FP64 if prec == "fp64" else L.LQCD_PREC_MIXED_BF16
        assert L.lqcd_dilution_pieces(dims, DIL_TSC | DIL_CUBE) == 12 * 4 * 8
        sp = L.stochastic_params(seed=5, n_lp=1, n_hp=0, tol_lp=1e-12, dilution=DIL_TSC | DIL_CUBE, chunk=100)
        rc, summ, ps, pt = _run(L, h, sp, L.solver_params(precision=pr), dims)
    assert rc == 0
    exact = olp.exact_loops_dense(U, kappa)
    assert np.max(np.abs(ps - exact)) < 1e-9 * np.max(np.abs(exact))
    ref = olp.stochastic_loops(U, kappa, dims, 5, [0], DIL_TSC | DIL_CUBE, tol=1e-13)
    assert rel_err(ps, ref) < 1e-9


def test_even_odd_dilution_matches_oracle():
    U = eps_su3_field(DIMS, 0.35, 3)
    kappa = 0.12
    with lattice(DIMS, U, kappa) as (L, h):
        sp = L.stochastic_params(seed=21, n_lp=1, n_hp=0, tol_lp=1e-11, dilution=DIL_TS | DIL_EO, chunk=24)
        rc, summ, ps, pt = _run(L, h, sp, L.solver_params(precision=L.LQCD_PREC_MIXED_BF16), DIMS)
    assert rc == 0
    ref = olp.stochastic_loops(U, kappa, DIMS, 21, [0], DIL_TS | DIL_EO, tol=1e-13)
    assert rel_err(ps, ref) < 1e-8
    assert rel_err(pt, olp.per_timeslice(ref)) < 1e-8


@pytest.mark.parametrize("dims", [(4, 6, 2, 6), (16, 16, 16, 32)])
def test_momentum_loops_match_oracle(dims):
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(3)
    per_site = rng.normal(size=(lt, lz, ly, lx, 6)) + 1j * rng.normal(size=(lt, lz, ly, lx, 6))
    moms = [(0, 0, 0), (1, 0, 0), (0, -1, 1), (2, 3, -1), (lx + 1, 0, -lz)] + [(k, 1, 0) for k in range(140)]
    if lx * ly * lz > 1000:
        moms = moms[:8] + moms[-3:]  # crossing the 128-momenta chunk is covered by the small lattice
    with lattice(dims) as (L, h):
        d = torch.from_numpy(per_site.reshape(-1, 6).copy()).cuda()
        out = torch.empty((len(moms), lt, 6), dtype=torch.complex128, device="cuda")
        L.lqcd_loops_momentum(h, d, moms, out)
        got = out.cpu().numpy()
    ref = olp.momentum_loops(per_site, moms)
    assert rel_err(got, ref) < 1e-12
    assert np.max(np.abs(got - ref)) < 1e-11 * np.sqrt(lx * ly * lz)


@pytest.mark.parametrize("n,unbiased", [(1, False), (2, True), (7, True), (7, False)])
def test_disconnected_correlator_matches_oracle(n, unbiased):
    L = __import__("tests._gpu", fromlist=["require_gpu"]).require_gpu()
    rng = np.random.default_rng(n)
    lt, l3 = 10, 64
    A = rng.normal(size=(n, lt, 6)) + 1j * rng.normal(size=(n, lt, 6))
    B = rng.normal(size=(n, lt, 6)) + 1j * rng.normal(size=(n, lt, 6))
    out = torch.empty((lt, 6, 6), dtype=torch.complex128, device="cuda")
    L.lqcd_disconnected_correlator(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), l3, out, unbiased)
    ref = olp.disconnected_correlator(A, B, l3, unbiased)
    assert rel_err(out.cpu().numpy(), ref) < 1e-12
    if n == 1:
        with pytest.raises(L.LqcdError):
            L.lqcd_disconnected_correlator(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), l3, out, True)


def test_correlator_from_momentum_loops_end_to_end():
    """Noise vectors -> diluted loops per vector (per site) -> momentum projection
    at +p and -p -> unbiased D_AB(p, t), against the oracle chain."""
    dims = (4, 4, 4, 6)
    U = eps_su3_field(dims, 0.35, 5)
    kappa = 0.12
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    moms = [(1, 0, 0), (-1, 0, 0)]
    nvec = 3
    with lattice(dims, U, kappa) as (L, h):
        loops_p = torch.empty((nvec, lt, 6), dtype=torch.complex128, device="cuda")
        loops_mp = torch.empty_like(loops_p)
        for r in range(nvec):
            ps = torch.zeros((V, 6), dtype=torch.complex128, device="cuda")
            sp = L.stochastic_params(seed=8, n_lp=1, n_hp=0, tol_lp=1e-11, dilution=DIL_TSC, first_noise=r)
            rc, _ = L.lqcd_loops_stochastic(h, sp, L.solver_params(precision=L.LQCD_PREC_MIXED_BF16), ps, None)
            assert rc == 0
            pm = torch.empty((2, lt, 6), dtype=torch.complex128, device="cuda")
            L.lqcd_loops_momentum(h, ps, moms, pm)
            loops_p[r], loops_mp[r] = pm[0], pm[1]
        D = torch.empty((lt, 6, 6), dtype=torch.complex128, device="cuda")
        L.lqcd_disconnected_correlator(loops_p, loops_mp, lx * ly * lz, D, True)
        got = D.cpu().numpy()
    per = [olp.stochastic_loops(U, kappa, dims, 8, [r], DIL_TSC, tol=1e-13) for r in range(nvec)]
    mp = np.stack([olp.momentum_loops(x, moms) for x in per])  # (nvec, 2, lt, 6)
    ref = olp.disconnected_correlator(mp[:, 0], mp[:, 1], lx * ly * lz, True)
    assert rel_err(got, ref) < 1e-8
