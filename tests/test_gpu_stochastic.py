"""GPU parity of the stochastic loops and the truncated solver method
(lqcd_loops_stochastic) against the oracle."""
import numpy as np
import pytest

from lattice_inputs import eps_su3_field, haar_su3_field
from oracle import loops as olp
from oracle.philox import DIL_TSC, DIL_NONE, DIL_TS
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
