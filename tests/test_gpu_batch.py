"""GPU tests of the uneven multi-lattice batch (one captured CUDA graph), the
captured single-lattice iteration graph, the FP64 CG solver and the autotuner,
against the oracle and against each other (bit-identical where the arithmetic
is the same)."""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, eps_su3_field, gaussian_spinors
from oracle.dense import dense_D, to_vec, from_vec
from oracle.solver import solve as osolve
from tests._gpu import lattice, to_dev, to_np, rel_err, require_gpu, torch

pytestmark = pytest.mark.gpu


def test_cg_fp64_matches_dense_lu():
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 0)
    kappa = 0.125
    b = gaussian_spinors(dims, 3, 31)
    with lattice(dims, U, kappa) as (L, h):
        x = torch.empty((3, 256, 4, 3), dtype=torch.complex128, device="cuda")
        rc, st = L.lqcd_solve_batch(h, to_dev(b.reshape(3, 256, 4, 3)), x,
                                    L.solver_params(tol=1e-12, solver=L.LQCD_SOLVER_CG, rhs_block=3))
        got = to_np(x, dims)
        assert rc == 0 and all(s["true_rel_residual"] <= 1e-12 for s in st)
        with pytest.raises(L.LqcdError):
            L.lqcd_solve_batch(h, to_dev(b.reshape(3, 256, 4, 3)), x,
                               L.solver_params(tol=1e-10, solver=L.LQCD_SOLVER_CG, precision=L.LQCD_PREC_MIXED_FP16))
    ref = from_vec(np.linalg.solve(dense_D(U, kappa, dims), to_vec(b).T).T, dims)
    for k in range(3):
        assert rel_err(got[k], ref[k]) < 1e-10


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_graph_replay_is_bit_identical_to_direct_launches(prec):
    dims = (8, 8, 8, 16)
    U = eps_su3_field(dims, 0.35, 1)
    b = gaussian_spinors(dims, 6, 3).reshape(6, -1, 4, 3)
    with lattice(dims, U, 0.12) as (L, h):
        pr = L.LQCD_PREC_MIXED_FP16 if prec == "fp16" else L.LQCD_PREC_MIXED_BF16
        bd = to_dev(b)
        x0 = torch.empty_like(bd)
        rc0, st0 = L.lqcd_solve_batch(h, bd, x0, L.solver_params(tol=1e-10, precision=pr))  # default stream: direct
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            x1 = torch.empty_like(bd)
            rc1, st1 = L.lqcd_solve_batch(h, bd, x1, L.solver_params(tol=1e-10, precision=pr))  # captured graph
            x2 = torch.empty_like(bd)
            rc2, st2 = L.lqcd_solve_batch(h, bd, x2, L.solver_params(tol=1e-10, precision=pr))  # graph replayed
        torch.cuda.synchronize()
        assert rc0 == rc1 == rc2 == 0
        assert torch.equal(x0, x1) and torch.equal(x1, x2)
        assert [a["iterations"] for a in st0] == [a["iterations"] for a in st1]


def test_uneven_batch_matches_single_solves_and_oracle():
    L = require_gpu()
    specs = [((4, 4, 4, 4), haar_su3_field((4, 4, 4, 4), 0), 0.125, 5),
             ((4, 4, 4, 8), eps_su3_field((4, 4, 4, 8), 0.35, 1), 0.120, 4),
             ((6, 6, 4, 8), haar_su3_field((6, 6, 4, 8), 2), 0.157, 3)]
    handles, bs, xs, refs = [], [], [], []
    batch = L.lqcd_batch_create()
    s = torch.cuda.Stream()
    try:
        for k, (dims, U, kappa, n) in enumerate(specs):
            h = L.lqcd_create(dims, 0)
            handles.append(h)
            L.lqcd_set_gauge(h, to_dev(U.reshape(-1)))
            L.lqcd_set_kappa(h, kappa)
            b = gaussian_spinors(dims, n, 60 + k)
            bs.append(to_dev(b.reshape(n, -1, 4, 3)))
            xs.append(torch.empty_like(bs[-1]))
            L.lqcd_batch_add(batch, h, bs[-1], xs[-1])
            refs.append(osolve(U, kappa, b, tol=1e-12)[0])
        total = sum(sp[3] for sp in specs)
        assert L.lqcd_batch_rhs(batch) == total
        # a stats array shorter than the batch is refused before any work
        with pytest.raises(L.LqcdError) as e:
            L.lqcd_batch_run(batch, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_FP16), total - 1, s)
        assert e.value.code == L.LQCD_ERR_INVALID
        rc, st = L.lqcd_batch_run(batch, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_FP16), total, s)
        torch.cuda.synchronize()
        assert rc == 0 and len(st) == total and all(r["true_rel_residual"] <= 1e-10 for r in st)
        for k, (dims, U, kappa, n) in enumerate(specs):
            solo = torch.empty_like(bs[k])
            L.lqcd_solve_batch(handles[k], bs[k], solo, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_FP16))
            assert torch.equal(solo, xs[k])
            got = to_np(xs[k], dims)
            for j in range(n):
                assert rel_err(got[j], refs[k][j]) < 1e-8
        # a second run replays the captured graph
        for x in xs:
            x.zero_()
        rc, st = L.lqcd_batch_run(batch, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_FP16), total, s)
        torch.cuda.synchronize()
        assert rc == 0
        got = to_np(xs[1], specs[1][0])
        assert rel_err(got[0], refs[1][0]) < 1e-8
    finally:
        L.lqcd_batch_destroy(batch)
        for h in handles:
            L.lqcd_destroy(h)


def test_autotune_keeps_results_bit_identical():
    dims = (8, 8, 8, 16)
    U = eps_su3_field(dims, 0.35, 1)
    b = gaussian_spinors(dims, 4, 8).reshape(4, -1, 4, 3)
    with lattice(dims, U, 0.12) as (L, h):
        bd = to_dev(b)
        x0 = torch.empty_like(bd)
        L.lqcd_solve_batch(h, bd, x0, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_FP16))
        best, variant = L.lqcd_autotune(h, 4, L.LQCD_PREC_MIXED_FP16, with_variant=True)
        assert best in (2, 4, 8, 16, 32, 64, 128, 256) and variant in (0, 1, 2, 3, 4, 7)  # FP16: pair variants only
        x1 = torch.empty_like(bd)
        L.lqcd_solve_batch(h, bd, x1, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_FP16))
        if variant < 4:  # the FP32-unit variants differ only in launch shape: same arithmetic
            assert torch.equal(x0, x1)
        else:  # tensor-core SU(3) products or rebuilt link rows: a different rounding, the same solution
            assert (x0 - x1).abs().max().item() <= 1e-8 * x0.abs().max().item()


def test_tuned_layout_choice_is_revised_from_iteration_counts(monkeypatch):
    """lqcd_tuned_choice reports the autotuner's pick until a BF16 solve revises
    the choice between the pair and the 128-RHS tile layout from the solve's
    per-RHS iteration counts: afterwards it is either the tile layout or the
    autotuner's best pair configuration, and a solve with the revised choice
    agrees with one forced onto the other layout."""
    monkeypatch.delenv("LQCD_HOP_VARIANT", raising=False)
    dims = (4, 4, 4, 8)
    U = eps_su3_field(dims, 0.35, 2)
    n = 128
    b = gaussian_spinors(dims, n, 41).reshape(n, -1, 4, 3)
    with lattice(dims, U, 0.12) as (L, h):
        pr = L.LQCD_PREC_MIXED_BF16
        bps, var = L.lqcd_autotune(h, n, pr, with_variant=True)
        assert L.lqcd_tuned_choice(h, n, pr) == (bps, var)
        bd = to_dev(b)
        x0 = torch.empty_like(bd)
        rc0, st0 = L.lqcd_solve_batch(h, bd, x0, L.solver_params(tol=1e-10, precision=pr))
        assert rc0 == 0
        bps2, var2 = L.lqcd_tuned_choice(h, n, pr)
        assert (bps2, var2) == (1, 5) or var2 in (0, 1, 2, 3, 4, 6, 7)
        if var == 5:
            assert var2 == 5 or (bps2, var2) != (bps, var)
        else:
            assert (bps2, var2) in ((bps, var), (1, 5))
        # the other layout gives the same solution to the solver's tolerance
        monkeypatch.setenv("LQCD_HOP_VARIANT", "1" if var2 == 5 else "5")
        x1 = torch.empty_like(bd)
        rc1, st1 = L.lqcd_solve_batch(h, bd, x1, L.solver_params(tol=1e-10, precision=pr))
        assert rc1 == 0
        assert all(s["true_rel_residual"] <= 1e-10 for s in st0 + st1)
        assert rel_err(to_np(x0, dims), to_np(x1, dims)) < 1e-8
