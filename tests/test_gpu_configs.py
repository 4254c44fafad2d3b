"""Full-size parity cases of the workloads the library is measured on
(16^3 x 32 eps = 0.35 field at kappa = 0.120, and the uneven batch), checked
against the oracle on sampled outputs and against exact loops statistically."""
import numpy as np
import pytest

from lattice_inputs import eps_su3_field, haar_su3_field, gaussian_spinors
from oracle import loops as olp, philox as oph
from oracle.solver import solve as osolve
from tests._gpu import lattice, to_dev, to_np, rel_err, require_gpu, torch

pytestmark = pytest.mark.gpu

DIMS = (16, 16, 16, 32)
V = 16 ** 3 * 32


@pytest.fixture(scope="module")
def eps_field():
    return eps_su3_field(DIMS, 0.35, 1)


@pytest.mark.parametrize("prec", ["fp64_plain", "mixed_bf16"])
def test_noise_vs_exact_subblock_16x16x16x32(eps_field, prec):
    """8 t+s+c-diluted vectors (384 pieces each): per-time-slice loops on the
    4x4 spatial sub-block (x, y < 4, z = 0) agree with the exact loops there
    within the spread of the 8 vectors; one diluted piece matches the oracle.
    fp64_plain is the configuration as stated: the plain single-right-hand-side
    FP64 solver (one RHS per solve) for the 3072 noise pieces and the 6144
    point sources of the sub-block; mixed_bf16 runs the same on the batched
    mixed-precision solver."""
    U = eps_field
    lx, ly, lz, lt = DIMS
    sub = [(t, 0, y, x) for t in range(lt) for y in range(4) for x in range(4)]
    sub_idx = np.array([x + lx * (y + ly * (z + lz * t)) for (t, z, y, x) in sub])
    with lattice(DIMS, U, 0.120) as (L, h):
        if prec == "fp64_plain":
            p = L.solver_params(tol=1e-10, precision=L.LQCD_PREC_FP64, rhs_block=1)
        else:
            p = L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_BF16)
        src = torch.empty((384, V, 4, 3), dtype=torch.complex128, device="cuda")
        x = torch.empty_like(src)
        per = []
        for r in range(8):
            L.lqcd_noise_generate(5, 0, r, DIMS, L.LQCD_DILUTE_TSC, 0, 384, src)
            rc, st = L.lqcd_solve_batch(h, src, x, p)
            assert rc == 0 and max(s["true_rel_residual"] for s in st) <= 1e-10
            ps = torch.zeros((V, 6), dtype=torch.complex128, device="cuda")
            L.lqcd_loops_batch(h, src, x, 1.0, ps, None)
            per.append(ps[torch.from_numpy(sub_idx).cuda()].cpu().numpy().reshape(lt, 16, 6).sum(axis=1))
            if r == 0:  # one sampled piece against the oracle at full size
                k = 12 * 7 + 3 * 2 + 1
                got = to_np(x[k:k + 1], DIMS)[0]
        # exact loops on the sub-block: 12 point sources per site
        exact = np.zeros((lt, 6), dtype=np.complex128)
        for c0 in range(0, len(sub_idx), 32):
            sites = sub_idx[c0:c0 + 32].tolist()
            ps_src = torch.empty((12 * len(sites), V, 4, 3), dtype=torch.complex128, device="cuda")
            L.lqcd_point_sources(h, sites, ps_src)
            xs = torch.empty_like(ps_src)
            rc, st = L.lqcd_solve_batch(h, ps_src, xs, p)
            assert rc == 0
            pt = torch.zeros((lt, 6), dtype=torch.complex128, device="cuda")
            L.lqcd_loops_batch(h, ps_src, xs, 1.0, None, pt)
            exact += pt.cpu().numpy()
    per = np.array(per)
    zs = []
    for part in (np.real, np.imag):
        d = part(per.mean(axis=0) - exact)
        e = part(per).std(axis=0, ddof=1) / np.sqrt(8)
        m = e > 1e-12
        zs.append(np.abs(d[m]) / e[m])
        assert np.all(np.abs(d[~m]) < 1e-7)
    z = np.concatenate(zs)
    # with 8 vectors z follows Student's t with 7 degrees of freedom (variance 1.4);
    # a wrong normalisation or sign would give z of order |L| / error ~ 100
    assert np.mean(z ** 2) < 3.0 and z.max() < 12.0, (np.mean(z ** 2), z.max())
    piece = oph.dilute(oph.z2_noise(DIMS, 5, 0, 0), oph.DIL_TSC, 12 * 7 + 3 * 2 + 1)
    ref, _ = osolve(U, 0.120, piece[None], tol=1e-12)
    assert rel_err(got, ref[0]) < 1e-8


def test_tsm_full_size_and_hp_vector_parity(eps_field):
    """TSM with 400 LP solves at 1e-3 and 20 HP vectors: convergence as stated,
    and the HP contribution of one vector equals the oracle's."""
    U = eps_field
    with lattice(DIMS, U, 0.120) as (L, h):
        pb = L.solver_params(precision=L.LQCD_PREC_MIXED_BF16)
        sp = L.stochastic_params(seed=9, n_lp=400, n_hp=20, tol_lp=1e-3, tol_hp=1e-10,
                                 dilution=L.LQCD_DILUTE_NONE, chunk=64)
        pt = torch.zeros((32, 6), dtype=torch.complex128, device="cuda")
        rc, summ = L.lqcd_loops_stochastic(h, sp, pb, None, pt)
        assert rc == 0
        assert summ[0]["true_rel_residual"] <= 1e-3 and summ[1]["true_rel_residual"] <= 1e-10
        assert 2 * summ[0]["iterations"] < summ[1]["iterations"]
        # one HP vector alone: its precise solution against the oracle's
        src = torch.empty((1, V, 4, 3), dtype=torch.complex128, device="cuda")
        L.lqcd_noise_generate(9, L.LQCD_STREAM_HP, 0, DIMS, L.LQCD_DILUTE_NONE, 0, 1, src)
        xg = torch.empty_like(src)
        rc, st = L.lqcd_solve_batch(h, src, xg, L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_BF16))
        one = torch.zeros((32, 6), dtype=torch.complex128, device="cuda")
        L.lqcd_loops_batch(h, src, xg, 1.0, None, one)
        got = one.cpu().numpy()
    xi = oph.z2_noise(DIMS, 9, 0, 1)[None]
    phi, _ = osolve(U, 0.120, xi, tol=1e-12)
    ref = olp.per_timeslice(olp.contract(xi, phi))
    assert rel_err(got, ref) < 1e-8


def test_uneven_batch_four_lattices_full_size():
    L = require_gpu()
    specs = [((8, 8, 8, 16), "haar", 0.157, 48), ((12, 12, 12, 24), "eps", 0.115, 24),
             ((16, 16, 16, 32), "eps", 0.120, 12), ((24, 24, 24, 48), "haar", 0.157, 6)]
    handles, bs, xs, fields = [], [], [], []
    batch = L.lqcd_batch_create()
    s = torch.cuda.Stream()
    try:
        for k, (dims, kind, kappa, n) in enumerate(specs):
            U = haar_su3_field(dims, 10 + k) if kind == "haar" else eps_su3_field(dims, 0.35, 10 + k)
            fields.append(U)
            h = L.lqcd_create(dims, 0)
            handles.append(h)
            L.lqcd_set_gauge(h, to_dev(U.reshape(-1)))
            L.lqcd_set_kappa(h, kappa)
            Vl = int(np.prod(dims))
            b = torch.empty((n, Vl, 4, 3), dtype=torch.complex128, device="cuda")
            L.lqcd_noise_generate(3, 0, k, dims, L.LQCD_DILUTE_TSC, 0, n, b)
            bs.append(b)
            xs.append(torch.empty_like(b))
            L.lqcd_batch_add(batch, h, b, xs[-1])
        total = sum(sp[3] for sp in specs)
        p = L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_BF16)
        rc, st = L.lqcd_batch_run(batch, p, total, s)
        torch.cuda.synchronize()
        assert rc == 0 and all(r["true_rel_residual"] <= 1e-10 for r in st)
        for k in range(len(specs)):
            solo = torch.empty_like(bs[k])
            L.lqcd_solve_batch(handles[k], bs[k], solo, p)
            assert torch.equal(solo, xs[k])
        # sampled oracle solve on the smallest lattice
        dims, _, kappa, n = specs[0]
        piece = oph.dilute(oph.z2_noise(dims, 3, 0, 0), oph.DIL_TSC, 5)
        ref, _ = osolve(fields[0], kappa, piece[None], tol=1e-12)
        assert rel_err(to_np(xs[0][5:6], dims)[0], ref[0]) < 1e-8
    finally:
        L.lqcd_batch_destroy(batch)
        for h in handles:
            L.lqcd_destroy(h)
