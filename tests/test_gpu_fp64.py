"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

Wilson operator D and D^+, plaquette, point sources, Z2 noise (bit-exact),
loop contraction, and the plain FP64 even-odd BiCGstab (vs dense LU and the
oracle), plus the error statuses made on the host (zero, NaN, iteration cap,
timeout, non-SU(3) links).
"""
import numpy as np
import pytest

from lattice_inputs import haar_su3_field, eps_su3_field, gaussian_spinors, unit_gauge_field
from oracle import dirac as od
from oracle import philox as oph
from oracle import loops as olp
from oracle.dense import dense_D, to_vec, from_vec
from tests._gpu import lattice, to_dev, to_np, rel_err, torch

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 4, 2, 8), (2, 2, 2, 2), (8, 6, 4, 10)]


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_dirac_matches_oracle(dims, dagger):
    U = haar_su3_field(dims, 1)
    kappa = 0.137
    psi = gaussian_spinors(dims, 3, 2)
    with lattice(dims, U, kappa) as (L, h):
        inp = to_dev(psi.reshape(3, -1, 4, 3))
        out = torch.empty_like(inp)
        L.lqcd_apply_dirac(h, inp, out, dagger)
        got = to_np(out, dims)
    ref = od.apply_Ddag(U, kappa, psi) if dagger else od.apply_D(U, kappa, psi)
    assert rel_err(got, ref) < 1e-14


def test_plaquette_matches_oracle():
    dims = (8, 8, 8, 16)
    for U in (eps_su3_field(dims, 0.35, 1), haar_su3_field(dims, 0), unit_gauge_field(dims)):
        with lattice(dims, U) as (L, h):
            assert abs(L.lqcd_plaquette(h) - od.plaquette(U)) < 1e-13


def test_set_gauge_rejects_non_su3():
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 0)
    U[1, 2, 3, 0, 2] *= 1.0 + 1e-9
    with lattice(dims) as (L, h):
        with pytest.raises(L.LqcdError) as e:
            L.lqcd_set_gauge(h, to_dev(U.reshape(-1)))
        assert e.value.code == L.LQCD_ERR_NOT_SU3
    U2 = haar_su3_field(dims, 0)
    U2[0, 0, 0, 0, 1] *= np.exp(1j * 0.3)  # unitary, det != 1
    with lattice(dims) as (L, h):
        with pytest.raises(L.LqcdError):
            L.lqcd_set_gauge(h, to_dev(U2.reshape(-1)))


def test_host_gauge_pointer_accepted():
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 3)
    with lattice(dims) as (L, h):
        L.lqcd_set_gauge(h, torch.from_numpy(U.reshape(-1)))  # host memory
        assert abs(L.lqcd_plaquette(h) - od.plaquette(U)) < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 2, 4, 6), (16, 16, 16, 32)])
@pytest.mark.parametrize("scheme", [oph.DIL_NONE, oph.DIL_T, oph.DIL_TS, oph.DIL_TSC, oph.DIL_EO,
                                    oph.DIL_TSC | oph.DIL_EO, oph.DIL_TSC | oph.DIL_CUBE, oph.DIL_T | oph.DIL_CUBE])
def test_noise_bit_exact(dims, scheme):
    L_ = __import__("tests._gpu", fromlist=["require_gpu"]).require_gpu()
    V = int(np.prod(dims))
    n = oph.dilution_count(dims, scheme)
    pick = sorted(set([0, n // 2, n - 1]))
    for stream in (0, 1):
        for first in pick:
            out = torch.empty((1, V, 4, 3), dtype=torch.complex128, device="cuda")
            L_.lqcd_noise_generate(0xC0FFEE, stream, 5, dims, scheme, first, 1, out)
            ref = oph.dilute(oph.z2_noise(dims, 0xC0FFEE, 5, stream), scheme, first)
            got = out.cpu().numpy().reshape(ref.shape)
            assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_noise_rejects_out_of_range_pieces():
    L_ = __import__("tests._gpu", fromlist=["require_gpu"]).require_gpu()
    out = torch.empty((1, 256, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(L_.LqcdError):
        L_.lqcd_noise_generate(1, 0, 0, (4, 4, 4, 4), L_.LQCD_DILUTE_TSC, 48, 1, out)


def test_point_sources():
    dims = (4, 4, 4, 4)
    V = 256
    sites = [0, 17, 255]
    with lattice(dims) as (L, h):
        out = torch.empty((36, V, 4, 3), dtype=torch.complex128, device="cuda")
        L.lqcd_point_sources(h, sites, out)
        got = to_np(out, dims)
    for k, s in enumerate(sites):
        x, y, z, t = s % 4, (s // 4) % 4, (s // 16) % 4, s // 64
        for sp in range(4):
            for c in range(3):
                assert np.array_equal(got[12 * k + 3 * sp + c], olp.point_source(dims, (t, z, y, x), sp, c))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
def test_loops_batch_matches_oracle(dims):
    src = gaussian_spinors(dims, 5, 1)
    sol = gaussian_spinors(dims, 5, 2)
    V = int(np.prod(dims))
    with lattice(dims) as (L, h):
        ps = torch.zeros((V, 6), dtype=torch.complex128, device="cuda")
        pt = torch.zeros((dims[3], 6), dtype=torch.complex128, device="cuda")
        L.lqcd_loops_batch(h, to_dev(src.reshape(5, V, 4, 3)), to_dev(sol.reshape(5, V, 4, 3)), 0.5, ps, pt)
        # accumulation: a second call adds
        L.lqcd_loops_batch(h, to_dev(src.reshape(5, V, 4, 3)), to_dev(sol.reshape(5, V, 4, 3)), 0.5, ps, pt)
        pth = torch.zeros((dims[3], 6), dtype=torch.complex128)
        L.lqcd_loops_batch(h, to_dev(src.reshape(5, V, 4, 3)), to_dev(sol.reshape(5, V, 4, 3)), 1.0, None, pth)
        got_s = ps.cpu().numpy().reshape(dims[3], dims[2], dims[1], dims[0], 6)
        got_t = pt.cpu().numpy()
        got_th = pth.numpy()
    ref = olp.contract(src, sol)
    assert rel_err(got_s, ref) < 1e-14
    assert rel_err(got_t, olp.per_timeslice(ref)) < 1e-14
    assert rel_err(got_th, olp.per_timeslice(ref)) < 1e-14


@pytest.mark.parametrize("dims,kappa,seed", [((4, 4, 4, 4), 0.125, 0), ((2, 2, 2, 2), 0.15, 1),
                                             ((4, 2, 4, 6), 0.157, 2)])
def test_fp64_solve_matches_dense_lu(dims, kappa, seed):
    U = haar_su3_field(dims, seed)
    b = gaussian_spinors(dims, 4, 10 + seed)
    V = int(np.prod(dims))
    with lattice(dims, U, kappa) as (L, h):
        x = torch.empty((4, V, 4, 3), dtype=torch.complex128, device="cuda")
        rc, stats = L.lqcd_solve_batch(h, to_dev(b.reshape(4, V, 4, 3)), x,
                                       L.solver_params(tol=1e-13, precision=L.LQCD_PREC_FP64))
        got = to_np(x, dims)
    assert rc == 0, stats
    ref = from_vec(np.linalg.solve(dense_D(U, kappa, dims), to_vec(b).T).T, dims)
    for k in range(4):
        assert rel_err(got[k], ref[k]) < 1e-12
        assert stats[k]["true_rel_residual"] <= 1e-13
        r = np.linalg.norm((b[k] - od.apply_D(U, kappa, got[k])).ravel()) / np.linalg.norm(b[k].ravel())
        assert abs(r - stats[k]["true_rel_residual"]) <= 1e-3 * r + 1e-16


def test_fp64_batched_equals_single_rhs_blocks():
    """Per-RHS reductions do not depend on the batch composition: bit-identical."""
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 0)
    b = gaussian_spinors(dims, 3, 4)
    with lattice(dims, U, 0.125) as (L, h):
        bd = to_dev(b.reshape(3, -1, 4, 3))
        x1 = torch.empty_like(bd)
        x3 = torch.empty_like(bd)
        L.lqcd_solve_batch(h, bd, x1, L.solver_params(tol=1e-10, rhs_block=1))
        L.lqcd_solve_batch(h, bd, x3, L.solver_params(tol=1e-10, rhs_block=3))
        assert torch.equal(x1, x3)


def test_fp64_exact_loops_all_point_sources_4444():
    """Exact G(x;x) from all 3072 point-source solves on a 4^4 Haar field (kappa = 0.125)."""
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 0)
    kappa = 0.125
    V = 256
    ref = olp.exact_loops_dense(U, kappa)  # (Lt, Lz, Ly, Lx, 6)
    with lattice(dims, U, kappa) as (L, h):
        ps = torch.zeros((V, 6), dtype=torch.complex128, device="cuda")
        pt = torch.zeros((4, 6), dtype=torch.complex128, device="cuda")
        chunk = 32
        for s0 in range(0, V, chunk):
            sites = list(range(s0, s0 + chunk))
            src = torch.empty((12 * chunk, V, 4, 3), dtype=torch.complex128, device="cuda")
            L.lqcd_point_sources(h, sites, src)
            x = torch.empty_like(src)
            rc, stats = L.lqcd_solve_batch(h, src, x, L.solver_params(tol=1e-10, rhs_block=12 * chunk))
            assert rc == 0 and max(s["true_rel_residual"] for s in stats) <= 1e-10
            L.lqcd_loops_batch(h, src, x, 1.0, ps, pt)
        got = ps.cpu().numpy().reshape(4, 4, 4, 4, 6)
        got_t = pt.cpu().numpy()
    # solutions at 1e-10 residual: loop error bounded by ~cond(D) * 1e-10
    assert np.max(np.abs(got - ref)) < 1e-8
    assert np.max(np.abs(got_t - olp.per_timeslice(ref))) < 1e-7


def test_fp64_status_codes():
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 0)
    V = 256
    b = gaussian_spinors(dims, 3, 7).reshape(3, V, 4, 3)
    b[1] = 0.0
    b[2, 5, 1, 1] = np.nan
    with lattice(dims, U, 0.125) as (L, h):
        x = torch.empty((3, V, 4, 3), dtype=torch.complex128, device="cuda")
        rc, st = L.lqcd_solve_batch(h, to_dev(b), x, L.solver_params(tol=1e-10, rhs_block=3))
        assert st[0]["status"] == 0 and st[1]["status"] == 0
        assert torch.all(x[1] == 0)
        assert st[2]["status"] == L.LQCD_ERR_NONFINITE
        assert rc == L.LQCD_ERR_NONFINITE
        # iteration cap
        rc, st = L.lqcd_solve_batch(h, to_dev(b[:1]), x[:1], L.solver_params(tol=1e-10, max_iter=3))
        assert rc == L.LQCD_ERR_NOT_CONVERGED and st[0]["status"] == L.LQCD_ERR_NOT_CONVERGED
        # wall-clock budget
        rc, st = L.lqcd_solve_batch(h, to_dev(b[:1]), x[:1], L.solver_params(tol=1e-14, timeout_ms=1e-6))
        assert rc == L.LQCD_ERR_TIMEOUT
        # invalid parameters
        with pytest.raises(L.LqcdError):
            L.lqcd_solve_batch(h, to_dev(b[:1]), x[:1], L.solver_params(tol=-1.0))


def test_solve_with_host_buffers():
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 0)
    b = gaussian_spinors(dims, 2, 8).reshape(2, 256, 4, 3)
    with lattice(dims, U, 0.125) as (L, h):
        bh = torch.from_numpy(b).pin_memory()
        xh = torch.empty_like(bh).pin_memory()
        rc, st = L.lqcd_solve_batch(h, bh, xh, L.solver_params(tol=1e-11))
        assert rc == 0
        xd = torch.empty((2, 256, 4, 3), dtype=torch.complex128, device="cuda")
        L.lqcd_solve_batch(h, to_dev(b), xd, L.solver_params(tol=1e-11))
        assert torch.equal(xh, xd.cpu())


def _golden_rows(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    return [line.split() for line in open(path) if line.strip() and not line.startswith("#")]


def test_noise_signs_match_golden_philox_words():
    """GPU noise against stored words of an independent Philox4x64-10 (tests/golden):
    bits 2k / 2k + 1 of word 0 are the signs of Re / Im of component k."""
    L_ = __import__("tests._gpu", fromlist=["require_gpu"]).require_gpu()
    dims = (16, 16, 16, 32)
    V = int(np.prod(dims))
    by_vec = {}
    for r in _golden_rows("philox4x64_words.txt"):
        seed, stream, ni, site, w0 = (int(v) for v in r[:5])
        by_vec.setdefault((seed, stream, ni), []).append((site, w0))
    for (seed, stream, ni), items in by_vec.items():
        out = torch.empty((1, V, 4, 3), dtype=torch.complex128, device="cuda")
        L_.lqcd_noise_generate(seed, stream, ni, dims, L_.LQCD_DILUTE_NONE, 0, 1, out)
        got = out.cpu().numpy().reshape(V, 12)
        for site, w0 in items:
            for k in range(12):
                re_neg, im_neg = (w0 >> (2 * k)) & 1, (w0 >> (2 * k + 1)) & 1
                assert (got[site, k].real < 0) == bool(re_neg) and (got[site, k].imag < 0) == bool(im_neg)
                assert abs(abs(got[site, k]) - 1.0) < 1e-15


def test_free_field_exact_loops_match_golden_traces():
    """Point-source FP64 solves of the free field against the closed-form traces (tests/golden)."""
    for r in _golden_rows("free_field_loops.txt"):
        dims = tuple(int(v) for v in r[:4])
        kappa, trace = float(r[4]), float(r[5])
        V = int(np.prod(dims))
        with lattice(dims, unit_gauge_field(dims), kappa) as (L, h):
            sites = [0, V - 1]
            src = torch.empty((12 * len(sites), V, 4, 3), dtype=torch.complex128, device="cuda")
            L.lqcd_point_sources(h, sites, src)
            x = torch.empty_like(src)
            rc, st = L.lqcd_solve_batch(h, src, x, L.solver_params(tol=1e-13, precision=L.LQCD_PREC_FP64))
            assert rc == 0
            per_site = torch.zeros((V, 6), dtype=torch.complex128, device="cuda")
            L.lqcd_loops_batch(h, src, x, 1.0, per_site, None)
            got = per_site.cpu().numpy()
        for s in sites:
            assert abs(got[s, 0] - trace) < 1e-10
            assert np.max(np.abs(got[s, 1:])) < 1e-12
