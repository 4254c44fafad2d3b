"""Checkpoint / resume of stochastic loop runs (paper_1108_2473_gb300/checkpoint.py).

CPU: the accumulators survive a save / load round trip exactly and the run hash
changes with every part of the run definition.  GPU: a run interrupted after two
noise vectors and resumed from its checkpoint in a fresh context reproduces the
uninterrupted run bit for bit, and a checkpoint of another run is refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _solver():
    from paper_1108_2473_gb300 import lqcd as L
    return L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_BF16)


def test_save_load_roundtrip_and_hash(tmp_path):
    from paper_1108_2473_gb300 import checkpoint as ck
    rng = np.random.default_rng(1)
    ps = torch.from_numpy(rng.normal(size=(16, 6)) + 1j * rng.normal(size=(16, 6)))
    pt = torch.from_numpy(rng.normal(size=(4, 6)) + 1j * rng.normal(size=(4, 6)))
    path = str(tmp_path / "run.npz")
    ck.save(path, ps, pt, 7, 7, "abc")
    a, b, nxt, done, h = ck.load(path)
    assert np.array_equal(a, ps.numpy()) and np.array_equal(b, pt.numpy())
    assert (nxt, done, h) == (7, 7, "abc")
    U = rng.normal(size=(2, 2, 2, 2, 4, 3, 3)) + 0j
    base = ck.config_hash((2, 2, 2, 2), 0.12, 5, 3, _solver(), U)
    assert base == ck.config_hash((2, 2, 2, 2), 0.12, 5, 3, _solver(), U.copy())
    U2 = U.copy()
    U2[0, 0, 0, 0, 0, 0, 0] += 1e-15
    others = [ck.config_hash((2, 2, 2, 4), 0.12, 5, 3, _solver(), U), ck.config_hash((2, 2, 2, 2), 0.13, 5, 3, _solver(), U),
              ck.config_hash((2, 2, 2, 2), 0.12, 6, 3, _solver(), U), ck.config_hash((2, 2, 2, 2), 0.12, 5, 2, _solver(), U),
              ck.config_hash((2, 2, 2, 2), 0.12, 5, 3, _solver(), U2)]
    assert len({base, *others}) == 6


@pytest.mark.gpu
def test_interrupted_run_resumes_bit_identically(tmp_path):
    from lattice_inputs import eps_su3_field
    from paper_1108_2473_gb300 import checkpoint as ck
    from tests._gpu import lattice
    dims = (4, 4, 4, 8)
    U = eps_su3_field(dims, 0.35, 3)
    kappa, seed, n = 0.12, 21, 4
    with lattice(dims, U, kappa) as (L, h):
        full_ps, full_pt, done = ck.run_stochastic(h, dims, kappa, seed, n, U)
        assert done == n
    path = str(tmp_path / "ck.npz")
    with lattice(dims, U, kappa) as (L, h):
        _, _, done = ck.run_stochastic(h, dims, kappa, seed, n, U, path=path, stop_after=2)
        assert done == 2
    with lattice(dims, U, kappa) as (L, h):  # a fresh context, as after a restart
        ps, pt, done = ck.run_stochastic(h, dims, kappa, seed, n, U, path=path)
        assert done == n
        assert torch.equal(ps, full_ps) and torch.equal(pt, full_pt)
        with pytest.raises(ValueError):
            ck.run_stochastic(h, dims, kappa + 0.001, seed, n, U, path=path)
