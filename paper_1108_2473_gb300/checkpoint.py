"""Checkpoint and resume for long stochastic loop runs.

The stochastic estimator (Eq. loop stochastic) is a sum over independent noise
vectors, and the Philox counters make every vector reproducible from (seed,
stream, noise index) alone.  A run therefore checkpoints as: the FP64 sums of the
per-site and per-time-slice loops over the vectors done so far, the index of the
next vector, and a hash of everything that defines the run (lattice, kappa, seed,
dilution, solver settings, gauge field).  Resuming adds the remaining vectors to
the loaded sums in the same order, so an interrupted run reproduces an
uninterrupted one bit for bit.  All arithmetic stays in liblqcd; this module only
moves the accumulators to and from disk.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import lqcd as L


def config_hash(dims, kappa, seed, dilution, solver, gauge) -> str:
    """sha256 over the run definition; gauge: the canonical complex128 link array (host or device)."""
    h = hashlib.sha256()
    h.update(json.dumps({"dims": [int(d) for d in dims], "kappa": float(kappa), "seed": int(seed),
                         "dilution": int(dilution),
                         "solver": {f: getattr(solver, f) for f, _ in solver._fields_}}, sort_keys=True).encode())
    g = gauge.detach().cpu().numpy() if isinstance(gauge, torch.Tensor) else np.asarray(gauge)
    h.update(np.ascontiguousarray(g, dtype=np.complex128).tobytes())
    return h.hexdigest()


def save(path, per_site, per_t, next_noise, n_done, chash):
    """Write the accumulators (FP64, exact) and the resume point atomically."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, per_site=per_site.detach().cpu().numpy(), per_t=per_t.detach().cpu().numpy(),
             next_noise=np.int64(next_noise), n_done=np.int64(n_done), config_hash=np.array(chash))
    os.replace(tmp, path)


def load(path):
    with np.load(path) as z:
        return (z["per_site"], z["per_t"], int(z["next_noise"]), int(z["n_done"]), str(z["config_hash"]))


def run_stochastic(h, dims, kappa, seed, n_vectors, gauge, dilution=L.LQCD_DILUTE_TSC, solver=None, path=None,
                   every=1, stop_after=None, device="cuda"):
    """Sum of the diluted loops of noise vectors 0 .. n_vectors - 1 (stream LP), with a
    checkpoint written to ``path`` every ``every`` vectors and resumed from it if present.

    Returns (per_site [V, 6], per_t [Lt, 6], vectors done) as device complex128 sums;
    the estimator is the sum divided by the number of vectors.  ``stop_after`` ends
    the call early after that many new vectors (an interruption, for tests).  A
    checkpoint written for a different run definition raises ValueError.
    """
    solver = solver or L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_BF16)
    V = int(np.prod(dims))
    chash = config_hash(dims, kappa, seed, dilution, solver, gauge)
    per_site = torch.zeros((V, 6), dtype=torch.complex128, device=device)
    per_t = torch.zeros((dims[3], 6), dtype=torch.complex128, device=device)
    start, done = 0, 0
    if path and os.path.exists(path):
        ps, pt, start, done, saved = load(path)
        if saved != chash:
            raise ValueError(f"checkpoint {path} belongs to a different run")
        per_site.copy_(torch.from_numpy(ps))
        per_t.copy_(torch.from_numpy(pt))
    new = 0
    for r in range(start, n_vectors):
        sp = L.stochastic_params(seed=seed, n_lp=1, n_hp=0, tol_lp=solver.tol, dilution=dilution, first_noise=r)
        rc, _ = L.lqcd_loops_stochastic(h, sp, solver, per_site, per_t)
        if rc != L.LQCD_OK:
            raise L.LqcdError(rc, f"noise vector {r} did not converge")
        done += 1
        new += 1
        if path and (done % every == 0 or r == n_vectors - 1):
            save(path, per_site, per_t, r + 1, done, chash)
        if stop_after is not None and new >= stop_after:
            break
    return per_site, per_t, done
