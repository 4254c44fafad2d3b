"""Shared helpers for the GPU tests: a lattice context driven through the C ABI."""
import contextlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1108_2473_gb300 import build_lib
    build_lib.build()
    from paper_1108_2473_gb300 import lqcd
    lqcd.load()
    return lqcd


@contextlib.contextmanager
def lattice(dims, U=None, kappa=None):
    L = require_gpu()
    h = L.lqcd_create(dims, 0)
    try:
        if U is not None:
            L.lqcd_set_gauge(h, torch.from_numpy(np.ascontiguousarray(U).reshape(-1)).cuda())
        if kappa is not None:
            L.lqcd_set_kappa(h, kappa)
        yield L, h
    finally:
        L.lqcd_destroy(h)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_np(t, dims=None):
    a = t.detach().cpu().numpy()
    if dims is not None:
        lx, ly, lz, lt = dims
        a = a.reshape(a.shape[:1] + (lt, lz, ly, lx, 4, 3))
    return a


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
