"""The no-allocation loop contraction against the regular one, through the C ABI.

lqcd_loops_batch_noalloc serves callers that cannot allocate device memory:
frameworks whose caching allocator already holds the GPU, pipelines that
cannot take the device synchronisation of cudaFree, services under a fixed
memory budget.  Its partial sums live in a fixed array inside the library that
every call shares, so this test calls it twice in a row with different inputs:
the second result must not be polluted by the first.  It also checks the size
limit, the per-site-only form (no partial sums at all) and that the call needs
no context.  This file is collected last so that a stop at its first failure
has already run every other test.
"""
import numpy as np
import pytest

from lattice_inputs import gaussian_spinors
from tests._gpu import lattice, to_dev, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (16, 16, 16, 32), (6, 4, 2, 8)])
def test_noalloc_matches_loops_batch_two_calls(dims):
    V = int(np.prod(dims))
    n = 3
    with lattice(dims) as (L, h):
        for call in range(2):
            src = to_dev(gaussian_spinors(dims, n, 40 + call).reshape(n, V, 4, 3))
            sol = to_dev(gaussian_spinors(dims, n, 50 + call).reshape(n, V, 4, 3))
            w = 0.25 + call
            ps_a = torch.zeros((V, 6), dtype=torch.complex128, device="cuda")
            pt_a = torch.zeros((dims[3], 6), dtype=torch.complex128, device="cuda")
            ps_b = torch.zeros_like(ps_a)
            pt_b = torch.zeros_like(pt_a)
            L.lqcd_loops_batch(h, src, sol, w, ps_a, pt_a)
            L.lqcd_loops_batch_noalloc(dims, src, sol, w, ps_b, pt_b)
            torch.cuda.synchronize()
            assert rel_err(ps_b.cpu().numpy(), ps_a.cpu().numpy()) < 1e-14
            assert rel_err(pt_b.cpu().numpy(), pt_a.cpu().numpy()) < 1e-14


def test_noalloc_per_site_only_two_calls():
    """per_t = NULL: only per-site loops, which need no partial sums."""
    dims = (8, 4, 4, 6)
    V = int(np.prod(dims))
    n = 2
    with lattice(dims) as (L, h):
        for call in range(2):
            src = to_dev(gaussian_spinors(dims, n, 60 + call).reshape(n, V, 4, 3))
            sol = to_dev(gaussian_spinors(dims, n, 70 + call).reshape(n, V, 4, 3))
            ps_a = torch.zeros((V, 6), dtype=torch.complex128, device="cuda")
            ps_b = torch.zeros_like(ps_a)
            L.lqcd_loops_batch(h, src, sol, 1.5, ps_a, None)
            L.lqcd_loops_batch_noalloc(dims, src, sol, 1.5, ps_b, None)
            torch.cuda.synchronize()
            assert rel_err(ps_b.cpu().numpy(), ps_a.cpu().numpy()) < 1e-14


def test_noalloc_rejects_lattice_beyond_scratch():
    """The library's own limit check (called through the raw C entry point, so
    that the binding's size checks do not stop the call first)."""
    import ctypes
    from tests._gpu import require_gpu
    L = require_gpu()
    dims = (32, 32, 32, 64)  # 64 * 256 = 16384 partial blocks > 8192
    buf = torch.zeros((64, 6), dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    rc = L.load().lqcd_loops_batch_noalloc(L._dims(dims), p, p, 1, 1.0, None, p, L._stream(buf))
    assert rc == L.LQCD_ERR_INVALID and "scratch" in L.lqcd_last_error(None)
    # a volume beyond 2^30 sites is refused before any size arithmetic
    rc = L.load().lqcd_loops_batch_noalloc(L._dims((2048, 2048, 2, 256)), p, p, 1, 1.0, p, None, L._stream(buf))
    assert rc == L.LQCD_ERR_INVALID


def test_noalloc_rejects_host_arrays():
    """A host array is refused by the binding and, through the raw C entry
    point, by the library itself (no kernel is launched on host memory)."""
    import ctypes
    from tests._gpu import require_gpu
    L = require_gpu()
    dims = (4, 4, 4, 4)
    src = torch.zeros((1, 256, 4, 3), dtype=torch.complex128, device="cuda")
    pt_host = torch.zeros((4, 6), dtype=torch.complex128)
    with pytest.raises(ValueError):
        L.lqcd_loops_batch_noalloc(dims, src, src, 1.0, None, pt_host)
    ps = ctypes.c_void_p(src.data_ptr())
    rc = L.load().lqcd_loops_batch_noalloc(L._dims(dims), ps, ps, 1, 1.0, None, ctypes.c_void_p(pt_host.data_ptr()),
                                           L._stream(src))
    assert rc == L.LQCD_ERR_INVALID and "per_t" in L.lqcd_last_error(None)
