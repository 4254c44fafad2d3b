"""The no-allocation loop contraction against the regular one, through the C ABI.

lqcd_loops_batch_noalloc serves callers that cannot allocate device memory
(inside stream capture, under a framework's caching allocator, or where the
device synchronisation of cudaFree is not acceptable).  Its partial sums live
in a fixed array inside the library that every call shares, so this test calls
it twice in a row with different inputs: the second result must not be
polluted by the first.  It also checks the size limit and that the call needs
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


def test_noalloc_rejects_lattice_beyond_scratch():
    from tests._gpu import require_gpu
    L = require_gpu()
    dims = (32, 32, 32, 64)  # 64 * 256 = 16384 partial blocks > 8192
    src = torch.zeros((1, 4, 3), dtype=torch.complex128, device="cuda")
    pt = torch.zeros((64, 6), dtype=torch.complex128, device="cuda")
    with pytest.raises(L.LqcdError) as e:
        L.lqcd_loops_batch_noalloc(dims, src, src, 1.0, None, pt)
    assert e.value.code == L.LQCD_ERR_INVALID and "scratch" in str(e.value)


def test_noalloc_rejects_host_arrays():
    from tests._gpu import require_gpu
    L = require_gpu()
    dims = (4, 4, 4, 4)
    src = torch.zeros((1, 256, 4, 3), dtype=torch.complex128, device="cuda")
    pt_host = torch.zeros((4, 6), dtype=torch.complex128)
    with pytest.raises(L.LqcdError):
        L.lqcd_loops_batch_noalloc(dims, src, src, 1.0, None, pt_host)
