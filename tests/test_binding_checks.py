"""The Python binding checks array arguments before any C call (no GPU needed):
a wrong dtype, a wrong element count or a host tensor where device memory is
required raises ValueError instead of letting a kernel run past an allocation."""
import pytest

torch = pytest.importorskip("torch")

from paper_1108_2473_gb300 import lqcd as L  # noqa: E402

DIMS = (4, 4, 4, 4)
V = 256


def test_noalloc_rejects_wrong_dtype_and_size():
    src = torch.zeros((2, V, 4, 3), dtype=torch.complex128)
    with pytest.raises(ValueError, match="complex128"):
        L.lqcd_loops_batch_noalloc(DIMS, src.to(torch.complex64), src, 1.0, None, None)
    with pytest.raises(ValueError, match="elements"):
        L.lqcd_loops_batch_noalloc(DIMS, src, src[:1], 1.0, None, None)
    with pytest.raises(ValueError, match="elements"):  # per_t must be [Lt][6]
        L.lqcd_loops_batch_noalloc(DIMS, src, src, 1.0, None, torch.zeros((5, 6), dtype=torch.complex128))
    with pytest.raises(ValueError, match="CUDA"):  # host arrays are refused before the C call
        L.lqcd_loops_batch_noalloc(DIMS, src, src, 1.0, None, torch.zeros((4, 6), dtype=torch.complex128))


def test_noise_output_size_checked():
    out = torch.zeros((2, V, 4, 3), dtype=torch.complex128)
    with pytest.raises(ValueError, match="elements"):
        L.lqcd_noise_generate(1, 0, 0, DIMS, L.LQCD_DILUTE_TSC, 0, 3, out)
    with pytest.raises(ValueError, match="complex128"):
        L.lqcd_noise_generate(1, 0, 0, DIMS, L.LQCD_DILUTE_TSC, 0, 2, out.real.contiguous())


def test_context_arrays_checked_against_the_lattice():
    # a context record as lqcd_create leaves it (dims and device), without a GPU
    fake = 0x1234
    L._CTX[fake] = (DIMS, 0)
    try:
        b = torch.zeros((3, V, 4, 3), dtype=torch.complex128)
        with pytest.raises(ValueError, match="elements"):
            L.lqcd_solve_batch(fake, b, torch.zeros((3, V + 2, 4, 3), dtype=torch.complex128), L.solver_params())
        with pytest.raises(ValueError, match="elements"):
            L.lqcd_loops_batch(fake, b, b, 1.0, None, torch.zeros((3, 6), dtype=torch.complex128))
        with pytest.raises(ValueError, match="coef"):
            L.lqcd_gradient(fake, b, b, [[0.0] * 6] * 3, L.solver_params())
    finally:
        del L._CTX[fake]
    with pytest.raises(ValueError, match="unknown"):
        L.lqcd_loops_batch(0x5678, b, b)
