"""CPU tests: the Python binding rejects tensors whose shape or dtype does not match
the sizes it passes to the C ABI, with ValueError, before any pointer reaches the
library (a mismatch there would read or write past the end of a device buffer)."""
import pytest

torch = pytest.importorskip("torch")

import paper_2004_02583_gb300 as tals


def _factors(dims, ranks, dtype=torch.float32):
    return [torch.zeros((d, r), dtype=dtype) for d, r in zip(dims, ranks)]


def test_project_checks_tensor_shape_and_dtypes():
    Us = _factors((6, 5, 4), (2, 3, 2))
    with pytest.raises(ValueError, match="shape"):
        tals.project(torch.zeros((6, 5, 5)), Us)
    with pytest.raises(ValueError, match="dtype"):
        tals.project(torch.zeros((6, 5, 4)), Us[:2] + [torch.zeros((4, 2), dtype=torch.float64)])
    with pytest.raises(ValueError, match="factors expected"):
        tals.project(torch.zeros((6, 5, 4)), Us[:2])
    with pytest.raises(ValueError, match="out"):
        tals.project(torch.zeros((6, 5, 4)), Us, out=torch.zeros((2, 3, 3)))


def test_reconstruct_and_adjoints_check_shapes():
    Us = _factors((6, 5, 4), (2, 3, 2))
    with pytest.raises(ValueError, match="shape"):
        tals.reconstruct(torch.zeros((6, 5, 4)), Us)          # G must be R1 x R2 x R3
    with pytest.raises(ValueError, match="out"):
        tals.reconstruct(torch.zeros((2, 3, 2)), Us, out=torch.zeros((6, 5, 5)))
    with pytest.raises(ValueError, match="G"):
        tals.reconstruct_backward(torch.zeros((2, 3, 3)), Us, torch.zeros((6, 5, 4)))
    with pytest.raises(ValueError, match="shape"):
        tals.reconstruct_backward(torch.zeros((2, 3, 2)), Us, torch.zeros((6, 5, 3)))
    with pytest.raises(ValueError, match="G_bar"):
        tals.project_backward(torch.zeros((6, 5, 4)), Us, torch.zeros((2, 2, 2)))
    with pytest.raises(ValueError, match="dtype"):
        tals.project_backward(torch.zeros((6, 5, 4)), Us, torch.zeros((2, 3, 2), dtype=torch.float64))


def test_sweep_pass_checks_basis():
    A = torch.zeros((8, 6, 4))
    with pytest.raises(ValueError, match="Q must be"):
        tals.sweep_pass(A, 0, torch.zeros((6, 2)))
    with pytest.raises(ValueError, match="FP32"):
        tals.sweep_pass(A, 0, torch.zeros((8, 2), dtype=torch.float64))
    with pytest.raises(ValueError, match="mode"):
        tals.sweep_pass(A, 3, torch.zeros((8, 2)))
    with pytest.raises(ValueError, match="engine"):
        tals.sweep_pass(A, 0, torch.zeros((8, 2)), engine="fp16")


def test_host_context_checks_buffer_sizes():
    hc = object.__new__(tals.HostContext)
    hc.ndim, hc.dims, hc.ranks, hc._code = 3, [6, 5, 4], [2, 3, 2], tals.TALS_F32
    good_u = [torch.zeros((6, 2)), torch.zeros((5, 3)), torch.zeros((4, 2))]
    hc._check_host(torch.zeros((6, 5, 4)), torch.zeros((2, 3, 2)), good_u)
    with pytest.raises(ValueError, match="A_host"):
        hc._check_host(torch.zeros((6, 5, 3)), torch.zeros((2, 3, 2)), good_u)
    with pytest.raises(ValueError, match="A_host"):
        hc._check_host(torch.zeros((6, 5, 4), dtype=torch.float64), torch.zeros((2, 3, 2)), good_u)
    with pytest.raises(ValueError, match="G_host"):
        hc._check_host(torch.zeros((6, 5, 4)), torch.zeros((2, 3, 3)), good_u)
    with pytest.raises(ValueError, match="U_host"):
        hc._check_host(torch.zeros((6, 5, 4)), torch.zeros((2, 3, 2)), good_u[:2] + [torch.zeros((4, 3))])
