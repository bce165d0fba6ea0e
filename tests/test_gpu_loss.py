"""The fused reconstruction loss f = ||G x_1 U1 ... x_N UN - A||^2
(reconstruction_loss / tucker_reconstruction_loss) against independent references:
f against the FP64 reconstruction computed with torch from the same G and U
(relative 1e-5 in FP32, 1e-12 in FP64); D = df/dB against 2 (B - A) with B the
library's own reconstruction (the loss form shares its accumulation: 1e-6 of the
largest entry); the gradients with respect to A, G and U against autograd of the
eager composite ((A - tucker_reconstruct(G, U))^2).sum() (1e-5 / 1e-10 relative),
with a unit and a non-unit output gradient. Shapes: views the register-tiled loss
form takes (the last expansion on a Q = 1 view and on a column view) and odd
sizes where it falls back to the elementwise pass."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W


@pytest.fixture(scope="module")
def tals():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2004_02583_gb300 as pkg
    pkg.lib()
    return pkg


CASES = [
    ((64, 48, 40), (8, 6, 4)),
    ((96, 80, 64), (16, 12, 8)),
    ((30, 21, 17), (5, 4, 3)),
    ((24, 20, 16, 12), (4, 5, 3, 2)),
]


def _inputs(dims, ranks, dtype, seed):
    A = torch.from_numpy(W.uniform_tensor(seed, dims, dtype=dtype)).cuda()
    G = torch.from_numpy(W.uniform_tensor(seed + 1, ranks, dtype=dtype)).cuda()
    Us = [torch.from_numpy(W.orthonormal(seed + 2 + n, d, r, dtype=dtype)).cuda() for n, (d, r) in
          enumerate(zip(dims, ranks))]
    return A, G, Us


def _reconstruct64(G, Us):
    b = G.double()
    for n, u in enumerate(Us):
        b = torch.movedim(torch.tensordot(u.double(), b, dims=([1], [n])), 0, n)
    return b


@pytest.mark.parametrize("dims,ranks", CASES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_loss_value_and_gradient_of_reconstruction(tals, dims, ranks, dtype):
    A, G, Us = _inputs(dims, ranks, dtype, W.SEED_BASE + 81)
    f, D = tals.reconstruction_loss(A, G, Us)
    b64 = _reconstruct64(G, Us)
    f_ref = float(((b64 - A.double()) ** 2).sum())
    tol = 1e-5 if dtype == np.float32 else 1e-12
    assert abs(float(f) - f_ref) <= tol * f_ref, (float(f), f_ref)
    B = tals.reconstruct(G, Us)
    d_ref = 2 * (B - A)
    assert float((D - d_ref).abs().max()) <= 1e-6 * float(d_ref.abs().max())


@pytest.mark.parametrize("dims,ranks", CASES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("scale", [1.0, 3.0])
def test_loss_gradients_match_eager_composite(tals, dims, ranks, dtype, scale):
    A0, G0, U0 = _inputs(dims, ranks, dtype, W.SEED_BASE + 82)
    grads = []
    for fused in (True, False):
        A = A0.clone().requires_grad_(True)
        G = G0.clone().requires_grad_(True)
        Us = [u.clone().requires_grad_(True) for u in U0]
        if fused:
            f = tals.tucker_reconstruction_loss(A, G, Us)
        else:
            f = ((A - tals.tucker_reconstruct(G, Us)) ** 2).sum().double()
        (scale * f).backward()
        grads.append([A.grad, G.grad] + [u.grad for u in Us])
    tol = 1e-5 if dtype == np.float32 else 1e-10
    for gf, ge in zip(*grads):
        assert float((gf - ge).norm()) <= tol * float(ge.norm()), (float((gf - ge).norm()), float(ge.norm()))


def test_loss_refuses_aliasing_output(tals):
    A, G, Us = _inputs((20, 16, 12), (3, 3, 3), np.float32, W.SEED_BASE + 83)
    import ctypes
    dims = (ctypes.c_int64 * 3)(20, 16, 12)
    ranks = (ctypes.c_int * 3)(3, 3, 3)
    f = torch.empty((), dtype=torch.float64, device="cuda")
    st = tals.lib().reconstruction_loss(G.data_ptr(), tals._ptrs(Us), A.data_ptr(), tals.TALS_F32, 3, dims, ranks,
                                        A.data_ptr(), f.data_ptr(), None)
    assert st == tals.TALS_EINVAL
