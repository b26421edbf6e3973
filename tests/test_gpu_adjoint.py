"""Adjoint (transpose) kernels against the FP64 oracle's transposes, the
dot-product identity, and central finite differences of an MSE loss through
the autograd wrapper."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SHAPES = [(2,), (33,), (1000,), (6, 5), (129, 129), (65, 33), (9, 6, 5), (33, 17, 9),
          (70, 70, 70), (100, 7, 5), (17, 100, 41)]


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import hpdr
    return hpdr


@pytest.mark.parametrize("shape", SHAPES, ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_recompose_adjoint_parity(oracle, H, shape, dtype):
    g = np.random.default_rng(21).standard_normal(shape).astype(dtype)
    got = H.hpdr_recompose_adjoint(torch.from_numpy(g).cuda()).cpu().numpy().astype(np.float64)
    ref = oracle.recompose_adjoint(g.astype(np.float64))
    tol = 1e-5 if dtype == np.float32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES, ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_decompose_adjoint_parity(oracle, H, shape, dtype):
    gc = np.random.default_rng(22).standard_normal(int(np.prod(shape))).astype(dtype)
    got = H.hpdr_decompose_adjoint(torch.from_numpy(gc).cuda(), shape).cpu().numpy().astype(np.float64)
    ref = oracle.decompose_adjoint(gc.astype(np.float64), shape)
    tol = 1e-5 if dtype == np.float32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(65, 65, 65), (257, 129), (500, 6)], ids=str)
def test_dot_product_identities(H, shape):
    rng = np.random.default_rng(23)
    n = int(np.prod(shape))
    c, g, u, h = (torch.from_numpy(rng.standard_normal(n)).cuda() for _ in range(4))
    Rc = H.hpdr_recompose(c, shape).reshape(-1)
    RTg = H.hpdr_recompose_adjoint(g.reshape(shape))
    assert abs((Rc @ g - c @ RTg).item()) <= 1e-12 * Rc.abs().max().item() * g.abs().sum().item()
    Du = H.hpdr_decompose(u.reshape(shape))
    DTh = H.hpdr_decompose_adjoint(h, shape).reshape(-1)
    assert abs((Du @ h - u @ DTh).item()) <= 1e-12 * Du.abs().max().item() * h.abs().sum().item()


def test_mse_gradient_matches_finite_differences():
    """Loss = mean((R(c) - t)^2); the loss is quadratic, so central
    differences (step 1e-3, FP64) equal the gradient up to rounding."""
    from paper_2503_06322_gb300 import autograd, fields, hpdr
    shape = (65, 65, 65)
    t = torch.from_numpy(fields.powerlaw_field(shape, seed=5, dtype=np.float64)).cuda()
    u0 = torch.from_numpy(fields.powerlaw_field(shape, seed=4, dtype=np.float64)).cuda()
    c = hpdr.hpdr_decompose(u0).requires_grad_(True)
    loss = ((autograd.recompose(c, shape) - t) ** 2).mean()
    loss.backward()
    grad = c.grad.detach()
    rng = np.random.default_rng(6)
    idx = rng.choice(c.numel(), size=64, replace=False)
    h = 1e-3
    with torch.no_grad():
        for i in idx:
            cp = c.detach().clone(); cp[i] += h
            cm = c.detach().clone(); cm[i] -= h
            lp = ((hpdr.hpdr_recompose(cp, shape) - t) ** 2).mean().item()
            lm = ((hpdr.hpdr_recompose(cm, shape) - t) ** 2).mean().item()
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad[i].item()) <= 1e-6 * abs(grad).max().item() + 1e-12


def test_mse_gradient_finite_differences_257():
    """Config of the differentiation workload: 257^3 coefficients of a
    power-law field (seed 4), target seed 5, loss = mean((R(c) - t)^2),
    central differences with step 1e-3 at 64 random coordinates (seed 6),
    in FP64.  The loss is quadratic, so the central difference equals the
    gradient up to rounding; it is summed as the mean of the per-element
    differences, so the mean over 1.7e7 elements does not swamp the
    ~1e-7 gradients.  The FP64 adjoint must match to 1e-8 of max|grad|,
    the FP32 adjoint to 1e-4."""
    from paper_2503_06322_gb300 import autograd, fields, hpdr
    shape = (257, 257, 257)
    t = torch.from_numpy(fields.powerlaw_field(shape, seed=5, dtype=np.float64)).cuda()
    u0 = torch.from_numpy(fields.powerlaw_field(shape, seed=4, dtype=np.float64)).cuda()
    grads = {}
    for dt in (torch.float64, torch.float32):
        c = hpdr.hpdr_decompose(u0.to(dt)).requires_grad_(True)
        loss = ((autograd.recompose(c, shape) - t.to(dt)) ** 2).mean()
        loss.backward()
        grads[dt] = c.grad.detach().double()
    c = hpdr.hpdr_decompose(u0)
    rng = np.random.default_rng(6)
    idx = rng.choice(c.numel(), size=64, replace=False)
    h = 1e-3
    gmax = grads[torch.float64].abs().max().item()
    with torch.no_grad():
        for i in idx:
            cp = c.clone(); cp[i] += h
            cm = c.clone(); cm[i] -= h
            rp = hpdr.hpdr_recompose(cp, shape) - t
            rm = hpdr.hpdr_recompose(cm, shape) - t
            fd = ((rp * rp - rm * rm).mean() / (2 * h)).item()
            assert abs(fd - grads[torch.float64][i].item()) <= 1e-8 * gmax
            assert abs(fd - grads[torch.float32][i].item()) <= 1e-4 * gmax


def test_fp32_backward_close_to_fp64():
    from paper_2503_06322_gb300 import autograd, fields, hpdr
    shape = (129, 129, 129)
    t = torch.from_numpy(fields.powerlaw_field(shape, seed=5)).cuda()
    u0 = torch.from_numpy(fields.powerlaw_field(shape, seed=4)).cuda()
    grads = []
    for dt in (torch.float32, torch.float64):
        c = hpdr.hpdr_decompose(u0.to(dt)).requires_grad_(True)
        loss = ((autograd.recompose(c, shape) - t.to(dt)) ** 2).mean()
        loss.backward()
        grads.append(c.grad.double())
    assert (grads[0] - grads[1]).abs().max().item() <= 1e-4 * grads[1].abs().max().item()


def test_decompose_autograd_round_trip():
    from paper_2503_06322_gb300 import autograd
    shape = (33, 17, 9)
    u = torch.randn(shape, dtype=torch.float64, device="cuda", requires_grad=True)
    c = autograd.decompose(u)
    w = torch.randn_like(c)
    (c * w).sum().backward()
    from paper_2503_06322_gb300 import hpdr
    ref = hpdr.hpdr_decompose_adjoint(w, shape)
    assert torch.allclose(u.grad, ref, rtol=0, atol=1e-12 * ref.abs().max().item())
