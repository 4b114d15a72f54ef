"""Autograd through the AM-QFT kernels: the gradient of a spectral loss
against the oracle's adjoint (2 F^H (w . X), float64) and against float64
central finite differences of the oracle's loss; the adjoint identity."""
import numpy as np
import pytest

import synth
from gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch

    from paper_1404_1810_gb300 import build, load

    assert torch.cuda.is_available()
    build.build()
    return load()


def _loss_and_grad(xr, w, variant):
    """GPU: real signals lifted to complex, L = sum_b sum_k w_k |X_bk|^2."""
    import torch

    from paper_1404_1810_gb300 import amqft_autograd as amqft

    xt = torch.tensor(xr, dtype=torch.float32, device="cuda", requires_grad=True)
    wt = torch.tensor(w, dtype=torch.float32, device="cuda")
    z = torch.complex(xt, torch.zeros_like(xt))
    X = amqft(z, variant)
    loss = (wt * (X.real ** 2 + X.imag ** 2)).sum()
    loss.backward()
    return float(loss.item()), xt.grad.double().cpu().numpy()


@pytest.mark.parametrize("v", [4, 2])
def test_gradient_matches_oracle_adjoint(orc, v):
    n, b = 1 << 14, 6
    xr = synth.real_signals(n, b, stream=3)
    w = synth.spectral_mask(n)
    _, g = _loss_and_grad(xr, w, v)
    x32 = xr.astype(np.float32).astype(np.float64)
    for i in range(b):
        X = orc.amqft(x32[i].astype(np.complex128), v)
        G = orc.amqft(w * X, v, sign=+1)          # F^H (w . X)
        ref = 2.0 * G.real
        assert rel(g[i], ref) < 1e-4, (v, i, rel(g[i], ref))


@pytest.mark.parametrize("v", [4, 2, 1, 8])
def test_gradient_finite_differences_n64(orc, v):
    n, b = 64, 2
    xr = synth.real_signals(n, b, stream=4)
    w = synth.spectral_mask(n, stream=2)
    _, g = _loss_and_grad(xr, w, v)
    x64 = xr.astype(np.float32).astype(np.float64)

    def loss64(x):
        return sum(float(np.sum(w * np.abs(orc.amqft(x[i].astype(np.complex128), v)) ** 2)) for i in range(b))

    h = 1e-6
    fd = np.zeros_like(x64)
    for i in range(b):
        for j in range(n):
            xp = x64.copy()
            xm = x64.copy()
            xp[i, j] += h
            xm[i, j] -= h
            fd[i, j] = (loss64(xp) - loss64(xm)) / (2 * h)
    assert rel(g, fd) < 1e-4, rel(g, fd)


@pytest.mark.parametrize("log2n", [10, 16, 17])
def test_adjoint_identity(log2n):
    """<F x, y> = <x, F^H y>, and the backward of the inverse is the forward."""
    import torch

    from paper_1404_1810_gb300 import amqft_autograd as amqft

    n, b = 1 << log2n, 2
    x = synth.device_normal_complex64(n, b, "cuda", seed_offset=11)
    y = synth.device_normal_complex64(n, b, "cuda", seed_offset=12)
    fx = amqft(x).reshape(-1).to(torch.complex128)
    yy = y.reshape(-1).to(torch.complex128)
    lhs = torch.vdot(fx, yy)
    rhs = torch.vdot(x.reshape(-1).to(torch.complex128), amqft(y, inverse=True).reshape(-1).to(torch.complex128))
    # float32 rounding bounds the difference relative to |Fx| |y| (Cauchy-Schwarz)
    scale = float(torch.linalg.norm(fx) * torch.linalg.norm(yy))
    assert abs(complex(lhs - rhs)) / scale < 1e-6
    xi = x.clone().requires_grad_(True)
    out = amqft(xi, inverse=True)
    (out.real.sum()).backward()
    # d/dx of sum Re(F^H x) = F (ones) under the conjugate convention
    ones = torch.ones_like(x)
    assert torch.allclose(xi.grad, amqft(ones), rtol=0, atol=0)


def test_rejects_cpu_tensors():
    import torch

    from paper_1404_1810_gb300 import amqft_autograd as amqft

    with pytest.raises(ValueError):
        amqft(torch.zeros(8, dtype=torch.complex64))
