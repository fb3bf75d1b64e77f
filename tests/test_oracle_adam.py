"""Pin of the Adam oracle against PyTorch's Adam (the optimiser of the 3DGS training routine)."""
import numpy as np
import pytest

from oracle import adam


def test_adam_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=200)
    grads = [rng.normal(size=200) * s for s in (1.0, 0.1, 3.0, 0.0, 1e-3, 1.0, 2.0)]
    for lr, eps in ((1e-3, 1e-15), (0.05, 1e-8), (1.6e-4, 1e-15)):
        p = p0.copy()
        m = np.zeros_like(p)
        v = np.zeros_like(p)
        tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
        opt = torch.optim.Adam([tp], lr=lr, betas=(0.9, 0.999), eps=eps)
        for t, g in enumerate(grads, start=1):
            adam.step(p, g, m, v, t, lr, eps=eps)
            tp.grad = torch.tensor(g, dtype=torch.float64)
            opt.step()
            np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_zero_gradient_and_infinite_parameter_stay_put():
    p = np.array([1.0, -np.inf])
    m = np.zeros(2)
    v = np.zeros(2)
    adam.step(p, np.zeros(2), m, v, 1, 0.1)
    assert p[0] == 1.0 and p[1] == -np.inf
