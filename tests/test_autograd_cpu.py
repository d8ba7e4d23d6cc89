"""CPU checks of the Python layer's differentiable helpers against the oracle."""

import numpy as np
import pytest

from oracle import tv
from paper_1705_07497_gb300 import inputs

torch = pytest.importorskip("torch")


def test_torch_gradient_helpers_match_oracle():
    from paper_1705_07497_gb300.autograd import grad2d, grad2d_adj, shrink

    n = 9
    u = inputs.random_vector(n * n * 2, 80).reshape(n * n, 2)
    w = inputs.random_vector(n * n * 4, 81).reshape(2, n * n, 2)
    gx, gy = grad2d(torch.tensor(u), n)
    for b in range(2):
        ox, oy = tv.grad(u[:, b].reshape(n, n))
        np.testing.assert_allclose(gx[:, b].numpy(), ox.ravel(), atol=1e-15)
        np.testing.assert_allclose(gy[:, b].numpy(), oy.ravel(), atol=1e-15)
        want = tv.grad_adj(w[0][:, b].reshape(n, n), w[1][:, b].reshape(n, n)).ravel()
        got = grad2d_adj(torch.tensor(w[0]), torch.tensor(w[1]), n)[:, b].numpy()
        np.testing.assert_allclose(got, want, atol=1e-15)
    x = torch.tensor(inputs.random_vector(50, 82) * 3)
    np.testing.assert_allclose(shrink(x, 1.3).numpy(), tv.shrink(x.numpy(), 1.3), atol=0)
