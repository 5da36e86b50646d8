"""The FP64 reference of the learned-guess network: analytic gradient
against central finite differences (CPU)."""
import numpy as np

from oracle import mlp


def test_reference_gradient_by_finite_differences():
    g = np.random.default_rng(3)
    n = 7
    p = g.normal(scale=0.05, size=mlp.H * mlp.IN + mlp.H + mlp.H * mlp.H + mlp.H + mlp.OUT * mlp.H + mlp.OUT)
    X = g.normal(size=(n, mlp.IN))
    T = g.normal(scale=0.1, size=(n, mlp.OUT))
    head = [0, 1, 2, 3, 4, 1, 3]
    loss, grad = mlp.loss_and_grad(p, X, T, head)
    idx = g.choice(p.size, 40, replace=False)
    idx = np.concatenate([idx, [0, mlp.H * mlp.IN, p.size - 1]])   # W1, b1, b3
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (mlp.loss_and_grad(p + e, X, T, head)[0] - mlp.loss_and_grad(p - e, X, T, head)[0]) / 2e-6
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, grad[i])
    # masking: outputs outside a sample's head do not change the loss
    T2 = T.copy()
    T2[0, 100:] += 5.0
    assert abs(mlp.loss_and_grad(p, X, T2, head)[0] - loss) < 1e-14
