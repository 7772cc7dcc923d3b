"""The FP64 reference network (oracle/mlp.py) against central finite
differences: its backpropagated gradient is what the GPU training kernels are
checked against."""
import numpy as np

from oracle import mlp


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    sizes = [5, 7, 6, 4]
    theta = rng.normal(0, 0.5, mlp.n_params(sizes))
    X = rng.normal(0, 1, (9, 5))
    Y = rng.normal(0, 1, (9, 4))
    xm, xs = rng.normal(0, 0.1, 5), rng.uniform(0.5, 2.0, 5)
    ym, ys = rng.normal(0, 0.1, 4), rng.uniform(0.5, 2.0, 4)
    loss, g = mlp.loss_and_grad(theta, sizes, X, Y, xm, xs, ym, ys)
    h = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (mlp.loss_and_grad(tp, sizes, X, Y, xm, xs, ym, ys)[0] -
                 mlp.loss_and_grad(tm, sizes, X, Y, xm, xs, ym, ys)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
    out, _ = mlp.forward(theta, sizes, X, xm, xs)
    assert loss == np.mean((out - (Y - ym) / ys) ** 2)


def test_mlp_layout_counts():
    assert mlp.n_params([5, 128, 128, 128, 64]) == 5 * 128 + 128 + 2 * (128 * 128 + 128) + 128 * 64 + 64
