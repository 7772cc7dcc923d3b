"""The warm-start network's CUDA training kernels against the FP64 reference
(oracle/mlp.py): loss and gradient, prediction, and training progress."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu
SIZES = [5, 128, 128, 128, 64]


def setup(lbm, seed=3, n=300):
    rng = np.random.default_rng(seed)
    net = lbm.WarmStartNet(seed=seed)
    theta = rng.normal(0, 0.08, net.n_params).astype(np.float32)
    net.set_params(theta)
    X = rng.uniform([0.5, 0.55, -0.4, 0.06, 10], [0.9, 1.2, -0.2, 1.0, 128], (n, 5)).astype(np.float32)
    Y = rng.normal(-3, 1.5, (n, 64)).astype(np.float32)
    xm, xs = X.mean(0), X.std(0)
    ym, ys = Y.mean(0), Y.std(0)
    net.set_scaling(xm, xs, ym, ys)
    return net, theta, X, Y, (xm, xs, ym, ys)


def test_gradient_matches_fp64_reference(lbm):
    net, theta, X, Y, sc = setup(lbm)
    loss, g = net.loss_grad(X, Y)
    ref_loss, ref_g = mlp.loss_and_grad(theta.astype(np.float64), SIZES, X, Y, *[s.astype(np.float64) for s in sc])
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    assert np.abs(g - ref_g).max() < 1e-4 * np.abs(ref_g).max()
    # per-layer relative error of the gradient blocks
    rel = np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g)
    assert rel < 1e-4
    net.close()


def test_predict_matches_fp64_reference(lbm):
    net, theta, X, Y, (xm, xs, ym, ys) = setup(lbm, seed=4, n=50)
    out = net.predict(X)
    ref, _ = mlp.forward(theta.astype(np.float64), SIZES, X, xm, xs)
    np.testing.assert_allclose(out, ref * ys + ym, rtol=0, atol=1e-4 * np.abs(ref * ys + ym).max())
    net.close()


def test_training_fits_a_smooth_map(lbm):
    """Adam on minibatches drives the loss on a smooth synthetic map (a tanh
    interface profile whose centre and levels depend on the inputs) down by
    two orders of magnitude."""
    rng = np.random.default_rng(9)
    n = 1500
    X = rng.uniform([0.5, 0.55, -0.304, 0.06, 10], [0.9, 1.2, -0.304, 1.0, 128], (n, 5)).astype(np.float32)
    s = (np.arange(64) + 0.5) / 32
    lo, hi = -6 + 4 * (X[:, :1] - 0.5), -1.0 + 0.3 * X[:, 3:4]
    Y = (lo + (hi - lo) * 0.5 * (1 - np.tanh((s[None, :] - 1) * (2 + X[:, 4:5] / 16)))).astype(np.float32)
    net = lbm.WarmStartNet(seed=1)
    xs = X.std(0)
    xs[xs == 0] = 1
    net.set_scaling(X.mean(0), xs, Y.mean(0), Y.std(0))
    l0, _ = net.loss_grad(X, Y)
    l1 = net.train(X, Y, epochs=300, batch=250, lr=2e-3, seed=1)
    assert l1 < l0 / 100
    pred = net.predict(X)
    assert np.abs(pred - Y).max() < 0.25
    net.close()
