"""Pins of the warm-start network oracle (oracle/mlp.py) against mathematics
and library routines: central finite differences, a least-squares fixed
point, torch's bfloat16 conversion and torch.optim.Adam."""
import numpy as np
import pytest
import torch

import lbm_inputs as I
from oracle import mlp as M


def _net(seed, n_in=3, width=5, n_layers=4, n_out=2, n=7):
    sizes = M.layer_sizes(n_in, width, n_layers, n_out)
    theta = I.mlp_init(seed, n_in, width, n_layers, n_out, bias_scale=0.3).astype(np.float64)
    x, t = I.mlp_batch(seed + 1, n, n_in, n_out)
    return sizes, theta, x.astype(np.float64), t.astype(np.float64)


@pytest.mark.parametrize("n_layers", [1, 2, 4])
def test_gradient_matches_finite_differences(n_layers):
    sizes, theta, x, t = _net(3, n_layers=n_layers)
    E, g = M.loss_grad(theta, sizes, x, t)
    h = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (M.loss_grad(tp, sizes, x, t)[0] - M.loss_grad(tm, sizes, x, t)[0]) / (2 * h)
    assert E > 0
    assert np.max(np.abs(g - fd)) <= 1e-8 * max(1.0, np.max(np.abs(fd)))


def test_one_layer_descent_reaches_least_squares():
    # A network of one linear layer is a linear least-squares fit with bias:
    # gradient descent on the mean squared error converges to lstsq's solution.
    rng = np.random.default_rng(5)
    n, n_in, n_out = 40, 3, 2
    x = rng.uniform(-1, 1, (n, n_in))
    t = rng.normal(size=(n, n_out))
    sizes = M.layer_sizes(n_in, 8, 1, n_out)
    theta = np.zeros(M.param_count(n_in, 8, 1, n_out))
    for _ in range(4000):
        theta -= 0.5 * M.loss_grad(theta, sizes, x, t)[1]
    A = np.hstack([x, np.ones((n, 1))])
    beta = np.linalg.lstsq(A, t, rcond=None)[0]  # [n_in + 1][n_out]
    (W, b), = M.unflatten(theta, sizes)
    np.testing.assert_allclose(W, beta[:n_in].T, atol=1e-9)
    np.testing.assert_allclose(b, beta[n_in], atol=1e-9)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        # exact ties: 1 + (2k+1) 2^-8 lies half-way between bfloat16 neighbours
                        1.0 + (2 * np.arange(64) + 1) * 2.0 ** -8, [0.0, -0.0, 1.0, -3.5]])
    v = v.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(v).float().to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(M.bf16_round(v), ref)


def test_adam_matches_torch():
    rng = np.random.default_rng(9)
    theta0 = rng.normal(size=50)
    p = torch.nn.Parameter(torch.from_numpy(theta0.copy()))
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.99), eps=1e-7)
    theta, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for k in range(1, 8):
        g = rng.normal(size=50) * k
        p.grad = torch.from_numpy(g.copy())
        opt.step()
        theta, m, v = M.adam_step(theta, g, m, v, k, 3e-3, 0.9, 0.99, 1e-7)
    np.testing.assert_allclose(theta, p.detach().numpy(), rtol=0, atol=1e-14)


def test_bf16_mode_is_a_small_perturbation():
    sizes, theta, x, t = _net(4, n_in=7, width=64, n_layers=4, n_out=3, n=256)
    E, g = M.loss_grad(theta, sizes, x, t)
    Eb, gb = M.loss_grad(theta, sizes, x, t, bf16=True)
    assert abs(Eb - E) < 2e-2 * E
    assert np.linalg.norm(gb - g) < 5e-2 * np.linalg.norm(g)
    # the stored quantities really are bfloat16 values
    y, hs = M.forward(theta, sizes, x, bf16=True)
    for h in hs:
        np.testing.assert_array_equal(M.bf16_round(h), h)
