"""GPU parity of the warm-start network kernels against the FP64 oracle
(oracle/mlp.py in bfloat16 mode, which rounds exactly the quantities the
kernels store in bfloat16): forward pass, loss and gradient, Adam step, and
the per-site feature / warm-start field kernels."""
import numpy as np
import pytest

import lbm_inputs as I
from oracle import mlp as M

pytestmark = pytest.mark.gpu

# Ragged shapes: widths that are not multiples of the 64-wide GEMM tiles,
# batches with partial tiles, one-row batches, and the warm-start shape.
SHAPES = [
    (7, 256, 4, 3, 1000),
    (7, 256, 4, 3, 4097),
    (5, 100, 3, 2, 63),
    (3, 40, 2, 5, 1),
    (9, 72, 1, 4, 130),
]


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _net(n_in, width, n_layers, n_out, n, seed=0):
    from paper_2108_08783_gb300 import MLP
    net = MLP(n_in, width, n_layers, n_out, max_batch=max(n, 16))
    theta = I.mlp_init(seed, n_in, width, n_layers, n_out, bias_scale=0.1)
    net.set_params(theta)
    x, t = I.mlp_batch(seed + 1, n, n_in, n_out, scale=0.5)
    return net, theta, x, t, M.layer_sizes(n_in, width, n_layers, n_out)


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(shape):
    import torch
    net, theta, x, _, sizes = _net(*shape)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref, _ = M.forward(theta, sizes, x, bf16=True)
    assert _rel(y, y_ref) < 2e-3
    np.testing.assert_array_equal(net.params(), theta)


def test_forward_in_chunks_matches_one_pass():
    import torch
    from paper_2108_08783_gb300 import MLP
    theta = I.mlp_init(4, 7, 64, 3, 3)
    x, _ = I.mlp_batch(5, 1000, 7, 3)
    small = MLP(7, 64, 3, 3, max_batch=96)
    big = MLP(7, 64, 3, 3, max_batch=1000)
    small.set_params(theta)
    big.set_params(theta)
    xd = torch.from_numpy(x).cuda()
    np.testing.assert_array_equal(small.forward(xd).cpu().numpy(), big.forward(xd).cpu().numpy())


@pytest.mark.parametrize("shape", SHAPES)
def test_loss_and_gradient_match_oracle(shape):
    import torch
    net, theta, x, t, sizes = _net(*shape)
    loss, g = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    E, g_ref = M.loss_grad(theta, sizes, x, t, bf16=True)
    assert abs(loss - E) <= 1e-3 * E
    assert _rel(g, g_ref) < 1e-2
    # and against the unrounded FP64 gradient, within the bfloat16 perturbation
    _, g64 = M.loss_grad(theta, sizes, x, t)
    assert _rel(g, g64) < 5e-2


def test_adam_step_matches_oracle():
    import torch
    net, theta, x, t, sizes = _net(7, 256, 4, 3, 2048, seed=7)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    th = theta.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for k in range(1, 4):
        _, g = net.loss_grad(xd, td)  # the gradient the step will use
        loss = net.train_step(xd, td, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=True)
        th, m, v = M.adam_step(th, g.astype(np.float64), m, v, k, 1e-3, 0.9, 0.999, 1e-8)
        p = net.params()
        assert np.max(np.abs(p - th)) < 2e-6
        th = p.astype(np.float64)  # follow the FP32 master copy
        assert loss > 0


def test_training_reduces_the_loss():
    import torch
    from paper_2108_08783_gb300 import MLP
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (8192, 7)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], x[:, 2] ** 2 - x[:, 3], np.cos(x[:, 4] + x[:, 5])],
                 1).astype(np.float32)
    net = MLP(7, 256, 4, 3, max_batch=2048)
    net.set_params(I.mlp_init(0, 7, 256, 4, 3))
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = net.loss_grad(xd[:2048], td[:2048])[0]
    for it in range(400):
        s = (it * 2048) % 8192
        net.train_step(xd[s:s + 2048], td[s:s + 2048], lr=2e-3)
    last = net.loss_grad(xd[:2048], td[:2048])[0]
    assert last < 0.05 * first


def test_create_rejects_bad_sizes():
    from paper_2108_08783_gb300 import MLP, LbmError
    for args in [(0, 8, 2, 3), (7, 8, 0, 3), (7, 2000, 2, 3), (7, 8, 2, 0), (17, 8, 2, 3)]:
        with pytest.raises(LbmError):
            MLP(*args, max_batch=16)


def _frame(geo, feats=(0.5, -0.25, 1.0, 0.3, 0.2)):
    from paper_2108_08783_gb300 import warm_frame
    c = geo.meta["centre"]
    return warm_frame((c[0], c[1], 0.0), (0, 0, 1), 0.5, geo.meta["length"], geo.radius, feats,
                      rho_scale=2e-3, u_scale=0.02)


def test_warm_features_and_fields():
    import torch
    from paper_2108_08783_gb300 import MLP, Lattice
    geo = I.tube(6, 24, u_mean=0.02)
    lat = Lattice(geo.labels, geo.iolets, storage="f64", tau=0.8)
    lat.set_wall("elastic", rho0=1.0, F=0.85, kappa=10.0)
    rho_g, u_g = I.random_fields(2, geo.shape, drho=1e-3, umax=0.02)
    coords = lat.coords()
    rho0, u0 = I.gather(rho_g, coords), I.gather(u_g, coords)
    lat.init_fields(rho0, u0)
    fr = _frame(geo)
    x, t = lat.warm_features(fr)
    x, t = x.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    # host restatement of the features and targets
    c = np.array([geo.meta["centre"][0], geo.meta["centre"][1]])
    d = coords[:, :2] - c
    r = np.hypot(d[:, 0], d[:, 1])
    er = np.where(r[:, None] > 1e-12, d / np.maximum(r, 1e-300)[:, None], 0.0)
    rho_m, u_m = lat.moments()
    np.testing.assert_allclose(x[:, :5], np.broadcast_to(np.float32([0.5, -0.25, 1.0, 0.3, 0.2]), (lat.n, 5)))
    np.testing.assert_allclose(x[:, 5], (coords[:, 2] - 0.5) / 24, rtol=1e-6)
    np.testing.assert_allclose(x[:, 6], r / 6, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(t[:, 0], (rho_m - 1) / 2e-3, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(t[:, 1], (u_m[:, 0] * er[:, 0] + u_m[:, 1] * er[:, 1]) / 0.02,
                               rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(t[:, 2], u_m[:, 2] / 0.02, rtol=1e-5, atol=1e-6)
    # warm start: network outputs mapped to (rho, u) and set as equilibrium
    net = MLP(7, 64, 3, 3, max_batch=256)
    theta = I.mlp_init(1, 7, 64, 3, 3, bias_scale=0.2)
    net.set_params(theta)
    lat.warm_start(net, fr)
    assert lat.step_count == 0
    y, _ = M.forward(theta, M.layer_sizes(7, 64, 3, 3), x, bf16=True)
    rho_w, u_w = lat.moments()
    np.testing.assert_allclose(rho_w, 1 + 2e-3 * y[:, 0], atol=2e-3 * 2e-3 * np.abs(y[:, 0]).max())
    u_ref = 0.02 * (y[:, 1:2] * np.hstack([er, np.zeros((lat.n, 1))]) + y[:, 2:3] * np.array([0, 0, 1.0]))
    assert _rel(u_w, u_ref) < 2e-3
    lat.step(10)
    lat.sync()


def test_warm_start_rejects_mismatched_network():
    from paper_2108_08783_gb300 import MLP, Lattice, LbmError
    geo = I.tube(4, 8)
    lat = Lattice(geo.labels, geo.iolets, storage="f32", tau=0.8)
    net = MLP(6, 16, 2, 3, max_batch=16)
    with pytest.raises(LbmError):
        lat.warm_start(net, _frame(geo))
