"""Seeded inputs of the warm-start network: initial parameters and batches.

Only random numbers: the layer layout (W_0, b_0, W_1, b_1, ... with W_l of
shape [rows_l][cols_l]) is the parameter-vector interface of the network.
"""
import numpy as np


def mlp_shapes(n_in, width, n_layers, n_out):
    dims = [n_in] + [width] * (n_layers - 1) + [n_out]
    return [(dims[l + 1], dims[l]) for l in range(n_layers)]


def mlp_init(seed, n_in, width, n_layers, n_out, bias_scale=0.0):
    """FP32 parameter vector: W_l uniform in +-sqrt(6/(rows + cols)) (Glorot),
    b_l uniform in +-bias_scale."""
    rng = np.random.default_rng(seed)
    parts = []
    for r, c in mlp_shapes(n_in, width, n_layers, n_out):
        a = np.sqrt(6.0 / (r + c))
        parts.append(rng.uniform(-a, a, r * c))
        parts.append(rng.uniform(-bias_scale, bias_scale, r) if bias_scale else np.zeros(r))
    return np.concatenate(parts).astype(np.float32)


def mlp_batch(seed, n, n_in, n_out, scale=1.0):
    """FP32 inputs x [n][n_in] uniform in [-1, 1] and targets t [n][n_out]
    uniform in +-scale."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1.0, 1.0, (n, n_in)).astype(np.float32)
    t = rng.uniform(-scale, scale, (n, n_out)).astype(np.float32)
    return x, t
