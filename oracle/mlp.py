"""FP64 CPU oracle of the learned warm start's network (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU legs may import this
module; the library never does.  The paper has no learned component: this is
the warm-start network the GPU path trains with its own kernels, written here
as its plain definition so that the GPU forward pass, loss, gradients and
optimiser step can be compared with it.

Network (L linear layers, widths n_in -> W -> ... -> W -> n_out):

    z_l = h_l W_l^T + b_l,   h_0 = x,
    h_{l+1} = tanh(z_l)      for l < L - 1,
    y = z_{L-1}.

Loss: mean squared error over the n x n_out outputs,
    E = sum (y - t)^2 / (n n_out).
Gradients by the chain rule (back-propagation):
    d_{L-1} = dE/dy = 2 (y - t) / (n n_out),
    dE/dW_l = d_l^T h_l,  dE/db_l = sum over rows of d_l,
    d_{l-1} = (d_l W_l) * (1 - h_l^2).
Optimiser: Adam (Kingma & Ba, 2015, Algorithm 1) with bias-corrected moments.

``bf16=True`` rounds (round to nearest, ties to even) to bfloat16 exactly the
quantities the mixed-precision GPU path stores in bfloat16: the inputs x, the
weights W_l, the hidden activations h_l (l >= 1), the output error d_{L-1} and
the back-propagated errors d_l; every product and sum is still FP64 (the GPU
accumulates in FP32).

Parameter vector layout (shared with the C ABI): W_0 (row-major
[n_out_0][n_in_0]), b_0, W_1, b_1, ..., FP32 on the GPU, FP64 here.

Pins (tests/test_oracle_mlp.py): gradients against central finite differences
of the loss, the one-layer network's gradient-descent fixed point against a
least-squares solve, bfloat16 rounding against torch's conversion, and the
optimiser step against torch.optim.Adam.
"""
import numpy as np


def layer_sizes(n_in, width, n_layers, n_out):
    """[(rows, cols)] of W_0 .. W_{L-1}."""
    dims = [n_in] + [width] * (n_layers - 1) + [n_out]
    return [(dims[l + 1], dims[l]) for l in range(n_layers)]


def param_count(n_in, width, n_layers, n_out):
    return sum(r * c + r for r, c in layer_sizes(n_in, width, n_layers, n_out))


def unflatten(theta, sizes):
    """Views [(W_l, b_l)] of a flat parameter vector."""
    out, o = [], 0
    for r, c in sizes:
        W = theta[o:o + r * c].reshape(r, c)
        o += r * c
        b = theta[o:o + r]
        o += r
        out.append((W, b))
    assert o == theta.size
    return out


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    A bfloat16 is the upper 16 bits of an IEEE binary32; the value is first
    rounded to binary32 (exact for every value the tests use), then the low 16
    bits are rounded away: add 0x7FFF plus the lowest kept bit and truncate.
    """
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    keep = (u >> 16) & 1
    r = ((u + 0x7FFF + keep) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64).reshape(f.shape)


def _q(a, bf16):
    return bf16_round(a) if bf16 else np.asarray(a, np.float64)


def forward(theta, sizes, x, bf16=False):
    """Outputs y [n][n_out] and the layer inputs h_0 .. h_{L-1}."""
    layers = unflatten(np.asarray(theta, np.float64), sizes)
    h = _q(x, bf16)
    hs = []
    for l, (W, b) in enumerate(layers):
        hs.append(h)
        z = h @ _q(W, bf16).T + b
        if l < len(layers) - 1:
            h = _q(np.tanh(z), bf16)
        else:
            return z, hs


def loss_grad(theta, sizes, x, t, bf16=False):
    """(E, dE/dtheta) for inputs x [n][n_in] and targets t [n][n_out]."""
    theta = np.asarray(theta, np.float64)
    layers = unflatten(theta, sizes)
    y, hs = forward(theta, sizes, x, bf16)
    t = np.asarray(t, np.float64)
    n, m = y.shape
    E = float(np.sum((y - t) ** 2) / (n * m))
    d = _q(2.0 * (y - t) / (n * m), bf16)
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gW = d.T @ hs[l]
        gb = d.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            d = _q((d @ _q(W, bf16)) * (1.0 - hs[l] ** 2), bf16)
    grads.reverse()
    return E, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t >= 1 counts steps); returns (theta, m, v), new arrays."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
