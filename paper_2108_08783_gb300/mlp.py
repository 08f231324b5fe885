"""Python binding of the warm-start network (``include/lbm_mlp.h``).

Argument marshalling only: the forward pass, loss, back-propagation and Adam
step run in the library's kernels.  Device arrays are torch CUDA tensors.
"""
import ctypes as C

import numpy as np

from . import _capi as A
from .lattice import _TorchAllocator, _ptr


class MLP:
    """Multilayer perceptron n_in -> width x (n_layers - 1) -> n_out with tanh
    between layers; bfloat16 operands, FP32 accumulation, FP32 Adam master
    parameters (``lbm_mlp_create``)."""

    def __init__(self, n_in, width=256, n_layers=4, n_out=3, max_batch=16384, device=0,
                 stream=None):
        import torch
        self._lib = A.lib()
        self.torch = torch
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.n_in, self.width, self.n_layers, self.n_out = n_in, width, n_layers, n_out
        self.max_batch = int(max_batch)
        self._alloc = _TorchAllocator(self.device, stream)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.lbm_mlp_create(n_in, width, n_layers, n_out, self.max_batch,
                                          C.byref(self._alloc.struct),
                                          C.c_void_p(stream.cuda_stream), C.byref(h))
        if rc != A.LBM_OK:
            raise A.LbmError(rc, "lbm_mlp_create(%d, %d, %d, %d, %d)"
                             % (n_in, width, n_layers, n_out, self.max_batch))
        self.h = h
        cnt = C.c_int64()
        self._check(self._lib.lbm_mlp_param_count(self.h, C.byref(cnt)))
        self.n_params = int(cnt.value)

    def close(self):
        h = getattr(self, "h", None)
        if h is not None:
            self._lib.lbm_mlp_destroy(h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != A.LBM_OK:
            raise A.LbmError(rc, self._lib.lbm_mlp_last_error(self.h).decode())
        return rc

    def _dev(self, a, cols):
        t = self.torch.as_tensor(a, dtype=self.torch.float32, device=self.device).contiguous()
        assert t.dim() == 2 and t.shape[1] == cols, t.shape
        return t

    def set_params(self, theta):
        theta = np.ascontiguousarray(np.asarray(theta, np.float32).ravel())
        assert theta.size == self.n_params
        self._check(self._lib.lbm_mlp_set_params(self.h, _ptr(theta), 0))

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        self._check(self._lib.lbm_mlp_get_params(self.h, _ptr(out), 0))
        return out

    def forward(self, x):
        x = self._dev(x, self.n_in)
        y = self.torch.empty((x.shape[0], self.n_out), dtype=self.torch.float32,
                             device=self.device)
        self._check(self._lib.lbm_mlp_forward(self.h, C.c_void_p(x.data_ptr()), x.shape[0],
                                              C.c_void_p(y.data_ptr())))
        return y

    def loss_grad(self, x, t):
        x, t = self._dev(x, self.n_in), self._dev(t, self.n_out)
        loss = C.c_double()
        g = np.zeros(self.n_params, np.float32)
        self._check(self._lib.lbm_mlp_loss_grad(self.h, C.c_void_p(x.data_ptr()),
                                                C.c_void_p(t.data_ptr()), x.shape[0],
                                                C.byref(loss), _ptr(g), 0))
        return float(loss.value), g

    def train_step(self, x, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=False):
        """One Adam step on the batch; returns its loss (before the update) when
        ``want_loss``, else None without waiting."""
        x, t = self._dev(x, self.n_in), self._dev(t, self.n_out)
        opt = A.LbmAdam(lr, beta1, beta2, eps)
        loss = C.c_double()
        self._check(self._lib.lbm_mlp_train_step(self.h, C.c_void_p(x.data_ptr()),
                                                 C.c_void_p(t.data_ptr()), x.shape[0],
                                                 C.byref(opt),
                                                 C.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def sync(self):
        self._check(self._lib.lbm_mlp_sync(self.h))


def warm_frame(centre, axis, z0, length, radius, features, rho_scale, u_scale):
    """lbm_warm_frame of a straight tube (see ``include/lbm_mlp.h``)."""
    f = A.LbmWarmFrame()
    for k in range(3):
        f.centre[k] = float(centre[k])
        f.axis[k] = float(axis[k])
    f.z0, f.length, f.radius = float(z0), float(length), float(radius)
    f.rho_scale, f.u_scale = float(rho_scale), float(u_scale)
    feats = list(features)
    assert len(feats) <= A.LBM_WARM_MAX_GLOBAL
    f.n_global = len(feats)
    for k, v in enumerate(feats):
        f.global_[k] = float(v)
    return f


def _throughput(rows=65536, train_rows=16384, reps=20):
    """CUDA-event timing of the warm-start network's forward pass and
    training step (seeded Glorot weights, uniform random inputs)."""
    import torch
    import lbm_inputs as I
    net = MLP(7, 256, 4, 3, max_batch=rows)
    net.set_params(I.mlp_init(0, 7, 256, 4, 3))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(rows, 7, device="cuda", generator=g)
    t = torch.rand(rows, 3, device="cuda", generator=g)
    for _ in range(3):
        net.forward(x)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(net.stream)
    for _ in range(reps):
        net.forward(x)
    e1.record(net.stream)
    e1.synchronize()
    fwd = e0.elapsed_time(e1) / reps
    flop = 2 * (7 * 256 + 2 * 256 * 256 + 256 * 3)
    e0.record(net.stream)
    for _ in range(reps):
        net.train_step(x[:train_rows], t[:train_rows], lr=1e-4)
    e1.record(net.stream)
    e1.synchronize()
    trn = e0.elapsed_time(e1) / reps
    net.sync()
    return {"forward_rows": rows, "forward_ms": fwd, "forward_tflops": rows * flop / fwd / 1e9,
            "train_rows": train_rows, "train_step_ms": trn,
            "train_tflops": 3 * train_rows * flop / trn / 1e9}


if __name__ == "__main__":
    import json
    import sys
    print(json.dumps(_throughput(int(sys.argv[1]) if len(sys.argv) > 1 else 65536)))
