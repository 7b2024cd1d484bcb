"""Learned warm start for the solve: a small 3D U-Net (encoder/decoder with
16/32/64 channels, 3x3x3 convolutions, ~355k parameters) that predicts
ln J of the converged solution from (log10 chi, log10 eps, B, ln J_start),
as a correction to ln J_start. Not in the paper. Its prediction only moves
the starting point of rt3d_solve, whose convergence is still certified by the
FP64 residual.

All arithmetic runs in the library's kernels (csrc/nn.cu: BF16 tensor-core
convolutions with FP32 accumulation, pooling, upsampling, loss, Adam); this
module holds the parameters and activations (torch tensors are used as device
memory only) and calls the kernels in order.

Layout: activations [S][V][C] BF16, V = nx*ny*nz (x fastest), C padded to a
multiple of 16; conv weights Wt[d][Ci][Co] with d = (dz+1)*9 + (dy+1)*3 + (dx+1).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import rt3d

_vp, _ci, _cf, _cll = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong

# name, Ci (padded), Co, ReLU, real input channels (for the initial scale)
LAYERS = [
    ("e1a", 16, 16, True, 4), ("e1b", 16, 16, True, 16),
    ("e2a", 16, 32, True, 16), ("e2b", 32, 32, True, 32),
    ("b_a", 32, 64, True, 32), ("b_b", 64, 64, True, 64),
    ("d2a", 96, 32, True, 96), ("d2b", 32, 32, True, 32),
    ("d1a", 48, 16, True, 48), ("d1b", 16, 16, True, 16),
    ("out", 16, 16, False, 16),
]


def _lib():
    lib = rt3d.load()
    if not getattr(lib, "_nn_ready", False):
        lib.rt3d_nn_conv3d.argtypes = [_vp, _vp, _vp, _vp, _vp, _ci, _ci, _ci, _ci, _ci, _ci, _ci,
                                       _ci, _vp]
        lib.rt3d_nn_conv3d_wgrad.argtypes = [_vp, _vp, _vp, _vp, _ci, _ci, _ci, _ci, _ci, _ci, _vp]
        lib.rt3d_nn_relu_bwd.argtypes = [_vp, _vp, _vp, _cll, _vp]
        lib.rt3d_nn_pool.argtypes = [_vp, _vp, _ci, _ci, _ci, _ci, _ci, _vp]
        lib.rt3d_nn_pool_bwd.argtypes = [_vp, _vp, _ci, _ci, _ci, _ci, _ci, _vp]
        lib.rt3d_nn_upsample.argtypes = [_vp, _vp, _ci, _ci, _ci, _ci, _ci, _ci, _ci, _vp]
        lib.rt3d_nn_upsample_bwd.argtypes = [_vp, _vp, _ci, _ci, _ci, _ci, _ci, _ci, _ci, _vp]
        lib.rt3d_nn_channel_copy.argtypes = [_vp, _ci, _ci, _vp, _ci, _ci, _ci, _cll, _vp]
        lib.rt3d_nn_f32_to_bf16.argtypes = [_vp, _vp, _cll, _vp]
        lib.rt3d_nn_add_bf16_f32.argtypes = [_vp, _vp, _vp, _cll, _vp]
        lib.rt3d_nn_features.argtypes = [_vp, _vp, _vp, _vp, _vp, _cll, _vp]
        lib.rt3d_nn_mse.argtypes = [_vp, _vp, _vp, _vp, _vp, _cll, _cf, _vp]
        lib.rt3d_nn_apply.argtypes = [_vp, _vp, _vp, _cll, _vp]
        lib.rt3d_nn_adam.argtypes = [_vp, _vp, _vp, _vp, _ci, _cf, _cf, _cf, _cf, _ci, _vp, _vp,
                                     _ci, _ci, _vp]
        lib._nn_ready = True
    return lib


def _p(t):
    return None if t is None else t.data_ptr()


def _ck(status):
    if status != 0:
        raise rt3d.RT3DError(status, rt3d.last_error())


def half(shape):
    return tuple((n + 1) // 2 for n in shape)


class UNet:
    """Parameters, optimiser state and the kernel sequence of the network."""

    def __init__(self, seed: int = 0, device="cuda"):
        self.dev = torch.device(device)
        g = torch.Generator().manual_seed(seed)
        self.W32, self.b32, self.Wt, self.WT = {}, {}, {}, {}
        self.mW, self.vW, self.mb, self.vb = {}, {}, {}, {}
        for name, ci, co, relu, real_ci in LAYERS:
            std = (2.0 / (27 * real_ci)) ** 0.5 if relu else (1.0 / (27 * real_ci)) ** 0.5
            if name == "out":
                std *= 0.1  # start close to "no correction"
            w = torch.randn(27, ci, co, generator=g) * std
            w[:, real_ci:, :] = 0.0
            if name == "out":
                w[:, :, 1:] = 0.0
            self.W32[name] = w.to(self.dev).contiguous()
            self.b32[name] = torch.zeros(co, device=self.dev)
            self.Wt[name] = self.W32[name].to(torch.bfloat16).contiguous()
            self.WT[name] = self.W32[name].transpose(1, 2).contiguous().to(torch.bfloat16)
            for d in (self.mW, self.vW):
                d[name] = torch.zeros_like(self.W32[name])
            for d in (self.mb, self.vb):
                d[name] = torch.zeros(co, device=self.dev)
        self.step = 0

    def n_params(self):
        return sum(int(w.numel()) for w in self.W32.values()) + sum(int(b.numel()) for b in self.b32.values())

    # ------------------------------------------------------------ layers
    def _conv(self, X, name, S, shape, relu, out_f32=False):
        lib = _lib()
        ci, co = self.W32[name].shape[1], self.W32[name].shape[2]
        nz, ny, nx = shape
        V = nx * ny * nz
        Y = torch.empty(S, V, co, dtype=torch.bfloat16, device=self.dev)
        Yf = torch.empty(S, V, co, dtype=torch.float32, device=self.dev) if out_f32 else None
        _ck(lib.rt3d_nn_conv3d(_p(X), _p(self.Wt[name]), _p(self.b32[name]), _p(Y), _p(Yf), S, nx,
                               ny, nz, ci, co, int(relu), 0, None))
        return Y, Yf

    def _conv_T(self, dY, name, S, shape):
        lib = _lib()
        ci, co = self.W32[name].shape[1], self.W32[name].shape[2]
        nz, ny, nx = shape
        dX = torch.empty(S, nx * ny * nz, ci, dtype=torch.bfloat16, device=self.dev)
        _ck(lib.rt3d_nn_conv3d(_p(dY), _p(self.WT[name]), None, _p(dX), None, S, nx, ny, nz, co, ci,
                               0, 1, None))
        return dX

    def _wgrad(self, X, dY, name, S, shape):
        # the layer's input activation and output gradient of the last
        # backward pass, kept (as references) for inspection
        self.wgrad_inputs[name] = (X, dY, shape)
        lib = _lib()
        ci, co = self.W32[name].shape[1], self.W32[name].shape[2]
        nz, ny, nx = shape
        _ck(lib.rt3d_nn_conv3d_wgrad(_p(X), _p(dY), _p(self.gW[name]), _p(self.gb[name]), S, nx,
                                     ny, nz, ci, co, None))

    def _relu_bwd(self, dY, Y):
        out = torch.empty_like(dY)
        _ck(_lib().rt3d_nn_relu_bwd(_p(dY), _p(Y), _p(out), dY.numel(), None))
        return out

    def _pool(self, X, S, shape, C):
        nz, ny, nx = shape
        hz, hy, hx = half(shape)
        P = torch.empty(S, hx * hy * hz, C, dtype=torch.bfloat16, device=self.dev)
        _ck(_lib().rt3d_nn_pool(_p(X), _p(P), S, nx, ny, nz, C, None))
        return P

    def _pool_bwd(self, dP, S, shape, C):
        nz, ny, nx = shape
        dX = torch.zeros(S, nx * ny * nz, C, dtype=torch.float32, device=self.dev)
        _ck(_lib().rt3d_nn_pool_bwd(_p(dP), _p(dX), S, nx, ny, nz, C, None))
        return dX

    def _up_concat(self, Xs, skip, S, shape, C, Cs):
        nz, ny, nx = shape
        V = nx * ny * nz
        U = torch.empty(S, V, C + Cs, dtype=torch.bfloat16, device=self.dev)
        _ck(_lib().rt3d_nn_upsample(_p(Xs), _p(U), S, nx, ny, nz, C, C + Cs, 0, None))
        _ck(_lib().rt3d_nn_channel_copy(_p(skip), Cs, 0, _p(U), C + Cs, C, Cs, S * V, None))
        return U

    def _split_concat(self, dU, S, shape, C, Cs):
        """(gradient of the upsampled input (small grid, BF16), of the skip (BF16))."""
        nz, ny, nx = shape
        V = nx * ny * nz
        hz, hy, hx = half(shape)
        d_small = torch.zeros(S, hx * hy * hz, C, dtype=torch.float32, device=self.dev)
        _ck(_lib().rt3d_nn_upsample_bwd(_p(dU), _p(d_small), S, nx, ny, nz, C, C + Cs, 0, None))
        d_skip = torch.empty(S, V, Cs, dtype=torch.bfloat16, device=self.dev)
        _ck(_lib().rt3d_nn_channel_copy(_p(dU), C + Cs, C, _p(d_skip), Cs, 0, Cs, S * V, None))
        return self._to_bf16(d_small), d_skip

    def _to_bf16(self, x32):
        out = torch.empty(x32.shape, dtype=torch.bfloat16, device=self.dev)
        _ck(_lib().rt3d_nn_f32_to_bf16(_p(x32), _p(out), x32.numel(), None))
        return out

    def _add(self, a_bf16, b_f32):
        out = torch.empty_like(a_bf16)
        _ck(_lib().rt3d_nn_add_bf16_f32(_p(a_bf16), _p(b_f32), _p(out), a_bf16.numel(), None))
        return out

    # ----------------------------------------------------------- network
    def features(self, chi, eps, B, J0):
        """[S][V][16] BF16 input from FP64 (S, nz, ny, nx) device tensors."""
        S = chi.shape[0]
        V = chi[0].numel()
        X = torch.empty(S, V, 16, dtype=torch.bfloat16, device=self.dev)
        _ck(_lib().rt3d_nn_features(_p(chi), _p(eps), _p(B), _p(J0), _p(X), S * V, None))
        return X

    def forward(self, X, shape):
        S = X.shape[0]
        s1s, s2s, s3s = shape, half(shape), half(half(shape))
        c = {}
        c["X"] = X
        c["a1"], _ = self._conv(X, "e1a", S, s1s, True)
        c["s1"], _ = self._conv(c["a1"], "e1b", S, s1s, True)
        c["p1"] = self._pool(c["s1"], S, s1s, 16)
        c["a2"], _ = self._conv(c["p1"], "e2a", S, s2s, True)
        c["s2"], _ = self._conv(c["a2"], "e2b", S, s2s, True)
        c["p2"] = self._pool(c["s2"], S, s2s, 32)
        c["a3"], _ = self._conv(c["p2"], "b_a", S, s3s, True)
        c["b"], _ = self._conv(c["a3"], "b_b", S, s3s, True)
        c["c2"] = self._up_concat(c["b"], c["s2"], S, s2s, 64, 32)
        c["a4"], _ = self._conv(c["c2"], "d2a", S, s2s, True)
        c["u2"], _ = self._conv(c["a4"], "d2b", S, s2s, True)
        c["c1"] = self._up_concat(c["u2"], c["s1"], S, s1s, 32, 16)
        c["a5"], _ = self._conv(c["c1"], "d1a", S, s1s, True)
        c["u1"], _ = self._conv(c["a5"], "d1b", S, s1s, True)
        _, c["y"] = self._conv(c["u1"], "out", S, s1s, False, out_f32=True)
        self.cache = (c, shape)
        return c["y"]

    def backward(self, dY):
        """Accumulates the parameter gradients of the last forward pass for the
        output gradient dY ([S][V][16] BF16, channel 0)."""
        c, shape = self.cache
        S = dY.shape[0]
        s1s, s2s, s3s = shape, half(shape), half(half(shape))
        self.gW = {n: torch.zeros_like(w) for n, w in self.W32.items()}
        self.wgrad_inputs = {}
        self.gb = {n: torch.zeros_like(b) for n, b in self.b32.items()}
        self._wgrad(c["u1"], dY, "out", S, s1s)
        d = self._conv_T(dY, "out", S, s1s)
        d = self._relu_bwd(d, c["u1"])
        self._wgrad(c["a5"], d, "d1b", S, s1s)
        d = self._conv_T(d, "d1b", S, s1s)
        d = self._relu_bwd(d, c["a5"])
        self._wgrad(c["c1"], d, "d1a", S, s1s)
        d = self._conv_T(d, "d1a", S, s1s)
        d_u2, d_s1_skip = self._split_concat(d, S, s1s, 32, 16)
        d = self._relu_bwd(d_u2, c["u2"])
        self._wgrad(c["a4"], d, "d2b", S, s2s)
        d = self._conv_T(d, "d2b", S, s2s)
        d = self._relu_bwd(d, c["a4"])
        self._wgrad(c["c2"], d, "d2a", S, s2s)
        d = self._conv_T(d, "d2a", S, s2s)
        d_b, d_s2_skip = self._split_concat(d, S, s2s, 64, 32)
        d = self._relu_bwd(d_b, c["b"])
        self._wgrad(c["a3"], d, "b_b", S, s3s)
        d = self._conv_T(d, "b_b", S, s3s)
        d = self._relu_bwd(d, c["a3"])
        self._wgrad(c["p2"], d, "b_a", S, s3s)
        d = self._conv_T(d, "b_a", S, s3s)
        d_s2 = self._add(d_s2_skip, self._pool_bwd(d, S, s2s, 32))
        d = self._relu_bwd(d_s2, c["s2"])
        self._wgrad(c["a2"], d, "e2b", S, s2s)
        d = self._conv_T(d, "e2b", S, s2s)
        d = self._relu_bwd(d, c["a2"])
        self._wgrad(c["p1"], d, "e2a", S, s2s)
        d = self._conv_T(d, "e2a", S, s2s)
        d_s1 = self._add(d_s1_skip, self._pool_bwd(d, S, s1s, 16))
        d = self._relu_bwd(d_s1, c["s1"])
        self._wgrad(c["a1"], d, "e1b", S, s1s)
        d = self._conv_T(d, "e1b", S, s1s)
        d = self._relu_bwd(d, c["a1"])
        self._wgrad(c["X"], d, "e1a", S, s1s)
        return self.gW, self.gb

    def loss_grad(self, Yf, target, J0):
        """MSE of the predicted ln J (= ln J0 + y) against ln(target); returns
        (loss, dY)."""
        rows = Yf.shape[0] * Yf.shape[1]
        dY = torch.empty(Yf.shape, dtype=torch.bfloat16, device=self.dev)
        sse = torch.zeros(1, dtype=torch.float32, device=self.dev)
        _ck(_lib().rt3d_nn_mse(_p(Yf), _p(target), _p(J0), _p(dY), _p(sse), rows,
                               1.0 / rows, None))
        return sse, dY

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        lib = _lib()
        self.step += 1
        for name, ci, co, relu, real in LAYERS:
            _ck(lib.rt3d_nn_adam(_p(self.W32[name]), _p(self.gW[name]), _p(self.mW[name]),
                                 _p(self.vW[name]), self.W32[name].numel(), lr, b1, b2, eps,
                                 self.step, _p(self.Wt[name]), _p(self.WT[name]), ci, co, None))
            _ck(lib.rt3d_nn_adam(_p(self.b32[name]), _p(self.gb[name]), _p(self.mb[name]),
                                 _p(self.vb[name]), co, lr, b1, b2, eps, self.step, None, None,
                                 1, co, None))

    def predict(self, chi, eps, B, J0):
        """J = exp(ln J0 + network correction) as FP64 (S, nz, ny, nx)."""
        shape = tuple(chi.shape[1:])
        X = self.features(chi, eps, B, J0)
        Yf = self.forward(X, shape)
        J = torch.empty_like(J0)
        _ck(_lib().rt3d_nn_apply(_p(Yf), _p(J0), _p(J), J0.numel(), None))
        return J


# ------------------------------------------------------------------ data
def solve_fields(grid, shape, seeds, eps_of_seed, scale_of_seed=None, tol=1e-9, max_iter=4000):
    """Converged solutions that the method itself produces: for every seed, a
    synthetic atmosphere (inputs.cartesian_config with that seed) solved by
    rt3d_solve from J = B. Returns a list of (chi, eps, B, J, I_bottom) device
    tensors shaped (1, nz, ny, nx) (faces (1, ny, nx))."""
    from . import inputs

    nz, ny, nx = shape
    out = []
    for seed in seeds:
        chi, eps, B, bc = inputs.cartesian_config((nx, ny, nz), eps_of_seed(seed), seed=seed)
        if scale_of_seed is not None:
            chi = chi * scale_of_seed(seed)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
        tchi, teps, tB, tbot = d(chi), d(eps), d(B), d(bc["I_bottom"])
        J = tB.clone()
        grid.solve(tchi, teps, tB, {"I_top": 0.0, "I_bottom": tbot}, J, tol=tol,
                   max_iter=max_iter)
        out.append((tchi[None], teps[None], tB[None], J[None], tbot[None]))
    return out


def train(net, data, steps, lr=2e-3, lr_final=2e-4, log_every=0):
    """Adam on the mean squared error of ln J over the samples, one sample per
    step (cycled). Returns the loss history."""
    hist = []
    shape = tuple(data[0][0].shape[1:])
    for step in range(steps):
        chi, eps, B, J, _ = data[step % len(data)]
        X = net.features(chi, eps, B, B)
        Yf = net.forward(X, shape)
        sse, dY = net.loss_grad(Yf, J, B)
        net.backward(dY)
        frac = step / max(1, steps - 1)
        net.adam(lr=lr * (lr_final / lr) ** frac)
        if log_every and (step % log_every == 0 or step == steps - 1):
            hist.append((step, float(sse.item()) / J.numel()))
    return hist
