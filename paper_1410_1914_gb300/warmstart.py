"""Learned warm start for the D3Q7 solve: a 4-level 3D U-Net (16/32/64/128
channels) that predicts the converged field from the structure.

Every operation of the forward pass, the backward pass and the Adam update
runs in the library's own kernels (``cl_nn_*`` entry points, BF16 tensor-core
convolutions with FP32 accumulation); this module only sequences them and
owns the device buffers (torch tensors, used as memory).

Input (16 channels per voxel, from ``cl_lbm_features``): active, solid,
ionomer, micropore, scaled log relative diffusivity, the linear ramp
between the two face concentrations, the series-resistor profile of the
planes along x and its deviation from the ramp (the part of the mean
profile that no bounded receptive field sees).
Output: the correction to the linear ramp, in units of (C_in - C_out)/nx, so
that the same local structure gives the same target at any box length; the
warm start is ramp + output / nx on active cells.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import _lib as L

CONV_LAYERS = [
    ("e1a", 16, 16), ("e1b", 16, 16),
    ("e2a", 16, 32), ("e2b", 32, 32),
    ("e3a", 32, 64), ("e3b", 64, 64),
    ("bta", 64, 128), ("btb", 128, 128),
    ("d3a", 192, 64), ("d3b", 64, 64),
    ("d2a", 96, 32), ("d2b", 32, 32),
    ("d1a", 48, 16), ("d1b", 16, 16),
]
FEATURES = 16

_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
_F = ctypes.c_float
_S = ctypes.c_int
_SIGS = {
    "cl_nn_conv3d": (_S, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _I, _I, _I, _I, _I, _P]),
    "cl_nn_wgrad_workspace": (_LL, [_I, _I, _I, _I, _I, _I]),
    "cl_nn_conv3d_wgrad": (_S, [_P, _P, _P, _P, _I, _I, _I, _I, _I, _I, _I, _I, _I, _I, _I, _P]),
    "cl_nn_wt_dgrad": (_S, [_P, _P, _I, _I, _P]),
    "cl_nn_bias_grad": (_S, [_P, _LL, _I, _I, _I, _P, _P]),
    "cl_nn_relu_bwd": (_S, [_P, _P, _LL, _I, _I, _I, _P]),
    "cl_nn_pool": (_S, [_P, _P, _I, _I, _I, _I, _I, _I, _I, _P]),
    "cl_nn_pool_bwd": (_S, [_P, _P, _I, _I, _I, _I, _I, _I, _I, _I, _P]),
    "cl_nn_upsample": (_S, [_P, _P, _I, _I, _I, _I, _I, _I, _I, _P]),
    "cl_nn_upsample_bwd": (_S, [_P, _P, _I, _I, _I, _I, _I, _I, _I, _P]),
    "cl_nn_copy_channels": (_S, [_P, _I, _I, _P, _I, _I, _LL, _I, _I, _P]),
    "cl_nn_head": (_S, [_P, _P, _P, _P, _LL, _I, _P]),
    "cl_nn_mse": (_S, [_P, _P, _P, _LL, _P, _P, _P]),
    "cl_nn_head_bwd": (_S, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _LL, _I, _P]),
    "cl_nn_adam": (_S, [_P, _P, _P, _P, _P, _LL, _F, _F, _F, _F, _I, _P]),
    "cl_nn_to_bf16": (_S, [_P, _P, _LL, _P]),
    "cl_nn_check": (_S, [_P]),
    "cl_lbm_features": (_S, [_P, _P]),
    "cl_lbm_target": (_S, [_P, _P]),
    "cl_lbm_init_warm": (_S, [_P, _P]),
}
_ready = False


def _lib():
    global _ready
    lib = L.load()
    if not _ready:
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _ready = True
    return lib


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _call(name, *args):
    s = getattr(_lib(), name)(*args)
    if s != L.CL_OK:
        raise L.ClError(s, name, L.last_error_message())


class UNet:
    """Parameters, Adam state and activation buffers for batch N of cubes D^3."""

    def __init__(self, seed: int = 0, device: str = "cuda"):
        import torch
        self.torch = torch
        self.dev = device
        g = torch.Generator().manual_seed(seed)
        self.params = {}
        for name, ci, co in CONV_LAYERS:
            w = torch.randn(27, co, ci, generator=g) * math.sqrt(2.0 / (27 * ci))
            self.params[name] = [w.to(device).contiguous(), torch.zeros(co, device=device)]
        self.params["head"] = [(torch.randn(16, generator=g) * 1e-2).to(device), torch.zeros(1, device=device)]
        self.wbf = {n: self.params[n][0].to(torch.bfloat16).contiguous() for n, _, _ in CONV_LAYERS}
        self.adam = {n: [[torch.zeros_like(t), torch.zeros_like(t)] for t in self.params[n]] for n in self.params}
        self.grads = {n: [torch.zeros_like(t) for t in self.params[n]] for n in self.params}
        self.t = 0
        self.shape = None

    # ------------------------------------------------------------ buffers
    _BUF_KEYS = ("a", "g", "out", "gy", "loss", "loss_ws", "wsp", "wd")

    def _alloc(self, N, D):
        """Activation, gradient and workspace buffers for batch N of D^3 cubes,
        kept per shape so that alternating shapes does not reallocate."""
        torch = self.torch
        if self.shape == (N, D):
            return
        if not hasattr(self, "_bufs"):
            self._bufs = {}
        if self.shape is not None:
            self._bufs[self.shape] = {k: getattr(self, k) for k in self._BUF_KEYS}
        self.shape = (N, D)
        if (N, D) in self._bufs:
            for k, v in self._bufs[(N, D)].items():
                setattr(self, k, v)
            return
        bf = dict(dtype=torch.bfloat16, device=self.dev)
        sizes = {1: D, 2: D // 2, 3: D // 4, 4: D // 8}
        chans = {"e1a": (1, 16), "cat1": (1, 48), "d1a": (1, 16), "d1": (1, 16),
                 "p1": (2, 16), "e2a": (2, 32), "cat2": (2, 96), "d2a": (2, 32), "d2": (2, 32),
                 "p2": (3, 32), "e3a": (3, 64), "cat3": (3, 192), "d3a": (3, 64), "d3": (3, 64),
                 "p3": (4, 64), "bta": (4, 128), "bt": (4, 128)}
        self.a = {k: torch.empty(N, sizes[l], sizes[l], sizes[l], c, **bf) for k, (l, c) in chans.items()}
        self.g = {k: torch.zeros_like(v) for k, v in self.a.items()}
        self.out = torch.empty(N * D ** 3, dtype=torch.float32, device=self.dev)
        self.gy = torch.empty_like(self.out)
        self.loss = torch.zeros(2, dtype=torch.float64, device=self.dev)
        self.loss_ws = torch.zeros(512, dtype=torch.float64, device=self.dev)
        ws = max(_lib().cl_nn_wgrad_workspace(N, sizes[l], sizes[l], sizes[l], ci, co)
                 for (name, ci, co), l in zip(CONV_LAYERS, [1, 1, 2, 2, 3, 3, 4, 4, 3, 3, 2, 2, 1, 1]))
        self.wsp = torch.empty(ws // 4 + 1, dtype=torch.float32, device=self.dev)
        self.wd = torch.empty(27 * 192 * 128, dtype=torch.bfloat16, device=self.dev)

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _conv(self, name, x, xs, xo, y, ys, yo, N, D, relu=True):
        _, ci, co = next(l for l in CONV_LAYERS if l[0] == name)
        _call("cl_nn_conv3d", _p(x), _p(self.wbf[name]), _p(self.params[name][1]), _p(y), N, D, D, D, ci, co, xs, xo,
              ys, yo, int(relu), 1, self._stream())

    # ------------------------------------------------------------ forward
    def forward(self, x, N, D):
        """x: bf16 [N, D, D, D, 16] features; returns fp32 prediction [N*D^3]."""
        self._alloc(N, D)
        a, s = self.a, self._stream()
        d1, d2, d3, d4 = D, D // 2, D // 4, D // 8
        self._conv("e1a", x, 16, 0, a["e1a"], 16, 0, N, d1)
        self._conv("e1b", a["e1a"], 16, 0, a["cat1"], 48, 32, N, d1)          # e1 -> cat1[32:48]
        _call("cl_nn_pool", _p(a["cat1"]), _p(a["p1"]), N, d1, d1, d1, 16, 48, 32, s)
        self._conv("e2a", a["p1"], 16, 0, a["e2a"], 32, 0, N, d2)
        self._conv("e2b", a["e2a"], 32, 0, a["cat2"], 96, 64, N, d2)          # e2 -> cat2[64:96]
        _call("cl_nn_pool", _p(a["cat2"]), _p(a["p2"]), N, d2, d2, d2, 32, 96, 64, s)
        self._conv("e3a", a["p2"], 32, 0, a["e3a"], 64, 0, N, d3)
        self._conv("e3b", a["e3a"], 64, 0, a["cat3"], 192, 128, N, d3)       # e3 -> cat3[128:192]
        _call("cl_nn_pool", _p(a["cat3"]), _p(a["p3"]), N, d3, d3, d3, 64, 192, 128, s)
        self._conv("bta", a["p3"], 64, 0, a["bta"], 128, 0, N, d4)
        self._conv("btb", a["bta"], 128, 0, a["bt"], 128, 0, N, d4)
        _call("cl_nn_upsample", _p(a["bt"]), _p(a["cat3"]), N, d3, d3, d3, 128, 192, 0, s)
        self._conv("d3a", a["cat3"], 192, 0, a["d3a"], 64, 0, N, d3)
        self._conv("d3b", a["d3a"], 64, 0, a["d3"], 64, 0, N, d3)
        _call("cl_nn_upsample", _p(a["d3"]), _p(a["cat2"]), N, d2, d2, d2, 64, 96, 0, s)
        self._conv("d2a", a["cat2"], 96, 0, a["d2a"], 32, 0, N, d2)
        self._conv("d2b", a["d2a"], 32, 0, a["d2"], 32, 0, N, d2)
        _call("cl_nn_upsample", _p(a["d2"]), _p(a["cat1"]), N, d1, d1, d1, 32, 48, 0, s)
        self._conv("d1a", a["cat1"], 48, 0, a["d1a"], 16, 0, N, d1)
        self._conv("d1b", a["d1a"], 16, 0, a["d1"], 16, 0, N, d1)
        hw, hb = self.params["head"]
        _call("cl_nn_head", _p(a["d1"]), _p(hw), _p(hb), _p(self.out), N * D ** 3, 16, s)
        self.x = x
        return self.out

    # ------------------------------------------------------------ backward
    def _conv_bwd(self, name, x, xs, xo, y, ys, yo, gy, gys, gyo, gx, gxs, gxo, N, D, need_gx=True):
        """y = relu(conv(x)); gy holds dL/d(pre-activation) (already masked by
        the ReLU) in channels [gyo, gyo+co) of a stride-gys buffer."""
        _, ci, co = next(l for l in CONV_LAYERS if l[0] == name)
        s = self._stream()
        M = N * D ** 3
        _call("cl_nn_conv3d_wgrad", _p(x), _p(gy), _p(self.wsp), _p(self.grads[name][0]), N, D, D, D, ci, co, xs, xo,
              gys, gyo, 1, s)
        _call("cl_nn_bias_grad", _p(gy), M, co, gys, gyo, _p(self.grads[name][1]), s)
        if need_gx:
            _call("cl_nn_wt_dgrad", _p(self.wbf[name]), _p(self.wd), co, ci, s)
            _call("cl_nn_conv3d", _p(gy), _p(self.wd), None, _p(gx), N, D, D, D, co, ci, gys, gyo, gxs, gxo, 0, 1, s)

    def backward(self, target, mask):
        """Masked MSE of the last forward against target (fp32 [N*D^3]);
        fills self.grads; returns nothing (loss in self.loss[0])."""
        N, D = self.shape
        a, g, s = self.a, self.g, self._stream()
        d1, d2, d3, d4 = D, D // 2, D // 4, D // 8
        M = N * D ** 3
        hw, hb = self.params["head"]
        _call("cl_nn_mse", _p(self.out), _p(target), _p(mask), M, _p(self.loss_ws), _p(self.loss), s)
        _call("cl_nn_head_bwd", _p(a["d1"]), _p(hw), _p(self.out), _p(target), _p(mask), _p(self.loss), _p(g["d1"]),
              _p(self.gy), _p(self.grads["head"][0]), _p(self.grads["head"][1]), M, 16, s)
        # level 1 decoder
        self._relu(a["d1"], g["d1"], M, 16, 16, 0)
        self._conv_bwd("d1b", a["d1a"], 16, 0, a["d1"], 16, 0, g["d1"], 16, 0, g["d1a"], 16, 0, N, d1)
        self._relu(a["d1a"], g["d1a"], M, 16, 16, 0)
        self._conv_bwd("d1a", a["cat1"], 48, 0, a["d1a"], 16, 0, g["d1a"], 16, 0, g["cat1"], 48, 0, N, d1)
        _call("cl_nn_upsample_bwd", _p(g["cat1"]), _p(g["d2"]), N, d1, d1, d1, 32, 48, 0, s)
        # level 2 decoder
        M2 = N * d2 ** 3
        self._relu(a["d2"], g["d2"], M2, 32, 32, 0)
        self._conv_bwd("d2b", a["d2a"], 32, 0, a["d2"], 32, 0, g["d2"], 32, 0, g["d2a"], 32, 0, N, d2)
        self._relu(a["d2a"], g["d2a"], M2, 32, 32, 0)
        self._conv_bwd("d2a", a["cat2"], 96, 0, a["d2a"], 32, 0, g["d2a"], 32, 0, g["cat2"], 96, 0, N, d2)
        _call("cl_nn_upsample_bwd", _p(g["cat2"]), _p(g["d3"]), N, d2, d2, d2, 64, 96, 0, s)
        # level 3 decoder
        M3 = N * d3 ** 3
        self._relu(a["d3"], g["d3"], M3, 64, 64, 0)
        self._conv_bwd("d3b", a["d3a"], 64, 0, a["d3"], 64, 0, g["d3"], 64, 0, g["d3a"], 64, 0, N, d3)
        self._relu(a["d3a"], g["d3a"], M3, 64, 64, 0)
        self._conv_bwd("d3a", a["cat3"], 192, 0, a["d3a"], 64, 0, g["d3a"], 64, 0, g["cat3"], 192, 0, N, d3)
        _call("cl_nn_upsample_bwd", _p(g["cat3"]), _p(g["bt"]), N, d3, d3, d3, 128, 192, 0, s)
        # bottom
        M4 = N * d4 ** 3
        self._relu(a["bt"], g["bt"], M4, 128, 128, 0)
        self._conv_bwd("btb", a["bta"], 128, 0, a["bt"], 128, 0, g["bt"], 128, 0, g["bta"], 128, 0, N, d4)
        self._relu(a["bta"], g["bta"], M4, 128, 128, 0)
        self._conv_bwd("bta", a["p3"], 64, 0, a["bta"], 128, 0, g["bta"], 128, 0, g["p3"], 64, 0, N, d4)
        # e3 = cat3[128:192] gets the skip gradient (already in g["cat3"]) plus the pooling path
        _call("cl_nn_pool_bwd", _p(g["p3"]), _p(g["cat3"]), N, d3, d3, d3, 64, 192, 128, 1, s)
        self._relu(a["cat3"], g["cat3"], M3, 64, 192, 128)
        self._conv_bwd("e3b", a["e3a"], 64, 0, a["cat3"], 192, 128, g["cat3"], 192, 128, g["e3a"], 64, 0, N, d3)
        self._relu(a["e3a"], g["e3a"], M3, 64, 64, 0)
        self._conv_bwd("e3a", a["p2"], 32, 0, a["e3a"], 64, 0, g["e3a"], 64, 0, g["p2"], 32, 0, N, d3)
        _call("cl_nn_pool_bwd", _p(g["p2"]), _p(g["cat2"]), N, d2, d2, d2, 32, 96, 64, 1, s)
        self._relu(a["cat2"], g["cat2"], M2, 32, 96, 64)
        self._conv_bwd("e2b", a["e2a"], 32, 0, a["cat2"], 96, 64, g["cat2"], 96, 64, g["e2a"], 32, 0, N, d2)
        self._relu(a["e2a"], g["e2a"], M2, 32, 32, 0)
        self._conv_bwd("e2a", a["p1"], 16, 0, a["e2a"], 32, 0, g["e2a"], 32, 0, g["p1"], 16, 0, N, d2)
        _call("cl_nn_pool_bwd", _p(g["p1"]), _p(g["cat1"]), N, d1, d1, d1, 16, 48, 32, 1, s)
        self._relu(a["cat1"], g["cat1"], M, 16, 48, 32)
        self._conv_bwd("e1b", a["e1a"], 16, 0, a["cat1"], 48, 32, g["cat1"], 48, 32, g["e1a"], 16, 0, N, d1)
        self._relu(a["e1a"], g["e1a"], M, 16, 16, 0)
        self._conv_bwd("e1a", self.x, 16, 0, a["e1a"], 16, 0, g["e1a"], 16, 0, None, 16, 0, N, d1, need_gx=False)

    def _relu(self, y, gy, M, C, stride, off):
        _call("cl_nn_relu_bwd", _p(y), _p(gy), M, C, stride, off, self._stream())

    # ------------------------------------------------------------ update
    def step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        s = self._stream()
        for n in self.params:
            for k, p in enumerate(self.params[n]):
                m, v = self.adam[n][k]
                pb = self.wbf[n] if (k == 0 and n != "head") else None
                _call("cl_nn_adam", _p(p), _p(self.grads[n][k]), _p(m), _p(v), _p(pb), p.numel(), lr, b1, b2, eps,
                      self.t, s)

    def check(self):
        """Raise if a bounded wait of a tensor-core convolution expired since
        the last check (synchronises the current stream)."""
        _call("cl_nn_check", self._stream())

    def loss_value(self) -> float:
        return float(self.loss[0].item())

    # ------------------------------------------------------------ io
    def state_dict(self):
        return {f"{n}.{k}": p.detach().cpu().numpy() for n in self.params for k, p in enumerate(self.params[n])}

    def load_state_dict(self, sd):
        torch = self.torch
        for n in self.params:
            for k in range(len(self.params[n])):
                self.params[n][k].copy_(torch.from_numpy(np.asarray(sd[f"{n}.{k}"])).to(self.dev))
        for n, _, _ in CONV_LAYERS:
            _call("cl_nn_to_bf16", _p(self.params[n][0]), _p(self.wbf[n]), self.params[n][0].numel(), self._stream())

    def num_params(self) -> int:
        return sum(p.numel() for n in self.params for p in self.params[n])


# ---------------------------------------------------------------- weights
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart_unet.npz")


def load_pretrained(path: str = WEIGHTS) -> "UNet":
    """The network with the weights trained by ``warmstart_train`` (float16
    on disk, FP32 masters and BF16 copies on the GPU)."""
    net = UNet(seed=0)
    with np.load(path) as z:
        net.load_state_dict({k: z[k] for k in z.files})
    return net


# ---------------------------------------------------------------- solver glue
def features(solver):
    """bf16 [1, nz, ny, nx, 16] network input for a loaded solver."""
    import torch
    nz, ny, nx = solver.shape
    f = torch.empty(1, nz, ny, nx, FEATURES, dtype=torch.bfloat16, device="cuda")
    _call("cl_lbm_features", ctypes.c_void_p(solver.h), _p(f))
    return f


def target(solver):
    """fp32 [N] training target: (C - ramp) * nx on active cells (scale-free)."""
    import torch
    t = torch.empty(solver.n, dtype=torch.float32, device="cuda")
    _call("cl_lbm_target", ctypes.c_void_p(solver.h), _p(t))
    return t


def active_mask(solver):
    import torch
    m = torch.from_numpy(solver.setup()["active"].reshape(-1)).cuda()
    return m


def warm_start(net: UNet, solver):
    """Initialise the solver from the network's prediction (cubes, edge a multiple of 8)."""
    nz, ny, nx = solver.shape
    assert nz == ny == nx and nx % 8 == 0, "the network runs on cubes whose edge is a multiple of 8"
    f = features(solver)
    pred = net.forward(f, 1, nx)
    net.check()
    _call("cl_lbm_init_warm", ctypes.c_void_p(solver.h), _p(pred))
