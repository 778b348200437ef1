"""FP64 CPU oracle of the warm-start network (test infrastructure only).

Plain numpy, double precision, written from the definitions:
  conv3d   O[n,z,y,x,o] = b[o] + sum_{t,i} I[n, z+dz_t, y+dy_t, x+dx_t, i] W[t,o,i]
           taps t = 9 kz + 3 ky + kx, offsets (kz-1, ky-1, kx-1); x is zero
           padded, y and z wrap (the structures are periodic in y and z);
  relu, 2x2x2 average pooling, 2x nearest upsampling, channel concatenation,
  a 1x1x1 head, and the masked mean-squared loss.
Gradients are not written out: tests differentiate this forward by central
finite differences, which pins the GPU's analytic backward without sharing
its formulas.  Layout NDHWC.

Network (4 levels, 16/32/64/128 channels):
  e1 = relu(conv(relu(conv(x, 16)), 16))                 full resolution
  e2 = two convs to 32 after pooling, e3 to 64, bottom to 128
  d3 = two convs (192 -> 64 -> 64) on [up(bottom), e3]
  d2 = two convs (96 -> 32 -> 32) on [up(d3), e2]
  d1 = two convs (48 -> 16 -> 16) on [up(d2), e1]
  out = head(d1) (1x1x1, 16 -> 1, no activation)
"""
from __future__ import annotations

import numpy as np

CONV_LAYERS = [
    # name, c_in, c_out
    ("e1a", 16, 16), ("e1b", 16, 16),
    ("e2a", 16, 32), ("e2b", 32, 32),
    ("e3a", 32, 64), ("e3b", 64, 64),
    ("bta", 64, 128), ("btb", 128, 128),
    ("d3a", 192, 64), ("d3b", 64, 64),
    ("d2a", 96, 32), ("d2b", 32, 32),
    ("d1a", 48, 16), ("d1b", 16, 16),
]
IN_CHANNELS = 16  # input features padded to 16 channels


def conv3d(x, w, b, periodic_yz=True):
    """x [N,D,H,W,Ci], w [27,Co,Ci], b [Co] -> [N,D,H,W,Co]."""
    N, D, H, W, Ci = x.shape
    Co = w.shape[1]
    out = np.broadcast_to(b, (N, D, H, W, Co)).astype(np.float64).copy()
    for t in range(27):
        dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
        xs = x
        if periodic_yz:
            xs = np.roll(xs, shift=(-dz, -dy), axis=(1, 2))
        else:
            pad = np.zeros_like(xs)
            zs = slice(max(0, dz), D + min(0, dz))
            zd = slice(max(0, -dz), D + min(0, -dz))
            ys = slice(max(0, dy), H + min(0, dy))
            yd = slice(max(0, -dy), H + min(0, -dy))
            pad[:, zd, yd] = xs[:, zs, ys]
            xs = pad
        shifted = np.zeros_like(xs)
        if dx >= 0:
            shifted[:, :, :, : W - dx] = xs[:, :, :, dx:]
        else:
            shifted[:, :, :, -dx:] = xs[:, :, :, : W + dx]
        out += np.einsum("ndhwi,oi->ndhwo", shifted, w[t])
    return out


def relu(x):
    return np.maximum(x, 0.0)


def pool(x):
    N, D, H, W, C = x.shape
    return x.reshape(N, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4, 6))


def up(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def forward(params, x, periodic_yz=True):
    """params: dict name -> (w [27,Co,Ci], b [Co]) and 'head' -> (w [Ci=16], b scalar)."""
    def block(h, a, b_):
        h = relu(conv3d(h, *params[a], periodic_yz))
        return relu(conv3d(h, *params[b_], periodic_yz))

    e1 = block(x, "e1a", "e1b")
    e2 = block(pool(e1), "e2a", "e2b")
    e3 = block(pool(e2), "e3a", "e3b")
    bt = block(pool(e3), "bta", "btb")
    d3 = block(np.concatenate([up(bt), e3], axis=-1), "d3a", "d3b")
    d2 = block(np.concatenate([up(d3), e2], axis=-1), "d2a", "d2b")
    d1 = block(np.concatenate([up(d2), e1], axis=-1), "d1a", "d1b")
    hw, hb = params["head"]
    return np.einsum("ndhwc,c->ndhw", d1, hw) + hb


def masked_mse(pred, target, mask):
    """mean over masked cells of (pred - target)^2."""
    m = mask.astype(np.float64)
    return float(np.sum(m * (pred - target) ** 2) / max(np.sum(m), 1.0))
