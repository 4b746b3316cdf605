"""Plain FP64 CPU oracle of the convolutional surrogate's forward and backward
passes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library.

The surrogate (the learned K-step map the method's statement asks for; the
paper itself has no learned component) is a U-Net on the periodic lattice:

* arrays are NHWC: (batch, H, W, channels);
* conv3x3: out[y, x, o] = b[o] + sum_{ky, kx, c} W[o, ky, kx, c]
  in[(y + ky - 1) mod H, (x + kx - 1) mod W, c] (circular padding: the
  domain is periodic), followed by ReLU except in the head;
* level l of L has C_l = C_0 2^l channels; the encoder applies two conv3x3 +
  ReLU per level and a 2x2 average pool between levels; the decoder
  upsamples by nearest-neighbour repetition, concatenates [upsampled, skip]
  along channels and applies two conv3x3 + ReLU; the head is a 1x1
  convolution to the output channels;
* loss = mean over all elements of (prediction - target)^2.

Backward passes are written out layer by layer (chain rule), pinned by
finite differences in tests/test_oracle_surrogate.py.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Net:
    levels: int
    c0: int
    c_in: int
    c_out: int
    # conv weights (O, 3, 3, C) and biases (O,), in the order of conv_specs()
    W: list = field(default_factory=list)
    b: list = field(default_factory=list)
    Wh: np.ndarray = None      # head (c_out, c0)
    bh: np.ndarray = None      # (c_out,)


def conv_specs(levels: int, c0: int, c_in: int):
    """(input channels, output channels) of every 3x3 convolution in order:
    encoder level 0..L-1 (two each), then decoder level L-2..0 (two each)."""
    ch = [c0 << l for l in range(levels)]
    specs = []
    prev = c_in
    for l in range(levels):
        specs += [(prev, ch[l]), (ch[l], ch[l])]
        prev = ch[l]
    for l in range(levels - 2, -1, -1):
        specs += [(ch[l + 1] + ch[l], ch[l]), (ch[l], ch[l])]
    return specs


def init_net(levels, c0, c_in, c_out, rng) -> Net:
    net = Net(levels, c0, c_in, c_out)
    for ci, co in conv_specs(levels, c0, c_in):
        net.W.append(rng.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci)))
        net.b.append(0.01 * rng.standard_normal(co))
    net.Wh = rng.standard_normal((c_out, c0)) * np.sqrt(1.0 / c0)
    net.bh = 0.01 * rng.standard_normal(c_out)
    return net


# ----------------------------------------------------------------- layers
def shifted(x, dy, dx):
    """s[:, y, x] = x[:, (y + dy) mod H, (x + dx) mod W]."""
    return np.roll(x, (-dy, -dx), axis=(1, 2))


def conv3x3(x, W, b):
    out = np.broadcast_to(b, x.shape[:3] + (W.shape[0],)).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("bhwc,oc->bhwo", shifted(x, ky - 1, kx - 1), W[:, ky, kx, :])
    return out


def conv3x3_backward(x, W, dz):
    """Gradients of conv3x3 given dL/d(out) = dz: (dx, dW, db)."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for ky in range(3):
        for kx in range(3):
            dW[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dz, shifted(x, ky - 1, kx - 1))
            # out[y] uses x[y + d]: the gradient flows back to x[y + d] from out[y]
            dx += shifted(np.einsum("bhwo,oc->bhwc", dz, W[:, ky, kx, :]), -(ky - 1), -(kx - 1))
    return dx, dW, dz.sum(axis=(0, 1, 2))


def relu(z):
    return np.maximum(z, 0.0)


def pool2(x):
    b, h, w, c = x.shape
    return x.reshape(b, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool2_backward(d):
    return np.repeat(np.repeat(d, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(d):
    b, h, w, c = d.shape
    return d.reshape(b, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


# --------------------------------------------------------------- network
def forward(net: Net, x):
    """Returns (prediction, cache) for NHWC input x."""
    L = net.levels
    cache = {"acts": [], "skips": []}
    k = 0
    h = x
    for l in range(L):
        if l > 0:
            h = pool2(h)
        for _ in range(2):
            cache["acts"].append(h)
            h = relu(conv3x3(h, net.W[k], net.b[k]))
            cache.setdefault("outs", []).append(h)
            k += 1
        cache["skips"].append(h)
    for l in range(L - 2, -1, -1):
        h = np.concatenate([up2(h), cache["skips"][l]], axis=3)
        for _ in range(2):
            cache["acts"].append(h)
            h = relu(conv3x3(h, net.W[k], net.b[k]))
            cache["outs"].append(h)
            k += 1
    cache["head_in"] = h
    pred = np.einsum("bhwc,oc->bhwo", h, net.Wh) + net.bh
    return pred, cache


def loss(pred, target):
    return float(np.mean((pred - target) ** 2))


def backward(net: Net, x, target):
    """Loss and gradients (dW list, db list, dWh, dbh) by the chain rule."""
    pred, cache = forward(net, x)
    L = net.levels
    n = pred.size
    dpred = 2.0 * (pred - target) / n
    h = cache["head_in"]
    dWh = np.einsum("bhwo,bhwc->oc", dpred, h)
    dbh = dpred.sum(axis=(0, 1, 2))
    dh = np.einsum("bhwo,oc->bhwc", dpred, net.Wh)
    nconv = len(net.W)
    dW = [None] * nconv
    db = [None] * nconv
    dskip = [np.zeros_like(s) for s in cache["skips"]]
    k = nconv - 1
    for l in range(0, L - 1):
        # decoder level l, convs in reverse
        for _ in range(2):
            dz = dh * (cache["outs"][k] > 0)
            dh, dW[k], db[k] = conv3x3_backward(cache["acts"][k], net.W[k], dz)
            k -= 1
        c_up = dh.shape[3] - cache["skips"][l].shape[3]
        dskip[l] += dh[..., c_up:]
        dh = up2_backward(dh[..., :c_up])
    for l in range(L - 1, -1, -1):
        dh = dh + dskip[l] if l < L - 1 else dh
        for _ in range(2):
            dz = dh * (cache["outs"][k] > 0)
            dh, dW[k], db[k] = conv3x3_backward(cache["acts"][k], net.W[k], dz)
            k -= 1
        if l > 0:
            dh = pool2_backward(dh)
    return loss(pred, target), dW, db, dWh, dbh
