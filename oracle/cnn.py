"""Oracle (test infrastructure): the learned-score CNN in FP64 numpy.

Plain definitions, no blocking or fusion:
  conv3x3 'same' (zero padding)   out[b,y,x,o] = bias[o] + sum_{ky,kx,c} in[b,y+ky-1,x+kx-1,c] w[o,ky,kx,c]
  ReLU after each of the 4 conv layers (channels 8 -> 32 -> 32 -> 32 -> 32)
  global mean pool                h[b,o] = mean_{y,x} a4[b,y,x,o]
  linear head                     pred[b] = v . h[b] + c
  loss                            (1/B) sum_b (pred[b] - y[b])^2
  gradients                       chain rule written out by hand (pinned by
                                  central finite differences in the tests)
  Adam                            Kingma & Ba (2015), bias-corrected.

The flat parameter vector follows the library's documented layout: for conv
layer l, W_l[o][k] with k = (3 ky + kx) * C_in + c (C_in = 8 for the input
layer, 32 after), the bias at k = 9 C_in, zeros up to 80 or 304 columns; then
the head v[32] and its bias.
"""
from __future__ import annotations

import numpy as np

CIN = (8, 32, 32, 32)
KPAD = (80, 304, 304, 304)
C = 32


def offsets():
    off, o = [], 0
    for k in KPAD:
        off.append(o)
        o += C * k
    off.append(o)
    return off, o + C + 1


def unpack(p: np.ndarray):
    """flat vector -> ([(w [32,3,3,cin], bias [32])] * 4, v [32], c)"""
    off, n = offsets()
    p = np.asarray(p, dtype=np.float64)
    assert p.size == n
    layers = []
    for l, (cin, kp) in enumerate(zip(CIN, KPAD)):
        m = p[off[l]:off[l] + C * kp].reshape(C, kp)
        w = m[:, :9 * cin].reshape(C, 3, 3, cin)
        layers.append((w, m[:, 9 * cin].copy()))
    v = p[off[4]:off[4] + C].copy()
    return layers, v, float(p[off[4] + C])


def pack(layers, v, c) -> np.ndarray:
    off, n = offsets()
    p = np.zeros(n)
    for l, ((w, bias), cin, kp) in enumerate(zip(layers, CIN, KPAD)):
        m = np.zeros((C, kp))
        m[:, :9 * cin] = w.reshape(C, 9 * cin)
        m[:, 9 * cin] = bias
        p[off[l]:off[l] + C * kp] = m.ravel()
    p[off[4]:off[4] + C] = v
    p[off[4] + C] = c
    return p


def conv3x3(x, w, bias):
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, H, W, w.shape[0])) + bias
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    return out


def conv3x3_input_grad(dout, w):
    """gradient of conv3x3 with respect to its input"""
    B, H, W, _ = dout.shape
    dxp = np.zeros((B, H + 2, W + 2, w.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("bhwo,oc->bhwc", dout, w[:, ky, kx, :])
    return dxp[:, 1:H + 1, 1:W + 1, :]


def conv3x3_weight_grad(x, dout):
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dw = np.zeros((dout.shape[3], 3, 3, x.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dout, xp[:, ky:ky + H, kx:kx + W, :])
    return dw, dout.sum(axis=(0, 1, 2))


def _keep(a):
    return a


def forward(p, x, store=_keep):
    """returns pred [B] and the intermediate values.  store(a) is applied to
    every activation as it would be stored between layers (identity: FP64
    throughout; a rounding function emulates a lower storage precision)."""
    layers, v, c = unpack(p)
    acts = [np.asarray(x, dtype=np.float64)]
    for w, bias in layers:
        acts.append(store(np.maximum(conv3x3(acts[-1], w, bias), 0.0)))
    h = acts[-1].mean(axis=(1, 2))
    return h @ v + c, (acts, h)


def loss_and_grad(p, x, y, store=_keep):
    """loss and flat gradient; store(a) is applied to activations and to the
    gradients with respect to pre-activations as they would be stored"""
    layers, v, c = unpack(p)
    pred, (acts, h) = forward(p, x, store)
    y = np.asarray(y, dtype=np.float64)
    B = len(y)
    loss = np.mean((pred - y) ** 2)
    dpred = 2.0 * (pred - y) / B
    gv = h.T @ dpred
    gc = dpred.sum()
    P = acts[-1].shape[1] * acts[-1].shape[2]
    da = np.broadcast_to((dpred[:, None] * v[None, :] / P)[:, None, None, :], acts[-1].shape).copy()
    grads = [None] * 4
    for l in range(3, -1, -1):
        dpre = store(da * (acts[l + 1] > 0))
        gw, gb = conv3x3_weight_grad(acts[l], dpre)
        grads[l] = (gw, gb)
        if l > 0:
            da = conv3x3_input_grad(dpre, layers[l][0])
    return loss, pack(grads, gv, gc)


class Adam:
    def __init__(self, n, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, p, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return p - self.lr * mh / (np.sqrt(vh) + self.eps)


def fields(c, f, factor, rho_scale, u_scale):
    """network input of one clone's populations f [9][ny][nx] (FP64): block
    means of (rho - 1, u_x, u_y) of the post-collision state, scaled, plus five
    zero channels -> [ny // factor][nx // factor][8].  The blocks tile the
    lattice from node (0, 0); rows and columns past the last whole block are
    not in the input."""
    from oracle import macro
    rho, ux, uy = macro(c, f)
    ny, nx = rho.shape
    H, W = ny // factor, nx // factor

    def pool(a):
        return a[:H * factor, :W * factor].reshape(H, factor, W, factor).mean(axis=(1, 3))
    out = np.zeros((H, W, 8))
    out[..., 0] = pool(rho - 1.0) * rho_scale
    out[..., 1] = pool(ux) * u_scale
    out[..., 2] = pool(uy) * u_scale
    return out
