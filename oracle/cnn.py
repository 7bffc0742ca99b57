"""CPU oracle of the early-stop network (TEST INFRASTRUCTURE ONLY).

Plain numpy in float64.  The network reads a syndrome of a size-L code as
two L x L maps (channel 0: the sigma_x generators, (L-1) x L, zero-padded;
channel 1: the sigma_z generators, L x (L-1), zero-padded), applies five 3x3
same-padded convolutions (2 -> 64 -> 64 -> 64 -> 64 -> 4, bias, ReLU after
the first four), averages each output channel over the map and returns the
log-softmax over the 4 classes.  The loss is the cross entropy with soft
targets, averaged over the batch.

`bf16=True` rounds weights, inputs and the stored post-ReLU activations to
bfloat16 (round to nearest even) at the same points as the tensor-core path,
which stores activations in bfloat16 and accumulates in float32.
"""
from __future__ import annotations

import numpy as np

C_HID = 64
K_CLS = 4
CHANNELS = [2, C_HID, C_HID, C_HID, C_HID, K_CLS]


def n_params() -> int:
    return sum(CHANNELS[i + 1] * 9 * CHANNELS[i] + CHANNELS[i + 1] for i in range(5))


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float64 values to bfloat16 (nearest even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(params: np.ndarray):
    """Flat parameter vector -> list of (W [co][3][3][ci], b [co]) per layer."""
    out, off = [], 0
    for i in range(5):
        ci, co = CHANNELS[i], CHANNELS[i + 1]
        w = params[off:off + co * 9 * ci].reshape(co, 3, 3, ci)
        off += co * 9 * ci
        b = params[off:off + co]
        off += co
        out.append((w, b))
    return out


def flatten(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def init_params(seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    layers = []
    for i in range(5):
        ci, co = CHANNELS[i], CHANNELS[i + 1]
        w = rng.normal(0, np.sqrt(2.0 / (9 * ci)), size=(co, 3, 3, ci))
        layers.append((w, np.zeros(co)))
    return flatten(layers)


def syndrome_maps(syn: np.ndarray, L: int) -> np.ndarray:
    """[n][2L(L-1)] 0/1 -> [n][L][L][2] maps (NHWC)."""
    syn = np.asarray(syn, np.float64).reshape(len(syn), -1)
    n = len(syn)
    x = np.zeros((n, L, L, 2))
    nx = (L - 1) * L
    x[:, :L - 1, :, 0] = syn[:, :nx].reshape(n, L - 1, L)
    x[:, :, :L - 1, 1] = syn[:, nx:].reshape(n, L, L - 1)
    return x


def _conv(x, w, b):
    """3x3 same conv, NHWC: y[n,y,x,co] = b[co] + sum w[co,kh,kw,ci] x[n,y+kh-1,x+kw-1,ci]."""
    n, H, W, ci = x.shape
    xp = np.zeros((n, H + 2, W + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((n, H, W, w.shape[0])) + b
    for kh in range(3):
        for kw in range(3):
            y += np.einsum("nhwc,oc->nhwo", xp[:, kh:kh + H, kw:kw + W, :], w[:, kh, kw, :])
    return y


def _conv_grad(x, w, dy):
    """Gradients of _conv: (dx, dw, db)."""
    n, H, W, ci = x.shape
    xp = np.zeros((n, H + 2, W + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for kh in range(3):
        for kw in range(3):
            dw[:, kh, kw, :] = np.einsum("nhwo,nhwc->oc", dy, xp[:, kh:kh + H, kw:kw + W, :])
            dxp[:, kh:kh + H, kw:kw + W, :] += np.einsum("nhwo,oc->nhwc", dy, w[:, kh, kw, :])
    return dxp[:, 1:-1, 1:-1, :], dw, dy.sum(axis=(0, 1, 2))


def forward(params, x, bf16=False, keep=False):
    """Log-probabilities [n][4] (and the activations if keep)."""
    layers = unflatten(params)
    rnd = bf16_round if bf16 else (lambda v: v)
    acts = [rnd(x)]
    a = acts[0]
    for i, (w, b) in enumerate(layers):
        z = _conv(a, rnd(w), b)
        if i < 4:
            a = rnd(np.maximum(z, 0.0))
            acts.append(a)
        else:
            acts.append(z)
    logits = acts[-1].mean(axis=(1, 2))
    m = logits.max(axis=1, keepdims=True)
    logp = logits - m - np.log(np.exp(logits - m).sum(axis=1, keepdims=True))
    return (logp, acts) if keep else logp


def loss_and_grad(params, x, targets, bf16=False):
    """Mean cross entropy with soft targets and its gradient (flat)."""
    layers = unflatten(params)
    rnd = bf16_round if bf16 else (lambda v: v)
    logp, acts = forward(params, x, bf16=bf16, keep=True)
    n, H, W = x.shape[:3]
    loss = -(targets * logp).sum() / n
    dlogits = (np.exp(logp) - targets) / n
    dz = np.broadcast_to(dlogits[:, None, None, :] / (H * W), acts[-1].shape).copy()
    grads = [None] * 5
    for i in range(4, -1, -1):
        w, b = layers[i]
        dx, dw, db = _conv_grad(acts[i], rnd(w), dz)
        grads[i] = (dw, db)
        if i > 0:
            dz = dx * (acts[i] > 0)
    return loss, flatten(grads)
