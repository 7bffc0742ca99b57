"""CPU oracle of the early-stop network (TEST INFRASTRUCTURE ONLY).

Plain numpy in float64.  The network reads a syndrome of a size-L code as
two L x L maps (channel 0: the sigma_x generators, (L-1) x L, zero-padded;
channel 1: the sigma_z generators, L x (L-1), zero-padded) and applies five
3x3 same-padded convolutions (2 -> 64 -> 64 -> 64 -> 64 -> 2, bias, ReLU
after the first four).

Readout.  A class is the logical coset of an error: bit a = parity of its
sigma_x part on qubit column 0, bit b = parity of its sigma_z part on qubit
row 0 (the class code of the decoder).  Let e0 be the decoder's pure error
(straight strings to the nearest boundary) with class code c0.  E + e0 has a
trivial syndrome, so its sigma_x parity is the same on every even qubit
column and its sigma_z parity the same on every even qubit row; the network
reads them on the middle ones, column 2m and row 2m with m = (L-1) div 2,
where they are set by local configurations.  Output channel 0 at map
position (i, m) is the logit s of "(E + e0)_x = 1 on qubit (2i, 2m)";
channel 1 at (m, j) that of "(E + e0)_z = 1 on qubit (2m, 2j)".  Taking the
flips as independent, P(parity odd) = (1 - M) / 2 with M = prod_i (1 - 2
sigmoid(s_i)) = prod_i (-tanh(s_i / 2)), M clipped to [-1 + 1e-6, 1 - 1e-6].
Class k = a + 2b then has log p_k = log P_x((a xor a0)) + log P_z((b xor
b0)) with c0 = a0 + 2 b0.  The loss is the cross entropy with soft targets,
averaged over the batch.

`bf16=True` rounds weights, inputs and the stored post-ReLU activations to
bfloat16 (round to nearest even) at the same points as the tensor-core path,
which stores activations in bfloat16 and accumulates in float32.
"""
from __future__ import annotations

import numpy as np

C_HID = 64
K_CLS = 4
N_OUT = 2
CHANNELS = [2, C_HID, C_HID, C_HID, C_HID, N_OUT]
CLIP = 1e-6
FLIP_BIAS = -4.0   # initial last-layer bias: flips start unlikely (M near 1)


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
        layers.append((w, np.full(co, FLIP_BIAS if i == 4 else 0.0)))
    return flatten(layers)


def midline(L: int) -> int:
    return (L - 1) // 2


def pure_error_codes(syn: np.ndarray, L: int) -> np.ndarray:
    """Class code c0 of the decoder's pure error of each syndrome."""
    import oracle as O
    syn = np.asarray(syn, np.uint8).reshape(len(syn), -1)
    return np.array([O.class_code(L, *O.pure_error(L, row)) for row in syn], np.int64)


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


def _readout(z5, L):
    """M_x, M_z (clipped products) and the factors, from the last layer."""
    m = midline(L)
    ta = -np.tanh(z5[:, :, m, 0] / 2.0)   # [n][L], rows i
    tb = -np.tanh(z5[:, m, :, 1] / 2.0)   # [n][L], columns j
    Ma, Mb = ta.prod(axis=1), tb.prod(axis=1)
    return ta, tb, Ma, Mb


def _class_logp(Ma, Mb, c0):
    Mac = np.clip(Ma, -1 + CLIP, 1 - CLIP)
    Mbc = np.clip(Mb, -1 + CLIP, 1 - CLIP)
    la = np.stack([np.log((1 + Mac) / 2), np.log((1 - Mac) / 2)], axis=1)   # parity of (E+e0)_x
    lb = np.stack([np.log((1 + Mbc) / 2), np.log((1 - Mbc) / 2)], axis=1)
    n = len(c0)
    a0, b0 = c0 & 1, c0 >> 1
    logp = np.empty((n, 4))
    for k in range(4):
        logp[:, k] = la[np.arange(n), (k & 1) ^ a0] + lb[np.arange(n), (k >> 1) ^ b0]
    return logp


def forward(params, syn, L, bf16=False, keep=False):
    """Log-probabilities [n][4] of the classes of n syndromes (and the
    activations if keep)."""
    x = syndrome_maps(syn, L)
    c0 = pure_error_codes(syn, L)
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
    _, _, Ma, Mb = _readout(acts[-1], L)
    logp = _class_logp(Ma, Mb, c0)
    return (logp, acts) if keep else logp


def loss_and_grad(params, syn, L, targets, bf16=False):
    """Mean cross entropy with soft targets and its gradient (flat)."""
    layers = unflatten(params)
    rnd = bf16_round if bf16 else (lambda v: v)
    logp, acts = forward(params, syn, L, bf16=bf16, keep=True)
    c0 = pure_error_codes(syn, L)
    n = len(c0)
    loss = -(targets * logp).sum() / n
    # d loss / d log P_x(v), d log P_z(v): targets summed over the classes using v
    a0, b0 = c0 & 1, c0 >> 1
    ga = np.zeros((n, 2))
    gb = np.zeros((n, 2))
    for k in range(4):
        ga[np.arange(n), (k & 1) ^ a0] -= targets[:, k] / n
        gb[np.arange(n), (k >> 1) ^ b0] -= targets[:, k] / n
    ta, tb, Ma, Mb = _readout(acts[-1], L)

    def d_prod(t, M, g):
        inside = (M > -1 + CLIP) & (M < 1 - CLIP)
        dM = np.where(inside, g[:, 0] / (1 + M) - g[:, 1] / (1 - M), 0.0)      # d loss / d M
        others = np.empty_like(t)
        for i in range(t.shape[1]):
            others[:, i] = np.prod(np.delete(t, i, axis=1), axis=1)
        dt_ds = -(1 - t * t) / 2.0          # t = -tanh(s/2): dt/ds = -(1 - tanh^2)/2
        return dM[:, None] * others * dt_ds

    m = midline(L)
    dz = np.zeros_like(acts[-1])
    dz[:, :, m, 0] = d_prod(ta, Ma, ga)
    dz[:, m, :, 1] = d_prod(tb, Mb, gb)
    grads = [None] * 5
    for i in range(4, -1, -1):
        w, b = layers[i]
        dx, dw, db = _conv_grad(acts[i], rnd(w), dz)
        grads[i] = (dw, db)
        if i > 0:
            dz = dx * (acts[i] > 0)
    return loss, flatten(grads)


def grad_magnitude(params, syn, L, targets, bf16=False):
    """Per parameter, the sum of the absolute values of the terms whose sum
    is its gradient (flat, like loss_and_grad): the backward pass of
    loss_and_grad with every factor replaced by its absolute value.  A
    gradient computed from the same terms with relative errors of at most u
    in each stored factor differs from the exact one by at most about
    (stored factors) x u x this magnitude; the GPU's float32 accumulation
    adds only a few units of 2^-24 relative to it."""
    layers = unflatten(params)
    rnd = bf16_round if bf16 else (lambda v: v)
    _, acts = forward(params, syn, L, bf16=bf16, keep=True)
    c0 = pure_error_codes(syn, L)
    n = len(c0)
    a0, b0 = c0 & 1, c0 >> 1
    ga = np.zeros((n, 2))
    gb = np.zeros((n, 2))
    for k in range(4):
        ga[np.arange(n), (k & 1) ^ a0] -= targets[:, k] / n
        gb[np.arange(n), (k >> 1) ^ b0] -= targets[:, k] / n
    ta, tb, Ma, Mb = _readout(acts[-1], L)

    def d_prod_abs(t, M, g):
        inside = (M > -1 + CLIP) & (M < 1 - CLIP)
        dM = np.where(inside, np.abs(g[:, 0] / (1 + M)) + np.abs(g[:, 1] / (1 - M)), 0.0)
        others = np.empty_like(t)
        for i in range(t.shape[1]):
            others[:, i] = np.prod(np.abs(np.delete(t, i, axis=1)), axis=1)
        return dM[:, None] * others * (1 - t * t) / 2.0

    m = midline(L)
    dz = np.zeros_like(acts[-1])
    dz[:, :, m, 0] = d_prod_abs(ta, Ma, ga)
    dz[:, m, :, 1] = d_prod_abs(tb, Mb, gb)
    grads = [None] * 5
    for i in range(4, -1, -1):
        w, b = layers[i]
        dx, dw, db = _conv_grad(np.abs(acts[i]), np.abs(rnd(w)), dz)
        grads[i] = (dw, db)
        if i > 0:
            dz = dx * (acts[i] > 0)
    return flatten(grads)
