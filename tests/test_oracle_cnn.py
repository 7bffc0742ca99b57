"""Pins of the network oracle: the analytic gradient against central finite
differences (float64, no rounding), the conv against a direct sum, the
syndrome maps against the syndrome layout, the bfloat16 rounding."""
import numpy as np
import pytest

import oracle as O
from oracle import cnn


def test_param_count():
    assert cnn.n_params() == 64 * 18 + 64 + 3 * (64 * 576 + 64) + 4 * 576 + 4


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3.14159265])
    r = cnn.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0              # tie to even
    assert r[2] == 1.0 + 2 ** -7                      # representable
    assert r[3] == 1.0 + 2 ** -6                      # tie to even (up)
    assert r[4] == -2.5 and abs(r[5] - 3.140625) < 1e-12


def test_conv_is_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 5, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = cnn._conv(x, w, b)
    for (n, i, j, o) in [(0, 0, 0, 0), (1, 4, 2, 3), (0, 2, 4, 1)]:
        s = b[o]
        for kh in range(3):
            for kw in range(3):
                ii, jj = i + kh - 1, j + kw - 1
                if 0 <= ii < 5 and 0 <= jj < 5:
                    s += (w[o, kh, kw, :] * x[n, ii, jj, :]).sum()
        assert abs(s - y[n, i, j, o]) < 1e-12


def test_syndrome_maps_layout():
    L = 5
    syn, _ = O.gen_syndromes(3, 0, 4, L, 0.2)
    x = cnn.syndrome_maps(syn, L)
    for i in range(4):
        for g in range(O.nstab(L)):
            t, r, c = O.stab_pos(L, g)
            if t == 0:
                assert x[i, (r - 1) // 2, c // 2, 0] == syn[i, g]
            else:
                assert x[i, r // 2, (c - 1) // 2, 1] == syn[i, g]
    assert x[:, L - 1, :, 0].sum() == 0 and x[:, :, L - 1, 1].sum() == 0


def test_gradient_matches_finite_differences():
    L = 4
    rng = np.random.default_rng(2)
    syn, _ = O.gen_syndromes(5, 0, 3, L, 0.25)
    x = cnn.syndrome_maps(syn, L)
    t = rng.dirichlet(np.ones(4), size=3)
    p = cnn.init_params(3) * 0.5
    p += rng.normal(0, 0.05, size=p.shape)        # nonzero biases
    loss, g = cnn.loss_and_grad(p, x, t)
    idx = rng.choice(len(p), size=60, replace=False)
    idx = np.concatenate([idx, [len(p) - 1, len(p) - 5, 64 * 18, 64 * 18 + 63]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        num = (cnn.loss_and_grad(p + e, x, t)[0] - cnn.loss_and_grad(p - e, x, t)[0]) / (2 * h)
        assert abs(num - g[i]) < 1e-6 + 1e-4 * abs(num), (i, num, g[i])


def test_logprob_normalised():
    L = 5
    syn, _ = O.gen_syndromes(8, 0, 6, L, 0.15)
    logp = cnn.forward(cnn.init_params(1), cnn.syndrome_maps(syn, L), bf16=True)
    assert np.allclose(np.exp(logp).sum(1), 1.0)
