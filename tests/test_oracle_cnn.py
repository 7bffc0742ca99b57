"""Pins of the network oracle: the analytic gradient against central finite
differences (float64, no rounding), the conv against a direct sum, the
syndrome maps against the syndrome layout, the bfloat16 rounding, the
parity readout against brute-force enumeration of flip patterns, and the
reading of a class bit on the middle column/row against column/row 0 for
operators with a trivial syndrome."""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle import cnn


def test_param_count():
    assert cnn.n_params() == 64 * 18 + 64 + 3 * (64 * 576 + 64) + 2 * 576 + 2


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
    t = rng.dirichlet(np.ones(4), size=3)
    p = cnn.init_params(3) * 0.5
    p += rng.normal(0, 0.05, size=p.shape)        # nonzero biases
    loss, g = cnn.loss_and_grad(p, syn, L, t)
    idx = rng.choice(len(p), size=60, replace=False)
    idx = np.concatenate([idx, [len(p) - 1, len(p) - 2, len(p) - 5, 64 * 18, 64 * 18 + 63]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        num = (cnn.loss_and_grad(p + e, syn, L, t)[0] - cnn.loss_and_grad(p - e, syn, L, t)[0]) / (2 * h)
        assert abs(num - g[i]) < 1e-6 + 1e-4 * abs(num), (i, num, g[i])


def test_gradient_magnitude_bounds_the_gradient():
    """grad_magnitude (the sum of |terms| of every gradient element) is at
    least |gradient| everywhere (triangle inequality), scales with the
    targets, and equals |gradient| where no terms cancel: with every flip
    logit of the last layer negative (its -4 start bias), every term of the
    last layer's bias gradient of channel 0 has one sign."""
    L = 5
    rng = np.random.default_rng(11)
    syn, _ = O.gen_syndromes(17, 0, 4, L, 0.12)
    t = rng.dirichlet(np.ones(4), size=4)
    p = cnn.init_params(4)
    _, g = cnn.loss_and_grad(p, syn, L, t, bf16=True)
    A = cnn.grad_magnitude(p, syn, L, t, bf16=True)
    assert (np.abs(g) <= A * (1 + 1e-12) + 1e-300).all()
    assert np.allclose(cnn.grad_magnitude(p, syn, L, 2 * t, bf16=True), 2 * A, rtol=1e-12, atol=0)
    _, acts = cnn.forward(p, syn, L, bf16=True, keep=True)
    m = cnn.midline(L)
    assert (acts[-1][:, :, m, 0] < 0).all()
    t1 = np.eye(4)[[0, 1, 2, 3]]
    _, g1 = cnn.loss_and_grad(p, syn, L, t1, bf16=True)
    A1 = cnn.grad_magnitude(p, syn, L, t1, bf16=True)
    # all four one-hot targets: per syndrome the parity term of channel 0 has
    # one sign across the middle column's positions; the bias of output
    # channel 0 is the last-but-one parameter
    one = np.eye(4)[[0]]
    for i in range(4):
        _, gi = cnn.loss_and_grad(p, syn[i:i + 1], L, one, bf16=True)
        Ai = cnn.grad_magnitude(p, syn[i:i + 1], L, one, bf16=True)
        assert abs(abs(gi[-2]) - Ai[-2]) <= 1e-12 * Ai[-2], (i, gi[-2], Ai[-2])
    assert (np.abs(g1) <= A1 * (1 + 1e-12)).all()


def test_logprob_normalised():
    L = 5
    syn, _ = O.gen_syndromes(8, 0, 6, L, 0.15)
    logp = cnn.forward(cnn.init_params(1), syn, L, bf16=True)
    assert np.allclose(np.exp(logp).sum(1), 1.0)


@pytest.mark.parametrize("L", [3, 4, 5])
def test_parity_readout_is_exact_for_independent_flips(L):
    """P(class) from the product rule equals the sum over all 2^L x 2^L flip
    patterns of the midline qubits (independent flips with probability
    sigmoid(s)) of the probability of the patterns with that parity pair."""
    rng = np.random.default_rng(L)
    m = cnn.midline(L)
    z5 = np.zeros((1, L, L, 2))
    sa, sb = rng.normal(0, 2, size=L), rng.normal(0, 2, size=L)
    z5[0, :, m, 0] = sa
    z5[0, m, :, 1] = sb
    for c0 in range(4):
        _, _, Ma, Mb = cnn._readout(z5, L)
        logp = cnn._class_logp(Ma, Mb, np.array([c0]))
        qa, qb = 1 / (1 + np.exp(-sa)), 1 / (1 + np.exp(-sb))

        def parity_probs(q):
            pr = np.zeros(2)
            for f in itertools.product([0, 1], repeat=len(q)):
                pr[sum(f) & 1] += np.prod([qi if fi else 1 - qi for qi, fi in zip(q, f)])
            return pr
        pa, pb = parity_probs(qa), parity_probs(qb)
        for k in range(4):
            want = pa[(k & 1) ^ (c0 & 1)] * pb[(k >> 1) ^ (c0 >> 1)]
            assert abs(np.exp(logp[0, k]) - want) < 1e-9


@pytest.mark.parametrize("L", [4, 5, 6, 7])
def test_class_bits_read_on_the_middle_lines(L):
    """For random stabilizer products times a random logical, the sigma_x
    parity on qubit column 2m and the sigma_z parity on qubit row 2m equal
    the class code (column 0 / row 0)."""
    rng = np.random.default_rng(100 + L)
    m = cnn.midline(L)
    n = 2 * L - 1
    qi = lambda r, c: (r * n + c) // 2
    for _ in range(30):
        ex = np.zeros(O.nq(L), np.uint8)
        ez = np.zeros(O.nq(L), np.uint8)
        for g in rng.choice(O.nstab(L), size=rng.integers(1, 3 * L), replace=True):
            t, _, _ = O.stab_pos(L, g)
            for q in O.stab_support(L, g):
                if t == 0:
                    ex[q] ^= 1
                else:
                    ez[q] ^= 1
        k = int(rng.integers(4))
        ex, ez = O.apply_logical(L, k, ex, ez)
        assert (O.syndrome(L, ex, ez) == 0).all()
        code = O.class_code(L, ex, ez)
        a_mid = int(sum(ex[qi(2 * i, 2 * m)] for i in range(L)) & 1)
        b_mid = int(sum(ez[qi(2 * m, 2 * j)] for j in range(L)) & 1)
        assert code == k and a_mid + 2 * b_mid == k
