"""Pins of the oracle under independent bit and phase flips (Sec. IV.B): each
qubit suffers sigma_x with probability p and, independently, sigma_z with
probability p, so a frame's weight is n = |x| + |z| and e^{-beta_bar} =
p / (1 - p).  Pinned by binomial tests of the generator, the closed-form
table, the factorisation of the class partition functions (the bit-flip and
phase-flip problems are independent), chi^2 over all states at L = 2, exact
<n> by enumeration at L = 3, and <n> = n_q at beta = 0."""
import math

import numpy as np
import pytest

import oracle as O
from test_oracle_mcmc import _class_states


def test_flip_generator_frequencies():
    L, p, n = 9, 0.1, 400
    nq = O.nq(L)
    xs = zs = both = 0
    for i in range(n):
        ex, ez = O.gen_error_flips(77, i, L, p)
        xs += int(ex.sum())
        zs += int(ez.sum())
        both += int((ex & ez).sum())
    N = n * nq
    for cnt, q in ((xs, p), (zs, p), (both, p * p)):
        assert abs(cnt - N * q) < 5 * math.sqrt(N * q * (1 - q)), (cnt, N * q)
    syn, tc = O.gen_syndromes(77, 0, 3, L, p, noise=1)
    for i in range(3):
        ex, ez = O.gen_error_flips(77, i, L, p)
        assert (O.syndrome(L, ex, ez) == syn[i]).all() and O.class_code(L, ex, ez) == tc[i]


def test_flip_thresholds_closed_form():
    for p in (0.05, 0.1, 0.2):
        T, bb = O.thresholds(p, noise=1)
        r = p / (1 - p)
        assert abs(bb - (-math.log(r))) < 1e-15
        for d in range(1, 5):
            assert abs(int(T[d]) - r ** d * 2 ** 32) <= 2


@pytest.mark.parametrize("L,seed", [(3, 1), (3, 2), (4, 3)])
def test_class_partition_functions_factorise(L, seed):
    """Z_(a,b) = Z_x(a) Z_z(b): log Z_(1,b) - log Z_(0,b) does not depend on b."""
    syn, _ = O.gen_syndromes(seed, 0, 1, L, 0.12, noise=1)
    logz, _ = O.exact_class_stats(L, syn[0], -math.log(0.12 / 0.88), noise=1)
    assert abs((logz[1] - logz[0]) - (logz[3] - logz[2])) < 1e-9
    assert abs((logz[2] - logz[0]) - (logz[3] - logz[1])) < 1e-9


def test_flip_mean_at_infinite_temperature():
    L = 3
    syn, _ = O.gen_syndromes(4, 0, 1, L, 0.1, noise=1)
    _, m = O.exact_class_stats(L, syn[0], 0.0, noise=1)
    assert np.allclose(m, O.nq(L), atol=1e-12)


def test_flip_l2_state_distribution_chi2():
    L, p, R, sweeps = 2, 0.3, 512, 48
    r = p / (1 - p)
    syn = np.array([1, 0, 1, 1], np.uint8)
    for scan in (0, 1):
        out = O.run_chains(L, 4, R, p, 4321 + scan, 0, syn, 0, sweeps, scan=scan, noise=1)
        for k in range(4):
            states = _class_states(L, syn, k)
            key = {bytes(np.concatenate(s)): i for i, s in enumerate(states)}
            w = np.array([r ** int(fx.sum() + fz.sum()) for fx, fz in states])
            w /= w.sum()
            cnt = np.zeros(16)
            for c in range(k * R, (k + 1) * R):
                cnt[key[bytes(np.concatenate([out["frames_x"][c], out["frames_z"][c]]))]] += 1
            e = w * R
            big = e >= 5
            obs = np.append(cnt[big], cnt[~big].sum())
            exp_ = np.append(e[big], e[~big].sum())
            if exp_[-1] == 0:
                obs, exp_ = obs[:-1], exp_[:-1]
            chi2 = ((obs - exp_) ** 2 / exp_).sum()
            dof = len(obs) - 1
            assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (scan, k, chi2, dof)


@pytest.mark.parametrize("L,p,seed", [(3, 0.1, 21), (3, 0.2, 22)])
def test_flip_mean_n_matches_enumeration(L, p, seed):
    R, sweeps, burn = 48, 300, 50
    syn, _ = O.gen_syndromes(seed, 0, 1, L, p, noise=1)
    syn = syn[0]
    _, bb = O.thresholds(p, noise=1)
    _, exact = O.exact_class_stats(L, syn, bb, noise=1)
    out = O.run_chains(L, 4, R, p, 900 + seed, 0, syn, 0, sweeps, burn_in=burn, noise=1)
    per_chain = out["chain_sum"].astype(np.float64) / (4 * (sweeps - burn))
    for k in range(4):
        x = per_chain[k * R:(k + 1) * R]
        se = x.std(ddof=1) / math.sqrt(R)
        assert abs(x.mean() - exact[k]) < 5 * se + 0.02, (k, x.mean(), exact[k], se)
    d = O.decode_one(L, p, 4, 4, 30, 5, 0, syn, noise=1)
    for c in range(16):
        fx, fz = d["frames_x"][c], d["frames_z"][c]
        assert d["chain_n"][c] == int(fx.sum() + fz.sum())
        assert (O.syndrome(L, fx, fz) == syn).all() and O.class_code(L, fx, fz) == c // 4
