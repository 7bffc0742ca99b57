"""Pins of the oracle's general Pauli channel (Eq. 1 with integer energies:
p_X : p_Y : p_Z : p_I = r^eX : r^eY : r^eZ : 1, Sec. IV's generalisation to
arbitrary channels of that form).  Pinned by the two special cases the paper
names (depolarizing = (1, 1, 1), independent flips = (1, 2, 1)), binomial
generator tests, chi^2 of random-scan chain states at L = 2, exact <E> by
enumeration at L = 3, and <E> = n_q (eX + eY + eZ) / 4 at beta = 0."""
import math

import numpy as np
import pytest

import oracle as O
from test_oracle_mcmc import _class_states


def test_rate_special_cases():
    for p in (0.03, 0.1, 0.2, 0.5):
        r = O.rate_general(p, (1, 1, 1))
        assert abs(r - (p / 3) / (1 - p)) < 1e-15 * max(1.0, r) + 1e-16
    for q in (0.02, 0.1, 0.3):
        p = 2 * q - q * q                    # some flip
        r = O.rate_general(p, (1, 2, 1))
        assert abs(r - q / (1 - q)) < 1e-12
    r = O.rate_general(0.75, (1, 1, 1))
    assert abs(r - 1.0) < 1e-12


def test_energy_histograms_match_the_named_models():
    L = 3
    syn, _ = O.gen_syndromes(5, 0, 1, L, 0.2)
    assert (O.exact_histogram(L, syn[0], 2, (1, 1, 1)) == O.exact_histogram(L, syn[0], 0)).all()
    assert (O.exact_histogram(L, syn[0], 2, (1, 2, 1)) == O.exact_histogram(L, syn[0], 1)).all()


def test_pauli_generator_frequencies():
    """The generator follows its definition (errors rebuilt from the Philox
    words give its syndromes and classes) and the Pauli frequencies match
    (pX, pY, pZ)."""
    L, n, e = 7, 40, (2, 3, 1)
    px, py, pz = O.pauli_probs(0.2, e)
    assert abs(px + py + pz - 0.2) < 1e-12
    syn, tc = O.gen_syndromes_pauli(31, 5, n, L, px, py, pz)
    key = np.array([31, 0x53594E44], np.uint32)
    t1, t2, t3 = (math.floor(px * 2 ** 32), math.floor((px + py) * 2 ** 32), math.floor((px + py + pz) * 2 ** 32))
    cnt = np.zeros(4)
    nq = O.nq(L)
    for i in range(n):
        ex = np.zeros(nq, np.uint8)
        ez = np.zeros(nq, np.uint8)
        for q in range(nq):
            u = int(O.philox(np.array([5 + i, q // 4, 2, 0], np.uint32), key)[q % 4])
            kind = 0 if u < t1 else 1 if u < t2 else 2 if u < t3 else 3
            cnt[kind] += 1
            ex[q] = kind in (0, 1)
            ez[q] = kind in (1, 2)
        assert (O.syndrome(L, ex, ez) == syn[i]).all() and O.class_code(L, ex, ez) == tc[i]
    N = cnt.sum()
    for c, pr in zip(cnt[:3], (px, py, pz)):
        assert abs(c - N * pr) < 5 * math.sqrt(N * pr * (1 - pr)) + 1


def test_general_channel_l2_chi2_random_scan():
    L, p, R, sweeps, e = 2, 0.4, 512, 60, (1, 3, 2)
    r = O.rate_general(p, e)
    E = {(0, 0): 0, (1, 0): e[0], (1, 1): e[1], (0, 1): e[2]}
    syn = np.array([1, 1, 0, 1], np.uint8)
    out = O.run_chains(L, 4, R, p, 777, 0, syn, 0, sweeps, scan=1, noise=2, energy=e)
    for k in range(4):
        states = _class_states(L, syn, k)
        key = {bytes(np.concatenate(s)): i for i, s in enumerate(states)}
        w = np.array([r ** sum(E[(int(x), int(z))] for x, z in zip(fx, fz)) for fx, fz in states])
        w /= w.sum()
        cnt = np.zeros(16)
        for c in range(k * R, (k + 1) * R):
            cnt[key[bytes(np.concatenate([out["frames_x"][c], out["frames_z"][c]]))]] += 1
        ex_ = w * R
        big = ex_ >= 5
        obs = np.append(cnt[big], cnt[~big].sum())
        exp_ = np.append(ex_[big], ex_[~big].sum())
        if exp_[-1] == 0:
            obs, exp_ = obs[:-1], exp_[:-1]
        chi2 = ((obs - exp_) ** 2 / exp_).sum()
        dof = len(obs) - 1
        assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (k, chi2, dof)


@pytest.mark.parametrize("e,p,seed", [((2, 3, 1), 0.15, 41), ((1, 1, 3), 0.25, 42)])
def test_general_channel_mean_matches_enumeration(e, p, seed):
    L, R, sweeps, burn = 3, 48, 200, 40
    px, py, pz = O.pauli_probs(p, e)
    syn, _ = O.gen_syndromes_pauli(seed, 0, 1, L, px, py, pz)
    bb = -math.log(O.rate_general(p, e))
    _, exact = O.exact_class_stats(L, syn[0], bb, noise=2, energy=e)
    out = O.run_chains(L, 4, R, p, 600 + seed, 0, syn[0], 0, sweeps, burn_in=burn, scan=1, noise=2, energy=e)
    per_chain = out["chain_sum"].astype(np.float64) / (O.nstab(L) * (sweeps - burn))
    for k in range(4):
        x = per_chain[k * R:(k + 1) * R]
        se = x.std(ddof=1) / math.sqrt(R)
        assert abs(x.mean() - exact[k]) < 5 * se + 0.03, (k, x.mean(), exact[k], se)
    _, m0 = O.exact_class_stats(L, syn[0], 0.0, noise=2, energy=e)
    assert np.allclose(m0, O.nq(L) * sum(e) / 4.0, atol=1e-9)
    d = O.decode_one(L, p, 4, 4, 20, 3, 0, syn[0], scan=1, noise=2, energy=e)
    Et = {(0, 0): 0, (1, 0): e[0], (1, 1): e[1], (0, 1): e[2]}
    for c in range(16):
        fx, fz = d["frames_x"][c], d["frames_z"][c]
        assert d["chain_n"][c] == sum(Et[(int(x), int(z))] for x, z in zip(fx, fz))
        assert (O.syndrome(L, fx, fz) == syn[0]).all() and O.class_code(L, fx, fz) == c // 4
