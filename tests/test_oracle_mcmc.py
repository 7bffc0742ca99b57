"""Statistical and exact pins of the oracle's Metropolis chains (no GPU).

The chains must sample Eq. 4's Boltzmann distribution within each class:
checked by a chi^2 test on every state at L=2, by exact enumeration of
<n>_{beta,k} at L=3 and L=4, by the beta -> 0 and beta -> infinity limits of
Sec. IV.A, and by the minimal example of Fig. 4.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


@pytest.mark.parametrize("p,d", [(0.15, 1), (0.3, 2), (0.5, 1), (0.5, 3)])
def test_acceptance_frequency(p, d):
    """P(accept | Delta n = d) = T[d] / 2^32 = r^d (Sec. IV, Eq. 2)."""
    T, _ = O.thresholds(p)
    Cn, N = 16, 0
    acc = 0
    for t in range(1500):
        for c in range(Cn):
            acc += O.chain_uniform_less(77, 3, t, 2, 5, c, Cn, int(T[d]))
            N += 1
    q = int(T[d]) / 2 ** 32
    sd = math.sqrt(N * q * (1 - q))
    assert abs(acc - N * q) < 5 * sd


def _class_states(L, syn, k):
    """All 2^{n_stab} frames of class k (start frame times generator products)."""
    ns, nq = O.nstab(L), O.nq(L)
    fx0, fz0, _ = O.start_frame(L, syn, k)
    sup = [(O.stab_pos(L, g)[0], O.stab_support(L, g)) for g in range(ns)]
    states = []
    for bits in itertools.product([0, 1], repeat=ns):
        fx, fz = fx0.copy(), fz0.copy()
        for g, b in enumerate(bits):
            if b:
                t, q = sup[g]
                if t == 0:
                    fx[q] ^= 1
                else:
                    fz[q] ^= 1
        states.append((fx, fz))
    return states


def test_l2_state_distribution_chi2():
    """L=2: final states of 512 independent chains per class against the
    exact Boltzmann weights e^{-beta n} of all 16 states of the class."""
    L, p, R, sweeps = 2, 0.4, 512, 48
    r = (p / 3) / (1 - p)
    syn = np.array([1, 0, 0, 1], np.uint8)
    out = O.run_chains(L, 4, R, p, 12345, 0, syn, 0, sweeps)
    for k in range(4):
        states = _class_states(L, syn, k)
        key = {bytes(np.concatenate(s)): i for i, s in enumerate(states)}
        assert len(key) == 16
        w = np.array([r ** int((fx | fz).sum()) for fx, fz in states])
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
        assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (k, chi2, dof)


@pytest.mark.parametrize("L,p,seed", [(3, 0.15, 5), (3, 0.25, 6), (4, 0.12, 7)])
def test_mean_n_matches_enumeration(L, p, seed):
    """<n>_{beta_bar,k} of Eq. 4 by exact enumeration of all 2^{n_stab}
    frames per class, against chain averages (independent replicas)."""
    R, sweeps, burn = 48, 300, 50
    syn, _ = O.gen_syndromes(seed, 0, 1, L, p)
    syn = syn[0]
    _, bb = O.thresholds(p)
    _, exact = O.exact_class_stats(L, syn, bb)
    out = O.run_chains(L, 4, R, p, 777 + seed, 0, syn, 0, sweeps, burn_in=burn)
    per_chain = out["chain_sum"].astype(np.float64) / (4 * (sweeps - burn))
    for k in range(4):
        x = per_chain[k * R:(k + 1) * R]
        se = x.std(ddof=1) / math.sqrt(R)
        assert abs(x.mean() - exact[k]) < 5 * se + 0.02, (k, x.mean(), exact[k], se)


def test_infinite_temperature_mean():
    """Sec. IV.A: as beta -> 0 every qubit carries I, X, Y, Z with probability
    1/4, so <n> -> 3/4 n_qubits.  Exact at beta = 0 for the enumeration; the
    chains are checked at a small positive beta (at beta = 0 exactly every
    proposal is accepted and a fixed-order sweep is deterministic, so the
    limit is taken from above)."""
    L = 3
    syn, _ = O.gen_syndromes(3, 0, 1, L, 0.2)
    target = GOLD["infinite_temperature_mean"]["fraction"] * O.nq(L)
    _, exact0 = O.exact_class_stats(L, syn[0], 0.0)
    assert np.allclose(exact0, target, rtol=0, atol=1e-12)
    p, scale, R, sweeps, burn = 0.15, 0.02, 64, 200, 20
    _, bb = O.thresholds(p)
    _, exact = O.exact_class_stats(L, syn[0], scale * bb)
    out = O.run_chains(L, 4, R, p, 99, 0, syn[0], 0, sweeps, burn_in=burn, beta_scale=scale)
    per_chain = out["chain_sum"].astype(np.float64) / (4 * (sweeps - burn))
    for k in range(4):
        x = per_chain[k * R:(k + 1) * R]
        se = x.std(ddof=1) / math.sqrt(R)
        assert abs(x.mean() - exact[k]) < 5 * se + 0.01
        assert abs(x.mean() - target) < 0.05 * target


def test_zero_temperature_never_increases():
    """Sec. IV.A: for beta* -> infinity n never increases."""
    L = 5
    syn, _ = O.gen_syndromes(11, 0, 4, L, 0.15)
    for i in range(4):
        out = O.run_chains(L, 4, 1, 0.15, 5, i, syn[i], 0, 30, beta_scale=float("inf"), trace=True)
        tr = out["trace"]
        assert (np.diff(tr) <= 0).all()


def test_minimal_example_fig4():
    """Fig. 4: a weight-3 configuration (Z on one qubit, X on two) turns into
    the weight-2 one (Y, X) by one sigma_x stabilizer; the zero-temperature
    chain finds it."""
    L = 5
    nq = O.nq(L)
    q = lambda r, c: (r * (2 * L - 1) + c) // 2
    fx = np.zeros(nq, np.uint8)
    fz = np.zeros(nq, np.uint8)
    fz[q(2, 4)] = 1
    fx[q(3, 3)] = 1
    fx[q(3, 5)] = 1
    assert int((fx | fz).sum()) == GOLD["minimal_example_weights"]["a"]
    syn = O.syndrome(L, fx, fz)
    frames = (np.tile(fx, (4, 1)), np.tile(fz, (4, 1)))
    out = O.run_chains(L, 4, 1, 0.1, 1, 0, syn, 0, 3, beta_scale=float("inf"), frames=frames, trace=True)
    tr = out["trace"]
    assert tr[0] == 3 and tr[1] == GOLD["minimal_example_weights"]["b"]
    gx, gz = out["frames_x"][0], out["frames_z"][0]
    assert gx[q(2, 4)] == 1 and gz[q(2, 4)] == 1          # the Y
    assert gx[q(4, 4)] == 1 and int((gx | gz).sum()) == 2
    assert (O.syndrome(L, gx, gz) == syn).all()


def test_chains_keep_syndrome_and_class():
    """Sec. IV: moves by stabilizers keep every chain in its class and
    compatible with the syndrome."""
    L, p, K, R = 5, 0.15, 4, 4
    syn, _ = O.gen_syndromes(1001, 0, 6, L, p)
    for i in range(6):
        d = O.decode_one(L, p, K, R, 40, 1101, i, syn[i])
        for c in range(K * R):
            fx, fz = d["frames_x"][c], d["frames_z"][c]
            assert (O.syndrome(L, fx, fz) == syn[i]).all()
            assert O.class_code(L, fx, fz) == c // R
            assert d["chain_n"][c] == int((fx | fz).sum())


def test_decide_rule():
    # argmin of the class sums, lowest class on ties (Sec. IV.A)
    K, R = 4, 2
    k, S, lr = O.decide(K, R, 10, 0, 1.5, np.array([5, 5, 3, 3, 2, 4, 9, 0], np.uint64))
    assert list(S) == [10, 6, 6, 9] and k == 1
    assert lr[1] == 0.0 and lr[2] == 0.0
    assert abs(lr[0] - (-1.5 * (10 - 6) / (4 * R * 10))) < 1e-15
    k, _, _ = O.decide(K, R, 10, 0, 1.5, np.zeros(8, np.uint64))
    assert k == 0


def test_resume_equals_uninterrupted():
    """The counter-based randomness is indexed by the sweep, so T1 sweeps
    followed by T - T1 sweeps equal T sweeps."""
    L, p, K, R, T, T1 = 5, 0.15, 4, 4, 30, 11
    syn, _ = O.gen_syndromes(1001, 0, 1, L, p)
    full = O.run_chains(L, K, R, p, 9, 0, syn[0], 0, T)
    a = O.run_chains(L, K, R, p, 9, 0, syn[0], 0, T1)
    b = O.run_chains(L, K, R, p, 9, 0, syn[0], T1, T, frames=(a["frames_x"], a["frames_z"]),
                     chain_sum=a["chain_sum"])
    assert (b["chain_sum"] == full["chain_sum"]).all()
    assert (b["frames_x"] == full["frames_x"]).all() and (b["frames_z"] == full["frames_z"]).all()


def test_decoder_below_p_at_l7():
    """Sec. IV.A: at p = 13% a code with L >= 6 brings the logical error rate
    below p.  The chains start from straight strings rather than from enhanced
    MWPM, so they get a longer run with a quarter of it as burn-in."""
    L, p, K, R, sweeps, burn = 7, 0.13, 4, 4, 3000, 750
    n = 240
    syn, tc = O.gen_syndromes(4242, 0, n, L, p)
    res = O.decode_batch(L, p, K, R, sweeps, 4343, range(n), syn, burn_in=burn)
    fails = sum(d["cls"] != t for d, t in zip(res, tc))
    assert fails / n < p


def test_anneal_stages_partition_the_burn_in():
    for B, S in [(800, 4), (7, 3), (5, 5), (1000, 7)]:
        stages = [O.anneal_stage(t, B, S) for t in range(B)]
        assert stages[0] == 0 and stages[-1] == S - 1
        assert all(b - a in (0, 1) for a, b in zip(stages, stages[1:]))
        assert O.anneal_stage(B, B, S) == -1
    assert O.anneal_scale(1.0, 0.3, 0, 4) == 0.3
    assert abs(O.anneal_scale(2.0, 0.3, 2, 4) - 2.0 * (0.3 + 0.7 * 0.5)) < 1e-15


def test_annealed_run_is_the_composition_of_fixed_temperature_runs():
    """The annealed burn-in is nothing but fixed-beta Metropolis runs (each
    pinned above) chained through their states, sweep index continuing."""
    L, p, K, R, S, B, T, a0 = 5, 0.12, 4, 4, 4, 18, 30, 0.3
    syn, _ = O.gen_syndromes(31, 0, 1, L, p)
    full = O.run_chains(L, K, R, p, 3, 0, syn[0], 0, T, burn_in=B, anneal_stages=S, anneal_beta0=a0)
    fr, cs = None, None
    bounds = [j * B // S for j in range(S + 1)]
    for j in range(S):
        o = O.run_chains(L, K, R, p, 3, 0, syn[0], bounds[j], bounds[j + 1], burn_in=bounds[j + 1],
                         beta_scale=O.anneal_scale(1.0, a0, j, S), frames=fr, chain_sum=cs)
        fr, cs = (o["frames_x"], o["frames_z"]), o["chain_sum"]
    o = O.run_chains(L, K, R, p, 3, 0, syn[0], B, T, burn_in=B, frames=fr, chain_sum=cs)
    assert (o["chain_sum"] == full["chain_sum"]).all()
    assert (o["frames_x"] == full["frames_x"]).all() and (o["frames_z"] == full["frames_z"]).all()
    assert (cs == 0).all()


def test_annealed_start_lowers_the_logical_error_rate():
    """Starting near low-energy configurations (Sec. IV) matters: the same
    sweep budget with the burn-in annealed from 0.3 beta_bar decodes better
    than with a burn-in at beta_bar, and stays below p at L=7, p=13%."""
    L, p, K, R, sweeps, burn = 7, 0.13, 4, 4, 600, 200
    n = 240
    syn, tc = O.gen_syndromes(4242, 0, n, L, p)
    plain = O.decode_batch(L, p, K, R, sweeps, 4343, range(n), syn, burn_in=burn)
    ann = O.decode_batch(L, p, K, R, sweeps, 4343, range(n), syn, burn_in=burn, anneal_stages=4, anneal_beta0=0.3)
    f_plain = sum(d["cls"] != t for d, t in zip(plain, tc)) / n
    f_ann = sum(d["cls"] != t for d, t in zip(ann, tc)) / n
    assert f_ann < p and f_ann < f_plain
