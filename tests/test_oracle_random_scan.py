"""Pins of the oracle's random-scan chains (Sec. IV as written: one generator
drawn at random per step, f(n) summed after every step).  Random-scan
Metropolis has the same stationary distribution as the colour sweeps, so the
same exact pins apply: chi^2 over all states at L = 2, exact <n> by
enumeration at L = 3, the beta -> infinity limit, class and syndrome
invariance, resumability, and the step/sample counts."""
import math

import numpy as np
import pytest

import oracle as O
from test_oracle_mcmc import _class_states


def test_l2_state_distribution_chi2_random_scan():
    L, p, R, sweeps = 2, 0.4, 512, 60
    r = (p / 3) / (1 - p)
    syn = np.array([1, 0, 0, 1], np.uint8)
    out = O.run_chains(L, 4, R, p, 2024, 0, syn, 0, sweeps, scan=1)
    for k in range(4):
        states = _class_states(L, syn, k)
        key = {bytes(np.concatenate(s)): i for i, s in enumerate(states)}
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


@pytest.mark.parametrize("L,p,seed", [(3, 0.15, 15), (3, 0.25, 16)])
def test_mean_n_matches_enumeration_random_scan(L, p, seed):
    R, sweeps, burn = 48, 300, 50
    syn, _ = O.gen_syndromes(seed, 0, 1, L, p)
    syn = syn[0]
    _, bb = O.thresholds(p)
    _, exact = O.exact_class_stats(L, syn, bb)
    out = O.run_chains(L, 4, R, p, 555 + seed, 0, syn, 0, sweeps, burn_in=burn, scan=1)
    per_chain = out["chain_sum"].astype(np.float64) / (O.nstab(L) * (sweeps - burn))
    for k in range(4):
        x = per_chain[k * R:(k + 1) * R]
        se = x.std(ddof=1) / math.sqrt(R)
        assert abs(x.mean() - exact[k]) < 5 * se + 0.02, (k, x.mean(), exact[k], se)


def test_one_proposal_per_step():
    """p = 3/4 gives r = 1: every proposal is accepted, so the accept count
    is exactly n_stab per sweep, and n is sampled n_stab times per sweep."""
    L, sweeps = 4, 7
    syn, _ = O.gen_syndromes(5, 0, 1, L, 0.3)
    out = O.run_chains(L, 4, 2, 0.75, 1, 0, syn[0], 0, sweeps, accepts=True, scan=1)
    assert (out["accepts"] == O.nstab(L) * sweeps).all()
    d = O.decode_one(L, 0.2, 4, 2, 9, 3, 0, syn[0], burn_in=4, scan=1)
    samples = O.nstab(L) * 2 * (9 - 4)
    k = int(np.argmin(d["class_sum"]))
    _, bb = O.thresholds(0.2)
    want = -bb * (d["class_sum"][1] / samples - d["class_sum"][k] / samples)
    assert d["cls"] == k and abs(d["log_ratio"][1] - want) < 1e-12


def test_zero_temperature_never_increases_random_scan():
    L = 5
    syn, _ = O.gen_syndromes(11, 0, 3, L, 0.15)
    for i in range(3):
        out = O.run_chains(L, 4, 1, 0.15, 5, i, syn[i], 0, 30, beta_scale=float("inf"), trace=True, scan=1)
        tr = out["trace"][:30]
        assert (np.diff(tr) <= 0).all()


def test_random_scan_keeps_syndrome_and_class_and_resumes():
    L, p, K, R, T, T1 = 5, 0.15, 4, 2, 20, 7
    syn, _ = O.gen_syndromes(1001, 0, 1, L, p)
    d = O.decode_one(L, p, K, R, T, 31, 0, syn[0], scan=1)
    for c in range(K * R):
        fx, fz = d["frames_x"][c], d["frames_z"][c]
        assert (O.syndrome(L, fx, fz) == syn[0]).all()
        assert O.class_code(L, fx, fz) == c // R
        assert d["chain_n"][c] == int((fx | fz).sum())
    full = O.run_chains(L, K, R, p, 31, 0, syn[0], 0, T, scan=1)
    a = O.run_chains(L, K, R, p, 31, 0, syn[0], 0, T1, scan=1)
    b = O.run_chains(L, K, R, p, 31, 0, syn[0], T1, T, frames=(a["frames_x"], a["frames_z"]),
                     chain_sum=a["chain_sum"], scan=1)
    assert (b["chain_sum"] == full["chain_sum"]).all()
    assert (b["frames_x"] == full["frames_x"]).all() and (b["frames_z"] == full["frames_z"]).all()
    assert (full["chain_sum"] == d["chain_sum"]).all()
