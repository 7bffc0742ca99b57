"""Detailed balance of the oracle's random-scan chain (Sec. IV: each step
draws one generator at random and applies it with the Metropolis
probability min(1, r^Delta n)).  Every step is reversible with respect to
the weights r^n of Eq. 4, so a sweep of n_stab steps is too: at stationarity
the pair (state before, state after) of a sweep is exchangeable, and the
number of sweeps s -> s' matches the number s' -> s for every pair of states.
At L = 2 (16 states per class) 4 x 512 chains are burnt in and then run
sweep by sweep (resumed from their frames); the transition counts of every
pair are tested for symmetry.  The stationary weights themselves are checked
in test_oracle_mcmc.py (chi^2 of the L = 2 states).

A chain that breaks reversibility (a Metropolis ratio inverted for one move
type, say) is stationary for no Boltzmann law, and it either moves the
occupancy off the exact weights or shows up here as a net circulation
between states."""
import itertools
import math

import numpy as np

import oracle as O


def _class_index(L, syn, k):
    ns = O.nstab(L)
    fx0, fz0, _ = O.start_frame(L, syn, k)
    sup = [(O.stab_pos(L, g)[0], O.stab_support(L, g)) for g in range(ns)]
    key = {}
    for i, bits in enumerate(itertools.product([0, 1], repeat=ns)):
        fx, fz = fx0.copy(), fz0.copy()
        for g, b in enumerate(bits):
            if b:
                t, q = sup[g]
                if t == 0:
                    fx[q] ^= 1
                else:
                    fz[q] ^= 1
        key[bytes(np.concatenate([fx, fz]))] = i
    assert len(key) == 2 ** ns
    return key


def _states(out, keys, R):
    s = np.empty(len(out["frames_x"]), np.int64)
    for c in range(len(s)):
        s[c] = keys[c // R][bytes(np.concatenate([out["frames_x"][c], out["frames_z"][c]]))]
    return s


def _symmetry_chi2(scan):
    """chi^2 of the sweep-to-sweep transition counts against symmetry, the
    number of state pairs tested and the number of moves seen."""
    L, p, K, R, burn, T = 2, 0.35, 4, 512, 16, 48
    syn = np.array([0, 1, 1, 0], np.uint8)
    keys = [_class_index(L, syn, k) for k in range(K)]
    out = O.run_chains(L, K, R, p, 4242, 0, syn, 0, burn, scan=scan)
    prev = _states(out, keys, R)
    counts = np.zeros((K, 16, 16), np.int64)
    for t in range(burn, burn + T):
        out = O.run_chains(L, K, R, p, 4242, 0, syn, t, t + 1, frames=(out["frames_x"], out["frames_z"]), scan=scan)
        cur = _states(out, keys, R)
        for c in range(K * R):
            counts[c // R, prev[c], cur[c]] += 1
        prev = cur
    chi2, dof, moved = 0.0, 0, 0
    for k in range(K):
        for i in range(16):
            for j in range(i + 1, 16):
                a, b = counts[k, i, j], counts[k, j, i]
                moved += a + b
                if a + b >= 10:
                    chi2 += (a - b) ** 2 / (a + b)
                    dof += 1
    return chi2, dof, moved / (K * R * T)


def test_random_scan_sweep_transitions_are_symmetric():
    chi2, dof, moved = _symmetry_chi2(scan=1)
    assert moved > 0.2 and dof >= 20   # the chains do move between many pairs
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (chi2, dof)


def test_colour_sweep_is_not_reversible():
    """The colour sweep applies the four colours in a fixed order: each
    colour's update is reversible and keeps the Boltzmann law, their product
    keeps it too (test_oracle_mcmc.py) but is not reversible.  The symmetry
    statistic sees that circulation: it can tell a reversible chain from one
    that only keeps its law."""
    chi2, dof, _ = _symmetry_chi2(scan=0)
    assert chi2 > 10 * (dof + 6 * math.sqrt(2 * dof) + 10), (chi2, dof)
