"""Pins of the oracle's per-chain accept counts (no GPU).  The Metropolis
step of Sec. IV applies a proposal when Delta n <= 0 and otherwise with
probability r^Delta n (Eq. 2): at p = 3/4 (r = 1) every proposal is applied,
so a chain accepts exactly one move per proposal; counts of a run split at
any sweep add up to the whole run's; they never exceed the proposals made."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("L,K,R", [(3, 4, 2), (5, 4, 1), (4, 16, 1)])
def test_every_proposal_accepted_at_r_one(L, K, R):
    sweeps = 7
    if K == 16:
        syn, _ = O.t_gen_syndromes(31, 0, 1, L, 0.2)
        n_stab = O.t_nstab(L)
    else:
        syn, _ = O.gen_syndromes(31, 0, 1, L, 0.2)
        n_stab = O.nstab(L)
    out = O.run_chains(L, K, R, 0.75, 9, 0, syn[0], 0, sweeps, accepts=True)
    assert (out["accepts"] == n_stab * sweeps).all()


@pytest.mark.parametrize("scan", [0, 1])
def test_counts_add_up_over_a_split_run(scan):
    L, K, R, p, T, T1 = 5, 4, 4, 0.12, 40, 13
    syn, _ = O.gen_syndromes(32, 0, 1, L, p)
    whole = O.run_chains(L, K, R, p, 5, 0, syn[0], 0, T, accepts=True, scan=scan)
    a = O.run_chains(L, K, R, p, 5, 0, syn[0], 0, T1, accepts=True, scan=scan)
    b = O.run_chains(L, K, R, p, 5, 0, syn[0], T1, T, frames=(a["frames_x"], a["frames_z"]),
                     chain_sum=a["chain_sum"], accepts=True, scan=scan)
    assert (a["accepts"] + b["accepts"] == whole["accepts"]).all()
    assert (b["frames_x"] == whole["frames_x"]).all() and (b["frames_z"] == whole["frames_z"]).all()


def test_counts_bounded_and_nonzero():
    L, K, R, p, T = 7, 4, 4, 0.1, 30
    syn, _ = O.gen_syndromes(33, 0, 1, L, p)
    out = O.run_chains(L, K, R, p, 6, 0, syn[0], 0, T, accepts=True)
    acc = out["accepts"]
    assert (acc > 0).all() and (acc <= O.nstab(L) * T).all()
