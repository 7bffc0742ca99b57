"""Pins of the oracle's toric code (the 16-class variant): geometry counts and
weights, commutation, GF(2) ranks (two encoded qubits), the logical algebra
and the 16 class codes, pure errors, colour disjointness, and the chains
against exact Boltzmann weights and exact <n> by enumeration on the 2 x 2
torus."""
import itertools
import math

import numpy as np
import pytest

import oracle as O


def _support_matrix(L):
    nq, ns = O.t_nq(L), O.t_nstab(L)
    M = np.zeros((ns, nq), np.uint8)
    for g in range(ns):
        M[g, O.t_stab_support(L, g)] = 1
    return M


def _gf2_rank(M):
    M = M.copy() % 2
    r = 0
    for c in range(M.shape[1]):
        piv = [i for i in range(r, M.shape[0]) if M[i, c]]
        if not piv:
            continue
        M[[r, piv[0]]] = M[[piv[0], r]]
        for i in range(M.shape[0]):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
    return r


@pytest.mark.parametrize("L", [2, 4, 6])
def test_toric_counts_weights_and_ranks(L):
    M = _support_matrix(L)
    assert M.shape == (2 * L * L, 2 * L * L)
    assert (M.sum(1) == 4).all()
    half = L * L
    assert (M[:half].sum(0) == 2).all() and (M[half:].sum(0) == 2).all()   # each qubit: 2 stars, 2 plaquettes
    assert ((M[:half].astype(int) @ M[half:].T.astype(int)) % 2 == 0).all()  # stars commute with plaquettes
    rs, rp = _gf2_rank(M[:half]), _gf2_rank(M[half:])
    assert rs == half - 1 and rp == half - 1
    assert O.t_nq(L) - (rs + rp) == 2          # sigma_x and sigma_z parts: two encoded qubits


@pytest.mark.parametrize("L", [2, 4])
def test_toric_logicals_and_class_codes(L):
    nq = O.t_nq(L)
    z = np.zeros(nq, np.uint8)
    ops = {}
    for k in (1, 2, 4, 8):
        ex, ez = O.t_apply_logical(L, k, z, z)
        assert (O.t_syndrome(L, ex, ez) == 0).all()           # commutes with every generator
        assert O.t_class_code(L, ex, ez) == k                  # and is not a stabilizer
        ops[k] = (ex, ez)
    # symplectic products: X1-Z1 and X2-Z2 anticommute, other pairs commute
    def sp(a, b):
        return int((a[0] & b[1]).sum() + (a[1] & b[0]).sum()) & 1
    assert sp(ops[1], ops[4]) == 1 and sp(ops[2], ops[8]) == 1
    for a, b in [(1, 2), (1, 8), (2, 4), (4, 8)]:
        assert sp(ops[a], ops[b]) == 0
    rng = np.random.default_rng(L)
    for _ in range(20):
        ex = rng.integers(0, 2, nq).astype(np.uint8)
        ez = rng.integers(0, 2, nq).astype(np.uint8)
        code = O.t_class_code(L, ex, ez)
        for g in rng.choice(O.t_nstab(L), size=5):
            t, _, _ = O.t_stab_pos(L, int(g))
            q = O.t_stab_support(L, int(g))
            fx, fz = ex.copy(), ez.copy()
            (fx if t == 0 else fz)[q] ^= 1
            assert O.t_class_code(L, fx, fz) == code
        k = int(rng.integers(16))
        fx, fz = O.t_apply_logical(L, k, ex, ez)
        assert O.t_class_code(L, fx, fz) == code ^ k


@pytest.mark.parametrize("L", [2, 4, 6])
def test_toric_pure_error_and_colours(L):
    syn, _ = O.t_gen_syndromes(9, 0, 30, L, 0.2)
    for s in syn:
        ex, ez = O.t_pure_error(L, s)
        assert (O.t_syndrome(L, ex, ez) == s).all()
        for k in (0, 5, 15):
            fx, fz, c0 = O.t_start_frame(L, s, k)
            assert (O.t_syndrome(L, fx, fz) == s).all() and O.t_class_code(L, fx, fz) == k
    for col in range(4):
        gs = [g for g in range(O.t_nstab(L)) if O.t_stab_colour(L, g) == col]
        assert len(gs) == L * L // 2
        seen = set()
        for g in gs:
            q = set(O.t_stab_support(L, g).tolist())
            assert not (q & seen)
            seen |= q


def _torus_states(L, syn, k):
    ns = O.t_nstab(L)
    fx0, fz0, _ = O.t_start_frame(L, syn, k)
    states = {}
    for bits in itertools.product([0, 1], repeat=ns):
        fx, fz = fx0.copy(), fz0.copy()
        for g, b in enumerate(bits):
            if b:
                t, _, _ = O.t_stab_pos(L, g)
                (fx if t == 0 else fz)[O.t_stab_support(L, g)] ^= 1
        states[bytes(np.concatenate([fx, fz]))] = int((fx | fz).sum())
    return states


def test_toric_l2_chi2_and_enumeration():
    """Random-scan chains on the 2 x 2 torus: final states against the exact
    weights and time averages against the exact <n> of all 16 classes.  (The
    fixed colour order is not used here: on 8 qubits it can trap a chain in a
    cycle of always-accepted Delta n = 0 moves; it is pinned on the 4 x 4
    torus below.)"""
    L, p, R, sweeps = 2, 0.3, 256, 40
    r = (p / 3) / (1 - p)
    syn, _ = O.t_gen_syndromes(21, 0, 1, L, p)
    syn = syn[0]
    out = O.run_chains(L, 16, R, p, 55, 0, syn, 0, sweeps, scan=1)
    for k in (0, 3, 9, 15):
        states = _torus_states(L, syn, k)
        assert len(states) == 64                    # 2^(n_stab - 2) distinct frames per class
        keys = list(states)
        w = np.array([r ** states[s] for s in keys])
        w /= w.sum()
        idx = {s: i for i, s in enumerate(keys)}
        cnt = np.zeros(len(keys))
        for c in range(k * R, (k + 1) * R):
            cnt[idx[bytes(np.concatenate([out["frames_x"][c], out["frames_z"][c]]))]] += 1
        e = w * R
        big = e >= 5
        obs = np.append(cnt[big], cnt[~big].sum())
        exp_ = np.append(e[big], e[~big].sum())
        chi2 = ((obs - exp_) ** 2 / exp_).sum()
        dof = len(obs) - 1
        assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (k, chi2, dof)
    # exact <n> per class from the enumeration against chain averages
    h = O.t_exact_histogram(L, syn).astype(np.float64)
    n = np.arange(h.shape[1])
    exact = (h * n * r ** n).sum(1) / (h * r ** n).sum(1)
    for scan, per_sweep in ((1, O.t_nstab(L)),):
        out = O.run_chains(L, 16, 24, p, 56, 0, syn, 0, 300, burn_in=40, scan=scan)
        per_chain = out["chain_sum"].astype(np.float64) / (per_sweep * 260)
        for k in range(16):
            x = per_chain[k * 24:(k + 1) * 24]
            se = x.std(ddof=1) / math.sqrt(24)
            assert abs(x.mean() - exact[k]) < 5 * se + 0.03, (scan, k, x.mean(), exact[k])
    d = O.decode_one(L, p, 16, 2, 20, 3, 0, syn)
    for c in range(32):
        fx, fz = d["frames_x"][c], d["frames_z"][c]
        assert (O.t_syndrome(L, fx, fz) == syn).all() and O.t_class_code(L, fx, fz) == c // 2


def test_toric_colour_sweeps_agree_with_random_scan_at_l4():
    """On the 4 x 4 torus the colour-sweep chains and the (exactly pinned)
    random-scan chains have the same class means."""
    L, p, R = 4, 0.2, 32
    syn, _ = O.t_gen_syndromes(23, 0, 2, L, p)
    for s in syn:
        a = O.run_chains(L, 16, R, p, 61, 0, s, 0, 240, burn_in=40)
        b = O.run_chains(L, 16, R, p, 62, 0, s, 0, 240, burn_in=40, scan=1)
        ma = a["chain_sum"].astype(np.float64) / (4 * 200)
        mb = b["chain_sum"].astype(np.float64) / (O.t_nstab(L) * 200)
        for k in range(16):
            xa, xb = ma[k * R:(k + 1) * R], mb[k * R:(k + 1) * R]
            se = math.sqrt(xa.var(ddof=1) / R + xb.var(ddof=1) / R)
            assert abs(xa.mean() - xb.mean()) < 5 * se + 0.05, (k, xa.mean(), xb.mean(), se)
