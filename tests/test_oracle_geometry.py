"""Pins of the oracle's code geometry, syndromes, start states and exact
enumeration against what the paper and the algebra fix (no GPU)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
LS = [2, 3, 4, 5, 6, 9, 13]


def _check_matrix(L):
    """Rows: generators as 0/1 vectors over qubits; returns (Hx, Hz)."""
    nq, ns = O.nq(L), O.nstab(L)
    H = np.zeros((ns, nq), np.uint8)
    types = np.zeros(ns, np.int32)
    for g in range(ns):
        H[g, O.stab_support(L, g)] = 1
        types[g] = O.stab_pos(L, g)[0]
    return H[types == 0], H[types == 1]


def _gf2_rank(M):
    M = (np.array(M, np.uint8) & 1).copy()
    rank = 0
    rows, cols = M.shape
    for c in range(cols):
        piv = [r for r in range(rank, rows) if M[r, c]]
        if not piv:
            continue
        M[[rank, piv[0]]] = M[[piv[0], rank]]
        for r in range(rows):
            if r != rank and M[r, c]:
                M[r] ^= M[rank]
        rank += 1
    return rank


@pytest.mark.parametrize("L", LS)
def test_counts(L):
    # Sec. II: n_stab = 2L(L-1); Sec. IV.A: n_qubits = n_stab + 1.
    assert O.nstab(L) == 2 * L * (L - 1)
    assert O.nq(L) == O.nstab(L) + 1


def test_paper_printed_qubit_counts():
    for L, n in GOLD["qubits_for_code_size"].items():
        if L.startswith("_"):
            continue
        assert O.nq(int(L)) == n


@pytest.mark.parametrize("L", LS)
def test_weights_and_boundaries(L):
    Hx, Hz = _check_matrix(L)
    w = np.concatenate([Hx.sum(1), Hz.sum(1)])
    assert set(w.tolist()) <= set(GOLD["n_stab_formula"]["stabilizer_weights"])
    # weight-3 generators sit on the boundary: sigma_x ones on the left/right
    # columns, sigma_z ones on the top/bottom rows, 2(L-1) of each type.
    assert (Hx.sum(1) == 3).sum() == 2 * (L - 1)
    assert (Hz.sum(1) == 3).sum() == 2 * (L - 1)
    # Sec. II: every single-qubit Pauli anticommutes with some generator:
    # each qubit lies in at least one sigma_x and one sigma_z generator.
    assert (Hx.sum(0) >= 1).all() and (Hz.sum(0) >= 1).all()


@pytest.mark.parametrize("L", LS)
def test_commutation_and_rank(L):
    Hx, Hz = _check_matrix(L)
    # Sec. II: all stabilizers commute -> even overlap of every X/Z pair.
    assert ((Hx.astype(np.int64) @ Hz.T.astype(np.int64)) % 2 == 0).all()
    # Sec. IV: each class has 2^{n_stab} members -> generators independent.
    assert _gf2_rank(Hx) == Hx.shape[0] == L * (L - 1)
    assert _gf2_rank(Hz) == Hz.shape[0] == L * (L - 1)


@pytest.mark.parametrize("L", LS)
def test_logicals(L):
    nq = O.nq(L)
    Hx, Hz = _check_matrix(L)
    zero = np.zeros(nq, np.uint8)
    xbar, _ = O.apply_logical(L, 1, zero, zero)
    _, zbar = O.apply_logical(L, 2, zero, zero)
    assert xbar.sum() == L and zbar.sum() == L
    # logicals commute with every generator (no syndrome) ...
    assert O.syndrome(L, xbar, zero).sum() == 0
    assert O.syndrome(L, zero, zbar).sum() == 0
    # ... anticommute with each other ...
    assert int(xbar.astype(int) @ zbar.astype(int)) % 2 == 1
    # ... and are not products of generators.
    assert _gf2_rank(np.vstack([Hx, xbar])) == Hx.shape[0] + 1
    assert _gf2_rank(np.vstack([Hz, zbar])) == Hz.shape[0] + 1
    # class codes: X-bar flips a, Z-bar flips b
    assert O.class_code(L, xbar, zero) == 1
    assert O.class_code(L, zero, zbar) == 2
    assert O.class_code(L, xbar, zbar) == 3


@pytest.mark.parametrize("L", [3, 5, 9])
def test_generators_preserve_syndrome_and_class(L):
    rng = np.random.default_rng(L)
    nq, ns = O.nq(L), O.nstab(L)
    for _ in range(20):
        ex = rng.integers(0, 2, nq).astype(np.uint8)
        ez = rng.integers(0, 2, nq).astype(np.uint8)
        s0, k0 = O.syndrome(L, ex, ez), O.class_code(L, ex, ez)
        g = int(rng.integers(0, ns))
        t = O.stab_pos(L, g)[0]
        q = O.stab_support(L, g)
        ex2, ez2 = ex.copy(), ez.copy()
        if t == 0:
            ex2[q] ^= 1
        else:
            ez2[q] ^= 1
        assert (O.syndrome(L, ex2, ez2) == s0).all()
        assert O.class_code(L, ex2, ez2) == k0


@pytest.mark.parametrize("L", [3, 5])
def test_boundary_absorption(L):
    # Sec. III: s-anyons (violated sigma_x generators) are absorbed by the
    # top/bottom boundaries, p-anyons by the left/right ones.
    nq = O.nq(L)
    zero = np.zeros(nq, np.uint8)
    q_top = (0 * (2 * L - 1) + 2) // 2          # grid (0, 2)
    q_left = (2 * (2 * L - 1) + 0) // 2         # grid (2, 0)
    q_mid = ((2 * (L // 2)) * (2 * L - 1) + 2 * (L // 2)) // 2
    ez = zero.copy(); ez[q_top] = 1
    s = O.syndrome(L, zero, ez)
    assert s.sum() == 1 and O.stab_pos(L, int(np.argmax(s)))[0] == 0
    ex = zero.copy(); ex[q_left] = 1
    s = O.syndrome(L, ex, zero)
    assert s.sum() == 1 and O.stab_pos(L, int(np.argmax(s)))[0] == 1
    ez = zero.copy(); ez[q_mid] = 1
    assert O.syndrome(L, zero, ez).sum() == 2


@pytest.mark.parametrize("L", LS)
def test_colours(L):
    # Sec. V: four groups whose members share no qubit; a sigma_x and a
    # sigma_z move must not share a group either (Delta n of one reads what
    # the other writes), hence X and Z generators get different colours.
    ns = O.nstab(L)
    members = []
    for col in range(4):
        cnt = O.colour_count(L, col)
        assert cnt == L * (L - 1) // 2
        ms = [O.colour_member(L, col, m) for m in range(cnt)]
        assert all(O.stab_colour(L, g) == col for g in ms)
        assert all(O.stab_pos(L, g)[0] == col // 2 for g in ms)
        seen = np.zeros(O.nq(L), np.int32)
        for g in ms:
            seen[O.stab_support(L, g)] += 1
        assert seen.max() <= 1
        members += ms
    assert sorted(members) == list(range(ns))


@pytest.mark.parametrize("L", [2, 3])
def test_pure_error_all_syndromes(L):
    ns = O.nstab(L)
    for bits in itertools.product([0, 1], repeat=ns):
        syn = np.array(bits, np.uint8)
        ex, ez = O.pure_error(L, syn)
        assert (O.syndrome(L, ex, ez) == syn).all()
        for k in range(4):
            fx, fz, _ = O.start_frame(L, syn, k)
            assert O.class_code(L, fx, fz) == k
            assert (O.syndrome(L, fx, fz) == syn).all()


@pytest.mark.parametrize("L", [5, 9, 13, 25])
def test_pure_error_random_and_distance(L):
    rng = np.random.default_rng(100 + L)
    ns = O.nstab(L)
    for _ in range(10):
        syn = (rng.random(ns) < 0.1).astype(np.uint8)
        ex, ez = O.pure_error(L, syn)
        assert (O.syndrome(L, ex, ez) == syn).all()
    # a single anyon is joined to its nearer absorbing boundary:
    # weight = distance to that boundary (Sec. III, Manhattan distance)
    for g in range(ns):
        syn = np.zeros(ns, np.uint8)
        syn[g] = 1
        t, r, c = O.stab_pos(L, g)
        ex, ez = O.pure_error(L, syn)
        if t == 1:
            d = min((c + 1) // 2, L - (c + 1) // 2)
            assert ex.sum() == d and ez.sum() == 0
        else:
            d = min((r + 1) // 2, L - (r + 1) // 2)
            assert ez.sum() == d and ex.sum() == 0


@pytest.mark.parametrize("L", [2, 3])
def test_enumeration_covers_all_paulis(L):
    """Eq. 3's sums over classes partition the Pauli group: summed over every
    syndrome and class, the weight histogram of the enumerated frames must be
    the number of n-qubit Pauli errors, C(nq, n) 3^n."""
    nq, ns = O.nq(L), O.nstab(L)
    total = np.zeros(nq + 1, np.float64)
    for s in range(1 << ns):
        syn = np.array([(s >> g) & 1 for g in range(ns)], np.uint8)
        h = O.exact_histogram(L, syn)
        assert (h.sum(1) == 2 ** ns).all()
        total += h.sum(0)
    expect = np.array([math.comb(nq, n) * 3 ** n for n in range(nq + 1)], np.float64)
    assert (total == expect).all()


def test_enumeration_l4_class_sizes():
    L = 4
    rng = np.random.default_rng(4)
    syn = (rng.random(O.nstab(L)) < 0.2).astype(np.uint8)
    h = O.exact_histogram(L, syn)
    assert (h.sum(1) == 2 ** O.nstab(L)).all()
    # the start frame of each class is one of the enumerated frames
    for k in range(4):
        fx, fz, _ = O.start_frame(L, syn, k)
        assert h[k, int((fx | fz).sum())] >= 1
