"""Qualitative end-to-end pins of the planar decoder under depolarizing noise
(Sec. IV.A, the discussion of Fig. 6): with a budget of at least L^4
proposals per chain,

* below the threshold (p = 0.10) the logical error rate falls with L;
* above it (p = 0.18) it does not fall;
* the distinguishability of the classes, min over the wrong classes of
  <n>_false minus <n>_true, grows with L below the threshold (p = 0.13).

The paper puts the threshold of algorithm C at 15-16 %.  Budget here:
20,000 sweeps of 2L(L-1) proposals each, the first 4,000 annealed from
0.1 beta_bar in 16 stages and not sampled (at least 4 L^4 sampled
proposals per chain up to L = 15), 4 classes x 4 chains, seeded synthetic
syndromes with their true classes.  The start states here are straight
strings, not the paper's matched ones, so the chains need the annealed
burn-in to mix: with the first 800 sweeps annealed from 0.3 beta_bar in 4
stages the error rate at p = 0.10 still rose from L = 11 to 15 (1.16 % to
2.67 %), and with 1,000 of 4,000 from 11 to 15 as well; with this schedule
it falls (2.91 / 0.78 / 0.48 % at L = 7 / 11 / 15)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = (7, 11, 15)
N = 65536
R = 4


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1302_2669_gb300 import build as b
    b.build()
    import paper_1302_2669_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


BURN, SWEEPS, STAGES, BETA0 = 4000, 20000, 16, 0.1


def _run(pkg, ctx, L, p, seed):
    burn, sweeps = BURN, SWEEPS
    assert (sweeps - burn) * 2 * L * (L - 1) >= 4 * L ** 4   # the paper's n_sample = L^4 per chain, four times over
    syn, tc = ctx.gen_syndromes(seed, 0, N, L, p, like=torch.zeros(1, device="cuda"))
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, anneal_stages=STAGES, anneal_beta0=BETA0)
    cls, csum, _ = ctx.decode(syn, L, p, opts, seed=seed + 100)
    torch.cuda.synchronize()
    cls, tc = cls.cpu().numpy(), tc.cpu().numpy().astype(np.int64)
    fails = int((cls != tc).sum())
    ler = fails / N
    sigma = math.sqrt(max(ler * (1 - ler), 1.0 / N) / N)
    samples = 4 * R * (sweeps - burn)                    # samples of n per class
    mean_n = csum.cpu().numpy().astype(np.float64) / samples   # <n>_k
    rows = np.arange(N)
    true = mean_n[rows, tc]
    wrong = mean_n.copy()
    wrong[rows, tc] = np.inf
    dist = float((wrong.min(axis=1) - true).mean())
    return ler, sigma, dist


def test_ler_falls_with_L_below_threshold(pkg, ctx):
    p = 0.10
    r = {L: _run(pkg, ctx, L, p, 6100 + L) for L in SIZES}
    for a, b in zip(SIZES, SIZES[1:]):
        (la, sa, _), (lb, sb, _) = r[a], r[b]
        assert lb + 3 * math.hypot(sa, sb) < la, (p, r)
    assert r[SIZES[-1]][0] < p


def test_ler_does_not_fall_with_L_above_threshold(pkg, ctx):
    p = 0.18
    r = {L: _run(pkg, ctx, L, p, 6200 + L) for L in SIZES}
    for a, b in zip(SIZES, SIZES[1:]):
        (la, sa, _), (lb, sb, _) = r[a], r[b]
        assert lb > la - 3 * math.hypot(sa, sb), (p, r)
    assert r[SIZES[-1]][0] > r[SIZES[0]][0], (p, r)


def test_distinguishability_grows_with_L_below_threshold(pkg, ctx):
    p = 0.13
    r = {L: _run(pkg, ctx, L, p, 6300 + L) for L in SIZES}
    d = [r[L][2] for L in SIZES]
    assert d[0] > 0 and all(b > a for a, b in zip(d, d[1:])), (p, r)
