"""GPU parity of the per-chain accept counts against the oracle, bit for bit.
The Metropolis step of Sec. IV either applies a proposed generator or not;
the oracle counts the applied ones of every chain while it runs the chains,
and the CUDA path reports the same counts: colour sweeps at every plane
width and several lane splits (including counters flushed many times and the
straggler queue of undecided proposals), annealed burn-in, random scan,
independent flips, the general channel, the toric code, resumption and host
buffers."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def _np(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


# (L, p, chains per class, sweeps, burn-in, options); the oracle takes the
# same options except the lane split, which does not change results (counting
# runs the colour sweeps with 32 lanes per bundle whatever the split asked).
CASES = [
    (5, 0.15, 4, 150, 0, {}),                                  # G = 16, two syndromes per bundle;
                                                               # > 255 increments per lane: flushes
    (5, 0.15, 1, 60, 0, {}),                                   # G = 4, eight syndromes per bundle
    (7, 0.05, 16, 40, 0, {}),                                  # low p: long digit comparisons, queue
    (9, 0.13, 16, 30, 5, dict(lanes_per_bundle=2)),            # counting runs 32 lanes per bundle
    (9, 0.13, 16, 30, 5, {}),
    (13, 0.10, 16, 12, 6, dict(anneal_stages=2, anneal_beta0=0.3)),
    (6, 0.10, 4, 20, 4, dict(scan=1)),
    (5, 0.09, 4, 20, 4, dict(noise=1, beta_scale=0.85)),
    (5, 0.10, 4, 14, 4, dict(noise=2, scan=1, pauli_energy=(2, 3, 1))),
]


@pytest.mark.parametrize("L,p,R,sweeps,burn,kw", CASES)
def test_accepts_match_oracle(ctx, pkg, L, p, R, sweeps, burn, kw):
    n = 10
    noise = kw.get("noise", 0)
    if noise == 2:
        syn, _ = O.gen_syndromes_pauli(5200 + L, 0, n, L, 0.03, 0.02, 0.04)
    else:
        syn, _ = O.gen_syndromes(5200 + L, 0, n, L, p, noise=noise)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, **kw)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=71, id0=4, accepts=True)
    torch.cuda.synchronize()
    okw = {k: v for k, v in kw.items() if k in ("anneal_stages", "anneal_beta0", "scan", "noise", "beta_scale")}
    if noise == 2:
        okw["energy"] = kw["pauli_energy"]
    acc = _np(out["accepts"])
    total = 0
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 71, 4 + i, syn[i], burn_in=burn, accepts=True, **okw)
        assert (acc[i] == ref["accepts"]).all(), i
        assert (_np(out["chain_sum"])[i] == ref["chain_sum"]).all()
        total += int(ref["accepts"].sum())
    assert total > 0


def test_accepts_toric(ctx, pkg):
    L, p, R, sweeps, burn, n = 4, 0.1, 2, 16, 4, 6
    syn, _ = O.t_gen_syndromes(8300, 0, n, L, p)
    opts = pkg.Opts(n_classes=16, chains_per_class=R, n_sweeps=sweeps, burn_in=burn)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=95, id0=1, accepts=True)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 16, R, sweeps, 95, 1 + i, syn[i], burn_in=burn, accepts=True)
        assert (_np(out["accepts"])[i] == ref["accepts"]).all()


def test_accepts_resume_and_host_buffers(ctx, pkg):
    """Counts of a run split at sweep T1 add up to the whole run's; host
    buffers give the same counts as device buffers; asking for the counts
    changes no other output."""
    L, p, R, T, T1, n = 7, 0.12, 8, 30, 11, 9
    syn, _ = O.gen_syndromes(5300, 0, n, L, p)
    dsyn = torch.from_numpy(syn).cuda()
    mk = lambda t: pkg.Opts(chains_per_class=R, n_sweeps=t, burn_in=3)
    full = ctx.decode_ex(dsyn, L, p, mk(T), seed=12, accepts=True)
    plain = ctx.decode_ex(dsyn, L, p, mk(T), seed=12)
    a = ctx.decode_ex(dsyn, L, p, mk(T1), seed=12, accepts=True)
    b = ctx.decode_ex(dsyn, L, p, mk(T), seed=12, sweep_begin=T1, init_frames=a["chain_frames"],
                      init_chain_sum=a["chain_sum"], accepts=True)
    h = ctx.decode_ex(syn, L, p, mk(T), seed=12, accepts=True)
    torch.cuda.synchronize()
    fa = _np(full["accepts"])
    assert (_np(a["accepts"]) + _np(b["accepts"]) == fa).all()
    assert (h["accepts"] == fa).all()
    for key in ("cls", "class_sum", "chain_sum", "chain_n", "chain_frames"):
        assert (_np(full[key]) == _np(plain[key])).all(), key
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, T, 12, i, syn[i], burn_in=3, accepts=True)
        assert (fa[i] == ref["accepts"]).all()
