"""Early stop through the C ABI: the stop rule and its results, checked
bit-exactly against plain decodes truncated at every checkpoint (a truncated
run is the prefix of the longer one, the chains being keyed by syndrome id),
and the gain of a trained network at a matched error rate."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import cnn

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


def _opts(pkg, sweeps=300, burn=60, R=4):
    return pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, anneal_stages=4, anneal_beta0=0.3)


def _net(pkg, ctx, L, seed):
    rng = np.random.default_rng(seed)
    p = cnn.init_params(seed) + rng.normal(0, 0.05, size=cnn.n_params())
    net = pkg.Network(ctx, L, max_batch=128)
    net.set_params(p.astype(np.float32))
    return net


def test_tau_infinite_is_plain_decode(pkg, ctx):
    L, n, p = 7, 300, 0.12
    syn, _ = O.gen_syndromes(6001, 0, n, L, p)
    net = _net(pkg, ctx, L, 1)
    o = _opts(pkg)
    cls, csum, sw = ctx.decode_early(net, syn, L, p, o, chunk_sweeps=50, tau=float("inf"), seed=77, id0=5)
    ref_cls, ref_sum, _ = ctx.decode(syn, L, p, o, seed=77, id0=5)
    assert (cls == ref_cls).all() and (csum == ref_sum).all()
    assert (sw == o.n_sweeps).all()
    net.close()


@pytest.mark.parametrize("device", [False, True])
def test_stop_rule_bit_exact(pkg, ctx, device):
    L, n, p, chunk = 7, 400, 0.12, 50
    syn, _ = O.gen_syndromes(6002, 0, n, L, p)
    net = _net(pkg, ctx, L, 2)
    o = _opts(pkg)
    lp = net.forward(syn).astype(np.float32)
    am = lp.argmax(1)
    masked = lp.copy()
    masked[np.arange(n), am] = -np.inf
    margin = lp[np.arange(n), am] - masked.max(1)
    tau = float(np.median(margin))
    marks = list(range(o.burn_in + chunk, o.n_sweeps, chunk)) + [o.n_sweeps]
    dec, sums = [], []
    for tk in marks:
        c, s, _ = ctx.decode(syn, L, p, pkg.Opts(**{**o.__dict__, "n_sweeps": tk}), seed=78, id0=9)
        dec.append(c)
        sums.append(s)
    stop = np.full(n, len(marks) - 1)
    for i in range(n):
        for k in range(len(marks) - 1):
            if margin[i] > np.float32(tau) and am[i] == dec[k][i]:
                stop[i] = k
                break
    x = torch.from_numpy(syn).cuda() if device else syn
    cls, csum, sw = ctx.decode_early(net, x, L, p, o, chunk_sweeps=chunk, tau=tau, seed=78, id0=9)
    if device:
        cls, csum, sw = cls.cpu().numpy(), csum.cpu().numpy(), sw.cpu().numpy()
    for i in range(n):
        k = stop[i]
        assert cls[i] == dec[k][i] and (csum[i] == sums[k][i]).all() and sw[i] == marks[k], i
    # both kinds of stop occur
    assert (stop < len(marks) - 1).sum() > 20 and (stop == len(marks) - 1).sum() > 20
    net.close()


def test_all_stop_at_first_checkpoint(pkg, ctx):
    """tau = -inf: a syndrome stops at the first checkpoint where the chains
    agree with the network; many items exercise the compaction."""
    L, n, p, chunk = 5, 3000, 0.1, 40
    syn, _ = O.gen_syndromes(6003, 0, n, L, p)
    net = _net(pkg, ctx, L, 3)
    o = _opts(pkg, sweeps=200, burn=40)
    cls, csum, sw = ctx.decode_early(net, syn, L, p, o, chunk_sweeps=chunk, tau=-float("inf"), seed=79)
    lp = net.forward(syn)
    am = lp.argmax(1)
    marks = list(range(o.burn_in + chunk, o.n_sweeps, chunk)) + [o.n_sweeps]
    for k, tk in enumerate(marks):
        c, s, _ = ctx.decode(syn, L, p, pkg.Opts(**{**o.__dict__, "n_sweeps": tk}), seed=79)
        here = sw == tk
        assert (cls[here] == c[here]).all() and (csum[here] == s[here]).all()
        if k + 1 < len(marks):
            assert (c[here] == am[here]).all()
            later = sw > tk
            assert (c[later] != am[later]).all()
    assert set(np.unique(sw)) <= set(marks)


def test_invalid(pkg, ctx):
    L = 5
    syn, _ = O.gen_syndromes(1, 0, 4, L, 0.1)
    net7 = _net(pkg, ctx, 7, 4)
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode_early(net7, syn, L, 0.1, _opts(pkg), chunk_sweeps=10)   # net for another L
    net5 = _net(pkg, ctx, 5, 4)
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode_early(net5, syn, L, 0.1, _opts(pkg), chunk_sweeps=0)
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode_early(net5, syn, L, 0.1, _opts(pkg), chunk_sweeps=10, tau=float("nan"))
    c, s, w = ctx.decode_early(net5, syn[:0], L, 0.1, _opts(pkg), chunk_sweeps=10)
    assert len(c) == 0


def test_trained_network_gain(pkg, ctx):
    """L = 7: a network trained on the library's own labels (p over
    [0.08, 0.18]) stops many syndromes early at p = 0.10; on a fresh test set
    of 131,072 syndromes the early-stop error rate stays within one binomial
    sigma of the long chains' (the bar for a matched error rate) and the throughput
    rises."""
    import argparse
    from paper_1302_2669_gb300 import early_stop as E
    ns = argparse.Namespace(L=7, train=1 << 16, val=65536, test=131072, p_lo=0.08, p_hi=0.18, n_p=8, label_R=4,
                            label_sweeps=400, epochs=4, batch=512, lr=2e-3, lr_final=2e-4, R=4, sweeps=2000,
                            burn_in=400, anneal_stages=16, anneal_beta0=0.1, chunk=200, seed=4001, eval_ps=[0.10])
    res = E.run(ns, log=lambda m: None)
    row = res["per_p"][0]
    row = {k: v for k, v in row.items() if k != "calibration"}
    assert row["tau"] is not None
    assert row["ler_early"] <= row["ler_long"] + row["sigma"], row
    assert row["mean_sweeps_early"] < 0.75 * ns.sweeps, row
    assert row["gain"] > 1.2, row


def _reorder_reference(L, p, R, o, chunk, tau, seed, id0, syn, lp):
    """Early stop with budget reordering, composed from the oracle's chain
    runs: the stop rule at every checkpoint; at the first checkpoint a
    survivor's chains of its two least likely classes (network ranking,
    ties to the lower class) take the states of the two most likely classes'
    chains and restart their sums, the classes' sums so far being frozen;
    later decisions compare class means exactly."""
    burn, T = o.burn_in, o.n_sweeps
    marks = list(range(burn + chunk, T, chunk)) + [T]
    kw = dict(burn_in=burn, anneal_stages=o.anneal_stages, anneal_beta0=o.anneal_beta0)
    spp = 4
    res = []
    for i in range(len(syn)):
        am = int(np.argmax(lp[i]))
        margin = lp[i][am] - max(lp[i][k] for k in range(4) if k != am)
        rank = sorted(range(4), key=lambda k: (-float(lp[i][k]), k))
        a, b, c, d = rank
        out = O.run_chains(L, 4, R, p, seed, id0 + i, syn[i], 0, marks[0], **kw)
        fx, fz, cs = out["frames_x"].copy(), out["frames_z"].copy(), out["chain_sum"].copy()
        frozen = None
        for k, tk in enumerate(marks):
            if k > 0:
                out = O.run_chains(L, 4, R, p, seed, id0 + i, syn[i], marks[k - 1], tk, frames=(fx, fz),
                                   chain_sum=cs, **kw)
                fx, fz, cs = out["frames_x"].copy(), out["frames_z"].copy(), out["chain_sum"].copy()
            S = [int(cs[q * R:(q + 1) * R].sum()) for q in range(4)]
            if frozen is None:
                N = [1, 1, 1, 1]
            else:
                S[a] += S[c]
                S[b] += S[d]
                S[c], S[d] = frozen
                n_top = spp * R * ((tk - burn) + (tk - marks[0]))
                n_low = spp * R * (marks[0] - burn)
                N = [0, 0, 0, 0]
                N[a] = N[b] = n_top
                N[c] = N[d] = n_low
            best = 0
            for q in range(1, 4):
                if S[q] * N[best] < S[best] * N[q]:
                    best = q
            final = k + 1 == len(marks)
            if final or (margin > np.float32(tau) and am == best):
                res.append((best, S, tk))
                break
            if frozen is None:
                frozen = (S[c], S[d])
                for r in range(R):
                    for src, dst in ((a, c), (b, d)):
                        fx[dst * R + r] = fx[src * R + r]
                        fz[dst * R + r] = fz[src * R + r]
                        cs[dst * R + r] = 0
    return res


@pytest.mark.parametrize("device", [False, True])
def test_budget_reordering_bit_exact(pkg, ctx, device):
    L, n, p, chunk, R = 5, 400, 0.13, 40, 4
    syn, _ = O.gen_syndromes(6010, 0, n, L, p)
    net = _net(pkg, ctx, L, 5)
    o = _opts(pkg, sweeps=240, burn=40, R=R)
    lp = net.forward(syn).astype(np.float32)
    am = lp.argmax(1)
    masked = lp.copy()
    masked[np.arange(n), am] = -np.inf
    tau = float(np.quantile(lp[np.arange(n), am] - masked.max(1), 0.25))
    x = torch.from_numpy(syn).cuda() if device else syn
    cls, csum, sw = ctx.decode_early(net, x, L, p, o, chunk_sweeps=chunk, tau=tau, seed=81, id0=3, reorder=True)
    if device:
        cls, csum, sw = cls.cpu().numpy(), csum.cpu().numpy(), sw.cpu().numpy()
    ref = _reorder_reference(L, p, R, o, chunk, tau, 81, 3, syn, lp)
    first = o.burn_in + chunk
    for i, (c, S, tk) in enumerate(ref):
        assert cls[i] == c and [int(v) for v in csum[i]] == S and sw[i] == tk, i
    # items stop at the first checkpoint, later after reordering, and at the end
    assert (sw == first).sum() > 10 and ((sw > first) & (sw < o.n_sweeps)).sum() > 5
    assert (sw == o.n_sweeps).sum() > 10
    # without reordering the same call is the plain early stop
    c0, s0, w0 = ctx.decode_early(net, syn, L, p, o, chunk_sweeps=chunk, tau=tau, seed=81, id0=3)
    assert (w0[sw == first] == first).all() and (c0[sw == first] == cls[sw == first]).all()
    net.close()
