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
    the early-stop error rate stays within two binomial sigmas of the long
    chains' and the throughput rises."""
    import argparse
    from paper_1302_2669_gb300 import early_stop as E
    ns = argparse.Namespace(L=7, train=1 << 16, val=32768, test=32768, p_lo=0.08, p_hi=0.18, n_p=8, label_R=4,
                            label_sweeps=400, epochs=4, batch=512, lr=2e-3, lr_final=2e-4, R=4, sweeps=2000,
                            burn_in=200, chunk=200, seed=4001, eval_ps=[0.10])
    res = E.run(ns, log=lambda m: None)
    row = res["per_p"][0]
    row = {k: v for k, v in row.items() if k != "calibration"}
    assert row["tau"] is not None
    assert row["ler_early"] <= row["ler_long"] + 2 * row["sigma"], row
    assert row["mean_sweeps_early"] < 0.75 * ns.sweeps, row
    assert row["gain"] > 1.2, row
