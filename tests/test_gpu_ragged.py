"""Ragged batches (several code sizes in one call) and their graph-captured
plans, against per-size plain decodes and the oracle, bit for bit."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LS = [5, 9, 13, 17, 25]


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


def _mixed(seed, n, p, id0=0):
    """Items with L drawn from LS; returns Ls, concatenated rows, rows, true classes."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(LS, size=n).astype(np.int32)
    rows, tcs = [], []
    for i, L in enumerate(Ls):
        s, t = O.gen_syndromes(seed, id0 + i, 1, int(L), p)
        rows.append(s[0])
        tcs.append(int(t[0]))
    return Ls, np.concatenate(rows).astype(np.uint8), rows, np.array(tcs)


def _sweeps(Ls, scale):
    return np.array([max(10, (int(L) * int(L)) // scale) for L in Ls], np.uint32)


@pytest.mark.parametrize("anneal", [False, True])
def test_ragged_matches_per_size_decodes(ctx, pkg, anneal):
    p, n, R = 0.14, 37, 4
    Ls, cat, rows, _ = _mixed(3001, n, p)
    sw = _sweeps(Ls, 4)
    kw = dict(n_sweeps=100, burn_in=40, anneal_stages=4, anneal_beta0=0.3) if anneal else dict(n_sweeps=100)
    opts = pkg.Opts(chains_per_class=R, **kw)
    cls, csum, lr = ctx.decode_ragged(torch.from_numpy(cat).cuda(), torch.from_numpy(Ls).cuda(), p, opts,
                                      n_sweeps=torch.from_numpy(sw).cuda(), seed=3101, id0=0)
    torch.cuda.synchronize()
    cls, csum, lr = cls.cpu().numpy(), csum.cpu().numpy(), lr.cpu().numpy()
    for i in range(n):
        L, s = int(Ls[i]), int(sw[i])
        burn = s * opts.burn_in // opts.n_sweeps
        o1 = pkg.Opts(chains_per_class=R, n_sweeps=s, burn_in=burn,
                      anneal_stages=opts.anneal_stages, anneal_beta0=opts.anneal_beta0)
        ref = ctx.decode_ex(torch.from_numpy(rows[i][None, :].copy()).cuda(), L, p, o1, seed=3101, id0=i)
        torch.cuda.synchronize()
        assert cls[i] == int(ref["cls"][0])
        assert (csum[i] == ref["class_sum"][0].cpu().numpy()).all()
        assert (lr[i] == ref["log_ratio"][0].cpu().numpy()).all()
        if i % 9 == 0 and L <= 13:
            orc = O.decode_one(L, p, 4, R, s, 3101, i, rows[i], burn_in=burn, anneal_stages=opts.anneal_stages,
                               anneal_beta0=opts.anneal_beta0)
            assert cls[i] == orc["cls"] and (csum[i] == orc["class_sum"]).all()


def test_ragged_explicit_ids_and_host_buffers(ctx, pkg):
    p, n, R = 0.12, 11, 4
    Ls, cat, rows, _ = _mixed(77, n, p)
    ids = np.random.default_rng(5).choice(100000, size=n, replace=False).astype(np.uint32)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=12)
    cls, csum, _ = ctx.decode_ragged(cat, Ls, p, opts, seed=9, ids=ids)
    for i in range(n):
        ref = O.decode_one(int(Ls[i]), p, 4, R, 12, 9, int(ids[i]), rows[i])
        assert cls[i] == ref["cls"] and (csum[i] == ref["class_sum"]).all()


def test_plan_replays_on_new_inputs(ctx, pkg):
    p, n, R = 0.14, 24, 4
    Ls, cat1, _, _ = _mixed(11, n, p)
    # same sizes, new syndromes
    rows2 = [O.gen_syndromes(12, i, 1, int(L), p)[0][0] for i, L in enumerate(Ls)]
    cat2 = np.concatenate(rows2).astype(np.uint8)
    sw = _sweeps(Ls, 10)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=50, burn_in=10, anneal_stages=2, anneal_beta0=0.4)
    d_syn = torch.from_numpy(cat1).cuda()
    d_cls = torch.empty(n, dtype=torch.int32, device="cuda")
    d_sum = torch.empty((n, 4), dtype=torch.uint64, device="cuda")
    d_lr = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    plan = pkg.RaggedPlan(ctx, Ls, p, d_syn, d_cls, d_sum, d_lr, opts=opts, n_sweeps=sw, seed=21)
    for cat in (cat1, cat2, cat1):
        d_syn.copy_(torch.from_numpy(cat))
        plan.launch()
        torch.cuda.synchronize()
        ref_cls, ref_sum, ref_lr = ctx.decode_ragged(torch.from_numpy(cat).cuda(), Ls, p, opts, n_sweeps=sw, seed=21)
        torch.cuda.synchronize()
        assert torch.equal(d_cls, ref_cls) and torch.equal(d_sum.cpu(), ref_sum.cpu()) and torch.equal(d_lr, ref_lr)
    plan.close()


def test_ragged_invalid(ctx, pkg):
    p = 0.1
    Ls = np.array([3, 4, 5, 6, 7, 8, 9, 10, 11], np.int32)   # 9 groups
    cat = np.zeros(sum(2 * L * (L - 1) for L in Ls), np.uint8)
    with pytest.raises(pkg.SurfmcmcError) as e:
        ctx.decode_ragged(cat, Ls, p, pkg.Opts(n_sweeps=4))
    assert e.value.code == pkg.EINVAL
    Ls = np.array([5, 9], np.int32)
    cat = np.zeros(40 + 144, np.uint8)
    with pytest.raises(pkg.SurfmcmcError):
        # item sweeps 4 -> burn-in 4*2/10 = 0 < 2 annealing stages
        ctx.decode_ragged(cat, Ls, p, pkg.Opts(n_sweeps=10, burn_in=2, anneal_stages=2, anneal_beta0=0.5),
                          n_sweeps=np.array([4, 10], np.uint32))
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode_ragged(cat, np.array([5, 40], np.int32), p, pkg.Opts(n_sweeps=4))


def test_ragged_full_size_sampled(ctx, pkg):
    """65,536 syndromes at p = 0.14 with L drawn from {5, 9, 13, 17, 25},
    sweeps = L^2, 4 classes x 4 chains, in one ragged call; sampled items
    against the oracle (two per size)."""
    p, n, R = 0.14, 65536, 4
    rng = np.random.default_rng(3001)
    Ls = rng.choice(LS, size=n).astype(np.int32)
    like = torch.zeros(1, device="cuda")
    rows = [None] * n
    for L in LS:
        idx = np.nonzero(Ls == L)[0]
        # ids = item index: generate each size's items at their ids
        for i in idx[:2].tolist() + idx[-1:].tolist():
            rows[i] = O.gen_syndromes(3001, i, 1, L, p)[0][0]
    # the rest from the GPU generator, one id at a time would be slow: use
    # contiguous runs of the GPU generator per size and pick the items' ids
    cat = np.empty(sum(2 * int(L) * (int(L) - 1) for L in Ls), np.uint8)
    off = np.concatenate([[0], np.cumsum([2 * int(L) * (int(L) - 1) for L in Ls])])
    for L in LS:
        g, _ = ctx.gen_syndromes(3001, 0, n, L, p, like=like)
        g = g.cpu().numpy()
        for i in np.nonzero(Ls == L)[0]:
            cat[off[i]:off[i + 1]] = g[i]
    sw = np.array([int(L) * int(L) for L in Ls], np.uint32)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=625)
    cls, csum, _ = ctx.decode_ragged(torch.from_numpy(cat).cuda(), torch.from_numpy(Ls).cuda(), p, opts,
                                     n_sweeps=torch.from_numpy(sw).cuda(), seed=3101)
    torch.cuda.synchronize()
    cls, csum = cls.cpu().numpy(), csum.cpu().numpy()
    picks = [i for i in range(n) if rows[i] is not None]
    for i in picks:
        assert (cat[off[i]:off[i + 1]] == rows[i]).all()
    for i in picks:
        L = int(Ls[i])
        ref = O.decode_one(L, p, 4, R, L * L, 3101, i, rows[i])
        assert cls[i] == ref["cls"] and (csum[i] == ref["class_sum"]).all(), (i, L)
