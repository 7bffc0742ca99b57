"""Serving: requests submitted while others are on the GPU are batched
continuously; every result equals the decode of that request alone (the
randomness is keyed by the request id), bit for bit."""
import threading

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


def _requests(n, p, seed=5001, sizes=(5, 9, 13)):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        L = int(rng.choice(sizes))
        rid = int(rng.integers(0, 2 ** 31))
        syn = O.gen_syndromes(seed, rid, 1, L, p)[0][0]
        reqs.append((rid, L, L + 3, syn))
    return reqs


def _alone(pkg, ctx, req, p, opts, seed):
    rid, L, sw, syn = req
    o = pkg.Opts(chains_per_class=opts.chains_per_class, n_sweeps=sw,
                 burn_in=sw * opts.burn_in // opts.n_sweeps, anneal_stages=opts.anneal_stages,
                 anneal_beta0=opts.anneal_beta0)
    cls, csum, _ = ctx.decode(syn[None, :].copy(), L, p, o, seed=seed, id0=rid)
    return int(cls[0]), csum[0]


def _collect(srv, n):
    got = {}
    while len(got) < n:
        ids, cls, sums, lat = srv.poll(wait_us=200000)
        for i, c, s, l in zip(ids, cls, sums, lat):
            got[int(i)] = (int(c), s.copy(), float(l))
    return got


# memory budgets: none; room for about two batches; less than two batches'
# scratch (a 32-request batch of these sizes charges ~90-170 kB), so that
# admissions must wait for a batch in flight to finish
@pytest.mark.parametrize("budget", [0, 300_000, 150_000])
def test_server_results_equal_alone(pkg, budget):
    p, seed = 0.12, 77
    opts = pkg.Opts(chains_per_class=4, n_sweeps=100, burn_in=40, anneal_stages=2, anneal_beta0=0.4)
    reqs = _requests(240, p)
    srv = pkg.Server(0, p, opts, seed=seed, max_batch=32, slots=3, max_L=13, memory_budget=budget, max_wait_us=300)
    # two submitting threads, interleaved with polling: requests arrive while batches run
    def submit(part):
        for r in part:
            srv.submit(r[0], r[1], r[2], r[3])
    th = [threading.Thread(target=submit, args=(reqs[k::2],)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = _collect(srv, len(reqs))
    stats = srv.stats()
    srv.close()
    assert stats["admitted"] == len(reqs) and stats["batches"] >= 2
    if budget == 0:
        assert stats["memory_stalls"] == 0
    if budget == 150_000:
        assert stats["memory_stalls"] > 0   # admission waited for memory to free up
    ctx = pkg.Context(0)
    for r in reqs:
        c, s, lat = got[r[0]]
        ac, asum = _alone(pkg, ctx, r, p, opts, seed)
        assert c == ac and (s == asum).all() and lat > 0
    ctx.close()


def test_server_single_request_and_errors(pkg):
    p = 0.12
    opts = pkg.Opts(chains_per_class=4, n_sweeps=10)
    srv = pkg.Server(0, p, opts, seed=1, max_batch=8, slots=1, max_L=9)
    req = _requests(1, p, seed=9, sizes=(9,))[0]
    srv.submit(*req)
    got = _collect(srv, 1)
    with pytest.raises(pkg.SurfmcmcError):
        srv.submit(1, 13, 5, np.zeros(312, np.uint8))   # L above max_L
    srv.close()
    ctx = pkg.Context(0)
    assert got[req[0]][0] == _alone(pkg, ctx, req, p, opts, 1)[0]
    ctx.close()
