"""GPU parity of the random-scan mode (Sec. IV as written: one random
generator per step, n summed after every step) against the oracle, bit for
bit: decisions, class sums, log-ratios, per-chain sums, final n and frames,
for every chain layout, with resumption, annealing, thermodynamic
integration and ragged batches."""
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


def _check(out, ref, i):
    assert int(_np(out["cls"])[i]) == ref["cls"]
    assert (_np(out["class_sum"])[i] == ref["class_sum"]).all()
    assert (_np(out["log_ratio"])[i] == ref["log_ratio"]).all()
    assert (_np(out["chain_sum"])[i] == ref["chain_sum"]).all()
    assert (_np(out["chain_n"])[i] == ref["chain_n"]).all()
    fr = _np(out["chain_frames"])[i]
    assert (fr[:, 0, :] == O.pack_bits(ref["frames_x"])).all()
    assert (fr[:, 1, :] == O.pack_bits(ref["frames_z"])).all()


@pytest.mark.parametrize("L,R,p,n", [(3, 1, 0.2, 9), (4, 2, 0.15, 7), (5, 4, 0.15, 20), (7, 8, 0.12, 5),
                                     (9, 16, 0.1, 3)])
def test_random_scan_matches_oracle(ctx, pkg, L, R, p, n):
    sweeps, burn = 14, 3
    syn, _ = O.gen_syndromes(3300 + L, 0, n, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, scan=1)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=91, id0=4)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 91, 4 + i, syn[i], burn_in=burn, scan=1)
        _check(out, ref, i)


def test_random_scan_resume_and_anneal(ctx, pkg):
    L, R, p, n, T, T1 = 5, 4, 0.14, 6, 20, 9
    syn, _ = O.gen_syndromes(3401, 0, n, L, p)
    kw = dict(anneal_stages=2, anneal_beta0=0.4)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=T, burn_in=6, scan=1, **kw)
    full = ctx.decode_ex(syn, L, p, opts, seed=5)
    a = ctx.decode_ex(syn, L, p, pkg.Opts(**{**opts.__dict__, "n_sweeps": T1}), seed=5)
    b = ctx.decode_ex(syn, L, p, opts, seed=5, sweep_begin=T1, init_frames=a["chain_frames"],
                      init_chain_sum=a["chain_sum"])
    for key in ("cls", "class_sum", "chain_sum", "chain_n", "chain_frames"):
        assert (b[key] == full[key]).all(), key
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, T, 5, i, syn[i], burn_in=6, scan=1, **kw)
        _check(full, ref, i)


def test_random_scan_ti(ctx, pkg):
    L, R, p, n, nb = 3, 4, 0.14, 4, 5
    syn, _ = O.gen_syndromes(3501, 0, n, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=12, burn_in=4, scan=1)
    cls, lz, mean = ctx.decode_ti(syn, L, p, opts, n_beta=nb, seed=8, id0=2)
    for i in range(n):
        k, rlz, rmean = O.decode_ti(L, p, 4, R, 12, 8, 2 + i, syn[i], n_beta=nb, burn_in=4, scan=1)
        assert cls[i] == k and (mean[i] == rmean).all() and (lz[i] == rlz).all()


def test_random_scan_ragged_equals_per_size(ctx, pkg):
    p, R = 0.12, 4
    sizes = [3, 5, 7, 5, 3, 7, 7]
    rows, per = [], {}
    for i, L in enumerate(sizes):
        s, _ = O.gen_syndromes(3600, i, 1, L, p)
        rows.append(s[0])
    syn = np.concatenate(rows).astype(np.uint8)
    Ls = np.array(sizes, np.int32)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=10, burn_in=2, scan=1)
    cls, csum, _ = ctx.decode_ragged(syn, Ls, p, opts, seed=12, ids=np.arange(len(sizes), dtype=np.uint32))
    for i, L in enumerate(sizes):
        ref = O.decode_one(L, p, 4, R, 10, 12, i, rows[i], burn_in=2, scan=1)
        assert cls[i] == ref["cls"] and (csum[i] == ref["class_sum"]).all()


def test_random_scan_invalid(ctx, pkg):
    syn, _ = O.gen_syndromes(1, 0, 2, 5, 0.1)
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 5, 0.1, pkg.Opts(scan=2))
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 5, 0.1, pkg.Opts(scan=1, lanes_per_bundle=8))
    ok = ctx.decode(syn, 5, 0.1, pkg.Opts(scan=1, lanes_per_bundle=32, n_sweeps=3))
    assert len(ok[0]) == 2
