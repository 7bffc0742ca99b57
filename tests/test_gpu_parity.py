"""GPU parity: every output of the CUDA path through the C ABI against the CPU
oracle on the same seeded inputs.  All quantities are integers (frames, n,
sums, classes) or one IEEE division/multiply from them (log-ratios), so the
bar is bit-exact equality."""
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


def _oracle_syndromes(seed, n, L, p, id0=0):
    syn, tc = O.gen_syndromes(seed, id0, n, L, p)
    return syn, tc


def _compare_decode(out, ref, i, Cn, L):
    assert int(_np(out["cls"])[i]) == ref["cls"]
    assert (_np(out["class_sum"])[i] == ref["class_sum"]).all()
    assert (_np(out["log_ratio"])[i] == ref["log_ratio"]).all()
    assert (_np(out["chain_sum"])[i] == ref["chain_sum"]).all()
    assert (_np(out["chain_n"])[i] == ref["chain_n"]).all()
    fr = _np(out["chain_frames"])[i]
    assert (fr[:, 0, :] == O.pack_bits(ref["frames_x"])).all()
    assert (fr[:, 1, :] == O.pack_bits(ref["frames_z"])).all()


@pytest.mark.parametrize("L,p,n", [(2, 0.3, 7), (3, 0.1, 33), (5, 0.15, 200), (13, 0.13, 129), (25, 0.18, 17),
                                   (31, 0.75, 5), (9, 0.0, 11)])
def test_gen_syndromes(ctx, L, p, n):
    syn, tc = _oracle_syndromes(2010, n, L, p, id0=3)
    like = torch.zeros(1, device="cuda")
    gs, gt = ctx.gen_syndromes(2010, 3, n, L, p, like=like)
    torch.cuda.synchronize()
    assert (_np(gs) == syn).all()
    assert (_np(gt) == tc).all()
    hs, ht = ctx.gen_syndromes(2010, 3, n, L, p)          # host buffers
    assert (hs == syn).all() and (ht == tc).all()


@pytest.mark.parametrize("L", [2, 3, 4, 5, 8, 13, 25, 31])
def test_start_frames(ctx, L):
    rng = np.random.default_rng(L)
    ns = O.nstab(L)
    syn = (rng.random((40, ns)) < rng.random((40, 1))).astype(np.uint8)
    syn[0] = 0
    syn[1] = 1
    fr, code = ctx.start_frames(torch.from_numpy(syn).cuda(), L)
    torch.cuda.synchronize()
    fr, code = _np(fr), _np(code)
    for i in range(len(syn)):
        ex, ez = O.pure_error(L, syn[i])
        assert (fr[i, 0] == O.pack_bits(ex)).all() and (fr[i, 1] == O.pack_bits(ez)).all()
        assert code[i] == O.class_code(L, ex, ez)


@pytest.mark.parametrize("R", [1, 2, 3, 4, 8, 12, 16])
def test_decode_chain_counts(ctx, pkg, R):
    """Plane widths G = 4, 8, 16, 32 and partly filled bundles."""
    L, p, n, sweeps = 5, 0.15, 11, 40
    syn, _ = _oracle_syndromes(1001, n, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=1101, id0=0)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 1101, i, syn[i])
        _compare_decode(out, ref, i, 4 * R, L)


def test_config1_all_200(ctx, pkg):
    """The small workload in full: L=5 (41 qubits), p=0.15, 4 classes x 4
    chains, 2000 sweeps, all 200 syndromes (syndrome seed 1001, decoder seed
    1101) against the oracle."""
    L, p, R, sweeps = 5, 0.15, 4, 2000
    syn, _ = _oracle_syndromes(1001, 200, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=1101, id0=0)
    torch.cuda.synchronize()
    idx = list(range(200))
    refs = O.decode_batch(L, p, 4, R, sweeps, 1101, idx, syn[idx])
    for i, ref in zip(idx, refs):
        _compare_decode(out, ref, i, 4 * R, L)


# (R = 6 and 12: 24 and 48 chains, 32-chain planes with a partly filled
# bundle, which the kernels specialised for whole bundles must not take)
@pytest.mark.parametrize("L,p,R,sweeps", [(2, 0.2, 4, 50), (3, 0.1, 16, 30), (4, 0.12, 8, 30),
                                          (7, 0.13, 16, 20), (13, 0.16, 16, 6), (17, 0.18, 4, 3),
                                          (25, 0.1, 8, 2), (31, 0.14, 4, 2), (9, 0.13, 12, 10),
                                          (5, 0.16, 6, 20)])
def test_decode_sizes(ctx, pkg, L, p, R, sweeps):
    n = 9
    syn, _ = _oracle_syndromes(2000 + L, n, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=77, id0=100)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 77, 100 + i, syn[i])
        _compare_decode(out, ref, i, 4 * R, L)


@pytest.mark.parametrize("lam", [2, 4, 8, 16, 32])
def test_lanes_per_bundle_do_not_change_results(ctx, pkg, lam):
    L, p, R, sweeps, n = 9, 0.14, 16, 25, 6
    syn, _ = _oracle_syndromes(3001, n, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, lanes_per_bundle=lam)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=5, id0=0)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 5, i, syn[i])
        _compare_decode(out, ref, i, 4 * R, L)


@pytest.mark.parametrize("beta_scale,p,burn", [(0.5, 0.12, 0), (2.0, 0.15, 3), (float("inf"), 0.15, 0),
                                               (0.0, 0.1, 0), (1.0, 0.75, 0), (1.0, 0.001, 5)])
def test_temperatures_and_burn_in(ctx, pkg, beta_scale, p, burn):
    L, R, sweeps, n = 5, 4, 30, 5
    syn, _ = _oracle_syndromes(4001, n, L, 0.15)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, beta_scale=beta_scale)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=6, id0=0)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 6, i, syn[i], burn_in=burn, beta_scale=beta_scale)
        _compare_decode(out, ref, i, 4 * R, L)


def test_resume_and_host_buffers(ctx, pkg):
    L, p, R, T, T1, n = 7, 0.13, 8, 40, 17, 5
    syn, _ = _oracle_syndromes(5001, n, L, p)
    dsyn = torch.from_numpy(syn).cuda()
    full = ctx.decode_ex(dsyn, L, p, pkg.Opts(chains_per_class=R, n_sweeps=T), seed=8)
    a = ctx.decode_ex(dsyn, L, p, pkg.Opts(chains_per_class=R, n_sweeps=T1), seed=8)
    b = ctx.decode_ex(dsyn, L, p, pkg.Opts(chains_per_class=R, n_sweeps=T), seed=8, sweep_begin=T1,
                      init_frames=a["chain_frames"], init_chain_sum=a["chain_sum"])
    # the same from host (numpy) buffers
    h = ctx.decode_ex(syn, L, p, pkg.Opts(chains_per_class=R, n_sweeps=T), seed=8)
    torch.cuda.synchronize()
    for k in ("cls", "class_sum", "log_ratio", "chain_sum", "chain_n", "chain_frames"):
        assert (_np(b[k]) == _np(full[k])).all(), k
        assert (_np(h[k]) == _np(full[k])).all(), k
    for i in range(n):
        _compare_decode(full, O.decode_one(L, p, 4, R, T, 8, i, syn[i]), i, 4 * R, L)


def test_batch_composition_does_not_matter(ctx, pkg):
    """A syndrome's result depends on its id only, not on its batch."""
    L, p, R, T = 5, 0.15, 4, 30
    syn, _ = _oracle_syndromes(6001, 20, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=T)
    whole = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=9, id0=50)
    part = ctx.decode_ex(torch.from_numpy(syn[7:12].copy()).cuda(), L, p, opts, seed=9, id0=57)
    torch.cuda.synchronize()
    assert (_np(part["chain_sum"]) == _np(whole["chain_sum"])[7:12]).all()


def test_empty_and_invalid(ctx, pkg):
    e = torch.zeros((0, O.nstab(5)), dtype=torch.uint8, device="cuda")
    cls, _, _ = ctx.decode(e, 5, 0.1)
    assert cls.numel() == 0
    syn = torch.zeros((2, O.nstab(5)), dtype=torch.uint8, device="cuda")
    bad = [dict(L=1), dict(L=32), dict(p=0.0), dict(p=0.8), dict(opts=pkg.Opts(n_classes=3)),
           dict(opts=pkg.Opts(chains_per_class=0)), dict(opts=pkg.Opts(n_sweeps=5, burn_in=6)),
           dict(opts=pkg.Opts(lanes_per_bundle=3)), dict(opts=pkg.Opts(beta_scale=-1.0)),
           dict(p=0.75, opts=pkg.Opts(beta_scale=float("inf"))),
           dict(opts=pkg.Opts(n_sweeps=10, burn_in=3, anneal_stages=4, anneal_beta0=0.3)),
           dict(opts=pkg.Opts(n_sweeps=10, burn_in=8, anneal_stages=4, anneal_beta0=0.0)),
           dict(opts=pkg.Opts(n_sweeps=10, burn_in=8, anneal_stages=-1))]
    for kw in bad:
        args = dict(L=5, p=0.1, opts=pkg.Opts(n_sweeps=2))
        args.update(kw)
        s = syn if args["L"] == 5 else torch.zeros((2, max(O.nstab(max(args["L"], 2)), 1)), dtype=torch.uint8,
                                                   device="cuda")
        with pytest.raises(pkg.SurfmcmcError) as ei:
            ctx.decode(s, args["L"], args["p"], args["opts"])
        assert ei.value.code == pkg.EINVAL, kw
    # the context stays usable after errors
    cls, _, _ = ctx.decode(syn, 5, 0.1, pkg.Opts(n_sweeps=2))
    torch.cuda.synchronize()
    assert cls.shape == (2,)


def test_ler_below_p_at_l7(ctx, pkg):
    """Same check as the oracle's pin (Sec. IV.A, p = 13%, L >= 6), through
    the GPU path on more syndromes."""
    L, p, n = 7, 0.13, 2000
    syn, tc = ctx.gen_syndromes(4242, 0, n, L, p, like=torch.zeros(1, device="cuda"))
    cls, _, _ = ctx.decode(syn, L, p, pkg.Opts(chains_per_class=4, n_sweeps=3000, burn_in=750), seed=4343)
    torch.cuda.synchronize()
    ler = float((cls != tc).float().mean())
    assert ler < p


@pytest.mark.parametrize("L,R,S,a0,burn,sweeps", [(5, 4, 4, 0.3, 40, 80), (9, 16, 3, 0.5, 7, 20), (4, 1, 2, 0.25, 9, 12),
                                                   (13, 16, 4, 0.3, 8, 10)])
def test_annealed_decode(ctx, pkg, L, R, S, a0, burn, sweeps):
    p, n = 0.13, 7
    syn, _ = _oracle_syndromes(8001 + L, n, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, anneal_stages=S, anneal_beta0=a0)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=12, id0=3)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 12, 3 + i, syn[i], burn_in=burn, anneal_stages=S, anneal_beta0=a0)
        _compare_decode(out, ref, i, 4 * R, L)


def test_annealed_resume_after_burn_in(ctx, pkg):
    L, p, R, T, T1, B, S = 7, 0.13, 8, 40, 23, 16, 4
    syn, _ = _oracle_syndromes(9001, 5, L, p)
    dsyn = torch.from_numpy(syn).cuda()
    mk = lambda t: pkg.Opts(chains_per_class=R, n_sweeps=t, burn_in=B, anneal_stages=S, anneal_beta0=0.3)
    full = ctx.decode_ex(dsyn, L, p, mk(T), seed=4)
    a = ctx.decode_ex(dsyn, L, p, mk(T1), seed=4)
    b = ctx.decode_ex(dsyn, L, p, mk(T), seed=4, sweep_begin=T1, init_frames=a["chain_frames"],
                      init_chain_sum=a["chain_sum"])
    torch.cuda.synchronize()
    for k in ("cls", "class_sum", "chain_sum", "chain_n", "chain_frames"):
        assert (_np(b[k]) == _np(full[k])).all(), k


def test_annealed_ler_l13(ctx, pkg):
    """With the annealed start the L=13 decoder is well below threshold at
    p = 10% (the paper's threshold for this algorithm is 15-16%)."""
    L, p, n = 13, 0.10, 2048
    syn, tc = ctx.gen_syndromes(7000, 0, n, L, p, like=torch.zeros(1, device="cuda"))
    opts = pkg.Opts(chains_per_class=16, n_sweeps=4000, burn_in=800, anneal_stages=4, anneal_beta0=0.3)
    cls, _, _ = ctx.decode(syn, L, p, opts, seed=7100)
    torch.cuda.synchronize()
    assert float((cls != tc).float().mean()) < 0.02


@pytest.mark.parametrize("L,R,nb,anneal", [(3, 8, 21, False), (5, 4, 7, True), (9, 16, 5, False)])
def test_decode_ti(ctx, pkg, L, R, nb, anneal):
    """Thermodynamic integration (Eq. 6, Simpson) against the oracle, bit for bit."""
    p, n, sweeps, burn = 0.14, 5, 24, 8
    syn, _ = _oracle_syndromes(1201 + L, n, L, p)
    kw = dict(anneal_stages=2, anneal_beta0=0.5) if anneal else {}
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, **kw)
    cls, lz, mean = ctx.decode_ti(torch.from_numpy(syn).cuda(), L, p, opts, n_beta=nb, seed=55, id0=7)
    torch.cuda.synchronize()
    cls, lz, mean = _np(cls), _np(lz), _np(mean)
    for i in range(n):
        k, rlz, rmean = O.decode_ti(L, p, 4, R, sweeps, 55, 7 + i, syn[i], n_beta=nb, burn_in=burn, **kw)
        assert cls[i] == k
        assert (mean[i] == rmean).all()
        assert (lz[i] == rlz).all()


def test_autotune_choice_keeps_results(ctx, pkg):
    """The autotuner picks the fastest (lanes per bundle, resident blocks per
    multiprocessor) for (L, R); decodes with the tuned shape give the same
    results as any explicit shape."""
    L, p, R, n = 9, 0.13, 16, 7
    best, best_b, ms = ctx.autotune(L, R, p, n_probe=2048, sweeps=10)
    assert best in pkg.TUNE_LANES and best_b in pkg.TUNE_BLOCKS
    assert ms[(best, best_b)] == min(v for v in ms.values() if v == v)
    assert len(ms) == len(pkg.TUNE_LANES) * len(pkg.TUNE_BLOCKS)
    syn, _ = _oracle_syndromes(2222, n, L, p)
    d = torch.from_numpy(syn).cuda()
    tuned = ctx.decode_ex(d, L, p, pkg.Opts(chains_per_class=R, n_sweeps=15), seed=3)
    fixed = ctx.decode_ex(d, L, p, pkg.Opts(chains_per_class=R, n_sweeps=15, lanes_per_bundle=4), seed=3)
    torch.cuda.synchronize()
    for k in ("cls", "class_sum", "chain_sum", "chain_frames"):
        assert (_np(tuned[k]) == _np(fixed[k])).all()


@pytest.mark.parametrize("p,seed,idx", [
    (0.13, 2013, [0, 1, 127, 128, 4097, 8191, 12288, 16383]),
    (0.10, 2010, [0, 5461, 10922, 16383]),
    (0.16, 2016, [2, 4096, 12287, 16381]),
    (0.18, 2018, [31, 8192, 8193, 16383])])
def test_bench_workload_full_size_sampled(ctx, pkg, p, seed, idx):
    """The benchmark's own workload at full size in its launch configuration,
    at each of its four error rates: L = 13, 16,384 syndromes (syndrome seed
    2010/2013/2016/2018, decoder seed + 100), 4 classes x 16 chains, 20,000
    sweeps of which the first 4,000 are annealed in 16 stages from 0.1
    beta_bar.  Syndromes spread over the batch (first, last, bundle and block
    boundaries) are decoded by the oracle at full length and must agree bit
    for bit: class, sums, log-ratios, per-chain sums, final n and final
    frames.  Each error rate has its own threshold table, digit-plane modes
    and annealing tables."""
    L, n, R, T, burn, stages, beta0 = 13, 16384, 16, 20000, 4000, 16, 0.1
    syn, _ = O.gen_syndromes(seed, 0, n, L, p)
    opts = pkg.Opts(chains_per_class=R, n_sweeps=T, burn_in=burn, anneal_stages=stages, anneal_beta0=beta0)
    dsyn = torch.from_numpy(syn).cuda()
    out = ctx.decode_ex(dsyn, L, p, opts, seed=seed + 100, id0=0)
    cls, csum, lr = ctx.decode(dsyn, L, p, opts, seed=seed + 100, id0=0)   # the call the benchmark times
    torch.cuda.synchronize()
    assert (_np(cls) == _np(out["cls"])).all() and (_np(csum) == _np(out["class_sum"])).all()
    assert (_np(lr) == _np(out["log_ratio"])).all()
    refs = O.decode_batch(L, p, 4, R, T, seed + 100, idx, syn[idx], burn_in=burn, anneal_stages=stages,
                          anneal_beta0=beta0)
    for i, ref in zip(idx, refs):
        _compare_decode(out, ref, i, 4 * R, L)
