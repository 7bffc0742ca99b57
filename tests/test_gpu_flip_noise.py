"""GPU parity under independent bit and phase flips (Sec. IV.B, opts.noise =
1): the generator, decodes in both scan modes, annealed and resumed runs and
thermodynamic integration against the oracle, bit for bit; and the decoder
at beta* = 0.85 beta_bar beating the physical flip rate with growing L."""
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


@pytest.mark.parametrize("L,p,n", [(2, 0.3, 9), (5, 0.1, 50), (13, 0.08, 40), (31, 0.2, 4)])
def test_flip_generator(ctx, L, p, n):
    syn, tc = O.gen_syndromes(4500, 2, n, L, p, noise=1)
    gs, gt = ctx.gen_syndromes(4500, 2, n, L, p, like=torch.zeros(1, device="cuda"), noise=1)
    assert (_np(gs) == syn).all() and (_np(gt) == tc).all()


@pytest.mark.parametrize("L,R,scan,anneal", [(3, 1, 0, False), (5, 4, 0, True), (7, 16, 0, False), (9, 2, 0, False),
                                             (5, 4, 1, False), (4, 8, 1, True)])
def test_flip_decode_matches_oracle(ctx, pkg, L, R, scan, anneal):
    p, n, sweeps, burn = 0.09, 12, 16, 4
    syn, _ = O.gen_syndromes(4600 + L, 0, n, L, p, noise=1)
    kw = dict(anneal_stages=2, anneal_beta0=0.5) if anneal else {}
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, beta_scale=0.85, scan=scan, noise=1, **kw)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=66, id0=3)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 66, 3 + i, syn[i], burn_in=burn, beta_scale=0.85, scan=scan, noise=1,
                           **kw)
        assert int(_np(out["cls"])[i]) == ref["cls"]
        assert (_np(out["class_sum"])[i] == ref["class_sum"]).all()
        assert (_np(out["log_ratio"])[i] == ref["log_ratio"]).all()
        assert (_np(out["chain_sum"])[i] == ref["chain_sum"]).all()
        assert (_np(out["chain_n"])[i] == ref["chain_n"]).all()
        fr = _np(out["chain_frames"])[i]
        assert (fr[:, 0, :] == O.pack_bits(ref["frames_x"])).all()
        assert (fr[:, 1, :] == O.pack_bits(ref["frames_z"])).all()


def test_flip_resume(ctx, pkg):
    L, p, n, T, T1 = 7, 0.1, 8, 20, 7
    syn, _ = O.gen_syndromes(4700, 0, n, L, p, noise=1)
    opts = pkg.Opts(chains_per_class=4, n_sweeps=T, burn_in=3, noise=1)
    full = ctx.decode_ex(syn, L, p, opts, seed=2)
    a = ctx.decode_ex(syn, L, p, pkg.Opts(**{**opts.__dict__, "n_sweeps": T1}), seed=2)
    b = ctx.decode_ex(syn, L, p, opts, seed=2, sweep_begin=T1, init_frames=a["chain_frames"],
                      init_chain_sum=a["chain_sum"])
    for key in ("cls", "class_sum", "chain_sum", "chain_n", "chain_frames"):
        assert (b[key] == full[key]).all(), key


def test_flip_ti(ctx, pkg):
    L, p, n, nb = 3, 0.1, 4, 7
    syn, _ = O.gen_syndromes(4800, 0, n, L, p, noise=1)
    opts = pkg.Opts(chains_per_class=4, n_sweeps=14, burn_in=4, noise=1)
    cls, lz, mean = ctx.decode_ti(syn, L, p, opts, n_beta=nb, seed=9, id0=1)
    for i in range(n):
        k, rlz, rmean = O.decode_ti(L, p, 4, 4, 14, 9, 1 + i, syn[i], n_beta=nb, burn_in=4, noise=1)
        assert cls[i] == k and (mean[i] == rmean).all() and (lz[i] == rlz).all()
        assert mean[i][0][0] == O.nq(L)


def test_flip_decoder_below_p_and_improving_with_L(ctx, pkg):
    """Sec. IV.B: at a flip probability well below threshold the logical
    error rate (either logical bit wrong) falls with L and is below p at
    L = 9 (beta* = 0.85 beta_bar)."""
    p, n = 0.05, 4096
    ler = {}
    like = torch.zeros(1, device="cuda")
    for L in (5, 9):
        syn, tc = ctx.gen_syndromes(4900 + L, 0, n, L, p, like=like, noise=1)
        opts = pkg.Opts(chains_per_class=4, n_sweeps=40 * L * L, burn_in=10 * L * L, beta_scale=0.85, noise=1,
                        anneal_stages=4, anneal_beta0=0.3)
        cls, _, _ = ctx.decode(syn, L, p, opts, seed=4999)
        ler[L] = float((cls != tc).float().mean())
    assert ler[9] < ler[5] and ler[9] < p, ler


def test_flip_invalid(ctx, pkg):
    syn, _ = O.gen_syndromes(1, 0, 2, 5, 0.1, noise=1)
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 5, 0.6, pkg.Opts(noise=1))          # flip p > 1/2
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 5, 0.1, pkg.Opts(noise=2))
    with pytest.raises(pkg.SurfmcmcError):
        ctx.gen_syndromes(1, 0, 2, 5, 0.1, noise=3)
