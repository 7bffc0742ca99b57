"""GPU parity of the toric-code variant (n_classes = 16) against the oracle,
bit for bit: the generator, decodes (16 to 64 chains per syndrome, annealed,
random scan, independent flips), resumption and thermodynamic integration;
and the logical error rate falling with L."""
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


@pytest.mark.parametrize("L,p,n", [(2, 0.3, 9), (4, 0.1, 40), (6, 0.15, 30), (30, 0.12, 3)])
def test_toric_generator(ctx, L, p, n):
    syn, tc = O.t_gen_syndromes(8100, 3, n, L, p)
    gs, gt = ctx.gen_syndromes_toric(8100, 3, n, L, p, like=torch.zeros(1, device="cuda"))
    assert (_np(gs) == syn).all() and (_np(gt) == tc).all()


@pytest.mark.parametrize("L,R,kw", [(2, 1, {}), (4, 2, {}), (6, 4, dict(anneal_stages=2, anneal_beta0=0.5)),
                                    (4, 1, dict(scan=1)), (6, 2, dict(noise=1, beta_scale=0.85))])
def test_toric_decode_matches_oracle(ctx, pkg, L, R, kw):
    p, n, sweeps, burn = 0.1, 6, 12, 4
    syn, _ = O.t_gen_syndromes(8200 + L, 0, n, L, p)
    opts = pkg.Opts(n_classes=16, chains_per_class=R, n_sweeps=sweeps, burn_in=burn, **kw)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=93, id0=2)
    torch.cuda.synchronize()
    okw = {k: v for k, v in kw.items() if k in ("anneal_stages", "anneal_beta0", "scan", "noise", "beta_scale")}
    for i in range(n):
        ref = O.decode_one(L, p, 16, R, sweeps, 93, 2 + i, syn[i], burn_in=burn, **okw)
        assert int(_np(out["cls"])[i]) == ref["cls"]
        assert (_np(out["class_sum"])[i] == ref["class_sum"]).all()
        assert (_np(out["log_ratio"])[i] == ref["log_ratio"]).all()
        assert (_np(out["chain_sum"])[i] == ref["chain_sum"]).all()
        assert (_np(out["chain_n"])[i] == ref["chain_n"]).all()
        fr = _np(out["chain_frames"])[i]
        assert (fr[:, 0, :] == O.pack_bits(ref["frames_x"])).all()
        assert (fr[:, 1, :] == O.pack_bits(ref["frames_z"])).all()


def test_toric_resume_and_ti(ctx, pkg):
    L, p, n = 4, 0.12, 4
    syn, _ = O.t_gen_syndromes(8300, 0, n, L, p)
    opts = pkg.Opts(n_classes=16, chains_per_class=2, n_sweeps=14, burn_in=4)
    full = ctx.decode_ex(syn, L, p, opts, seed=4)
    a = ctx.decode_ex(syn, L, p, pkg.Opts(**{**opts.__dict__, "n_sweeps": 6}), seed=4)
    b = ctx.decode_ex(syn, L, p, opts, seed=4, sweep_begin=6, init_frames=a["chain_frames"],
                      init_chain_sum=a["chain_sum"])
    for key in ("cls", "class_sum", "chain_sum", "chain_n", "chain_frames"):
        assert (b[key] == full[key]).all(), key
    cls, lz, mean = ctx.decode_ti(syn, L, p, opts, n_beta=5, seed=7, id0=1)
    assert mean.shape == (n, 16, 5)
    for i in range(n):
        k, rlz, rmean = O.decode_ti(L, p, 16, 2, 14, 7, 1 + i, syn[i], n_beta=5, burn_in=4)
        assert cls[i] == k and (mean[i] == rmean).all() and (lz[i] == rlz).all()


def test_toric_ler_falls_with_L(ctx, pkg):
    p, n = 0.05, 4096
    like = torch.zeros(1, device="cuda")
    ler = {}
    for L in (4, 8):
        syn, tc = ctx.gen_syndromes_toric(8400 + L, 0, n, L, p, like=like)
        opts = pkg.Opts(n_classes=16, chains_per_class=2, n_sweeps=20 * L * L, burn_in=5 * L * L,
                        anneal_stages=4, anneal_beta0=0.3)
        cls, _, _ = ctx.decode(syn, L, p, opts, seed=8499)
        ler[L] = float((cls != tc).float().mean())
    assert ler[8] < ler[4] and ler[8] < p, ler


def test_toric_invalid(ctx, pkg):
    syn, _ = O.t_gen_syndromes(1, 0, 2, 4, 0.1)
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 5, 0.1, pkg.Opts(n_classes=16))                 # odd L
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 4, 0.1, pkg.Opts(n_classes=8))
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode_ragged(syn.reshape(-1), np.array([4, 4], np.int32), 0.1, pkg.Opts(n_classes=16))
    with pytest.raises(pkg.SurfmcmcError):
        ctx.gen_syndromes_toric(1, 0, 2, 3, 0.1)
