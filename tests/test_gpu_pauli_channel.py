"""GPU parity of the general Pauli channel (opts.noise = 2, integer energies
(eX, eY, eZ), random scan) against the oracle, bit for bit: the generator,
decodes for several chain layouts and sizes (annealed, beta* != beta_bar),
resumption and thermodynamic integration."""
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


@pytest.mark.parametrize("L,e,p,n", [(2, (1, 1, 1), 0.3, 7), (5, (2, 3, 1), 0.15, 40), (13, (1, 4, 2), 0.1, 20),
                                     (31, (3, 1, 2), 0.2, 3)])
def test_pauli_generator(ctx, L, e, p, n):
    px, py, pz = O.pauli_probs(p, e)
    syn, tc = O.gen_syndromes_pauli(7100, 4, n, L, px, py, pz)
    gs, gt = ctx.gen_syndromes_pauli(7100, 4, n, L, px, py, pz, like=torch.zeros(1, device="cuda"))
    assert (_np(gs) == syn).all() and (_np(gt) == tc).all()


@pytest.mark.parametrize("L,R,e,anneal", [(3, 1, (2, 3, 1), False), (5, 4, (1, 4, 2), True), (7, 8, (3, 1, 2), False),
                                          (4, 2, (1, 1, 1), False)])
def test_pauli_decode_matches_oracle(ctx, pkg, L, R, e, anneal):
    p, n, sweeps, burn = 0.15, 8, 12, 4
    px, py, pz = O.pauli_probs(p, e)
    syn, _ = O.gen_syndromes_pauli(7200 + L, 0, n, L, px, py, pz)
    kw = dict(anneal_stages=2, anneal_beta0=0.5) if anneal else {}
    opts = pkg.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, beta_scale=0.9, scan=1, noise=2,
                    pauli_energy=e, **kw)
    out = ctx.decode_ex(torch.from_numpy(syn).cuda(), L, p, opts, seed=88, id0=6)
    torch.cuda.synchronize()
    for i in range(n):
        ref = O.decode_one(L, p, 4, R, sweeps, 88, 6 + i, syn[i], burn_in=burn, beta_scale=0.9, scan=1, noise=2,
                           energy=e, **kw)
        assert int(_np(out["cls"])[i]) == ref["cls"]
        assert (_np(out["class_sum"])[i] == ref["class_sum"]).all()
        assert (_np(out["log_ratio"])[i] == ref["log_ratio"]).all()
        assert (_np(out["chain_sum"])[i] == ref["chain_sum"]).all()
        assert (_np(out["chain_n"])[i] == ref["chain_n"]).all()
        fr = _np(out["chain_frames"])[i]
        assert (fr[:, 0, :] == O.pack_bits(ref["frames_x"])).all()
        assert (fr[:, 1, :] == O.pack_bits(ref["frames_z"])).all()


def test_pauli_resume_and_ti(ctx, pkg):
    L, p, n, e = 3, 0.12, 4, (2, 3, 1)
    px, py, pz = O.pauli_probs(p, e)
    syn, _ = O.gen_syndromes_pauli(7300, 0, n, L, px, py, pz)
    opts = pkg.Opts(chains_per_class=4, n_sweeps=14, burn_in=4, scan=1, noise=2, pauli_energy=e)
    full = ctx.decode_ex(syn, L, p, opts, seed=3)
    a = ctx.decode_ex(syn, L, p, pkg.Opts(**{**opts.__dict__, "n_sweeps": 6}), seed=3)
    b = ctx.decode_ex(syn, L, p, opts, seed=3, sweep_begin=6, init_frames=a["chain_frames"],
                      init_chain_sum=a["chain_sum"])
    for key in ("cls", "class_sum", "chain_sum", "chain_n", "chain_frames"):
        assert (b[key] == full[key]).all(), key
    cls, lz, mean = ctx.decode_ti(syn, L, p, opts, n_beta=5, seed=9, id0=1)
    for i in range(n):
        k, rlz, rmean = O.decode_ti(L, p, 4, 4, 14, 9, 1 + i, syn[i], n_beta=5, burn_in=4, scan=1, noise=2,
                                    energy=e)
        assert cls[i] == k and (mean[i] == rmean).all() and (lz[i] == rlz).all()


def test_pauli_invalid(ctx, pkg):
    syn, _ = O.gen_syndromes(1, 0, 2, 5, 0.1)
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 5, 0.1, pkg.Opts(noise=2, pauli_energy=(1, 2, 1)))           # needs scan = 1
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 5, 0.1, pkg.Opts(noise=2, scan=1, pauli_energy=(0, 2, 1)))
    with pytest.raises(pkg.SurfmcmcError):
        ctx.decode(syn, 5, 0.1, pkg.Opts(noise=2, scan=1, pauli_energy=(1, 9, 1)))
    with pytest.raises(pkg.SurfmcmcError):
        ctx.gen_syndromes_pauli(1, 0, 2, 5, 0.5, 0.2, 0.1)
