"""GPU parity of the early-stop network: the tensor-core forward pass and the
gradient against the float64 network oracle that rounds weights, inputs and
activations to bfloat16 at the same points.

Tolerances.  Forward: both sides round the same tensors to bfloat16; they
differ by the float32 (tensor-core) against float64 accumulation, which moves
a stored activation by one bfloat16 step (2^-8 relative) where the exact value
lies within ~1e-6 of a rounding boundary.  Log-probabilities therefore agree to
~1e-3; the bar is max |difference| < 2e-2 and mean < 2e-3.  Gradient: the GPU
additionally stores the back-propagated gradients in bfloat16 (relative error
2^-9 each), so per layer the relative L2 error of the gradient must be
< 3e-2 and its cosine with the oracle's > 0.999.
"""
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


def _params(seed):
    rng = np.random.default_rng(seed)
    p = cnn.init_params(seed)
    return p + rng.normal(0, 0.05, size=p.shape)   # nonzero biases, some dead ReLUs


def _layer_slices():
    out, off = [], 0
    for i in range(5):
        ci, co = cnn.CHANNELS[i], cnn.CHANNELS[i + 1]
        out.append(("w%d" % (i + 1), slice(off, off + co * 9 * ci)))
        off += co * 9 * ci
        out.append(("b%d" % (i + 1), slice(off, off + co)))
        off += co
    return out


def _forward_check(gpu, ref):
    d = np.abs(gpu.astype(np.float64) - ref)
    assert d.max() < 2e-2, d.max()
    assert d.mean() < 2e-3, d.mean()


# L = 3 (the smallest network size), an even L, and L = 31 (the largest:
# widest input strips and halo tiles, the longest middle lines)
@pytest.mark.parametrize("L,n,seed", [(3, 5, 1), (4, 9, 4), (5, 13, 2), (9, 7, 3), (31, 3, 5)])
def test_forward_parity_small(pkg, ctx, L, n, seed):
    syn, _ = O.gen_syndromes(700 + seed, 0, n, L, 0.15)
    p = _params(seed)
    net = pkg.Network(ctx, L, max_batch=64)
    net.set_params(p.astype(np.float32))
    lp = net.forward(syn)
    ref = cnn.forward(p.astype(np.float32).astype(np.float64), syn, L, bf16=True)
    _forward_check(lp, ref)
    net.close()


def test_forward_parity_many_tiles(pkg, ctx):
    """L = 17, 1024 syndromes: 2312 position tiles, many per block, so both
    accumulators and every pipeline stage are reused; the oracle checks a
    sample of syndromes spread over the batch, including the last."""
    L, n = 17, 1024
    syn, _ = O.gen_syndromes(4003, 0, n, L, 0.13)
    p = _params(11)
    net = pkg.Network(ctx, L, max_batch=n)
    net.set_params(p.astype(np.float32))
    dev = torch.from_numpy(syn).cuda()
    lp = net.forward(dev).cpu().numpy()
    idx = np.array(sorted(set(np.linspace(0, n - 1, 20).astype(int).tolist())))
    ref = cnn.forward(p.astype(np.float32).astype(np.float64), syn[idx], L, bf16=True)
    _forward_check(lp[idx], ref)
    net.close()


def test_forward_batching_and_buffers(pkg, ctx):
    """Results do not depend on the batch a syndrome is in (rows of a tile are
    independent) nor on host or device buffers: bit-identical."""
    L, n = 7, 300
    syn, _ = O.gen_syndromes(4100, 0, n, L, 0.12)
    p = _params(5).astype(np.float32)
    a = pkg.Network(ctx, L, max_batch=n)
    b = pkg.Network(ctx, L, max_batch=64)
    a.set_params(p)
    b.set_params(torch.from_numpy(p).cuda())
    la = a.forward(syn)
    lb = b.forward(torch.from_numpy(syn).cuda()).cpu().numpy()
    lc = a.forward(syn[123:124])
    assert (la == lb).all()
    assert (la[123:124] == lc).all()
    assert np.allclose(np.exp(la).sum(1), 1.0, atol=1e-5)
    assert (b.get_params() == p).all()
    a.close()
    b.close()


# element-wise gradient tolerance relative to the sum of the terms' absolute
# values: six bf16 steps (2^-8 each)
GRAD_REL = 6 * 2.0 ** -8


@pytest.mark.parametrize("L,n,seed", [(5, 7, 21), (6, 11, 25), (9, 37, 22), (17, 64, 23), (31, 4, 24)])
def test_gradient_parity(pkg, ctx, L, n, seed):
    rng = np.random.default_rng(seed)
    syn, _ = O.gen_syndromes(800 + seed, 0, n, L, 0.14)
    q = rng.dirichlet(np.ones(4) * 0.5, size=n)
    p = _params(seed).astype(np.float32)
    net = pkg.Network(ctx, L, max_batch=n)
    net.set_params(p)
    loss, g = net.gradient(syn, q.astype(np.float32))
    rl, rg = cnn.loss_and_grad(p.astype(np.float64), syn, L, q, bf16=True)
    mag = cnn.grad_magnitude(p.astype(np.float64), syn, L, q, bf16=True)
    assert abs(loss - rl) < 1e-3 * max(1.0, abs(rl)), (loss, rl)
    for name, sl in _layer_slices():
        a, b = g[sl].astype(np.float64), rg[sl]
        # element by element: every term of a gradient is a product of
        # stored factors, and the GPU stores the back-propagated gradients
        # (and the activations) in bf16, 2^-9 relative each, with up to four
        # stores between the loss and the first layer's weights; float32
        # accumulation adds ~2^-24 relative.  The bound is taken against the
        # sum of the terms' absolute values (grad_magnitude), since the terms
        # cancel; a dropped or misplaced term moves its element by a sizeable
        # fraction of that sum.
        tol = GRAD_REL * mag[sl] + 1e-6 * mag[sl].max()
        err = np.abs(a - b)
        worst = int(np.argmax(err / np.maximum(tol, 1e-300)))
        assert (err <= tol).all(), (name, worst, a[worst], b[worst], mag[sl][worst],
                                    float((err / np.maximum(mag[sl], 1e-300)).max()))
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.abs(a).max() < 1e-6, name
            continue
        rel = np.linalg.norm(a - b) / nb
        cos = (a @ b) / (np.linalg.norm(a) * nb)
        assert rel < 3e-2 and cos > 0.999, (name, rel, cos)
    # deterministic: fixed-order reductions only
    loss2, g2 = net.gradient(syn, q.astype(np.float32))
    assert loss2 == loss and (g2 == g).all()
    net.close()


def test_wait_time_out_reports_and_recovers(pkg, ctx):
    """The bounded pipeline waits of the network kernels give up cleanly.
    With a bound of one poll (the first poll never suspends) the forward of
    an L = 5 batch finds an mbarrier phase still pending, the block drains
    its copies and MMAs and exits, and the call returns ECUDA with the
    device flag's time-out message; with the default bound the same network
    then gives exactly its earlier result."""
    L, n = 5, 4096
    syn, _ = O.gen_syndromes(4300, 0, n, L, 0.12)
    dsyn = torch.from_numpy(syn).cuda()
    net = pkg.Network(ctx, L, max_batch=n)
    net.set_params(_params(5).astype(np.float32))
    ref = net.forward(dsyn).cpu().numpy()
    net.set_wait_limit(1)
    with pytest.raises(pkg.SurfmcmcError) as e:
        net.forward(dsyn)
    assert e.value.code == pkg.ECUDA and "timed out" in str(e.value)
    net.set_wait_limit(0)
    again = net.forward(dsyn).cpu().numpy()
    assert (again == ref).all()
    net.status()                      # the flag was cleared by the failing call
    net.close()


def test_training_reduces_loss(pkg, ctx):
    """Adam on one fixed batch (one-hot targets of the true classes): the
    loss falls well below its start."""
    L, n = 5, 256
    syn, tc = O.gen_syndromes(4200, 0, n, L, 0.08)
    q = np.eye(4, dtype=np.float32)[tc]
    net = pkg.Network(ctx, L, max_batch=n)
    net.set_params(cnn.init_params(7).astype(np.float32))
    dsyn = torch.from_numpy(syn).cuda()
    dq = torch.from_numpy(q).cuda()
    first = net.train_step(dsyn, dq, 1e-3)
    for _ in range(300):
        last = net.train_step(dsyn, dq, 1e-3)
    assert np.isfinite(last) and last < 0.7 * first, (first, last)
    # the parameters moved and the forward pass agrees with the reported loss
    lp = net.forward(syn)
    assert abs(-(q * lp).sum(1).mean() - net.gradient(syn, q)[0]) < 1e-5
    net.close()


def test_invalid_args(pkg, ctx):
    with pytest.raises(pkg.SurfmcmcError):
        pkg.Network(ctx, 2, 16)
    with pytest.raises(pkg.SurfmcmcError):
        pkg.Network(ctx, 5, 0)
    net = pkg.Network(ctx, 5, max_batch=8)
    syn, _ = O.gen_syndromes(1, 0, 9, 5, 0.1)
    q = np.full((9, 4), 0.25, np.float32)
    with pytest.raises(pkg.SurfmcmcError):
        net.gradient(syn, q)                      # n > max_batch
    with pytest.raises(pkg.SurfmcmcError):
        net.train_step(syn[:4], q[:4], 0.0)       # lr must be > 0
    assert net.forward(syn[:0]).shape == (0, 4)
    net.status()
    net.close()
