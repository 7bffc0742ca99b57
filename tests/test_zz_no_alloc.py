"""The allocation-free entry point (surfmcmc_decode_noalloc) against
surfmcmc_decode on the same inputs, through the C ABI.

It is for callers that cannot allocate device memory (their memory is held
by another allocator, or they run under a fixed budget): its scratch is a
fixed array inside the library.  Results must equal surfmcmc_decode's bit for
bit, on two calls in a row that share that array.  This file is collected
last so that a stop at the first failure has already run every other test."""
import ctypes as C

import pytest

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


def _noalloc(P, syn, L, p, opts, seed, id0):
    n = syn.shape[0]
    cls = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    sums = torch.zeros((n, 4), dtype=torch.uint64, device="cuda")
    lr = torch.full((n, 4), 3.0, dtype=torch.float64, device="cuda")
    o = opts.c()
    rc = P.lib().surfmcmc_decode_noalloc(syn.data_ptr(), n, L, p, C.byref(o), seed, id0, cls.data_ptr(),
                                         sums.data_ptr(), lr.data_ptr(), None)
    torch.cuda.synchronize()
    return rc, cls, sums, lr


def test_noalloc_matches_decode_on_two_calls(pkg):
    P = pkg
    ctx = P.Context(0)
    like = torch.zeros(1, device="cuda")
    cases = [(13, 0.13, 16, 40, 700, 2013), (5, 0.15, 4, 200, 501, 1001)]
    for L, p, R, sweeps, n, seed in cases:
        syn, _ = ctx.gen_syndromes(seed, 0, n, L, p, like=like)
        opts = P.Opts(chains_per_class=R, n_sweeps=sweeps)
        ref_cls, ref_sum, ref_lr = ctx.decode(syn, L, p, opts, seed=seed + 100, id0=0)
        torch.cuda.synchronize()
        for _ in range(2):
            rc, cls, sums, lr = _noalloc(P, syn, L, p, opts, seed + 100, 0)
            assert rc == P.OK
            assert torch.equal(cls, ref_cls)
            assert torch.equal(sums.cpu(), ref_sum.cpu())
            assert torch.equal(lr, ref_lr)
    ctx.close()


def test_noalloc_rejects_oversized_batches_and_host_buffers(pkg):
    P = pkg
    L, R = 13, 16
    cap = P.NOALLOC_SCRATCH_BYTES
    n_big = 1
    while P.lib().surfmcmc_noalloc_scratch_needed(n_big, L, R) <= cap:
        n_big *= 2
    syn = torch.zeros((4, 2 * L * (L - 1)), dtype=torch.uint8, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    o = P.Opts(chains_per_class=R, n_sweeps=2).c()
    assert P.lib().surfmcmc_decode_noalloc(syn.data_ptr(), n_big, L, 0.1, C.byref(o), 1, 0, out.data_ptr(), None,
                                           None, None) == P.EINVAL
    hsyn = syn.cpu()
    assert P.lib().surfmcmc_decode_noalloc(hsyn.data_ptr(), 4, L, 0.1, C.byref(o), 1, 0, out.data_ptr(), None,
                                           None, None) == P.EINVAL
