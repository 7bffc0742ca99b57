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


# (L, p, chains per class, sweeps, burn-in, beta_scale, n, seed): the bench
# size, the small size, a burn-in with a tempered table (the exp path of the
# acceptance table), beta* = 0 (every move accepted), beta* = infinity (no
# uphill move accepted), beta* = beta_bar / 2, and one chain per class
# (plane width 4: eight syndromes share a bundle).
CASES = [(13, 0.13, 16, 40, 0, 1.0, 700, 2013), (5, 0.15, 4, 200, 0, 1.0, 501, 1001),
         (5, 0.12, 4, 60, 20, 0.7, 300, 1201), (5, 0.15, 4, 30, 0, 0.0, 64, 1301),
         (7, 0.10, 4, 30, 10, float("inf"), 64, 1401), (9, 0.14, 8, 50, 5, 0.5, 200, 1501),
         (5, 0.15, 1, 100, 10, 1.0, 333, 1601)]


def test_noalloc_matches_decode_on_two_calls(pkg):
    P = pkg
    ctx = P.Context(0)
    like = torch.zeros(1, device="cuda")
    for L, p, R, sweeps, burn, bs, n, seed in CASES:
        syn, _ = ctx.gen_syndromes(seed, 0, n, L, p, like=like)
        opts = P.Opts(chains_per_class=R, n_sweeps=sweeps, burn_in=burn, beta_scale=bs)
        ref_cls, ref_sum, ref_lr = ctx.decode(syn, L, p, opts, seed=seed + 100, id0=0)
        torch.cuda.synchronize()
        for _ in range(2):
            rc, cls, sums, lr = _noalloc(P, syn, L, p, opts, seed + 100, 0)
            assert rc == P.OK, (L, p, R, bs)
            assert torch.equal(cls, ref_cls), (L, p, R, bs)
            assert torch.equal(sums.cpu(), ref_sum.cpu()), (L, p, R, bs)
            assert torch.equal(lr.isnan(), ref_lr.isnan()), (L, p, R, bs)
            assert torch.equal(lr.nan_to_num(), ref_lr.nan_to_num()), (L, p, R, bs)
    ctx.close()


def test_noalloc_allocates_no_device_memory(pkg):
    """After one warm-up pass (which may load kernel code), further calls,
    one of them close to the scratch capacity, leave the device's free memory
    and torch's reserved memory unchanged."""
    P = pkg
    L, p, R, sweeps = 9, 0.12, 4, 6
    n_max = 1
    while P.lib().surfmcmc_noalloc_scratch_needed(2 * n_max, L, R) <= P.NOALLOC_SCRATCH_BYTES:
        n_max *= 2
    while P.lib().surfmcmc_noalloc_scratch_needed(n_max + 1024, L, R) <= P.NOALLOC_SCRATCH_BYTES:
        n_max += 1024
    assert P.lib().surfmcmc_noalloc_scratch_needed(n_max, L, R) <= P.NOALLOC_SCRATCH_BYTES
    ctx = P.Context(0)
    syn, _ = ctx.gen_syndromes(77, 0, n_max, L, p, like=torch.zeros(1, device="cuda"))
    ctx.close()
    opts = P.Opts(chains_per_class=R, n_sweeps=sweeps)
    small = syn[:100].contiguous()
    outs = {}
    for s in (small, syn):
        n = s.shape[0]
        outs[n] = (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty((n, 4), dtype=torch.uint64,
                                                                                    device="cuda"))
    o = opts.c()

    def call(s):
        cls, sums = outs[s.shape[0]]
        return P.lib().surfmcmc_decode_noalloc(s.data_ptr(), s.shape[0], L, p, C.byref(o), 5, 0, cls.data_ptr(),
                                               sums.data_ptr(), None, None)

    for s in (small, syn):   # warm-up
        assert call(s) == P.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        for s in (small, syn):
            assert call(s) == P.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


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
