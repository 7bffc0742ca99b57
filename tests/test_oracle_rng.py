"""Pins of the oracle's randomness, acceptance table and noise generator (no GPU)."""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle as O

_TRITON_SCRIPT = textwrap.dedent(
    """
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c0, c1, c2, c3, k0p, k1p, out, N: tl.constexpr):
        i = tl.arange(0, N)
        a = tl.load(c0 + i); b = tl.load(c1 + i); c = tl.load(c2 + i); d = tl.load(c3 + i)
        k0 = tl.load(k0p + i); k1 = tl.load(k1p + i)
        r0, r1, r2, r3 = tl.philox_impl(a, b, c, d, k0, k1, 10)
        tl.store(out + i * 4 + 0, r0); tl.store(out + i * 4 + 1, r1)
        tl.store(out + i * 4 + 2, r2); tl.store(out + i * 4 + 3, r3)

    inp = np.frombuffer(sys.stdin.buffer.read(), dtype=np.uint32).reshape(6, -1)
    N = inp.shape[1]
    t = [torch.from_numpy(inp[j].copy()) for j in range(6)]
    out = torch.zeros(N * 4, dtype=torch.uint32)
    k[(1,)](t[0], t[1], t[2], t[3], t[4], t[5], out, N=N)
    sys.stdout.buffer.write(out.numpy().tobytes())
    """
)


def test_philox_matches_independent_implementation():
    """Philox4x32-10 of the oracle against triton's implementation of the same
    published generator, run by triton's CPU interpreter."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    N = 64
    inp = rng.integers(0, 2 ** 32, size=(6, N), dtype=np.uint64).astype(np.uint32)
    inp[:, 0] = 0
    inp[:, 1] = 0xFFFFFFFF
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=inp.tobytes(), capture_output=True,
                          timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr.decode()[-300:])
    ref = np.frombuffer(proc.stdout, dtype=np.uint32).reshape(N, 4)
    for i in range(N):
        got = O.philox(inp[0:4, i], inp[4:6, i])
        assert (got == ref[i]).all(), i


def test_philox_uniformity():
    # chi^2 of the top 4 bits of 64k words: 16 cells
    words = np.array([O.philox([i, 3, 5, 7], [11, 13]) for i in range(16384)], np.uint32).ravel()
    cells = np.bincount(words >> 28, minlength=16)
    e = len(words) / 16
    chi2 = ((cells - e) ** 2 / e).sum()
    assert chi2 < 45  # 15 dof, p ~ 1e-4


@pytest.mark.parametrize("Cn", [1, 4, 16, 24, 32, 64, 80])
def test_uniform_less_is_comparison(Cn):
    """The digit-by-digit comparison equals u < T on the assembled u."""
    rng = np.random.default_rng(Cn)
    for _ in range(300):
        seed = int(rng.integers(0, 2 ** 63))
        s, t = int(rng.integers(0, 2 ** 32)), int(rng.integers(0, 2 ** 20))
        col, m, c = int(rng.integers(0, 4)), int(rng.integers(0, 300)), int(rng.integers(0, Cn))
        u = O.chain_uniform(seed, s, t, col, m, c, Cn)
        for T in (int(rng.integers(0, 2 ** 32)), u, u + 1, max(u - 1, 0), 0, 2 ** 32, 2 ** 32 - 1,
                  (u & 0xFFFF0000) | 0x8000):
            assert O.chain_uniform_less(seed, s, t, col, m, c, Cn, T) == (u < T)


def test_plane_width():
    assert [O.plane_width(c) for c in (1, 2, 3, 4, 5, 16, 17, 32, 33, 64, 128)] == \
        [1, 2, 4, 4, 8, 16, 32, 32, 32, 32, 32]


def test_chain_uniforms_independent():
    # different chains and proposals draw different, uncorrelated uniforms
    Cn = 64
    u = np.array([[O.chain_uniform(99, 5, t, 1, 3, c, Cn) for c in range(Cn)] for t in range(200)], np.float64)
    u /= 2.0 ** 32
    assert abs(u.mean() - 0.5) < 0.02
    cc = np.corrcoef(u.T)
    off = cc[~np.eye(Cn, dtype=bool)]
    assert np.abs(off).max() < 0.35
    assert abs(off.mean()) < 0.02


@pytest.mark.parametrize("p", [0.01, 0.1, 0.13, 0.15, 0.189, 0.5])
def test_thresholds_closed_form(p):
    # Eq. 2: e^{-beta_bar} = (p/3)/(1-p); T[d] = floor(r^d 2^32)
    T, bb = O.thresholds(p)
    r = (p / 3) / (1 - p)
    assert abs(bb - (-math.log(r))) < 1e-12
    for d in range(1, 5):
        assert abs(int(T[d]) - r ** d * 2 ** 32) <= 1.0 + 1e-9 * r ** d * 2 ** 32
    assert all(T[d] > T[d + 1] for d in range(1, 4))


def test_thresholds_limits():
    T, _ = O.thresholds(0.75)                     # r = 1: beta_bar = 0, accept all
    assert all(int(T[d]) == 2 ** 32 for d in range(1, 5))
    T, _ = O.thresholds(0.1, beta_scale=0.0)      # beta* = 0
    assert all(int(T[d]) == 2 ** 32 for d in range(1, 5))
    T, _ = O.thresholds(0.1, beta_scale=float("inf"))   # beta* -> infinity
    assert all(int(T[d]) == 0 for d in range(1, 5))
    T2, _ = O.thresholds(0.1, beta_scale=2.0)
    r = (0.1 / 3) / 0.9
    assert abs(int(T2[1]) - r ** 2 * 2 ** 32) <= 2


@pytest.mark.parametrize("p", [0.05, 0.15, 0.75])
def test_noise_frequencies(p):
    """Eq. 1 with p_x = p_y = p_z = p/3 (Sec. II): binomial check per Pauli."""
    L = 13
    n_syn = 400
    cnt = np.zeros(4)
    for i in range(n_syn):
        ex, ez = O.gen_error(2024, i, L, p)
        cnt[0] += ((ex == 1) & (ez == 0)).sum()
        cnt[1] += ((ex == 1) & (ez == 1)).sum()
        cnt[2] += ((ex == 0) & (ez == 1)).sum()
        cnt[3] += ((ex == 0) & (ez == 0)).sum()
    N = n_syn * O.nq(L)
    for j, pj in enumerate([p / 3, p / 3, p / 3, 1 - p]):
        sd = math.sqrt(N * pj * (1 - pj))
        assert abs(cnt[j] - N * pj) < 5 * sd + 1


def test_gen_syndromes_consistent():
    L, p = 5, 0.15
    syn, tc = O.gen_syndromes(1001, 0, 50, L, p)
    for i in range(50):
        ex, ez = O.gen_error(1001, i, L, p)
        assert (O.syndrome(L, ex, ez) == syn[i]).all()
        assert O.class_code(L, ex, ez) == tc[i]
    syn2, tc2 = O.gen_syndromes(1001, 10, 5, L, p)
    assert (syn2 == syn[10:15]).all() and (tc2 == tc[10:15]).all()
    z, _ = O.gen_syndromes(1, 0, 3, L, 0.0)
    assert z.sum() == 0
