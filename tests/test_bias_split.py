"""The first layer's bias enters the tensor-core GEMM as three bf16 operand
values b1 = bf16(b), b2 = bf16(b - b1), b3 = bf16(b - b1 - b2) multiplied by
constant-one operand columns (the products are exact and summed in float32).
The split is exact, b1 + b2 + b3 == b, for every float32 b with |b| >=
2^-100 (the remainders stay in the normal range), so the bias the network
adds is the float32 master bias itself; for smaller biases the error stays
below 2^-126 in absolute value.  Checked here with
round-to-nearest-even bf16 written from its definition (the nearest
8-significant-bit value, ties to an even last bit), independently of the
CUDA conversion."""
import numpy as np


def bf16_rne(x):
    """float32 array -> nearest bf16 value (ties to even), as float32."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def test_bf16_rne_reference_values():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to the even bf16 (1.0);
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to 1 + 2^-6
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, -2.5, 3.0e-3],
                    dtype=np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, None], dtype=object)
    got = bf16_rne(vals)
    for g, w in zip(got[:5], want[:5]):
        assert float(g) == float(w)
    # the nearest 8-bit-significand value by brute force for the last one
    x = float(vals[5])
    e = int(np.floor(np.log2(abs(x))))
    cand = [m * 2.0 ** (e - 7) for m in range(2 ** 7, 2 ** 8 + 1)]
    best = min(cand, key=lambda c: (abs(c - x), int(round(c / 2.0 ** (e - 7))) % 2))
    assert float(got[5]) == best


def test_three_part_split_is_exact():
    rng = np.random.default_rng(20240)
    n = 200_000
    mant = rng.integers(2 ** 23, 2 ** 24, size=n).astype(np.float64)
    expo = rng.integers(-100, 100, size=n)
    sign = rng.choice([-1.0, 1.0], size=n)
    b = (sign * mant * np.exp2(expo - 23)).astype(np.float32)
    edge = np.array([1.0, -1.0, 0.5 + 2.0 ** -24, 1.0 - 2.0 ** -24, 3.0e38, 2.0 ** -100, 0.0, 0.1, -0.7],
                    dtype=np.float32)
    b = np.concatenate([b, edge])
    b1 = bf16_rne(b)
    r1 = (b - b1).astype(np.float32)
    b2 = bf16_rne(r1)
    r2 = (r1 - b2).astype(np.float32)
    b3 = bf16_rne(r2)
    assert (b3 == r2).all()   # the remainder already has at most 8 significant bits
    total = b1.astype(np.float64) + b2.astype(np.float64) + b3.astype(np.float64)
    assert (total == b.astype(np.float64)).all()


def test_three_part_split_tiny_biases():
    rng = np.random.default_rng(20241)
    n = 100_000
    mant = rng.integers(2 ** 23, 2 ** 24, size=n).astype(np.float64)
    b = (mant * np.exp2(rng.integers(-126, -100, size=n) - 23)).astype(np.float32)
    b1 = bf16_rne(b)
    b2 = bf16_rne((b - b1).astype(np.float32))
    b3 = bf16_rne((b - b1 - b2).astype(np.float32))
    err = np.abs(b1.astype(np.float64) + b2.astype(np.float64) + b3.astype(np.float64) - b.astype(np.float64))
    assert err.max() < 2.0 ** -126
