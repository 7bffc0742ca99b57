"""Pins of the thermodynamic-integration estimate (Eq. 6 with Simpson's rule
over 21 equidistant temperatures, Sec. IV and IV.A)."""
import math

import numpy as np
import pytest

import oracle as O


def test_simpson_exact_on_cubics():
    # composite Simpson integrates polynomials of degree <= 3 exactly
    bb = 2.7
    beta = np.linspace(0, bb, 21)
    coef = np.array([[1.0, -2.0, 0.5, 0.25], [3.0, 0.0, -1.0, 0.1]])
    f = np.array([c[0] + c[1] * beta + c[2] * beta ** 2 + c[3] * beta ** 3 for c in coef])
    I = O.simpson_integral(f, bb)
    exact = [c[0] * bb + c[1] * bb ** 2 / 2 + c[2] * bb ** 3 / 3 + c[3] * bb ** 4 / 4 for c in coef]
    assert np.allclose(I, exact, rtol=1e-13, atol=1e-12)
    with pytest.raises(ValueError):
        O.simpson_integral(f[:, :20], bb)


def test_simpson_error_bound_on_smooth_function():
    # |error| <= (b-a) h^4 max|f''''| / 180
    bb = 3.0
    beta = np.linspace(0, bb, 21)
    f = np.exp(-beta)[None, :]
    h = bb / 20
    I = O.simpson_integral(f, bb)[0]
    assert abs(I - (1 - math.exp(-bb))) <= bb * h ** 4 / 180 + 1e-15


@pytest.mark.parametrize("p,seed", [(0.10, 1), (0.15, 2), (0.2, 3)])
def test_eq6_with_exact_means_at_l3(p, seed):
    """log Z_k(beta_bar) - n_stab log 2 = -int_0^beta_bar <n>_k (Eq. 6): the
    Simpson integral of the exact enumerated means over 21 points reproduces
    the exact log Z_k within the quadrature error."""
    L = 3
    syn, _ = O.gen_syndromes(seed, 0, 1, L, p)
    _, bb = O.thresholds(p)
    grid = np.linspace(0, bb, 21)
    means = np.array([O.exact_class_stats(L, syn[0], b)[1] for b in grid]).T   # [4][21]
    I = O.simpson_integral(means, bb)
    logZ, _ = O.exact_class_stats(L, syn[0], bb)
    lhs = logZ - O.nstab(L) * math.log(2)
    assert np.allclose(-I, lhs, atol=2e-3 * abs(lhs).max())
    # class ratios, which is what the decoder uses
    assert np.allclose(-(I - I[0]), logZ - logZ[0], atol=5e-3)


def test_ti_decode_matches_exact_log_ratios_at_l3():
    """TI from chains (R replicas per class and temperature) against exact
    log Z_k / Z_best by enumeration."""
    L, p, K, R, sweeps, burn = 3, 0.15, 4, 64, 120, 20
    syn, _ = O.gen_syndromes(9, 0, 1, L, p)
    k, lz, mean = O.decode_ti(L, p, K, R, sweeps, 31, 0, syn[0], burn_in=burn)
    _, bb = O.thresholds(p)
    logZ, _ = O.exact_class_stats(L, syn[0], bb)
    exact = logZ - logZ.max()
    assert k == int(np.argmax(logZ))
    assert np.allclose(lz, exact, atol=0.15)
    assert (mean[:, 0] == 0.75 * O.nq(L)).all()
