"""Input recipes of the benchmark modules (no GPU): the general Pauli
channel's probabilities (Eq. 1 with integer energies: p_P = (1 - p) r^e_P,
sum over P = p) reduce to the named channels."""
import math

import pytest

from paper_1302_2669_gb300.variants_bench import general_channel_probs


@pytest.mark.parametrize("p", [0.01, 0.1, 0.3])
def test_depolarizing_energies_give_p_over_3(p):
    px, py, pz = general_channel_probs(p, (1, 1, 1))
    for v in (px, py, pz):
        assert math.isclose(v, p / 3, rel_tol=1e-12)


@pytest.mark.parametrize("q", [0.02, 0.05, 0.2])
def test_flip_energies_give_independent_flips(q):
    # independent bit and phase flips with probability q: total error
    # probability 1 - (1 - q)^2, X and Z with q (1 - q), Y with q^2
    p = 1 - (1 - q) ** 2
    px, py, pz = general_channel_probs(p, (1, 2, 1))
    assert math.isclose(px, q * (1 - q), rel_tol=1e-10)
    assert math.isclose(pz, q * (1 - q), rel_tol=1e-10)
    assert math.isclose(py, q * q, rel_tol=1e-10)


def test_probabilities_sum_to_p():
    for e in ((2, 3, 1), (1, 4, 2), (3, 1, 2)):
        px, py, pz = general_channel_probs(0.1, e)
        assert math.isclose(px + py + pz, 0.1, rel_tol=1e-12)
        assert px > 0 and py > 0 and pz > 0
