"""Host logic of the early-stop study, on the CPU: checkpoint sweeps, the
replay of the stop rule on per-checkpoint decisions (a syndrome stops at the
first checkpoint before the last where the network's margin exceeds tau and
its argmax equals the chains' decision; otherwise it runs to the end), and
the calibration that keeps the smallest tau whose error rate is within one
binomial sigma of the long chains'."""
import math
from types import SimpleNamespace

import numpy as np

from paper_1302_2669_gb300 import early_stop as ES


def test_checkpoint_marks():
    o = SimpleNamespace(burn_in=100, n_sweeps=1000)
    assert ES.checkpoint_marks(o, 300) == [400, 700, 1000]
    o = SimpleNamespace(burn_in=0, n_sweeps=900)
    assert ES.checkpoint_marks(o, 300) == [300, 600, 900]
    o = SimpleNamespace(burn_in=50, n_sweeps=60)
    assert ES.checkpoint_marks(o, 100) == [60]   # no intermediate checkpoint


def _lp(rows):
    return np.log(np.asarray(rows, dtype=np.float64))


def test_replay_stop_rule():
    marks = [10, 20, 30, 40]
    # network log-probabilities: items 0-2 confident in class 2 (margin
    # log(0.7/0.1)), item 3 unsure, item 4 a tie between classes 0 and 1
    logprob = _lp([[0.1, 0.1, 0.7, 0.1],
                   [0.1, 0.1, 0.7, 0.1],
                   [0.1, 0.1, 0.7, 0.1],
                   [0.3, 0.2, 0.3 - 1e-3, 0.2 + 1e-3],
                   [0.4, 0.4, 0.1, 0.1]])
    dec = np.array([[2, 2, 2, 2],    # agrees at once: stops at the first checkpoint
                    [1, 0, 2, 1],    # agrees at the third
                    [1, 1, 1, 3],    # never agrees before the last: runs to the end
                    [0, 0, 0, 0],    # margin too small
                    [0, 0, 0, 1]],   # zero margin
                   dtype=np.int32)
    tau = 1.0
    cls, sw = ES.replay(logprob, dec, marks, tau)
    assert cls.tolist() == [2, 2, 3, 0, 1]
    assert sw.tolist() == [10, 30, 40, 40, 40]
    # the last checkpoint never stops early: a decision there is the full run
    cls, sw = ES.replay(logprob, dec, marks, float("inf"))
    assert (cls == dec[:, -1]).all() and (sw == 40).all()
    # a negative threshold lets the zero-margin tie stop where argmax (the
    # first of the tied classes, 0) agrees
    cls, sw = ES.replay(logprob, dec, marks, -1.0)
    assert cls[4] == 0 and sw[4] == 10
    # the margin is compared strictly: tau equal to the margin does not stop
    margin = float(np.float32(np.log(0.7)) - np.float32(np.log(0.1)))
    _, sw = ES.replay(logprob, dec, marks, margin)
    assert sw[0] == 40
    _, sw = ES.replay(logprob, dec, marks, np.nextafter(np.float32(margin), np.float32(0)))
    assert sw[0] == 10


def test_calibrate_picks_smallest_tau_not_above_the_long_chains():
    rng = np.random.default_rng(5)
    n, marks = 4000, [10, 20]
    true = rng.integers(0, 4, size=n).astype(np.int32)
    long_dec = true.copy()
    wrong = rng.random(n) < 0.05                      # long chains: 5% errors
    long_dec[wrong] = (true[wrong] + 1) % 4
    early = long_dec.copy()
    flip = rng.random(n) < 0.5                        # the first checkpoint is often wrong
    early[flip] = (long_dec[flip] + 2) % 4
    dec = np.stack([early, long_dec], axis=1)
    # the network agrees with the early decision; confident (margin 3) where
    # that decision is right, unsure (margin 0.5) where it is wrong
    lp = np.full((n, 4), -10.0)
    right = early == true
    lp[np.arange(n), early] = np.where(right, -0.05, -0.5)
    other = (early + 1) % 4
    lp[np.arange(n), other] = np.where(right, -3.05, -1.0)
    best, ler_long, sigma, rows = ES.calibrate(lp, dec, marks, true, [0.0, 1.0, 2.0, 4.0])
    assert abs(ler_long - (long_dec != true).mean()) < 1e-12
    assert abs(sigma - math.sqrt(ler_long * (1 - ler_long) / n)) < 1e-12
    lers = {r["tau"]: r["ler"] for r in rows}
    assert lers[0.0] > ler_long + sigma               # tau = 0 stops the wrong ones too
    assert lers[1.0] <= ler_long + sigma               # only the confident, right ones stop
    assert best == 1.0
    sweeps = [r["mean_sweeps"] for r in sorted(rows, key=lambda r: r["tau"])]
    assert all(a <= b for a, b in zip(sweeps, sweeps[1:]))   # a larger tau never stops earlier
    assert lers[4.0] == ler_long                       # nothing stops: the long chains' rate
    assert lers[1.0] <= ler_long                       # the default margin: no excess at all
    # with a margin of one sigma tau = 0 is still out
    assert ES.calibrate(lp, dec, marks, true, [0.0, 1.0, 2.0, 4.0], margin_sigma=1.0)[0] == 1.0
