"""Pins of the oracle's jackknife combination (Sec. 4.1: error bars from blocks of
the data; the blocks here are groups of walkers), in closed form.

* Three replicates (1, 2, 4), worked by hand: mean 7/3, squared deviations
  16/9 + 1/9 + 25/9 = 14/3, times (n - 1)/n = 2/3 gives 28/9, error sqrt(28)/3.
* The estimate is a block mean: its leave-one-out replicates are
  v_b = (sum x - x_b)/(n - 1), so v_b - vbar = -(x_b - xbar)/(n - 1) and the
  jackknife error equals the standard error of the mean of the blocks,
  sqrt(sum (x_b - xbar)^2 / (n (n - 1))).  A factor n/(n - 1) in place of
  (n - 1)/n, or a missing one, fails this by the square of that factor.
* Linear in the replicates: err(a v + c) = |a| err(v); constant replicates give 0.
* Fewer than two replicates give NaN; a NaN replicate spoils only its column.
"""
import math

import numpy as np


def test_three_blocks_by_hand(orc):
    assert math.isclose(orc.jackknife([1.0, 2.0, 4.0]), math.sqrt(28.0) / 3.0, rel_tol=1e-15)


def test_block_mean_gives_the_standard_error_of_the_mean(orc):
    rng = np.random.default_rng(11)
    for n in (2, 3, 16, 64):
        x = rng.normal(3.0, 2.0, size=(n, 5))
        reps = (x.sum(0)[None, :] - x) / (n - 1)
        sem = x.std(0, ddof=1) / np.sqrt(n)
        assert np.allclose(orc.jackknife(reps), sem, rtol=1e-12, atol=0), n


def test_linear_in_the_replicates(orc):
    rng = np.random.default_rng(12)
    v = rng.normal(size=(10, 7))
    base = orc.jackknife(v)
    assert np.allclose(orc.jackknife(-2.5 * v + 4.0), 2.5 * base, rtol=1e-12)
    assert np.all(orc.jackknife(np.full((6, 3), 1.7)) == 0.0)


def test_degenerate_cases(orc):
    assert math.isnan(orc.jackknife([3.0]))
    v = np.arange(12.0).reshape(4, 3)
    v[2, 1] = np.nan
    err = orc.jackknife(v)
    assert np.isnan(err[1]) and np.isfinite(err[0]) and np.isfinite(err[2])
