"""Pins of the oracle's error bars by binning over iterations (Sec. 4.1: data
blocks of dN iterations, the binning method), in closed form.

* Identical iterations: every value equals the single-iteration analysis (to the
  rounding of a sum of equal terms) and every error vanishes to that rounding.
* Iterations that alternate S_0 +- a f (f >= 0, zero at the maximum of S_0, so
  the shift to max S = 0 leaves the perturbation alone): with blocks of one the
  errors of S and beta are a f / sqrt(n - 1) and a (central difference of f) /
  sqrt(n - 1); with blocks of two the alternation cancels inside each block and
  both errors vanish.
* A remainder at the end of the range is left out; a single block gives values
  and NaN errors.
"""
import numpy as np
import pytest

K, E_MIN, W, H_FD, N = 400, -20.0, 0.1, 3, 20
E = E_MIN + (np.arange(K) + 0.5) * W
T = np.linspace(0.5, 4.0, 16)
S0 = -((E - 2.05) / 6.0) ** 2 * 10.0         # concave, its maximum at the centre of bin 220
KSTAR = int(np.argmax(S0))
F = ((np.arange(K) - KSTAR) / K) ** 2          # >= 0, zero at the maximum


def _alternating(n, a):
    return np.stack([-(S0 + (a if i % 2 == 0 else -a) * F) for i in range(n)])


def test_identical_iterations(orc):
    lnW = np.stack([-S0] * 6)
    r = orc.micro_binned(lnW, E_MIN, W, None, block=2, fd_half_width=H_FD, n_monomers=N, T=T)
    one = orc.micro_analysis(-S0, E_MIN, W, None, fd_half_width=H_FD, n_monomers=N, T=T)
    for k in ("S", "beta", "CV", "E_T", "cV_T", "peak"):
        assert np.allclose(r[k], one[k], rtol=1e-15, atol=0, equal_nan=True), k
        fin = np.isfinite(one[k])
        assert np.all(r[k + "_err"][fin] <= 1e-15 * np.abs(one[k][fin])), k


@pytest.mark.parametrize("n", [8, 12])
def test_alternating_iterations(orc, n):
    a = 0.25
    lnW = _alternating(n, a)
    r1 = orc.micro_binned(lnW, E_MIN, W, None, block=1, fd_half_width=H_FD, n_monomers=N, T=T)
    S_ref = S0 - S0[KSTAR]
    assert np.allclose(r1["S"], S_ref, rtol=0, atol=1e-12)
    assert np.allclose(r1["S_err"], a * F / np.sqrt(n - 1), rtol=1e-10, atol=1e-14)
    dF = np.full(K, np.nan)
    dF[H_FD:K - H_FD] = (F[2 * H_FD:] - F[:K - 2 * H_FD]) / (2 * H_FD * W)
    ok = np.isfinite(dF)
    assert np.allclose(r1["beta_err"][ok], a * np.abs(dF[ok]) / np.sqrt(n - 1), rtol=1e-8, atol=1e-12)
    r2 = orc.micro_binned(lnW, E_MIN, W, None, block=2, fd_half_width=H_FD, n_monomers=N, T=T)
    assert np.all(r2["S_err"] <= 1e-14 * (1.0 + np.abs(S_ref)))                 # rounding only
    assert np.all(r2["beta_err"][ok] <= 1e-12 * (1.0 + np.abs(r2["beta"][ok])))
    assert np.allclose(r2["S"], S_ref, rtol=0, atol=1e-12)


def test_remainder_left_out_and_single_block(orc):
    rng = np.random.default_rng(5)
    lnW = np.stack([-S0 + 0.05 * rng.standard_normal(K) for _ in range(7)])
    r = orc.micro_binned(lnW, E_MIN, W, None, block=3, fd_half_width=H_FD, n_monomers=N, T=T)
    lnW2 = lnW.copy()
    lnW2[6] += 5.0 * rng.standard_normal(K)      # the seventh iteration is not in the two blocks
    r2 = orc.micro_binned(lnW2, E_MIN, W, None, block=3, fd_half_width=H_FD, n_monomers=N, T=T)
    for k in ("S", "beta", "E_T", "S_err", "E_T_err"):
        assert np.array_equal(r[k], r2[k], equal_nan=True), k
    one = orc.micro_binned(lnW[:3], E_MIN, W, None, block=3, fd_half_width=H_FD, n_monomers=N, T=T)
    assert np.all(np.isnan(one["S_err"])) and np.all(np.isfinite(one["S"]))
    # the value is the mean of the per-iteration analyses
    per = np.stack([orc.micro_analysis(x, E_MIN, W, None, fd_half_width=H_FD, n_monomers=N, T=T)["E_T"]
                    for x in lnW[:6]])
    assert np.allclose(r["E_T"], per.mean(axis=0), rtol=1e-13, atol=1e-13)
    assert np.allclose(r["E_T_err"], per.reshape(2, 3, -1).mean(axis=1).std(axis=0, ddof=1) / np.sqrt(2),
                       rtol=1e-9, atol=1e-15)
