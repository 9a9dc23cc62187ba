"""Pins of the oracle's free energy (Eq. 7) and Maxwell construction.

An entropy made of two concave parabolas S1 = -(E - a)^2 / 2c and
S2 = h - (E - b)^2 / 2c, S = max(S1, S2), has the common tangent of slope
beta_c = h / (b - a) touching at E1 = a - c beta_c and E2 = b - c beta_c; the hull
exceeds S by min((E - E1)^2, (E - E2)^2) / 2c, so the free-energy barrier is
(b - a)^2 / (8 c) / (beta_c N) and the latent heat (b - a) / N: closed forms.
"""
import numpy as np
import pytest

E_MIN, W, K, N = -0.05, 0.1, 100, 10


def _E():
    return E_MIN + (np.arange(K) + 0.5) * W


def _two_parabolas(a=2.0, b=6.0, c=2.0, h=1.0):
    E = _E()
    return np.maximum(-(E - a) ** 2 / (2 * c), h - (E - b) ** 2 / (2 * c))


def test_two_parabolas_closed_form(orc):
    a, b, c, h = 2.0, 6.0, 2.0, 1.0
    f, r = orc.maxwell(_two_parabolas(a, b, c, h), E_MIN, W, N)
    beta_c = h / (b - a)
    assert r["found"] == 1.0
    assert r["beta_c"] == pytest.approx(beta_c, rel=1e-12)
    assert r["eps_1"] == pytest.approx((a - c * beta_c) / N, rel=1e-12)
    assert r["eps_2"] == pytest.approx((b - c * beta_c) / N, rel=1e-12)
    assert r["latent"] == pytest.approx((b - a) / N, rel=1e-12)
    assert r["barrier"] == pytest.approx((b - a) ** 2 / (8 * c) / (beta_c * N), rel=1e-9)
    S = _two_parabolas(a, b, c, h)
    assert np.allclose(f, (_E() - S / beta_c) / N, rtol=1e-12, atol=1e-12)
    # the two coexisting states have equal free energy
    assert f[15] == pytest.approx(f[55], rel=1e-9, abs=1e-12)


def test_linear_term_shifts_beta_only(orc):
    S = _two_parabolas()
    _, r0 = orc.maxwell(S, E_MIN, W, N)
    _, r1 = orc.maxwell(S + 0.7 * _E(), E_MIN, W, N)
    assert r1["beta_c"] == pytest.approx(r0["beta_c"] + 0.7, rel=1e-12)
    assert r1["latent"] == pytest.approx(r0["latent"], rel=1e-12)
    assert r1["barrier"] * r1["beta_c"] == pytest.approx(r0["barrier"] * r0["beta_c"], rel=1e-9)


def test_concave_entropy_has_no_transition(orc):
    E = _E()
    S = -(E - 4.0) ** 2 / 3.0
    f, r = orc.maxwell(S, E_MIN, W, N)
    assert r["found"] == 0.0 and np.isnan(r["beta_c"]) and np.all(np.isnan(f))
    f, r = orc.maxwell(S, E_MIN, W, N, beta_c=0.8)        # a given beta_c: free energy only
    assert r["found"] == 0.0 and r["beta_c"] == 0.8
    assert np.allclose(f, (E - S / 0.8) / N, rtol=1e-14, atol=1e-14)


def test_tolerances_filter_the_construction(orc):
    S = _two_parabolas()
    _, r = orc.maxwell(S, E_MIN, W, N, tol_L=0.41)          # latent heat 0.4 < Tol_L
    assert r["found"] == 0.0
    _, r = orc.maxwell(S, E_MIN, W, N, tol_L=0.39)
    assert r["found"] == 1.0
    _, r = orc.maxwell(S, E_MIN, W, N, tol_beta=1e3)         # beta never rises that much
    assert r["found"] == 0.0


def test_largest_intruder_wins_and_holes_are_skipped(orc):
    E = _E()
    S = _two_parabolas()
    S = S + np.where(E > 8.0, 0.05 * np.exp(-((E - 8.6) ** 2) / 0.02), 0.0)   # a small second S-bend
    _, r = orc.maxwell(S, E_MIN, W, N)
    assert r["latent"] == pytest.approx(0.4, rel=1e-12)
    holes = S.copy()
    holes[[3, 30, 40, 70]] = np.nan                            # unvisited bins
    _, rh = orc.maxwell(holes, E_MIN, W, N)
    assert rh["latent"] == pytest.approx(0.4, rel=1e-12)
    assert rh["beta_c"] == pytest.approx(r["beta_c"], rel=1e-12)


def test_negative_temperature_bend_is_no_transition(orc):
    # the mirror image of the two parabolas (E -> const - E): its common tangent
    # falls (beta_c < 0, a negative temperature) and is not a transition; the
    # unmirrored entropy on the same bins gives the closed-form beta_c > 0
    E = _E()
    S = _two_parabolas()
    f, r = orc.maxwell(S[::-1].copy(), E_MIN, W, N)
    assert r["found"] == 0.0 and np.isnan(r["beta_c"]) and np.all(np.isnan(f))
    _, r = orc.maxwell(S, E_MIN, W, N)
    assert r["found"] == 1.0 and r["beta_c"] > 0.0
