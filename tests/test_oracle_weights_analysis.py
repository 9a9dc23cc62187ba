"""Pins of the oracle's Berg recursion and microcanonical analysis.

Berg (Sec. 2.2): from g_acc = 0 one step must equal the paper's naive
recursion W^{n+1} = W^n / H^n on visited bins; a flat histogram must leave the
weights unchanged; unvisited bins keep their slope.
Analysis (Eq. 4-6): central differences are exact on a quadratic entropy, so
beta and C_V have closed forms there; canonical averages of a Gaussian density
of states and of a two-level system are known in closed form; the trimer's
canonical <E>_T follows from a 1-D integral over c.
"""
import numpy as np
import pytest
from scipy import integrate, optimize


def test_first_berg_step_is_naive_recursion(orc):
    rng = np.random.default_rng(1)
    K = 50
    lnW = rng.normal(size=K)
    H = rng.integers(1, 1000, size=K).astype(float)
    new, g, flat = orc.berg_update(H, lnW, np.zeros(K - 1), 0.1)
    naive = lnW - np.log(H)
    assert np.allclose(new - new[0], naive - naive[0], atol=1e-12)
    assert np.allclose(g, H[:-1] * H[1:] / (H[:-1] + H[1:]))


def test_berg_flat_histogram_is_fixed_point(orc):
    K = 30
    lnW = np.cumsum(np.linspace(-1, 1, K))
    new, _, flat = orc.berg_update(np.full(K, 7.0), lnW, np.full(K - 1, 3.0), 0.05)
    assert np.allclose(new, lnW - lnW[0], atol=1e-13)
    assert flat[0] == K and flat[1] == 7.0 and flat[2] == 0.0 and flat[3] == 0.0


def test_berg_unvisited_bins_keep_slope(orc):
    K = 20
    lnW = np.linspace(0, -5, K) ** 2 * 0.1
    H = np.zeros(K)
    H[5:12] = [3, 8, 20, 40, 20, 8, 3]
    new, g, _ = orc.berg_update(H, lnW, np.zeros(K - 1), 0.1)
    d_old, d_new = -np.diff(lnW), -np.diff(new)
    untouched = np.ones(K - 1, bool)
    untouched[5:11] = False
    assert np.allclose(d_new[untouched], d_old[untouched], atol=1e-13)
    assert np.all(g[untouched] == 0)
    # inside the visited window the step is the naive one
    naive = lnW - np.where(H > 0, np.log(np.maximum(H, 1)), 0)
    assert np.allclose(d_new[5:11], -np.diff(naive)[5:11], atol=1e-12)


def test_berg_error_weighting(orc):
    # second step with g_acc from the first: ghat = g0 / (g_acc + g0)
    K = 4
    H1 = np.array([10.0, 10.0, 10.0, 10.0])
    H2 = np.array([10.0, 40.0, 10.0, 10.0])
    lnW, g, _ = orc.berg_update(H1, np.zeros(K), np.zeros(K - 1), 1.0)
    lnW2, g2, _ = orc.berg_update(H2, lnW, g, 1.0)
    g0 = H2[0] * H2[1] / (H2[0] + H2[1])                 # 8
    ghat = g0 / (5.0 + g0)
    assert lnW2[1] - lnW2[0] == pytest.approx(-ghat * np.log(4.0), abs=1e-14)
    assert g2[0] == pytest.approx(13.0)


def test_flatness_statistics(orc):
    H = np.array([0.0, 1.0, 2.0, 3.0, 0.0])
    _, _, f = orc.berg_update(H, np.zeros(5), np.zeros(4), 1.0)
    assert f[0] == 3 and f[1] == 2.0
    assert f[2] == pytest.approx(np.sqrt(2.0 / 3.0) / 2.0)
    assert f[3] == pytest.approx(0.5)


def test_quadratic_entropy_derivatives_exact(orc):
    K, e_min, w = 200, -5.0, 0.05
    Ek = e_min + (np.arange(K) + 0.5) * w
    a, b = 1.3, 0.2
    S = a * Ek - b * Ek ** 2
    for h in (1, 3, 7):
        out = orc.micro_analysis(-S, e_min, w, fd_half_width=h)
        inner = slice(h, K - h)
        beta = a - 2 * b * Ek
        assert np.allclose(out["beta"][inner], beta[inner], rtol=1e-9, atol=1e-9)
        assert np.allclose(out["CV"][inner], beta[inner] ** 2 / (2 * b), rtol=1e-7, atol=1e-9)
        assert np.all(np.isnan(out["beta"][:h])) and np.all(np.isnan(out["beta"][K - h:]))
        assert np.nanmax(out["S"]) == 0.0


def test_reweighted_entropy_uses_histogram(orc):
    K = 40
    lnW = np.linspace(0, 3, K)
    H = np.exp(np.sin(np.arange(K) / 5.0)) * 100
    H[[0, 1, 39]] = 0
    out = orc.micro_analysis(lnW, 0.0, 1.0, H=H)
    ok = H > 0
    S = -lnW[ok] + np.log(H[ok])
    assert np.allclose(out["S"][ok], S - S.max(), atol=1e-13)
    assert np.all(np.isnan(out["S"][~ok]))


def test_gaussian_dos_canonical(orc):
    sigma, N = 3.0, 10
    e_min, w, K = -80.0, 0.01, 16000
    Ek = e_min + (np.arange(K) + 0.5) * w
    S = -Ek ** 2 / (2 * sigma ** 2)
    T = np.array([0.5, 1.0, 2.0, 4.0])
    out = orc.micro_analysis(-S, e_min, w, n_monomers=N, T=T)
    assert np.allclose(out["E_T"], -sigma ** 2 / T, rtol=1e-6)
    assert np.allclose(out["cV_T"], sigma ** 2 / (N * T ** 2), rtol=1e-5)


def test_two_level_peak(orc):
    g = 50.0
    lnW = np.zeros(11)
    H = np.zeros(11)                            # only bins 0 and 10 are populated
    H[0], H[10] = 1.0, g
    T = np.linspace(0.05, 1.0, 400)
    e_min, w = -0.05, 0.1                       # bin centres 0 and 1.0
    out = orc.micro_analysis(lnW, e_min, w, H=H, n_monomers=1, T=T)
    x = g * np.exp(-1.0 / T)
    assert np.allclose(out["E_T"], x / (1 + x), rtol=1e-10)
    cv = lambda t: g * np.exp(-1 / t) / (1 + g * np.exp(-1 / t)) ** 2 / t ** 2
    assert np.allclose(out["cV_T"], cv(T), rtol=1e-10)
    t_star = optimize.minimize_scalar(lambda t: -cv(t), bounds=(0.05, 1.0), method="bounded",
                                      options={"xatol": 1e-12}).x
    assert out["peak"][0] == pytest.approx(t_star, abs=(T[1] - T[0]) ** 2 * 10)
    assert out["peak"][1] == pytest.approx(cv(t_star), rel=1e-4)


def test_trimer_canonical_energy_by_quadrature(orc):
    # S_k = ln(mass_k) of the exact trimer DOS; <E>_T from the 1-D integral over c
    C = 1.0
    E = lambda c: 0.25 * (1 - c) + 4 * ((2 + 2 * c) ** -6 - C * (2 + 2 * c) ** -3)
    e_min, w, K = -1.0, 0.002, 5000
    G = 4_000_000
    c = -1 + (np.arange(G) + 0.5) * (2 / G)
    k = np.floor((E(c) - e_min) / w)
    ok = (k >= 0) & (k < K)
    mass = np.bincount(k[ok].astype(int), minlength=K) / G
    lnW = np.where(mass > 0, -np.log(np.where(mass > 0, mass, 1)), 0.0)
    H = (mass > 0).astype(float)
    T = np.array([0.15, 0.3, 0.6, 1.2])
    out = orc.micro_analysis(lnW, e_min, w, H=H, T=T)
    cmin = optimize.brentq(lambda x: E(x) - (e_min + K * w), -1 + 1e-9, 0.0)
    for Ti, got in zip(T, out["E_T"]):
        num = integrate.quad(lambda x: E(x) * np.exp(-E(x) / Ti), cmin, 1, limit=200, points=[-0.37])[0]
        den = integrate.quad(lambda x: np.exp(-E(x) / Ti), cmin, 1, limit=200, points=[-0.37])[0]
        assert got == pytest.approx(num / den, abs=2 * w)
