"""Pins of the oracle's container, FENE bonds and the bond-length and
spherical-cap moves (the paper's own geometry, Sec. 2.1 Eq. 2 and Sec. 3.2).

* FENE: zero at r0, even in r - r0, the harmonic limit -k C_F (r - r0)^2 for
  small stretches, infinite beyond |r - r0| >= R.
* The container is a hard wall: (x^2 + y^2) + z^2 <= R^2 inside, +inf outside.
* Bond-length moves change exactly one bond, by delta, along its direction, on
  the shorter side, and -delta undoes them; caps keep the bond to their centre.
* E_after - E_before = dE for every move type; long runs stay inside the wall.
* Bond-length moves carry the Hastings factor ((r + delta) / r)^2 of their
  radial map, so that they sample the Cartesian measure of the bead
  coordinates: a collinear trimer with bond-length moves only, under flat
  weights, samples each bond length r with density proportional to r^2 on the
  FENE range (capped by the last bin), which makes its energy histogram and its
  stretch distribution exact integrals (a plain Metropolis rule would sample r
  uniformly and fail both).
"""
import dataclasses

import numpy as np
import pytest

from paper_1702_01770_gb300 import inputs

from helpers import oracle_model, oracle_muca


def _line(r1, r2):
    return np.array([[0.0, 0, 0], [r1, 0, 0], [r1 + r2, 0, 0]])


def _fene_trimer(**kw):
    s = dataclasses.replace(inputs.trimer("AAB"), k_bend=0.0, k_lj_intra=0.0, k_fene=-20.0, fene_r0=1.0,
                            fene_R=0.3, **kw)
    return s


def test_fene_rest_symmetry_and_range(orc):
    m = oracle_model(orc, _fene_trimer())
    _, t = orc.energy(m, _line(1.0, 1.0), terms=True)
    assert t[4] == 0.0
    _, tp = orc.energy(m, _line(1.125, 1.0), terms=True)
    _, tm = orc.energy(m, _line(0.875, 1.0), terms=True)
    assert tp[4] == tm[4] > 0.0
    assert orc.energy(m, _line(1.3, 1.0)) == np.inf            # |r - r0| = R: outside the range
    assert np.isfinite(orc.energy(m, _line(1.29, 1.0)))


def test_fene_harmonic_limit(orc):
    m = oracle_model(orc, _fene_trimer())
    a = 1e-3
    _, t = orc.energy(m, _line(1.0 + a, 1.0), terms=True)
    # k R^2 C_F ln(1 - x^2) = -k C_F a^2 (1 + a^2 / (2 R^2) + ...), k = -20, C_F = 1
    assert t[4] == pytest.approx(20.0 * a * a, rel=1e-4)


def test_container_is_a_hard_wall(orc):
    s = dataclasses.replace(inputs.trimer("AAA"), sphere_R=2.0)
    m = oracle_model(orc, s)
    x = _line(1.0, 1.0) - np.array([1.0, 0, 0])
    assert np.isfinite(orc.energy(m, x))
    x[2, 0] = 2.0                                            # exactly on the wall: inside
    assert np.isfinite(orc.energy(m, x))
    x[2, 0] = np.nextafter(2.0, 3.0)
    assert orc.energy(m, x) == np.inf


def _bonds(x, chain_len):
    out, o = [], 0
    for n in chain_len:
        out.append(np.linalg.norm(np.diff(x[o:o + n], axis=0), axis=1))
        o += n
    return np.concatenate(out)


def test_bond_length_moves(orc):
    s = inputs.fene_sphere(1)
    m = oracle_model(orc, s)
    rng = np.random.default_rng(1)
    x = s.xyz0
    for _ in range(200):
        c, l = int(rng.integers(2)), int(rng.integers(12))
        d = float(rng.uniform(-0.05, 0.05))
        n, y = orc.apply_move(m, orc.make_move(orc.BOND, c, l, angle=d), x)
        assert n == min(l + 1, 12 - l) or (l + 1 == 12 - l and n == 12 - l)
        b0, b1 = _bonds(x, s.chain_len), _bonds(y, s.chain_len)
        k = 12 * c + l
        assert b1[k] == pytest.approx(b0[k] + d, abs=1e-14)
        assert np.allclose(np.delete(b1, k), np.delete(b0, k), rtol=0, atol=1e-14)
        u0 = x[13 * c + l + 1] - x[13 * c + l]
        u1 = y[13 * c + l + 1] - y[13 * c + l]
        assert np.allclose(u1 / np.linalg.norm(u1), u0 / np.linalg.norm(u0), atol=1e-14)
        moved = np.nonzero(np.any(y != x, axis=1))[0]
        head = l + 1 < 12 - l
        want = np.arange(13 * c, 13 * c + l + 1) if head else np.arange(13 * c + l + 1, 13 * c + 13)
        assert set(moved) <= set(want)
        _, z = orc.apply_move(m, orc.make_move(orc.BOND, c, l, angle=-d), y)
        assert np.allclose(z, x, rtol=0, atol=1e-13)
        J = orc.move_jacobian(m, x, orc.make_move(orc.BOND, c, l, angle=d))
        assert J == pytest.approx(((b0[k] + d) / b0[k]) ** 2, rel=1e-14)
        x = y
    # a step that takes the bond through zero length is no move
    n, _ = orc.apply_move(m, orc.make_move(orc.BOND, 0, 3, angle=-1.5), x)
    assert n == 0
    for t in (orc.PIVOT, orc.TRANS, orc.ROT, orc.CRANK, orc.CAP):
        assert orc.move_jacobian(m, x, orc.make_move(t, 0, 3, angle=0.3)) == 1.0


def test_spherical_cap_moves(orc):
    s = inputs.fene_sphere(1)
    m = oracle_model(orc, s)
    rng = np.random.default_rng(2)
    for _ in range(100):
        c, i = int(rng.integers(2)), int(rng.integers(13))
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        n, y = orc.apply_move(m, orc.make_move(orc.CAP, c, i, axis=tuple(ax), angle=float(rng.uniform(-0.5, 0.5))),
                              s.xyz0)
        assert n == 1
        j, ctr = 13 * c + i, 13 * c + (i - 1 if i > 0 else 1)
        assert np.array_equal(np.delete(y, j, axis=0), np.delete(s.xyz0, j, axis=0))
        assert np.linalg.norm(y[j] - y[ctr]) == pytest.approx(np.linalg.norm(s.xyz0[j] - s.xyz0[ctr]), abs=1e-14)


@pytest.mark.parametrize("mtype", ["PIVOT", "TRANS", "ROT", "CRANK", "BOND", "CAP"])
def test_delta_energy_of_every_move_type(orc, mtype):
    s = inputs.fene_sphere(1)
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    t_want = getattr(orc, mtype)
    x = s.xyz0.copy()
    done = 0
    for t in range(4000):
        mv, _ = orc.propose(m, mu, 99, t)
        if mv.type != t_want:
            continue
        E0 = orc.energy(m, x)
        dE, y = orc.delta_energy(m, x, mv)
        E1 = orc.energy(m, y)
        if np.isinf(E1):
            assert dE == np.inf
            continue
        assert dE == pytest.approx(E1 - E0, rel=1e-11, abs=1e-11 * max(1.0, abs(E0), abs(E1)))
        x = y
        done += 1
        if done == 60:
            break
    assert done >= 30


def test_runs_stay_inside_and_in_range(orc):
    s = inputs.fene_sphere(1)
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    w = orc.new_walker(m, mu, s.xyz0, 5)
    _, st, rec = orc.sweep_walker(m, mu, np.zeros(s.n_bins), w, 26 * 400, record=True)
    assert np.all(np.linalg.norm(w.xyz, axis=1) <= 8.0)
    b = _bonds(w.xyz, s.chain_len)
    assert np.all(np.abs(b - 1.0) < 0.3)
    assert w.E == pytest.approx(orc.energy(m, w.xyz), rel=1e-9, abs=1e-9)
    assert np.all(st[:6] > 0) and np.all(st[6:12] > 0)             # every move type tried and taken
    assert np.sum(np.isinf(rec["dE"])) > 0                       # the wall / bond range rejected some


R_F, KR2 = 0.3, 1.8      # the trimer's FENE range and -k R^2 (k = -20)


def _g(e):
    """|x| at which E_F(x) = -KR2 ln(1 - x^2) equals e (0 below 0)."""
    return np.sqrt(1.0 - np.exp(-np.maximum(e, 0.0) / KR2))


def _G(e):
    """Integral of the Cartesian weight (1 + R x)^2 over {x : E_F(x) < e}."""
    g = _g(e)
    return 2.0 * g + (2.0 / 3.0) * R_F * R_F * g ** 3


def _stretch_energy_histogram(e_min, w, K):
    """P(E in bin) for E = E_F(x1) + E_F(x2), x = (r - 1) / R with density
    (1 + R x1)^2 (1 + R x2)^2 on (-1, 1)^2, restricted to E < e_min + K w."""
    x1, wq = np.polynomial.legendre.leggauss(4000)
    E1 = -KR2 * np.log(1.0 - x1 * x1)
    edges = e_min + w * np.arange(K + 1)
    G = _G(edges[None, :] - E1[:, None])
    mass = np.sum((wq * (1.0 + R_F * x1) ** 2)[:, None] * np.diff(G, axis=1), axis=0)
    return mass / mass.sum()


def _stretch_marginal(edges, e_max):
    """P(x1 in each interval of edges): density (1 + R x1)^2 G(e_max - E_F(x1))."""
    out = []
    for a, b in zip(edges[:-1], edges[1:]):
        x, wq = np.polynomial.legendre.leggauss(200)
        x = 0.5 * (b - a) * x + 0.5 * (a + b)
        E1 = -KR2 * np.log(1.0 - x * x)
        out.append(0.5 * (b - a) * np.sum(wq * (1.0 + R_F * x) ** 2 * _G(e_max - E1)))
    out = np.array(out)
    return out / out.sum()


def _bond_only_trimer():
    return dataclasses.replace(_fene_trimer(), k_tors=0.0, e_min=0.0, bin_width=0.05, n_bins=80,
                               p=(0.0, 0.0, 0.0, 0.0, 1.0, 0.0), amax=(0.5, 0.5, 0.3, 0.5, 0.06, 0.5))


def test_bond_moves_sample_the_cartesian_measure(orc):
    s = _bond_only_trimer()
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    H = np.zeros(s.n_bins, np.uint64)
    for seed in range(8):
        wk = orc.new_walker(m, mu, _line(1.0, 1.0), seed)
        orc.sweep_walker(m, mu, np.zeros(s.n_bins), wk, 2000)             # equilibrate
        H, _, _ = orc.sweep_walker(m, mu, np.zeros(s.n_bins), wk, 200000, hist=H)
    p = _stretch_energy_histogram(s.e_min, s.bin_width, s.n_bins)
    n = H.sum()
    exp_ = n * p
    keep = exp_ > 50
    # successive samples are correlated (steps of 0.06 on a range of 0.6): compare
    # with a generous multiple of the Poisson error
    z = (H[keep] - exp_[keep]) / np.sqrt(exp_[keep])
    assert np.max(np.abs(z)) < 25.0, np.max(np.abs(z))
    assert np.sum(np.abs(H[keep] / exp_[keep] - 1.0) > 0.1) == 0


def test_bond_moves_stretch_distribution(orc):
    # the energy sees only x^2; the stretch itself shows the odd part of the
    # r^2 weight: <x> is about 0.06 here, 0 for a uniform density
    s = _bond_only_trimer()
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    xs = []
    for seed in range(4):
        wk = orc.new_walker(m, mu, _line(1.0, 1.0), 100 + seed)
        orc.sweep_walker(m, mu, np.zeros(s.n_bins), wk, 2000)
        for _ in range(3000):
            orc.sweep_walker(m, mu, np.zeros(s.n_bins), wk, 60)
            r = np.linalg.norm(np.diff(wk.xyz, axis=0), axis=1)
            xs.extend((r - 1.0) / R_F)
    xs = np.array(xs)
    edges = np.linspace(-1.0, 1.0, 11)
    p = _stretch_marginal(edges, s.e_min + s.bin_width * s.n_bins)
    h = np.histogram(xs, edges)[0] / xs.size
    keep = p > 0.01
    assert np.max(np.abs(h[keep] / p[keep] - 1.0)) < 0.08, (h, p)
    x_mean = np.sum(p * 0.5 * (edges[1:] + edges[:-1]))
    assert x_mean > 0.04
    assert abs(xs.mean() - x_mean) < 0.02, (xs.mean(), x_mean)
