"""Pins of the oracle's energy (Eq. 1-3 plus torsion) against closed forms.

Each expected value below is derived by hand for a hand-built conformation
(straight chains: integer distances, cos(theta) = 1; right angles: r^2 = 2;
planar 4-mers: cos(tau) = +1, -1, 0) and evaluated with exact rationals, so a
dropped term, a wrong sign, a wrong coupling index or a wrong pair range in the
oracle fails one of them.
"""
import json
import os
from fractions import Fraction as Fr
from itertools import product

import numpy as np
import pytest

from paper_1702_01770_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
C_AB = {("A", "A"): Fr(1), ("B", "B"): Fr(1, 2), ("A", "B"): Fr(-1, 2), ("B", "A"): Fr(-1, 2)}


def model_for(orc, seq, box_L=0.0, k_tors=0.0, chain_len=None):
    s = inputs.str_to_seq(seq)
    cl = [len(seq)] if chain_len is None else chain_len
    return orc.Model(np.array(cl), s, box_L=box_L, k_tors=k_tors)


def lj(r2: Fr, c: Fr) -> Fr:
    """4 (r^-12 - C r^-6) for rational r^2."""
    return 4 * (1 / r2 ** 6 - c / r2 ** 3)


def test_paper_constants_are_the_defaults(orc):
    g = GOLD["C_LJ"]
    m = orc.Model(np.array([3]), np.zeros(3, np.uint8))
    assert m.C == (g["AA"], g["AB"], g["AB"], g["BB"])
    h = GOLD["set_hamiltonian"]
    assert m.k_bend == h["c_KC"] and m.k_lj_intra == h["c_KLJ_intra"] and m.k_lj_inter == h["c_KLJ_inter"]
    s = inputs.config0()
    assert (s.k_bend, s.k_lj_intra, s.C) == (h["c_KC"], h["c_KLJ_intra"], m.C)


@pytest.mark.parametrize("seq", ["".join(p) for p in product("AB", repeat=3)])
def test_straight_trimer(orc, seq):
    m = model_for(orc, seq)
    E = orc.energy(m, inputs.straight_chain(3))
    expect = lj(Fr(4), C_AB[(seq[0], seq[2])])        # bend 0, only pair (0,2) at r = 2
    assert E == pytest.approx(float(expect), abs=1e-15)


@pytest.mark.parametrize("seq", ["".join(p) for p in product("AB", repeat=3)])
def test_right_angle_trimer(orc, seq):
    m = model_for(orc, seq)
    x = np.array([[1.0, 0, 0], [0, 0, 0], [0, 1.0, 0]])
    E, t = orc.energy(m, x, terms=True)
    expect = Fr(1, 4) * (1 - 0) + lj(Fr(2), C_AB[(seq[0], seq[2])])
    assert E == pytest.approx(float(expect), abs=1e-15)
    assert t[0] == pytest.approx(0.25, abs=1e-15) and t[1] == 0.0 and t[3] == 0.0


def test_trimer_decimal_values(orc):
    # the same closed forms, as decimal numbers
    for seq, straight, right in [("AAA", -0.0615234375, -0.1875), ("BBB", -0.0302734375, 0.0625),
                                 ("AAB", 0.0322265625, 0.5625)]:
        m = model_for(orc, seq)
        assert orc.energy(m, inputs.straight_chain(3)) == pytest.approx(straight, abs=1e-15)
        x = np.array([[1.0, 0, 0], [0, 0, 0], [0, 1.0, 0]])
        assert orc.energy(m, x) == pytest.approx(right, abs=1e-15)


def straight_closed_form(seq: str) -> Fr:
    n = len(seq)
    return sum((lj(Fr((j - i) ** 2), C_AB[(seq[i], seq[j])])
                for i in range(n) for j in range(i + 2, n)), Fr(0))


@pytest.mark.parametrize("seq", ["ABBABBABABBAB", "BBBBBAAAB", "BBBABAAABB", "AAAAAAA"])
def test_straight_chain(orc, seq):
    m = model_for(orc, seq, k_tors=-0.5)   # straight: every dihedral is degenerate -> 0
    E, t = orc.energy(m, inputs.straight_chain(len(seq)), terms=True)
    assert E == pytest.approx(float(straight_closed_form(seq)), rel=1e-14, abs=1e-15)
    assert t[0] == 0.0 and t[1] == 0.0


def test_fibonacci_13_straight_value(orc):
    m = model_for(orc, "ABBABBABABBAB")
    assert orc.energy(m, inputs.straight_chain(13)) == pytest.approx(-0.0122108020835, abs=1e-12)


# planar and twisted 4-mers: x0 = e_y, x1 = 0, x2 = e_x, x3 as listed; both bends
# are right angles; (x3, cos tau, r03^2), with r02^2 = r13^2 = 2 in all three
FOURMERS = {
    "cis": ([1.0, 1.0, 0.0], Fr(1), Fr(1)),
    "trans": ([1.0, -1.0, 0.0], Fr(-1), Fr(5)),
    "perp": ([1.0, 0.0, 1.0], Fr(0), Fr(3)),
}


@pytest.mark.parametrize("shape", list(FOURMERS))
@pytest.mark.parametrize("seq", ["AAAA", "ABBA", "BABA"])
def test_fourmer_torsion(orc, shape, seq):
    x3, cos_tau, r03 = FOURMERS[shape]
    x = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0], x3])
    kappa = Fr(-1, 2)
    m = model_for(orc, seq, k_tors=float(kappa))
    bend = Fr(1, 4) * 2
    tors = -kappa * cos_tau
    ljs = (lj(Fr(2), C_AB[(seq[0], seq[2])]) + lj(Fr(2), C_AB[(seq[1], seq[3])])
           + lj(r03, C_AB[(seq[0], seq[3])]))
    E, t = orc.energy(m, x, terms=True)
    assert t[0] == pytest.approx(float(bend), abs=1e-15)
    assert t[1] == pytest.approx(float(tors), abs=1e-15)
    assert E == pytest.approx(float(bend + tors + ljs), abs=1e-14)


def test_two_chains_periodic(orc):
    """Two straight trimers at separation d along y: inter term closed form,
    unchanged under a shift by L and under the minimum image."""
    L, d = 10.0, 1.5
    seq = "ABA" + "BBA"
    m = model_for(orc, seq, box_L=L, chain_len=[3, 3])
    a = inputs.straight_chain(3)
    b = inputs.straight_chain(3, origin=(0.0, d, 0.0))
    inter = sum(lj(Fr(d) ** 2 + (i - j) ** 2, C_AB[(seq[i], seq[3 + j])])
                for i in range(3) for j in range(3))
    intra = lj(Fr(4), C_AB[("A", "A")]) + lj(Fr(4), C_AB[("B", "A")])
    E, t = orc.energy(m, np.concatenate([a, b]), terms=True)
    assert t[3] == pytest.approx(float(inter), rel=1e-13)
    assert t[2] == pytest.approx(float(intra), rel=1e-13)
    for shift in ([L, 0, 0], [0, -L, 0], [3 * L, 2 * L, -L]):
        E2 = orc.energy(m, np.concatenate([a, b + np.array(shift)]))
        assert E2 == pytest.approx(E, rel=1e-12)
    # chain b moved to y = L - d: its minimum image sits at y = -d, the mirror image
    E3 = orc.energy(m, np.concatenate([a, b + np.array([0.0, L - 2 * d, 0.0])]))
    assert E3 == pytest.approx(E, rel=1e-12)
    # without the box the far chain hardly interacts
    m_open = model_for(orc, seq, box_L=0.0, chain_len=[3, 3])
    E4, t4 = orc.energy(m_open, np.concatenate([a, b + np.array([0, L - 2 * d, 0])]), terms=True)
    assert abs(t4[3]) < 1e-4


def test_invariances(orc):
    rng = np.random.default_rng(5)
    s = inputs.config1(walkers=1)
    m = orc.Model(s.chain_len, s.seq, box_L=0.0, k_tors=-0.5)   # open: rigid motions are exact symmetries
    x = s.xyz0.copy()
    E = orc.energy(m, x)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    Ex = orc.energy(m, x @ q.T + rng.normal(size=3) * 7)
    assert Ex == pytest.approx(E, rel=1e-11, abs=1e-11)
    # relabel chains: reverse chain order together with their sequences
    n = 9
    perm = np.concatenate([np.arange(c * n, (c + 1) * n) for c in reversed(range(4))])
    m2 = orc.Model(s.chain_len, s.seq[perm], box_L=0.0, k_tors=-0.5)
    assert orc.energy(m2, x[perm]) == pytest.approx(E, rel=1e-12, abs=1e-12)
    # reverse the direction of every chain (monomer order within each chain)
    rev = np.concatenate([np.arange((c + 1) * n - 1, c * n - 1, -1) for c in range(4)])
    m3 = orc.Model(s.chain_len, s.seq[rev], box_L=0.0, k_tors=-0.5)
    assert orc.energy(m3, x[rev]) == pytest.approx(E, rel=1e-12, abs=1e-12)
    # periodic: translating one chain by a lattice vector changes nothing
    mp = orc.Model(s.chain_len, s.seq, box_L=20.0, k_tors=-0.5)
    Ep = orc.energy(mp, x)
    y = x.copy()
    y[9:18] += np.array([20.0, -40.0, 20.0])
    assert orc.energy(mp, y) == pytest.approx(Ep, rel=1e-12, abs=1e-12)


def test_config_initial_energies_in_range(orc):
    for s in [inputs.config0(), inputs.config1(4)] + inputs.config2(2):
        m = orc.Model(s.chain_len, s.seq, box_L=s.box_L, k_tors=s.k_tors)
        E = orc.energy(m, s.xyz0)
        assert s.e_min <= E < s.e_max, (s.name, E)


@pytest.mark.parametrize("eps,resolved", [(0.0, False), (1e-12, False), (1e-6, True), (1e-3, True)])
def test_nearly_collinear_dihedral(orc, eps, resolved):
    """The degenerate-dihedral rule of the torsion term: bonds b0, b1 at an angle eps
    make n1 = b0 x b1 of length sin(eps).  With b1 = e_x, b2 = e_y and b0 tilted by eps
    in the plane at azimuth phi about e_x, cos tau = -cos(phi) whatever eps; the term
    counts while |n1|^2 |n2|^2 = sin^2(eps) >= 1e-20 and is 0 below (eps = 1e-12: 1e-24,
    and exactly collinear bonds)."""
    phi = np.pi / 3
    b0 = np.array([np.cos(eps), np.sin(eps) * np.cos(phi), np.sin(eps) * np.sin(phi)])
    x = np.array([-b0, [0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 1.0, 0.0]])
    kappa = -0.5
    m = model_for(orc, "AAAA", k_tors=kappa)
    _, t = orc.energy(m, x, terms=True)
    expected = -kappa * (-np.cos(phi)) if resolved else 0.0
    assert t[1] == pytest.approx(expected, abs=1e-8), (eps, t[1])
