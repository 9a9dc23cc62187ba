"""Pins of the oracle's energy derivatives and reweighted sensitivities.

* A straight AAB trimer's gradient and dE/dC_AB in closed form (exact binary values).
* The FENE bond term's gradient through the finite differences of a stretched
  two-13-mer conformation in the sphere (bond terms about 8 of its 11 units).
* dE/dx against central finite differences of the (separately pinned) energy, at
  h = 1e-3 and, tighter, at h = 1e-5, on conformations of several workloads.
* dE/dp is exact: the energy is linear in every parameter.
* Translation invariance (all systems) and rotation invariance (open systems).
* Reweighted d<E>_T/dC_AB and dc_V/dC_AB of the AAB trimer against finite
  differences in C_AB of its canonical averages by quadrature (cos theta is
  uniform on [-1, 1] under the pivot moves' measure), the samples being the
  quadrature nodes with their weights as multicanonical weights.
"""
import numpy as np
import pytest

from paper_1702_01770_gb300 import inputs

from helpers import oracle_model, random_conformations


def _cases():
    s3, x3 = inputs.config3(2, seed=11)
    s13 = inputs.config0()
    x13 = random_conformations(s13, 1, 5)[0]
    s2 = inputs.config2(1)[2]          # two 34-mers, periodic L = 40
    x2 = random_conformations(s2, 1, 6)[0]
    s8 = inputs.config2(1)[3]          # eight 9-mers, periodic L = 30
    x8 = random_conformations(s8, 1, 7, d_min=0.85)[0]
    sf = inputs.fene_sphere(1)         # FENE bonds stretched up to 0.8 R, inside the sphere
    return [("fib55", s3, x3[0]), ("fib13", s13, x13), ("2x34", s2, x2), ("8x9", s8, x8),
            ("fene", sf, _fene_state(sf))]


def _fene_state(s):
    import oracle as orc
    from helpers import oracle_muca
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    wk = orc.new_walker(m, mu, s.xyz0, 3)
    orc.sweep_walker(m, mu, -0.05 * np.arange(s.n_bins), wk, 26 * 50)
    return wk.xyz.copy()


CASES = _cases()


def test_straight_trimer_closed_form(orc):
    s = inputs.trimer("AAB")
    m = oracle_model(orc, s)
    x = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]])
    e, gx, gp = orc.energy_grad(m, x)
    assert e == orc.energy(m, x)
    # r13 = 2, s = 1/4: dphi/d(r^2) = 4 s (3 C s^3 - 6 s^6) with C = C_AB = -1/2
    f = 2.0 * 4.0 * 0.25 * (3.0 * -0.5 / 64.0 - 6.0 / 4096.0)
    assert gx[0, 0] == -2.0 * f and gx[2, 0] == 2.0 * f       # d = x0 - x2 = (-2, 0, 0)
    assert np.all(gx[1] == 0.0) and np.all(gx[:, 1:] == 0.0)  # a straight chain has no bending force
    assert list(gp) == [0.0, 0.0, -4.0 / 64.0, 0.0, 0.0]


@pytest.mark.parametrize("name,s,x", CASES, ids=[c[0] for c in CASES])
def test_gradient_against_central_differences(orc, name, s, x):
    m = oracle_model(orc, s)
    e, gx, _ = orc.energy_grad(m, x)
    assert e == pytest.approx(orc.energy(m, x), rel=1e-12, abs=1e-12)
    scale = np.max(np.abs(gx))
    for h, tol in ((1e-3, 2e-4), (1e-5, 2e-7)):
        fd = np.zeros_like(gx)
        for i in range(x.shape[0]):
            for d in range(3):
                xp, xm = x.copy(), x.copy()
                xp[i, d] += h
                xm[i, d] -= h
                fd[i, d] = (orc.energy(m, xp) - orc.energy(m, xm)) / (2 * h)
        err = np.max(np.abs(fd - gx))
        assert err <= tol * scale + 1e-9, (name, h, err, scale)


@pytest.mark.parametrize("name,s,x", CASES, ids=[c[0] for c in CASES])
def test_parameter_derivatives_are_exact(orc, name, s, x):
    import dataclasses
    e, _, gp = orc.energy_grad(oracle_model(orc, s), x)
    base = dict(C=tuple(s.C), k_tors=s.k_tors, k_bend=s.k_bend)
    for k, delta in enumerate([0.5, 0.5, 0.5, 0.5, 0.5]):
        def energy_at(sign):
            C = list(base["C"])
            kt, kb = base["k_tors"], base["k_bend"]
            if k == 0:
                C[0] += sign * delta
            elif k == 1:
                C[3] += sign * delta
            elif k == 2:
                C[1] += sign * delta
                C[2] += sign * delta
            elif k == 3:
                kt += sign * delta
            else:
                kb += sign * delta
            return orc.energy(oracle_model(orc, dataclasses.replace(s, C=tuple(C), k_tors=kt, k_bend=kb)), x)
        fd = (energy_at(+1) - energy_at(-1)) / (2 * delta)
        assert fd == pytest.approx(gp[k], rel=1e-11, abs=1e-11 * (1 + abs(e))), (name, k)


@pytest.mark.parametrize("name,s,x", CASES, ids=[c[0] for c in CASES])
def test_translation_and_rotation_invariance(orc, name, s, x):
    _, gx, _ = orc.energy_grad(oracle_model(orc, s), x)
    mag = np.sum(np.abs(gx))
    assert np.max(np.abs(gx.sum(axis=0))) <= 1e-12 * mag
    if s.box_L == 0:
        torque = np.cross(x - x.mean(axis=0), gx).sum(axis=0)
        assert np.max(np.abs(torque)) <= 1e-11 * np.sum(np.abs(x - x.mean(axis=0))[:, :, None] * np.abs(gx)[:, None, :])


def _trimer_E(c, C_ab, k_bend=0.25):
    r2 = 2.0 + 2.0 * c
    return k_bend * (1.0 - c) + 4.0 * (r2 ** -6 - C_ab * r2 ** -3)


def _canonical(c, w, C_ab, T):
    E = _trimer_E(c, C_ab)
    a = -E / T
    p = w * np.exp(a - a.max())
    Z = p.sum()
    mE = np.sum(p * E) / Z
    return mE, np.sum(p * (E - mE) ** 2) / Z / (3 * T * T)


def test_reweighted_sensitivities_of_the_trimer(orc):
    s = inputs.trimer("AAB")
    m = oracle_model(orc, s)
    c, w = np.polynomial.legendre.leggauss(2000)
    E, D = np.zeros(c.size), np.zeros(c.size)
    for n, cn in enumerate(c):
        x = np.array([[-1.0, 0, 0], [0.0, 0, 0], [cn, np.sqrt(1.0 - cn * cn), 0.0]])
        E[n], _, gp = orc.energy_grad(m, x)
        D[n] = gp[2]
    ok = E < 100.0                      # away from the r13 -> 0 end, where r^2 = 2 + 2c cancels
    assert np.allclose(E[ok], _trimer_E(c[ok], -0.5), rtol=1e-12, atol=1e-12)
    T = np.array([0.15, 0.3, 0.6, 1.0])
    out = orc.reweight_sensitivity(E, D, -np.log(w), 3, T)
    dl = 1e-4
    for i, t in enumerate(T):
        e0, cv0 = _canonical(c, w, -0.5, t)
        ep, cvp = _canonical(c, w, -0.5 + dl, t)
        em, cvm = _canonical(c, w, -0.5 - dl, t)
        assert out["E_T"][i] == pytest.approx(e0, rel=1e-10)
        assert out["cV_T"][i] == pytest.approx(cv0, rel=1e-9)
        assert out["dE_T"][i] == pytest.approx((ep - em) / (2 * dl), rel=1e-6, abs=1e-9)
        assert out["dcV_T"][i] == pytest.approx((cvp - cvm) / (2 * dl), rel=1e-5, abs=1e-8)


def test_reweighting_constant_derivative(orc):
    rng = np.random.default_rng(3)
    E = rng.normal(size=500)
    lnW = rng.normal(size=500)
    out = orc.reweight_sensitivity(E, np.full(500, 2.5), lnW, 7, [0.5, 2.0])
    assert np.allclose(out["dE_T"], 2.5, rtol=0, atol=1e-12)     # an additive constant shifts <E> only
    assert np.allclose(out["dcV_T"], 0.0, atol=1e-12)
