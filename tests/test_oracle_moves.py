"""Pins of the oracle's move geometry, proposal stream and dE.

* Philox4x32-10 equals cuRAND's own host Philox4_32_10 generator (an
  independent implementation, run through libcurand) word for word.
* Rotations built from the Taylor sin/cos agree with libm's sin/cos.
* Moves keep every bond at unit length; pivots keep distances to the pivot;
  rigid moves keep every intra-chain distance (Sec. 3.2 move set).
* dE by affected terms equals E(new) - E(old) of the full energy.
* The pair-evaluation count equals a brute-force count of changed distances.
* Proposal statistics: type frequencies, uniform chains/indices/angles,
  isotropic axes.
"""
import ctypes as C
import os

import numpy as np
import pytest

from paper_1702_01770_gb300 import inputs


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return C.CDLL(p)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator(orc):
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    for seed in (0, 1, 0x123456789ABCDEF0, 2**64 - 1):
        gen = C.c_void_p()
        if cr.curandCreateGeneratorHost(C.byref(gen), C.c_int(161)) != 0:   # CURAND_RNG_PSEUDO_PHILOX4_32_10
            pytest.skip("cuRAND host generator unavailable")
        try:
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
            n = 4 * 300
            out = np.zeros(n, np.uint32)
            assert cr.curandGenerate(gen, out.ctypes.data_as(C.POINTER(C.c_uint32)), C.c_size_t(n)) == 0
        finally:
            cr.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        # cuRAND's host ordering: element i is word i % 4 of block (0, 0, i // 4, 0)
        mine = np.concatenate([orc.philox([0, 0, b, 0], key) for b in range(n // 4)])
        assert np.array_equal(out, mine)


def test_philox_counter_words_all_matter(orc):
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(orc.philox(c, [5, 6]), base)
    assert not np.array_equal(orc.philox([1, 2, 3, 4], [5, 7]), base)


def _model(orc, s, box=None):
    return orc.Model(s.chain_len, s.seq, box_L=s.box_L if box is None else box, k_tors=s.k_tors)


def test_rotation_matches_libm(orc):
    s = inputs.trimer("AAA")
    m = _model(orc, s)
    x = np.array([[-1.0, 0, 0], [0.0, 0, 0], [0.0, 1.0, 0]])
    for a in np.linspace(-1.0, 1.0, 41):
        mv = orc.make_move(orc.PIVOT, 0, 1, axis=(0.0, 0.0, 1.0), angle=a)
        n, y = orc.apply_move(m, mv, x)
        assert n == 1
        # monomer 2 at e_y rotated about z through the origin lands on (-sin a, cos a, 0)
        assert y[2, 0] == pytest.approx(-np.sin(a), rel=2.3e-16, abs=1e-300)
        assert y[2, 1] == pytest.approx(np.cos(a), rel=2.3e-16)
        assert np.array_equal(y[:2], x[:2])


def _bonds(x, chain_len):
    out, o = [], 0
    for n in chain_len:
        out.append(np.linalg.norm(np.diff(x[o:o + n], axis=0), axis=1))
        o += n
    return np.concatenate(out)


@pytest.mark.parametrize("cfg", ["c0", "c1", "c2x34"])
def test_moves_preserve_geometry(orc, cfg):
    s = {"c0": inputs.config0(), "c1": inputs.config1(1), "c2x34": inputs.config2(1)[2]}[cfg]
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=(0.4, 0.2, 0.2, 0.2), amax=s.amax)
    m = _model(orc, s)
    x = s.xyz0.copy()
    N = s.n_total
    offs = np.concatenate([[0], np.cumsum(s.chain_len)])
    for t in range(300):
        mv, _ = orc.propose(m, mu, 77, t)
        n, y = orc.apply_move(m, mv, x)
        assert n > 0
        assert np.allclose(_bonds(y, s.chain_len), 1.0, atol=1e-13)
        o, e = offs[mv.chain], offs[mv.chain + 1]
        moved = np.any(y != x, axis=1)
        assert not moved[:o].any() and not moved[e:].any()
        if mv.type == orc.PIVOT:
            k = o + mv.index
            d0 = np.linalg.norm(x[o:e] - x[k], axis=1)
            d1 = np.linalg.norm(y[o:e] - y[k], axis=1)
            assert np.allclose(d0, d1, atol=1e-12)
            assert np.array_equal(x[k], y[k])
            side = np.arange(o, e)[moved[o:e]]
            head, tail = mv.index, (e - o) - 1 - mv.index
            if side.size:
                assert (side.max() < k) if head < tail else (side.min() > k)
        elif mv.type in (orc.TRANS, orc.ROT):
            dx = x[o:e, None, :] - x[None, o:e, :]
            dy = y[o:e, None, :] - y[None, o:e, :]
            assert np.allclose(np.linalg.norm(dx, axis=2), np.linalg.norm(dy, axis=2), atol=1e-12)
            if mv.type == orc.ROT:
                assert np.allclose(x[o:e].mean(0), y[o:e].mean(0), atol=1e-12)
        else:
            i = o + mv.index
            assert moved[o:e].sum() <= 1
            assert np.linalg.norm(y[i] - y[i - 1]) == pytest.approx(1.0, abs=1e-13)
            assert np.linalg.norm(y[i] - y[i + 1]) == pytest.approx(1.0, abs=1e-13)
        x = y
    assert N == x.shape[0]


@pytest.mark.parametrize("cfg", ["c0", "c1", "c2x34", "c2_8x9"])
def test_delta_equals_energy_difference(orc, cfg):
    s = {"c0": inputs.config0(), "c1": inputs.config1(1), "c2x34": inputs.config2(1)[2],
         "c2_8x9": inputs.config2(1)[3]}[cfg]
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=(0.4, 0.2, 0.2, 0.2), amax=s.amax)
    m = _model(orc, s)
    x = s.xyz0.copy()
    worst = 0.0
    for t in range(400):
        mv, _ = orc.propose(m, mu, 5, t)
        dE, y = orc.delta_energy(m, x, mv)
        E0, E1 = orc.energy(m, x), orc.energy(m, y)
        full = E1 - E0
        assert np.isfinite(dE)
        # the full difference carries the rounding of every unchanged term
        scale = max(1.0, abs(E0), abs(E1))
        err = abs(dE - full)
        worst = max(worst, err / scale)
        assert err <= 1e-12 * scale, (t, dE, full)
        if t % 3 == 0 and E1 < s.e_max:
            x = y   # walk on (within the bin range) so later moves see varied conformations
    assert worst < 1e-12


def test_pair_evals_brute_force(orc):
    s = inputs.config2(1)[3]     # eight 9-mers, periodic
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=(0.4, 0.2, 0.2, 0.2), amax=s.amax)
    m = _model(orc, s)
    x = s.xyz0.copy()
    N = s.n_total
    chain = np.repeat(np.arange(len(s.chain_len)), s.chain_len)
    idx = np.arange(N)
    for t in range(120):
        mv, _ = orc.propose(m, mu, 9, t)
        _, y = orc.apply_move(m, mv, x)
        moved = np.any(y != x, axis=1)
        count = 0
        for i in idx[moved]:
            for j in idx[~moved]:
                if chain[i] == chain[j] and abs(i - j) < 2:
                    continue
                d0, d1 = x[i] - x[j], y[i] - y[j]
                if chain[i] != chain[j]:
                    d0, d1 = d0 - s.box_L * np.rint(d0 / s.box_L), d1 - s.box_L * np.rint(d1 / s.box_L)
                if abs(np.linalg.norm(d0) - np.linalg.norm(d1)) > 1e-9:
                    count += 2
        assert orc.pair_evals(m, mv) == count, (t, mv.type)


def test_proposal_statistics(orc):
    s = inputs.config2(1)[3]
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=(0.5, 0.2, 0.2, 0.1), amax=(0.5, 0.4, 0.3, 0.2))
    m = _model(orc, s)
    n = 8000
    types, chains, idx, ang, axes, uacc = [], [], [], [], [], []
    for t in range(n):
        mv, u = orc.propose(m, mu, 1234, t)
        types.append(mv.type)
        chains.append(mv.chain)
        uacc.append(u)
        if mv.type in (orc.PIVOT, orc.CRANK):
            idx.append(mv.index)
        if mv.type in (orc.PIVOT, orc.ROT):
            axes.append(list(mv.axis))
            ang.append(mv.angle / mu.amax[mv.type])
    types = np.array(types)
    for k, p in enumerate(mu.p):
        f = np.mean(types == k)
        assert abs(f - p) < 5 * np.sqrt(p * (1 - p) / n)
    cnt = np.bincount(chains, minlength=8)
    assert np.all(np.abs(cnt - n / 8) < 5 * np.sqrt(n / 8))
    idx = np.array(idx)
    assert idx.min() == 1 and idx.max() == 7
    axes = np.array(axes)
    assert np.allclose(np.linalg.norm(axes, axis=1), 1.0, atol=1e-15)
    assert np.all(np.abs(axes.mean(0)) < 5 / np.sqrt(len(axes) * 3))
    assert np.allclose((axes ** 2).mean(0), 1 / 3, atol=5 * np.sqrt(4 / 45 / len(axes)))
    ang = np.array(ang)
    assert ang.min() >= -1 and ang.max() <= 1 and abs(ang.mean()) < 5 / np.sqrt(3 * len(ang))
    u = np.array(uacc)
    assert 0 < u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    # translation components uniform in [-0.4, 0.4]
    d = np.array([list(orc.propose(m, orc.Muca(0, 1, 1, p=(0, 1, 0, 0), amax=(0.5, 0.4, 0.3, 0.2)), 7, t)[0].disp)
                  for t in range(2000)])
    assert np.abs(d).max() <= 0.4 and np.all(np.abs(d.mean(0)) < 5 * 0.4 / np.sqrt(3 * 2000))


def test_proposal_is_deterministic(orc):
    s = inputs.config1(1)
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=s.p, amax=s.amax)
    m = _model(orc, s)
    a = orc.propose(m, mu, 42, 1000)
    b = orc.propose(m, mu, 42, 1000)
    assert bytes(a[0]) == bytes(b[0]) and a[1] == b[1]
    c = orc.propose(m, mu, 43, 1000)
    assert bytes(a[0]) != bytes(c[0])


def test_delta_scale_trimer_closed_form(orc):
    """The changed-term magnitude of a trimer pivot: |pair (0,2)| before and
    after plus |bend| before and after, by hand."""
    s = inputs.trimer("AAA")
    m = _model(orc, s)
    x = np.array([[-1.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])   # straight
    a = 0.7
    mv = orc.make_move(orc.PIVOT, 0, 1, axis=(0.0, 0.0, 1.0), angle=a)
    r2_new = (1.0 + np.cos(a)) ** 2 + np.sin(a) ** 2
    lj = lambda r2: 4.0 * (r2 ** -6 - r2 ** -3)
    bend_new = 0.25 * (1.0 - np.cos(a))
    expect = abs(lj(4.0)) + abs(lj(r2_new)) + 0.0 + bend_new
    assert orc.delta_scale(m, x, mv) == pytest.approx(expect, rel=1e-12)
