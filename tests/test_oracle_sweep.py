"""Pins of the oracle's multicanonical sweep (Sec. 2.2, MONTE_CARLO.f of Sec. 3.2).

The trimer is solvable: under pivot rotations with isotropic axes and
symmetric angles the bond-bond cosine c is uniform on [-1, 1], and
E(c) = kappa_C (1 - c) + 4 (u^-6 - C u^-3) with u = r13^2 = 2 + 2c.  So the
probability mass of every energy bin is known without the oracle, and a
sampler with piecewise-constant weights W_k must visit bin k with probability
proportional to mass_k W_k.  That pins the proposal (isotropy, symmetry), the
acceptance rule min(1, W'/W), the bin map and the histogram bookkeeping.
"""
import numpy as np
import pytest

from paper_1702_01770_gb300 import inputs

C_OF = {"AAA": 1.0, "BBB": 0.5, "AAB": -0.5, "ABA": 1.0}


def trimer_masses(seq, e_min, width, K, G=4_000_000):
    c = -1.0 + (np.arange(G) + 0.5) * (2.0 / G)
    u = 2.0 + 2.0 * c
    E = 0.25 * (1.0 - c) + 4.0 * (u ** -6 - C_OF[seq] * u ** -3)
    k = np.floor((E - e_min) / width)
    ok = (k >= 0) & (k < K)
    return np.bincount(k[ok].astype(np.int64), minlength=K) / G


def run_walkers(orc, s, lnW, n_walkers, n_moves, burn=200, seed0=100):
    m = orc.Model(s.chain_len, s.seq, box_L=s.box_L, k_tors=s.k_tors)
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=s.p, amax=s.amax)
    H = np.zeros((n_walkers, s.n_bins))
    for w in range(n_walkers):
        wk = orc.new_walker(m, mu, s.xyz0, seed0 + w)
        orc.sweep_walker(m, mu, lnW, wk, burn)
        h, _, _ = orc.sweep_walker(m, mu, lnW, wk, n_moves)
        H[w] = h
    return H


def group_compare(H, expect, n_groups=10):
    """Per-walker fractions in groups of bins vs the expected fractions."""
    K = expect.size
    nz = np.nonzero(expect > 0)[0]
    edges = np.linspace(nz[0], nz[-1] + 1, n_groups + 1).astype(int)
    f = H / H.sum(1, keepdims=True)
    zs = []
    for a, b in zip(edges[:-1], edges[1:]):
        fw = f[:, a:b].sum(1)
        e = expect[a:b].sum()
        sem = fw.std(ddof=1) / np.sqrt(len(fw))
        zs.append((fw.mean() - e) / max(sem, 1e-12))
    return np.array(zs)


@pytest.mark.parametrize("seq", ["AAA", "AAB"])
def test_trimer_flat_weights_give_exact_dos(orc, seq):
    s = inputs.trimer(seq)
    mass = trimer_masses(seq, s.e_min, s.bin_width, s.n_bins)
    H = run_walkers(orc, s, np.zeros(s.n_bins), 64, 4000)
    z = group_compare(H, mass / mass.sum())
    assert np.all(np.abs(z) < 5.0), z


def test_trimer_arbitrary_weights(orc):
    s = inputs.trimer("AAA")
    mass = trimer_masses("AAA", s.e_min, s.bin_width, s.n_bins)
    k = np.arange(s.n_bins)
    lnW = 1.5 * np.sin(k / 6.0) - 0.02 * k
    p = mass * np.exp(lnW)
    H = run_walkers(orc, s, lnW, 64, 4000, seed0=900)
    z = group_compare(H, p / p.sum())
    assert np.all(np.abs(z) < 5.0), z


def test_trimer_exact_weights_flatten_histogram(orc):
    s = inputs.trimer("AAA")
    mass = trimer_masses("AAA", s.e_min, s.bin_width, s.n_bins)
    ok = mass > 0
    lnW = np.where(ok, -np.log(np.where(ok, mass, 1.0)), 0.0)
    H = run_walkers(orc, s, lnW, 32, 20000, seed0=5000).sum(0)
    Hv = H[ok]
    assert np.all(H[~ok] == 0)
    # flat within counting noise inflated by autocorrelation (a few sweeps)
    assert Hv.std() / Hv.mean() < 0.08


def test_berg_iterations_recover_trimer_entropy(orc):
    s = inputs.trimer("AAA")
    mass = trimer_masses("AAA", s.e_min, s.bin_width, s.n_bins)
    lnW = np.zeros(s.n_bins)
    g = np.zeros(s.n_bins - 1)
    for it in range(6):
        H = run_walkers(orc, s, lnW, 16, 8000, burn=100, seed0=10000 * (it + 1)).sum(0)
        lnW, g, flat = orc.berg_update(H, lnW, g, s.bin_width)
    # compare S = -lnW with ln(mass) on bins with appreciable mass
    ok = mass > 2e-3
    S = -lnW[ok] - np.log(mass[ok])
    assert S.std() < 0.15, S.std()
    assert flat[2] < 0.3


def test_resume_is_bit_exact(orc):
    s = inputs.config1(1)
    m = orc.Model(s.chain_len, s.seq, box_L=s.box_L, k_tors=s.k_tors)
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=s.p, amax=s.amax, recompute_every=2)
    lnW = np.linspace(0, -3, s.n_bins)
    a = orc.new_walker(m, mu, s.xyz0, 3)
    b = orc.new_walker(m, mu, s.xyz0, 3)
    ha, sa, _ = orc.sweep_walker(m, mu, lnW, a, 36 * 10)
    hb, _, _ = orc.sweep_walker(m, mu, lnW, b, 36 * 4)
    hb, _, _ = orc.sweep_walker(m, mu, lnW, b, 36 * 6, hist=hb)
    assert np.array_equal(ha, hb)
    assert np.array_equal(a.xyz, b.xyz) and a.E == b.E and a.bin == b.bin and a.t == b.t == 360
    assert sa[orc.ST_RECOMPUTES] == 5 and sa[orc.ST_DRIFT] < 1e-10      # recomputes at sweeps 2,4,...,10; tiny FP64 drift
    assert ha.sum() == 360


def test_forced_decisions(orc):
    s = inputs.config1(1)
    m = orc.Model(s.chain_len, s.seq, box_L=s.box_L, k_tors=s.k_tors)
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=s.p, amax=s.amax)
    lnW = np.zeros(s.n_bins)
    a = orc.new_walker(m, mu, s.xyz0, 8)
    ha, sa, rec = orc.sweep_walker(m, mu, lnW, a, 500, record=True)
    b = orc.new_walker(m, mu, s.xyz0, 8)
    hb, sb, recb = orc.sweep_walker(m, mu, lnW, b, 500, force=rec["accepted"].astype(np.int8), record=True)
    assert sb[orc.ST_MISMATCHES] == 0 and np.array_equal(ha, hb) and np.array_equal(rec, recb)
    f = rec["accepted"].astype(np.int8).copy()
    flip = np.nonzero(f == 0)[0][:3]
    f[flip] = 1
    c = orc.new_walker(m, mu, s.xyz0, 8)
    _, sc, _ = orc.sweep_walker(m, mu, lnW, c, 500, force=f)
    assert sc[orc.ST_MISMATCHES] >= 1


def test_out_of_range_start_is_an_error(orc):
    s = inputs.config0()
    m = orc.Model(s.chain_len, s.seq)
    mu = orc.Muca(5.0, 0.05, 10)       # range [5, 5.5) excludes the straight chain
    w = orc.new_walker(m, mu, s.xyz0, 0)
    assert w.bin == -1
    with pytest.raises(ValueError):
        orc.sweep_walker(m, mu, np.zeros(10), w, 10)


def test_moves_out_of_range_are_rejected(orc):
    s = inputs.config0()
    m = orc.Model(s.chain_len, s.seq)
    E0 = orc.energy(m, s.xyz0)
    mu = orc.Muca(E0 - 0.001, 0.002, 1)   # a single narrow bin around the start
    w = orc.new_walker(m, mu, s.xyz0, 0)
    h, st, rec = orc.sweep_walker(m, mu, np.zeros(1), w, 200, record=True)
    assert h[0] == 200
    # only moves whose energy stays in the bin are accepted
    acc = rec["accepted"] == 1
    assert np.all(np.abs(rec["E_after"][acc] - E0) < 0.002)
