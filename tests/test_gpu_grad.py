"""Energy derivatives and reweighted sensitivities on the GPU, through the C ABI,
against the FP64 oracle, central differences and the trimer's exact canonical
averages."""
import dataclasses

import numpy as np
import pytest
import torch

from paper_1702_01770_gb300 import inputs

from helpers import oracle_model, random_conformations

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def phast():
    from paper_1702_01770_gb300 import phast
    phast.lib()
    return phast


def _batches():
    s3, x3 = inputs.config3(12, seed=21)
    s2 = inputs.config2(1)[2]
    s8 = inputs.config2(1)[3]
    s4 = inputs.config4(1)
    return [("fib55", s3, x3), ("2x34", s2, random_conformations(s2, 3, 31)),
            ("8x9", s8, random_conformations(s8, 3, 32, d_min=0.85)), ("8x55", s4, random_conformations(s4, 2, 33))]


BATCHES = _batches()


def _oracle(orc, s, x):
    m = oracle_model(orc, s)
    out = [orc.energy_grad(m, xb) for xb in x]
    return (np.array([o[0] for o in out]), np.stack([o[1] for o in out]), np.stack([o[2] for o in out]))


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name,s,x", BATCHES, ids=[b[0] for b in BATCHES])
def test_energy_grad_matches_oracle(phast, orc, name, s, x, precision):
    E, gx, gf = phast.phast_energy_grad(s, torch.from_numpy(x).cuda(), precision)
    E, gx, gf = E.cpu().numpy(), gx.cpu().numpy(), gf.cpu().numpy()
    Eo, gxo, gfo = _oracle(orc, s, x)
    for b in range(x.shape[0]):
        gmax = max(1.0, np.max(np.abs(gxo[b])))
        if precision == 64:
            assert E[b] == pytest.approx(Eo[b], rel=1e-11, abs=1e-11)
            assert np.max(np.abs(gx[b] - gxo[b])) <= 1e-10 * gmax
            assert np.allclose(gf[b], gfo[b], rtol=1e-11, atol=1e-11)
        else:
            assert abs(E[b] - Eo[b]) <= 1e-4 * max(1.0, abs(Eo[b])), (name, b)
            assert np.max(np.abs(gx[b] - gxo[b])) <= 1e-4 * gmax, (name, b)
            assert np.all(np.abs(gf[b] - gfo[b]) <= 1e-4 * np.maximum(1.0, np.abs(gfo[b]))), (name, b)


def test_differentiation_batch_full_size(phast, orc):
    """The 65536-conformation batch of the 55-mer in FP32: sampled conformations
    against the oracle, every conformation's forces summing to zero."""
    s, x = inputs.config3()
    xt = torch.from_numpy(x).cuda()
    E, gx, gf = phast.phast_energy_grad(s, xt, 32)
    torch.cuda.synchronize()
    assert torch.isfinite(E).all() and torch.isfinite(gx).all() and torch.isfinite(gf).all()
    net = gx.sum(dim=1).abs().max(dim=1).values
    mag = gx.abs().sum(dim=(1, 2))
    assert bool((net <= 1e-5 * mag + 1e-6).all())
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(x.shape[0], 24, replace=False))
    Eo, gxo, gfo = _oracle(orc, s, x[idx])
    E, gx, gf = E.cpu().numpy()[idx], gx.cpu().numpy()[idx], gf.cpu().numpy()[idx]
    for k in range(idx.size):
        assert abs(E[k] - Eo[k]) <= 1e-4 * max(1.0, abs(Eo[k]))
        assert np.max(np.abs(gx[k] - gxo[k])) <= 1e-4 * max(1.0, np.max(np.abs(gxo[k])))
        assert np.all(np.abs(gf[k] - gfo[k]) <= 1e-4 * np.maximum(1.0, np.abs(gfo[k])))


@pytest.mark.parametrize("precision", [64, 32])
def test_autograd_function(phast, precision):
    s, x = inputs.config3(4, seed=41)
    xyz = torch.from_numpy(x).cuda().requires_grad_(True)
    params = torch.tensor(phast.ff_params(s), dtype=torch.float64, requires_grad=True)
    w = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64, device="cuda")
    E = phast.energy(xyz, params, s, precision)
    (w * E).sum().backward()
    _, gx, gf = phast.phast_energy_grad(s, torch.from_numpy(x).cuda(), precision)
    assert torch.allclose(xyz.grad, w.view(-1, 1, 1) * gx, rtol=0, atol=0)
    assert torch.allclose(params.grad, (w.view(-1, 1) * gf).sum(0).cpu(), rtol=1e-12, atol=1e-12)
    if precision == 64:   # central differences, h = 1e-3, FP64
        rng = np.random.default_rng(9)
        h = 1e-3
        for _ in range(12):
            b, i, d = rng.integers(4), rng.integers(55), rng.integers(3)
            xp, xm = x.copy(), x.copy()
            xp[b, i, d] += h
            xm[b, i, d] -= h
            Ep = phast.phast_energy(s, torch.from_numpy(xp).cuda())[b]
            Em = phast.phast_energy(s, torch.from_numpy(xm).cuda())[b]
            fd = float(Ep - Em) / (2 * h)
            assert fd == pytest.approx(float(gx[b, i, d]), abs=2e-4 * max(1.0, float(gx[b].abs().max())))
        for k in range(5):   # the energy is linear in each parameter
            pp, pm = list(phast.ff_params(s)), list(phast.ff_params(s))
            pp[k] += 0.5
            pm[k] -= 0.5
            Ep = phast.energy(torch.from_numpy(x).cuda(), torch.tensor(pp, dtype=torch.float64), s, 64)
            Em = phast.energy(torch.from_numpy(x).cuda(), torch.tensor(pm, dtype=torch.float64), s, 64)
            assert torch.allclose((Ep - Em).cpu(), gf[:, k].cpu(), rtol=1e-10, atol=1e-10)


def test_reweighting_matches_oracle(phast, orc):
    rng = np.random.default_rng(13)
    n = 20000
    E = rng.normal(-20.0, 6.0, n)
    D = -0.3 * E + rng.normal(0.0, 2.0, n)
    lnW = 0.5 * E + rng.normal(0.0, 1.0, n)
    T = np.linspace(0.1, 1.0, 64)
    g = phast.reweight_sensitivity(*(torch.from_numpy(v).cuda() for v in (E, D, lnW)), 55, torch.from_numpy(T).cuda())
    o = orc.reweight_sensitivity(E, D, lnW, 55, T)
    for k in ("E_T", "cV_T", "dE_T", "dcV_T"):
        assert np.allclose(g[k].cpu().numpy(), o[k], rtol=1e-10, atol=1e-12), k


def _trimer_canonical(c, w, C_ab, T, k_bend=0.25, e_max=np.inf):
    r2 = 2.0 + 2.0 * c
    E = k_bend * (1.0 - c) + 4.0 * (r2 ** -6 - C_ab * r2 ** -3)
    a = -E / T
    p = w * np.exp(a - a.max()) * (E < e_max)
    mE = np.sum(p * E) / p.sum()
    return mE, np.sum(p * (E - mE) ** 2) / p.sum() / (3 * T * T)


def _trimer_truth(T, dl=1e-4, e_max=np.inf):
    c, w = np.polynomial.legendre.leggauss(4000)
    if np.isfinite(e_max):   # the sampled domain {c : E(c) < e_max} is an interval [c*, 1]
        lo, hi = -1.0, 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            r2 = 2.0 + 2.0 * mid
            if 0.25 * (1.0 - mid) + 4.0 * (r2 ** -6 + 0.5 * r2 ** -3) >= e_max:
                lo = mid
            else:
                hi = mid
        c = 0.5 * (1.0 - hi) * c + 0.5 * (1.0 + hi)
        w = 0.5 * (1.0 - hi) * w
    out = []
    for t in T:
        e0, cv0 = _trimer_canonical(c, w, -0.5, t)
        ep, cvp = _trimer_canonical(c, w, -0.5 + dl, t)
        em, cvm = _trimer_canonical(c, w, -0.5 - dl, t)
        out.append((e0, cv0, (ep - em) / (2 * dl), (cvp - cvm) / (2 * dl)))
    return np.array(out)


def test_trimer_sensitivities_by_quadrature_nodes(phast):
    """Quadrature nodes as samples with their weights as multicanonical weights:
    the GPU pipeline (derivative kernel, reweighting kernel) gives the exact
    canonical derivatives of the AAB trimer."""
    s = inputs.trimer("AAB")
    c, w = np.polynomial.legendre.leggauss(4000)
    x = np.zeros((c.size, 3, 3))
    x[:, 0, 0] = -1.0
    x[:, 2, 0] = c
    x[:, 2, 1] = np.sqrt(1.0 - c * c)
    E, _, gf = phast.phast_energy_grad(s, torch.from_numpy(x).cuda(), 64, want_xyz=False)
    T = np.array([0.15, 0.3, 0.6, 1.0])
    g = phast.reweight_sensitivity(E, gf[:, 2], torch.from_numpy(-np.log(w)).cuda(), 3, torch.from_numpy(T).cuda())
    truth = _trimer_truth(T)
    assert np.allclose(g["E_T"].cpu().numpy(), truth[:, 0], rtol=1e-9)
    assert np.allclose(g["dE_T"].cpu().numpy(), truth[:, 2], rtol=1e-5, atol=1e-9)
    assert np.allclose(g["dcV_T"].cpu().numpy(), truth[:, 3], rtol=1e-4, atol=1e-8)


def test_muca_run_trimer_sensitivities(phast, orc):
    """A multicanonical run of the AAB trimer on flat weights (its walkers then
    sample cos theta uniformly): reweighted d<E>_T/dC_AB and dc_V/dC_AB from the
    run's snapshots match the exact values within five jackknife errors."""
    s = dataclasses.replace(inputs.trimer("AAB"), walkers=512, seed_base=100)
    ctx = phast.Context(s, pair_precision=32)
    lnW = ctx.lnW_zeros()
    T = torch.tensor([0.3, 0.5, 1.0], dtype=torch.float64, device="cuda")
    ctx.sweep(20, lnW)                                    # forget the straight start
    chunks, per = 240, 4
    Es, Ds = [], []
    for _ in range(chunks):
        ctx.sweep(per, lnW)
        st = ctx.get_state()
        E, _, gf = phast.phast_energy_grad(s, ctx.xyz_of(st, 0), 32, want_xyz=False)
        Es.append(E)
        Ds.append(gf[:, 2])
    E = torch.stack(Es)            # [chunks, walkers]
    D = torch.stack(Ds)
    zeros = torch.zeros_like(E)
    blocks = 16
    per_block = s.walkers // blocks
    full = phast.reweight_sensitivity(E.reshape(-1), D.reshape(-1), zeros.reshape(-1), 3, T)
    reps = []
    for b in range(blocks):    # jackknife over blocks of walkers
        keep = torch.ones(s.walkers, dtype=torch.bool, device="cuda")
        keep[b * per_block:(b + 1) * per_block] = False
        r = phast.reweight_sensitivity(E[:, keep].reshape(-1), D[:, keep].reshape(-1),
                                       zeros[:, keep].reshape(-1), 3, T)
        reps.append(torch.stack([r["dE_T"], r["dcV_T"]]).cpu().numpy())
    reps = np.array(reps)
    err = orc.jackknife(reps)
    truth = _trimer_truth(T.cpu().numpy(), e_max=s.e_min + s.n_bins * s.bin_width)   # the sampled range
    est = np.stack([full["dE_T"].cpu().numpy(), full["dcV_T"].cpu().numpy()])
    ref = np.stack([truth[:, 2], truth[:, 3]])
    assert np.all(np.abs(est - ref) <= 5.0 * err + 1e-9), (est, ref, err)
    assert np.all(err < 0.1 * np.abs(ref) + 1e-6)         # the test has teeth
    ctx.close()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name,s,x", BATCHES[:3], ids=[b[0] for b in BATCHES[:3]])
def test_device_parameters_equal_host_parameters(phast, name, s, x, precision):
    """phast_energy_grad_params with the five parameters in device memory gives what
    phast_energy_grad gives for a force field holding the same values."""
    p = [1.3, 0.2, -0.7, -0.9, 0.4]                    # C_AA, C_BB, C_AB, kappa, kappa_C
    xt = torch.from_numpy(x).cuda()
    Ea, gxa, gfa = phast.phast_energy_grad(phast.with_ff_params(s, p), xt, precision)
    Eb, gxb, gfb = phast.phast_energy_grad(s, xt, precision, params=torch.tensor(p, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(Ea, Eb) and torch.equal(gxa, gxb) and torch.equal(gfa, gfb)
    with pytest.raises(phast.PhastError, match="NULL params"):
        st = phast._Structs([s])
        phast._check(phast.lib().phast_energy_grad_params(st.sys, st.ff, x.shape[0], xt.data_ptr(), precision, None,
                                                          None, None, None, phast._stream(None)))


def _straight_stretches(n_chain, n_chains, seed, box_L=0.0):
    """Chains that started straight along an irrational direction and took three
    pivots of +-0.4 rad each (FP64): their straight stretches hold dihedrals of
    collinear bonds (FP64 term 0) whose FP32 normals are rounding noise."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_chains):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        x = np.arange(n_chain)[:, None] * u[None, :] + np.array([0.0, 6.0 * c, 0.0]) + rng.normal(size=3) * 0.1
        for k in rng.choice(np.arange(2, n_chain - 2), 3, replace=False):
            a = rng.normal(size=3)
            a /= np.linalg.norm(a)
            t = rng.choice([-0.4, 0.4])
            K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
            R = np.eye(3) + np.sin(t) * K + (1 - np.cos(t)) * K @ K
            x[k + 1:] = (x[k + 1:] - x[k]) @ R.T + x[k]
        out.append(x)
    return np.concatenate(out)[None]


@pytest.mark.parametrize("name", ["fib55", "2x34"])
def test_fp32_straight_stretches(phast, orc, name):
    """FP32 energies and gradients of conformations with straight stretches: the
    dihedrals FP32 cannot resolve are taken in FP64, so the FP32 results keep the
    FP32 tolerance against the oracle (without that they were off by several
    energy units)."""
    if name == "fib55":
        s, x = inputs.config3(1)[0], _straight_stretches(55, 1, 61)
    else:
        s, x = inputs.config2(1)[2], _straight_stretches(34, 2, 62, box_L=40.0)
    E, gx, gf = phast.phast_energy_grad(s, torch.from_numpy(x).cuda(), 32)
    E, gx, gf = E.cpu().numpy(), gx.cpu().numpy(), gf.cpu().numpy()
    Eo, gxo, gfo = _oracle(orc, s, x)
    assert abs(E[0] - Eo[0]) <= 1e-4 * max(1.0, abs(Eo[0])), (E[0], Eo[0])
    assert np.max(np.abs(gx[0] - gxo[0])) <= 1e-4 * max(1.0, np.max(np.abs(gxo[0])))
    assert np.all(np.abs(gf[0] - gfo[0]) <= 1e-4 * np.maximum(1.0, np.abs(gfo[0])))
    E32 = phast.phast_energy(s, torch.from_numpy(x).cuda(), pair_precision=32).cpu().numpy()
    assert abs(E32[0] - Eo[0]) <= 1e-4 * max(1.0, abs(Eo[0])), (E32[0], Eo[0])
