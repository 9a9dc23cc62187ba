"""The paper's own geometry on the GPU -- steric container, FENE bonds,
bond-length and spherical-cap moves -- against the oracle."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

from paper_1702_01770_gb300 import inputs

from helpers import check_fp32_trace_dE, oracle_model, oracle_muca

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def phast():
    from paper_1702_01770_gb300 import phast
    phast.lib()
    return phast


def _states(orc, s, n, seed):
    """n conformations from an oracle run of the workload (inside the wall, bonds in range)."""
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    wk = orc.new_walker(m, mu, s.xyz0, seed)
    out = []
    for _ in range(n):
        orc.sweep_walker(m, mu, np.zeros(s.n_bins), wk, 26 * 20)
        out.append(wk.xyz.copy())
    return np.stack(out)


@pytest.mark.parametrize("precision", [64, 32])
def test_energy_with_wall_and_bonds(phast, orc, precision):
    s = inputs.fene_sphere(1)
    x = _states(orc, s, 6, 3)
    bad = x[0].copy()
    bad[5] *= 8.5 / np.linalg.norm(bad[5])            # a monomer beyond the wall
    xs = np.concatenate([x, bad[None]])
    E = phast.phast_energy(s, torch.from_numpy(xs).cuda(), precision).cpu().numpy()
    m = oracle_model(orc, s)
    for b in range(x.shape[0]):
        Eo = orc.energy(m, x[b])
        tol = 1e-11 if precision == 64 else 1e-4
        assert abs(E[b] - Eo) <= tol * max(1.0, abs(Eo))
    assert E[-1] == np.inf


@pytest.mark.parametrize("precision", [64, 32])
def test_delta_energy_every_move_type(phast, orc, precision):
    s = inputs.fene_sphere(1)
    x = _states(orc, s, 1, 4)[0]
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    mvs = [orc.propose(m, mu, 1234, t)[0] for t in range(400)]
    arr = np.zeros(len(mvs), phast.MOVE_DTYPE)
    for i, mv in enumerate(mvs):
        arr[i] = (mv.type, mv.chain, mv.index, 0, tuple(mv.axis), mv.angle, tuple(mv.disp))
    xs = torch.from_numpy(np.broadcast_to(x, (len(mvs),) + x.shape).copy()).cuda()
    dE, xn = phast.phast_delta_energy(s, xs, arr, precision, want_xyz=True)
    dE, xn = dE.cpu().numpy(), xn.cpu().numpy()
    seen = set()
    for i, mv in enumerate(mvs):
        dEo, yo = orc.delta_energy(m, x, mv)
        seen.add(mv.type)
        if np.isinf(dEo):
            assert dE[i] == np.inf, i
            continue
        assert np.array_equal(xn[i], yo), (i, mv.type)          # exact FP64 geometry, bit for bit
        if precision == 64:
            assert dE[i] == pytest.approx(dEo, rel=1e-9, abs=1e-9), (i, mv.type)
        else:
            A = orc.delta_scale(m, x, mv)
            assert abs(dE[i] - dEo) <= 1e-4 * max(1.0, abs(dEo)) + 2e-5 * A, (i, mv.type)
    assert seen == set(range(6))


@pytest.mark.parametrize("tile", [None, (1, 32)])
@pytest.mark.parametrize("precision", [64, 32])
def test_sweep_lockstep_with_oracle(phast, orc, precision, tile):
    s = inputs.fene_sphere(32)
    n_tr, n_sweeps = 4, 150
    ctx = phast.Context(s, pair_precision=precision)
    if tile:
        ctx.set_tile(*tile)
    k = np.arange(s.n_bins)
    lnW = -0.03 * k + 0.5 * np.sin(k / 13.0)
    trace = ctx.trace_buffer(n_sweeps, n_tr)
    ctx.sweep(n_sweeps, torch.from_numpy(lnW).cuda(), trace=trace, trace_walkers=n_tr)
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    tr = trace.cpu().numpy().view(phast.TRACE_DTYPE).reshape(n_tr, -1)
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    n_moves = n_sweeps * s.n_total
    seeds = s.seeds()

    def one(w):
        wk = orc.new_walker(m, mu, s.xyz0, int(seeds[w]))
        f = tr[w]["accepted"].astype(np.int8)
        h, stats, rec = orc.sweep_walker(m, mu, lnW, wk, n_moves, force=f, record=True)
        return wk, stats, rec, f

    with ThreadPoolExecutor(max_workers=4) as ex:
        res = list(ex.map(one, range(n_tr)))
    xyz = st["xyz"].numpy().reshape(s.walkers, s.n_total, 3)
    for w, (wk, stats, rec, f) in enumerate(res):
        dg = tr[w]["dE"].copy()
        inf_o, inf_g = np.isinf(rec["dE"]), np.isinf(dg)
        if precision == 64:
            assert np.array_equal(inf_o, inf_g), w                   # the wall and the bond range agree
        else:
            # in FP32 a bond at the edge of its range can be infinite on one side and
            # finite on the other, but then far above every bin: rejected by both
            E_prev = np.concatenate([[orc.energy(m, s.xyz0)], rec["E_after"][:-1]])
            one = inf_o != inf_g
            fin = np.where(inf_o, dg, rec["dE"])
            assert np.all(E_prev[one] + fin[one] >= s.e_max), w
            assert not np.any(tr[w]["accepted"][one]), w
            dg[one] = rec["dE"][one]
        ok = ~inf_o & np.isfinite(rec["dE"])
        if precision == 64:
            assert np.allclose(dg[ok], rec["dE"][ok], rtol=1e-9, atol=1e-9)
        else:
            check_fp32_trace_dE(orc, s, lnW, seeds[w], dg, rec, f, label=f"walker {w}")
        assert stats[orc.ST_MISMATCHES] <= 2                          # near-ties of the decision only
        assert np.array_equal(xyz[w], wk.xyz), w                      # exact coordinates, bit for bit
        assert stats[4] > 0 and stats[5] > 0 and stats[10] > 0 and stats[11] > 0
    assert np.all(np.linalg.norm(xyz, axis=2) <= 8.0)
    ctx.close()


def test_plain_and_batched_fp64_agree(phast):
    s = inputs.fene_sphere(16)
    a = phast.Context(s, pair_precision=64)
    b = phast.Context(s, pair_precision=64)
    lnW = torch.zeros(s.n_bins, dtype=torch.float64, device="cuda")
    a.sweep(40, lnW, form=phast.FORM_PLAIN)
    b.sweep(40, lnW, form=phast.FORM_BATCHED)
    sa, sb = a.get_state("cpu"), b.get_state("cpu")
    torch.cuda.synchronize()
    assert torch.equal(sa["xyz"], sb["xyz"]) and torch.equal(sa["bin"], sb["bin"])
    assert torch.allclose(sa["E"], sb["E"], rtol=0, atol=1e-9)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_gradient_with_bonds(phast, orc, precision):
    s = inputs.fene_sphere(1)
    x = _states(orc, s, 4, 8)
    E, gx, gf = phast.phast_energy_grad(s, torch.from_numpy(x).cuda(), precision)
    E, gx, gf = E.cpu().numpy(), gx.cpu().numpy(), gf.cpu().numpy()
    m = oracle_model(orc, s)
    for b in range(x.shape[0]):
        Eo, go, po = orc.energy_grad(m, x[b])
        gmax = max(1.0, np.max(np.abs(go)))
        tol = 1e-10 if precision == 64 else 1e-4
        assert abs(E[b] - Eo) <= (1e-11 if precision == 64 else 1e-4) * max(1.0, abs(Eo))
        assert np.max(np.abs(gx[b] - go)) <= tol * gmax
        assert np.all(np.abs(gf[b] - po) <= tol * np.maximum(1.0, np.abs(po)))


@pytest.mark.parametrize("precision", [64, 32])
def test_bond_moves_sample_the_cartesian_measure(phast, precision):
    # bond-length moves alone on a collinear trimer under flat weights: every
    # walker's final state is one sample of two independent bond lengths with
    # density proportional to r^2 on the FENE range (capped by the last bin)
    import dataclasses

    from test_oracle_geometry import R_F, _bond_only_trimer, _line, _stretch_marginal
    s = dataclasses.replace(_bond_only_trimer(), walkers=8192, xyz0=_line(1.0, 1.0))
    ctx = phast.Context(s, pair_precision=precision)
    ctx.sweep(1500, torch.zeros(s.n_bins, dtype=torch.float64, device="cuda"))
    xyz = ctx.get_state("cpu")["xyz"].numpy().reshape(s.walkers, 3, 3)
    torch.cuda.synchronize()
    ctx.close()
    x = ((np.linalg.norm(np.diff(xyz, axis=1), axis=2) - 1.0) / R_F).ravel()
    edges = np.linspace(-1.0, 1.0, 11)
    p = _stretch_marginal(edges, s.e_min + s.bin_width * s.n_bins)
    h = np.histogram(x, edges)[0] / x.size
    keep = p > 0.02
    assert np.max(np.abs(h[keep] / p[keep] - 1.0)) < 0.15, (h, p)
    x_mean = np.sum(p * 0.5 * (edges[1:] + edges[:-1]))
    assert abs(x.mean() - x_mean) < 0.02, (x.mean(), x_mean)     # 0 without the Hastings factor


@pytest.mark.parametrize("form", ["plain", "batched", "lane"])
def test_fp64_sweeps_follow_the_oracle_unforced(phast, orc, form):
    # no imposed decisions: the GPU and the oracle walk the same chains move for
    # move, so histograms, coordinates and per-type acceptance counts agree
    from test_gpu_sweep import oracle_walkers
    s = inputs.fene_sphere(8)
    ctx = phast.Context(s, pair_precision=64)
    if form == "lane":
        ctx.set_tile(1, 32)
    k = np.arange(s.n_bins)
    lnW = -0.02 * k + 0.6 * np.sin(k / 23.0)
    n_sweeps = 500
    hw = ctx.hist_walker_zeros()
    ctx.sweep(n_sweeps, torch.from_numpy(lnW).cuda(), form=phast.FORM_PLAIN if form == "plain" else phast.FORM_BATCHED,
              hist_walker=hw)
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    hw = hw.cpu().numpy().reshape(s.walkers, s.n_bins)
    res = oracle_walkers(orc, s, lnW, n_sweeps * s.n_total)
    xyz = st["xyz"].numpy().reshape(s.walkers, s.n_total, 3)
    stt = ctx.stats()
    for w, (wk, h, stats, _) in enumerate(res):
        assert np.array_equal(hw[w].astype(np.uint64), h), f"walker {w}: histogram differs"
        assert np.array_equal(xyz[w], wk.xyz), f"walker {w}: coordinates differ"
        assert abs(float(st["E"][w]) - wk.E) < 1e-9 and int(st["bin"][w]) == wk.bin
        assert np.array_equal(stt["attempts"][w], np.array(stats[:orc.N_MOVES]).astype(np.uint64))
        assert np.array_equal(stt["accepts"][w], np.array(stats[orc.N_MOVES:2 * orc.N_MOVES]).astype(np.uint64))
        assert stats[orc.N_MOVES + orc.BOND] > 0 and stats[orc.N_MOVES + orc.CAP] > 0
    ctx.close()


def _tight_sphere(walkers):
    """One Fibonacci 13-mer with FENE bonds pressed into a sphere of radius 2.6:
    its monomers meet the wall all the time."""
    import dataclasses
    rng = np.random.Generator(np.random.Philox(11))
    while True:
        x = inputs.random_saw(13, 1.0, rng)
        x = x - x.mean(axis=0)
        if np.max(np.linalg.norm(x, axis=1)) <= 2.0:
            break
    return dataclasses.replace(inputs.fene_sphere(walkers), name="tight_sphere", chain_len=np.array([13], np.int32),
                               seq=inputs.fibonacci_sequence(13), sphere_R=2.6, xyz0=x)


@pytest.mark.parametrize("tile", [None, (1, 64)])
@pytest.mark.parametrize("precision", [32, 64])
def test_tight_sphere_stays_inside(phast, orc, precision, tile):
    # near the wall the FP32 sweep decides with the exact positions, which must
    # include the accepted moves still waiting for their exact replay
    s = _tight_sphere(4096)
    ctx = phast.Context(s, pair_precision=precision)
    if tile:
        ctx.set_tile(*tile)
    n_tr, n_sweeps = 6, 300
    k = np.arange(s.n_bins)
    lnW = -0.02 * k
    trace = ctx.trace_buffer(n_sweeps, n_tr)
    ctx.sweep(n_sweeps, torch.from_numpy(lnW).cuda(), trace=trace, trace_walkers=n_tr)
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    xyz = st["xyz"].numpy().reshape(s.walkers, s.n_total, 3)
    r2 = (xyz[..., 0] * xyz[..., 0] + xyz[..., 1] * xyz[..., 1]) + xyz[..., 2] * xyz[..., 2]
    assert np.all(r2 <= s.sphere_R ** 2), int(np.sum(np.any(r2 > s.sphere_R ** 2, axis=1)))
    assert np.mean(np.max(r2, axis=1) > (0.95 * s.sphere_R) ** 2) > 0.3     # the chains do press on the wall
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    E = st["E"].numpy()
    for w in range(0, s.walkers, 97):
        assert abs(orc.energy(m, xyz[w]) - E[w]) <= 1e-3 * max(1.0, abs(E[w])), w
    # the traced walkers' wall rejections agree with the oracle's replay
    tr = trace.cpu().numpy().view(phast.TRACE_DTYPE).reshape(n_tr, -1)
    seeds = s.seeds()
    for w in range(n_tr):
        wk = orc.new_walker(m, mu, s.xyz0, int(seeds[w]))
        f = tr[w]["accepted"].astype(np.int8)
        _, stats, rec = orc.sweep_walker(m, mu, lnW, wk, n_sweeps * s.n_total, force=f, record=True)
        # a bond at the edge of its FENE range, or a monomer at the wall, is decided on
        # the exact positions in FP32 mode too: infinite on both sides or on neither
        assert np.array_equal(np.isinf(rec["dE"]), np.isinf(tr[w]["dE"])), w
        assert np.array_equal(xyz[w], wk.xyz), w
    ctx.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_bond_move_edge_cases(phast, orc, precision):
    # a bond shrunk through zero length is no move (NaN, coordinates unchanged);
    # a stretch beyond the FENE range and a step into the wall are infinite
    s = inputs.fene_sphere(1)
    x = _states(orc, s, 1, 5)[0]
    m = oracle_model(orc, s)
    r3 = float(np.linalg.norm(x[4] - x[3]))
    mvs = [orc.make_move(orc.BOND, 0, 3, angle=-(r3 + 0.5)),     # through zero length
           orc.make_move(orc.BOND, 0, 3, angle=0.35),            # |r - r0| beyond R = 0.3
           orc.make_move(orc.BOND, 1, 6, angle=0.02),            # an ordinary stretch
           orc.make_move(orc.TRANS, 0, 0, disp=(30.0, 0.0, 0.0))]  # into the wall
    arr = np.zeros(len(mvs), phast.MOVE_DTYPE)
    for i, mv in enumerate(mvs):
        arr[i] = (mv.type, mv.chain, mv.index, 0, tuple(mv.axis), mv.angle, tuple(mv.disp))
    xs = torch.from_numpy(np.broadcast_to(x, (len(mvs),) + x.shape).copy()).cuda()
    dE, xn = phast.phast_delta_energy(s, xs, arr, precision, want_xyz=True)
    dE, xn = dE.cpu().numpy(), xn.cpu().numpy()
    ref = [orc.delta_energy(m, x, mv) for mv in mvs]
    assert np.isnan(ref[0][0]) and np.isnan(dE[0]) and np.array_equal(xn[0], x)
    assert ref[1][0] == np.inf and dE[1] == np.inf
    assert np.isfinite(dE[2]) and np.array_equal(xn[2], ref[2][1])
    assert abs(dE[2] - ref[2][0]) <= (1e-9 if precision == 64 else 1e-4) * max(1.0, abs(ref[2][0]))
    assert ref[3][0] == np.inf and dE[3] == np.inf


@pytest.mark.parametrize("tile", [(16, 32), (1, 128)])
def test_fene_divergence_is_decided_exactly(phast, tile):
    # weights that favour high energies drive bonds to the edge of their FENE range,
    # where an FP32 bond length cannot tell a finite term from the divergence: no
    # accepted move may leave a state whose exact FP64 energy is infinite
    s = inputs.fene_sphere(16384)
    ctx = phast.Context(s, pair_precision=32)
    ctx.set_tile(*tile)
    k = np.arange(s.n_bins)
    lnW = -0.02 * k + 0.5 * np.sin(k / 13.0)
    ctx.sweep(400, torch.from_numpy(lnW).cuda())
    st, stt = ctx.get_state("cpu"), ctx.stats()
    torch.cuda.synchronize()
    xyz = st["xyz"].numpy().reshape(s.walkers, s.n_total, 3)
    E64 = phast.phast_energy(s, torch.from_numpy(xyz).cuda(), 64).cpu().numpy()
    assert np.all(np.isfinite(E64)), int(np.sum(~np.isfinite(E64)))
    drift = stt["drift_max"]
    assert np.all(np.isfinite(drift)) and drift.max() < 0.05, drift.max()
    # the last move of the run is followed by a recompute: the running energy is the FP64 one
    assert np.allclose(st["E"].numpy(), E64, rtol=1e-12, atol=1e-9)
    b = np.concatenate([np.linalg.norm(xyz[:, o + 1:o + 13] - xyz[:, o:o + 12], axis=2) for o in (0, 13)], axis=1)
    x2 = ((b - s.fene_r0) / s.fene_R) ** 2
    print(f"bonds with x^2 > 0.99: {int(np.sum(x2 > 0.99))}, largest x^2 {x2.max():.6f}")
    assert x2.max() < 1.0 and np.sum(x2 > 0.95) > 0          # the bonds do reach the edge of their range
    ctx.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_wall_at_the_edge_of_the_fp32_band(phast, orc, precision):
    # translations that leave a monomer a hair off the wall, around r^2 - R^2 =
    # +-1e-5 R^2 where FP32 mode hands the decision to the exact positions (a few
    # FP32 ulps of r^2 either side): the wall is infinite exactly where the
    # oracle's FP64 test puts it
    s = inputs.fene_sphere(1)
    x = _states(orc, s, 1, 6)[0]
    m = oracle_model(orc, s)
    R2 = s.sphere_R ** 2
    c = x[:13]
    rng = np.random.Generator(np.random.Philox(12))
    targets = R2 * np.concatenate([1e-5 + rng.uniform(-4e-7, 4e-7, 300), -1e-5 + rng.uniform(-4e-7, 4e-7, 100)])
    mvs = []
    for tg in targets:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        lo, hi = 0.0, 20.0                      # max_k |c_k + d u|^2 - R^2 - tg changes sign in [lo, hi]
        for _ in range(200):
            d = 0.5 * (lo + hi)
            f = np.max(np.sum((c + d * u) ** 2, axis=1)) - R2 - tg
            lo, hi = (d, hi) if f < 0 else (lo, d)
        mvs.append(orc.make_move(orc.TRANS, 0, 0, disp=tuple(hi * u)))
    arr = np.zeros(len(mvs), phast.MOVE_DTYPE)
    for i, mv in enumerate(mvs):
        arr[i] = (mv.type, mv.chain, mv.index, 0, tuple(mv.axis), mv.angle, tuple(mv.disp))
    xs = torch.from_numpy(np.broadcast_to(x, (len(mvs),) + x.shape).copy()).cuda()
    dE = phast.phast_delta_energy(s, xs, arr, precision).cpu().numpy()
    dEo = np.array([orc.delta_energy(m, x, mv)[0] for mv in mvs])
    assert np.sum(np.isinf(dEo)) >= 250 and np.sum(np.isfinite(dEo)) >= 80
    bad = np.nonzero(np.isinf(dE) != np.isinf(dEo))[0]
    assert bad.size == 0, [(int(i), float(targets[i] / R2), float(dE[i]), float(dEo[i])) for i in bad[:5]]
