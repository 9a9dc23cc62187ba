"""The sweep and the analysis at the build's hard limits (PHAST_MAX_CHAINS,
PHAST_MAX_MONOMERS, PHAST_MAX_BINS, PHAST_MAX_SYSTEMS) against the oracle."""
import dataclasses

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


def _largest(walkers):
    """16 chains x 32 monomers (512, both limits) in a periodic box of side 48,
    16384 bins of 0.125 on [-1024, 1024)."""
    rng = np.random.Generator(np.random.Philox(21))
    seq = np.concatenate([inputs.random_sequence(32, 0.5, rng) for _ in range(16)])
    chains = [inputs.random_saw(32, 1.0, rng) for _ in range(16)]
    xyz0 = inputs.place_chains(chains, 48.0, 1.0, rng)
    return inputs.System("16x32", np.full(16, 32, np.int32), seq, 48.0, k_tors=-0.5, e_min=-1024.0,
                         bin_width=0.125, n_bins=16384, p=(0.7, 0.1, 0.1, 0.1), amax=(0.5, 0.5, 0.3, 0.5),
                         recompute_every=1, walkers=walkers, xyz0=xyz0)


def test_limits_are_the_header_limits(phast):
    s = _largest(1)
    assert s.n_total == 512 and len(s.chain_len) == 16 and s.n_bins == 16384


def _oracle_walker(orc, s, lnW, n_moves, w, force=None, record=False):
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    wk = orc.new_walker(m, mu, s.xyz0, int(s.seeds()[w]))
    h, st, rec = orc.sweep_walker(m, mu, lnW, wk, n_moves, force=force, record=record)
    return wk, h, st, rec


def test_largest_system_fp64_follows_the_oracle(phast, orc):
    s = _largest(3)
    ctx = phast.Context(s, pair_precision=64)
    k = np.arange(s.n_bins)
    lnW = -0.01 * k + 0.3 * np.sin(k / 300.0)
    hw = ctx.hist_walker_zeros()
    n_sweeps = 2
    ctx.sweep(n_sweeps, torch.from_numpy(lnW).cuda(), hist_walker=hw)
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    hw = hw.cpu().numpy().reshape(s.walkers, s.n_bins)
    xyz = st["xyz"].numpy().reshape(s.walkers, s.n_total, 3)
    stt = ctx.stats()
    for w in range(s.walkers):
        wk, h, stats, _ = _oracle_walker(orc, s, lnW, n_sweeps * s.n_total, w)
        assert np.array_equal(hw[w].astype(np.uint64), h), w
        assert np.array_equal(xyz[w], wk.xyz), w
        assert abs(float(st["E"][w]) - wk.E) < 1e-9 and int(st["bin"][w]) == wk.bin
        assert int(stt["recomputes"][w]) == n_sweeps                 # a full FP64 energy every sweep
    ctx.close()


def test_largest_system_fp32_lockstep(phast, orc):
    s = _largest(2)
    ctx = phast.Context(s, pair_precision=32)
    k = np.arange(s.n_bins)
    lnW = -0.01 * k
    n_sweeps, n_tr = 2, 2
    trace = ctx.trace_buffer(n_sweeps, n_tr)
    ctx.sweep(n_sweeps, torch.from_numpy(lnW).cuda(), trace=trace, trace_walkers=n_tr)
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    tr = trace.cpu().numpy().view(phast.TRACE_DTYPE).reshape(n_tr, -1)
    xyz = st["xyz"].numpy().reshape(s.walkers, s.n_total, 3)
    for w in range(n_tr):
        f = tr[w]["accepted"].astype(np.int8)
        wk, _, stats, rec = _oracle_walker(orc, s, lnW, n_sweeps * s.n_total, w, force=f, record=True)
        check_fp32_trace_dE(orc, s, lnW, s.seeds()[w], tr[w]["dE"], rec, f, label=f"walker {w}")
        assert stats[orc.ST_MISMATCHES] <= 2
        assert np.array_equal(xyz[w], wk.xyz), w
    ctx.close()


def test_eight_system_types_in_one_context(phast, orc):
    types = inputs.config2(walkers_each=3) + [
        dataclasses.replace(inputs.config0(3), name="fib13b", seed_base=100),
        dataclasses.replace(inputs.config1(3), seed_base=200),
        dataclasses.replace(inputs.fene_sphere(3), seed_base=300),
        dataclasses.replace(inputs.trimer("ABA"), walkers=3, seed_base=400)]
    assert len(types) == 8
    ctx = phast.Context(types, pair_precision=64)
    lnW = torch.cat([torch.from_numpy(-0.02 * np.arange(t.n_bins)) for t in types]).cuda()
    hw = ctx.hist_walker_zeros()
    n_sweeps = 6
    ctx.sweep(n_sweeps, lnW, hist_walker=hw)
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    hw = hw.cpu().numpy()
    h_off = w_off = 0
    for i, t in enumerate(types):
        xyz = ctx.xyz_of(st, i).numpy()
        lw = -0.02 * np.arange(t.n_bins)
        for w in range(t.walkers):
            wk, h, _, _ = _oracle_walker(orc, t, lw, n_sweeps * t.n_total, w)
            got = hw[h_off + w * t.n_bins: h_off + (w + 1) * t.n_bins]
            assert np.array_equal(got.astype(np.uint64), h), (t.name, w)
            assert np.array_equal(xyz[w], wk.xyz), (t.name, w)
            assert abs(float(st["E"][w_off + w]) - wk.E) < 1e-9, (t.name, w)
        h_off += t.walkers * t.n_bins
        w_off += t.walkers
    ctx.close()


def test_analysis_at_the_largest_binning(phast, orc):
    rng = np.random.default_rng(16384)
    K, e_min, w, h, N, B = 16384, -1024.0, 0.125, 8, 512, 4
    Ek = e_min + (np.arange(K) + 0.5) * w
    S = np.maximum(-((Ek + 300.0) / 200.0) ** 2, 1.5 - ((Ek - 250.0) / 200.0) ** 2) * 40.0
    lnW = -S
    H = rng.poisson(50, size=(B, K)).astype(np.int64)
    H[:, :500] = 0
    T = np.linspace(2.0, 30.0, 64)
    r = phast.phast_micro_analysis(torch.from_numpy(lnW).cuda(), e_min, w, hist=torch.from_numpy(H).cuda(),
                                   fd_half_width=h, n_monomers=N, T=torch.from_numpy(T).cuda())
    f, rep, err = phast.phast_maxwell(torch.from_numpy(lnW).cuda(), torch.from_numpy(H).cuda(), e_min, w, N,
                                      fd_half_width=h)
    torch.cuda.synchronize()
    Hs = H.sum(0)
    om = orc.micro_analysis(lnW, e_min, w, H=Hs, fd_half_width=h, n_monomers=N, T=T)
    assert np.allclose(r.S.cpu().numpy(), om["S"], rtol=1e-12, atol=1e-12, equal_nan=True)
    assert np.allclose(r.cV_T.cpu().numpy(), om["cV_T"], rtol=1e-9, atol=1e-12)
    with np.errstate(divide="ignore"):
        S_in = np.where(Hs > 0, -lnW + np.log(np.where(Hs > 0, Hs, 1)), np.nan)
    fo, ro = orc.maxwell(S_in - np.nanmax(S_in), e_min, w, N, fd_half_width=h)
    row = rep[0].cpu().numpy()
    assert ro["found"] == 1.0 and row[5] == 1.0
    for q, k in enumerate(("beta_c", "eps_1", "eps_2", "latent", "barrier")):
        assert row[q] == pytest.approx(ro[k], rel=1e-12, abs=1e-12), k
    assert np.allclose(f.cpu().numpy(), fo, rtol=1e-12, atol=1e-12, equal_nan=True)
