"""GPU parity of the multicanonical sweep (phast_muca_sweep) against the FP64 oracle.

* FP64 pairs (plain form and batched form): every decision and every
  per-walker histogram count equals the oracle's on the same seeds (the
  Fibonacci 13-mer workload: 8 walkers, keys 0..7, 5 Berg iterations of 10^4
  sweeps), and the walkers' coordinates agree bit for bit.
* FP32 pairs (batched form): lockstep replay -- the oracle re-runs each traced
  walker imposing the GPU's decisions and recomputes every dE in FP64; every
  dE agrees within 1e-4 relative (floor 1 energy unit) plus 2e-5 of the
  magnitude of the changed terms, and the few decisions the oracle would have
  taken differently are near-ties at a bin edge.
* Bookkeeping: jackknife-block histograms, pair-evaluation counts, resume,
  checkpoint / restore, tile invariance, error paths.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

from paper_1702_01770_gb300 import inputs
from helpers import all_move_types, check_fp32_trace_dE, oracle_model, oracle_muca, paper_cross_seeding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def phast():
    from paper_1702_01770_gb300 import phast
    phast.lib()
    return phast


def oracle_walkers(orc, s, lnW, n_moves, walkers=None, force=None, record=False, xyz=None, state=None):
    """Run the oracle on walkers of system s (threads over walkers); returns per-walker results."""
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    seeds = s.seeds()
    walkers = range(s.walkers) if walkers is None else walkers

    def one(w):
        wk = orc.new_walker(m, mu, s.xyz0 if xyz is None else xyz[w], int(seeds[w]))
        if state is not None:
            wk.E, wk.bin, wk.t = state[w]
        h, st, rec = orc.sweep_walker(m, mu, lnW, wk, n_moves, force=None if force is None else force[w],
                                      record=record)
        return wk, h, st, rec

    with ThreadPoolExecutor(max_workers=8) as ex:
        return list(ex.map(one, walkers))


def smooth_lnW(K, seed=0):
    k = np.arange(K)
    return -0.04 * k + 0.8 * np.sin(k / 17.0 + seed)


@pytest.mark.parametrize("form,tile", [("plain", None), ("batched", (8, 8)), ("batched", (32, 2)),
                                       ("batched", (1, 32))])
def test_fp64_decisions_and_histograms_bit_exact(phast, orc, form, tile):
    s = inputs.config0()
    ctx = phast.Context(s, pair_precision=64)
    if tile:
        ctx.set_tile(*tile)
    lnW = smooth_lnW(s.n_bins)
    n_sweeps = 1000
    hw = ctx.hist_walker_zeros()
    trace = ctx.trace_buffer(n_sweeps, 2)
    ctx.sweep(n_sweeps, torch.from_numpy(lnW).cuda(), form=phast.FORM_PLAIN if form == "plain" else phast.FORM_BATCHED,
              hist_walker=hw, trace=trace, trace_walkers=2)
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    hw = hw.cpu().numpy().reshape(s.walkers, s.n_bins)
    tr = trace.cpu().numpy().view(phast.TRACE_DTYPE).reshape(2, -1)
    res = oracle_walkers(orc, s, lnW, n_sweeps * s.n_total, record=True)
    xyz = st["xyz"].numpy().reshape(s.walkers, s.n_total, 3)
    for w, (wk, h, stats, rec) in enumerate(res):
        assert np.array_equal(hw[w].astype(np.uint64), h), f"walker {w}: histogram differs"
        assert np.array_equal(xyz[w], wk.xyz), f"walker {w}: coordinates differ"
        assert abs(float(st["E"][w]) - wk.E) < 1e-9 and int(st["bin"][w]) == wk.bin
        assert int(st["t"][w]) == wk.t == n_sweeps * s.n_total
        if w < 2:
            assert np.array_equal(tr[w]["accepted"], rec["accepted"])
            assert np.array_equal(tr[w]["bin_after"], rec["bin_after"])
            assert np.allclose(tr[w]["dE"], rec["dE"], rtol=1e-10, atol=1e-10)
    stt = ctx.stats()
    assert np.all(stt["attempts"].sum(1) == n_sweeps * s.n_total)
    assert np.array_equal(stt["accepts"][:, 0], np.array([r[2][orc.N_MOVES] for r in res]))
    assert np.array_equal(stt["pair_evals"], np.array([r[2][orc.ST_PAIR_EVALS] for r in res]).astype(np.uint64))
    ctx.close()


def test_config0_berg_iterations_end_to_end(phast, orc):
    """The Fibonacci 13-mer workload as specified: 8 walkers, keys 0..7, 5 Berg
    iterations of 10^4 sweeps, FP64.  Every histogram count matches the oracle,
    and the updated weights match the oracle's recursion applied to them."""
    s = inputs.config0()
    ctx = phast.Context(s, pair_precision=64)
    K = s.n_bins
    lnW = torch.zeros(K, dtype=torch.float64, device="cuda")
    g = torch.zeros(K - 1, dtype=torch.float64, device="cuda")
    flat = torch.zeros(4, dtype=torch.float64, device="cuda")
    n_sweeps = 10_000
    state = None
    xyz = None
    for it in range(5):
        lnw_in = lnW.cpu().numpy().copy()
        hw = ctx.hist_walker_zeros()
        hs = ctx.hist_sum_zeros()
        ctx.sweep(n_sweeps, lnW, form=phast.FORM_BATCHED, hist_walker=hw, hist_sum=hs)
        phast.phast_weight_update(hs, lnW, g, s.bin_width, flat_out=flat)
        torch.cuda.synchronize()
        hw = hw.cpu().numpy().reshape(s.walkers, K)
        res = oracle_walkers(orc, s, lnw_in, n_sweeps * s.n_total, xyz=xyz, state=state)
        for w, (wk, h, _, _) in enumerate(res):
            assert np.array_equal(hw[w].astype(np.uint64), h), f"iteration {it}, walker {w}"
        H = hw.sum(0).astype(np.float64)
        assert np.array_equal(hs.cpu().numpy(), hw.sum(0))
        g_ref = np.zeros(K - 1) if it == 0 else g_prev
        ref, g_ref, flat_ref = orc.berg_update(H, lnw_in, g_ref, s.bin_width)
        assert np.allclose(lnW.cpu().numpy(), ref, rtol=0, atol=1e-9)
        assert np.allclose(g.cpu().numpy(), g_ref, rtol=1e-12)
        assert np.allclose(flat.cpu().numpy(), flat_ref, rtol=1e-12)
        g_prev = g.cpu().numpy()
        xyz = [r[0].xyz for r in res]
        state = [(r[0].E, r[0].bin, r[0].t) for r in res]
    # the recursion flattens the histogram of the 13-mer over its visited range
    assert flat_ref[2] < 1.0
    ctx.close()


def _near_tie(E_o, dE_o, dE_g, s, lnW, u, b0, tol):
    """True when the two decisions can differ through the FP32 rounding of dE."""
    lo, hi = E_o + min(dE_o, dE_g) - tol, E_o + max(dE_o, dE_g) + tol
    edges = s.e_min + s.bin_width * np.arange(s.n_bins + 1)
    if np.any((edges >= lo) & (edges <= hi)):
        return True
    return False


@pytest.mark.parametrize("tile", [None, (1, 64)])
@pytest.mark.parametrize("name", ["4x9", "xseed"])
def test_fp32_lockstep_with_oracle(phast, orc, name, tile):
    s = inputs.config1(64) if name == "4x9" else paper_cross_seeding(64)
    n_tr, n_sweeps = 4, 300
    ctx = phast.Context(s, pair_precision=32)
    if tile:
        ctx.set_tile(*tile)
    lnW = smooth_lnW(s.n_bins, 1)
    trace = ctx.trace_buffer(n_sweeps, n_tr)
    ctx.sweep(n_sweeps, torch.from_numpy(lnW).cuda(), trace=trace, trace_walkers=n_tr)
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    tr = trace.cpu().numpy().view(phast.TRACE_DTYPE).reshape(n_tr, -1)
    n_moves = n_sweeps * s.n_total
    force = [tr[w]["accepted"].astype(np.int8) for w in range(n_tr)]
    res = oracle_walkers(orc, s, lnW, n_moves, walkers=range(n_tr), force=force, record=True)
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    total_mis = 0
    worst = 0.0
    for w, (wk, h, stats, rec) in enumerate(res):
        worst = max(worst, check_fp32_trace_dE(orc, s, lnW, s.seeds()[w], tr[w]["dE"], rec, force[w],
                                               label=f"walker {w}"))
        E_prev = np.concatenate([[orc.energy(m, s.xyz0)], rec["E_after"][:-1]])
        b_prev = np.concatenate([[orc.bin_of(mu, E_prev[0])], rec["bin_after"][:-1]])
        mis = 0
        for it in range(n_moves):
            E_new = E_prev[it] + rec["dE"][it]
            b = orc.bin_of(mu, E_new)
            own = 0
            if b >= 0:
                _, u = orc.propose(m, mu, int(s.seeds()[w]), it)
                dl = lnW[b] - lnW[b_prev[it]]
                own = int(dl >= 0 or u < np.exp(dl))
            if own != tr[w]["accepted"][it]:
                mis += 1
                assert _near_tie(E_prev[it], rec["dE"][it], tr[w]["dE"][it], s, lnW, 0, b_prev[it], 1e-4 * max(1.0, abs(E_new))), \
                    f"walker {w} move {it}: unexplained decision mismatch"
        assert mis == stats[orc.ST_MISMATCHES]
        total_mis += mis
        # the GPU's running energy tracks the oracle's within the FP32 budget
        assert abs(float(st["E"][w]) - wk.E) < 1e-3 * max(1.0, abs(wk.E))
    assert total_mis <= max(3, n_tr * n_moves // 2000)
    ctx.close()


def test_fp32_drift_recompute(phast, orc):
    s = inputs.config1(32)
    ctx = phast.Context(s, pair_precision=32)
    lnW = torch.zeros(s.n_bins, dtype=torch.float64, device="cuda")
    ctx.sweep(250, lnW)
    st = ctx.get_state("cpu")
    stt = ctx.stats()
    assert np.all(stt["recomputes"] == 2)
    assert stt["drift_max"].max() < 1e-3
    m = oracle_model(orc, s)
    xyz = st["xyz"].numpy().reshape(s.walkers, s.n_total, 3)
    for w in range(0, s.walkers, 7):
        Ew = orc.energy(m, xyz[w])
        assert abs(Ew - float(st["E"][w])) < 1e-3 * max(1.0, abs(Ew))
        assert orc.bin_of(oracle_muca(orc, s), float(st["E"][w])) == int(st["bin"][w])
    bonds = np.linalg.norm(np.diff(xyz.reshape(s.walkers, 4, 9, 3), axis=2), axis=3)
    assert np.allclose(bonds, 1.0, atol=1e-12)
    ctx.close()


@pytest.mark.parametrize("tile", [None, (1, 32)])
def test_uneven_batch_plain_equals_batched_fp64(phast, orc, tile):
    systems = inputs.config2(walkers_each=8)
    systems = [all_move_types(x) for x in systems]
    a = phast.Context(systems, pair_precision=64)
    b = phast.Context(systems, pair_precision=64)
    if tile:
        b.set_tile(*tile)
    lnW = torch.cat([torch.from_numpy(smooth_lnW(x.n_bins, i)) for i, x in enumerate(systems)]).cuda()
    ha, hb = a.hist_walker_zeros(), b.hist_walker_zeros()
    a.sweep(20, lnW, form=phast.FORM_PLAIN, hist_walker=ha)
    b.sweep(20, lnW, form=phast.FORM_BATCHED, hist_walker=hb)
    sa, sb = a.get_state("cpu"), b.get_state("cpu")
    torch.cuda.synchronize()
    assert torch.equal(ha.cpu(), hb.cpu())
    assert torch.equal(sa["xyz"], sb["xyz"]) and torch.equal(sa["bin"], sb["bin"])
    assert torch.allclose(sa["E"], sb["E"], rtol=0, atol=1e-9)
    # one walker of each type against the oracle
    hw = ha.cpu().numpy()
    off = 0
    for i, x in enumerate(systems):
        K = x.n_bins
        res = oracle_walkers(orc, x, smooth_lnW(K, i), 20 * x.n_total, walkers=[0, x.walkers - 1])
        for j, w in enumerate([0, x.walkers - 1]):
            assert np.array_equal(hw[off + w * K: off + (w + 1) * K].astype(np.uint64), res[j][1]), (x.name, w)
        off += x.walkers * K
    a.close()
    b.close()


@pytest.mark.parametrize("tile", [(8, 8), (1, 32)])
def test_jackknife_block_histograms(phast, tile):
    s = inputs.config1(40)
    ctx = phast.Context(s, pair_precision=32)
    ctx.set_tile(*tile)
    lnW = torch.zeros(s.n_bins, dtype=torch.float64, device="cuda")
    n_jk = 6                                # blocks of 6 or 7 walkers, tiles of 8: ragged tiles
    hs = ctx.hist_sum_zeros(n_jk)
    hw = ctx.hist_walker_zeros()
    ctx.sweep(3, lnW, n_jk=n_jk, hist_sum=hs, hist_walker=hw)
    torch.cuda.synchronize()
    hs = hs.cpu().numpy().reshape(n_jk, s.n_bins)
    hw = hw.cpu().numpy().reshape(s.walkers, s.n_bins).astype(np.int64)
    for b in range(n_jk):
        lo, hi = b * s.walkers // n_jk, (b + 1) * s.walkers // n_jk
        assert np.array_equal(hs[b], hw[lo:hi].sum(0))
    assert hs.sum() == s.walkers * 3 * s.n_total
    ctx.close()


@pytest.mark.parametrize("flush", [1, 4, 64])
def test_shared_histogram_flush_is_exact(phast, orc, flush):
    """The tile's 32-bit shared histogram moves a bin into the 64-bit sums whenever
    an increment takes it to a multiple of the flush count.  With a small flush
    count the flush runs constantly; the block sums must equal the run with the
    default count, the per-walker histograms summed per block, and the oracle's."""
    s = inputs.config0(walkers=9728)        # 608 tiles of 16 walkers: whole rounds of the grid
    lnW = torch.from_numpy(smooth_lnW(s.n_bins, 3)).cuda()
    n_jk, n_sweeps = 16, 60
    runs = []
    for count in (0, flush):
        ctx = phast.Context(s, pair_precision=64)
        ctx.set_tile(32, 16)
        ctx.set_hist_flush(count)
        hs, hw = ctx.hist_sum_zeros(n_jk), ctx.hist_walker_zeros()
        ctx.sweep(n_sweeps, lnW, n_jk=n_jk, hist_sum=hs, hist_walker=hw)
        torch.cuda.synchronize()
        runs.append((hs.cpu().numpy().reshape(n_jk, s.n_bins), hw.cpu().numpy().reshape(s.walkers, s.n_bins)))
        ctx.close()
    (hs0, hw0), (hs1, hw1) = runs
    assert np.array_equal(hs0, hs1) and np.array_equal(hw0, hw1)
    per = s.walkers // n_jk
    for b in range(n_jk):
        assert np.array_equal(hs1[b], hw1[b * per:(b + 1) * per].astype(np.int64).sum(0))
    picks = [0, 777, 4100, s.walkers - 1]
    res = oracle_walkers(orc, s, smooth_lnW(s.n_bins, 3), n_sweeps * s.n_total, walkers=picks)
    for w, r in zip(picks, res):
        assert np.array_equal(hw1[w].astype(np.uint64), r[1]), w
    assert hs1.sum() == s.walkers * n_sweeps * s.n_total


def test_histogram_bounds_are_refused(phast):
    s = inputs.config0(walkers=4)
    ctx = phast.Context(s, pair_precision=64)
    lnW = torch.zeros(s.n_bins, dtype=torch.float64, device="cuda")
    hw = ctx.hist_walker_zeros()
    n_max = (2 ** 32 - 1) // s.n_total            # the most sweeps whose counts fit a uint32
    with pytest.raises(phast.PhastError, match="2\\^32"):
        ctx.sweep(n_max + 1, lnW, hist_walker=hw)
    for bad in (3, 2 ** 31 + 1, 2 ** 32 - 1):
        with pytest.raises(phast.PhastError, match="power of two"):
            ctx.set_hist_flush(bad)
    ctx.set_hist_flush(2 ** 31)
    ctx.sweep(1, lnW, hist_walker=hw)            # a call within the bound runs
    torch.cuda.synchronize()
    assert int(hw.sum()) == 4 * s.n_total
    assert np.all(ctx.stats()["recompute_outside"] == 0)
    ctx.close()


def test_resume_and_checkpoint_bit_exact(phast):
    s = inputs.config1(16)
    lnW = torch.from_numpy(smooth_lnW(s.n_bins, 2)).cuda()
    a = phast.Context(s, pair_precision=64)
    a.sweep(10, lnW)
    b = phast.Context(s, pair_precision=64)
    b.sweep(4, lnW)
    blob = b.checkpoint()
    b.sweep(6, lnW)
    sa, sb = a.get_state("cpu"), b.get_state("cpu")
    torch.cuda.synchronize()
    for k in ("xyz", "E", "bin", "t"):
        assert torch.equal(sa[k], sb[k]), k
    b.restore(blob)
    b.sweep(6, lnW)
    sc = b.get_state("cpu")
    torch.cuda.synchronize()
    for k in ("xyz", "E", "bin", "t"):
        assert torch.equal(sa[k], sc[k]), k
    bad = bytearray(blob)
    bad[200] ^= 0xFF
    with pytest.raises(phast.PhastError, match="CRC"):
        b.restore(bytes(bad))
    with pytest.raises(phast.PhastError):
        b.restore(blob[:-8])
    a.close()
    b.close()


def test_tile_invariance_fp64(phast):
    s = paper_cross_seeding(24)
    lnW = torch.from_numpy(smooth_lnW(s.n_bins, 3)).cuda()
    out = []
    for tile in [(4, 8), (8, 16), (16, 4), (32, 2), (1, 32), (1, 64)]:
        c = phast.Context(s, pair_precision=64)
        c.set_tile(*tile)
        h = c.hist_walker_zeros()
        c.sweep(8, lnW, hist_walker=h)
        st = c.get_state("cpu")
        torch.cuda.synchronize()
        out.append((h.cpu(), st["xyz"], st["bin"]))
        c.close()
    for o in out[1:]:
        assert all(torch.equal(x, y) for x, y in zip(out[0], o))


def test_autotune_keeps_state(phast):
    s = inputs.config1(64)
    c = phast.Context(s, pair_precision=32)
    lnW = c.lnW_zeros()
    before = c.get_state("cpu")
    tile = c.autotune(lnW, sweeps=1)
    after = c.get_state("cpu")
    torch.cuda.synchronize()
    assert tile[0] in (1, 4, 8, 16, 32) and tile[0] * tile[1] % 32 == 0
    assert torch.equal(before["xyz"], after["xyz"]) and torch.equal(before["t"], after["t"])
    c.sweep(1, lnW)
    c.close()


def test_error_paths(phast):
    s = inputs.config0(walkers=2)
    import dataclasses
    far = dataclasses.replace(s, e_min=10.0)            # straight chain starts below the range
    with pytest.raises(phast.PhastError, match="PHAST_ERANGE"):
        phast.Context(far, pair_precision=64)
    c = phast.Context(s, pair_precision=64)
    lnW = c.lnW_zeros()
    with pytest.raises(phast.PhastError, match="n_jk"):
        c.sweep(1, lnW, n_jk=3, hist_sum=c.hist_sum_zeros(3))
    with pytest.raises(phast.PhastError):
        c.set_tile(5, 8)
    with pytest.raises(phast.PhastError):
        c.sweep(1, lnW, form=7)
    c.sweep(0, lnW)                                     # zero sweeps: no-op
    assert int(c.get_state("cpu")["t"][0]) == 0
    c.close()
