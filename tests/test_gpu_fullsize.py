"""Full-size parity: the eight-55-mer aggregation workload (16384 walkers,
L = 40, 8000 bins) in the launch configuration the benchmark times.

The oracle cannot follow 16384 walkers, so it checks samples and properties:
lockstep replay of traced walkers (every dE within the FP32 tolerance of
tests/helpers.py, decisions equal except near-ties), oracle energies of sampled walkers' final
coordinates against the GPU's running energies, bin consistency, histogram
totals per jackknife block, bond lengths, pair-evaluation counts.
"""
import numpy as np
import pytest
import torch

from paper_1702_01770_gb300 import inputs
from helpers import check_fp32_trace_dE, oracle_model, oracle_muca

pytestmark = pytest.mark.gpu


def test_config4_full_size(orc):
    from paper_1702_01770_gb300 import phast
    s = inputs.config4()
    ctx = phast.Context(s, pair_precision=32)
    n_sweeps, n_jk, n_tr = 1, 16, 2
    lnW = torch.zeros(s.n_bins, dtype=torch.float64, device="cuda")
    hs = ctx.hist_sum_zeros(n_jk)
    trace = ctx.trace_buffer(n_sweeps, n_tr)
    ctx.sweep(n_sweeps, lnW, n_jk=n_jk, hist_sum=hs, trace=trace, trace_walkers=n_tr)
    st = ctx.get_state("cpu")
    stats = ctx.stats()
    torch.cuda.synchronize()
    N = s.n_total
    hs = hs.cpu().numpy().reshape(n_jk, s.n_bins)
    assert np.all(hs.sum(1) == (s.walkers // n_jk) * n_sweeps * N)
    assert np.all(stats["attempts"].sum(1) == n_sweeps * N)
    xyz = st["xyz"].numpy().reshape(s.walkers, N, 3)
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    for w in np.linspace(0, s.walkers - 1, 12).astype(int):
        Eo = orc.energy(m, xyz[w])
        assert abs(Eo - float(st["E"][w])) <= 1e-4 * max(1.0, abs(Eo)), (w, Eo, float(st["E"][w]))
        assert orc.bin_of(mu, float(st["E"][w])) == int(st["bin"][w])
        bonds = np.linalg.norm(np.diff(xyz[w].reshape(8, 55, 3), axis=1), axis=2)
        assert np.allclose(bonds, 1.0, atol=1e-12)
    # lockstep replay of the traced walkers
    tr = trace.cpu().numpy().view(phast.TRACE_DTYPE).reshape(n_tr, -1)
    for w in range(n_tr):
        wk = orc.new_walker(m, mu, s.xyz0, int(s.seeds()[w]))
        _, so, rec = orc.sweep_walker(m, mu, lnW.cpu().numpy(), wk, n_sweeps * N,
                                      force=tr[w]["accepted"].astype(np.int8), record=True)
        check_fp32_trace_dE(orc, s, lnW.cpu().numpy(), s.seeds()[w], tr[w]["dE"], rec,
                            tr[w]["accepted"].astype(np.int8), label=f"walker {w}")
        assert so[orc.ST_MISMATCHES] <= 2                      # decisions the oracle would take differently (near-ties)
        assert int(stats["pair_evals"][w]) == int(so[orc.ST_PAIR_EVALS])
        assert abs(wk.E - float(st["E"][w])) <= 1e-4 * max(1.0, abs(wk.E))
    ctx.close()


def test_config2_full_size(orc):
    """The four uneven system types at full size (1024 walkers each) in the launch
    configuration the benchmark times: one persistent launch on the tile the
    autotuner picks there (32 lanes x 8 walkers), one multicanonical iteration
    captured as a CUDA graph (histogram clear, the sweeps, Berg's step per type).
    With the FP64 recompute due at the iteration's last move, every walker's energy
    must be the oracle's FP64 energy of its final coordinates; the histogram totals
    per jackknife block and the Berg step are checked against the oracle too."""
    import dataclasses

    from paper_1702_01770_gb300 import phast
    S, n_jk = 10, 16
    systems = [dataclasses.replace(x, recompute_every=S) for x in inputs.config2(walkers_each=1024)]
    ctx = phast.Context(systems, pair_precision=32)
    ctx.set_tile(32, 8)
    lnW = ctx.lnW_zeros()
    g = torch.zeros_like(lnW)
    hs = ctx.hist_sum_zeros(n_jk)
    flat = torch.zeros(len(systems), 4, dtype=torch.float64, device="cuda")
    graph = ctx.capture_iteration(S, lnW, hs, g, n_jk=n_jk, flat_out=flat)
    graph.launch()
    st = ctx.get_state("cpu")
    torch.cuda.synchronize()
    stats = st["stats"].numpy().view(phast.STATS_DTYPE)
    hs_all, lnW_all, g_all, flat_all = hs.cpu().numpy(), lnW.cpu().numpy(), g.cpu().numpy(), flat.cpu().numpy()
    hoff = 0
    for k, x in enumerate(systems):
        N, K, W = x.n_total, x.n_bins, x.walkers
        H = hs_all[hoff: hoff + n_jk * K].reshape(n_jk, K)
        hoff += n_jk * K
        assert np.all(H.sum(1) == (W // n_jk) * S * N), x.name
        # Berg's step from flat weights, against the oracle's on the summed histogram
        o = ctx.lnw_off[k]
        lw, ga, fl = orc.berg_update(H.sum(0).astype(np.float64), np.zeros(K), np.zeros(K - 1), x.bin_width)
        assert np.allclose(lnW_all[o: o + K], lw, rtol=1e-9, atol=1e-9), x.name
        assert np.allclose(g_all[o: o + K - 1], ga, rtol=1e-9, atol=1e-9), x.name
        assert np.allclose(flat_all[k], fl, rtol=1e-9, atol=1e-12), x.name
        sl = slice(ctx.walker_off[k], ctx.walker_off[k] + W)
        sk = stats[sl]
        assert np.all(sk["attempts"].sum(1) == S * N), x.name
        assert np.all(sk["recomputes"] == 1), x.name
        # the running FP32 energy of every walker stayed near its FP64 energy (the
        # single chains start straight: their near-collinear dihedrals are taken in FP64)
        assert sk["drift_max"].max() <= 0.02, (x.name, float(sk["drift_max"].max()))
        xyz = ctx.xyz_of(st, k).numpy()
        E, b = st["E"].numpy()[sl], st["bin"].numpy()[sl]
        m, mu = oracle_model(orc, x), oracle_muca(orc, x)
        for w in np.linspace(0, W - 1, 8).astype(int):
            Eo = orc.energy(m, xyz[w])
            assert abs(Eo - E[w]) <= 1e-10 * max(1.0, abs(Eo)), (x.name, w, Eo, E[w])
            bo = orc.bin_of(mu, Eo)
            assert b[w] == (bo if bo >= 0 else (0 if Eo < x.e_min else K - 1)), (x.name, w)
            # the running FP32 energy before the recompute stayed near the FP64 one
            assert sk["drift_max"][w] <= 1e-3 * max(1.0, abs(Eo)), (x.name, w, sk["drift_max"][w])
            off = np.concatenate([[0], np.cumsum(x.chain_len)])
            for c in range(len(x.chain_len)):
                bonds = np.linalg.norm(np.diff(xyz[w][off[c]: off[c + 1]], axis=0), axis=1)
                assert np.allclose(bonds, 1.0, atol=1e-12), (x.name, w, c)
    graph.close()
    ctx.close()
