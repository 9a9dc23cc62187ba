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
