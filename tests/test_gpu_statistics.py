"""Statistical parity of the FP32 sweep with the FP64 oracle on a multi-chain
workload (four 9-mers in a periodic box, L = 20, torsion kappa = -0.5, the
70/15/15 move mix; Sec. 2.2 Eq. 4-6, Sec. 4.1).

The weights come from Berg iterations of the GPU in FP32.  With those weights
fixed, the GPU (FP32 pair terms, 2048 walkers, with a group of lanes per walker or one
walker per thread) and the oracle (FP64, 64 walkers
on independent seeds) each run the same production phase from the workload's
starting conformation (equilibration, then counting); each estimates S(E) =
-lnW + ln H (Eq. 4), and the canonical specific heat c_V(T) with its peak, with
jackknife errors over 16 blocks of walkers.  The two estimates must agree within
statistical errors: S on every well-visited bin within five combined jackknife
errors (after removing the free additive constant), a chi-square per bin of
order one, and the c_V peak's temperature and height within five combined
errors.  The oracle's errors must be small enough for the test to have teeth.
"""
import dataclasses
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

from paper_1702_01770_gb300 import inputs
from helpers import oracle_model, oracle_muca

pytestmark = pytest.mark.gpu

N_BLOCKS = 16
T_GRID = np.linspace(0.3, 1.5, 64)
H_HALF = 5          # finite-difference half-width (bins) of beta(E)
EQ, PROD = 500, 8000


def _oracle_production(orc, s, lnW, walkers, seed0):
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)

    def one(i):
        wk = orc.new_walker(m, mu, s.xyz0, seed0 + i)
        orc.sweep_walker(m, mu, lnW, wk, EQ * s.n_total)
        return orc.sweep_walker(m, mu, lnW, wk, PROD * s.n_total)[0].astype(np.float64)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        H = np.array(list(ex.map(one, range(walkers))))
    Hb = H.reshape(N_BLOCKS, -1, s.n_bins).sum(1)
    kw = dict(fd_half_width=H_HALF, n_monomers=s.n_total, T=T_GRID)
    full = orc.micro_analysis(lnW, s.e_min, s.bin_width, H=Hb.sum(0), **kw)
    reps = [orc.micro_analysis(lnW, s.e_min, s.bin_width, H=Hb.sum(0) - Hb[b], **kw) for b in range(N_BLOCKS)]
    err = {k: orc.jackknife([r[k] for r in reps]) for k in ("S", "peak")}
    return full, err, Hb.sum(0)


@pytest.mark.parametrize("tile", [None, (1, 64)])
def test_fp32_entropy_and_specific_heat_agree_with_the_oracle(orc, tile):
    from paper_1702_01770_gb300 import phast
    s = inputs.config1(walkers=2048)
    K, w = s.n_bins, s.bin_width
    ctx = phast.Context(s, pair_precision=32)
    lnW = torch.zeros(K, dtype=torch.float64, device="cuda")
    g = torch.zeros(K - 1, dtype=torch.float64, device="cuda")
    hs = ctx.hist_sum_zeros(N_BLOCKS)
    for _ in range(16):                                   # Berg iterations (FP32 sweeps)
        hs.zero_()
        ctx.sweep(100, lnW, n_jk=N_BLOCKS, hist_sum=hs)
        phast.phast_weight_update(hs.view(N_BLOCKS, K), lnW, g, w)
    ctx.close()
    # production with the weights fixed, from the start, on fresh walker streams
    ctx = phast.Context(dataclasses.replace(s, seed_base=500_000), pair_precision=32)
    if tile:   # one walker per thread
        ctx.set_tile(*tile)
    ctx.sweep(EQ, lnW)
    hs.zero_()
    ctx.sweep(PROD, lnW, n_jk=N_BLOCKS, hist_sum=hs)
    r = phast.phast_micro_analysis(lnW, s.e_min, w, hist=hs.view(N_BLOCKS, K), fd_half_width=H_HALF,
                                   n_monomers=s.n_total, T=torch.from_numpy(T_GRID).cuda())
    torch.cuda.synchronize()
    S_g, S_ge = r.S.cpu().numpy(), r.S_err.cpu().numpy()
    pk_g, pk_ge = r.peak.cpu().numpy(), r.peak_err.cpu().numpy()
    H_g = hs.view(N_BLOCKS, K).sum(0).cpu().numpy()
    lnw = lnW.cpu().numpy()
    ctx.close()

    full, err, H_o = _oracle_production(orc, s, lnw, 64, seed0=10 ** 7)
    sel = (H_o >= 500) & (H_g >= 500) & np.isfinite(full["S"]) & np.isfinite(S_g)
    assert sel.sum() >= K // 2, f"only {sel.sum()} bins well visited by both"
    d = S_g[sel] - full["S"][sel]
    sig = np.sqrt(S_ge[sel] ** 2 + err["S"][sel] ** 2)
    sig = np.maximum(sig, np.median(sig))                 # the normalising bin shows no error of its own
    c = np.sum(d / sig ** 2) / np.sum(1.0 / sig ** 2)     # S is defined up to a constant
    z = np.abs(d - c) / sig
    print(f"S(E): {sel.sum()} bins, max z {z.max():.2f}, chi2/dof {np.mean(z ** 2):.3f}, "
          f"median sigma {np.median(sig):.4f}; peak gpu {pk_g} +- {pk_ge}, oracle {full['peak']} +- {err['peak']}")
    assert z.max() <= 5.0
    assert np.mean(z ** 2) <= 1.5
    assert np.median(sig) < 0.1                           # the comparison has teeth
    zp = np.abs(pk_g - full["peak"]) / np.sqrt(pk_ge ** 2 + err["peak"] ** 2)
    assert np.all(zp <= 5.0), (pk_g, pk_ge, full["peak"], err["peak"])
    assert T_GRID[2] < full["peak"][0] < T_GRID[-3]       # an interior peak
    assert err["peak"][0] < 0.05 and err["peak"][1] < 0.1 * full["peak"][1]
