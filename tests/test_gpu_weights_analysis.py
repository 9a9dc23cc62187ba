"""GPU parity of phast_weight_update (Berg recursion) and phast_micro_analysis
(Eq. 4-6, canonical reweighting, jackknife) against the FP64 oracle.

The Berg kernel integrates lnW by a parallel scan, so lnW agrees with the
oracle's running sum to rounding (1e-9 absolute over 8000 bins); every other
output is elementwise within 1e-10 relative.  Jackknife errors are compared
with the oracle run once per leave-one-block-out replicate.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def phast():
    from paper_1702_01770_gb300 import phast
    phast.lib()
    return phast


def random_hist(rng, n_blocks, K, holes=True):
    base = np.exp(3 * np.sin(np.arange(K) / 40.0)) * 50
    H = rng.poisson(base[None, :].repeat(n_blocks, 0)).astype(np.int64)
    if holes:
        H[:, : K // 10] = 0
        H[:, K // 2: K // 2 + 5] = 0
        H[:, -3:] = 0
    return H


@pytest.mark.parametrize("K,n_blocks", [(2, 1), (7, 3), (720, 1), (2000, 4), (8000, 16), (16384, 2)])
def test_weight_update_matches_oracle(phast, orc, K, n_blocks):
    rng = np.random.default_rng(K + n_blocks)
    w = 0.05
    lnW = np.cumsum(rng.normal(0, 0.1, K))
    g = np.abs(rng.normal(0, 5, K - 1)) * (rng.random(K - 1) < 0.7)
    H = random_hist(rng, n_blocks, K, holes=K > 10)
    lnW_d = torch.from_numpy(lnW.copy()).cuda()
    g_d = torch.from_numpy(g.copy()).cuda()
    beta = torch.zeros(max(K - 1, 1), dtype=torch.float64, device="cuda")
    flat = torch.zeros(4, dtype=torch.float64, device="cuda")
    phast.phast_weight_update(torch.from_numpy(H).cuda(), lnW_d, g_d, w, beta_out=beta, flat_out=flat)
    ref, g_ref, flat_ref = orc.berg_update(H.sum(0).astype(float), lnW, g, w)
    torch.cuda.synchronize()
    assert np.allclose(lnW_d.cpu().numpy(), ref, rtol=0, atol=1e-9)
    assert np.allclose(g_d.cpu().numpy(), g_ref, rtol=1e-12, atol=0)
    assert np.allclose(beta.cpu().numpy()[: K - 1], -np.diff(ref) / w, rtol=1e-6, atol=1e-6)
    assert np.allclose(flat.cpu().numpy(), flat_ref, rtol=1e-10)


def _orc_replicates(orc, lnW, H, e_min, w, h, N, T):
    full = orc.micro_analysis(lnW, e_min, w, H=H.sum(0).astype(float), fd_half_width=h, n_monomers=N, T=T)
    reps = [orc.micro_analysis(lnW, e_min, w, H=(H.sum(0) - H[b]).astype(float), fd_half_width=h, n_monomers=N, T=T)
            for b in range(H.shape[0])]
    return full, reps




def _close(a, b, rtol):
    a, b = np.asarray(a), np.asarray(b)
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(a)
    assert np.allclose(a[ok], b[ok], rtol=rtol, atol=rtol), np.max(np.abs(a[ok] - b[ok]))


@pytest.mark.parametrize("n_blocks", [1, 4, 16])
def test_micro_analysis_matches_oracle(phast, orc, n_blocks):
    rng = np.random.default_rng(n_blocks)
    K, e_min, w, h, N = 3000, -120.0, 0.1, 5, 40
    Ek = e_min + (np.arange(K) + 0.5) * w
    lnW = -(-((Ek + 40) / 30.0) ** 2 + 0.5 * np.tanh((Ek + 60) / 5.0)) * 20
    H = random_hist(rng, n_blocks, K)
    T = np.linspace(0.2, 2.0, 64)
    r = phast.phast_micro_analysis(torch.from_numpy(lnW).cuda(), e_min, w, hist=torch.from_numpy(H).cuda(),
                                   fd_half_width=h, n_monomers=N, T=torch.from_numpy(T).cuda())
    torch.cuda.synchronize()
    full, reps = _orc_replicates(orc, lnW, H, e_min, w, h, N, T)
    _close(r.S.cpu(), full["S"], 1e-12)
    _close(r.beta.cpu(), full["beta"], 1e-9)
    _close(r.CV.cpu(), full["CV"], 1e-7)
    _close(r.E_T.cpu(), full["E_T"], 1e-10)
    _close(r.cV_T.cpu(), full["cV_T"], 1e-9)
    _close(r.peak.cpu(), full["peak"], 1e-9)
    if n_blocks >= 2:
        _close(r.S_err.cpu(), orc.jackknife([x["S"] for x in reps]), 1e-8)
        _close(r.beta_err.cpu(), orc.jackknife([x["beta"] for x in reps]), 1e-6)
        _close(r.E_T_err.cpu(), orc.jackknife([x["E_T"] for x in reps]), 1e-7)
        _close(r.cV_T_err.cpu(), orc.jackknife([x["cV_T"] for x in reps]), 1e-6)
        _close(r.peak_err.cpu(), orc.jackknife([x["peak"] for x in reps]), 1e-6)
    else:
        assert r.S_err is None


def test_micro_analysis_weights_only(phast, orc):
    K, e_min, w = 500, -5.0, 0.02
    Ek = e_min + (np.arange(K) + 0.5) * w
    lnW = -(1.3 * Ek - 0.2 * Ek ** 2)
    r = phast.phast_micro_analysis(torch.from_numpy(lnW).cuda(), e_min, w, fd_half_width=3, n_monomers=7,
                                   T=torch.tensor([0.5, 1.0, 2.0], dtype=torch.float64, device="cuda"))
    ref = orc.micro_analysis(lnW, e_min, w, fd_half_width=3, n_monomers=7, T=[0.5, 1.0, 2.0])
    _close(r.S.cpu(), ref["S"], 1e-12)
    _close(r.beta.cpu(), ref["beta"], 1e-9)
    _close(r.CV.cpu(), ref["CV"], 1e-7)
    _close(r.E_T.cpu(), ref["E_T"], 1e-10)


def test_full_muca_on_trimer_recovers_exact_entropy(phast, orc):
    """Sweep -> Berg -> analysis on the GPU for the trimer, whose density of
    states is exact: S(E) within 5 jackknife errors of ln(mass)."""
    from paper_1702_01770_gb300 import inputs
    s = inputs.trimer("AAA")
    s.walkers = 512
    s.seed_base = 1000
    ctx = phast.Context(s, pair_precision=32)
    K = s.n_bins
    lnW = torch.zeros(K, dtype=torch.float64, device="cuda")
    g = torch.zeros(K - 1, dtype=torch.float64, device="cuda")
    for it in range(6):
        hs = ctx.hist_sum_zeros(16)
        ctx.sweep(400, lnW, n_jk=16, hist_sum=hs)
        if it < 5:
            phast.phast_weight_update(hs, lnW, g, s.bin_width)
    r = phast.phast_micro_analysis(lnW, s.e_min, s.bin_width, hist=hs.view(16, K), fd_half_width=2)
    torch.cuda.synchronize()
    c = -1 + (np.arange(4_000_000) + 0.5) * (2 / 4_000_000)
    u = 2 + 2 * c
    E = 0.25 * (1 - c) + 4 * (u ** -6 - u ** -3)
    k = np.floor((E - s.e_min) / s.bin_width)
    okk = (k >= 0) & (k < K)
    mass = np.bincount(k[okk].astype(int), minlength=K) / 4_000_000
    S, err = r.S.cpu().numpy(), r.S_err.cpu().numpy()
    sel = (mass > 5e-3) & ~np.isnan(S)
    exact = np.log(mass[sel])
    d = S[sel] - exact
    # S is normalised to max S = 0, so its maximum bin shows zero jackknife
    # error although it carries the normalisation's uncertainty: use the typical
    # error as a floor and remove the free additive constant
    e = np.maximum(err[sel], np.median(err[sel]))
    d -= np.average(d, weights=1 / e ** 2)
    assert np.all(np.abs(d) < 5 * e), np.max(np.abs(d) / e)
    ctx.close()


@pytest.mark.parametrize("with_hist", [True, False])
def test_binning_over_iterations_matches_oracle(phast, orc, with_hist):
    # twelve iterations of weights and histograms, blocks of three (Sec. 4.1)
    rng = np.random.default_rng(12)
    n_it, K, e_min, w, h, N, block = 12, 1500, -60.0, 0.1, 4, 30, 3
    Ek = e_min + (np.arange(K) + 0.5) * w
    base = -(-((Ek + 20) / 25.0) ** 2 + 0.4 * np.tanh((Ek + 30) / 4.0)) * 15
    lnW = np.stack([base + 0.05 * np.cumsum(rng.standard_normal(K)) / np.sqrt(K) for _ in range(n_it)])
    H = rng.poisson(200, size=(n_it, K)).astype(np.int64) if with_hist else None
    if with_hist:
        H[:, :40] = 0
        H[5, 700] = 0                                 # one iteration leaves a bin unvisited
    T = np.linspace(0.3, 3.0, 48)
    r = phast.phast_micro_analysis_binned(torch.from_numpy(lnW).cuda(), e_min, w,
                                          hist=None if H is None else torch.from_numpy(H).cuda(), block=block,
                                          fd_half_width=h, n_monomers=N, T=torch.from_numpy(T).cuda())
    torch.cuda.synchronize()
    o = orc.micro_binned(lnW, e_min, w, H, block=block, fd_half_width=h, n_monomers=N, T=T)
    for k, tol in (("S", 1e-12), ("beta", 1e-9), ("CV", 1e-7), ("E_T", 1e-10), ("cV_T", 1e-9), ("peak", 1e-9)):
        _close(getattr(r, k).cpu(), o[k], tol)
        _close(getattr(r, k + "_err").cpu(), o[k + "_err"], 1e-6)
    if with_hist:
        assert np.isnan(r.S[700].item()) and np.isnan(r.S_err[700].item())
    assert np.all(np.isfinite(r.S_err.cpu().numpy()[100:600]))


def test_binning_needs_a_full_block(phast):
    lnW = torch.zeros(2, 100, dtype=torch.float64, device="cuda")
    with pytest.raises(phast.PhastError, match="block"):
        phast.phast_micro_analysis_binned(lnW, 0.0, 0.1, block=3, fd_half_width=2)


def test_entropy_is_invariant_to_the_walker_count(phast):
    """The analogue of the paper's data collapse over processor counts (Fig. 4):
    the Fibonacci 13-mer with 256 walkers x 200 sweeps and with 1024 walkers x 50
    sweeps per iteration (the same statistics), six Berg iterations each; the
    final S(E) of the two runs agree within five combined jackknife errors on
    the well-visited bins, up to the free additive constant."""
    from paper_1702_01770_gb300 import inputs

    def run(walkers, sweeps, seed_base):
        s = inputs.config0(walkers)
        s.seed_base = seed_base
        ctx = phast.Context(s, pair_precision=32)
        K = s.n_bins
        lnW = torch.zeros(K, dtype=torch.float64, device="cuda")
        g = torch.zeros(K - 1, dtype=torch.float64, device="cuda")
        for it in range(7):
            hs = ctx.hist_sum_zeros(16)
            ctx.sweep(sweeps, lnW, n_jk=16, hist_sum=hs)
            if it < 6:
                phast.phast_weight_update(hs, lnW, g, s.bin_width)
        r = phast.phast_micro_analysis(lnW, s.e_min, s.bin_width, hist=hs.view(16, K), fd_half_width=2)
        H = hs.view(16, K).sum(0).cpu().numpy()
        torch.cuda.synchronize()
        out = r.S.cpu().numpy(), r.S_err.cpu().numpy(), H
        ctx.close()
        return out

    Sa, ea, Ha = run(256, 200, 0)
    Sb, eb, Hb = run(1024, 50, 5000)
    sel = (Ha > 300) & (Hb > 300) & np.isfinite(Sa) & np.isfinite(Sb)
    assert sel.sum() > 50, (int(sel.sum()), int(Ha.max()), int(Hb.max()), int((Ha > 0).sum()))
    e = np.sqrt(ea[sel] ** 2 + eb[sel] ** 2)
    e = np.maximum(e, np.median(e))             # the normalising bin shows no error of its own
    d = Sa[sel] - Sb[sel]
    d -= np.average(d, weights=1 / e ** 2)
    assert np.all(np.abs(d) < 5 * e), np.max(np.abs(d) / e)
