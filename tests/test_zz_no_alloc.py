"""phast_micro_analysis_noalloc: the analysis for callers that cannot allocate
device memory at the point where they run it (for example a plug-in living in
another program's CUDA context under a fixed memory budget).  It takes no
workspace and uses the library's static device scratch instead.

Checked through the C ABI against the workspace-taking phast_micro_analysis on
the same inputs, on two calls in a row with different sizes (so a second call
cannot lean on what the first left in the shared scratch); both run the same
kernels, so the results must be identical.  Also: the call leaves the device's
allocations unchanged (torch's reserved bytes and the driver's free bytes), the
weights-only form (no histogram), the argument errors it forwards, and the
size limit.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

FIELDS = ("S", "beta", "CV", "E_T", "cV_T", "peak", "S_err", "beta_err", "CV_err", "E_T_err", "cV_T_err", "peak_err")


def _inputs(seed, K, n_blocks, n_T):
    rng = np.random.default_rng(seed)
    e_min, w = -120.0, 0.1
    Ek = e_min + (np.arange(K) + 0.5) * w
    lnW = -(-((Ek + 40) / 30.0) ** 2 + 0.5 * np.tanh((Ek + 60) / 5.0)) * 20
    base = np.exp(3 * np.sin(np.arange(K) / 40.0)) * 50
    H = rng.poisson(base[None, :].repeat(n_blocks, 0)).astype(np.int64)
    H[:, : K // 10] = 0
    T = np.linspace(0.2, 2.0, n_T)
    return (torch.from_numpy(lnW).cuda(), e_min, w, torch.from_numpy(H).cuda(), torch.from_numpy(T).cuda())


def _same(a, b):
    if a is None or b is None:
        assert a is None and b is None
        return
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert np.array_equal(a, b, equal_nan=True)


def test_noalloc_matches_the_workspace_entry_point():
    from paper_1702_01770_gb300 import phast
    for call, (K, n_blocks, n_T, seed) in enumerate([(8000, 16, 64, 1), (3000, 4, 17, 2)]):
        lnW, e_min, w, H, T = _inputs(seed, K, n_blocks, n_T)
        ref = phast.phast_micro_analysis(lnW, e_min, w, hist=H, fd_half_width=5, n_monomers=440, T=T)
        got = phast.phast_micro_analysis(lnW, e_min, w, hist=H, fd_half_width=5, n_monomers=440, T=T, noalloc=True)
        torch.cuda.synchronize()
        for f in FIELDS:
            _same(getattr(got, f), getattr(ref, f))
        assert np.isfinite(got.peak.cpu().numpy()).all(), call


def test_noalloc_allocates_nothing():
    from paper_1702_01770_gb300 import phast
    lnW, e_min, w, H, T = _inputs(5, 6000, 8, 32)
    out = phast.phast_micro_analysis(lnW, e_min, w, hist=H, fd_half_width=5, n_monomers=440, T=T, noalloc=True)
    torch.cuda.synchronize()
    # the result tensors of a second call exist before it: only the call itself is measured
    ref = phast.MicroResult(*[torch.empty_like(getattr(out, f)) for f in FIELDS])
    reserved, (free, _) = torch.cuda.memory_reserved(), torch.cuda.mem_get_info()
    phast.fill_micro_analysis_noalloc(ref, lnW, e_min, w, hist=H, fd_half_width=5, n_monomers=440, T=T)
    torch.cuda.synchronize()
    assert torch.cuda.memory_reserved() == reserved
    assert torch.cuda.mem_get_info()[0] == free
    for f in FIELDS:
        _same(getattr(ref, f), getattr(out, f))


def test_noalloc_weights_only_and_argument_errors():
    from paper_1702_01770_gb300 import phast
    lnW, e_min, w, H, T = _inputs(6, 2000, 2, 8)
    ref = phast.phast_micro_analysis(lnW, e_min, w, hist=None, fd_half_width=3, n_monomers=40, T=T)
    got = phast.phast_micro_analysis(lnW, e_min, w, hist=None, fd_half_width=3, n_monomers=40, T=T, noalloc=True)
    torch.cuda.synchronize()
    for f in FIELDS:
        _same(getattr(got, f), getattr(ref, f))
    with pytest.raises(phast.PhastError, match="fd_half_width"):
        phast.phast_micro_analysis(lnW, e_min, w, hist=H, fd_half_width=0, n_monomers=40, T=T, noalloc=True)


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_1702_01770_gb300 import phast
    lnW, e_min, w, H, T = _inputs(3, 16384, 16, 64)     # 17 * (3 * 16384 + 130) doubles > 524288
    with pytest.raises(phast.PhastError, match="static workspace"):
        phast.phast_micro_analysis(lnW, e_min, w, hist=H, fd_half_width=5, n_monomers=440, T=T, noalloc=True)
