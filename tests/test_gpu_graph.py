"""One multicanonical iteration captured as a CUDA graph (phast_ctx_capture_iteration)
replays exactly what the same calls made one by one compute."""
import numpy as np
import pytest
import torch

from paper_1702_01770_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def phast():
    from paper_1702_01770_gb300 import phast
    phast.lib()
    return phast


def _hs_offsets(ctx, n_jk):
    off, out = 0, []
    for K in ctx.n_bins:
        out.append(off)
        off += n_jk * K
    return out


@pytest.mark.parametrize("tile", [None, (1, 32)])
@pytest.mark.parametrize("workload", ["four types", "sphere"])
@pytest.mark.parametrize("precision", [32, 64])
def test_graph_iterations_equal_eager_calls(phast, precision, workload, tile):
    if workload == "four types":
        systems = inputs.config2(walkers_each=8)  # four uneven system types in one launch
    else:
        systems = [inputs.fene_sphere(24)]        # FENE bonds, the sphere, all six move types
    n_jk, S, iters = 2, 15, 3
    a = phast.Context(systems, pair_precision=precision)
    b = phast.Context(systems, pair_precision=precision)
    if tile:
        a.set_tile(*tile)
        b.set_tile(*tile)
    lnWa, lnWb = a.lnW_zeros(), b.lnW_zeros()
    ga, gb = torch.zeros_like(lnWa), torch.zeros_like(lnWb)
    hsa, hsb = a.hist_sum_zeros(n_jk), b.hist_sum_zeros(n_jk)
    fa = torch.zeros(len(systems), 4, dtype=torch.float64, device="cuda")
    fb = torch.zeros_like(fa)
    graph = b.capture_iteration(S, lnWb, hsb, gb, n_jk=n_jk, flat_out=fb)
    torch.cuda.synchronize()
    assert int(hsb.abs().sum()) == 0                # capturing ran nothing
    hoff = _hs_offsets(a, n_jk)
    for _ in range(iters):
        hsa.zero_()
        a.sweep(S, lnWa, n_jk=n_jk, hist_sum=hsa)
        for s, x in enumerate(systems):
            K, o = a.n_bins[s], a.lnw_off[s]
            phast.phast_weight_update(hsa[hoff[s]: hoff[s] + n_jk * K].view(n_jk, K), lnWa[o: o + K],
                                      ga[o: o + K - 1], x.bin_width, flat_out=fa[s])
        graph.launch()
    torch.cuda.synchronize()
    assert torch.equal(hsa, hsb)
    assert torch.equal(lnWa, lnWb)
    assert torch.equal(fa, fb)
    sa, sb = a.get_state("cpu"), b.get_state("cpu")
    torch.cuda.synchronize()
    for k in ("xyz", "E", "bin", "t"):
        assert torch.equal(sa[k], sb[k]), k
    # the weights moved away from flat and every type visited bins
    assert float(lnWb.abs().max()) > 0.0
    assert np.all(fb.cpu().numpy()[:, 0] > 0)
    graph.close()
    a.close()
    b.close()


def test_capture_refuses_the_default_stream(phast):
    s = inputs.config1(8)
    ctx = phast.Context(s)
    lnW = ctx.lnW_zeros()
    with pytest.raises(phast.PhastError, match="default stream"):
        ctx.capture_iteration(2, lnW, ctx.hist_sum_zeros(), torch.zeros_like(lnW),
                              stream=torch.cuda.default_stream())
    ctx.close()
