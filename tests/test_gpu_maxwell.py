"""Free energy and Maxwell construction on the GPU (phast_maxwell) against the
oracle: synthetic entropies with a known common tangent, jackknife replicates
from block histograms, and a tabulated entropy from a multicanonical run."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

FIELDS = ("beta_c", "eps_1", "eps_2", "latent", "barrier", "found")


@pytest.fixture(scope="module")
def phast():
    from paper_1702_01770_gb300 import phast
    phast.lib()
    return phast


def _S_from(lnW, H):
    """The analysis' entropy: -lnW + ln H on visited bins, shifted to max 0."""
    with np.errstate(divide="ignore"):
        S = np.where(H > 0, -lnW + np.log(np.where(H > 0, H, 1.0)), np.nan)
    return S - np.nanmax(S)


def _check_row(row, ref):
    for q, k in enumerate(FIELDS):
        if np.isnan(ref[k]):
            assert np.isnan(row[q]), k
        else:
            assert row[q] == pytest.approx(ref[k], rel=1e-12, abs=1e-12), k


@pytest.mark.parametrize("tol_L", [0.0, 0.41])
def test_two_parabolas_against_oracle(phast, orc, tol_L):
    K, e_min, w, N = 100, -0.05, 0.1, 10
    E = e_min + (np.arange(K) + 0.5) * w
    S = np.maximum(-(E - 2.0) ** 2 / 4.0, 1.0 - (E - 6.0) ** 2 / 4.0)
    lnW = -S
    H = np.ones((1, K), np.int64)
    f, rep, err = phast.phast_maxwell(torch.from_numpy(lnW).cuda(), torch.from_numpy(H).cuda(), e_min, w, N,
                                      tol_L=tol_L)
    fo, ro = orc.maxwell(_S_from(lnW, H[0]), e_min, w, N, tol_L=tol_L)
    _check_row(rep[0].cpu().numpy(), ro)
    assert np.allclose(f.cpu().numpy(), fo, rtol=1e-12, atol=1e-12, equal_nan=True)
    if tol_L == 0.0:
        assert ro["found"] == 1.0 and ro["latent"] == pytest.approx(0.4, rel=1e-12)


def test_replicates_and_jackknife(phast, orc):
    K, e_min, w, N, B = 400, -10.0, 0.05, 13, 8
    E = e_min + (np.arange(K) + 0.5) * w
    S = np.maximum(-(E + 5.0) ** 2 / 6.0, 0.8 - (E - 2.0) ** 2 / 6.0)   # an S-bend
    rng = np.random.default_rng(4)
    lnW = -S
    H = rng.poisson(2000, size=(B, K)).astype(np.int64)
    H[:, :7] = 0                                                          # unvisited low end
    f, rep, err = phast.phast_maxwell(torch.from_numpy(lnW).cuda(), torch.from_numpy(H).cuda(), e_min, w, N,
                                      fd_half_width=3, tol_beta=0.05)
    rep, err = rep.cpu().numpy(), err.cpu().numpy()
    rows = []
    for r in range(B + 1):
        Hr = H.sum(0) if r == 0 else H.sum(0) - H[r - 1]
        fo, ro = orc.maxwell(_S_from(lnW, Hr), e_min, w, N, fd_half_width=3, tol_beta=0.05)
        _check_row(rep[r], ro)
        rows.append([ro[k] for k in FIELDS])
        if r == 0:
            assert np.allclose(f.cpu().numpy(), fo, rtol=1e-12, atol=1e-12, equal_nan=True)
    rows = np.array(rows)
    assert np.all(rows[:, 5] == 1.0)
    jk = orc.jackknife(rows[1:, :5])
    assert np.allclose(err[:5], jk, rtol=1e-9, atol=1e-15)
    assert err[5] == B


def test_given_beta_and_plain_weights(phast, orc):
    K, e_min, w, N = 720, -6.0, 0.05, 13
    E = e_min + (np.arange(K) + 0.5) * w
    lnW = 0.02 * (E - 3.0) ** 2                                            # S = -lnW, concave
    f, rep, err = phast.phast_maxwell(torch.from_numpy(lnW).cuda(), None, e_min, w, N, beta_c=1.3)
    S = -lnW - np.max(-lnW)
    fo, ro = orc.maxwell(S, e_min, w, N, beta_c=1.3)
    _check_row(rep[0].cpu().numpy(), ro)
    assert np.allclose(f.cpu().numpy(), fo, rtol=1e-12, atol=1e-12)
    assert rep.shape == (1, 6) and float(err[5]) == 0.0


def test_full_size_noisy_against_oracle(phast, orc):
    # the benchmark's binning (8000 bins of 0.1 on [-400, 400), 440 monomers, 16
    # blocks): an S-bend with Poisson noise and unvisited holes, so the hull has
    # many short edges, gaps in the chain and one long edge scanned in chunks
    K, e_min, w, N, B = 8000, -400.0, 0.1, 440, 16
    E = e_min + (np.arange(K) + 0.5) * w
    S = np.maximum(-(E + 150.0) ** 2 / 4000.0, 3.0 - (E - 120.0) ** 2 / 4000.0)
    rng = np.random.default_rng(9)
    lnW = -S
    H = rng.poisson(40, size=(B, K)).astype(np.int64)
    H[:, :300] = 0
    H[:, 5000:5013] = 0
    H[:, 7900:] = 0
    f, rep, err = phast.phast_maxwell(torch.from_numpy(lnW).cuda(), torch.from_numpy(H).cuda(), e_min, w, N,
                                      fd_half_width=5, tol_beta=0.001, tol_L=0.05)
    rep = rep.cpu().numpy()
    for r in range(B + 1):
        Hr = H.sum(0) if r == 0 else H.sum(0) - H[r - 1]
        fo, ro = orc.maxwell(_S_from(lnW, Hr), e_min, w, N, fd_half_width=5, tol_beta=0.001, tol_L=0.05)
        _check_row(rep[r], ro)
        if r == 0:
            assert ro["found"] == 1.0
            assert np.allclose(f.cpu().numpy(), fo, rtol=1e-12, atol=1e-12, equal_nan=True)


def test_negative_temperature_bend_is_no_transition(phast, orc):
    K, e_min, w, N = 100, -0.05, 0.1, 10
    E = e_min + (np.arange(K) + 0.5) * w
    S = np.maximum(-(E - 2.0) ** 2 / 4.0, 1.0 - (E - 6.0) ** 2 / 4.0)[::-1].copy()   # falling common tangent
    lnW = -S
    f, rep, err = phast.phast_maxwell(torch.from_numpy(lnW).cuda(), None, e_min, w, N)
    fo, ro = orc.maxwell(S - S.max(), e_min, w, N)
    _check_row(rep[0].cpu().numpy(), ro)
    assert ro["found"] == 0.0 and np.all(np.isnan(f.cpu().numpy()))
