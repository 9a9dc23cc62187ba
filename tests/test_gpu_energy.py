"""GPU parity of phast_energy and phast_delta_energy (Eq. 2/3 plus torsion)
against the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 pairs 1e-11 relative to max(1, |E|); FP32 pairs 1e-4
relative to max(1, |E|) (energies are in units of the Lennard-Jones well depth,
so 1 is the natural floor); the moved coordinates must equal the oracle's bit
for bit (both sides round every geometry operation the same way).
"""
import numpy as np
import pytest
import torch

from paper_1702_01770_gb300 import inputs
from helpers import all_move_types, oracle_model, paper_cross_seeding, random_conformations

pytestmark = pytest.mark.gpu

SYSTEMS = {
    "fib13": lambda: inputs.config0(),
    "4x9": lambda: inputs.config1(1),
    "fib21": lambda: inputs.config2(1)[1],
    "2x34": lambda: inputs.config2(1)[2],
    "8x9": lambda: inputs.config2(1)[3],
    "8x55": lambda: inputs.config4(1),
    "xseed": lambda: paper_cross_seeding(1),
    "trimer": lambda: inputs.trimer("AAB", k_tors=-0.5),
}


@pytest.fixture(scope="module")
def phast():
    from paper_1702_01770_gb300 import phast
    phast.lib()
    return phast


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("prec", [64, 32])
def test_energy_matches_oracle(phast, orc, name, prec):
    s = SYSTEMS[name]()
    B = 24 if s.n_total < 200 else 6
    x = random_conformations(s, B, seed=sum(map(ord, name)) + prec)
    E = phast.phast_energy(s, torch.from_numpy(x).cuda(), pair_precision=prec).cpu().numpy()
    m = oracle_model(orc, s)
    ref = np.array([orc.energy(m, xb) for xb in x])
    tol = (1e-11 if prec == 64 else 1e-4) * np.maximum(1.0, np.abs(ref))
    assert np.all(np.abs(E - ref) <= tol), np.max(np.abs(E - ref) / np.maximum(1.0, np.abs(ref)))


def test_energy_empty_batch(phast):
    s = inputs.config0()
    E = phast.phast_energy(s, torch.empty((0, 13, 3), dtype=torch.float64, device="cuda"))
    assert E.numel() == 0


def _moves_from_oracle(orc, s, B, seed):
    m = oracle_model(orc, s)
    mu = orc.Muca(s.e_min, s.bin_width, s.n_bins, p=s.p, amax=s.amax)
    mvs = [orc.propose(m, mu, seed, t)[0] for t in range(B)]
    arr = np.zeros(B, dtype=[("type", "<i4"), ("chain", "<i4"), ("index", "<i4"), ("pad", "<i4"),
                              ("axis", "<f8", 3), ("angle", "<f8"), ("disp", "<f8", 3)])
    for i, mv in enumerate(mvs):
        arr[i] = (mv.type, mv.chain, mv.index, 0, tuple(mv.axis), mv.angle, tuple(mv.disp))
    return mvs, arr


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("prec", [64, 32])
def test_delta_energy_matches_oracle(phast, orc, name, prec):
    s = all_move_types(SYSTEMS[name]())
    B = 96 if s.n_total < 200 else 24
    x = random_conformations(s, B, seed=7 + prec)
    mvs, arr = _moves_from_oracle(orc, s, B, seed=31)
    dE, xn = phast.phast_delta_energy(s, torch.from_numpy(x).cuda(), arr, pair_precision=prec, want_xyz=True)
    dE, xn = dE.cpu().numpy(), xn.cpu().numpy()
    m = oracle_model(orc, s)
    for b in range(B):
        ref, xr = orc.delta_energy(m, x[b], mvs[b])
        assert np.array_equal(xn[b], xr), f"move {b} (type {mvs[b].type}): geometry differs from the oracle"
        tol = (1e-10 if prec == 64 else 1e-4) * max(1.0, abs(ref))
        assert abs(dE[b] - ref) <= tol, (b, mvs[b].type, dE[b], ref)


def test_delta_energy_invalid_and_degenerate_moves(phast):
    s = inputs.config1(1)
    x = np.repeat(s.xyz0[None], 5, axis=0).copy()
    # degenerate crankshaft: neighbours of monomer 1 of chain 0 put on top of each other
    x[4, 2] = x[4, 0]
    moves = [dict(type=0, chain=9, index=1), dict(type=0, chain=0, index=0),
             dict(type=2, chain=0, angle=3.0, axis=(0, 0, 1)), dict(type=7, chain=0),
             dict(type=3, chain=0, index=1, angle=0.2)]
    dE = phast.phast_delta_energy(s, torch.from_numpy(x).cuda(), moves).cpu().numpy()
    assert np.all(np.isnan(dE))


def test_rotation_moves_preserve_bonds_on_device(phast):
    s = inputs.config4(1)
    x = np.repeat(s.xyz0[None], 64, axis=0).copy()
    rng = np.random.default_rng(3)
    moves = []
    for b in range(64):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        moves.append(dict(type=b % 3 if b % 3 != 1 else 2, chain=b % 8, index=1 + b % 53,
                          axis=tuple(ax), angle=rng.uniform(-1, 1)))
    _, xn = phast.phast_delta_energy(s, torch.from_numpy(x).cuda(), moves, want_xyz=True)
    xn = xn.cpu().numpy()
    bonds = np.linalg.norm(np.diff(xn.reshape(64, 8, 55, 3), axis=2), axis=3)
    assert np.allclose(bonds, 1.0, atol=1e-13)
