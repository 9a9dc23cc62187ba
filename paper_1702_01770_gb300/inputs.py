"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the method's arithmetic: it only builds AB sequences,
initial conformations, walker keys and the five workload descriptions (sizes,
couplings, bins, move mix).  Energies, moves, weights and analysis live in the
CUDA library (product) and, independently, in ``oracle/`` (tests).

Workloads follow the paper's systems (Sec. 4: a 2 x 9-mer dimer and a
2 x 10 + 2 x 9 cross-seeding system, Sec. 2.1 AB model with C_LJ of Eq. 1):
  * sequences: Fibonacci AB words (S0 = A, S1 = B, S_{i+1} = S_{i-1} S_i) for
    single chains, Bernoulli(f_A) draws otherwise (the paper's PDB-derived
    sequences are not available; these stand in for them);
  * conformations: straight chains, or random self-avoiding off-lattice walks
    with unit bonds and a minimum non-bonded distance, placed in a periodic
    cube with a minimum inter-chain (minimum-image) distance.
Random draws use numpy's Philox bit generator seeded per workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

A, B = 0, 1


def fibonacci_sequence(n: int) -> np.ndarray:
    """AB Fibonacci word of length n (n must be a Fibonacci number >= 1)."""
    a, b = "A", "B"
    words = [a, b]
    while len(words[-1]) < n:
        words.append(words[-2] + words[-1])
    w = next((x for x in words if len(x) == n), None)
    if w is None:
        raise ValueError(f"{n} is not the length of a Fibonacci AB word")
    return np.array([A if ch == "A" else B for ch in w], dtype=np.uint8)


def seq_to_str(seq) -> str:
    return "".join("A" if int(s) == A else "B" for s in seq)


def str_to_seq(s: str) -> np.ndarray:
    return np.array([A if ch == "A" else B for ch in s.strip()], dtype=np.uint8)


def random_sequence(n: int, frac_a: float, rng: np.random.Generator) -> np.ndarray:
    return (rng.random(n) >= frac_a).astype(np.uint8)   # A with probability frac_a


def straight_chain(n: int, origin=(0.0, 0.0, 0.0), direction=(1.0, 0.0, 0.0)) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.asarray(origin, dtype=np.float64)[None, :] + np.arange(n, dtype=np.float64)[:, None] * d


def _unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def random_saw(n: int, d_min: float, rng: np.random.Generator, max_tries: int = 200) -> np.ndarray:
    """Random self-avoiding walk: unit bonds, non-bonded distances >= d_min."""
    while True:
        x = np.zeros((n, 3))
        ok = True
        for i in range(1, n):
            for _ in range(max_tries):
                cand = x[i - 1] + _unit(rng)
                if i < 2 or np.min(np.sum((x[: i - 1] - cand) ** 2, axis=1)) >= d_min * d_min:
                    x[i] = cand
                    break
            else:
                ok = False
                break
        if ok:
            return x


def random_saws(B: int, n: int, d_min: float, rng: np.random.Generator, max_tries: int = 200) -> np.ndarray:
    """B independent random self-avoiding walks grown together (unit bonds,
    non-bonded distances >= d_min), (B, n, 3); a walk whose monomer finds no
    place in max_tries draws restarts from scratch."""
    out = np.empty((B, n, 3))
    todo = np.arange(B)
    while todo.size:
        m = todo.size
        x = np.zeros((m, n, 3))
        alive = np.ones(m, bool)
        for i in range(1, n):
            placed = np.zeros(m, bool)
            placed[~alive] = True
            for _ in range(max_tries):
                idx = np.nonzero(~placed)[0]
                if idx.size == 0:
                    break
                v = rng.normal(size=(idx.size, 3))
                v /= np.linalg.norm(v, axis=1, keepdims=True)
                cand = x[idx, i - 1] + v
                if i >= 2:
                    d2 = np.sum((x[idx, : i - 1] - cand[:, None, :]) ** 2, axis=2)
                    ok = np.min(d2, axis=1) >= d_min * d_min
                else:
                    ok = np.ones(idx.size, bool)
                x[idx[ok], i] = cand[ok]
                placed[idx[ok]] = True
            alive &= placed
        out[todo[alive]] = x[alive]
        todo = todo[~alive]
    return out


def _min_image_d2(a: np.ndarray, b: np.ndarray, L: float) -> float:
    d = a[:, None, :] - b[None, :, :]
    if L > 0:
        d = d - L * np.rint(d / L)
    return float(np.min(np.sum(d * d, axis=2)))


def place_chains(chains, box_L: float, d_min: float, rng: np.random.Generator) -> np.ndarray:
    """Translate each chain (centroid) to a uniform point of the box, rejecting
    placements closer than d_min (minimum image) to chains already placed."""
    placed = []
    for c in chains:
        c0 = c - c.mean(axis=0)
        for _ in range(10000):
            cand = c0 + rng.random(3) * box_L
            if all(_min_image_d2(cand, p, box_L) >= d_min * d_min for p in placed):
                placed.append(cand)
                break
        else:
            raise RuntimeError("could not place chains")
    return np.concatenate(placed, axis=0)


@dataclass
class System:
    """One system type: chains, sequence, box, force field and MUCA set-up."""
    name: str
    chain_len: np.ndarray
    seq: np.ndarray
    box_L: float
    k_bend: float = 0.25
    k_tors: float = 0.0
    k_lj_intra: float = 4.0
    k_lj_inter: float = 4.0
    C: tuple = (1.0, -0.5, -0.5, 0.5)          # C_LJ at 2*s_i + s_j: AA, AB, BA, BB (Eq. 1)
    sphere_R: float = 0.0                      # steric spherical container about the origin (0: none)
    k_fene: float = 0.0                        # FENE bond term of Eq. 2 (0: AB limit, rigid bonds)
    fene_r0: float = 1.0
    fene_R: float = 0.5
    C_F: tuple = (1.0, 1.0, 1.0, 1.0)          # C_F at 2*s_l + s_{l+1}
    e_min: float = -6.0
    bin_width: float = 0.05
    n_bins: int = 720
    p: tuple = (1.0, 0.0, 0.0, 0.0)            # pivot, translation, rotation, crankshaft[, bond, cap]
    amax: tuple = (0.5, 0.5, 0.3, 0.5)         # angles (rad), translation step[, bond step, cap angle]
    recompute_every: int = 0
    walkers: int = 1
    xyz0: np.ndarray = field(default=None)     # (N, 3) initial conformation shared by the walkers
    seed_base: int = 0                         # walker w gets key seed_base + w

    @property
    def n_total(self) -> int:
        return int(np.sum(self.chain_len))

    @property
    def e_max(self) -> float:
        return self.e_min + self.n_bins * self.bin_width

    def seeds(self) -> np.ndarray:
        return self.seed_base + np.arange(self.walkers, dtype=np.uint64)

    def walker_xyz(self) -> np.ndarray:
        """(walkers, N, 3) initial coordinates."""
        return np.broadcast_to(self.xyz0, (self.walkers,) + self.xyz0.shape).copy()


def _bins(e_lo: float, e_hi: float, width: float) -> int:
    return int(round((e_hi - e_lo) / width))


def config0(walkers: int = 8) -> System:
    """Fibonacci 13-mer ABBABBABABBAB, straight start, pivot only, bins of 0.05
    on [-6, 30), no torsion, FP64; walker keys 0..7."""
    seq = fibonacci_sequence(13)
    return System("fib13", np.array([13], np.int32), seq, 0.0, k_tors=0.0,
                  e_min=-6.0, bin_width=0.05, n_bins=_bins(-6, 30, 0.05), p=(1, 0, 0, 0),
                  walkers=walkers, xyz0=straight_chain(13), seed_base=0)


MIX = (0.70, 0.15, 0.15, 0.0)


def _multichain(name, n_chains, n, frac_a, seq_seed, box_L, e_lo, e_hi, width, walkers,
                recompute_every, xyz_seed, d_min=1.0) -> System:
    rng = np.random.Generator(np.random.Philox(seq_seed))
    seq = np.concatenate([random_sequence(n, frac_a, rng) for _ in range(n_chains)])
    rng_x = np.random.Generator(np.random.Philox(xyz_seed))
    chains = [random_saw(n, d_min, rng_x) for _ in range(n_chains)]
    xyz0 = place_chains(chains, box_L, d_min, rng_x)
    return System(name, np.full(n_chains, n, np.int32), seq, box_L, k_tors=-0.5,
                  e_min=e_lo, bin_width=width, n_bins=_bins(e_lo, e_hi, width), p=MIX,
                  amax=(0.5, 0.5, 0.3, 0.5), recompute_every=recompute_every,
                  walkers=walkers, xyz0=xyz0, seed_base=0)


def config1(walkers: int = 256) -> System:
    """Four 9-mers, Bernoulli(0.5) sequences from seed 1, periodic L = 20,
    torsion kappa = -0.5, 70/15/15 pivot/translation/rotation, bins 0.05 on
    [-40, 60), FP32 pairs, FP64 recompute every 100 sweeps."""
    return _multichain("4x9", 4, 9, 0.5, 1, 20.0, -40.0, 60.0, 0.05, walkers, 100, 101)


def config2(walkers_each: int = 1024) -> list:
    """Four uneven system types in one launch: a Fibonacci 13-mer, a Fibonacci
    21-mer, two 34-mers (L = 40) and eight 9-mers (L = 30), seed-2 Bernoulli(0.4)
    sequences for the multi-chain types."""
    s13 = System("fib13", np.array([13], np.int32), fibonacci_sequence(13), 0.0, k_tors=-0.5,
                 e_min=-6.0, bin_width=0.05, n_bins=_bins(-6, 30, 0.05), p=(1, 0, 0, 0),
                 recompute_every=100, walkers=walkers_each, xyz0=straight_chain(13))
    s21 = System("fib21", np.array([21], np.int32), fibonacci_sequence(21), 0.0, k_tors=-0.5,
                 e_min=-12.0, bin_width=0.05, n_bins=_bins(-12, 45, 0.05), p=(1, 0, 0, 0),
                 recompute_every=100, walkers=walkers_each, xyz0=straight_chain(21))
    s2x34 = _multichain("2x34", 2, 34, 0.4, 2, 40.0, -40.0, 80.0, 0.05, walkers_each, 100, 202)
    s8x9 = _multichain("8x9", 8, 9, 0.4, 2, 30.0, -80.0, 80.0, 0.05, walkers_each, 100, 203)
    base = 0
    for s in (s13, s21, s2x34, s8x9):
        s.seed_base = base
        base += s.walkers
    return [s13, s21, s2x34, s8x9]


def place_in_sphere(chains, sphere_R: float, d_min: float, rng: np.random.Generator) -> np.ndarray:
    """Translate each chain (centroid) to a uniform point of the ball that keeps it
    inside the sphere, rejecting placements closer than d_min to chains placed."""
    placed = []
    for c in chains:
        c0 = c - c.mean(axis=0)
        reach = sphere_R - np.max(np.linalg.norm(c0, axis=1)) - 0.5
        assert reach > 0, "chain too large for the container"
        while True:
            v = rng.uniform(-reach, reach, 3)
            if np.linalg.norm(v) > reach:
                continue
            cand = c0 + v
            if all(np.min(np.sum((p[:, None, :] - cand[None]) ** 2, axis=2)) >= d_min * d_min for p in placed):
                placed.append(cand)
                break
    return np.concatenate(placed)


def fene_sphere(walkers: int = 64, seed: int = 7) -> System:
    """The paper's own geometry: two Fibonacci 13-mers in the steric spherical
    container (radius 8) with FENE bonds (k_fene = -20, i.e. -K/2 with K = 40,
    r0 = 1, R = 0.3) and all six move types."""
    rng = np.random.Generator(np.random.Philox(seed))
    chains = [random_saw(13, 1.0, rng) for _ in range(2)]
    xyz0 = place_in_sphere(chains, 8.0, 1.0, rng)
    seq = np.concatenate([fibonacci_sequence(13), fibonacci_sequence(13)])
    return System("fene_sphere", np.array([13, 13], np.int32), seq, 0.0, k_tors=-0.5, sphere_R=8.0,
                  k_fene=-20.0, fene_r0=1.0, fene_R=0.3, e_min=-30.0, bin_width=0.05, n_bins=_bins(-30.0, 60.0, 0.05),
                  p=(0.4, 0.1, 0.1, 0.1, 0.15, 0.15), amax=(0.5, 0.3, 0.3, 0.5, 0.05, 0.5),
                  recompute_every=10, walkers=walkers, xyz0=xyz0)


def config3(batch: int = 65536, seed: int = 3):
    """Differentiation workload: one Fibonacci 55-mer (open boundaries, torsion
    kappa = -0.5) and a batch of seed-3 random self-avoiding walks of it (unit
    bonds, non-bonded distances >= 0.8).  Returns (System, xyz [batch, 55, 3])."""
    s = System("fib55", np.array([55], np.int32), fibonacci_sequence(55), 0.0, k_tors=-0.5,
               e_min=-100.0, bin_width=0.1, n_bins=_bins(-100.0, 100.0, 0.1), p=(1, 0, 0, 0),
               recompute_every=100, walkers=1, xyz0=straight_chain(55))
    rng = np.random.Generator(np.random.Philox(seed))
    return s, random_saws(batch, 55, 0.8, rng)


def config4(walkers: int = 16384) -> System:
    """Eight 55-mers (440 monomers), seed-4 Bernoulli(0.45) sequences, periodic
    L = 40, torsion kappa = -0.5, 70/15/15 mix, bins 0.1 on [-400, 400)."""
    return _multichain("8x55", 8, 55, 0.45, 4, 40.0, -400.0, 400.0, 0.1, walkers, 100, 404)


def trimer(seq: str = "AAA", k_tors: float = 0.0) -> System:
    """Three monomers, open boundaries: its density of states is known exactly."""
    return System("trimer", np.array([3], np.int32), str_to_seq(seq), 0.0, k_tors=k_tors,
                  e_min=-1.0, bin_width=0.05, n_bins=_bins(-1.0, 3.0, 0.05), p=(1, 0, 0, 0),
                  amax=(1.0, 0.5, 0.3, 0.5), walkers=1, xyz0=straight_chain(3))
