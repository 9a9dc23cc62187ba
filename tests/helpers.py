"""Shared test helpers: seeded conformations and oracle mirrors of the workloads."""
import numpy as np

from paper_1702_01770_gb300 import inputs


def random_conformations(s: inputs.System, B: int, seed: int, d_min: float = 0.9) -> np.ndarray:
    """B random self-avoiding conformations of system s, (B, N, 3) FP64."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.empty((B, s.n_total, 3))
    for b in range(B):
        chains = [inputs.random_saw(int(n), d_min, rng) for n in s.chain_len]
        if s.box_L > 0:
            out[b] = inputs.place_chains(chains, s.box_L, d_min, rng)
        else:
            x = np.concatenate(chains)
            out[b] = x + rng.normal(size=3) * 5.0
    return out


def oracle_model(orc, s: inputs.System):
    return orc.Model(s.chain_len, s.seq, box_L=s.box_L, k_bend=s.k_bend, k_tors=s.k_tors,
                     k_lj_intra=s.k_lj_intra, k_lj_inter=s.k_lj_inter, C=s.C)


def oracle_muca(orc, s: inputs.System):
    return orc.Muca(s.e_min, s.bin_width, s.n_bins, p=s.p, amax=s.amax, recompute_every=s.recompute_every)


def paper_cross_seeding(walkers: int = 64, box_L: float = 20.0) -> inputs.System:
    """The hIAPP/Abeta cross-seeding system of Sec. 4.2 (two 10-mers, two 9-mers),
    in a periodic box standing in for the paper's spherical container."""
    seqs = ["BBBABAAABB", "BBBABAAABB", "BBBBBAAAB", "BBBBBAAAB"]
    seq = np.concatenate([inputs.str_to_seq(q) for q in seqs])
    rng = np.random.Generator(np.random.Philox(77))
    chains = [inputs.random_saw(len(q), 1.0, rng) for q in seqs]
    xyz0 = inputs.place_chains(chains, box_L, 1.0, rng)
    return inputs.System("paper_xseed", np.array([len(q) for q in seqs], np.int32), seq, box_L, k_tors=0.0,
                         e_min=-40.0, bin_width=0.05, n_bins=2000, p=inputs.MIX, amax=(0.5, 0.5, 0.3, 0.5),
                         recompute_every=10, walkers=walkers, xyz0=xyz0)


def all_move_types(s: inputs.System) -> inputs.System:
    """Copy of s proposing all four move types (crankshaft included)."""
    import dataclasses
    p = (0.4, 0.2, 0.2, 0.2) if len(s.chain_len) > 1 else (0.7, 0.0, 0.0, 0.3)
    return dataclasses.replace(s, p=p)
