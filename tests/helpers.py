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
                     k_lj_intra=s.k_lj_intra, k_lj_inter=s.k_lj_inter, C=s.C, sphere_R=s.sphere_R,
                     k_fene=s.k_fene, fene_r0=s.fene_r0, fene_R=s.fene_R, C_F=s.C_F)


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


def fp32_dE_tolerance(dE_ref: float, scale: float) -> float:
    """Tolerance of an FP32-pair dE against the FP64 oracle: 1e-4 relative with
    a floor of one energy unit, plus 2e-5 of the magnitude of the terms the move
    changes (FP32 coordinates carry ~1e-7 relative rounding, which a
    Lennard-Jones term near contact amplifies ~12/r times)."""
    return 1e-4 * max(1.0, abs(dE_ref)) + 2e-5 * scale


STRICT_LOG = []   # one record per checked trace: how the FP32 dE meets the strict 1e-4 relative bound


def strict_dE_stats(dE_gpu, dE_ref) -> dict:
    """How a trace of FP32 dE meets the strict bound |err| <= 1e-4 |dE| (no floor):
    moves, failures of the strict bound, failures of the bound with a floor of
    one energy unit, the largest and 99th-percentile ratio err / (1e-4 |dE|), and
    the largest absolute error."""
    ok = np.isfinite(dE_ref) & np.isfinite(dE_gpu)
    err = np.abs(dE_gpu[ok] - dE_ref[ok])
    ref = np.abs(dE_ref[ok])
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(ref > 0, err / (1e-4 * ref), np.where(err > 0, np.inf, 0.0))
    return {"moves": int(ok.sum()), "strict_fail": int((ratio > 1.0).sum()),
            "floor1_fail": int((err > 1e-4 * np.maximum(1.0, ref)).sum()),
            "max_ratio": float(ratio.max()) if ratio.size else 0.0,
            "p99_ratio": float(np.percentile(ratio, 99)) if ratio.size else 0.0,
            "max_abs_err": float(err.max()) if err.size else 0.0}


def check_fp32_trace_dE(orc, s, lnW, seed, dE_gpu, rec, force, label=""):
    """Every finite dE of a replayed FP32 trace within fp32_dE_tolerance; the
    scale is computed (by a prefix replay) only for moves over the 1e-4 floor."""
    m, mu = oracle_model(orc, s), oracle_muca(orc, s)
    ok = np.isfinite(rec["dE"])
    assert np.array_equal(ok, np.isfinite(dE_gpu)), label
    st = strict_dE_stats(np.asarray(dE_gpu, float), np.asarray(rec["dE"], float))
    STRICT_LOG.append({"system": s.name, "label": label, **st})
    print(f"strict dE bound [{s.name} {label}]: {st}")
    err = np.zeros(ok.shape)
    err[ok] = np.abs(dE_gpu[ok] - rec["dE"][ok])
    base = 1e-4 * np.maximum(1.0, np.abs(np.where(ok, rec["dE"], 0.0)))
    worst = 0.0
    for k in np.nonzero(err > base)[0]:
        wk = orc.new_walker(m, mu, s.xyz0, int(seed))
        if k > 0:
            orc.sweep_walker(m, mu, lnW, wk, int(k), force=force[:k])
        mv, _ = orc.propose(m, mu, int(seed), int(k))
        A = orc.delta_scale(m, wk.xyz, mv)
        tol = fp32_dE_tolerance(rec["dE"][k], A)
        worst = max(worst, err[k] / tol)
        assert err[k] <= tol, (label, int(k), float(dE_gpu[k]), float(rec["dE"][k]), A)
    return worst
