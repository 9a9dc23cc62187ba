"""Plain FP64 CPU oracle of the PHAST multicanonical sweep (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The CUDA
product path never imports it, and it never imports the product path.  The C source (``oracle.c``) is the oracle; this file only moves
numpy arrays across the C boundary.

Paper: arXiv 1702.01770 (PHAST).  Eq. 2/3 energy, Sec. 2.2 multicanonical
sweep and Berg recursion, Eq. 4-6 microcanonical analysis.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

PIVOT, TRANS, ROT, CRANK, BOND, CAP = 0, 1, 2, 3, 4, 5
N_MOVES = 6
# orc_sweep_walker statistics: attempts[6], accepts[6], then these
ST_PAIR_EVALS, ST_RECOMPUTES, ST_DRIFT, ST_MISMATCHES = 12, 13, 14, 15


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, FP64, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(C.Structure):
    _fields_ = [("n_chains", C.c_int), ("chain_len", C.POINTER(C.c_int32)),
                ("seq", C.POINTER(C.c_uint8)), ("box_L", C.c_double),
                ("k_bend", C.c_double), ("k_tors", C.c_double),
                ("k_lj_intra", C.c_double), ("k_lj_inter", C.c_double),
                ("C", C.c_double * 4), ("sphere_R", C.c_double), ("k_fene", C.c_double),
                ("fene_r0", C.c_double), ("fene_R", C.c_double), ("C_F", C.c_double * 4)]


class _Muca(C.Structure):
    _fields_ = [("e_min", C.c_double), ("bin_width", C.c_double), ("n_bins", C.c_int32),
                ("p", C.c_double * 6), ("amax", C.c_double * 6),
                ("recompute_every", C.c_int32)]


class Move(C.Structure):
    _fields_ = [("type", C.c_int32), ("chain", C.c_int32), ("index", C.c_int32),
                ("pad", C.c_int32), ("axis", C.c_double * 3), ("angle", C.c_double),
                ("disp", C.c_double * 3)]


class _Record(C.Structure):
    _fields_ = [("dE", C.c_double), ("E_after", C.c_double),
                ("bin_after", C.c_int32), ("accepted", C.c_int32)]


RECORD_DTYPE = np.dtype([("dE", "<f8"), ("E_after", "<f8"), ("bin_after", "<i4"),
                         ("accepted", "<i4")])

_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_energy.argtypes = [P(_Model), P(C.c_double), P(C.c_double)]
        L.orc_energy.restype = C.c_double
        L.orc_energy_grad.argtypes = [P(_Model), P(C.c_double), P(C.c_double), P(C.c_double)]
        L.orc_energy_grad.restype = C.c_double
        L.orc_reweight_sensitivity.argtypes = [C.c_int64, P(C.c_double), P(C.c_double), P(C.c_double), C.c_int32,
                                               C.c_int32, P(C.c_double), P(C.c_double), P(C.c_double),
                                               P(C.c_double), P(C.c_double)]
        L.orc_reweight_sensitivity.restype = None
        L.orc_maxwell.argtypes = [C.c_int32, C.c_double, C.c_double, P(C.c_double), C.c_int32, C.c_int32,
                                  C.c_double, C.c_double, C.c_double, P(C.c_double), P(C.c_double)]
        L.orc_maxwell.restype = None
        L.orc_propose.argtypes = [P(_Model), P(_Muca), C.c_uint64, C.c_uint64, P(Move), P(C.c_double)]
        L.orc_apply_move.argtypes = [P(_Model), P(Move), P(C.c_double), P(C.c_double)]
        L.orc_apply_move.restype = C.c_int
        L.orc_move_jacobian.argtypes = [P(_Model), P(C.c_double), P(Move)]
        L.orc_move_jacobian.restype = C.c_double
        L.orc_delta_energy.argtypes = [P(_Model), P(C.c_double), P(Move), P(C.c_double)]
        L.orc_delta_energy.restype = C.c_double
        L.orc_delta_scale.argtypes = [P(_Model), P(C.c_double), P(Move)]
        L.orc_delta_scale.restype = C.c_double
        L.orc_pair_evals.argtypes = [P(_Model), P(Move)]
        L.orc_pair_evals.restype = C.c_int64
        L.orc_bin.argtypes = [P(_Muca), C.c_double]
        L.orc_bin.restype = C.c_int32
        L.orc_sweep_walker.argtypes = [P(_Model), P(_Muca), P(C.c_double), C.c_uint64, C.c_int64,
                                       P(C.c_double), P(C.c_double), P(C.c_int32), P(C.c_uint64),
                                       P(C.c_uint64), P(C.c_int8), C.c_void_p, P(C.c_double)]
        L.orc_sweep_walker.restype = C.c_int
        L.orc_berg_update.argtypes = [C.c_int32, C.c_double, P(C.c_double), P(C.c_double),
                                      P(C.c_double), P(C.c_double)]
        L.orc_micro_analysis.argtypes = [C.c_int32, C.c_double, C.c_double, P(C.c_double),
                                         P(C.c_double), C.c_int32, C.c_int32, C.c_int32,
                                         P(C.c_double), P(C.c_double), P(C.c_double),
                                         P(C.c_double), P(C.c_double), P(C.c_double),
                                         P(C.c_double)]
        L.orc_jackknife.argtypes = [C.c_int32, C.c_int32, P(C.c_double), P(C.c_double)]
        L.orc_micro_binned.argtypes = ([C.c_int32, C.c_double, C.c_double, P(C.c_double), P(C.c_double),
                                        C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P(C.c_double)]
                                       + [P(C.c_double)] * 12)
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


@dataclass
class Model:
    """Force field and system: chains, AB sequence, periodic box, couplings."""
    chain_len: np.ndarray
    seq: np.ndarray
    box_L: float = 0.0
    k_bend: float = 0.25
    k_tors: float = 0.0
    k_lj_intra: float = 4.0
    k_lj_inter: float = 4.0
    C: tuple = (1.0, -0.5, -0.5, 0.5)
    sphere_R: float = 0.0
    k_fene: float = 0.0
    fene_r0: float = 1.0
    fene_R: float = 0.5
    C_F: tuple = (1.0, 1.0, 1.0, 1.0)

    def __post_init__(self):
        self.chain_len = np.ascontiguousarray(self.chain_len, dtype=np.int32)
        self.seq = np.ascontiguousarray(self.seq, dtype=np.uint8)
        assert self.seq.size == int(self.chain_len.sum())

    @property
    def n_total(self) -> int:
        return int(self.chain_len.sum())

    def c_struct(self) -> _Model:
        s = _Model()
        s.n_chains = int(self.chain_len.size)
        s.chain_len = _ptr(self.chain_len, C.c_int32)
        s.seq = _ptr(self.seq, C.c_uint8)
        s.box_L = float(self.box_L)
        s.k_bend, s.k_tors = float(self.k_bend), float(self.k_tors)
        s.k_lj_intra, s.k_lj_inter = float(self.k_lj_intra), float(self.k_lj_inter)
        s.C = (C.c_double * 4)(*[float(c) for c in self.C])
        s.sphere_R = float(self.sphere_R)
        s.k_fene, s.fene_r0, s.fene_R = float(self.k_fene), float(self.fene_r0), float(self.fene_R)
        s.C_F = (C.c_double * 4)(*[float(c) for c in self.C_F])
        return s


@dataclass
class Muca:
    e_min: float
    bin_width: float
    n_bins: int
    p: tuple = (1.0, 0.0, 0.0, 0.0)
    amax: tuple = (0.5, 0.5, 0.3, 0.5)
    recompute_every: int = 0

    def c_struct(self) -> _Muca:
        s = _Muca()
        s.e_min, s.bin_width, s.n_bins = float(self.e_min), float(self.bin_width), int(self.n_bins)
        p = list(self.p) + [0.0] * (6 - len(self.p))
        a = list(self.amax) + [0.0] * (6 - len(self.amax))
        s.p = (C.c_double * 6)(*[float(x) for x in p])
        s.amax = (C.c_double * 6)(*[float(x) for x in a])
        s.recompute_every = int(self.recompute_every)
        return s


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def energy(model: Model, xyz, terms: bool = False):
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    assert x.size == 3 * model.n_total
    t = np.zeros(5)
    m = model.c_struct()
    e = lib().orc_energy(C.byref(m), _ptr(x, C.c_double), _ptr(t, C.c_double))
    return (e, t) if terms else e


def energy_grad(model: Model, xyz):
    """(E, dE/dxyz [N, 3], dE/d(C_AA, C_BB, C_AB, kappa, kappa_C) [5]) of one conformation."""
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    assert x.size == 3 * model.n_total
    gx, gp = np.zeros(x.size), np.zeros(5)
    m = model.c_struct()
    e = lib().orc_energy_grad(C.byref(m), _ptr(x, C.c_double), _ptr(gx, C.c_double), _ptr(gp, C.c_double))
    return e, gx.reshape(-1, 3), gp


def reweight_sensitivity(E, D, lnW, n_monomers: int, T):
    """<E>_T, c_V(T) per monomer and their derivatives in a parameter from
    multicanonical samples (energies E, derivatives D, sampling log-weights lnW)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    assert E.size == D.size == lnW.size
    out = [np.zeros(max(T.size, 1)) for _ in range(4)]
    lib().orc_reweight_sensitivity(C.c_int64(E.size), _ptr(E, C.c_double), _ptr(D, C.c_double),
                                   _ptr(lnW, C.c_double), C.c_int32(n_monomers), C.c_int32(T.size),
                                   _ptr(T, C.c_double), *[_ptr(o, C.c_double) for o in out])
    return dict(E_T=out[0][: T.size], cV_T=out[1][: T.size], dE_T=out[2][: T.size], dcV_T=out[3][: T.size])


def maxwell(S, e_min: float, bin_width: float, n_monomers: int, fd_half_width: int = 1, beta_c: float = 0.0,
            tol_beta: float = 0.0, tol_L: float = 0.0):
    """Free energy per monomer f [K] and the Maxwell construction {beta_c, eps_1, eps_2,
    latent, barrier, found} from S [K] (NaN on unvisited bins)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    f, res = np.zeros(S.size), np.zeros(6)
    lib().orc_maxwell(C.c_int32(S.size), C.c_double(e_min), C.c_double(bin_width), _ptr(S, C.c_double),
                      C.c_int32(n_monomers), C.c_int32(fd_half_width), C.c_double(beta_c), C.c_double(tol_beta),
                      C.c_double(tol_L), _ptr(f, C.c_double), _ptr(res, C.c_double))
    return f, dict(zip(("beta_c", "eps_1", "eps_2", "latent", "barrier", "found"), res))


def propose(model: Model, muca: Muca, seed: int, t: int):
    mv = Move()
    u = C.c_double()
    m, mu = model.c_struct(), muca.c_struct()
    lib().orc_propose(C.byref(m), C.byref(mu), C.c_uint64(seed), C.c_uint64(t), C.byref(mv), C.byref(u))
    return mv, u.value


def make_move(type_, chain, index=0, axis=(0.0, 0.0, 1.0), angle=0.0, disp=(0.0, 0.0, 0.0)) -> Move:
    mv = Move()
    mv.type, mv.chain, mv.index = int(type_), int(chain), int(index)
    mv.axis = (C.c_double * 3)(*axis)
    mv.angle = float(angle)
    mv.disp = (C.c_double * 3)(*disp)
    return mv


def apply_move(model: Model, mv: Move, xyz):
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    out = np.empty_like(x)
    m = model.c_struct()
    n = lib().orc_apply_move(C.byref(m), C.byref(mv), _ptr(x, C.c_double), _ptr(out, C.c_double))
    return n, out.reshape(-1, 3)


def move_jacobian(model: Model, xyz, mv: Move) -> float:
    """Hastings factor of the move from xyz (1 except for bond-length moves)."""
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    m = model.c_struct()
    return lib().orc_move_jacobian(C.byref(m), _ptr(x, C.c_double), C.byref(mv))


def delta_energy(model: Model, xyz, mv: Move):
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    out = np.empty_like(x)
    m = model.c_struct()
    dE = lib().orc_delta_energy(C.byref(m), _ptr(x, C.c_double), C.byref(mv), _ptr(out, C.c_double))
    return dE, out.reshape(-1, 3)


def delta_scale(model: Model, xyz, mv: Move) -> float:
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1)
    m = model.c_struct()
    return float(lib().orc_delta_scale(C.byref(m), _ptr(x, C.c_double), C.byref(mv)))


def pair_evals(model: Model, mv: Move) -> int:
    m = model.c_struct()
    return int(lib().orc_pair_evals(C.byref(m), C.byref(mv)))


def bin_of(muca: Muca, E: float) -> int:
    mu = muca.c_struct()
    return int(lib().orc_bin(C.byref(mu), C.c_double(E)))


@dataclass
class Walker:
    """State of one walker: coordinates, running energy, bin, move index, key."""
    xyz: np.ndarray
    E: float
    bin: int
    t: int
    seed: int


def new_walker(model: Model, muca: Muca, xyz, seed: int, t: int = 0) -> Walker:
    x = np.array(xyz, dtype=np.float64).reshape(-1, 3).copy()
    E = energy(model, x)
    return Walker(x, E, bin_of(muca, E), t, seed)


def sweep_walker(model: Model, muca: Muca, lnW, w: Walker, n_moves: int, hist=None,
                 force=None, record: bool = False):
    """Run n_moves attempts of walker w in place.  Returns (hist, stats, records)."""
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    if hist is None:
        hist = np.zeros(muca.n_bins, np.uint64)
    assert hist.dtype == np.uint64 and hist.size == muca.n_bins
    E = C.c_double(w.E)
    b = C.c_int32(w.bin)
    t = C.c_uint64(w.t)
    stats = np.zeros(16)
    rec = np.zeros(n_moves, RECORD_DTYPE) if record else None
    f = None
    if force is not None:
        f = np.ascontiguousarray(force, dtype=np.int8)
        assert f.size == n_moves
    m, mu = model.c_struct(), muca.c_struct()
    w.xyz = np.ascontiguousarray(w.xyz, dtype=np.float64)
    rc = lib().orc_sweep_walker(C.byref(m), C.byref(mu), _ptr(lnW, C.c_double), C.c_uint64(w.seed),
                                C.c_int64(n_moves), _ptr(w.xyz, C.c_double), C.byref(E), C.byref(b),
                                C.byref(t), _ptr(hist, C.c_uint64),
                                _ptr(f, C.c_int8) if f is not None else None,
                                rec.ctypes.data if rec is not None else None,
                                _ptr(stats, C.c_double))
    if rc != 0:
        raise ValueError("walker energy out of the bin range")
    w.E, w.bin, w.t = E.value, b.value, t.value
    return hist, stats, rec


def berg_update(H, lnW, g_acc, bin_width: float = 1.0):
    H = np.ascontiguousarray(H, dtype=np.float64)
    lnW = np.array(lnW, dtype=np.float64)
    g_acc = np.array(g_acc, dtype=np.float64)
    flat = np.zeros(4)
    lib().orc_berg_update(C.c_int32(H.size), C.c_double(bin_width), _ptr(H, C.c_double),
                          _ptr(lnW, C.c_double), _ptr(g_acc, C.c_double), _ptr(flat, C.c_double))
    return lnW, g_acc, flat


def jackknife(replicates):
    """Jackknife errors (Sec. 4.1, error bars from data blocks) from leave-one-block-out
    replicates [n, ...]: sqrt((n-1)/n sum_b (v_b - mean)^2) elementwise, NaN for n < 2."""
    v = np.ascontiguousarray(replicates, dtype=np.float64)
    n = v.shape[0]
    rest = v.shape[1:]
    m = int(np.prod(rest)) if rest else 1
    flat = v.reshape(n, m) if n else np.zeros((0, m))
    flat = np.ascontiguousarray(flat)
    err = np.zeros(m)
    lib().orc_jackknife(C.c_int32(n), C.c_int32(m), _ptr(flat, C.c_double) if n else None, _ptr(err, C.c_double))
    return err.reshape(rest) if rest else float(err[0])


def micro_binned(lnW, e_min: float, bin_width: float, H=None, block: int = 1, fd_half_width: int = 1,
                 n_monomers: int = 1, T=()):
    """Binning over iterations: lnW [n_it, K] and H [n_it, K] (or None) one row per
    iteration; returns the values and their *_err, as micro_analysis's keys."""
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    n_it, K = lnW.shape
    Hh = None if H is None else np.ascontiguousarray(H, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    nT = max(T.size, 1)
    out = {k: np.zeros(n) for k, n in (("S", K), ("beta", K), ("CV", K), ("E_T", nT), ("cV_T", nT), ("peak", 2))}
    err = {k + "_err": np.zeros(v.size) for k, v in out.items()}
    lib().orc_micro_binned(C.c_int32(K), C.c_double(e_min), C.c_double(bin_width), _ptr(lnW, C.c_double),
                           _ptr(Hh, C.c_double) if Hh is not None else None, C.c_int32(n_it), C.c_int32(block),
                           C.c_int32(fd_half_width), C.c_int32(n_monomers), C.c_int32(T.size), _ptr(T, C.c_double),
                           *[_ptr(out[k], C.c_double) for k in ("S", "beta", "CV", "E_T", "cV_T", "peak")],
                           *[_ptr(err[k + "_err"], C.c_double) for k in ("S", "beta", "CV", "E_T", "cV_T", "peak")])
    res = {**out, **err}
    for k in ("E_T", "cV_T", "E_T_err", "cV_T_err"):
        res[k] = res[k][: T.size]
    return res


def micro_analysis(lnW, e_min: float, bin_width: float, H=None, fd_half_width: int = 1,
                   n_monomers: int = 1, T=()):
    lnW = np.ascontiguousarray(lnW, dtype=np.float64)
    K = lnW.size
    Hh = None if H is None else np.ascontiguousarray(H, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    S, beta, CV = np.zeros(K), np.zeros(K), np.zeros(K)
    E_T, cV_T, peak = np.zeros(max(T.size, 1)), np.zeros(max(T.size, 1)), np.full(2, np.nan)
    lib().orc_micro_analysis(C.c_int32(K), C.c_double(e_min), C.c_double(bin_width),
                             _ptr(lnW, C.c_double), _ptr(Hh, C.c_double) if Hh is not None else None,
                             C.c_int32(fd_half_width), C.c_int32(n_monomers), C.c_int32(T.size),
                             _ptr(T, C.c_double), _ptr(S, C.c_double), _ptr(beta, C.c_double),
                             _ptr(CV, C.c_double), _ptr(E_T, C.c_double), _ptr(cV_T, C.c_double),
                             _ptr(peak, C.c_double))
    return dict(S=S, beta=beta, CV=CV, E_T=E_T[: T.size], cV_T=cV_T[: T.size], peak=peak)
