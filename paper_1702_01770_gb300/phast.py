"""Python binding of libphast.so (include/phast.h), argument marshalling only.

Every computation happens in the CUDA library; torch tensors provide device
memory and the stream.  The functions keep the C names.  The library must be
built (``__graft_entry__.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libphast.so")

PIVOT, TRANS, ROT, CRANK = 0, 1, 2, 3
FORM_BATCHED, FORM_PLAIN = 0, 1
MAX_SYSTEMS, MAX_CHAINS, MAX_MONOMERS, MAX_BINS = 8, 16, 512, 16384
ERRORS = {0: "PHAST_OK", -1: "PHAST_EINVAL", -2: "PHAST_ERANGE", -3: "PHAST_ENOMEM", -4: "PHAST_ECUDA",
          -5: "PHAST_ETIMEOUT", -6: "PHAST_EDEVICE", -7: "PHAST_ENONFINITE"}
SYMBOLS = ["phast_energy", "phast_delta_energy", "phast_ctx_create", "phast_ctx_destroy", "phast_ctx_info",
           "phast_ctx_get_state", "phast_ctx_set_state", "phast_ctx_set_tile", "phast_ctx_get_tile",
           "phast_ctx_autotune", "phast_muca_sweep", "phast_weight_update", "phast_micro_workspace_size",
           "phast_micro_analysis", "phast_micro_analysis_noalloc", "phast_ctx_checkpoint", "phast_ctx_restore", "phast_last_error",
           "phast_version", "phast_ctx_capture_iteration", "phast_graph_launch",
           "phast_graph_destroy", "phast_energy_grad",
           "phast_reweight_sensitivity", "phast_maxwell", "phast_micro_binned_workspace_size",
           "phast_micro_analysis_binned", "phast_ctx_set_hist_flush", "phast_energy_grad_params"]


class PhastError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


N_MOVES = 6   # pivot, translation, rotation, crankshaft, bond length, spherical cap


class _System(C.Structure):
    _fields_ = [("n_chains", C.c_int32), ("chain_len", C.POINTER(C.c_int32)),
                ("seq", C.POINTER(C.c_uint8)), ("box_L", C.c_double), ("sphere_R", C.c_double)]


class _FF(C.Structure):
    _fields_ = [("k_bend", C.c_double), ("k_tors", C.c_double), ("k_lj_intra", C.c_double),
                ("k_lj_inter", C.c_double), ("C", C.c_double * 4), ("k_fene", C.c_double),
                ("fene_r0", C.c_double), ("fene_R", C.c_double), ("C_F", C.c_double * 4)]


class _Muca(C.Structure):
    _fields_ = [("e_min", C.c_double), ("bin_width", C.c_double), ("n_bins", C.c_int32),
                ("recompute_every", C.c_int32), ("p", C.c_double * N_MOVES), ("amax", C.c_double * N_MOVES),
                ("pair_precision", C.c_int32), ("pad", C.c_int32)]


class _MicroOut(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("S", "beta", "CV", "E_T", "cV_T", "peak", "S_err", "beta_err",
                                            "CV_err", "E_T_err", "cV_T_err", "peak_err")]


MOVE_DTYPE = np.dtype([("type", "<i4"), ("chain", "<i4"), ("index", "<i4"), ("pad", "<i4"),
                       ("axis", "<f8", 3), ("angle", "<f8"), ("disp", "<f8", 3)])
STATS_DTYPE = np.dtype([("attempts", "<u8", N_MOVES), ("accepts", "<u8", N_MOVES), ("pair_evals", "<u8"),
                        ("pair_evals_inter", "<u8"), ("recomputes", "<u8"), ("drift_max", "<f8"),
                        ("recompute_outside", "<u8"), ("pad", "<u8")])
TRACE_DTYPE = np.dtype([("dE", "<f8"), ("bin_after", "<i4"), ("accepted", "<i4")])

_lib = None


def lib():
    """Load libphast.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl, P = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.POINTER
        L.phast_energy.argtypes = [P(_System), P(_FF), i32, vp, i32, vp, vp]
        L.phast_delta_energy.argtypes = [P(_System), P(_FF), i32, vp, vp, i32, vp, vp, vp]
        L.phast_ctx_create.argtypes = [P(vp), i32, P(_System), P(_FF), P(_Muca), vp, vp, vp, vp]
        L.phast_ctx_destroy.argtypes = [vp]
        L.phast_ctx_destroy.restype = None
        L.phast_ctx_info.argtypes = [vp, i32, vp]
        L.phast_ctx_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.phast_ctx_set_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.phast_ctx_set_tile.argtypes = [vp, i32, i32]
        L.phast_ctx_get_tile.argtypes = [vp, P(i32), P(i32)]
        L.phast_ctx_set_hist_flush.argtypes = [vp, C.c_uint32]
        L.phast_ctx_autotune.argtypes = [vp, vp, i32, vp]
        L.phast_muca_sweep.argtypes = [vp, i64, vp, i32, i32, vp, vp, vp, i32, vp]
        L.phast_weight_update.argtypes = [i32, dbl, vp, i32, vp, vp, vp, vp, vp]
        L.phast_micro_workspace_size.argtypes = [i32, i32, i32]
        L.phast_micro_workspace_size.restype = C.c_size_t
        L.phast_micro_binned_workspace_size.argtypes = [i32, i32, i32]
        L.phast_micro_binned_workspace_size.restype = C.c_size_t
        L.phast_micro_analysis_binned.argtypes = [i32, dbl, dbl, vp, vp, i32, i32, i32, i32, i32, vp, P(_MicroOut),
                                                  vp, C.c_size_t, vp]
        L.phast_micro_analysis.argtypes = [i32, dbl, dbl, vp, vp, i32, i32, i32, i32, vp, P(_MicroOut), vp,
                                           C.c_size_t, vp]
        L.phast_micro_analysis_noalloc.argtypes = [i32, dbl, dbl, vp, vp, i32, i32, i32, i32, vp, P(_MicroOut),
                                                   vp]
        L.phast_maxwell.argtypes = [i32, dbl, dbl, vp, vp, i32, i32, i32, dbl, dbl, dbl, vp, vp, vp, vp]
        L.phast_energy_grad.argtypes = [P(_System), P(_FF), i32, vp, i32, vp, vp, vp, vp]
        L.phast_energy_grad_params.argtypes = [P(_System), P(_FF), i32, vp, i32, vp, vp, vp, vp, vp]
        L.phast_reweight_sensitivity.argtypes = [i64, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp]
        L.phast_ctx_capture_iteration.argtypes = [vp, i64, vp, i32, vp, vp, vp, P(vp), vp]
        L.phast_graph_launch.argtypes = [vp, vp]
        L.phast_graph_destroy.argtypes = [vp]
        L.phast_graph_destroy.restype = None
        L.phast_ctx_checkpoint.argtypes = [vp, vp, P(C.c_size_t), vp]
        L.phast_ctx_restore.argtypes = [vp, vp, C.c_size_t, vp]
        L.phast_last_error.restype = C.c_char_p
        L.phast_last_error.argtypes = []
        L.phast_version.argtypes = []
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise PhastError(rc, lib().phast_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous(), "tensors crossing the C ABI must be contiguous"
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    raise TypeError(type(t))


class _Structs:
    """ABI structs of a list of systems, with the host arrays they point to kept alive."""

    def __init__(self, systems, pair_precision: int | None = None):
        n = len(systems)
        self.keep = []
        self.sys = (_System * n)()
        self.ff = (_FF * n)()
        self.mp = (_Muca * n)()
        for i, s in enumerate(systems):
            cl = np.ascontiguousarray(s.chain_len, dtype=np.int32)
            sq = np.ascontiguousarray(s.seq, dtype=np.uint8)
            self.keep += [cl, sq]
            self.sys[i].n_chains = cl.size
            self.sys[i].chain_len = cl.ctypes.data_as(C.POINTER(C.c_int32))
            self.sys[i].seq = sq.ctypes.data_as(C.POINTER(C.c_uint8))
            self.sys[i].box_L = float(s.box_L)
            self.sys[i].sphere_R = float(s.sphere_R)
            self.ff[i].k_bend, self.ff[i].k_tors = float(s.k_bend), float(s.k_tors)
            self.ff[i].k_lj_intra, self.ff[i].k_lj_inter = float(s.k_lj_intra), float(s.k_lj_inter)
            self.ff[i].C = (C.c_double * 4)(*[float(c) for c in s.C])
            self.ff[i].k_fene, self.ff[i].fene_r0, self.ff[i].fene_R = float(s.k_fene), float(s.fene_r0), float(s.fene_R)
            self.ff[i].C_F = (C.c_double * 4)(*[float(c) for c in s.C_F])
            self.mp[i].e_min, self.mp[i].bin_width = float(s.e_min), float(s.bin_width)
            self.mp[i].n_bins, self.mp[i].recompute_every = int(s.n_bins), int(s.recompute_every)
            p = list(s.p) + [0.0] * (N_MOVES - len(s.p))
            a = list(s.amax) + [0.0] * (N_MOVES - len(s.amax))
            self.mp[i].p = (C.c_double * N_MOVES)(*[float(x) for x in p])
            self.mp[i].amax = (C.c_double * N_MOVES)(*[float(x) for x in a])
            self.mp[i].pair_precision = int(pair_precision or 64)


def phast_energy(system, xyz: torch.Tensor, pair_precision: int = 64, stream=None) -> torch.Tensor:
    """Energies (FP64, device) of xyz [B, N, 3] FP64 on the device."""
    st = _Structs([system])
    xyz = xyz.contiguous()
    B = xyz.shape[0] if xyz.numel() else 0
    E = torch.empty(B, dtype=torch.float64, device=xyz.device)
    _check(lib().phast_energy(st.sys, st.ff, B, _ptr(xyz), pair_precision, _ptr(E), _stream(stream)))
    return E


FF_PARAMS = ("C_AA", "C_BB", "C_AB", "kappa", "kappa_C")


def ff_params(system) -> list:
    """(C_AA, C_BB, C_AB, kappa, kappa_C) of a system: the Lennard-Jones coefficients of
    Eq. 1, the torsion weight (E_tors = -kappa sum cos tau) and the bending weight."""
    return [float(system.C[0]), float(system.C[3]), float(system.C[1]), float(system.k_tors), float(system.k_bend)]


def with_ff_params(system, params):
    """Copy of system with the five force-field parameters set."""
    import dataclasses
    caa, cbb, cab, kappa, kappa_c = [float(x) for x in params]
    return dataclasses.replace(system, C=(caa, cab, cab, cbb), k_tors=kappa, k_bend=kappa_c)


def phast_energy_grad(system, xyz: torch.Tensor, pair_precision: int = 32, want_xyz: bool = True,
                      want_ff: bool = True, stream=None, params: torch.Tensor | None = None):
    """(E [B], dE/dxyz [B, N, 3] or None, dE/d(C_AA, C_BB, C_AB, kappa, kappa_C) [B, 5] or None),
    FP64 on the device, of xyz [B, N, 3] FP64 on the device.  params: FP64 [5] on the device
    (ff_params order) in place of the system's values (phast_energy_grad_params)."""
    st = _Structs([system])
    xyz = xyz.contiguous()
    B = xyz.shape[0] if xyz.numel() else 0
    E = torch.empty(B, dtype=torch.float64, device=xyz.device)
    gx = torch.empty_like(xyz) if want_xyz else None
    gf = torch.empty(B, 5, dtype=torch.float64, device=xyz.device) if want_ff else None
    if params is None:
        _check(lib().phast_energy_grad(st.sys, st.ff, B, _ptr(xyz), pair_precision, _ptr(E), _ptr(gx), _ptr(gf),
                                       _stream(stream)))
    else:
        assert params.dtype == torch.float64 and params.numel() == 5 and params.device == xyz.device
        _check(lib().phast_energy_grad_params(st.sys, st.ff, B, _ptr(xyz), pair_precision, _ptr(params.contiguous()),
                                              _ptr(E), _ptr(gx), _ptr(gf), _stream(stream)))
    return E, gx, gf


class EnergyFunction(torch.autograd.Function):
    """E(xyz, params) for a batch of conformations of one system; params are the five
    force-field parameters (ff_params order).  The backward pass recomputes the forward
    one in the same kernel (nothing is kept but the inputs)."""

    @staticmethod
    def forward(ctx, xyz, params, system, pair_precision):
        # the parameters stay where they are (no copy to the host, no synchronisation)
        p = params.detach().to(device=xyz.device, dtype=torch.float64).contiguous()
        E, _, _ = phast_energy_grad(system, xyz.detach().to(torch.float64), pair_precision, want_xyz=False,
                                    want_ff=False, params=p)
        ctx.save_for_backward(xyz, params)
        ctx.system, ctx.pair_precision = system, pair_precision
        return E

    @staticmethod
    def backward(ctx, gE):
        xyz, params = ctx.saved_tensors
        p = params.detach().to(device=xyz.device, dtype=torch.float64).contiguous()
        _, gx, gf = phast_energy_grad(ctx.system, xyz.detach().to(torch.float64), ctx.pair_precision, params=p)
        gE = gE.to(torch.float64)
        g_xyz = (gE.view(-1, 1, 1) * gx).to(xyz.dtype) if ctx.needs_input_grad[0] else None
        g_par = (gE.view(-1, 1) * gf).sum(0).to(params.device, params.dtype) if ctx.needs_input_grad[1] else None
        return g_xyz, g_par, None, None


def energy(xyz: torch.Tensor, params: torch.Tensor, system, pair_precision: int = 32) -> torch.Tensor:
    """Differentiable energies [B] of xyz [B, N, 3] (device) under params [5] (ff_params order)."""
    return EnergyFunction.apply(xyz, params, system, pair_precision)


def reweight_sensitivity(E: torch.Tensor, D: torch.Tensor, lnW: torch.Tensor, n_monomers: int,
                         T: torch.Tensor, stream=None) -> dict:
    """<E>_T, c_V(T) and their derivatives in a parameter from multicanonical samples
    (energies E, derivatives D = dE/dlambda, sampling log-weights lnW), device FP64."""
    E, D, lnW, T = (x.to(torch.float64).contiguous() for x in (E, D, lnW, T))
    out = {k: torch.empty(T.numel(), dtype=torch.float64, device=E.device) for k in ("E_T", "cV_T", "dE_T", "dcV_T")}
    _check(lib().phast_reweight_sensitivity(E.numel(), _ptr(E), _ptr(D), _ptr(lnW), n_monomers, T.numel(), _ptr(T),
                                            _ptr(out["E_T"]), _ptr(out["cV_T"]), _ptr(out["dE_T"]),
                                            _ptr(out["dcV_T"]), _stream(stream)))
    return out


def moves_tensor(moves, device) -> torch.Tensor:
    """Pack moves (a MOVE_DTYPE array or a list of dicts) into device bytes."""
    if not isinstance(moves, np.ndarray):
        arr = np.zeros(len(moves), MOVE_DTYPE)
        for i, m in enumerate(moves):
            for k, v in m.items():
                arr[i][k] = v
        moves = arr
    raw = np.ascontiguousarray(moves.astype(MOVE_DTYPE)).view(np.uint8)
    return torch.from_numpy(raw.copy()).to(device)


def phast_delta_energy(system, xyz: torch.Tensor, moves, pair_precision: int = 64, want_xyz: bool = False,
                       stream=None):
    st = _Structs([system])
    xyz = xyz.contiguous()
    B = xyz.shape[0]
    mv = moves if isinstance(moves, torch.Tensor) else moves_tensor(moves, xyz.device)
    dE = torch.empty(B, dtype=torch.float64, device=xyz.device)
    xn = torch.empty_like(xyz) if want_xyz else None
    _check(lib().phast_delta_energy(st.sys, st.ff, B, _ptr(xyz), _ptr(mv), pair_precision, _ptr(dE), _ptr(xn),
                                    _stream(stream)))
    return (dE, xn) if want_xyz else dE


class Context:
    """Walker state of one or more system types on the current device (phast_ctx)."""

    def __init__(self, systems, pair_precision: int = 32, xyz0=None, seeds=None, stream=None):
        if isinstance(systems, inputs.System):
            systems = [systems]
        self.systems = list(systems)
        self._st = _Structs(self.systems, pair_precision)
        walkers = np.array([s.walkers for s in self.systems], dtype=np.int32)
        if seeds is None:
            seeds = np.concatenate([s.seeds() for s in self.systems]).astype(np.uint64)
        if xyz0 is None:
            xyz0 = np.concatenate([s.walker_xyz().reshape(-1) for s in self.systems])
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        xyz0 = np.ascontiguousarray(xyz0, dtype=np.float64).reshape(-1)
        self._keep = [walkers, seeds, xyz0]
        h = C.c_void_p()
        _check(lib().phast_ctx_create(C.byref(h), len(self.systems), self._st.sys, self._st.ff, self._st.mp,
                                      walkers.ctypes.data, seeds.ctypes.data, xyz0.ctypes.data, _stream(stream)))
        self.h = h
        self.W = int(walkers.sum())
        self.pair_precision = pair_precision
        info = [self.info(s) for s in range(len(self.systems))]
        self.N = [i[1] for i in info]
        self.n_bins = [i[2] for i in info]
        self.walker_off = [i[3] for i in info]
        self.xyz_off = [i[4] for i in info]
        self.lnw_off = [i[5] for i in info]
        self.xyz_total = sum(s.walkers * n * 3 for s, n in zip(self.systems, self.N))

    def info(self, s: int):
        out = np.zeros(8, np.int64)
        _check(lib().phast_ctx_info(self.h, s, out.ctypes.data))
        return [int(x) for x in out]

    def close(self):
        if getattr(self, "h", None):
            lib().phast_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state ------------------------------------------------------------------
    def get_state(self, device="cuda", stream=None) -> dict:
        dev = torch.device(device)
        xyz = torch.empty(self.xyz_total, dtype=torch.float64, device=dev)
        E = torch.empty(self.W, dtype=torch.float64, device=dev)
        b = torch.empty(self.W, dtype=torch.int32, device=dev)
        t = torch.empty(self.W, dtype=torch.int64, device=dev)
        stats = torch.empty(self.W * STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        _check(lib().phast_ctx_get_state(self.h, _ptr(xyz), _ptr(E), _ptr(b), _ptr(t), _ptr(stats),
                                         _stream(stream)))
        return dict(xyz=xyz, E=E, bin=b, t=t, stats=stats)

    def set_state(self, xyz=None, E=None, bin=None, t=None, stats=None, stream=None):
        _check(lib().phast_ctx_set_state(self.h, _ptr(xyz), _ptr(E), _ptr(bin), _ptr(t), _ptr(stats),
                                         _stream(stream)))

    def stats(self) -> np.ndarray:
        st = self.get_state()
        torch.cuda.synchronize()
        return st["stats"].cpu().numpy().view(STATS_DTYPE)

    def xyz_of(self, state: dict, s: int) -> torch.Tensor:
        """Coordinates of system type s as [walkers, N, 3]."""
        n = self.systems[s].walkers * self.N[s] * 3
        return state["xyz"][self.xyz_off[s]: self.xyz_off[s] + n].view(self.systems[s].walkers, self.N[s], 3)

    # tiles ------------------------------------------------------------------
    def set_tile(self, threads_per_walker: int = 0, walkers_per_cta: int = 0):
        _check(lib().phast_ctx_set_tile(self.h, threads_per_walker, walkers_per_cta))

    def get_tile(self):
        a, b = C.c_int32(), C.c_int32()
        _check(lib().phast_ctx_get_tile(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_hist_flush(self, count: int = 0):
        """Count at which a tile's shared histogram bin moves into hist_sum (0: default 2^31)."""
        _check(lib().phast_ctx_set_hist_flush(self.h, int(count)))

    def autotune(self, lnW: torch.Tensor, sweeps: int = 1, stream=None):
        _check(lib().phast_ctx_autotune(self.h, _ptr(lnW), sweeps, _stream(stream)))
        return self.get_tile()

    # the sweep --------------------------------------------------------------
    def lnW_zeros(self, device="cuda") -> torch.Tensor:
        return torch.zeros(sum(self.n_bins), dtype=torch.float64, device=device)

    def hist_sum_zeros(self, n_jk: int = 1, device="cuda") -> torch.Tensor:
        return torch.zeros(n_jk * sum(self.n_bins), dtype=torch.int64, device=device)

    def hist_walker_zeros(self, device="cuda") -> torch.Tensor:
        return torch.zeros(sum(s.walkers * k for s, k in zip(self.systems, self.n_bins)), dtype=torch.int32,
                           device=device)

    def sweep(self, n_sweeps: int, lnW: torch.Tensor, form: int = FORM_BATCHED, n_jk: int = 1,
              hist_sum: torch.Tensor | None = None, hist_walker: torch.Tensor | None = None,
              trace: torch.Tensor | None = None, trace_walkers: int = 0, stream=None):
        _check(lib().phast_muca_sweep(self.h, int(n_sweeps), _ptr(lnW), form, n_jk, _ptr(hist_sum),
                                      _ptr(hist_walker), _ptr(trace), trace_walkers, _stream(stream)))

    def capture_iteration(self, n_sweeps: int, lnW: torch.Tensor, hist_sum: torch.Tensor, g_acc: torch.Tensor,
                          n_jk: int = 1, flat_out: torch.Tensor | None = None, stream=None) -> "IterationGraph":
        """One multicanonical iteration (clear hist_sum, n_sweeps batched sweeps, Berg's step per
        system type) captured as a CUDA graph; g_acc is laid out like lnW.  Captured on `stream`
        (a side stream by default), replayed by IterationGraph.launch."""
        cap = stream if stream is not None else torch.cuda.Stream()
        cap.wait_stream(torch.cuda.current_stream())
        h = C.c_void_p()
        _check(lib().phast_ctx_capture_iteration(self.h, int(n_sweeps), _ptr(lnW), n_jk, _ptr(hist_sum), _ptr(g_acc),
                                                 _ptr(flat_out), C.byref(h), _stream(cap)))
        return IterationGraph(h, keep=(self, lnW, hist_sum, g_acc, flat_out))

    def trace_buffer(self, n_sweeps: int, walkers: int, device="cuda") -> torch.Tensor:
        n = walkers * n_sweeps * self.N[0]
        return torch.zeros(n * TRACE_DTYPE.itemsize, dtype=torch.uint8, device=device)

    # checkpoint -------------------------------------------------------------
    def checkpoint(self, stream=None) -> bytes:
        n = C.c_size_t()
        _check(lib().phast_ctx_checkpoint(self.h, None, C.byref(n), _stream(stream)))
        buf = C.create_string_buffer(n.value)
        _check(lib().phast_ctx_checkpoint(self.h, buf, C.byref(n), _stream(stream)))
        return buf.raw

    def restore(self, blob: bytes, stream=None):
        buf = C.create_string_buffer(blob, len(blob))
        _check(lib().phast_ctx_restore(self.h, buf, len(blob), _stream(stream)))


MAXWELL_FIELDS = ("beta_c", "eps_1", "eps_2", "latent", "barrier", "found")


def phast_maxwell(lnW: torch.Tensor, hist: torch.Tensor | None, e_min: float, bin_width: float, n_monomers: int,
                  fd_half_width: int = 1, beta_c: float = 0.0, tol_beta: float = 0.0, tol_L: float = 0.0,
                  stream=None):
    """Free energy per monomer f [K] and the Maxwell construction: rows [(1 + R), 6] of
    (MAXWELL_FIELDS) for all blocks and each leave-one-block-out replicate, and their
    jackknife errors [6]; hist int64 [n_blocks, K] (or [K], or None for S = -lnW)."""
    K = lnW.numel()
    n_blocks = 0 if hist is None else hist.numel() // K
    R = n_blocks if n_blocks >= 2 else 0
    f = torch.empty(K, dtype=torch.float64, device=lnW.device)
    rep = torch.empty(1 + R, 6, dtype=torch.float64, device=lnW.device)
    err = torch.empty(6, dtype=torch.float64, device=lnW.device)
    _check(lib().phast_maxwell(K, float(e_min), float(bin_width), _ptr(lnW), _ptr(hist), n_blocks, fd_half_width,
                               n_monomers, float(beta_c), float(tol_beta), float(tol_L), _ptr(f), _ptr(rep),
                               _ptr(err), _stream(stream)))
    return f, rep, err


class IterationGraph:
    """A captured multicanonical iteration (phast_ctx_capture_iteration); holds the
    context and buffers it was captured with."""

    def __init__(self, handle, keep):
        self.h = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(lib().phast_graph_launch(self.h, _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().phast_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def phast_weight_update(hist: torch.Tensor, lnW: torch.Tensor, g_acc: torch.Tensor, bin_width: float,
                        beta_out: torch.Tensor | None = None, flat_out: torch.Tensor | None = None, stream=None):
    """One Berg step in place on lnW [K] and g_acc [K-1]; hist int64 [n_blocks, K] (or [K])."""
    K = lnW.numel()
    n_blocks = hist.numel() // K
    _check(lib().phast_weight_update(K, float(bin_width), _ptr(hist), n_blocks, _ptr(lnW), _ptr(g_acc),
                                     _ptr(beta_out), _ptr(flat_out), _stream(stream)))


@dataclass
class MicroResult:
    S: torch.Tensor
    beta: torch.Tensor
    CV: torch.Tensor
    E_T: torch.Tensor
    cV_T: torch.Tensor
    peak: torch.Tensor
    S_err: torch.Tensor | None = None
    beta_err: torch.Tensor | None = None
    CV_err: torch.Tensor | None = None
    E_T_err: torch.Tensor | None = None
    cV_T_err: torch.Tensor | None = None
    peak_err: torch.Tensor | None = None


def phast_micro_analysis(lnW: torch.Tensor, e_min: float, bin_width: float, hist: torch.Tensor | None = None,
                         fd_half_width: int = 1, n_monomers: int = 1, T: torch.Tensor | None = None,
                         workspace: torch.Tensor | None = None, stream=None, noalloc: bool = False) -> MicroResult:
    """Eq. 4-6 plus canonical reweighting; hist int64 [n_blocks, K]; errors when n_blocks >= 2.

    noalloc=True calls phast_micro_analysis_noalloc, which takes no workspace
    (it uses the library's static device scratch); the result tensors are still
    allocated here by torch."""
    dev = lnW.device
    K = lnW.numel()
    n_blocks = 0 if hist is None else hist.numel() // K
    if T is None:
        T = torch.empty(0, dtype=torch.float64, device=dev)
    n_T = T.numel()
    f = lambda n: torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    errs = n_blocks >= 2
    r = MicroResult(f(K), f(K), f(K), f(n_T), f(n_T), f(2))
    if errs:
        r.S_err, r.beta_err, r.CV_err, r.E_T_err, r.cV_T_err, r.peak_err = f(K), f(K), f(K), f(n_T), f(n_T), f(2)
    if noalloc:
        return fill_micro_analysis_noalloc(r, lnW, e_min, bin_width, hist, fd_half_width, n_monomers, T, stream)
    o = _micro_out(r)
    need = lib().phast_micro_workspace_size(K, n_T, n_blocks)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    _check(lib().phast_micro_analysis(K, float(e_min), float(bin_width), _ptr(lnW), _ptr(hist), n_blocks,
                                      fd_half_width, n_monomers, n_T, _ptr(T), C.byref(o), _ptr(workspace),
                                      workspace.numel(), _stream(stream)))
    return r


def _micro_out(r: MicroResult) -> _MicroOut:
    o = _MicroOut()
    for name in _MicroOut._fields_:
        v = getattr(r, name[0])
        setattr(o, name[0], None if v is None else v.data_ptr())
    return o


def fill_micro_analysis_noalloc(r: MicroResult, lnW: torch.Tensor, e_min: float, bin_width: float,
                                hist: torch.Tensor | None = None, fd_half_width: int = 1, n_monomers: int = 1,
                                T: torch.Tensor | None = None, stream=None) -> MicroResult:
    """phast_micro_analysis_noalloc into the caller's result tensors r (no device allocation
    on this path; T may be None only when r's E_T and cV_T are empty)."""
    K = lnW.numel()
    n_blocks = 0 if hist is None else hist.numel() // K
    n_T = 0 if T is None else T.numel()
    _check(lib().phast_micro_analysis_noalloc(K, float(e_min), float(bin_width), _ptr(lnW), _ptr(hist), n_blocks,
                                              fd_half_width, n_monomers, n_T, _ptr(T), C.byref(_micro_out(r)),
                                              _stream(stream)))
    return r


def phast_micro_analysis_binned(lnW: torch.Tensor, e_min: float, bin_width: float, hist: torch.Tensor | None = None,
                                block: int = 1, fd_half_width: int = 1, n_monomers: int = 1,
                                T: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                                stream=None) -> MicroResult:
    """Binning over iterations: lnW [n_it, K] and hist int64 [n_it, K] (or None), one
    row per iteration; values and errors over n_it // block blocks of iterations."""
    dev = lnW.device
    lnW = lnW.contiguous()
    n_it, K = lnW.shape
    if T is None:
        T = torch.empty(0, dtype=torch.float64, device=dev)
    n_T = T.numel()
    f = lambda n: torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    r = MicroResult(f(K), f(K), f(K), f(n_T), f(n_T), f(2))
    r.S_err, r.beta_err, r.CV_err, r.E_T_err, r.cV_T_err, r.peak_err = f(K), f(K), f(K), f(n_T), f(n_T), f(2)
    o = _MicroOut()
    for name in _MicroOut._fields_:
        v = getattr(r, name[0])
        setattr(o, name[0], None if v is None else v.data_ptr())
    need = lib().phast_micro_binned_workspace_size(K, n_T, n_it)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    _check(lib().phast_micro_analysis_binned(K, float(e_min), float(bin_width), _ptr(lnW), _ptr(hist),
                                             n_it, int(block), fd_half_width, n_monomers, n_T, _ptr(T), C.byref(o),
                                             _ptr(workspace), workspace.numel(), _stream(stream)))
    return r


def phast_version() -> int:
    return lib().phast_version()
