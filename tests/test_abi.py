"""The C-ABI library builds, loads and exports every entry point include/phast.h declares.

CPU-only: no compute calls (there may be no GPU); host-side argument checks
that fail before any device work are exercised.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libphast():
    from paper_1702_01770_gb300 import build
    build.build()
    from paper_1702_01770_gb300 import phast
    return phast


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "phast.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(phast_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("phast_energy", "phast_delta_energy", "phast_muca_sweep", "phast_weight_update",
                     "phast_micro_analysis", "phast_ctx_create", "phast_ctx_checkpoint", "phast_ctx_restore"):
        assert required in names


def test_library_exports_every_declared_symbol(libphast):
    L = C.CDLL(libphast.LIB_PATH)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(libphast.SYMBOLS) == sorted(n for n in declared_symbols())


def test_version_and_error_string(libphast):
    L = libphast.lib()
    assert L.phast_version() == 2
    assert isinstance(L.phast_last_error(), bytes)


def test_host_side_validation(libphast):
    """Invalid arguments are rejected before any device work."""
    from paper_1702_01770_gb300 import inputs
    L = libphast.lib()
    s = inputs.config0()
    st = libphast._Structs([s])
    # bad pair precision
    assert L.phast_energy(st.sys, st.ff, 1, None, 16, None, None) == -1
    assert b"pair_precision" in L.phast_last_error()
    # B = 0 is a no-op that touches nothing
    assert L.phast_energy(st.sys, st.ff, 0, None, 64, None, None) == 0
    assert L.phast_delta_energy(st.sys, st.ff, 0, None, None, 32, None, None, None) == 0
    # chain shorter than 3
    bad = inputs.System("bad", np.array([2], np.int32), np.zeros(2, np.uint8), 0.0)
    sb = libphast._Structs([bad])
    assert L.phast_energy(sb.sys, sb.ff, 1, None, 64, None, None) == -1
    # too many chains
    many = inputs.System("many", np.full(17, 3, np.int32), np.zeros(51, np.uint8), 10.0)
    sm = libphast._Structs([many])
    assert L.phast_energy(sm.sys, sm.ff, 1, None, 64, None, None) == -1
    # sequence letters other than 0/1
    seq = np.zeros(13, np.uint8)
    seq[3] = 2
    s2 = inputs.System("x", np.array([13], np.int32), seq, 0.0)
    assert L.phast_energy(libphast._Structs([s2]).sys, libphast._Structs([s2]).ff, 1, None, 64, None, None) == -1
    # weight update / analysis argument checks
    assert L.phast_weight_update(0, 0.1, None, 1, None, None, None, None, None) == -1
    assert L.phast_weight_update(10, -1.0, None, 1, None, None, None, None, None) == -1
    assert L.phast_micro_workspace_size(100, 8, 4) == 8 * 5 * (3 * 100 + 2 * 8 + 2)
    out = libphast._MicroOut()
    assert L.phast_micro_analysis(100, 0.0, 0.1, None, None, 0, 60, 1, 0, None, C.byref(out), None, 0, None) == -1
    # context creation rejects bad move mixes before touching the device
    s3 = inputs.config0(walkers=1)
    st3 = libphast._Structs([s3])
    st3.mp[0].p = (C.c_double * libphast.N_MOVES)(0.5, 0.2, 0.2, 0.2, 0.0, 0.0)
    h = C.c_void_p()
    w = np.array([1], np.int32)
    seeds = np.zeros(1, np.uint64)
    xyz = s3.walker_xyz().reshape(-1)
    assert L.phast_ctx_create(C.byref(h), 1, st3.sys, st3.ff, st3.mp, w.ctypes.data, seeds.ctypes.data,
                              xyz.ctypes.data, None) == -1
    assert b"probabilities" in L.phast_last_error()
    st4 = libphast._Structs([s3])
    st4.mp[0].amax = (C.c_double * libphast.N_MOVES)(1.5, 0.5, 0.3, 0.5, 0.0, 0.0)
    assert L.phast_ctx_create(C.byref(h), 1, st4.sys, st4.ff, st4.mp, w.ctypes.data, seeds.ctypes.data,
                              xyz.ctypes.data, None) == -1
    # bond-length / cap moves need the FENE term; a container excludes a periodic box
    st6 = libphast._Structs([s3])
    st6.mp[0].p = (C.c_double * libphast.N_MOVES)(0.8, 0.0, 0.0, 0.0, 0.2, 0.0)
    assert L.phast_ctx_create(C.byref(h), 1, st6.sys, st6.ff, st6.mp, w.ctypes.data, seeds.ctypes.data,
                              xyz.ctypes.data, None) == -1
    assert b"k_fene" in L.phast_last_error()
    st7 = libphast._Structs([s3])
    st7.sys[0].sphere_R, st7.sys[0].box_L = 10.0, 20.0
    assert L.phast_energy(st7.sys, st7.ff, 1, None, 64, None, None) == -1
    assert b"container" in L.phast_last_error()
    xyz_nan = xyz.copy()
    xyz_nan[4] = np.nan
    st5 = libphast._Structs([s3])
    assert L.phast_ctx_create(C.byref(h), 1, st5.sys, st5.ff, st5.mp, w.ctypes.data, seeds.ctypes.data,
                              xyz_nan.ctypes.data, None) == -7


def test_product_path_does_not_touch_the_oracle():
    """The CUDA package never imports or includes the test oracle, and the oracle never uses the package."""
    pkg = os.path.join(ROOT, "paper_1702_01770_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), fn
            assert "liboracle" not in src, fn
    for fn in os.listdir(os.path.join(pkg, "csrc")):
        src = open(os.path.join(pkg, "csrc", fn)).read()
        assert not re.search(r"#include\s*[<\"].*oracle", src), fn
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read() + open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_1702_01770_gb300" not in src and "phast.h" not in src
