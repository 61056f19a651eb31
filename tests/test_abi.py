"""The C-ABI library builds, loads and exports every symbol include/tnmc.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tnmc(?:3d)?_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2104_13264_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.LIB_PATH


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("tnmc_build_env", "tnmc_sample", "tnmc_logq", "tnmc_mh_step", "tnmc_init_chains",
                     "tnmc_env_free", "tnmc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header():
    from paper_2104_13264_gb300 import binding
    assert set(declared_symbols()) <= set(binding.SIGNATURES)


def test_argument_errors_reported_without_gpu(libpath):
    """Argument checks run before any CUDA call, so they work on a machine without a GPU."""
    from paper_2104_13264_gb300 import binding
    L = binding.lib()
    out = ctypes.c_void_p()
    st = L.tnmc_build_env(None, 1.0, 4, 0, None, ctypes.byref(out))
    assert st == 1
    assert b"non-null" in L.tnmc_last_error()
    import numpy as np
    h = np.zeros((2, 2))
    J = np.ones((2, 1))
    lat = binding._Lattice(2, 2, J.ctypes.data, J.ctypes.data, h.ctypes.data)
    assert L.tnmc_build_env(ctypes.byref(lat), 1.0, 0, 0, None, ctypes.byref(out)) == 1
    assert L.tnmc_build_env(ctypes.byref(lat), 1.0, 65, 0, None, ctypes.byref(out)) == 1
    assert L.tnmc_build_env(ctypes.byref(lat), float("nan"), 4, 0, None, ctypes.byref(out)) == 1
    hb = np.array([[0.0, float("inf")], [0.0, 0.0]])
    lat2 = binding._Lattice(2, 2, J.ctypes.data, J.ctypes.data, hb.ctypes.data)
    assert L.tnmc_build_env(ctypes.byref(lat2), 1.0, 4, 0, None, ctypes.byref(out)) == 1
    assert b"not finite" in L.tnmc_last_error()


def test_allocator_and_batch_argument_errors_without_gpu(libpath):
    """tnmc_set_allocator wants both functions or neither; the batch calls check their
    arguments before touching the device."""
    from paper_2104_13264_gb300 import binding
    L = binding.lib()

    @binding.ALLOC_FN
    def _alloc(n, s, ctx):
        return None

    assert L.tnmc_set_allocator(ctypes.cast(_alloc, ctypes.c_void_p), None, None) == 1
    assert b"both" in L.tnmc_last_error()
    assert L.tnmc_set_allocator(None, None, None) == 0
    out = ctypes.c_void_p()
    assert L.tnmc_batch_create(0, None, None, 1, 1, 128, 1, None, ctypes.byref(out)) == 1
    assert L.tnmc_build_env_batched(-1, None, None, None, 0, None, None) == 1
    assert L.tnmc_sample_batched(None, None, None, None, None, None) == 1
    assert L.tnmc_mh_batched(None, None, None, None, None, None, None, None, None, None) == 1


def test_newer_entry_points_check_arguments_without_gpu(libpath):
    """The bond-basis, variational, site-order and 3D calls reject bad arguments with
    TNMC_E_INVALID_ARG and a message before touching the device."""
    import numpy as np

    from paper_2104_13264_gb300 import binding
    L = binding.lib()
    out = ctypes.c_void_p()
    h = np.zeros((2, 2))
    J = np.ones((2, 1))
    lat = binding._Lattice(2, 2, J.ctypes.data, J.ctypes.data, h.ctypes.data)
    # bond basis: the sampling bond 2 chi must fit
    assert L.tnmc_build_env_bond(ctypes.byref(lat), 1.0, 1 << 20, 0, None, ctypes.byref(out)) == 1
    assert b"chi" in L.tnmc_last_error()
    # variational rounds out of range
    assert L.tnmc_build_env_variational(ctypes.byref(lat), 1.0, 4, -1, 0, None, ctypes.byref(out)) == 1
    assert L.tnmc_build_env_variational(ctypes.byref(lat), 1.0, 4, 65, 0, None, ctypes.byref(out)) == 1
    assert b"sweeps" in L.tnmc_last_error()
    # site order on a null env
    assert L.tnmc_env_set_order(None, 0) == 1
    # MH step on a null env
    assert L.tnmc_mh_step(None, 1, 1, None, None, None, None, None, None, 0, 0, None, None, None) == 1
    # 3D: D, chi, beta and non-finite couplings
    h3 = np.zeros((2, 2, 2))
    J3 = np.ones(8)
    lat3 = binding._Lattice3D(2, 2, 2, J3.ctypes.data, J3.ctypes.data, J3.ctypes.data, h3.ctypes.data)
    for fn in (L.tnmc3d_build_env, L.tnmc3d_build_env_bond):
        assert fn(None, 1.0, 2, 2, None, ctypes.byref(out)) == 1
        assert fn(ctypes.byref(lat3), 1.0, 0, 2, None, ctypes.byref(out)) == 1
        assert b"D = 0" in L.tnmc_last_error()
        assert fn(ctypes.byref(lat3), 1.0, 2, 0, None, ctypes.byref(out)) == 1
        assert fn(ctypes.byref(lat3), -1.0, 2, 2, None, ctypes.byref(out)) == 1
    h3b = h3.copy()
    h3b[1, 1, 1] = float("nan")
    lat3b = binding._Lattice3D(2, 2, 2, J3.ctypes.data, J3.ctypes.data, J3.ctypes.data, h3b.ctypes.data)
    assert L.tnmc3d_build_env(ctypes.byref(lat3b), 1.0, 2, 2, None, ctypes.byref(out)) == 1
    assert b"not finite" in L.tnmc_last_error()
    assert L.tnmc3d_sample(None, 0, 1, 0, 0, None, None, None, None, None) == 1
    assert L.tnmc3d_mh_step(None, 1, 1, None, None, None, None, None, None, 0, 0, None, None, None) == 1
