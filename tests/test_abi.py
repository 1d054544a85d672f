"""CPU checks of the C ABI: the library builds, loads, exports every declared symbol, and rejects
invalid configurations before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as G

    G.build()
    from paper_1202_6074_gb300 import cmlbm

    return cmlbm


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "cmlbm.h")).read()
    return sorted(set(re.findall(r"CMLBM_API\s+[\w\s\*]+?\b(cmlbm_\w+)\s*\(", text)))


def test_header_declarations_match_binding(lib):
    assert declared_symbols() == sorted(lib.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(so, name), name


def test_config_struct_size_matches(lib):
    # the ctypes mirror of cmlbm_config must have the C layout: 4+12+4+12 ints, 18+8 doubles, ...
    c = lib.Config()
    assert ctypes.sizeof(c) == 8 * ((ctypes.sizeof(c) + 7) // 8)
    assert lib.Config.tau.offset % 8 == 0 and lib.Config.stream.offset % 8 == 0


@pytest.mark.parametrize("kw,msg", [
    (dict(lattice="D2Q9", nz=2), "nz == 1"),
    (dict(nx=0), ">= 1"),
    (dict(tau=0.5), "tau"),
    (dict(omega_3=2.0), "omega_3"),
    (dict(omega_bulk=-1.0), "omega_bulk"),
    (dict(storage=7), "storage"),
    (dict(van_driest=(26.0, 1.0), smagorinsky_cs=0.1), "walls in y"),
    (dict(van_driest=(26.0, 1.0), bc=("periodic", "bounceback", "periodic")), "smagorinsky_cs"),
    (dict(nx=2048, ny=1024, nz=1024), "2^31"),
    (dict(lattice="D2Q9", nx=65536, ny=8192, nz=1), "9*nx*ny < 2^32"),
    (dict(attractor=3), "attractor"),
    (dict(reduced_compressibility=True, rho0=0.0), "rho0"),
    (dict(bc=("halo", "periodic", "periodic")), "CMLBM_HALO on z"),
    (dict(kernel=9), "unknown kernel"),
    (dict(lattice="D2Q9", nz=1, bc=("periodic", "periodic", "halo")), "CMLBM_HALO needs D3Q27"),
    (dict(nx=1024, ny=1024, nz=151, bc=("periodic", "periodic", "halo")), "(nz+2)"),
])
def test_invalid_configs_are_rejected_without_a_gpu(lib, kw, msg):
    c = lib.make_config(**kw)
    h = ctypes.c_void_p()
    so = lib.load()
    rc = so.cmlbm_create(ctypes.byref(c), ctypes.byref(h))
    assert rc == lib.ERR_INVALID
    assert h.value is None
    assert msg in so.cmlbm_last_error(None).decode()


@pytest.mark.parametrize("kw", [
    # D3Q27 with 27 N >= 2^32 runs 64-bit-offset variants of the pair kernel (FP32 / 16-bit: periodic
    # x, nx a multiple of 64) or of the one-cell kernel (FP64); everything else is refused
    dict(nx=1024, ny=1024, nz=200, bc=("bounceback", "periodic", "periodic")),
    dict(nx=1000, ny=1024, nz=200),
    dict(nx=1024, ny=1024, nz=200, kernel="tma"),
    dict(nx=1024, ny=1024, nz=200, kernel="pair_two_steps"),
    dict(nx=1024, ny=1024, nz=200, kernel="direct"),
])
def test_large_grid_forms_without_64bit_variants_are_unsupported(lib, kw):
    c = lib.make_config(**kw)
    h = ctypes.c_void_p()
    so = lib.load()
    assert so.cmlbm_create(ctypes.byref(c), ctypes.byref(h)) == lib.ERR_UNSUPPORTED
    assert h.value is None
    assert "2^32" in so.cmlbm_last_error(None).decode()


def test_tma_on_a_slab_is_unsupported_without_a_gpu(lib):
    c = lib.make_config(nx=128, ny=4, nz=4, bc=("periodic", "periodic", "halo"), kernel="tma")
    h = ctypes.c_void_p()
    so = lib.load()
    assert so.cmlbm_create(ctypes.byref(c), ctypes.byref(h)) == lib.ERR_UNSUPPORTED
    assert "slab" in so.cmlbm_last_error(None).decode()


def test_null_handle_calls_fail_cleanly(lib):
    so = lib.load()
    assert so.cmlbm_halo_bytes(None) == 0
    assert so.cmlbm_step_kernel(None) == lib.ERR_INVALID
    assert so.cmlbm_halo_pack(None, 0, None, 0) == lib.ERR_INVALID
    assert so.cmlbm_halo_unpack(None, 0, None, 0) == lib.ERR_INVALID
    assert so.cmlbm_step(None, 1) == lib.ERR_INVALID
    assert so.cmlbm_state_bytes(None) == 0
    assert so.cmlbm_launch_count(None) == 0
    so.cmlbm_destroy(None)
