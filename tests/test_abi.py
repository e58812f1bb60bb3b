"""The C ABI library builds, loads and exports every function include/dg.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    from paper_1806_11456_gb300 import dg
    return dg


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(dg_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    # the calls of the boundary: mesh with an order map, residual, V-cycle,
    # tau estimate, adaptation, steady solve
    for must in ["dg_mesh_create", "dg_mesh_layout", "dg_mesh_destroy", "dg_residual", "dg_pmg_vcycle",
                 "dg_tau_estimate", "dg_adapt", "dg_solve_steady"]:
        assert must in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) == set(built.EXPORTS)


def test_binding_fails_loudly_without_gpu(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1806_11456_gb300 import synthetic as syn
    mesh = syn.periodic_box(1, 1, 1)
    with pytest.raises(built.DGError):
        built.Mesh(mesh, syn.uniform_orders(1, 3, 2), syn.flow_params())


def test_noalloc_transfer_rejects_bad_nvar_before_any_device_call(built):
    """The allocation-free transfer checks its arguments on the host first: a
    variable count outside [1, 64] is DG_EINVAL with a message, and nothing
    touches the (here dummy) device pointers."""
    lib = ctypes.CDLL(built.LIB_PATH)
    lib.dg_last_error.restype = ctypes.c_char_p
    o = (ctypes.c_int32 * 6)(1, 1, 0, 2, 2, 0)
    dummy = ctypes.c_void_p(16)
    for nvar in (0, 65, 1 << 30):
        rc = lib.dg_transfer_noalloc(2, 2, o, o, nvar, dummy, dummy, None)
        assert rc == -1
        assert b"nvar" in lib.dg_last_error()
