"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every function declared in include/iblbm.h; the binding's signature
table covers the header; argument validation that fails before any device
call."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iblbm.h")


def header_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(iblbm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_boundary_calls():
    names = header_functions()
    for required in ("iblbm_create", "iblbm_add_body", "iblbm_step", "iblbm_body_forces",
                     "iblbm_move_body", "iblbm_destroy", "iblbm_strerror", "iblbm_step_batch"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2609_02298_b300 import build
    path = build.build()
    lib = C.CDLL(path)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_2609_02298_b300 as L
    bound = {s[0] for s in L.SIGNATURES}
    assert set(header_functions()) <= bound


def test_strerror_names_every_code():
    import paper_2609_02298_b300 as L
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10, -11):
        assert L.strerror(code) != "unknown status"
    assert L.strerror(-999) == "unknown status"


def test_struct_layout_matches_header():
    """ctypes mirrors of the descriptors have the C sizes (compiled probe-free:
    sizes follow from the field lists in the header)."""
    import paper_2609_02298_b300 as L
    # nx, ny, storage, bc[4], padding to 8, u_bc, three doubles, force, init_rho, init_u,
    # cuda_stream, wall_closure, tail padding to 8
    assert L.LatticeDesc.wall_closure.offset == 4 * 2 + 4 + 16 + 4 + 64 + 8 * 3 + 16 + 8 + 16 + 8
    assert C.sizeof(L.LatticeDesc) == L.LatticeDesc.wall_closure.offset + 4 + 4
    assert C.sizeof(L.BodyDesc) % 8 == 0


def test_create_rejects_bad_arguments_without_device_work():
    """Validation happens before any CUDA call, so it runs on a CPU-only host."""
    import paper_2609_02298_b300 as L
    lib = L.load_library()
    d = L.LatticeDesc()
    d.nx, d.ny, d.storage, d.init_rho = 2, 10, L.F32, 1.0
    h = C.c_void_p()
    assert lib.iblbm_create(C.byref(d), L.BGK, 0.8, C.byref(h)) == -1      # nx < 3
    d.nx = 10
    d.bc[0], d.bc[1] = L.BC_PERIODIC, L.BC_VELOCITY                        # half-periodic axis
    assert lib.iblbm_create(C.byref(d), L.BGK, 0.8, C.byref(h)) == -1
    d.bc[1] = L.BC_PERIODIC
    assert lib.iblbm_create(C.byref(d), L.BGK, 0.5, C.byref(h)) == -1      # tau <= 1/2
    assert lib.iblbm_create(C.byref(d), 7, 0.8, C.byref(h)) == -1          # unknown collision
    d.wall_closure = 2                                                     # only 0 or 1
    assert lib.iblbm_create(C.byref(d), L.BGK, 0.8, C.byref(h)) == -1
    d.wall_closure = 0
    assert lib.iblbm_create(None, L.BGK, 0.8, C.byref(h)) == -1
    assert lib.iblbm_step(None, 1) == -1
    assert lib.iblbm_step_batch(None, 0, 1) == -1


def test_diagnostics_and_marker_velocity_reject_bad_arguments():
    """The Sec. 2.8 diagnostics and the per-marker velocity call validate their
    arguments before any CUDA call (null context, null output)."""
    import paper_2609_02298_b300 as L
    lib = L.load_library()
    out = (C.c_double * 8)()
    assert lib.iblbm_local_diagnostics(None, 0, 0.1, 2.0, out, None) == -1
    assert lib.iblbm_set_marker_velocity(None, 0, None) == -1
