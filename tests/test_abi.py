"""The C ABI library loads without a GPU, exports every function include/pc.h declares, and
rejects malformed descriptors with the documented status before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc
    return pc.load()


def declared_functions():
    names = set()
    for fname in os.listdir(os.path.join(ROOT, "include")):
        if fname.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fname)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(pc_\w+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "pc_project" in names and "pc_plan_create" in names and len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2304_14690_gb300 import pc
    assert set(declared_functions()) <= set(pc.FUNCTIONS)


def test_status_strings(lib):
    assert lib.pc_status_string(0) == b"ok"
    assert lib.pc_status_string(5) == b"device-memory budget exceeded"
    assert lib.pc_status_string(99) == b"unknown status"


def _desc(**over):
    from paper_2304_14690_gb300 import pc, workloads as wl
    prob = wl.generic(dim=2, n=(8, 8), seed=0)
    xyz = np.ascontiguousarray(prob.nodes)
    typ = np.ascontiguousarray(prob.node_type)
    d = pc.make_desc(prob, node_xyz=xyz, node_type=typ)
    for k, v in over.items():
        if k in ("n", "bc_lo", "bc_hi"):
            for i, x in enumerate(v):
                getattr(d, k)[i] = x
        else:
            setattr(d, k, v)
    return d, (xyz, typ)


@pytest.mark.parametrize("over,status", [
    (dict(dim=4), 1),
    (dict(knn=3), 1),
    (dict(knn=64), 1),
    (dict(n=(9, 8, 1)), 2),          # odd cell count: no real-to-real transform of odd length
    (dict(n=(2, 8, 1)), 1),          # fewer than 3 cells per axis: no gradient block
    (dict(n=(14, 8, 1)), 2),         # n/2 = 7 is not 2^a 3^b 5^c
    (dict(bc_lo=(0, 1, 0), bc_hi=(1, 1, 0)), 1),   # periodic paired with a wall
    (dict(precision=7), 1),
    (dict(refine_iters=99), 1),
    (dict(wls_eps=-1.0), 1),
    (dict(node_xyz=None), 1),
    (dict(eigenvalues=2), 1),                        # neither FD nor pseudo-spectral
    (dict(eigenvalues=1, precision=1), 2),           # pseudo-spectral with the mixed refinement
    (dict(divergence=5), 1),                         # neither MAC faces nor direct WLS
    (dict(grid_type=2), 1),                          # neither cells nor vertices
    (dict(grid_type=1), 2),                          # vertices with MAC-face divergence
])
def test_descriptor_validation(lib, over, status):
    d, keep = _desc(**over)
    h = ctypes.c_void_p()
    s = lib.pc_plan_create(ctypes.byref(d), 0, 0, None, ctypes.byref(h))
    assert s == status, lib.pc_last_error_message()
    assert lib.pc_last_error_message() != b""


@pytest.mark.parametrize("over", [
    dict(dim=3, n=(4096, 4096, 128)),   # 2^31 cells: beyond the kernels' 32-bit row numbers
    dict(num_nodes=1 << 31),            # 2^31 nodes
    dict(num_nodes=(1 << 31) - (1 << 16) + 1),
])
def test_plan_beyond_row_limits_is_refused_before_the_device(lib, over):
    """Row arrays are indexed with 64-bit offsets and 32-bit row numbers, so a plan whose cells,
    faces or nodes exceed 2^31 - 2^16 is refused (PC_ERR_UNSUPPORTED) by validation, before any
    device call; the node arrays are never read."""
    d, keep = _desc(**over)
    h = ctypes.c_void_p()
    s = lib.pc_plan_create(ctypes.byref(d), 0, 0, None, ctypes.byref(h))
    assert s == 2, lib.pc_last_error_message()
    assert b"at most" in lib.pc_last_error_message()
    assert not h.value


def _grid_desc(**over):
    from paper_2304_14690_gb300 import pc
    d = pc.GridDesc()
    d.dim = 2
    for a in range(3):
        d.n[a] = 16 if a < 2 else 1
        d.h[a] = 0.1
        d.bc_lo[a] = d.bc_hi[a] = pc.BC["W"]
    d.grid_type = 1
    for k, v in over.items():
        if k in ("n", "bc_lo", "bc_hi", "h"):
            for i, x in enumerate(v):
                getattr(d, k)[i] = x
        else:
            setattr(d, k, v)
    return d


@pytest.mark.parametrize("over,status", [
    (dict(dim=1), 1),
    (dict(grid_type=2), 1),
    (dict(precision=7), 1),
    (dict(gauge=3), 1),
    (dict(eigenvalues=4), 1),
    (dict(eigenvalues=1, precision=1), 2),           # pseudo-spectral with the mixed refinement
    (dict(n=(3, 16)), 1),
    (dict(h=(0.1, -1.0)), 1),
    (dict(bc_lo=(0, 1)), 1),                          # periodic paired with a wall
    (dict(bc_lo=(3, 1), n=(15, 16)), 2),              # a D-N vertex axis: quarter-wave pair of odd length
    (dict(n=(4096, 16)), 2),                          # an N-N vertex axis of 4096 cells: DCT-I FFT of 4096
    (dict(n=(14, 16)), 2),                            # a cell axis of 14 (half 7): no transform
])
def test_grid_descriptor_validation(lib, over, status):
    d = _grid_desc(**over)
    if "n" in over and over["n"] == (14, 16):
        d.grid_type = 0
    h = ctypes.c_void_p()
    s = lib.pc_grid_plan_create(ctypes.byref(d), 0, None, ctypes.byref(h))
    assert s == status, lib.pc_last_error_message()
    assert lib.pc_last_error_message() != b""


def test_momentum_entry_points_reject_null(lib):
    """The predictor's entry points check their arguments before touching a device."""
    h = ctypes.c_void_p()
    assert lib.pc_momentum_create(None, None, 12, 0.0, None, None, ctypes.byref(h)) == 1
    assert lib.pc_last_error_message() != b""
    assert lib.pc_momentum_predict(None, 0.1, None, None, None, None) == 1
    assert lib.pc_momentum_reset(None) == 1
    assert lib.pc_momentum_destroy(None) == 0
