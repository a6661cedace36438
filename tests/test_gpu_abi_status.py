"""Status codes of pc_plan_create that need the real library on a device (host-safe inputs).

- A degenerate node cloud (every node on one line) leaves the WLS normal matrices of Eq. 14
  rank deficient: the quadratic basis of Eq. 16 has six unknowns in 2D, points on a line
  determine three. The plan is refused with PC_ERR_WLS_SINGULAR.
- A device-memory budget far below what the plan holds is refused with PC_ERR_BUDGET before
  the rows are built.
Both return cleanly: no plan handle, a message, and the device stays usable (a valid plan is
built afterwards).
"""
import ctypes

import numpy as np
import pytest

from paper_2304_14690_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc as mod
    return mod


def _create(pc, prob, xyz, typ, budget=0, precision="fp64"):
    lib = pc.load()
    d = pc.make_desc(prob, precision=precision, node_xyz=xyz, node_type=typ)
    d.num_nodes = xyz.shape[1]
    h = ctypes.c_void_p()
    s = lib.pc_plan_create(ctypes.byref(d), 0, budget, None, ctypes.byref(h))
    return s, h, lib.pc_last_error_message()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_collinear_cloud_is_wls_singular(pc, precision):
    prob = wl.generic(dim=2, n=(16, 16), bc_lo=("W", "W"), bc_hi=("W", "W"), seed=3)
    N = 400
    rng = np.random.default_rng(4)
    L = prob.n[0] * prob.h[0]
    x = np.sort(rng.uniform(0.0, L, N))
    xyz = np.ascontiguousarray(np.stack([x, np.full(N, 0.5 * prob.n[1] * prob.h[1])]))
    typ = np.zeros(N, dtype=np.uint8)
    s, h, msg = _create(pc, prob, xyz, typ, precision=precision)
    assert s == 3, msg
    assert not h.value and b"WLS" in msg


def test_tiny_budget_is_refused(pc):
    prob = wl.generic(dim=2, n=(32, 32), bc_lo=("P", "W"), bc_hi=("P", "W"), seed=5)
    xyz = np.ascontiguousarray(prob.nodes)
    typ = np.ascontiguousarray(prob.node_type)
    s, h, msg = _create(pc, prob, xyz, typ, budget=1024)
    assert s == 5, msg
    assert not h.value and b"budget" in msg
    # the device is still usable: the same problem without a budget builds
    s, h, msg = _create(pc, prob, xyz, typ)
    assert s == 0, msg
    assert pc.load().pc_destroy(h) == 0
