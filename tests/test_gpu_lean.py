"""GPU parity of the compile-time FP32 transform passes (the default FP32 schedule at the line
lengths n = 2M, M in {16, 32, 48, 64, 96, 128, 192, 256, 384, 512}; variant 0, and variant 1
with fewer slots per thread) against the CPU oracle's
Poisson solve (§2.3 three-step solve), through the C ABI.

Every length is taken along the contiguous axis (row tiles: forward-only and inverse-only
passes) and along axis 0 (column tiles: forward, division, inverse), with the other axis short
and not a multiple of the tile's line count (ragged tiles), for every boundary pair (real DFT,
DCT-II, DST-II, DCT-IV, DST-IV), including singular problems (zero mode). 3D cases add column
passes of axis 1. Tolerances as in test_gpu_parity: FP32 unrefined 1e-5, mixed 1e-10 (relative
L2 of p). The general passes (4 slots per thread) must agree with the same oracle, and a batch
call with the compile-time passes must equal its single calls bit for bit.
"""
import numpy as np
import pytest

from oracle import grid as G
from oracle import poisson as P
from paper_2304_14690_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

LEAN_M = [16, 32, 48, 64, 96, 128, 192, 256, 384, 512]
KINDS = {"PP": ("P", "P"), "NN": ("W", "W"), "DD": ("D", "D"), "ND": ("I", "D"), "DN": ("D", "W")}
OTHER = ["NN", "PP", "DD", "ND", "DN"]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc
    assert torch.cuda.is_available()
    return pc, torch, torch.device("cuda", 0)


def _case(kinds, n, seed):
    dim = len(n)
    rng = np.random.default_rng(seed)
    h = tuple(rng.uniform(0.5, 2.0) / n[a] for a in range(dim))
    g = G.Grid(dim, tuple(n), tuple([0.0] * dim), h, tuple(KINDS[k][0] for k in kinds),
               tuple(KINDS[k][1] for k in kinds))
    s = rng.normal(size=n)
    return g, s


def _plan(pc, g, precision):
    prob = wl.generic(dim=g.dim, n=g.n, h=g.h, lo=g.lo, bc_lo=g.bc_lo, bc_hi=g.bc_hi, seed=7)
    return pc.Plan(prob, precision=precision)


def _solve(pc, torch, dev, g, s, precision, slots=None):
    plan = _plan(pc, g, precision)
    if slots is not None:
        for a in range(g.dim):
            plan.set_slots(a, slots, precision="fp32")
    p, _ = plan.solve_poisson(torch.as_tensor(s, device=dev))
    out = p.cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("M", LEAN_M)
@pytest.mark.parametrize("orient", ["col", "row"])
def test_lean_lengths_match_oracle(env, M, orient):
    """Each lean length along axis 0 (column tiles) or axis 1 (row tiles), every boundary pair;
    the other axis has 20 cells (ragged tiles for every tile line count)."""
    pc, torch, dev = env
    for i, kind in enumerate(KINDS):
        other = OTHER[i]
        kinds = (kind, other) if orient == "col" else (other, kind)
        n = (2 * M, 20) if orient == "col" else (20, 2 * M)
        g, s = _case(kinds, n, 4000 + 17 * M + i)
        ref, _ = P.solve(s, g)
        for precision, tol in (("fp32", 1e-5), ("mixed", 1e-10)):
            e = rel(_solve(pc, torch, dev, g, s, precision), ref)
            assert e <= tol, (M, orient, kinds, precision, e)
        # the small-slots variant and the general passes reach the same oracle result
        for slots in (1, 4):
            e = rel(_solve(pc, torch, dev, g, s, "fp32", slots=slots), ref)
            assert e <= 1e-5, (M, orient, kinds, slots, e)


@pytest.mark.parametrize("n", [(20, 64, 10), (12, 96, 36), (10, 12, 128), (6, 256, 18), (192, 10, 12)])
def test_lean_3d_match_oracle(env, n):
    """3D grids with a lean length on one axis: the column passes of axis 1 (forward-only and
    inverse-only) and the rows of the last axis."""
    pc, torch, dev = env
    for i, kinds in enumerate([("NN", "NN", "NN"), ("PP", "DD", "ND"), ("DN", "PP", "NN")]):
        g, s = _case(kinds, n, 5000 + i + sum(n))
        ref, _ = P.solve(s, g)
        for precision, tol in (("fp32", 1e-5), ("mixed", 1e-10)):
            e = rel(_solve(pc, torch, dev, g, s, precision), ref)
            assert e <= tol, (n, kinds, precision, e)


@pytest.mark.parametrize("slots", [0, 1])
def test_lean_batch_equals_single(env, slots):
    """Projections of several problems with lean lengths (either variant): a batch call equals
    the single calls bit for bit (both run the same kernel bodies)."""
    pc, torch, dev = env
    specs = [((64, 96), ("P", "P"), ("P", "P")), ((128, 48), ("W", "W"), ("W", "W")),
             ((96, 192), ("P", "W"), ("P", "W")), ((32, 256), ("W", "P"), ("W", "P")),
             ((384, 64), ("I", "W"), ("D", "W"))]
    plans, args, singles = [], [], []
    for i, (n, lo, hi) in enumerate(specs):
        prob = wl.generic(dim=2, n=n, h=(1.0 / 64, 1.0 / 64), bc_lo=lo, bc_hi=hi, seed=30 + i,
                          obstacles=[("circle", (0.3 * n[0] / 64, 0.5 * n[1] / 64), 0.1)])
        plan = pc.Plan(prob, precision="mixed")
        for a in range(2):
            plan.set_slots(a, slots)
        u = torch.as_tensor(prob.u_star, device=dev)
        singles.append([t.clone() for t in plan.project(u)[:3]])
        outs = plan.alloc_outputs()
        plans.append(plan)
        args.append(dict(dt=prob.dt, u_star=u, f_ib=None, p=outs[0], u=outs[1], f=outs[2]))
    pc.project_batch(plans, args)
    torch.cuda.synchronize()
    for i, a in enumerate(args):
        for name, got, want in zip("puf", (a["p"], a["u"], a["f"]), singles[i]):
            assert torch.equal(got, want), (i, name)
    for plan in plans:
        plan.close()


def test_lean_misaligned_arrays_fall_back(env):
    """Row tiles of the compile-time passes use 16-byte accesses; a source or result array that
    is only 8-byte aligned (a view one element into a buffer) takes the general passes instead,
    and the solve still matches the oracle and the aligned call."""
    pc, torch, dev = env
    for kinds in (("NN", "PP"), ("ND", "DD")):
        g, s = _case(kinds, (64, 128), 6100 + len(kinds[0]))
        ref, _ = P.solve(s, g)
        for precision, tol in (("fp32", 1e-5), ("mixed", 1e-10)):
            plan = _plan(pc, g, precision)
            aligned, _ = plan.solve_poisson(torch.as_tensor(s, device=dev))
            sb = torch.zeros(s.size + 1, dtype=torch.float64, device=dev)
            pb = torch.zeros(s.size + 1, dtype=torch.float64, device=dev)
            s_view = sb[1:].view(g.shape)
            s_view.copy_(torch.as_tensor(s, device=dev))
            p_view = pb[1:].view(g.shape)
            plan.solve_poisson(s_view, p_out=p_view)
            torch.cuda.synchronize()
            assert rel(p_view.cpu().numpy(), ref) <= tol, (kinds, precision)
            assert rel(p_view.cpu().numpy(), aligned.cpu().numpy()) <= tol, (kinds, precision)
            plan.close()
