"""The mixed-precision refinement and its device-side stopping rule (§8 S6 reading).

A mixed solve runs the FP32 transform solve, then sweeps p += solve32(s - mean - L_h p) with
the residual in double-float arithmetic. The rule, decided on the device after each residual:
stop at ||r|| <= refine_tol ||s||, or when the residual no longer falls at the rate of the first
sweep (it has reached the rounding floor of its own evaluation), or after refine_iters sweeps,
which is reported as PC_ERR_NOT_CONVERGED with the statistics filled.

Checked here: the largest accepted axis length (4096) and the largest served sizes (1024^2,
192^3) against the oracle's exact solve at 1e-10; the sweep count and the convergence flag in
the statistics; the non-converged status; and that a rule that stops after two sweeps gives the
bits of two fixed sweeps.
"""
import numpy as np
import pytest

from oracle import grid as G
from oracle import poisson as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc
    return pc, torch, torch.device("cuda", 0)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,n,h,lo,hi", [
    (2, (4096, 1024), (1 / 256, 1 / 128), ("I", "W"), ("D", "W")),   # the longest accepted axis
    (2, (1024, 1024), (1 / 128, 1 / 128), ("W", "P"), ("W", "P")),   # largest served 2D size
    (3, (192, 192, 192), (1 / 64,) * 3, ("W", "W", "I"), ("W", "W", "W")),   # largest served 3D size
])
def test_large_grids_match_oracle(env, dim, n, h, lo, hi):
    pc, torch, dev = env
    g = G.Grid(dim, n, (0.0,) * dim, h, lo, hi)
    s = np.random.default_rng(sum(n)).normal(size=n)
    ref, _ = P.solve(s, g)
    sd = torch.as_tensor(s, device=dev)
    plan = pc.GridPlan(dim, n, h, lo, hi, precision="mixed")
    p, st = plan.solve_poisson(sd, stats=True)
    e = rel(p.cpu().numpy(), ref)
    assert e <= 1e-10, e
    assert st["refine_converged"] and 1 <= st["refine_iters_done"] <= 4, st
    r = st["residual_norm"]
    assert r[-1] <= 1e-9 * st["source_norm"], st
    plan.close()
    p64 = pc.GridPlan(dim, n, h, lo, hi, precision="fp64")
    q, _ = p64.solve_poisson(sd)
    assert rel(q.cpu().numpy(), ref) <= 1e-12
    p64.close()


def test_served_1024_projection_mixed_matches_fp64(env):
    """A 1024^2 inflow/outflow channel with a cylinder (the largest 2D served request): the mixed
    projection with the stopping rule against the plain FP64 path, 1e-10 on p and u."""
    pc, torch, dev = env
    from paper_2304_14690_gb300 import workloads as wl
    prob = wl.generic(dim=2, n=(1024, 1024), h=(1 / 64, 1 / 64), bc_lo=("I", "W"), bc_hi=("D", "W"),
                      obstacles=[("circle", (6.0, 8.0), 0.8)], seed=41)
    u = torch.as_tensor(prob.u_star, device=dev)
    mixed = pc.Plan(prob, precision="mixed")
    fp64 = pc.Plan(prob, precision="fp64")
    p, uo, _, st = mixed.project(u, stats=True)
    p64, u64, _, _ = fp64.project(u)
    assert st["refine_converged"], st
    assert rel(p.cpu().numpy(), p64.cpu().numpy()) <= 1e-10
    assert rel(uo.cpu().numpy(), u64.cpu().numpy()) <= 1e-10
    mixed.close()
    fp64.close()


def test_rule_stops_at_the_floor_like_two_fixed_sweeps(env):
    """On a problem whose residual reaches its rounding floor after two sweeps the rule stops
    there, and p is bitwise that of exactly two sweeps; the skipped sweeps change nothing."""
    pc, torch, dev = env
    n, h = (256, 192), (1 / 64, 1 / 64)
    s = torch.as_tensor(np.random.default_rng(3).normal(size=n), device=dev)
    ad = pc.GridPlan(2, n, h, ("I", "W"), ("D", "W"), precision="mixed", refine_iters=4, refine_tol=1e-13)
    fx = pc.GridPlan(2, n, h, ("I", "W"), ("D", "W"), precision="mixed", refine_iters=2, refine_tol=0.0)
    pa, st = ad.solve_poisson(s, stats=True)
    pf, sf = fx.solve_poisson(s, stats=True)
    assert st["refine_iters_done"] == 2 and st["refine_converged"], st
    assert sf["refine_iters_done"] == 2
    assert torch.equal(pa, pf)
    # without statistics (graph replay), the same bits
    pa2, _ = ad.solve_poisson(s)
    torch.cuda.synchronize()
    assert torch.equal(pa2, pf)
    ad.close()
    fx.close()


def test_not_converged_is_reported(env):
    """One sweep allowed and a tolerance below the floor: the call returns
    PC_ERR_NOT_CONVERGED with the statistics filled and p written (one sweep's accuracy)."""
    pc, torch, dev = env
    n, h = (512, 256), (1 / 64, 1 / 64)
    g = G.Grid(2, n, (0.0, 0.0), h, ("W", "W"), ("W", "W"))
    s = np.random.default_rng(5).normal(size=n)
    ref, _ = P.solve(s, g)
    plan = pc.GridPlan(2, n, h, ("W", "W"), ("W", "W"), precision="mixed", refine_iters=1, refine_tol=1e-13)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    with pytest.raises(pc.PcError) as e:
        plan.solve_poisson(torch.as_tensor(s, device=dev), p_out=out, stats=True)
    assert e.value.status == 7
    st = e.value.stats
    assert st is not None and st["refine_iters_done"] == 1 and not st["refine_converged"]
    assert rel(out.cpu().numpy(), ref) <= 1e-6
    plan.close()


def test_batched_rule_matches_single_calls(env):
    """Batched projections apply the rule per problem and give the bits of single calls."""
    pc, torch, dev = env
    from paper_2304_14690_gb300 import workloads as wl
    probs = [wl.generic(dim=2, n=n, bc_lo=bl, bc_hi=bh, seed=60 + i)
             for i, (n, bl, bh) in enumerate([((64, 48), ("P", "W"), ("P", "W")), ((96, 64), ("W", "I"), ("W", "D")),
                                              ((128, 128), ("P", "P"), ("P", "P"))])]
    plans = [pc.Plan(pr, precision="mixed") for pr in probs]
    args, singles = [], []
    for pl, pr in zip(plans, probs):
        u = torch.as_tensor(pr.u_star, device=dev)
        p, uo, fo = pl.alloc_outputs()
        args.append(dict(dt=pr.dt, u_star=u, p=p, u=uo, f=fo))
    pc.project_batch(plans, args)
    torch.cuda.synchronize()
    for pl, a in zip(plans, args):
        p, uo, fo, st = pl.project(a["u_star"], stats=True)
        assert st["refine_converged"]
        assert torch.equal(p, a["p"]) and torch.equal(uo, a["u"])
    for pl in plans:
        pl.close()
