"""The AB2 momentum predictor (pc_momentum, Eq. 3) against the oracle, alone and chained with the
pressure correction into full time steps."""
import math

import numpy as np
import pytest

from oracle import grid as G
from oracle import momentum as M
from oracle import projection as PR
from paper_2304_14690_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CASES = [
    dict(dim=2, n=(32, 24), bc_lo=("I", "W"), bc_hi=("D", "W"), obstacles=[("circle", (1.0, 0.75), 0.25)]),
    dict(dim=3, n=(12, 10, 8), bc_lo=("W", "D", "P"), bc_hi=("W", "W", "P"), obstacles=[("sphere", (0.4, 0.3, 0.25), 0.12)]),
]


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
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


def _grid(p):
    return G.Grid(p.dim, p.n, p.lo, p.h, p.bc_lo, p.bc_hi)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_predictor_matches_oracle(env, case, precision, tol):
    """Each step's u* from the same u^n (the oracle's chain) against the oracle's predictor, with
    prescribed boundary velocities and a body force; the first step is Euler."""
    pc, torch, dev = env
    prob = wl.generic(seed=700 + case, **CASES[case])
    g = _grid(prob)
    oplan = PR.build_plan(g, prob.nodes, prob.node_type, K=prob.knn)
    force = np.arange(1.0, prob.dim + 1) * 0.1
    m_ref = M.build(g, prob.nodes, prob.node_type, K=prob.knn, nu=0.05, force=force)
    plan = pc.Plan(prob, precision=precision)
    mom = pc.Momentum(plan, nu=0.05, force=force)
    rng = np.random.default_rng(case)
    ub = rng.normal(size=prob.u_star.shape)
    ub_d = torch.as_tensor(ub, device=dev)
    dt = 0.01
    u = prob.u_star.copy()
    for step in range(4):
        us_ref = M.predict(m_ref, dt, u, ub)
        us = mom.predict(torch.as_tensor(u, device=dev), dt, u_boundary=ub_d)
        e = rel(us.cpu().numpy(), us_ref)
        assert e <= tol, (case, precision, step, e)
        u = PR.project(oplan, dt, us_ref)["u"]
    mom.close()
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_time_steps_match_oracle(env, precision, tol):
    """Five full time steps (predictor, then the IB-force iteration of the correction) run on the
    device alone, against the same chain in the oracle."""
    pc, torch, dev = env
    prob = wl.generic(seed=710, **CASES[0])
    g = _grid(prob)
    oplan = PR.build_plan(g, prob.nodes, prob.node_type, K=prob.knn)
    m_ref = M.build(g, prob.nodes, prob.node_type, K=prob.knn, nu=0.02)
    plan = pc.Plan(prob, precision=precision)
    mom = pc.Momentum(plan, nu=0.02)
    dt = 0.005
    u_ref = prob.u_star.copy()
    u = torch.as_tensor(prob.u_star, device=dev)
    for step in range(5):
        r = PR.project_ib(oplan, dt, M.predict(m_ref, dt, u_ref), tol=0.0, max_iters=3)
        u_ref = r["u"]
        us = mom.predict(u, dt)
        p, u, f, info = plan.project_ib(us, dt=dt, tol=0.0, max_iters=3)
        assert info["iterations"] == 3
        assert rel(u.cpu().numpy(), u_ref) <= tol, (step, rel(u.cpu().numpy(), u_ref))
        assert rel(p.cpu().numpy(), r["p"]) <= tol, step
    mom.close()
    plan.close()


def test_taylor_green_decay(env):
    """The periodic Taylor-Green vortex stepped on the device decays at exp(-2 nu t)."""
    pc, torch, dev = env
    nu, dt, steps = 0.1, 0.02, 15
    prob = wl.periodic_taylor_green(n=64, seed=9)
    x, y = prob.nodes
    tg = np.stack([np.sin(x) * np.cos(y), -np.cos(x) * np.sin(y)])
    plan = pc.Plan(prob, precision="mixed")
    mom = pc.Momentum(plan, nu=nu)
    u = torch.as_tensor(tg, device=dev)
    for _ in range(steps):
        _, u, _, _ = plan.project(mom.predict(u, dt), dt=dt)
    exact = tg * math.exp(-2 * nu * dt * steps)
    err = np.abs(u.cpu().numpy() - exact).max() / np.abs(exact).max()
    assert err < 2e-3, err
    mom.close()
    plan.close()


def test_dt_change_and_reset(env):
    pc, torch, dev = env
    prob = wl.generic(seed=720, **CASES[0])
    plan = pc.Plan(prob, precision="fp64")
    mom = pc.Momentum(plan, nu=0.01)
    u = torch.as_tensor(prob.u_star, device=dev)
    first = mom.predict(u, 0.01).clone()
    mom.predict(u, 0.01)
    with pytest.raises(pc.PcError):
        mom.predict(u, 0.02)
    mom.reset()
    assert torch.equal(mom.predict(u, 0.01), first)
    mom.close()
    plan.close()
