"""Pins of the AB2 momentum predictor of the oracle (oracle/momentum.py), no GPU."""
import math

import numpy as np
import pytest

from oracle import grid as G
from oracle import momentum as M
from oracle import projection as PR
from paper_2304_14690_gb300 import workloads as wl


def _grid(p):
    return G.Grid(p.dim, p.n, p.lo, p.h, p.bc_lo, p.bc_hi)


@pytest.mark.parametrize("case", [
    dict(dim=2, n=(20, 16), bc_lo=("W", "D"), bc_hi=("I", "W"), obstacles=[("circle", (0.6, 0.5), 0.15)]),
    dict(dim=3, n=(8, 8, 6), bc_lo=("W", "W", "D"), bc_hi=("W", "W", "D")),
])
def test_node_rows_reproduce_quadratics(case):
    """Gradient and Laplacian rows at every node reproduce a quadratic velocity exactly, so R of
    a quadratic field is exact: -u.grad u + nu lap u + F."""
    prob = wl.generic(seed=31, **case)
    g = _grid(prob)
    d = prob.dim
    rng = np.random.default_rng(2)
    c0, A, B = rng.normal(size=d), rng.normal(size=(d, d)), rng.normal(size=(d, d, d))
    B = 0.5 * (B + np.transpose(B, (0, 2, 1)))
    x = prob.nodes
    u = c0[:, None] + A @ x + np.einsum("aij,im,jm->am", B, x, x)
    grad = A[:, :, None] + 2.0 * np.einsum("abj,jm->abm", B, x)           # d u_a / d x_b
    lap = 2.0 * np.trace(B, axis1=1, axis2=2)                               # (d,)
    m = M.build(g, prob.nodes, prob.node_type, K=prob.knn, nu=0.3, force=np.arange(1.0, d + 1))
    R = M.rhs(m, u)
    want = -np.einsum("bm,abm->am", u, grad) + 0.3 * lap[:, None] + np.arange(1.0, d + 1)[:, None]
    assert np.abs(R - want).max() < 1e-7 * (1 + np.abs(want).max())


def test_taylor_green_rhs_converges():
    """R of the Taylor-Green field: -(sin 2x, sin 2y)/2 - 2 nu u; the meshless error falls with h."""
    errs = []
    for n in (16, 32, 64):
        prob = wl.periodic_taylor_green(n=n, seed=3)
        x, y = prob.nodes
        u = np.stack([np.sin(x) * np.cos(y), -np.cos(x) * np.sin(y)])
        m = M.build(_grid(prob), prob.nodes, prob.node_type, K=12, nu=0.05)
        want = -0.5 * np.stack([np.sin(2 * x), np.sin(2 * y)]) - 2 * 0.05 * u
        errs.append(np.abs(M.rhs(m, u) - want).max())
    assert errs[-1] < 2e-2, errs
    assert all(errs[i] / errs[i + 1] > 1.6 for i in range(2)), errs


def test_ab2_step_by_hand():
    """The first step is forward Euler; the second combines R^n, R^{n-1} and the pressure
    gradient recovered from u*^{n-1} and u^n; boundary and virtual nodes are overwritten."""
    prob = wl.generic(dim=2, n=(12, 10), bc_lo=("W", "W"), bc_hi=("W", "W"),
                      obstacles=[("circle", (0.4, 0.3), 0.12)], seed=4)
    g = _grid(prob)
    m = M.build(g, prob.nodes, prob.node_type, K=12, nu=0.1, force=(0.2, -0.1))
    rng = np.random.default_rng(5)
    dt = 0.01
    u0 = rng.normal(size=prob.u_star.shape)
    ub = rng.normal(size=u0.shape)
    s1 = M.predict(m, dt, u0, ub)
    fl = prob.node_type == 0
    assert np.allclose(s1[:, fl], (u0 + dt * M.rhs(m, u0))[:, fl], rtol=0, atol=1e-14)
    assert np.array_equal(s1[:, prob.node_type == 1], ub[:, prob.node_type == 1])
    assert np.all(s1[:, prob.node_type == 2] == 0.0)
    gp = rng.normal(size=u0.shape)
    u1 = s1 - 1.5 * dt * gp
    s2 = M.predict(m, dt, u1, ub)
    want = u1 + dt * (1.5 * M.rhs(m, u1) - 0.5 * (M.rhs(m, u0) - gp))
    assert np.abs(s2[:, fl] - want[:, fl]).max() < 1e-12


def test_taylor_green_decay_with_projection():
    """AB2 predictor + pressure correction on the periodic Taylor-Green vortex: the velocity
    follows the viscous decay exp(-2 nu t), with the error falling as the nodes refine."""
    nu, dt, steps = 0.1, 0.02, 15
    errs = []
    for n in (16, 32):
        prob = wl.periodic_taylor_green(n=n, seed=9)
        g = _grid(prob)
        plan = PR.build_plan(g, prob.nodes, prob.node_type, K=12)
        m = M.build(g, prob.nodes, prob.node_type, K=12, nu=nu)
        x, y = prob.nodes
        tg = np.stack([np.sin(x) * np.cos(y), -np.cos(x) * np.sin(y)])
        u = tg.copy()
        for _ in range(steps):
            us = M.predict(m, dt, u)
            u = PR.project(plan, dt, us)["u"]
        exact = tg * math.exp(-2 * nu * dt * steps)
        errs.append(np.abs(u - exact).max() / np.abs(exact).max())
    assert errs[-1] < 5e-3, errs
    assert errs[0] / errs[1] > 2.0, errs
