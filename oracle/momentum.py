"""The first fractional step around the pressure correction (test infrastructure; see package
header): the second-order Adams-Bashforth predictor (Eq. 3, §2.1) on the node cloud.

Eq. 3 advances the momentum equations (Eq. 2) to the intermediate velocity
  u* = u^n + (3/2) dt R^n - (1/2) dt R^{n-1},
  R^n     = -u^n . grad u^n + nu lap u^n + F,                 (no pressure term)
  R^{n-1} = -u^{n-1} . grad u^{n-1} - grad p^{n-1} + nu lap u^{n-1} + F,
and the pressure correction (oracle.projection / oracle.vertex) adds back (3/2) dt grad p^n.
The spatial operators are meshless (§2.2): at every node, the first-derivative rows and the
Laplacian row of the WLS fit over its K nearest nodes (itself included), with the weight,
support radius and basis of the transfer rows.

Readings:
  * grad p^{n-1} at a fluid node is the gradient the previous correction applied there:
    u^n = u*^{n-1} - beta dt grad p^{n-1} (Eq. 18 with beta = 3/2), so it is recovered as
    (u*^{n-1} - u^n) / (beta dt); dt is constant over the run.
  * The first step has no R^{n-1}: it takes R^{-1} = R^0 and no pressure term (forward Euler).
  * Boundary points carry their prescribed velocity in u* (no-slip: zero, or the given
    boundary values); virtual points carry u* = 0 (§2.3).

Parity: pinned by tests/test_oracle_momentum.py - the node rows reproduce gradients and
Laplacians of quadratics exactly; R of the Taylor-Green field converges to its closed form; a
Taylor-Green run with the projection decays at the analytic viscous rate.
"""
from dataclasses import dataclass

import numpy as np

from . import knn as KNN
from . import wls as W
from . import projection as PR


@dataclass
class Momentum:
    col: np.ndarray            # (N, K) node indices
    G: np.ndarray              # (d, N, K) first-derivative rows
    L: np.ndarray              # (N, K) Laplacian rows
    nu: float
    force: np.ndarray          # (d,)
    node_type: np.ndarray
    beta: float = 1.5
    R_prev: np.ndarray = None  # R^{n-1} without its pressure term
    ustar_prev: np.ndarray = None
    steps: int = 0


def build(g, nodes, node_type, K=12, eps=6.3, support_factor=3.0, nu=0.0, force=None, beta=1.5):
    """Rows of the meshless momentum operators at every node (§2.2)."""
    pts = np.asarray(nodes, dtype=np.float64).T.copy()
    lo, lengths, periodic = PR._box(g)
    idx, _ = KNN.knn(pts, pts, K, lo, lengths, periodic)
    delta = pts[idx] - pts[:, None, :]
    for a in range(g.dim):
        if periodic[a]:
            L = lengths[a]
            da = delta[..., a]
            delta[..., a] = np.where(da > 0.5 * L, da - L, np.where(da < -0.5 * L, da + L, da))
    d2 = KNN.squared_distance(delta)
    _, grad, lap = W.rows(delta, d2, eps, support_factor, laplacian=True)
    f = np.zeros(g.dim) if force is None else np.asarray(force, dtype=np.float64)
    return Momentum(idx, np.transpose(grad, (1, 0, 2)), lap, float(nu), f,
                    np.asarray(node_type, dtype=np.uint8), beta)


def rhs(m, u):
    """R = -u . grad u + nu lap u + F at every node (d, N)."""
    u = np.asarray(u, dtype=np.float64)
    d = u.shape[0]
    vals = u[:, m.col]                                   # (d, N, K): u_a at the neighbours
    grad = np.einsum("bnk,ank->abn", m.G, vals)          # grad[a, b] = d u_a / d x_b
    lap = np.einsum("nk,ank->an", m.L, vals)
    adv = np.einsum("bn,abn->an", u, grad)
    return -adv + m.nu * lap + m.force[:, None]


def predict(m, dt, u_n, u_boundary=None):
    """u* of the AB2 step from u^n (d, N); updates the stored R^{n-1} and u*^{n-1}."""
    u_n = np.asarray(u_n, dtype=np.float64)
    R = rhs(m, u_n)
    if m.steps == 0:
        R_old, gp = R, np.zeros_like(R)
    else:
        R_old = m.R_prev
        gp = (m.ustar_prev - u_n) / (m.beta * dt)
    ustar = u_n + dt * (1.5 * R - 0.5 * (R_old - gp))
    bnd = m.node_type == PR.BOUNDARY
    ustar[:, bnd] = 0.0 if u_boundary is None else np.asarray(u_boundary, dtype=np.float64)[:, bnd]
    ustar[:, m.node_type == PR.VIRTUAL] = 0.0
    m.R_prev, m.ustar_prev, m.steps = R, ustar.copy(), m.steps + 1
    return ustar


def reset(m):
    m.R_prev, m.ustar_prev, m.steps = None, None, 0
