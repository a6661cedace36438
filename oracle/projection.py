"""The pressure-correction sub-step of the hybrid method, end to end (test infrastructure).

Steps, in the paper's order (§2.3, one pass of the IB-force iteration with a given force):

1. Plan (§2.2 last paragraph: coefficients depend only on positions and are computed once):
   - transfer rows: for every face centre of the staggered grid that carries a flux, the
     value row (row 0 of C^-1 A, Eq. 13 with the f-unknown basis of Eq. 16) over its K
     nearest nodes (velocity, boundary and virtual points alike, §2.3 Fig. 1);
   - gradient rows: for every node, the first-derivative rows of C^-1 A over the 3^d block of
     pressure points (cell centres) around it: along each axis the cell holding the node and
     its two neighbours, the block shifted inward at a non-periodic wall and wrapped on a
     periodic axis. §2.3 takes this gradient "from the pressure points" by WLS without fixing
     the stencil; a K-nearest choice can put every point into two layers next to a 3D wall,
     where the quadratic basis is rank deficient, while a 3-per-axis block always determines
     a quadratic exactly.
2. Transfer of u~ = u* + dt f~ to the faces. The modified PPE (Eq. 20) has the right-hand side
   (2/(3 dt)) div u* + (2/3) div f~ = (1/(beta dt)) div(u* + dt f~) with beta = 3/2.
   Wall faces carry no flux (§3.3 workaround); inflow and Dirichlet faces keep the
   transferred flux (Eq. 7: u^{n+1}.n = u*.n at an inflow).
3. Source s = D_h U / (beta dt), set to zero outside an optional RHS mask (§3.5); discrete
   solve L_h p = s (oracle.poisson; or the pseudo-spectral solve of the same source). The
   paper's own variant takes s from WLS derivative rows at the cell centres over the K nearest
   nodes (div_mode "wls_direct"), without face fluxes.
4. Gradient of p at the nodes with the gradient rows, then (Eqs. 18-19)
     fluid node:             u^{n+1} = u* - beta dt grad p,          f~ = 0
     boundary/virtual node:  f~ = -u*/dt + beta grad p,              u^{n+1} = 0
   (Eq. 18 with Eq. 19 substituted gives exactly 0 at those nodes.)
5. Check quantity: corrected face flux U - beta dt G_h p and its divergence D_h, which is
   round-off (or the removed mean of s, when the compatibility projection acted).

Node types: 0 fluid (velocity point), 1 boundary point, 2 virtual point (§2.3).

6. The IB-force iteration (§2.3, project_ib): passes 2-4 repeated with the force of the
   previous pass until its mean squared change is below a tolerance times its mean square.

Parity: the grid-level invariants (round-off divergence, idempotence), linearity, Taylor-Green
recovery and the IB relations are pinned in tests/test_oracle_projection.py; the IB iteration
against the fixed point of its affine map found by a direct dense solve on a small problem.
"""
from dataclasses import dataclass
import numpy as np

from . import grid as G
from . import knn as KNN
from . import wls as W
from . import poisson as P

FLUID, BOUNDARY, VIRTUAL = 0, 1, 2


@dataclass
class Plan:
    grid: G.Grid
    nodes: np.ndarray           # (d, N)
    node_type: np.ndarray       # (N,)
    K: int
    eps: float
    support_factor: float
    face_col: list              # per axis: (num_faces, K) int64 node indices
    face_w: list                # per axis: (num_faces, K) value-row weights (0 on wall faces)
    node_col: np.ndarray        # (N, 3^d) cell linear indices of the gradient block
    node_D: np.ndarray          # (d, N, 3^d) derivative-row weights
    cell_col: np.ndarray = None  # (cells, K) node indices of the direct-divergence rows
    cell_D: np.ndarray = None    # (d, cells, K) derivative-row weights at the cell centres


def _box(g):
    lengths = [g.length(a) for a in range(g.dim)]
    periodic = [g.periodic(a) for a in range(g.dim)]
    return list(g.lo[: g.dim]), lengths, periodic


def _wls_block(points, queries, idx, g, eps, support_factor):
    _, lengths, periodic = _box(g)
    nb = points[idx]                                              # (Q, K, d)
    delta = nb - queries[:, None, :]
    for a in range(g.dim):
        if periodic[a]:
            L = lengths[a]
            da = delta[..., a]
            delta[..., a] = np.where(da > 0.5 * L, da - L, np.where(da < -0.5 * L, da + L, da))
    d2 = KNN.squared_distance(delta)
    return W.rows(delta, d2, eps, support_factor)


def build_plan(g, nodes, node_type, K=12, eps=6.3, support_factor=3.0, chunk=200000):
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = nodes.T.copy()                                          # (N, d)
    lo, lengths, periodic = _box(g)
    face_col, face_w = [], []
    for a in range(g.dim):
        fp = g.face_points(a)
        idx, _ = KNN.knn(pts, fp, K, lo, lengths, periodic)
        w = np.empty(idx.shape)
        for s0 in range(0, fp.shape[0], chunk):
            s1 = min(s0 + chunk, fp.shape[0])
            val, _ = _wls_block(pts, fp[s0:s1], idx[s0:s1], g, eps, support_factor)
            w[s0:s1] = val
        wall = g.face_is_wall(a).ravel()
        w[wall] = 0.0
        face_col.append(idx)
        face_w.append(w)
    cp = g.cell_points()
    idx = gradient_block(g, pts)
    D = np.empty((g.dim,) + idx.shape)
    for s0 in range(0, pts.shape[0], chunk):
        s1 = min(s0 + chunk, pts.shape[0])
        _, grad = _wls_block(cp, pts[s0:s1], idx[s0:s1], g, eps, support_factor)
        D[:, s0:s1, :] = np.transpose(grad, (1, 0, 2))
    return Plan(g, nodes, np.asarray(node_type, dtype=np.uint8), K, eps, support_factor,
                face_col, face_w, idx, D)


def gradient_block(g, pts):
    """Cell linear indices (N, 3^d) of the block of 3 cells per axis around each node, listed in
    C order of the block offsets."""
    N = pts.shape[0]
    per_axis = []
    for a in range(g.dim):
        c = np.floor((pts[:, a] - g.lo[a]) / g.h[a]).astype(np.int64)
        c = np.clip(c, 0, g.n[a] - 1)
        start = c - 1
        if g.periodic(a):
            cells = np.mod(start[:, None] + np.arange(3)[None, :], g.n[a])
        else:
            start = np.clip(start, 0, g.n[a] - 3)
            cells = start[:, None] + np.arange(3)[None, :]
        per_axis.append(cells)                                     # (N, 3)
    idx = np.zeros((N, 1), dtype=np.int64)
    for a in range(g.dim):
        idx = (idx[:, :, None] * g.n[a] + per_axis[a][:, None, :]).reshape(N, -1)
    return idx


def cell_rows(plan, chunk=200000):
    """Derivative rows at every cell centre over its K nearest nodes (§2.2 rows at the pressure
    points, for the paper's own divergence of u~ at the pressure points, §2.3). Built on first
    use and kept on the plan."""
    if plan.cell_col is None:
        g = plan.grid
        pts = plan.nodes.T.copy()
        lo, lengths, periodic = _box(g)
        cp = g.cell_points()
        idx, _ = KNN.knn(pts, cp, plan.K, lo, lengths, periodic)
        D = np.empty((g.dim,) + idx.shape)
        for s0 in range(0, cp.shape[0], chunk):
            s1 = min(s0 + chunk, cp.shape[0])
            _, grad = _wls_block(pts, cp[s0:s1], idx[s0:s1], g, plan.eps, plan.support_factor)
            D[:, s0:s1, :] = np.transpose(grad, (1, 0, 2))
        plan.cell_col, plan.cell_D = idx, D
    return plan.cell_col, plan.cell_D


def direct_divergence(plan, u_tilde):
    """div u~ at the cell centres from the WLS derivative rows: sum_a sum_k D_a,k u~_a,k."""
    col, D = cell_rows(plan)
    g = plan.grid
    div = np.zeros(col.shape[0])
    for a in range(g.dim):
        div += np.sum(D[a] * u_tilde[a][col], axis=1)
    return div.reshape(g.shape)


def transfer(plan, u_tilde):
    """Face fluxes U_a = sum_k w_k u~_{a,k} (value rows), wall faces 0."""
    g = plan.grid
    out = []
    for a in range(g.dim):
        U = np.sum(plan.face_w[a] * u_tilde[a][plan.face_col[a]], axis=1)
        out.append(U.reshape(g.face_shape(a)))
    return out


def node_gradient(plan, p):
    pf = np.asarray(p, dtype=np.float64).ravel()
    vals = pf[plan.node_col]                                       # (N, K)
    return np.sum(plan.node_D * vals[None, :, :], axis=2)          # (d, N)


def project(plan, dt, u_star, f_ib=None, beta=1.5, gauge="mean", eigenvalues="fd", rhs_mask=None,
            div_mode="faces"):
    """One pressure-correction pass. Returns a dict with p, u, f, U (faces), s, div_after, removed.
    rhs_mask (cells, nonzero = flow domain): the source is set to zero outside it before the
    solve (§3.5, the polar cavity's source/sink term outside the flow domain).
    div_mode "faces": s from the compact divergence of the WLS face fluxes; "wls_direct": s
    from WLS derivative rows at the cell centres (§2.3 as printed), with U and div_after None."""
    g = plan.grid
    u_star = np.asarray(u_star, dtype=np.float64).reshape(g.dim, -1)
    if f_ib is None:
        u_tilde = u_star
    else:
        u_tilde = u_star + dt * np.asarray(f_ib, dtype=np.float64).reshape(g.dim, -1)
    if div_mode == "faces":
        U = transfer(plan, u_tilde)
        s = G.divergence(U, g) / (beta * dt)
    elif div_mode == "wls_direct":
        U = None
        s = direct_divergence(plan, u_tilde) / (beta * dt)
    else:
        raise ValueError(div_mode)
    if rhs_mask is not None:
        s = np.where(np.asarray(rhs_mask).reshape(g.shape) != 0, s, 0.0)
    p, removed = P.solve(s, g, gauge=gauge, eigenvalues=eigenvalues)
    grad = node_gradient(plan, p)
    ib = plan.node_type != FLUID
    u_new = u_star - beta * dt * grad
    u_new[:, ib] = 0.0
    f_new = np.zeros_like(u_star)
    f_new[:, ib] = -u_star[:, ib] / dt + beta * grad[:, ib]
    U_new, div_after = None, None
    if U is not None:
        U_new = [U[a] - beta * dt * G.face_gradient(p, g, a) for a in range(g.dim)]
        for a in range(g.dim):
            U_new[a][g.face_is_wall(a)] = 0.0
        div_after = G.divergence(U_new, g)
    return dict(p=p, u=u_new, f=f_new, U=U, s=s, grad=grad, U_new=U_new,
                div_after=div_after, removed=removed)


def ib_change(f_new, f_old, node_type):
    """(mean over boundary/virtual nodes of |f_new - f_old|^2, mean of |f_old|^2)."""
    ib = np.asarray(node_type) != FLUID
    if not ib.any():
        return 0.0, 0.0
    d = np.asarray(f_new, dtype=np.float64)[:, ib] - np.asarray(f_old, dtype=np.float64)[:, ib]
    o = np.asarray(f_old, dtype=np.float64)[:, ib]
    n = int(ib.sum())
    return float(np.sum(d * d)) / n, float(np.sum(o * o)) / n


def ib_converged(diff, prev, tol):
    """§2.3 stopping rule: the mean squared change of the IB force below tol times the mean squared
    force of the previous iterate (a zero previous force converges only with zero change)."""
    return diff == 0.0 if prev == 0.0 else diff <= tol * prev


def project_ib(plan, dt, u_star, f_init=None, tol=1e-3, max_iters=50, beta=1.5, gauge="mean",
               eigenvalues="fd", rhs_mask=None, div_mode="faces"):
    """The IB-force iteration of §2.3 around the pressure correction: solve the modified PPE
    (Eq. 20) with the current force, update the force at the boundary and virtual points by
    Eq. 19 from the new pressure gradient, and repeat until ib_converged (or max_iters). The
    force starts from f_init (zero when None: the first iteration of a time step). Returns the
    last pass (p, u, f with the force consistent with that pressure) plus the iteration count
    and the sequence of (diff, prev) pairs."""
    u_star = np.asarray(u_star, dtype=np.float64)
    f = np.zeros_like(u_star) if f_init is None else np.asarray(f_init, dtype=np.float64)
    hist = []
    out = None
    for it in range(1, max_iters + 1):
        out = project(plan, dt, u_star, f, beta=beta, gauge=gauge, eigenvalues=eigenvalues, rhs_mask=rhs_mask,
                      div_mode=div_mode)
        diff, prev = ib_change(out["f"], f, plan.node_type)
        hist.append((diff, prev))
        f = out["f"]
        if ib_converged(diff, prev, tol):
            break
    out["iterations"] = it
    out["history"] = hist
    return out
