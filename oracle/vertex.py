"""Regular (vertex) pressure grid (test infrastructure; see package header).

§2.3 solves the pressure Poisson equation with the same three steps on either grid type: the
transforms and eigenvalues depend on whether the pressure points are the vertices of the
grid ("regular") or the cell centres ("staggered", oracle.poisson), and on the boundary kinds.
§3.2 presents results on a regular grid. This module is the regular-grid solve: the pressure
points of an axis with n cells of spacing h are the vertices x_j = lo + j h, j = 0..n.

Unknowns of an axis and the ghost rules of the 3-point operator (p_{j-1} - 2 p_j + p_{j+1}) / h^2,
per boundary pair lo-hi (Neumann = 'W' or 'I'):
  P-P  j = 0..n-1   periodic wrap (vertex n is vertex 0)
  N-N  j = 0..n     mirror at both ends: p_{-1} = p_1, p_{n+1} = p_{n-1}
  D-D  j = 1..n-1   p_0 = p_n = 0 (boundary values, not unknowns)
  N-D  j = 0..n-1   mirror at 0, p_n = 0
  D-N  j = 1..n     p_0 = 0, mirror at n

Eigenvectors in the unknowns' order, with the angle theta of each (FD eigenvalue
-(2/h)^2 sin^2(theta/2), pseudo-spectral -(theta/h)^2, as for the cell grid):
  P-P  1, cos(2 pi k j/n), sin(2 pi k j/n), (-1)^j    theta = 2 pi k/n
  N-N  cos(pi k j/n), k = 0..n                      theta = pi k/n        (DCT-I)
  D-D  sin(pi k j/n), k = 1..n-1                    theta = pi k/n        (DST-I)
  N-D  cos(pi (k+1/2) j/n), k = 0..n-1              theta = pi (k+1/2)/n
  D-N  sin(pi (k+1/2) j/n), k = 0..n-1              theta = pi (k+1/2)/n

Zero mode (every axis P-P or N-N): the constant vector. Its coefficient in the expansion of s
is dropped (the compatibility projection; on an N-N axis it is the trapezoid-weighted mean of
s) and reported, and the solution has no constant part. An optional corner gauge sets the
first unknown to zero.

The solve expands the source in the eigenvectors with one dense basis per axis (numpy.linalg
.solve finds the coefficients), divides by the summed eigenvalues and sums the expansion back.

The pressure-correction pass on the vertex grid (build_plan, project, project_ib) takes the
divergence of u~ at the pressure points from WLS derivative rows over their K nearest nodes
(§2.3 as printed: there are no faces on this grid), solves on the unknowns, and takes the
gradient at each node from the derivative rows over the 3^d block of lattice vertices around
it (the nearest vertex and its neighbours, shifted inward at a non-periodic end, wrapped on a
periodic axis). A Dirichlet boundary vertex is a point of that block with its known value 0.
The node updates are those of the cell-grid pass (Eqs. 18-19).

Parity: pinned by tests/test_oracle_vertex.py - the eigenvector relations against the operator
applied by its ghost rules, a brute-force dense solve of the assembled operator on small 2D and
3D grids, a manufactured solution converging at second order, continuous modes solved exactly
with the pseudo-spectral eigenvalues, and the identity with the cell-grid periodic solve
(oracle.poisson) of the symmetric extension of the source. The pass: the derivative rows at the
pressure points and at the nodes reproduce quadratics exactly; a gradient field is projected out
with the pressure recovered at second order; the IB relations hold.
"""
from dataclasses import dataclass

import numpy as np

from .grid import NEUMANN
from . import knn as KNN
from . import projection as PR


def axis_kind(lo, hi):
    if lo == "P":
        return "PP"
    return ("N" if lo in NEUMANN else "D") + ("N" if hi in NEUMANN else "D")


def unknowns(kind, n):
    """Number of pressure unknowns on an axis of n cells and their first vertex index."""
    return {"PP": (n, 0), "NN": (n + 1, 0), "DD": (n - 1, 1), "ND": (n, 0), "DN": (n, 1)}[kind]


def _lam(theta, h, eigenvalues):
    if eigenvalues == "fd":
        return -(4.0 / (h * h)) * np.sin(theta / 2.0) ** 2
    if eigenvalues == "spectral":
        return -(theta / h) ** 2
    raise ValueError(eigenvalues)


def eigenbasis(kind, n, h, eigenvalues="fd"):
    """(Phi, lam): Phi[:, k] the k-th eigenvector over the axis's unknowns, lam[k] its eigenvalue."""
    m, j0 = unknowns(kind, n)
    j = (np.arange(m, dtype=np.float64) + j0)[:, None]
    if kind == "PP":
        cols, wav = [np.ones(n)], [0]
        for k in range(1, (n - 1) // 2 + 1):
            cols.append(np.cos(2.0 * np.pi * k * j[:, 0] / n))
            cols.append(np.sin(2.0 * np.pi * k * j[:, 0] / n))
            wav += [k, k]
        if n % 2 == 0:
            cols.append(np.cos(np.pi * j[:, 0]))
            wav.append(n // 2)
        return np.stack(cols, axis=1), _lam(2.0 * np.pi * np.asarray(wav, dtype=np.float64) / n, h, eigenvalues)
    if kind == "NN":
        k = np.arange(n + 1, dtype=np.float64)
        theta = np.pi * k / n
        return np.cos(theta[None, :] * j), _lam(theta, h, eigenvalues)
    if kind == "DD":
        k = np.arange(1, n, dtype=np.float64)
        theta = np.pi * k / n
        return np.sin(theta[None, :] * j), _lam(theta, h, eigenvalues)
    k = np.arange(n, dtype=np.float64)
    theta = np.pi * (k + 0.5) / n
    basis = np.cos(theta[None, :] * j) if kind == "ND" else np.sin(theta[None, :] * j)
    return basis, _lam(theta, h, eigenvalues)


def _pad(p, kind, a):
    """p with one ghost layer on each side of axis a, by the axis's ghost rules."""
    pm = np.moveaxis(p, a, 0)
    if kind == "PP":
        lo, hi = pm[-1:], pm[:1]
    elif kind == "NN":
        lo, hi = pm[1:2], pm[-2:-1]
    elif kind == "DD":
        lo, hi = np.zeros_like(pm[:1]), np.zeros_like(pm[:1])
    elif kind == "ND":
        lo, hi = pm[1:2], np.zeros_like(pm[:1])
    else:   # DN
        lo, hi = np.zeros_like(pm[:1]), pm[-2:-1]
    return np.moveaxis(np.concatenate([lo, pm, hi], axis=0), 0, a)


def laplacian(p, kinds, h):
    """The 2d+1-point operator on the unknowns of a vertex grid (kinds: one per axis)."""
    p = np.asarray(p, dtype=np.float64)
    out = np.zeros_like(p)
    for a, kind in enumerate(kinds):
        q = _pad(p, kind, a)
        sl = lambda i0, i1: tuple(slice(i0, i1) if b == a else slice(None) for b in range(p.ndim))
        m = p.shape[a]
        out += (q[sl(0, m)] - 2.0 * p + q[sl(2, m + 2)]) / (h[a] * h[a])
    return out


def _solve_along(M, x, a):
    xa = np.moveaxis(x, a, 0)
    shp = xa.shape
    y = np.linalg.solve(M, xa.reshape(shp[0], -1)).reshape(shp)
    return np.moveaxis(y, 0, a)


def _apply(M, x, a):
    return np.moveaxis(np.tensordot(M, x, axes=([1], [a])), 0, a)


def solve(s, n, h, bc_lo, bc_hi, gauge="mean", eigenvalues="fd"):
    """Return (p, removed) with the vertex-grid operator applied to p equal to s, less the
    dropped zero-mode coefficient `removed` when every axis is P-P or N-N. s and p have the
    unknowns' shape (unknowns(kind, n[a])[0] per axis)."""
    dim = len(n)
    kinds = [axis_kind(bc_lo[a], bc_hi[a]) for a in range(dim)]
    bases = [eigenbasis(kinds[a], n[a], h[a], eigenvalues) for a in range(dim)]
    s = np.asarray(s, dtype=np.float64)
    shape = tuple(unknowns(kinds[a], n[a])[0] for a in range(dim))
    if s.shape != shape:
        raise ValueError(f"source shape {s.shape}, expected {shape}")
    coef = s
    for a in range(dim):                       # step 1: forward expansion, axis by axis
        coef = _solve_along(bases[a][0], coef, a)
    lam = np.zeros(shape)                      # step 2: divide by the summed eigenvalues
    for a in range(dim):
        sh = [1] * dim
        sh[a] = shape[a]
        lam = lam + bases[a][1].reshape(sh)
    singular = all(k in ("PP", "NN") for k in kinds)
    zero = tuple([0] * dim)
    removed = 0.0
    if singular:
        removed = float(coef[zero])            # the constant mode: the basis vectors at k = 0 are 1
        coef = coef.copy()
        coef[zero] = 0.0
        lam[zero] = 1.0
    p = coef / lam
    for a in range(dim):                       # step 3: backward expansion
        p = _apply(bases[a][0], p, a)
    if singular and gauge == "corner":
        p = p - p[zero]
    return p, removed


# ----------------------------------------------------------------------------- the pass (§2.3)
def lattice_shape(g):
    """Vertices per axis of grid g: n on a periodic axis (vertex n is vertex 0), else n + 1."""
    return tuple(int(g.n[a]) if g.periodic(a) else int(g.n[a]) + 1 for a in range(g.dim))


def kinds_of(g):
    return [axis_kind(g.bc_lo[a], g.bc_hi[a]) for a in range(g.dim)]


def unknown_slices(g):
    """Per axis, the slice of the lattice that holds the unknowns."""
    out = []
    for a, k in enumerate(kinds_of(g)):
        m, j0 = unknowns(k, int(g.n[a]))
        out.append(slice(j0, j0 + m))
    return tuple(out)


def _points(g, index_axes):
    axes = [g.lo[a] + np.asarray(ix, dtype=np.float64) * g.h[a] for a, ix in enumerate(index_axes)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.ravel() for m in mesh], axis=1)


def lattice_points(g):
    return _points(g, [np.arange(m) for m in lattice_shape(g)])


def pressure_points(g):
    """Coordinates (unknowns, d) of the pressure unknowns, C order of the unknowns' shape."""
    return _points(g, [np.arange(sl.start, sl.stop) for sl in unknown_slices(g)])


def vertex_block(g, pts):
    """Lattice linear indices (N, 3^d) of the 3 vertices per axis around each node: the nearest
    vertex and its two neighbours, shifted inward at a non-periodic end, wrapped on a periodic
    axis; C order of the block offsets."""
    shape = lattice_shape(g)
    N = pts.shape[0]
    per_axis = []
    for a in range(g.dim):
        c = np.floor((pts[:, a] - g.lo[a]) / g.h[a] + 0.5).astype(np.int64)
        if g.periodic(a):
            c = np.mod(c, shape[a])
            v = np.mod(c[:, None] - 1 + np.arange(3)[None, :], shape[a])
        else:
            c = np.clip(c, 0, shape[a] - 1)
            start = np.clip(c - 1, 0, shape[a] - 3)
            v = start[:, None] + np.arange(3)[None, :]
        per_axis.append(v)
    idx = np.zeros((N, 1), dtype=np.int64)
    for a in range(g.dim):
        idx = (idx[:, :, None] * shape[a] + per_axis[a][:, None, :]).reshape(N, -1)
    return idx


@dataclass
class VertexPlan:
    grid: object
    nodes: np.ndarray           # (d, N)
    node_type: np.ndarray       # (N,)
    K: int
    eps: float
    support_factor: float
    pt_col: np.ndarray          # (unknowns, K) node indices of the divergence rows
    pt_D: np.ndarray            # (d, unknowns, K) derivative-row weights at the pressure points
    node_col: np.ndarray        # (N, 3^d) lattice indices of the gradient block
    node_D: np.ndarray          # (d, N, 3^d) derivative-row weights at the nodes


def build_plan(g, nodes, node_type, K=12, eps=6.3, support_factor=3.0):
    """Rows of the vertex-grid pass (§2.2: computed once from the positions)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = nodes.T.copy()
    lo, lengths, periodic = PR._box(g)
    qp = pressure_points(g)
    idx, _ = KNN.knn(pts, qp, K, lo, lengths, periodic)
    _, grad = PR._wls_block(pts, qp, idx, g, eps, support_factor)
    pt_D = np.transpose(grad, (1, 0, 2))
    lp = lattice_points(g)
    nidx = vertex_block(g, pts)
    _, ngrad = PR._wls_block(lp, pts, nidx, g, eps, support_factor)
    return VertexPlan(g, nodes, np.asarray(node_type, dtype=np.uint8), K, eps, support_factor,
                      idx, pt_D, nidx, np.transpose(ngrad, (1, 0, 2)))


def direct_divergence(plan, u_tilde):
    """div u~ at the pressure points: sum_a sum_k D_a,k u~_a,k, in the unknowns' shape."""
    g = plan.grid
    div = np.zeros(plan.pt_col.shape[0])
    for a in range(g.dim):
        div += np.sum(plan.pt_D[a] * u_tilde[a][plan.pt_col], axis=1)
    return div.reshape(tuple(sl.stop - sl.start for sl in unknown_slices(g)))


def embed(p, g):
    """The unknowns p placed on the whole lattice, Dirichlet boundary vertices at 0."""
    full = np.zeros(lattice_shape(g))
    full[unknown_slices(g)] = p
    return full


def node_gradient(plan, p_full):
    vals = np.asarray(p_full, dtype=np.float64).ravel()[plan.node_col]
    return np.sum(plan.node_D * vals[None, :, :], axis=2)


def project(plan, dt, u_star, f_ib=None, beta=1.5, gauge="mean", eigenvalues="fd", rhs_mask=None):
    """One pressure-correction pass on the vertex grid: source from the direct divergence,
    the vertex-grid solve, gradient and node updates (Eqs. 18-20). rhs_mask (unknowns' shape,
    nonzero = flow domain) zeroes the source outside it before the solve (§3.5). Returns p
    (unknowns), p_full (lattice), u, f, s, grad, removed."""
    g = plan.grid
    u_star = np.asarray(u_star, dtype=np.float64).reshape(g.dim, -1)
    u_tilde = u_star if f_ib is None else u_star + dt * np.asarray(f_ib, dtype=np.float64).reshape(g.dim, -1)
    s = direct_divergence(plan, u_tilde) / (beta * dt)
    if rhs_mask is not None:
        s = np.where(np.asarray(rhs_mask).reshape(s.shape) != 0, s, 0.0)
    p, removed = solve(s, g.n[: g.dim], g.h[: g.dim], g.bc_lo, g.bc_hi, gauge=gauge, eigenvalues=eigenvalues)
    p_full = embed(p, g)
    grad = node_gradient(plan, p_full)
    ib = plan.node_type != PR.FLUID
    u_new = u_star - beta * dt * grad
    u_new[:, ib] = 0.0
    f_new = np.zeros_like(u_star)
    f_new[:, ib] = -u_star[:, ib] / dt + beta * grad[:, ib]
    return dict(p=p, p_full=p_full, u=u_new, f=f_new, s=s, grad=grad, removed=removed)


def project_ib(plan, dt, u_star, f_init=None, tol=1e-3, max_iters=50, beta=1.5, gauge="mean", eigenvalues="fd",
               rhs_mask=None):
    """The IB-force iteration of §2.3 around the vertex-grid pass, with the stopping rule of
    oracle.projection (ib_change, ib_converged)."""
    u_star = np.asarray(u_star, dtype=np.float64)
    f = np.zeros_like(u_star) if f_init is None else np.asarray(f_init, dtype=np.float64)
    hist = []
    out = None
    for it in range(1, max_iters + 1):
        out = project(plan, dt, u_star, f, beta=beta, gauge=gauge, eigenvalues=eigenvalues, rhs_mask=rhs_mask)
        diff, prev = PR.ib_change(out["f"], f, plan.node_type)
        hist.append((diff, prev))
        f = out["f"]
        if PR.ib_converged(diff, prev, tol):
            break
    out["iterations"] = it
    out["history"] = hist
    return out
