"""Pins of the regular (vertex) grid Poisson solve of the oracle (oracle/vertex.py)."""
import itertools

import numpy as np
import pytest

from oracle import grid as G
from oracle import poisson as P
from oracle import vertex as V

KINDS = {"PP": ("P", "P"), "NN": ("W", "W"), "DD": ("D", "D"), "ND": ("I", "D"), "DN": ("D", "W")}


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("n", [6, 8, 12, 15])
def test_eigenvectors(kind, n):
    """Every basis vector satisfies the 3-point relation with the axis's ghost rules."""
    if kind == "PP" and n % 2:
        pytest.skip("periodic axes of odd length are not used")
    h = 0.3
    Phi, lam = V.eigenbasis(kind, n, h)
    assert Phi.shape[0] == V.unknowns(kind, n)[0] == Phi.shape[1]
    for k in range(Phi.shape[1]):
        Lv = V.laplacian(Phi[:, k], [kind], [h])
        assert np.abs(Lv - lam[k] * Phi[:, k]).max() <= 1e-11 * max(1.0, abs(lam[k]))
    assert np.linalg.matrix_rank(Phi) == Phi.shape[1]


def _weights(kind, m):
    w = np.ones(m)
    if kind == "NN":
        w[0] = w[-1] = 0.5
    return w


def _brute(s, kinds, n, h):
    """Dense operator assembled by applying the ghost rules to unit vectors; singular problems
    are bordered with the trapezoid-weighted constraint (the operator's left null vector)."""
    shape = s.shape
    m = s.size
    A = np.zeros((m, m))
    for c in range(m):
        e = np.zeros(m)
        e[c] = 1.0
        A[:, c] = V.laplacian(e.reshape(shape), kinds, h).ravel()
    singular = all(k in ("PP", "NN") for k in kinds)
    if not singular:
        return np.linalg.solve(A, s.ravel()).reshape(shape), 0.0
    w = np.ones(shape)
    for a, k in enumerate(kinds):
        sh = [1] * len(shape)
        sh[a] = shape[a]
        w = w * _weights(k, shape[a]).reshape(sh)
    B = np.zeros((m + 1, m + 1))
    B[:m, :m] = A
    B[:m, m] = 1.0
    B[m, :m] = w.ravel()
    x = np.linalg.solve(B, np.concatenate([s.ravel(), [0.0]]))
    return x[:m].reshape(shape), x[m]


@pytest.mark.parametrize("n", [(6, 5), (8, 4, 5)])
def test_brute_force(n):
    dim = len(n)
    h = [0.2, 0.3, 0.25][:dim]
    combos = list(itertools.product(list(KINDS), repeat=dim))
    if dim == 3:
        combos = combos[::9]
    rng = np.random.default_rng(3)
    for kinds in combos:
        if any(k == "PP" and n[a] % 2 for a, k in enumerate(kinds)):
            continue
        shape = tuple(V.unknowns(k, n[a])[0] for a, k in enumerate(kinds))
        s = rng.normal(size=shape)
        p, removed = V.solve(s, n, h, [KINDS[k][0] for k in kinds], [KINDS[k][1] for k in kinds])
        pb, mu = _brute(s, list(kinds), n, h)
        assert np.abs(p - pb).max() <= 1e-11 * max(1.0, np.abs(pb).max()), kinds
        assert removed == pytest.approx(mu, abs=1e-12), kinds


def test_manufactured_second_order():
    """p = cos(pi x/L0) sin(pi y/L1) on an N-N x D-D vertex grid: the FD error falls by 4 per
    halving of h."""
    errs = []
    for n0 in (16, 32, 64):
        n = (n0, n0 // 2)
        L = (2.0, 1.0)
        h = (L[0] / n[0], L[1] / n[1])
        x = np.arange(n[0] + 1) * h[0]
        y = np.arange(1, n[1]) * h[1]
        X, Y = np.meshgrid(x, y, indexing="ij")
        pe = np.cos(np.pi * X / L[0]) * np.sin(np.pi * Y / L[1])
        s = -((np.pi / L[0]) ** 2 + (np.pi / L[1]) ** 2) * pe
        p, _ = V.solve(s, n, h, ("W", "D"), ("W", "D"))
        errs.append(np.abs(p - pe).max())
    r = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.6 < x < 4.4 for x in r), r


@pytest.mark.parametrize("kinds", [("NN", "DD"), ("ND", "DN"), ("PP", "NN")])
def test_spectral_exact_on_continuous_modes(kinds):
    """With the pseudo-spectral eigenvalues a sampled continuous eigenfunction is solved exactly."""
    n, h = (12, 10), (0.1, 0.2)
    L = (n[0] * h[0], n[1] * h[1])
    s = np.ones(tuple(V.unknowns(k, n[a])[0] for a, k in enumerate(kinds)))
    lam = 0.0
    for a, k in enumerate(kinds):
        m, j0 = V.unknowns(k, n[a])
        x = (np.arange(m) + j0) * h[a]
        if k == "PP":
            kk = 2.0 * np.pi * 2 / L[a]
            f = np.cos(kk * x + 0.4)
        elif k in ("NN", "DD"):
            kk = np.pi * 3 / L[a]
            f = np.cos(kk * x) if k == "NN" else np.sin(kk * x)
        else:
            kk = np.pi * 2.5 / L[a]
            f = np.cos(kk * x) if k == "ND" else np.sin(kk * x)
        sh = [1, 1]
        sh[a] = m
        s = s * f.reshape(sh)
        lam -= kk * kk
    p, _ = V.solve(s, n, h, [KINDS[k][0] for k in kinds], [KINDS[k][1] for k in kinds], eigenvalues="spectral")
    assert np.abs(p - s / lam).max() <= 1e-12 * np.abs(s / lam).max()
    pfd, _ = V.solve(s, n, h, [KINDS[k][0] for k in kinds], [KINDS[k][1] for k in kinds])
    assert np.abs(pfd - s / lam).max() > 1e-5 * np.abs(s / lam).max()


def _extend_axis(kind, n):
    """(extended length, [(unknown index or -1, sign)] per extended cell) of the symmetric
    extension: even about a Neumann end, odd about a Dirichlet end, periodic of period m."""
    m, j0 = V.unknowns(kind, n)
    if kind == "PP":
        return n, [(e, 1.0) for e in range(n)]
    period = 2 * n if kind in ("NN", "DD") else 4 * n
    even_lo, even_hi = kind[0] == "N", kind[1] == "N"
    out = []
    for e in range(period):
        # fold e into [0, n] with the reflections, tracking the sign
        x, sign = e, 1.0
        for _ in range(4):
            if x > n:                       # reflect about n
                x = 2 * n - x
                sign *= 1.0 if even_hi else -1.0
            elif x < 0:                     # reflect about 0
                x = -x
                sign *= 1.0 if even_lo else -1.0
            else:
                break
        if x > n or x < 0:
            x = x % period
        j = x
        if (j == 0 and not even_lo) or (j == n and not even_hi):
            out.append((-1, 0.0))
        else:
            out.append((j - j0, sign))
    return period, out


@pytest.mark.parametrize("kinds", [("NN", "DD"), ("ND", "PP"), ("DN", "NN"), ("DD", "ND")])
def test_symmetric_extension_identity(kinds):
    """The vertex solution equals the restriction of the periodic cell-grid solve (oracle.poisson,
    a separate solver) of the source extended evenly about Neumann ends and oddly about
    Dirichlet ends: the real DFT of such an extension is the DCT-I / DST-I (or the quarter-wave
    pair) of the vertex values."""
    n, h = (8, 6), (0.25, 0.4)
    rng = np.random.default_rng(11)
    shape = tuple(V.unknowns(k, n[a])[0] for a, k in enumerate(kinds))
    s = rng.normal(size=shape)
    p, removed = V.solve(s, n, h, [KINDS[k][0] for k in kinds], [KINDS[k][1] for k in kinds])
    ext = [_extend_axis(k, n[a]) for a, k in enumerate(kinds)]
    m = tuple(e[0] for e in ext)
    se = np.zeros(m)
    for e0 in range(m[0]):
        u0, g0 = ext[0][1][e0]
        for e1 in range(m[1]):
            u1, g1 = ext[1][1][e1]
            if u0 >= 0 and u1 >= 0:
                se[e0, e1] = g0 * g1 * s[u0, u1]
    g = G.Grid(2, m, (0.0, 0.0), h, ("P", "P"), ("P", "P"))
    pe, removed_e = P.solve(se, g)
    j0 = [V.unknowns(k, n[a])[1] for a, k in enumerate(kinds)]
    back = pe[j0[0]:j0[0] + shape[0], j0[1]:j0[1] + shape[1]]
    assert np.abs(back - p).max() <= 1e-11 * np.abs(p).max()
    assert removed_e == pytest.approx(removed, abs=1e-12)


# ----------------------------------------------------------------------------- the vertex-grid pass
from paper_2304_14690_gb300 import workloads as wl   # noqa: E402


def _grid(prob):
    return G.Grid(prob.dim, prob.n, prob.lo, prob.h, prob.bc_lo, prob.bc_hi)


def test_pressure_points_and_block():
    """Unknown positions per boundary pair, and the gradient block: nearest vertex and its
    neighbours, shifted inward at ends, wrapped on a periodic axis."""
    g = G.Grid(2, (6, 4), (0.0, 0.0), (1.0, 1.0), ("D", "P"), ("W", "P"))
    assert V.lattice_shape(g) == (7, 4)
    pp = V.pressure_points(g)
    assert sorted(set(pp[:, 0])) == [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]     # D-N: vertices 1..n
    assert sorted(set(pp[:, 1])) == [0.0, 1.0, 2.0, 3.0]               # P-P: 0..n-1
    g2 = G.Grid(2, (6, 4), (0.0, 0.0), (1.0, 1.0), ("D", "I"), ("D", "D"))
    assert sorted(set(V.pressure_points(g2)[:, 0])) == [1.0, 2.0, 3.0, 4.0, 5.0]   # D-D
    assert sorted(set(V.pressure_points(g2)[:, 1])) == [0.0, 1.0, 2.0, 3.0]        # N-D
    pts = np.array([[0.2, 0.2], [5.9, 3.7], [2.6, 1.4], [6.0, 3.45]])
    idx = V.vertex_block(g, pts)
    rows = [sorted({int(c) // 4 for c in r}) for r in idx]
    cols = [sorted({int(c) % 4 for c in r}) for r in idx]
    assert rows == [[0, 1, 2], [4, 5, 6], [2, 3, 4], [4, 5, 6]]
    assert cols == [[0, 1, 3], [0, 1, 3], [0, 1, 2], [0, 2, 3]]


@pytest.mark.parametrize("case", [
    dict(dim=2, n=(20, 16), bc_lo=("W", "D"), bc_hi=("I", "W"), obstacles=[("circle", (0.6, 0.5), 0.15)]),
    dict(dim=2, n=(16, 20), bc_lo=("D", "D"), bc_hi=("W", "D")),
    dict(dim=3, n=(8, 10, 6), bc_lo=("W", "D", "I"), bc_hi=("W", "W", "D")),
])
def test_vertex_rows_reproduce_quadratics(case):
    """Derivative rows at the pressure points (divergence of a quadratic velocity) and at the
    nodes over the vertex block (gradient of a quadratic pressure) are exact, at boundary
    vertices and next to obstacles."""
    prob = wl.generic(seed=21, **case)
    g = _grid(prob)
    pl = V.build_plan(g, prob.nodes, prob.node_type, K=prob.knn)
    d = prob.dim
    rng = np.random.default_rng(4)
    A, B, c0 = rng.normal(size=(d, d)), rng.normal(size=(d, d, d)), rng.normal(size=d)
    x = prob.nodes
    u = c0[:, None] + A @ x + np.einsum("aij,im,jm->am", B, x, x)
    div = V.direct_divergence(pl, u).ravel()
    q = V.pressure_points(g).T
    expect = np.trace(A) + sum((B[a, a, :] + B[a, :, a]) @ q for a in range(d))
    np.testing.assert_allclose(div, expect, rtol=0, atol=1e-9 * (1 + np.abs(expect).max()))
    Q, b = rng.normal(size=(d, d)), rng.normal(size=d)
    Q = Q + Q.T
    lp = V.lattice_points(g).T
    p_full = (b @ lp + 0.5 * np.einsum("im,ij,jm->m", lp, Q, lp)).reshape(V.lattice_shape(g))
    gr = V.node_gradient(pl, p_full)
    ex = b[:, None] + Q @ x
    assert np.abs(gr - ex).max() < 1e-9 * (1 + np.abs(ex).max())


def _phi(kinds, L):
    """A smooth pressure meeting each axis's boundary pair, with its gradient."""
    f, df = [], []
    for k, l in zip(kinds, L):
        if k == "PP":
            f.append(lambda x, l=l: np.sin(2 * np.pi * x / l)); df.append(lambda x, l=l: 2 * np.pi / l * np.cos(2 * np.pi * x / l))
        elif k == "NN":
            f.append(lambda x, l=l: np.cos(np.pi * x / l)); df.append(lambda x, l=l: -np.pi / l * np.sin(np.pi * x / l))
        elif k == "DD":
            f.append(lambda x, l=l: np.sin(np.pi * x / l)); df.append(lambda x, l=l: np.pi / l * np.cos(np.pi * x / l))
        elif k == "ND":
            f.append(lambda x, l=l: np.cos(0.5 * np.pi * x / l)); df.append(lambda x, l=l: -0.5 * np.pi / l * np.sin(0.5 * np.pi * x / l))
        else:
            f.append(lambda x, l=l: np.sin(0.5 * np.pi * x / l)); df.append(lambda x, l=l: 0.5 * np.pi / l * np.cos(0.5 * np.pi * x / l))

    def phi(x):
        return np.prod([f[a](x[a]) for a in range(len(kinds))], axis=0)

    def grad(x):
        return np.stack([df[a](x[a]) * np.prod([f[b](x[b]) for b in range(len(kinds)) if b != a], axis=0)
                         for a in range(len(kinds))])
    return phi, grad


@pytest.mark.parametrize("kinds", [("NN", "DD"), ("NN", "NN"), ("PP", "ND"), ("DN", "PP")])
def test_vertex_projection_recovers_pressure(kinds):
    """u* = beta dt grad(phi) with phi meeting the boundary conditions: the pass returns p -> phi
    at the vertices and u -> 0 at the nodes, both at second order in h."""
    ep, eu = [], []
    for n in (32, 64, 128):
        h = (1.0 / n, 1.0 / n)
        prob = wl.generic(dim=2, n=(n, n), h=h, bc_lo=tuple(KINDS[k][0] for k in kinds),
                          bc_hi=tuple(KINDS[k][1] for k in kinds), seed=13)
        g = _grid(prob)
        pl = V.build_plan(g, prob.nodes, prob.node_type, K=12)
        phi, grad = _phi(kinds, (1.0, 1.0))
        u_star = prob.beta * prob.dt * grad(prob.nodes)
        r = V.project(pl, prob.dt, u_star)
        ref = phi(V.pressure_points(g).T).reshape(r["p"].shape)
        ep.append(np.abs(r["p"] - ref).max())
        eu.append(np.abs(r["u"]).max())
    assert ep[-1] < 1e-3 and eu[-1] < 1e-2, (ep, eu)
    assert all(ep[i] / ep[i + 1] > 3.3 for i in range(2)), ep
    assert all(eu[i] / eu[i + 1] > 3.3 for i in range(2)), eu


def test_vertex_ib_relations_and_iteration():
    """IB nodes: u = 0 and f = -u*/dt + beta grad p; the iteration stops by the §2.3 rule and its
    last pass is the pass with the previous force."""
    prob = wl.generic(dim=2, n=(24, 16), bc_lo=("I", "W"), bc_hi=("D", "W"),
                      obstacles=[("circle", (0.7, 0.5), 0.2)], seed=2, with_force=True)
    g = _grid(prob)
    pl = V.build_plan(g, prob.nodes, prob.node_type, K=12)
    r = V.project(pl, prob.dt, prob.u_star, prob.f_ib)
    ib = prob.node_type != 0
    assert ib.any()
    assert np.all(r["u"][:, ib] == 0.0) and np.all(r["f"][:, ~ib] == 0.0)
    np.testing.assert_allclose(r["f"][:, ib], -prob.u_star[:, ib] / prob.dt + prob.beta * r["grad"][:, ib],
                               rtol=1e-12, atol=1e-12)
    it = V.project_ib(pl, prob.dt, prob.u_star, tol=1e-3, max_iters=40)
    assert 2 <= it["iterations"] < 40
    diff, prev = it["history"][-1]
    assert diff <= 1e-3 * prev
    assert all(d > 1e-3 * p for d, p in it["history"][:-1])


def test_vertex_rhs_mask_zeroes_source():
    """The masked source is zero outside the mask and unchanged inside; an all-ones mask changes
    nothing."""
    prob = wl.generic(dim=2, n=(16, 12), bc_lo=("W", "W"), bc_hi=("D", "W"), seed=6)
    g = _grid(prob)
    pl = V.build_plan(g, prob.nodes, prob.node_type, K=12)
    r0 = V.project(pl, prob.dt, prob.u_star)
    mask = np.random.default_rng(1).random(r0["s"].shape) > 0.3
    r1 = V.project(pl, prob.dt, prob.u_star, rhs_mask=mask)
    assert np.array_equal(r1["s"][mask], r0["s"][mask]) and np.all(r1["s"][~mask] == 0.0)
    r2 = V.project(pl, prob.dt, prob.u_star, rhs_mask=np.ones_like(mask))
    assert np.array_equal(r2["p"], r0["p"])
