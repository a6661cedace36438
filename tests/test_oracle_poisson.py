"""Pins of the oracle's Poisson solve against the mathematics (no GPU).

* every 1D eigenbasis satisfies the three-point relation of a matrix assembled here, entry by
  entry, from the ghost-cell rules (independent of oracle.grid);
* the solve inverts a brute-force dense Laplacian (LU) on 8x8, 16x16 and 4x4x4 grids for every
  boundary pairing, with a bordered system for the singular (all periodic/Neumann) cases;
* manufactured smooth solutions converge at second order (error ratio ~4 per halving of h);
* an eigenfunction source is solved to round-off in 2D and 3D, including 3*2^m sizes.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import grid as G
from oracle import poisson as P

KINDS = {"PP": ("P", "P"), "NN": ("W", "W"), "DD": ("D", "D"), "ND": ("I", "D"), "DN": ("D", "W")}


def dense_1d(kind, n, h):
    """Three-point second difference with the ghost rule of each end written out."""
    M = np.zeros((n, n))
    for j in range(n):
        M[j, j] -= 2.0
        if j > 0:
            M[j, j - 1] += 1.0
        if j < n - 1:
            M[j, j + 1] += 1.0
    if kind == "PP":
        M[0, n - 1] += 1.0
        M[n - 1, 0] += 1.0
    else:
        lo, hi = kind[0], kind[1]
        M[0, 0] += 1.0 if lo == "N" else -1.0        # ghost p_-1 = +-p_0
        M[n - 1, n - 1] += 1.0 if hi == "N" else -1.0
    return M / (h * h)


def dense_nd(kinds, n, h):
    """Kronecker sum of the 1D matrices (C order: last axis fastest)."""
    dim = len(n)
    total = None
    for a in range(dim):
        mats = [np.eye(n[b]) for b in range(dim)]
        mats[a] = dense_1d(kinds[a], n[a], h[a])
        m = mats[0]
        for b in range(1, dim):
            m = np.kron(m, mats[b])
        total = m if total is None else total + m
    return total


def make_grid(kinds, n, h):
    dim = len(n)
    return G.Grid(dim, tuple(n), tuple([0.0] * dim), tuple(h),
                  tuple(KINDS[k][0] for k in kinds), tuple(KINDS[k][1] for k in kinds))


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("n", [8, 9, 12, 16, 24, 96])
def test_eigenbasis_matches_stencil(kind, n):
    h = 0.37
    M = dense_1d(kind, n, h)
    Phi, lam = P.eigenbasis(kind, n, h)
    assert Phi.shape == (n, n)
    assert np.linalg.matrix_rank(Phi) == n
    err = np.abs(M @ Phi - Phi * lam[None, :]).max()
    assert err <= 1e-12 * 4.0 / (h * h)


def test_eigenvalue_closed_forms():
    """Spot values of the 1D eigenvalues from their closed forms (h = 1)."""
    n = 8
    _, lam = P.eigenbasis("NN", n, 1.0)
    assert lam[0] == 0.0
    assert abs(lam[4] - (-2.0)) < 1e-15                      # -4 sin^2(pi/4)
    _, lam = P.eigenbasis("DD", n, 1.0)
    assert abs(lam[n - 1] - (-4.0)) < 1e-15                  # -4 sin^2(pi/2)
    _, lam = P.eigenbasis("PP", n, 1.0)
    assert abs(sorted(lam)[0] - (-4.0)) < 1e-15              # Nyquist mode
    _, lam = P.eigenbasis("ND", 1, 1.0)
    assert abs(lam[0] - (-2.0)) < 1e-15                      # n=1: ghosts +p0, -p0


def _bruteforce(kinds, n, h, s):
    A = dense_nd(kinds, n, h)
    N = A.shape[0]
    singular = all(k in ("PP", "NN") for k in kinds)
    if singular:
        B = np.zeros((N + 1, N + 1))
        B[:N, :N] = A
        B[:N, N] = 1.0
        B[N, :N] = 1.0
        rhs = np.concatenate([s.ravel(), [0.0]])
        x = np.linalg.solve(B, rhs)
        return x[:N].reshape(n), x[N]
    return np.linalg.solve(A, s.ravel()).reshape(n), 0.0


@pytest.mark.parametrize("n", [(8, 8), (16, 16), (8, 12), (4, 4, 4)])
def test_bruteforce_dense(n, rng):
    dim = len(n)
    for kinds in itertools.product(list(KINDS), repeat=dim):
        if dim == 3 and len(set(kinds)) == 3 and rng.uniform() < 0.7:
            continue  # keep the 3D sweep short
        h = tuple(rng.uniform(0.5, 2.0) for _ in range(dim))
        g = make_grid(kinds, n, h)
        s = rng.normal(size=n)
        p_ref, mu = _bruteforce(kinds, n, h, s)
        p, removed = P.solve(s, g)
        scale = np.abs(p_ref).max()
        assert np.abs(p - p_ref).max() <= 1e-13 * scale * max(n), kinds
        assert abs(removed - mu) <= 1e-12 * max(1.0, abs(mu))


def _manufactured(kind, x, L):
    """(p, -k^2) with p satisfying the boundary pair of kind on [0, L]."""
    if kind == "PP":
        k = 2 * math.pi / L
        return np.sin(k * x), -k * k
    if kind == "NN":
        k = math.pi / L
        return np.cos(k * x), -k * k
    if kind == "DD":
        k = math.pi / L
        return np.sin(k * x), -k * k
    if kind == "ND":
        k = math.pi / (2 * L)
        return np.cos(k * x), -k * k
    if kind == "DN":
        k = math.pi / (2 * L)
        return np.sin(k * x), -k * k
    raise ValueError(kind)


@pytest.mark.parametrize("kinds", [("PP", "PP"), ("NN", "NN"), ("DD", "DD"), ("ND", "NN"),
                                   ("DN", "PP"), ("PP", "DD"), ("ND", "DN")])
def test_manufactured_second_order(kinds):
    L = (2.0, 1.5)
    errs = []
    for m in (16, 32, 64, 128):
        n = (m, m)
        h = (L[0] / m, L[1] / m)
        g = make_grid(kinds, n, h)
        xs = [(np.arange(m) + 0.5) * h[a] for a in range(2)]
        px, kx = _manufactured(kinds[0], xs[0], L[0])
        py, ky = _manufactured(kinds[1], xs[1], L[1])
        pex = np.outer(px, py)
        s = (kx + ky) * pex
        p, _ = P.solve(s, g)
        if g.singular():
            p = p - p.mean()
            pex = pex - pex.mean()
        errs.append(np.abs(p - pex).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios), (errs, ratios)


@pytest.mark.parametrize("n", [(8, 8), (12, 16), (96, 64), (6, 8, 10), (12, 8, 6)])
def test_eigenfunction_source(n, rng):
    dim = len(n)
    for kinds in itertools.product(list(KINDS), repeat=dim):
        if dim == 3 and rng.uniform() < 0.8:
            continue
        h = tuple(rng.uniform(0.5, 2.0) for _ in range(dim))
        g = make_grid(kinds, n, h)
        ks = [int(rng.integers(0, n[a])) for a in range(dim)]
        bases = [P.eigenbasis(kinds[a], n[a], h[a]) for a in range(dim)]
        s = bases[0][0][:, ks[0]]
        lam = bases[0][1][ks[0]]
        for a in range(1, dim):
            s = np.multiply.outer(s, bases[a][0][:, ks[a]])
            lam = lam + bases[a][1][ks[a]]
        p, removed = P.solve(s, g)
        if lam == 0.0:
            assert np.abs(p).max() <= 1e-13
            assert abs(removed - s.mean()) <= 1e-14
        else:
            # dense LU of an n x n basis: round-off grows like n * eps
            assert np.abs(p - s / lam).max() <= 1e-14 * max(n) * np.abs(s / lam).max()


def test_corner_gauge():
    g = make_grid(("NN", "PP"), (8, 8), (1.0, 1.0))
    s = np.random.default_rng(1).normal(size=(8, 8))
    p, _ = P.solve(s, g, gauge="corner")
    assert p[0, 0] == 0.0
    pm, _ = P.solve(s, g)
    assert np.abs((p - p.mean()) - pm).max() < 1e-13


@pytest.mark.parametrize("bc", [("P", "P"), ("W", "W"), ("I", "D"), ("D", "W")])
def test_compensated_residual_is_exact(bc, rng):
    """grid.residual_compensated against exact rational arithmetic (fractions.Fraction), on a
    source that nearly cancels L_h p (residual ~1e-9 of terms ~1e4): the double-double
    evaluation gives the exact residual to a few ulps of the residual itself, where an FP64
    evaluation would be wrong in every digit."""
    from fractions import Fraction
    n = (6, 5)
    g = G.Grid(2, n, (0.0, 0.0), (0.3, 0.7), (bc[0], "W"), (bc[1], "W"))
    p = rng.normal(size=n) * 1e3
    s = G.laplacian(p, g) + rng.normal(size=n) * 1e-9
    got = G.residual_compensated(s, p, g)
    pad = [G._ghost_pad(p, g, a) for a in range(2)]
    for i in range(n[0]):
        for j in range(n[1]):
            acc = Fraction(s[i, j])
            for a, (di, dj) in enumerate(((1, 0), (0, 1))):
                q = pad[a]
                ci, cj = i + di, j + dj              # centre in the padded array
                t = Fraction(q[ci - di, cj - dj]) - 2 * Fraction(q[ci, cj]) + Fraction(q[ci + di, cj + dj])
                acc -= t / Fraction(g.h[a] * g.h[a])
            exact = float(acc)
            assert abs(got[i, j] - exact) <= 4 * np.finfo(float).eps * abs(exact)


def test_refined_solve_is_a_fixed_point(rng):
    """On a 1024 x 512 grid with the channel's boundary pairs, the oracle's solve (dense
    expansion + one compensated refinement sweep) is at the fixed point of refinement: a
    further sweep changes it by less than 1e-15 (relative L2)."""
    g = G.Grid(2, (1024, 512), (0.0, 0.0), (20.0 / 1024, 10.0 / 512), ("I", "W"), ("D", "W"))
    s = rng.normal(size=g.shape)
    p, _ = P.solve(s, g)
    bases = [P.eigenbasis(P.axis_kind(g, a), g.n[a], g.h[a]) for a in range(2)]
    d = P._expand_solve(G.residual_compensated(s, p, g), g, bases, False)
    assert np.linalg.norm(d) <= 1e-15 * np.linalg.norm(p)


# ----------------------------------------------------------------------------- pseudo-spectral
def _continuous_mode(kind, m, n, h):
    """The continuous eigenfunction of d2/dx2 with the axis's boundary conditions, sampled at the
    cell centres x = (j + 1/2) h, and its eigenvalue (independent of the grid)."""
    L = n * h
    x = (np.arange(n) + 0.5) * h
    if kind == "PP":
        k = 2.0 * np.pi * m / L
        return np.cos(k * x + 0.3), -k * k
    if kind == "NN":
        k = np.pi * m / L
        return np.cos(k * x), -k * k
    if kind == "DD":
        k = np.pi * m / L
        return np.sin(k * x), -k * k
    k = np.pi * (m + 0.5) / L
    return (np.cos(k * x) if kind == "ND" else np.sin(k * x)), -k * k


@pytest.mark.parametrize("kinds,n", [(("PP", "NN"), (24, 16)), (("DD", "ND"), (20, 12)),
                                     (("DN", "PP"), (16, 18)), (("NN", "DD", "DN"), (8, 10, 12))])
def test_spectral_solve_is_exact_on_continuous_modes(kinds, n):
    """§2.3 pseudo-spectral eigenvalues: a product of sampled continuous eigenfunctions (each
    resolvable on its axis) is solved exactly, p = s / (sum of continuous eigenvalues), and the
    FD eigenvalues are not (second-order error)."""
    letters = {"PP": ("P", "P"), "NN": ("W", "W"), "DD": ("D", "D"), "ND": ("I", "D"), "DN": ("D", "I")}
    h = [0.1, 0.07, 0.05][:len(n)]
    g = G.Grid(len(n), n, [0.0] * len(n), h, [letters[k][0] for k in kinds], [letters[k][1] for k in kinds])
    rng = np.random.default_rng(31)
    for _ in range(3):
        s = np.ones(n)
        lam = 0.0
        for a, kind in enumerate(kinds):
            m = int(rng.integers(1, n[a] // 2 - 1))
            f, la = _continuous_mode(kind, m, n[a], h[a])
            shape = [1] * len(n)
            shape[a] = n[a]
            s = s * f.reshape(shape)
            lam += la
        p, removed = P.solve(s, g, eigenvalues="spectral")
        assert removed == pytest.approx(0.0, abs=1e-12)
        np.testing.assert_allclose(p, s / lam, rtol=0, atol=1e-12 * np.abs(s / lam).max())
        pfd, _ = P.solve(s, g)
        assert np.abs(pfd - s / lam).max() > 1e-6 * np.abs(s / lam).max()


def test_spectral_accuracy_on_smooth_periodic_function():
    """p = exp(sin x) on [0, 2 pi): from s = p'' the pseudo-spectral solve recovers p - mean(p)
    to rounding at n = 64, while the FD solve keeps its O(h^2) error."""
    n = 64
    h = 2.0 * np.pi / n
    g = G.Grid(2, (n, 4), (0.0, 0.0), (h, 1.0), ("P", "P"), ("P", "P"))
    x = (np.arange(n) + 0.5) * h
    pe = np.exp(np.sin(x))
    se = (np.cos(x) ** 2 - np.sin(x)) * pe
    s = np.repeat(se[:, None], 4, axis=1)
    ref = np.repeat((pe - pe.mean())[:, None], 4, axis=1)
    p, _ = P.solve(s, g, eigenvalues="spectral")
    assert np.abs(p - ref).max() <= 1e-12
    pfd, _ = P.solve(s, g)
    assert np.abs(pfd - ref).max() > 1e-4
