"""Pins of the oracle's neighbour search and WLS rows (no GPU).

* cell-list KNN equals brute force over all pairs (Python sort on (d2, index)), with periodic
  wrap, exact ties on a lattice, 2D and 3D;
* the WLS rows reproduce every quadratic exactly: the value row gives f(x), the derivative
  rows give grad f(x) (so the value row sums to 1 and derivative rows sum to 0);
* the Gaussian weight of Eq. 17 at its closed-form points.
"""
import math

import numpy as np
import pytest

from oracle import knn as KNN
from oracle import wls as W


def brute_knn(points, queries, K, lengths, periodic):
    out = []
    for q in queries:
        rows = []
        for i, p in enumerate(points):
            d2 = 0.0
            for a in range(len(q)):
                da = float(p[a]) - float(q[a])
                if periodic[a]:
                    if da > 0.5 * lengths[a]:
                        da -= lengths[a]
                    elif da < -0.5 * lengths[a]:
                        da += lengths[a]
                d2 = d2 + da * da
            rows.append((d2, i))
        rows.sort()
        out.append([i for _, i in rows[:K]])
    return np.array(out)


@pytest.mark.parametrize("dim,periodic", [(2, (True, True)), (2, (False, True)), (2, (False, False)),
                                          (3, (True, False, True)), (3, (False, False, False))])
def test_knn_bruteforce(dim, periodic, rng):
    lengths = [1.0, 0.75, 0.5][:dim]
    lo = [0.0] * dim
    M = 700 if dim == 2 else 900
    pts = rng.uniform(0, 1, size=(M, dim)) * np.asarray(lengths)
    qs = rng.uniform(0, 1, size=(60, dim)) * np.asarray(lengths)
    K = 12 if dim == 2 else 27
    idx, d2 = KNN.knn(pts, qs, K, lo, lengths, list(periodic), occupancy=3.0)
    ref = brute_knn(pts, qs, K, lengths, periodic)
    assert np.array_equal(idx, ref)
    assert np.all(np.diff(d2, axis=1) >= 0)


def test_knn_lattice_ties():
    """On an exact lattice many distances tie; the order must be (d2, index)."""
    n = 10
    g = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    qs = pts[[0, 5, 37, 99]]
    for periodic in ([True, True], [False, False]):
        idx, _ = KNN.knn(pts, qs, 12, [0.0, 0.0], [1.0, 1.0], periodic, occupancy=2.0)
        ref = brute_knn(pts, qs, 12, [1.0, 1.0], periodic)
        assert np.array_equal(idx, ref)


def _cloud(dim, rng, m=9, jitter=0.3):
    g = np.arange(-(m // 2), m // 2 + 1, dtype=np.float64)
    mesh = np.meshgrid(*([g] * dim), indexing="ij")
    pts = np.stack([x.ravel() for x in mesh], 1) * 0.1
    return pts + rng.uniform(-jitter, jitter, pts.shape) * 0.1


@pytest.mark.parametrize("dim", [2, 3])
def test_polynomial_reproduction(dim, rng):
    K = 12 if dim == 2 else 27
    pts = _cloud(dim, rng)
    queries = rng.uniform(-0.05, 0.05, size=(40, dim))
    idx, d2 = KNN.knn(pts, queries, K, [-1.0] * dim, [2.0] * dim, [False] * dim)
    delta = pts[idx] - queries[:, None, :]
    val, grad = W.rows(delta, d2, 6.3, 3.0)
    # a random quadratic f(x) = c + b.x + x^T A x
    c = rng.normal()
    b = rng.normal(size=dim)
    A = rng.normal(size=(dim, dim))
    A = A + A.T

    def f(x):
        return c + x @ b + np.einsum("...i,ij,...j->...", x, A, x)

    def df(x):
        return b + 2.0 * x @ A

    fk = f(pts[idx])                                      # (Q, K)
    assert np.abs(np.sum(val * fk, axis=1) - f(queries)).max() < 1e-12
    g_est = np.einsum("qdk,qk->qd", grad, fk)
    assert np.abs(g_est - df(queries)).max() < 1e-10
    assert np.abs(val.sum(axis=1) - 1.0).max() < 1e-13
    assert np.abs(grad.sum(axis=2)).max() < 1e-10


def test_cubic_is_not_reproduced(rng):
    """Sanity of the pin above: a cubic term is not reproduced, so the test can fail."""
    pts = _cloud(2, rng)
    q = np.array([[0.013, -0.021]])
    idx, d2 = KNN.knn(pts, q, 12, [-1.0, -1.0], [2.0, 2.0], [False, False])
    val, _ = W.rows(pts[idx] - q[:, None, :], d2, 6.3, 3.0)
    fk = pts[idx][..., 0] ** 3
    assert abs(np.sum(val * fk) - q[0, 0] ** 3) > 1e-9


def test_gaussian_weight_closed_form():
    eps = 6.3
    assert W.gaussian_weight(np.array(0.0), 2.0, eps) == 1.0
    assert abs(W.gaussian_weight(np.array(4.0), 2.0, eps) - math.exp(-eps)) < 1e-16
    assert W.gaussian_weight(np.array(4.0000001), 2.0, eps) == 0.0
    assert abs(W.gaussian_weight(np.array(1.0), 2.0, eps) - math.exp(-eps / 4)) < 1e-16


def test_support_radius_reading():
    """hs = 3 x local spacing; spacing from the K-th distance (2D: r_K sqrt(pi/K))."""
    hs = W.support_radius(np.array(4.0), 12, 2, 3.0)
    assert abs(hs - 3.0 * 2.0 * math.sqrt(math.pi / 12)) < 1e-15
    hs3 = W.support_radius(np.array(4.0), 27, 3, 3.0)
    assert abs(hs3 - 3.0 * 2.0 * (4 * math.pi / 81) ** (1 / 3)) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_laplacian_row_reproduces_quadratics(dim, rng):
    """The Laplacian row (sum of the pure second-derivative rows of C^-1 A) returns 2 tr(A) for
    f = c + b.x + x^T A x at every query, sums to 0, and misses the x^3 term's Laplacian."""
    K = 12 if dim == 2 else 27
    pts = _cloud(dim, rng)
    queries = rng.uniform(-0.05, 0.05, size=(40, dim))
    idx, d2 = KNN.knn(pts, queries, K, [-1.0] * dim, [2.0] * dim, [False] * dim)
    delta = pts[idx] - queries[:, None, :]
    val, grad, lap = W.rows(delta, d2, 6.3, 3.0, laplacian=True)
    val0, grad0 = W.rows(delta, d2, 6.3, 3.0)
    assert np.array_equal(val, val0) and np.array_equal(grad, grad0)
    c, b, A = rng.normal(), rng.normal(size=dim), rng.normal(size=(dim, dim))
    A = A + A.T
    fk = c + pts[idx] @ b + np.einsum("qki,ij,qkj->qk", pts[idx], A, pts[idx])
    assert np.abs(np.sum(lap * fk, axis=1) - 2.0 * np.trace(A)).max() < 1e-7 * (1 + abs(np.trace(A)))
    assert np.abs(lap.sum(axis=1)).max() < 1e-6 * np.abs(lap).max()
    cub = pts[idx][..., 0] ** 3
    assert np.abs(np.sum(lap * cub, axis=1) - 6.0 * queries[:, 0]).max() > 1e-9
