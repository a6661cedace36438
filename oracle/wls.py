"""Weighted-least-squares rows of §2.2 (test infrastructure; see package header).

For a query point x with neighbours x_1..x_K, §2.2 writes a Taylor expansion (Eq. 9) whose
unknowns, when f(x) itself is unknown, are a = [f, f_1, f_2, f_11, f_12, f_22] with the
polynomial vector q_i = [1, dx_1, dx_2, dx_1^2/2, dx_1 dx_2, dx_2^2/2] (Eq. 16). Minimising the
weighted error J (Eq. 12) gives a = C^-1 A b with C = sum_i w_i q_i q_i^T (Eq. 14) and
A = [w_1 q_1, ..., w_K q_K] (Eq. 15), so the rows of C^-1 A are stencil coefficients (Eq. 13):
row 0 reproduces f(x), rows 1..d its first derivatives. In 3D the basis has the 10 terms of
the complete quadratic (the extension §2.2 calls straightforward).

Weight (Eq. 17): w = exp(-eps r^2 / hs^2) for r <= hs, else 0, eps = 6.3, with hs the support
radius. §2.2 sets hs to three times the average spacing of the points. With a fixed stencil of
K points the local average spacing is read off the distance r_K to the farthest of them:
  2D: s = r_K sqrt(pi / K)      3D: s = r_K (4 pi / (3 K))^(1/3),      hs = support_factor * s,
so every stencil point lies inside the support (hs > 1.5 r_K for the stencils used here).

Numerical reading (exact in exact arithmetic): the offsets are scaled, xi = dx / hs, before
forming C; derivative rows are divided by hs afterwards. The solve uses Gaussian elimination
with partial pivoting (numpy.linalg.solve).

Parity: pinned by polynomial reproduction (any quadratic is reproduced exactly, so the value
row sums to 1 and derivative rows sum to 0) in tests/test_oracle_wls.py.
"""
import math
import numpy as np


def num_basis(dim):
    return 6 if dim == 2 else 10


def basis(xi):
    """Polynomial vector of Eq. 16 (2D) or its 3D analogue, in scaled offsets xi[..., d]."""
    d = xi.shape[-1]
    one = np.ones(xi.shape[:-1])
    if d == 2:
        x, y = xi[..., 0], xi[..., 1]
        terms = [one, x, y, 0.5 * x * x, x * y, 0.5 * y * y]
    else:
        x, y, z = xi[..., 0], xi[..., 1], xi[..., 2]
        terms = [one, x, y, z, 0.5 * x * x, x * y, x * z, 0.5 * y * y, y * z, 0.5 * z * z]
    return np.stack(terms, axis=-1)


def support_radius(kth_d2, K, dim, support_factor):
    rK = np.sqrt(kth_d2)
    if dim == 2:
        s = rK * math.sqrt(math.pi / K)
    else:
        s = rK * (4.0 * math.pi / (3.0 * K)) ** (1.0 / 3.0)
    return support_factor * s


def gaussian_weight(r2, hs, eps):
    """Eq. 17 evaluated from the squared distance r2."""
    w = np.exp(-eps * r2 / (hs * hs))
    return np.where(r2 <= hs * hs, w, 0.0)


def pure_second_terms(dim):
    """Basis indices of f_11, f_22 (, f_33): with the 1/2 factors of Eq. 16 their rows of C^-1 A
    are the second derivatives themselves."""
    return (3, 5) if dim == 2 else (4, 7, 9)


def rows(delta, d2, eps, support_factor, laplacian=False):
    """WLS coefficient rows for a batch of queries.

    delta (Q, K, d): stencil offsets x_k - x (minimum image); d2 (Q, K): squared distances.
    The local spacing comes from the farthest stencil point (the K-th neighbour of a K-nearest
    stencil). Returns (value_row (Q, K), grad_rows (Q, d, K)), and with laplacian=True also the
    Laplacian row (Q, K): the sum of the pure second-derivative rows (scaled by 1/hs^2).
    """
    Q, K, d = delta.shape
    hs = support_radius(d2.max(axis=1), K, d, support_factor)     # (Q,)
    w = gaussian_weight(d2, hs[:, None], eps)                       # (Q, K)
    xi = delta / hs[:, None, None]
    q = basis(xi)                                                   # (Q, K, m)
    A = np.transpose(q * w[:, :, None], (0, 2, 1))                  # (Q, m, K): [w_k q_k]
    C = A @ q                                                       # (Q, m, m): sum w q q^T
    ev = np.linalg.eigvalsh(C)
    if np.any(ev[:, 0] <= 1e-13 * ev[:, -1]):
        raise np.linalg.LinAlgError("WLS normal matrix C is singular for some query")
    R = np.linalg.solve(C, A)                                       # (Q, m, K) = C^-1 A
    value = R[:, 0, :]
    grad = R[:, 1:1 + d, :] / hs[:, None, None]
    if not laplacian:
        return value, grad
    lap = R[:, list(pure_second_terms(d)), :].sum(axis=1) / (hs * hs)[:, None]
    return value, grad, lap
