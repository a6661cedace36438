"""Exact solve of the discrete pressure Poisson equation (test infrastructure; see package header).

§2.3 solves the (modified) PPE on the regular grid in three steps: forward one-dimensional
transforms along each axis in turn, division by the eigenvalues (the sum of the 1D
eigenvalues), backward transforms. With the central finite-difference eigenvalues this is an
exact inverse of the 2d+1-point Laplacian L_h. The oracle states that inverse in its plain
form: it expands the source in the eigenvectors of the 1D three-point operator with the
ghost rules of oracle.grid (one dense basis per axis), divides by the summed eigenvalues and
sums the expansion back. No fast transform is used; numpy.linalg.solve finds the expansion
coefficients from the dense basis.

1D eigenbases on a cell-centred axis (j, k = 0..n-1; Neumann = 'W' or 'I'):
  periodic      1, cos(2 pi k j/n), sin(2 pi k j/n), (-1)^j     lambda = -(4/h^2) sin^2(pi k/n)
  Neumann-Neumann   cos(pi k (j+1/2)/n)                          lambda = -(4/h^2) sin^2(pi k/(2n))
  Dirichlet-Dirichlet sin(pi (k+1)(j+1/2)/n)                     lambda = -(4/h^2) sin^2(pi (k+1)/(2n))
  Neumann-Dirichlet cos(pi (k+1/2)(j+1/2)/n)                     lambda = -(4/h^2) sin^2(pi (2k+1)/(4n))
  Dirichlet-Neumann sin(pi (k+1/2)(j+1/2)/n)                     same lambda
The last two pairs put different homogeneous conditions at the two ends of one axis, which
§2.3 does not list (it asks for the same type on both ends); they are still diagonalised
exactly by these bases and are used for an inflow/outflow channel.

§2.3 allows two sets of eigenvalues with the same transforms: the central finite-difference
ones above (the exact inverse of L_h), and the pseudo-spectral ones. Writing each FD eigenvalue
as -(2/h)^2 sin^2(theta/2), theta = 2 pi k/n (periodic, k the wavenumber), pi k/n (N-N),
pi (k+1)/n (D-D) or pi (k+1/2)/n (N-D, D-N), the pseudo-spectral eigenvalue of the same basis
vector is -(theta/h)^2: the eigenvalue of the continuous second derivative for the continuous
eigenfunction that the basis vector samples at the cell centres. The pseudo-spectral solve is
defined by its expansion alone (its operator has no compact stencil), so it takes no
refinement sweep; at the sizes where it is compared the expansion is at FP64 rounding.

Zero mode: when every axis is periodic or Neumann-Neumann the summed eigenvalue of the
constant mode is 0. Its source coefficient is the mean of s, which is dropped (the
compatibility projection) and the solution gets no constant part (mean(p) = 0). An optional
corner gauge p[0,...,0] = 0 matches the reference pressure of §3.1.

Parity: pinned by tests/test_oracle_poisson.py - eigenvector relations against an
independently assembled matrix, a brute-force dense LU solve on 8x8, 16x16 and 4x4x4 grids,
manufactured solutions converging at second order, and the compensated residual of large
solves at the FP64 floor.
"""
import numpy as np

from .grid import NEUMANN, residual_compensated


def axis_kind(g, a):
    lo, hi = g.bc_lo[a], g.bc_hi[a]
    if lo == "P":
        return "PP"
    lo = "N" if lo in NEUMANN else "D"
    hi = "N" if hi in NEUMANN else "D"
    return lo + hi


def _lam(theta, h, eigenvalues):
    """FD or pseudo-spectral eigenvalue of the basis vector with angle theta (§2.3)."""
    if eigenvalues == "fd":
        return -(4.0 / (h * h)) * np.sin(theta / 2.0) ** 2
    if eigenvalues == "spectral":
        return -(theta / h) ** 2
    raise ValueError(eigenvalues)


def eigenbasis(kind, n, h, eigenvalues="fd"):
    """(Phi, lam): Phi[:, k] is the k-th eigenvector of the 1D operator, lam[k] its eigenvalue
    (central finite-difference or pseudo-spectral, see the module header)."""
    j = np.arange(n, dtype=np.float64)[:, None]
    if kind == "PP":
        cols, wav = [np.ones(n)], [0]
        for k in range(1, (n - 1) // 2 + 1):
            cols.append(np.cos(2.0 * np.pi * k * j[:, 0] / n))
            cols.append(np.sin(2.0 * np.pi * k * j[:, 0] / n))
            wav += [k, k]
        if n % 2 == 0:
            cols.append(np.cos(np.pi * j[:, 0]))
            wav.append(n // 2)
        Phi = np.stack(cols, axis=1)
        return Phi, _lam(2.0 * np.pi * np.asarray(wav, dtype=np.float64) / n, h, eigenvalues)
    k = np.arange(n, dtype=np.float64)[None, :]
    if kind == "NN":
        Phi = np.cos(np.pi * k * (j + 0.5) / n)
        theta = np.pi * k[0] / n
    elif kind == "DD":
        Phi = np.sin(np.pi * (k + 1.0) * (j + 0.5) / n)
        theta = np.pi * (k[0] + 1.0) / n
    elif kind == "ND":
        Phi = np.cos(np.pi * (k + 0.5) * (j + 0.5) / n)
        theta = np.pi * (k[0] + 0.5) / n
    elif kind == "DN":
        Phi = np.sin(np.pi * (k + 0.5) * (j + 0.5) / n)
        theta = np.pi * (k[0] + 0.5) / n
    else:
        raise ValueError(kind)
    return Phi, _lam(theta, h, eigenvalues)


def _apply(M, x, a):
    """Multiply the matrix M onto axis a of x."""
    y = np.tensordot(M, x, axes=([1], [a]))
    return np.moveaxis(y, 0, a)


def _solve_along(M, x, a):
    """Solve M y = x along axis a of x (dense LU per axis, all lines at once)."""
    xa = np.moveaxis(x, a, 0)
    shp = xa.shape
    y = np.linalg.solve(M, xa.reshape(shp[0], -1)).reshape(shp)
    return np.moveaxis(y, 0, a)


def _expand_solve(s, g, bases, singular):
    """Steps 1-3 of §2.3 with the dense bases: the solution with no constant part (the zero-mode
    coefficient is dropped when the problem is singular)."""
    coef = s
    for a in range(g.dim):                      # step 1: forward expansion, axis by axis
        coef = _solve_along(bases[a][0], coef, a)
    lam = np.zeros(g.shape)                     # step 2: divide by the summed eigenvalues
    for a in range(g.dim):
        shape = [1] * g.dim
        shape[a] = g.n[a]
        lam = lam + bases[a][1].reshape(shape)
    zero = tuple([0] * g.dim)
    if singular:
        lam[zero] = 1.0
        coef = coef.copy()
        coef[zero] = 0.0
    p = coef / lam
    for a in range(g.dim):                      # step 3: backward expansion
        p = _apply(bases[a][0], p, a)
    return p


def solve(s, g, gauge="mean", eigenvalues="fd"):
    """Return (p, removed_mean) with L_h p = s (s minus its mean when the problem is singular);
    with eigenvalues="spectral" the pseudo-spectral solve of the same source instead.

    removed_mean is the mean of s dropped by the compatibility projection (0 otherwise).

    The dense expansion alone loses accuracy with the conditioning of L_h: on a 1024 x 512
    grid its result is 1e-13 to 1e-12 (relative L2) away from the exact discrete solution,
    depending on the BLAS. One sweep of iterative refinement, p += solve(s - L_h p) with the
    residual in double-double arithmetic (grid.residual_compensated), brings it to FP64
    rounding of the exact solution that the three-step algorithm defines."""
    s = np.asarray(s, dtype=np.float64).reshape(g.shape)
    bases = [eigenbasis(axis_kind(g, a), g.n[a], g.h[a], eigenvalues) for a in range(g.dim)]
    singular = g.singular()
    removed = float(np.mean(s)) if singular else 0.0
    p = _expand_solve(s, g, bases, singular)
    if eigenvalues == "fd":
        r = residual_compensated(s - removed if singular else s, p, g)
        p = p + _expand_solve(r, g, bases, singular)
    if singular and gauge == "corner":
        p = p - p[tuple([0] * g.dim)]
    return p, removed
