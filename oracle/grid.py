"""Staggered pressure grid of the hybrid method (test infrastructure; see package header).

The pressure points of §2.3 (double discretization, Fig. 1) are the centres of a uniform
Cartesian grid covering the extended rectangle. Velocity components of the transferred field
live on the cell faces (a staggered / MAC arrangement, the grid type the paper uses in §3.3).

Boundary kinds per domain face (one letter each):
  'P' periodic (must pair with 'P' on the same axis),
  'W' wall: homogeneous Neumann, Eq. 7; the normal flux through the face is zero, following
      the workaround of §3.3 (u*.n cancels on a staggered grid and may be set to zero),
  'I' inflow: homogeneous Neumann, Eq. 7 (u^{n+1}.n = u*.n), the face keeps its transferred flux,
  'D' homogeneous Dirichlet (p = 0 on the face); the face keeps its transferred flux.

Ghost-cell rules of the 2d+1-point Laplacian (p_{-1} and p_n are the ghost values):
  Neumann (W, I): p_{-1} = p_0,     p_n = p_{n-1}
  Dirichlet (D):  p_{-1} = -p_0,    p_n = -p_{n-1}
  periodic:       p_{-1} = p_{n-1}, p_n = p_0
With these rules the face gradient G_h and the cell divergence D_h satisfy D_h G_h = L_h
exactly, which is what makes "discrete divergence after projection at round-off" checkable.

Parity: pinned by tests/test_oracle_poisson.py (brute-force matrix assembled independently,
manufactured solutions at second order) and tests/test_oracle_projection.py (D_h G_h = L_h).
"""
from dataclasses import dataclass
import numpy as np

NEUMANN = ("W", "I")


@dataclass(frozen=True)
class Grid:
    dim: int
    n: tuple          # cells per axis
    lo: tuple         # lower domain corner
    h: tuple          # spacing per axis
    bc_lo: tuple      # one letter per axis (see module doc)
    bc_hi: tuple

    @property
    def shape(self):
        return tuple(int(v) for v in self.n[: self.dim])

    def length(self, a):
        # The domain length is defined as n*h (one rounded product) on every side of the parity.
        return float(self.n[a]) * float(self.h[a])

    def periodic(self, a):
        return self.bc_lo[a] == "P"

    def num_faces(self, a):
        """Distinct faces normal to axis a along that axis (periodic: face n == face 0)."""
        return self.n[a] if self.periodic(a) else self.n[a] + 1

    def face_shape(self, a):
        s = list(self.shape)
        s[a] = self.num_faces(a)
        return tuple(s)

    def cell_centres(self, a):
        """Coordinate along axis a of the cell centres: lo + (i + 1/2) h."""
        i = np.arange(self.n[a], dtype=np.float64)
        return self.lo[a] + (i + 0.5) * self.h[a]

    def face_coords(self, a, b):
        """Coordinate along axis b of the faces normal to axis a."""
        if a == b:
            i = np.arange(self.num_faces(a), dtype=np.float64)
            return self.lo[a] + i * self.h[a]
        return self.cell_centres(b)

    def face_points(self, a):
        """All face centres normal to axis a, shape (num, dim), in C order of face_shape(a)."""
        axes = [self.face_coords(a, b) for b in range(self.dim)]
        mesh = np.meshgrid(*axes, indexing="ij")
        return np.stack([m.ravel() for m in mesh], axis=1)

    def cell_points(self):
        axes = [self.cell_centres(b) for b in range(self.dim)]
        mesh = np.meshgrid(*axes, indexing="ij")
        return np.stack([m.ravel() for m in mesh], axis=1)

    def face_is_wall(self, a):
        """Boolean array over face_shape(a): True where the face is a wall (flux forced to 0)."""
        m = np.zeros(self.face_shape(a), dtype=bool)
        if not self.periodic(a):
            idx = [slice(None)] * self.dim
            if self.bc_lo[a] == "W":
                idx[a] = 0
                m[tuple(idx)] = True
            if self.bc_hi[a] == "W":
                idx[a] = self.n[a]
                m[tuple(idx)] = True
        return m

    def singular(self):
        """True when the Laplacian has a constant null space (no Dirichlet face anywhere)."""
        return all(self.bc_lo[a] != "D" and self.bc_hi[a] != "D" for a in range(self.dim))


def _ghost_pad(p, g, a):
    """Pad p by one ghost layer on each side of axis a with the ghost rules above."""
    first = np.take(p, [0], axis=a)
    last = np.take(p, [p.shape[a] - 1], axis=a)
    if g.periodic(a):
        lo_ghost, hi_ghost = last, first
    else:
        lo_ghost = -first if g.bc_lo[a] == "D" else first
        hi_ghost = -last if g.bc_hi[a] == "D" else last
    return np.concatenate([lo_ghost, p, hi_ghost], axis=a)


def laplacian(p, g):
    """L_h p: sum over axes of (p_{j-1} - 2 p_j + p_{j+1}) / h_a^2 with the ghost rules."""
    out = np.zeros_like(p)
    for a in range(g.dim):
        q = _ghost_pad(p, g, a)
        n = p.shape[a]
        left = np.take(q, range(0, n), axis=a)
        mid = np.take(q, range(1, n + 1), axis=a)
        right = np.take(q, range(2, n + 2), axis=a)
        out += (left - 2.0 * mid + right) / (g.h[a] * g.h[a])
    return out


# Error-free transformations for a compensated residual (Knuth's TwoSum; Dekker's splitting
# and product, 1971). numpy evaluates each elementwise operation separately (no fused
# multiply-add), as these algorithms require.
def _two_sum(a, b):
    s = a + b
    z = s - a
    return s, (a - (s - z)) + (b - z)


_DEKKER = 134217729.0          # 2^27 + 1


def _split(x):
    t = _DEKKER * x
    hi = t - (t - x)
    return hi, x - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _dd_add(ah, al, bh, bl):
    s, e = _two_sum(ah, bh)
    e = e + (al + bl)
    h = s + e
    return h, e - (h - s)


def _dd_div(ah, al, b):
    q = ah / b
    p, e = _two_prod(q, b)
    r = ((ah - p) - e + al) / b
    h = q + r
    return h, r - (h - q)


def residual_compensated(s, p, g):
    """s - L_h p in double-double arithmetic (about 106 significant bits), rounded to FP64.

    Same operator as laplacian(): (p_{j-1} - 2 p_j + p_{j+1}) / (h_a h_a) per axis with the
    ghost rules; only the arithmetic differs."""
    rh = np.array(s, dtype=np.float64, copy=True)
    rl = np.zeros_like(rh)
    for a in range(g.dim):
        q = _ghost_pad(p, g, a)
        n = p.shape[a]
        left = np.take(q, range(0, n), axis=a)
        mid = np.take(q, range(1, n + 1), axis=a)
        right = np.take(q, range(2, n + 2), axis=a)
        th, tl = _two_sum(left, right)
        th, tl = _dd_add(th, tl, -2.0 * mid, np.zeros_like(mid))
        th, tl = _dd_div(th, tl, g.h[a] * g.h[a])
        rh, rl = _dd_add(rh, rl, -th, -tl)
    return rh + rl


def face_gradient(p, g, a):
    """G_h p on the faces normal to axis a: (p_right - p_left)/h_a using the ghost rules.

    Wall and inflow faces get 0 (homogeneous Neumann, Eq. 7), Dirichlet faces
    (p_0 - (-p_0))/h at the low end and (-p_{n-1} - p_{n-1})/h at the high end."""
    q = _ghost_pad(p, g, a)
    n = p.shape[a]
    if g.periodic(a):
        left = np.take(q, range(0, n), axis=a)      # face i sits between cells i-1 and i
        right = np.take(q, range(1, n + 1), axis=a)
    else:
        left = np.take(q, range(0, n + 1), axis=a)
        right = np.take(q, range(1, n + 2), axis=a)
    return (right - left) / g.h[a]


def divergence(faces, g):
    """D_h U: sum over axes of (U(i+1/2) - U(i-1/2)) / h_a, one value per cell."""
    out = np.zeros(g.shape)
    for a in range(g.dim):
        U = faces[a]
        n = g.n[a]
        lo = np.take(U, range(0, n), axis=a)
        if g.periodic(a):
            hi = np.take(U, [(i + 1) % n for i in range(n)], axis=a)
        else:
            hi = np.take(U, range(1, n + 1), axis=a)
        out += (hi - lo) / g.h[a]
    return out
