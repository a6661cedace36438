"""Seeded synthetic inputs shaped like the paper's test cases.

This module only draws inputs: node clouds (velocity, boundary and virtual points of the
double discretization in §2.3), node types, provisional velocities and grid descriptions.
It holds none of the method's arithmetic, so both the CUDA path and the CPU oracle may use
it. Every generator is deterministic in its seed.

Workloads (sizes follow the paper's cases: 2D grids of a few hundred cells per axis, node
clouds of ~1e5 points refined near obstacles, §3.1-§3.4):
  periodic_taylor_green   2D periodic [0,2pi]^2, 64x64 cells, 4096 jittered nodes,
                          Taylor-Green velocity plus a gradient perturbation.
  channel_cylinder        2D channel [0,20]x[0,10], 1024x512 cells, inflow/outflow in x,
                          walls in y, cylinder D=1 at (5,5), ~4e5 nodes refined radially.
  box_sphere              3D box [0,8]x[0,4]x[0,4], 256x128x128 cells, walls everywhere,
                          sphere D=1 at (2,2,2), ~4.2e6 nodes, random-field velocity (FP32).
  batch_2d                512 independent 2D problems of mixed sizes and boundary types.
  generic                 parametric builder used by the tests for small cases.
"""
from dataclasses import dataclass, field
import math
import numpy as np

FLUID, BOUNDARY, VIRTUAL = 0, 1, 2
BC_CODES = {"P": 0, "W": 1, "I": 2, "D": 3}


@dataclass
class Problem:
    name: str
    dim: int
    n: tuple
    lo: tuple
    h: tuple
    bc_lo: tuple
    bc_hi: tuple
    nodes: np.ndarray            # (dim, N) float64, structure of arrays
    node_type: np.ndarray        # (N,) uint8: 0 fluid, 1 boundary, 2 virtual
    u_star: np.ndarray           # (dim, N) float64 or float32
    f_ib: np.ndarray = None      # (dim, N) or None
    dt: float = 1.0
    beta: float = 1.5
    knn: int = 12
    eps: float = 6.3
    support_factor: float = 3.0
    obstacles: list = field(default_factory=list)   # (kind, centre tuple, radius)

    def __post_init__(self):
        # dense structure-of-arrays layout, as the C ABI expects
        self.nodes = np.ascontiguousarray(self.nodes, dtype=np.float64)
        self.node_type = np.ascontiguousarray(self.node_type, dtype=np.uint8)
        self.u_star = np.ascontiguousarray(self.u_star)
        if self.f_ib is not None:
            self.f_ib = np.ascontiguousarray(self.f_ib, dtype=self.u_star.dtype)

    @property
    def num_nodes(self):
        return int(self.nodes.shape[1])

    @property
    def num_cells(self):
        return int(np.prod(self.n[: self.dim]))

    def lengths(self):
        return tuple(float(self.n[a]) * float(self.h[a]) for a in range(self.dim))


# ----------------------------------------------------------------------------- helpers

def jittered_lattice(lo, lengths, spacing, jitter, rng):
    """Points at the centres of a lattice of the given spacing, moved by U(-j, j) * spacing."""
    dim = len(lo)
    counts = [max(1, int(round(lengths[a] / spacing))) for a in range(dim)]
    axes = [lo[a] + (np.arange(counts[a]) + 0.5) * (lengths[a] / counts[a]) for a in range(dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([m.ravel() for m in mesh], axis=0)
    pts = pts + rng.uniform(-jitter, jitter, size=pts.shape) * spacing
    return pts


def _inside_box(pts, lo, lengths, margin):
    ok = np.ones(pts.shape[1], dtype=bool)
    for a in range(pts.shape[0]):
        ok &= (pts[a] > lo[a] + margin) & (pts[a] < lo[a] + lengths[a] - margin)
    return ok


def _wrap(pts, lo, lengths, periodic):
    for a, per in enumerate(periodic):
        if per:
            pts[a] = lo[a] + np.mod(pts[a] - lo[a], lengths[a])
    return pts


def circle_points(centre, radius, spacing, rng):
    m = max(8, int(round(2.0 * math.pi * radius / spacing)))
    th = rng.uniform(0.0, 2.0 * math.pi) + 2.0 * math.pi * np.arange(m) / m
    return np.stack([centre[0] + radius * np.cos(th), centre[1] + radius * np.sin(th)])


def sphere_points(centre, radius, spacing, rng):
    """Fibonacci-spiral points on a sphere at roughly the given spacing, randomly rotated."""
    m = max(12, int(round(4.0 * math.pi * radius * radius / (spacing * spacing))))
    i = np.arange(m) + 0.5
    z = 1.0 - 2.0 * i / m
    r = np.sqrt(1.0 - z * z)
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i + rng.uniform(0, 2 * math.pi)
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), z])
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    pts = q @ pts
    return np.asarray(centre, dtype=np.float64)[:, None] + radius * pts


def lamb_oseen(pts, centres, gammas, cores):
    """Sum of 2D Lamb-Oseen vortices u_theta = G/(2 pi r) (1 - exp(-r^2/rc^2))."""
    u = np.zeros_like(pts[:2])
    for (cx, cy), G, rc in zip(centres, gammas, cores):
        dx, dy = pts[0] - cx, pts[1] - cy
        r2 = dx * dx + dy * dy
        small = r2 < 1e-12 * rc * rc
        fac = np.where(small, G / (2 * math.pi * rc * rc),
                       G / (2 * math.pi * np.where(small, 1.0, r2)) * (1 - np.exp(-r2 / (rc * rc))))
        u[0] += -fac * dy
        u[1] += fac * dx
    return u


def gaussian_gradient(pts, lo, lengths, periodic, rng, count=8, sigma=0.5):
    """Gradient of phi = sum_m a_m exp(-|x-c_m|^2/(2 sigma^2)) (minimum image on periodic axes)."""
    dim = pts.shape[0]
    g = np.zeros_like(pts)
    for _ in range(count):
        a = rng.choice([-1.0, 1.0])
        c = np.array([rng.uniform(lo[k], lo[k] + lengths[k]) for k in range(dim)])
        d = pts - c[:, None]
        for k in range(dim):
            if periodic[k]:
                L = lengths[k]
                d[k] = d[k] - L * np.round(d[k] / L)
        e = np.exp(-np.sum(d * d, axis=0) / (2 * sigma * sigma))
        g += -a * d / (sigma * sigma) * e
    return g


def _obstacle_cloud(dim, lo, lengths, periodic, spacing, obstacles, rng, jitter=0.3,
                    bnd_spacing=None):
    """Jittered lattice with obstacles: inside -> virtual, surface -> boundary points."""
    pts = jittered_lattice(lo, lengths, spacing, jitter, rng)
    pts = _wrap(pts, lo, lengths, periodic)
    keep = np.ones(pts.shape[1], dtype=bool)
    for a in range(dim):
        if not periodic[a]:
            keep &= (pts[a] > lo[a]) & (pts[a] < lo[a] + lengths[a])
    pts = pts[:, keep]
    types = np.zeros(pts.shape[1], dtype=np.uint8)
    extra, extra_t = [], []
    bs = bnd_spacing or spacing
    for kind, c, R in obstacles:
        r = np.sqrt(np.sum((pts - np.asarray(c)[:, None]) ** 2, axis=0))
        band = np.abs(r - R) < 0.5 * spacing
        types[r < R] = VIRTUAL
        pts, types = pts[:, ~band], types[~band]
        surf = circle_points(c, R, bs, rng) if dim == 2 else sphere_points(c, R, bs, rng)
        extra.append(surf)
        extra_t.append(np.full(surf.shape[1], BOUNDARY, dtype=np.uint8))
    if extra:
        pts = np.concatenate([pts] + extra, axis=1)
        types = np.concatenate([types] + extra_t)
    return pts, types


# ----------------------------------------------------------------------------- workloads

def generic(dim=2, n=(32, 32, 32), h=None, lo=(0.0, 0.0, 0.0), bc_lo=("P", "P", "P"),
            bc_hi=("P", "P", "P"), spacing_factor=1.0, obstacles=(), seed=0, knn=None,
            jitter=0.3, velocity="vortex", dtype=np.float64, with_force=False, dt=1.0):
    """Small parametric problem: jittered lattice, optional circular/spherical obstacles."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n[:dim])
    if h is None:
        h = tuple(1.0 / 16 for _ in range(dim))
    h = tuple(float(v) for v in h[:dim])
    lo = tuple(float(v) for v in lo[:dim])
    bc_lo, bc_hi = tuple(bc_lo[:dim]), tuple(bc_hi[:dim])
    lengths = tuple(n[a] * h[a] for a in range(dim))
    periodic = [b == "P" for b in bc_lo]
    spacing = spacing_factor * min(h)
    pts, types = _obstacle_cloud(dim, lo, lengths, periodic, spacing, list(obstacles), rng,
                                 jitter=jitter)
    u = _velocity(pts, types, lo, lengths, periodic, rng, velocity)
    f = None
    if with_force:
        f = np.zeros_like(u)
        ib = types != FLUID
        f[:, ib] = rng.normal(size=(dim, int(ib.sum())))
    return Problem("generic", dim, n, lo, h, bc_lo, bc_hi, pts, types, u.astype(dtype),
                   None if f is None else f.astype(dtype), dt=dt,
                   knn=knn or (12 if dim == 2 else 27), obstacles=list(obstacles))


def _velocity(pts, types, lo, lengths, periodic, rng, kind):
    dim = pts.shape[0]
    if kind == "vortex":
        u = np.zeros_like(pts)
        u[0] += 1.0
        nv = 6
        centres = [tuple(rng.uniform(lo[k], lo[k] + lengths[k]) for k in range(2)) for _ in range(nv)]
        gam = rng.uniform(0.5, 1.0, nv) * rng.choice([-1, 1], nv)
        core = rng.uniform(0.1, 0.3, nv) * min(lengths[:2])
        u[:2] += lamb_oseen(pts, centres, gam, core)
        if dim == 3:
            u[2] += 0.3 * np.sin(2 * math.pi * (pts[0] - lo[0]) / lengths[0])
        gp = gaussian_gradient(pts, lo, lengths, periodic, rng, count=4,
                               sigma=0.15 * min(lengths))
        u += 0.2 * gp / max(1e-300, np.abs(gp).max())
    elif kind == "random":
        u = rng.normal(size=pts.shape)
    else:
        raise ValueError(kind)
    u[:, types == VIRTUAL] = 0.0
    return u


def periodic_taylor_green(n=64, seed=14690):
    """2D periodic [0,2pi]^2, n x n cells, n^2 nodes at cell centres jittered by +-0.3h.

    u* = Taylor-Green (sin x cos y, -cos x sin y) + 0.1 grad(phi)/max|grad(phi)|, phi a sum of
    8 periodic Gaussians of width 0.5 with random signs and centres."""
    rng = np.random.default_rng(seed)
    L = 2.0 * math.pi
    h = L / n
    pts = jittered_lattice((0.0, 0.0), (L, L), h, 0.3, rng)
    pts = _wrap(pts, (0.0, 0.0), (L, L), [True, True])
    x, y = pts
    u = np.stack([np.sin(x) * np.cos(y), -np.cos(x) * np.sin(y)])
    gp = gaussian_gradient(pts, (0.0, 0.0), (L, L), [True, True], rng, count=8, sigma=0.5)
    u = u + 0.1 * gp / np.abs(gp).max()
    types = np.zeros(pts.shape[1], dtype=np.uint8)
    return Problem("periodic_taylor_green", 2, (n, n), (0.0, 0.0), (h, h), ("P", "P"),
                   ("P", "P"), pts, types, u)


def _channel_rings(g, R0, s0, s_cap, rng, outward):
    """Concentric rings around the cylinder; spacing s0 * g^m capped at s_cap."""
    rings = []
    r, s = R0, s0
    while s < s_cap:
        r = r + s if outward else r - s
        if r <= 0.5 * s:
            break
        rings.append((r, s))
        s = s * g
    return rings, r


def channel_cylinder(nx=1024, ny=512, target_nodes=400000, seed=14691):
    """2D channel [0,20]x[0,10] with a cylinder of diameter 1 at (5,5).

    x: Neumann inflow at x=0, homogeneous Dirichlet outflow at x=20; y: walls.
    Nodes: 628 boundary points on the circle (spacing 0.005), concentric rings outside and
    inside the circle with spacing 0.005 g^m (capped at 0.04, g found by bisection so that
    the total is within 1% of target_nodes), a jittered lattice of spacing 0.04 beyond the
    rings (fluid) and inside them (virtual). u* = (1, 0) + 32 Lamb-Oseen vortices
    (|Gamma| in [0.5, 1], core 0.2-0.5), 0 on virtual nodes."""
    Lx, Ly = 20.0, 10.0
    c, R = (5.0, 5.0), 0.5
    s0, cap = 0.005, 0.04

    def build(g, rng):
        out_rings, r_out = _channel_rings(g, R, s0, cap, rng, True)
        in_rings, r_in = _channel_rings(g, R, s0, cap, rng, False)
        parts, types = [], []
        bnd = circle_points(c, R, s0, rng)
        parts.append(bnd)
        types.append(np.full(bnd.shape[1], BOUNDARY, np.uint8))
        for rings, t in ((out_rings, FLUID), (in_rings, VIRTUAL)):
            for rr, s in rings:
                p = circle_points(c, rr, s, rng)
                parts.append(p)
                types.append(np.full(p.shape[1], t, np.uint8))
        lat = jittered_lattice((0.0, 0.0), (Lx, Ly), cap, 0.3, rng)
        rl = np.sqrt((lat[0] - c[0]) ** 2 + (lat[1] - c[1]) ** 2)
        far = rl > r_out + 0.5 * cap
        near_in = rl < r_in - 0.5 * cap
        parts += [lat[:, far], lat[:, near_in]]
        types += [np.full(int(far.sum()), FLUID, np.uint8), np.full(int(near_in.sum()), VIRTUAL, np.uint8)]
        pts = np.concatenate(parts, axis=1)
        typ = np.concatenate(types)
        ok = _inside_box(pts, (0.0, 0.0), (Lx, Ly), 0.25 * s0)
        return pts[:, ok], typ[ok]

    lo_g, hi_g = 1.0005, 1.2
    for _ in range(40):
        mid = 0.5 * (lo_g + hi_g)
        pts, _ = build(mid, np.random.default_rng(seed))
        if pts.shape[1] > target_nodes:
            lo_g = mid
        else:
            hi_g = mid
        if abs(pts.shape[1] - target_nodes) < 0.01 * target_nodes:
            break
    rng = np.random.default_rng(seed)
    pts, types = build(mid, rng)
    vr = np.random.default_rng(seed + 1000)
    centres = []
    while len(centres) < 32:
        p = (vr.uniform(0, Lx), vr.uniform(0, Ly))
        if (p[0] - c[0]) ** 2 + (p[1] - c[1]) ** 2 > (R + 0.3) ** 2:
            centres.append(p)
    gam = vr.uniform(0.5, 1.0, 32) * vr.choice([-1.0, 1.0], 32)
    core = vr.uniform(0.2, 0.5, 32)
    u = lamb_oseen(pts, centres, gam, core)
    u[0] += 1.0
    u[:, types == VIRTUAL] = 0.0
    h = (Lx / nx, Ly / ny)
    return Problem("channel_cylinder", 2, (nx, ny), (0.0, 0.0), h, ("I", "W"), ("D", "W"),
                   pts, types, u, obstacles=[("circle", c, R)])


def box_sphere(n=(256, 128, 128), seed=14692, spectrum_kmax=64):
    """3D box [0,8]x[0,4]x[0,4], walls on all six faces, sphere D=1 at (2,2,2).

    Nodes: jittered lattice at the grid spacing h (virtual inside the sphere), boundary points
    on the sphere at spacing h/2, three fluid shells and two virtual shells at h/2 steps.
    u*: Gaussian random field with E(k) ~ k^(-5/3) for 1 <= |k| <= kmax, independent
    components, normalised to RMS 1, zero on virtual nodes, stored as float32."""
    rng = np.random.default_rng(seed)
    L = (8.0, 4.0, 4.0)
    h = tuple(L[a] / n[a] for a in range(3))
    hm = min(h)
    c, R = (2.0, 2.0, 2.0), 0.5
    lat = jittered_lattice((0.0, 0.0, 0.0), L, hm, 0.3, rng)
    r = np.sqrt(np.sum((lat - np.asarray(c)[:, None]) ** 2, axis=0))
    band = (r > R - 1.25 * hm) & (r < R + 1.75 * hm)
    lat_t = np.where(r < R, VIRTUAL, FLUID).astype(np.uint8)
    parts, types = [lat[:, ~band]], [lat_t[~band]]
    for m, t in ((0, BOUNDARY), (1, FLUID), (2, FLUID), (3, FLUID), (-1, VIRTUAL), (-2, VIRTUAL)):
        p = sphere_points(c, R + m * 0.5 * hm, 0.5 * hm, rng)
        parts.append(p)
        types.append(np.full(p.shape[1], t, np.uint8))
    pts = np.concatenate(parts, axis=1)
    typ = np.concatenate(types)
    ok = _inside_box(pts, (0.0, 0.0, 0.0), L, 1e-6)
    pts, typ = pts[:, ok], typ[ok]
    u = _random_field(pts, (0.0, 0.0, 0.0), L, n, spectrum_kmax, rng)
    u[:, typ == VIRTUAL] = 0.0
    return Problem("box_sphere", 3, tuple(n), (0.0, 0.0, 0.0), h, ("W", "W", "W"),
                   ("W", "W", "W"), pts, typ, u.astype(np.float32), knn=27,
                   obstacles=[("sphere", c, R)])


def _random_field(pts, lo, L, n, kmax, rng):
    """Three independent periodic Gaussian fields with E(k) ~ k^(-5/3), sampled trilinearly."""
    dim = len(n)
    ks = [np.fft.fftfreq(n[a]) * n[a] for a in range(dim)]
    K = np.sqrt(sum(np.meshgrid(*[k * k for k in ks], indexing="ij")))
    Ks = np.where(K >= 1, K, 1.0)
    amp = np.where((K >= 1) & (K <= kmax), Ks ** (-5.0 / 6.0 - (dim - 1) / 2.0), 0.0)
    out = []
    for _ in range(dim):
        noise = rng.normal(size=tuple(n)) + 1j * rng.normal(size=tuple(n))
        f = np.real(np.fft.ifftn(noise * amp))
        f = f / np.sqrt(np.mean(f * f))
        out.append(f)
    # trilinear sampling at node positions (periodic wrap of the field)
    u = np.zeros((dim, pts.shape[1]))
    idx = []
    fr = []
    for a in range(dim):
        x = (pts[a] - lo[a]) / (L[a] / n[a]) - 0.5
        i0 = np.floor(x).astype(np.int64)
        idx.append(i0)
        fr.append(x - i0)
    for corner in range(1 << dim):
        wgt = np.ones(pts.shape[1])
        ii = []
        for a in range(dim):
            b = (corner >> a) & 1
            wgt = wgt * (fr[a] if b else 1.0 - fr[a])
            ii.append(np.mod(idx[a] + b, n[a]))
        for c in range(dim):
            u[c] += wgt * out[c][tuple(ii)]
    return u


BATCH_SIZES = (64, 96, 128, 192, 256, 384, 512)


def batch_2d(count=512, seed=14693, sizes=BATCH_SIZES):
    """Independent 2D problems: n0, n1 drawn from sizes, h = 1/64, BC pair from
    {periodic-periodic, periodic x / walls y, walls-walls}, nodes = jittered lattice at h,
    0-2 non-overlapping circles of diameter 5-15% of the shorter side, u* vortices plus a
    gradient perturbation."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        n0, n1 = int(rng.choice(sizes)), int(rng.choice(sizes))
        h = 1.0 / 64
        kind = int(rng.integers(0, 3))
        if kind == 0:
            bl, bh = ("P", "P"), ("P", "P")
        elif kind == 1:
            bl, bh = ("P", "W"), ("P", "W")
        else:
            bl, bh = ("W", "W"), ("W", "W")
        L0, L1 = n0 * h, n1 * h
        nob = int(rng.integers(0, 3))
        obs = []
        tries = 0
        while len(obs) < nob and tries < 100:
            tries += 1
            D = rng.uniform(0.05, 0.15) * min(L0, L1)
            Rr = 0.5 * D
            cc = (rng.uniform(Rr + 4 * h, L0 - Rr - 4 * h), rng.uniform(Rr + 4 * h, L1 - Rr - 4 * h))
            if all((cc[0] - o[1][0]) ** 2 + (cc[1] - o[1][1]) ** 2 > (Rr + o[2] + 4 * h) ** 2 for o in obs):
                obs.append(("circle", cc, Rr))
        p = generic(dim=2, n=(n0, n1), h=(h, h), bc_lo=bl, bc_hi=bh, obstacles=obs,
                    seed=int(rng.integers(0, 2**31)))
        p.name = f"batch_{i}"
        probs.append(p)
    return probs


SERVE_SIZES_2D = (128, 192, 256, 384, 512, 768, 1024)
SERVE_SIZES_3D = (64, 96, 128, 192)


def serving_pool(count=64, seed=14695, frac_2d=0.7, sizes_2d=SERVE_SIZES_2D, sizes_3d=SERVE_SIZES_3D):
    """Geometries of the request stream: 2D n x n (h = 1/n, inflow/outflow along x, walls
    along y, one cylinder) or 3D n^3 (h = 1/n, walls, one sphere) with n drawn uniformly from
    the size lists; obstacle diameter 10-30% of the box, centre inside it; nodes on a jittered
    lattice at h; u* vortices plus a gradient perturbation."""
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(count):
        two = rng.uniform() < frac_2d
        dim = 2 if two else 3
        n = int(rng.choice(sizes_2d if two else sizes_3d))
        h = 1.0 / n
        D = rng.uniform(0.1, 0.3)
        c = tuple(float(rng.uniform(0.5 * D + 4 * h, 1.0 - 0.5 * D - 4 * h)) for _ in range(dim))
        obs = [("circle" if two else "sphere", c, 0.5 * D)]
        if two:
            bl, bh = ("I", "W"), ("D", "W")
        else:
            bl, bh = ("W", "W", "W"), ("W", "W", "W")
        p = generic(dim=dim, n=(n,) * dim, h=(h,) * dim, bc_lo=bl, bc_hi=bh, obstacles=obs,
                    seed=int(rng.integers(0, 2**31)))
        p.name = f"serve_{i}_{dim}d_{n}"
        pool.append(p)
    return pool


def serving_trace(count=20000, rate=2000.0, pool_size=64, seed=14696):
    """Poisson arrivals: (arrival seconds, geometry index, u* scale) per request, exponential
    gaps of mean 1/rate, geometry uniform over the pool, scale uniform in [0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    g = rng.integers(0, pool_size, size=count)
    s = rng.uniform(0.5, 1.5, size=count)
    return [(float(t[i]), int(g[i]), float(s[i])) for i in range(count)]
