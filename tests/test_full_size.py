"""GPU parity at the full sizes of the measured workloads, through the C ABI.

The channel workload also runs on the vertex grid (one pass and the IB iteration against the
oracle's vertex pass) and through the AB2 predictor (two steps against the oracle); vertex
solves run at the largest axes the vertex transforms take.

Channel with cylinder, 1024x512 cells, ~4.0e5 nodes (the benchmark workload): the oracle runs
the whole projection, and the IB-force iteration at tolerance 1e-3, so p, u and f are compared
element by element (FP64 1e-12, mixed 1e-10 relative L2).

Box with sphere, 256x128x128 cells, ~4.3e6 nodes, K = 27: the oracle's neighbour search and
WLS setup for 1.3e7 face rows would take minutes, so the comparison is split:
  - the transform solve on the full grid against the oracle's separable eigen-solve;
  - WLS rows at sampled faces and nodes (columns bit-exact, weights within the kappa bound);
  - the corrected velocity at sampled nodes from the oracle's rows applied to the GPU pressure;
  - the source at sampled cells: the oracle's transfer and divergence there against
    L_h p + removed mean of the GPU solution (1e-9 of max|s|: a direct FP64 solve on this grid,
    kappa(L_h) ~ 1e5, leaves residuals near 1e-11);
  - mixed against FP64 on the whole field (p to 1e-10; u and f are stored in FP32 like u*, so
    to FP32 rounding), and the divergence after projection.
"""
import numpy as np
import pytest

from oracle import grid as G
from oracle import knn as KNN
from oracle import poisson as P
from oracle import projection as PR
from paper_2304_14690_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ULP = np.finfo(np.float64).eps


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def grid_of(p):
    return G.Grid(p.dim, p.n, p.lo, p.h, p.bc_lo, p.bc_hi)


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc
    assert torch.cuda.is_available()
    return pc, torch, torch.device("cuda", 0)


@pytest.fixture(scope="module")
def channel():
    prob = wl.channel_cylinder()
    return prob, PR.build_plan(grid_of(prob), prob.nodes, prob.node_type, K=prob.knn)


def test_channel_full_projection(env, channel):
    pc, torch, dev = env
    prob, oplan = channel
    ref = PR.project(oplan, prob.dt, prob.u_star)
    u = torch.as_tensor(prob.u_star, device=dev)
    got = {}
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-10)):
        plan = pc.Plan(prob, precision=precision)
        if precision == "mixed":
            plan.autotune()                   # the benchmark's launch configuration
        p, uo, fo, st = plan.project(u, stats=True)
        assert rel(p.cpu().numpy(), ref["p"]) <= tol, precision
        assert rel(uo.cpu().numpy(), ref["u"]) <= tol, precision
        assert rel(fo.cpu().numpy(), ref["f"]) <= tol, precision
        assert st["max_div_after"] * min(prob.h) / st["max_abs_u_star"] <= 1e-9
        got[precision] = p.cpu().numpy()
        plan.close()
    # The refinement reaches the floor of its double-float residual (about 2^-44 of the source):
    # mixed against the FP64 GPU path measured 4.5e-15 to 1.5e-14 on this grid.
    # 1e-13 keeps a margin and catches a residual or source whose rounding raises that floor
    # (a second difference formed as (p_l + p_r) - 2 p_c gave 9.4e-13).
    assert rel(got["mixed"], got["fp64"]) <= 1e-13


def test_channel_ib_iteration(env, channel):
    """The IB-force iteration at the paper's tolerance 1e-3 on the full channel (~2.4e4
    boundary/virtual nodes), in the launch configuration the benchmark times: same number of
    passes as the oracle (every pass ratio is far from the threshold), p, u, f element by element."""
    pc, torch, dev = env
    prob, oplan = channel
    ref = PR.project_ib(oplan, prob.dt, prob.u_star, tol=1e-3, max_iters=50)
    ratios = [d / p for d, p in ref["history"] if p > 0]
    assert all(abs(r / 1e-3 - 1.0) > 0.05 for r in ratios)
    u = torch.as_tensor(prob.u_star, device=dev)
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-10)):
        plan = pc.Plan(prob, precision=precision)
        if precision == "mixed":
            plan.autotune()
        p, uo, fo, info = plan.project_ib(u, tol=1e-3, max_iters=50)
        assert info["iterations"] == ref["iterations"] and info["converged"], precision
        assert rel(p.cpu().numpy(), ref["p"]) <= tol, precision
        assert rel(uo.cpu().numpy(), ref["u"]) <= tol, precision
        assert rel(fo.cpu().numpy(), ref["f"]) <= tol, precision
        plan.close()


def test_channel_vertex_projection(env, channel):
    """The channel workload on the regular (vertex) pressure grid (1024 x 513 unknowns, N-D by
    N-N: quarter-wave and DCT-I transforms), in the benchmark's launch configuration:
    one pass against the oracle's vertex pass, p, u, f element by element."""
    from oracle import vertex as V
    pc, torch, dev = env
    prob, _ = channel
    vpl = V.build_plan(grid_of(prob), prob.nodes, prob.node_type, K=prob.knn)
    ref = V.project(vpl, prob.dt, prob.u_star)
    u = torch.as_tensor(prob.u_star, device=dev)
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-10)):
        plan = pc.Plan(prob, precision=precision, div_mode="wls_direct", grid_type="vertices")
        if precision == "mixed":
            plan.autotune()
        p, uo, fo, _ = plan.project(u)
        assert p.shape == ref["p"].shape
        assert rel(p.cpu().numpy(), ref["p"]) <= tol, precision
        assert rel(uo.cpu().numpy(), ref["u"]) <= tol, precision
        assert rel(fo.cpu().numpy(), ref["f"]) <= tol, precision
        plan.close()


def test_channel_vertex_ib_iteration(env, channel):
    """The IB-force iteration at tolerance 1e-3 on the channel's vertex grid: same number of
    passes as the oracle, p, u, f element by element."""
    from oracle import vertex as V
    pc, torch, dev = env
    prob, _ = channel
    vpl = V.build_plan(grid_of(prob), prob.nodes, prob.node_type, K=prob.knn)
    ref = V.project_ib(vpl, prob.dt, prob.u_star, tol=1e-3, max_iters=50)
    ratios = [d / p for d, p in ref["history"] if p > 0]
    assert all(abs(r / 1e-3 - 1.0) > 0.05 for r in ratios)
    u = torch.as_tensor(prob.u_star, device=dev)
    plan = pc.Plan(prob, precision="mixed", div_mode="wls_direct", grid_type="vertices")
    plan.autotune()
    p, uo, fo, info = plan.project_ib(u, tol=1e-3, max_iters=50)
    assert info["iterations"] == ref["iterations"] and info["converged"]
    for got, want in ((p, ref["p"]), (uo, ref["u"]), (fo, ref["f"])):
        assert rel(got.cpu().numpy(), want) <= 1e-10
    plan.close()


def test_channel_predictor_full_size(env, channel):
    """The AB2 predictor on the channel's 398,401 nodes (K = 12) in the launch configuration of
    the bench's time step: two steps (Euler start, then AB2 with the recovered pressure
    gradient) against the oracle, the correction between them taken from the oracle."""
    from oracle import momentum as M
    pc, torch, dev = env
    prob, oplan = channel
    m_ref = M.build(grid_of(prob), prob.nodes, prob.node_type, K=12, nu=0.01)
    dt = 1e-4
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-10)):
        M.reset(m_ref)
        plan = pc.Plan(prob, precision=precision)
        mom = pc.Momentum(plan, nu=0.01)
        u = prob.u_star.copy()
        for step in range(2):
            want = M.predict(m_ref, dt, u)
            got = mom.predict(torch.as_tensor(u, device=dev), dt)
            assert rel(got.cpu().numpy(), want) <= tol, (precision, step)
            u = PR.project(oplan, dt, want)["u"]
        mom.close()
        plan.close()


@pytest.mark.parametrize("kinds", [(("I", "D"), ("W", "W")), (("D", "W"), ("P", "P"))])
def test_vertex_solve_maximum_sizes(env, kinds):
    """Vertex-grid solves at the largest axes the vertex transforms take: a 4096-cell N-D or D-N
    axis (quarter-wave pair, FFT of 2048) with a 2048-cell N-N axis (DCT-I, FFT of 2048 on the
    even extension) or a 1024-cell P-P axis, against the oracle's DCT-I / quarter-wave expansion."""
    from oracle import vertex as V
    pc, torch, dev = env
    (lo0, hi0), (lo1, hi1) = kinds
    n = (4096, 2048) if lo1 != "P" else (4096, 1024)
    h = (1.0 / n[0], 1.0 / n[1])
    lo, hi = (lo0, lo1), (hi0, hi1)
    shape = tuple(V.unknowns(V.axis_kind(lo[a], hi[a]), n[a])[0] for a in range(2))
    s = np.random.default_rng(17).normal(size=shape)
    ref, _ = V.solve(s, n, h, lo, hi)
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-10)):
        plan = pc.GridPlan(2, n, h, lo, hi, grid_type="vertices", precision=precision)
        p, _ = plan.solve_poisson(torch.as_tensor(s, device=dev))
        assert rel(p.cpu().numpy(), ref) <= tol, (kinds, precision)
        plan.close()


@pytest.fixture(scope="module")
def box(env):
    pc, torch, dev = env
    prob = wl.box_sphere()
    g = grid_of(prob)
    p64 = pc.Plan(prob, precision="fp64")
    pmx = pc.Plan(prob, precision="mixed")
    pmx.autotune()
    u = torch.as_tensor(prob.u_star, device=dev)
    r64 = p64.project(u, stats=True)
    rmx = pmx.project(u, stats=True)
    yield prob, g, p64, pmx, r64, rmx
    p64.close()
    pmx.close()


def test_box_transform_solve(env, box):
    pc, torch, dev = env
    prob, g, p64, pmx, _, _ = box
    s = np.random.default_rng(2024).normal(size=g.shape)
    ref, _ = P.solve(s, g)
    sd = torch.as_tensor(s, device=dev)
    assert rel(p64.solve_poisson(sd)[0].cpu().numpy(), ref) <= 1e-12
    assert rel(pmx.solve_poisson(sd)[0].cpu().numpy(), ref) <= 1e-10


def _sample_rows_kappa(points, queries, idx, g):
    delta = points[idx] - queries[:, None, :]
    from oracle import wls as W
    d2 = KNN.squared_distance(delta)
    hs = W.support_radius(d2.max(axis=1), idx.shape[1], g.dim, 3.0)
    w = W.gaussian_weight(d2, hs[:, None], 6.3)
    q = W.basis(delta / hs[:, None, None])
    return np.linalg.cond(np.einsum("qk,qki,qkj->qij", w, q, q))


def test_box_sampled_rows(env, box):
    prob, g, p64, _, _, _ = box
    rng = np.random.default_rng(7)
    pts = prob.nodes.T.copy()
    lo, lengths, periodic = list(g.lo[:3]), [g.length(a) for a in range(3)], [False] * 3
    # face rows of axis 0 at sampled non-wall faces
    fp = g.face_points(0)
    wall = g.face_is_wall(0).ravel()
    cand = np.flatnonzero(~wall)
    sel = rng.choice(cand, 2048, replace=False)
    idx, _ = KNN.knn(pts, fp[sel], prob.knn, lo, lengths, periodic)
    val, _ = PR._wls_block(pts, fp[sel], idx, g, 6.3, 3.0)
    col, w = p64.rows(0)
    assert np.array_equal(col[sel], idx)
    kap = _sample_rows_kappa(pts, fp[sel], idx, g)
    tol = 64 * ULP * kap[:, None] * np.abs(val).max(axis=1, keepdims=True)
    assert np.all(np.abs(w[sel] - val) <= tol)
    # node derivative rows at sampled nodes
    nsel = rng.choice(prob.num_nodes, 2048, replace=False)
    cidx = PR.gradient_block(g, pts[nsel])
    _, grad = PR._wls_block(g.cell_points(), pts[nsel], cidx, g, 6.3, 3.0)
    col, D = p64.rows(prob.dim)
    assert np.array_equal(col[nsel], cidx)
    kap = _sample_rows_kappa(g.cell_points(), pts[nsel], cidx, g)
    Dref = np.transpose(grad, (1, 0, 2))                          # (d, Q, 27)
    tol = 64 * ULP * kap[None, :, None] * np.abs(Dref).max(axis=2, keepdims=True)
    assert np.all(np.abs(D[:, nsel, :] - Dref) <= tol)


def test_box_sampled_correction(env, box):
    """u = u* - beta dt g at sampled nodes, g from the oracle's rows on the GPU pressure."""
    prob, g, _, _, r64, _ = box
    p = r64[0].cpu().numpy()
    uo = r64[1].cpu().numpy()
    rng = np.random.default_rng(8)
    pts = prob.nodes.T.copy()
    nsel = rng.choice(np.flatnonzero(prob.node_type == 0), 4096, replace=False)
    cidx = PR.gradient_block(g, pts[nsel])
    _, grad = PR._wls_block(g.cell_points(), pts[nsel], cidx, g, 6.3, 3.0)   # (Q, d, 27)
    gn = np.einsum("qak,qk->aq", grad, p.ravel()[cidx])
    ref = prob.u_star[:, nsel].astype(np.float64) - 1.5 * prob.dt * gn
    # u is stored in the input's dtype (FP32 here): compare to FP32 rounding
    tol = 1e-12 if uo.dtype == np.float64 else 2.0 ** -23
    assert rel(uo[:, nsel], ref) <= tol
    ib = np.flatnonzero(prob.node_type != 0)
    assert np.all(uo[:, ib] == 0.0)


def test_box_sampled_source(env, box):
    """At sampled cells: the oracle's source (its own face rows and u*) equals L_h p + removed
    mean of the GPU FP64 solution (the solve is direct, so this holds to round-off)."""
    prob, g, _, _, r64, _ = box
    p = r64[0].cpu().numpy()
    removed = r64[3]["removed_mean"]
    rng = np.random.default_rng(9)
    shape = g.shape
    cells = np.stack([rng.integers(0, shape[a], 1024) for a in range(3)], axis=1)
    pts = prob.nodes.T.copy()
    lo, lengths, periodic = list(g.lo[:3]), [g.length(a) for a in range(3)], [False] * 3
    ut = prob.u_star.astype(np.float64)
    s = np.zeros(len(cells))
    for a in range(3):
        fs = g.face_shape(a)
        walls = g.face_is_wall(a)
        for side in (0, 1):
            fi = cells.copy()
            fi[:, a] += side
            lin = np.ravel_multi_index(fi.T, fs)
            fp = g.face_points(a)[lin]
            idx, _ = KNN.knn(pts, fp, prob.knn, lo, lengths, periodic)
            val, _ = PR._wls_block(pts, fp, idx, g, 6.3, 3.0)
            U = np.sum(val * ut[a][idx], axis=1)
            U[walls.ravel()[lin]] = 0.0
            s += (U if side else -U) / g.h[a]
    s /= 1.5 * prob.dt
    lap = G.laplacian(p, g)[tuple(cells.T)]
    assert np.max(np.abs(lap + removed - s)) <= 1e-9 * np.max(np.abs(s))


def test_box_mixed_vs_fp64(env, box):
    prob, _, _, _, r64, rmx = box
    assert rel(rmx[0].cpu().numpy(), r64[0].cpu().numpy()) <= 1e-10
    for i in (1, 2):                  # u, f in FP32 storage: equal up to FP32 rounding
        assert rel(rmx[i].cpu().numpy(), r64[i].cpu().numpy()) <= 2.0 ** -23
    st = rmx[3]
    assert st["max_div_after"] * min(prob.h) / st["max_abs_u_star"] <= 1e-9
