"""The vertex ("regular") pressure grid of §2.3 (the grid of the §3.2 results) against the oracle.

Grid-only plans: the Poisson solve for every boundary pairing, and the cell-centred solve without
nodes. On the device the vertex solve runs one transform pass per axis on the unknowns (DCT-I and
DST-I through the real DFT of the even or odd extension of each line in shared memory, the
quarter-wave bases through the DCT-II / DST-II pair in the other order); the oracle expands in the
DCT-I / DST-I / quarter-wave eigenvectors with dense bases.

Vertex-grid projection plans: the WLS rows at the vertex unknowns and at the nodes, one pass, the
IB-force iteration, host arrays, clones and the RHS mask."""
import itertools

import numpy as np
import pytest

from oracle import grid as G
from oracle import poisson as P
from oracle import vertex as V

pytestmark = pytest.mark.gpu

KINDS = {"PP": ("P", "P"), "NN": ("W", "W"), "DD": ("D", "D"), "ND": ("I", "D"), "DN": ("D", "W")}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc
    assert torch.cuda.is_available()
    return pc, torch, torch.device("cuda", 0)


def _vertex_case(kinds, n, seed):
    dim = len(n)
    rng = np.random.default_rng(seed)
    h = tuple(rng.uniform(0.5, 2.0) / n[a] for a in range(dim))
    lo = tuple(KINDS[k][0] for k in kinds)
    hi = tuple(KINDS[k][1] for k in kinds)
    shape = tuple(V.unknowns(k, n[a])[0] for a, k in enumerate(kinds))
    return h, lo, hi, rng.normal(size=shape)


def _combos(dim):
    combos = list(itertools.product(list(KINDS), repeat=dim))
    return combos if dim == 2 else combos[::6]


@pytest.mark.parametrize("n", [(8, 8), (24, 20), (30, 16), (12, 10, 8), (6, 16, 10)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10), ("fp32", 1e-5)])
def test_vertex_poisson_matches_oracle(env, n, precision, tol):
    pc, torch, dev = env
    dim = len(n)
    for i, kinds in enumerate(_combos(dim)):
        h, lo, hi, s = _vertex_case(kinds, n, 3000 + i)
        ref, removed = V.solve(s, n, h, lo, hi)
        plan = pc.GridPlan(dim, n, h, lo, hi, grid_type="vertices", precision=precision)
        assert plan.shape == s.shape
        p, st = plan.solve_poisson(torch.as_tensor(s, device=dev), stats=True)
        e = rel(p.cpu().numpy(), ref)
        assert e <= tol, (kinds, n, precision, e)
        # the dropped zero-mode coefficient of the vertex problem (0 when a Dirichlet end exists)
        assert abs(st["removed_mean"] - removed) <= 1e-12 * (1 + np.abs(s).max()), (kinds, st["removed_mean"], removed)
        plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10), ("fp32", 1e-5)])
def test_vertex_odd_lengths(env, precision, tol):
    """DCT-I and DST-I axes of an odd number of cells (an FFT of odd length 15 or 25 on the
    extension, radices 3 and 5 only), and a quarter-wave axis of 30 cells (FFT of 15)."""
    pc, torch, dev = env
    cases = [((15, 25), ("NN", "DD")), ((25, 15), ("DD", "NN")), ((15, 15), ("NN", "NN")),
             ((30, 25), ("ND", "NN")), ((25, 30), ("DD", "DN")), ((15, 9, 25), ("NN", "DD", "NN"))]
    for i, (n, kinds) in enumerate(cases):
        h, lo, hi, s = _vertex_case(kinds, n, 8000 + i)
        ref, removed = V.solve(s, n, h, lo, hi)
        plan = pc.GridPlan(len(n), n, h, lo, hi, grid_type="vertices", precision=precision)
        p, st = plan.solve_poisson(torch.as_tensor(s, device=dev), stats=True)
        assert rel(p.cpu().numpy(), ref) <= tol, (kinds, n, precision, rel(p.cpu().numpy(), ref))
        assert abs(st["removed_mean"] - removed) <= 1e-12 * (1 + np.abs(s).max()), (kinds, st["removed_mean"], removed)
        plan.close()


def test_vertex_quarter_wave_odd_length_refused(env):
    """A quarter-wave axis runs a DCT-II/DST-II pair of its own length, which must be even."""
    pc, torch, dev = env
    with pytest.raises(pc.PcError) as e:
        pc.GridPlan(2, (15, 16), (0.1, 0.1), ("W", "W"), ("D", "W"), grid_type="vertices")
    assert e.value.status == 2


@pytest.mark.parametrize("n", [(24, 20), (10, 8, 12)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_vertex_spectral_matches_oracle(env, n, precision, tol):
    pc, torch, dev = env
    dim = len(n)
    for i, kinds in enumerate(_combos(dim)):
        h, lo, hi, s = _vertex_case(kinds, n, 4000 + i)
        ref, _ = V.solve(s, n, h, lo, hi, eigenvalues="spectral")
        plan = pc.GridPlan(dim, n, h, lo, hi, grid_type="vertices", precision=precision, eigenvalues="spectral")
        p, _ = plan.solve_poisson(torch.as_tensor(s, device=dev))
        e = rel(p.cpu().numpy(), ref)
        assert e <= tol, (kinds, n, precision, e)
        plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_vertex_corner_gauge(env, precision, tol):
    """The corner gauge fixes the first unknown at zero on problems with a zero mode."""
    pc, torch, dev = env
    n = (16, 12)
    for i, kinds in enumerate([("NN", "NN"), ("PP", "NN"), ("PP", "PP"), ("NN", "DD")]):
        h, lo, hi, s = _vertex_case(kinds, n, 5000 + i)
        ref, _ = V.solve(s, n, h, lo, hi, gauge="corner")
        plan = pc.GridPlan(2, n, h, lo, hi, grid_type="vertices", precision=precision, gauge=1)
        p, _ = plan.solve_poisson(torch.as_tensor(s, device=dev))
        p = p.cpu().numpy()
        assert rel(p, ref) <= tol, (kinds, rel(p, ref))
        if all(k in ("PP", "NN") for k in kinds):
            assert p[0, 0] == 0.0
        plan.close()


def test_vertex_host_arrays_match_device(env):
    """Host (pinned and pageable) source and solution arrays give the device result bit for bit."""
    pc, torch, dev = env
    n = (20, 24)
    kinds = ("ND", "DN")
    h, lo, hi, s = _vertex_case(kinds, n, 6000)
    plan = pc.GridPlan(2, n, h, lo, hi, grid_type="vertices", precision="mixed")
    p_dev, _ = plan.solve_poisson(torch.as_tensor(s, device=dev))
    p_dev = p_dev.cpu().numpy()
    for pin in (False, True):
        hs = torch.as_tensor(s.copy())
        hp = torch.empty(plan.shape, dtype=torch.float64)
        if pin:
            hs, hp = hs.pin_memory(), hp.pin_memory()
        p_host, _ = plan.solve_poisson(hs, hp)
        assert np.array_equal(p_host.numpy(), p_dev), pin
    plan.close()


def test_vertex_solution_satisfies_operator(env):
    """Independent of the oracle's expansion: the vertex-grid 5-point operator (ghost rules of
    each boundary pairing) applied to the device solution returns the source less its zero mode."""
    pc, torch, dev = env
    n = (32, 24)
    for i, kinds in enumerate(_combos(2)):
        h, lo, hi, s = _vertex_case(kinds, n, 7000 + i)
        plan = pc.GridPlan(2, n, h, lo, hi, grid_type="vertices", precision="fp64")
        p, st = plan.solve_poisson(torch.as_tensor(s, device=dev), stats=True)
        lap = V.laplacian(p.cpu().numpy(), list(kinds), h)
        want = s - st["removed_mean"]
        assert rel(lap, want) <= 1e-11, (kinds, rel(lap, want))
        plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_cell_grid_plan_matches_oracle(env, precision, tol):
    """A grid-only plan on the cell-centred grid solves as the full plan's Poisson step."""
    pc, torch, dev = env
    n = (24, 20)
    for i, kinds in enumerate(_combos(2)):
        rng = np.random.default_rng(8000 + i)
        h = tuple(rng.uniform(0.5, 2.0) / n[a] for a in range(2))
        lo = tuple(KINDS[k][0] for k in kinds)
        hi = tuple(KINDS[k][1] for k in kinds)
        g = G.Grid(2, n, (0.0, 0.0), h, lo, hi)
        s = rng.normal(size=n)
        ref, _ = P.solve(s, g)
        plan = pc.GridPlan(2, n, h, lo, hi, grid_type="cells", precision=precision)
        p, _ = plan.solve_poisson(torch.as_tensor(s, device=dev))
        assert rel(p.cpu().numpy(), ref) <= tol, (kinds, rel(p.cpu().numpy(), ref))
        plan.close()


def test_grid_plan_refuses_node_calls(env):
    pc, torch, dev = env
    plan = pc.GridPlan(2, (16, 16), (0.1, 0.1), ("W", "W"), ("W", "W"), grid_type="vertices")
    h = plan.handle
    lib = pc.load()
    u = torch.zeros(4, device=dev, dtype=torch.float64)
    st = lib.pc_project(h, 0.1, u.data_ptr(), None, u.data_ptr(), u.data_ptr(), None, None, None)
    assert st == pc.PC_ERR_INVALID_ARG
    st = lib.pc_plan_set_rhs_mask(h, u.data_ptr(), None)
    assert st == pc.PC_ERR_INVALID_ARG
    out = torch.empty(2, dtype=torch.int64)
    import ctypes
    st = lib.pc_plan_rows(h, 0, ctypes.cast(out.data_ptr(), ctypes.POINTER(ctypes.c_int64)), None, None)
    assert st == pc.PC_ERR_INVALID_ARG
    with pytest.raises(pc.PcError):
        plan.clone()
    plan.close()


def test_grid_plan_autotune_keeps_results(env):
    """The transform schedule chosen by the autotuner changes no bit of a vertex solve."""
    pc, torch, dev = env
    n = (48, 40)
    kinds = ("NN", "DN")
    h, lo, hi, s = _vertex_case(kinds, n, 9000)
    plan = pc.GridPlan(2, n, h, lo, hi, grid_type="vertices", precision="mixed")
    sd = torch.as_tensor(s, device=dev)
    p0, _ = plan.solve_poisson(sd)
    p0 = p0.cpu().numpy()
    plan.autotune()
    p1, _ = plan.solve_poisson(sd)
    ref, _ = V.solve(s, n, h, lo, hi)
    assert rel(p1.cpu().numpy(), ref) <= 1e-10
    assert rel(p0, ref) <= 1e-10
    plan.close()


# ----------------------------------------------------------------------------- the vertex-grid pass
from paper_2304_14690_gb300 import workloads as wl   # noqa: E402

VCASES = [
    dict(dim=2, n=(32, 24), bc_lo=("I", "W"), bc_hi=("D", "W"), obstacles=[("circle", (1.0, 0.75), 0.25)]),
    dict(dim=2, n=(40, 40), bc_lo=("P", "P"), bc_hi=("P", "P"), obstacles=[("circle", (1.25, 1.25), 0.3)]),
    dict(dim=2, n=(24, 32), bc_lo=("D", "W"), bc_hi=("W", "D")),
    dict(dim=3, n=(12, 10, 8), bc_lo=("W", "D", "P"), bc_hi=("W", "W", "P"), obstacles=[("sphere", (0.4, 0.3, 0.25), 0.12)]),
]


@pytest.fixture(scope="module")
def vproblems():
    out = []
    for i, c in enumerate(VCASES):
        p = wl.generic(seed=500 + i, with_force=True, **c)
        g = G.Grid(p.dim, p.n, p.lo, p.h, p.bc_lo, p.bc_hi)
        pl = V.build_plan(g, p.nodes, p.node_type, K=p.knn)
        out.append((p, pl, V.project(pl, p.dt, p.u_star, p.f_ib)))
    return out


def _vplan(pc, prob, precision, **kw):
    return pc.Plan(prob, precision=precision, div_mode="wls_direct", grid_type="vertices", **kw)


def _row_kappa(points, queries, idx, g, support_factor=3.0, eps=6.3):
    """Condition number of the WLS normal matrix of every row (for the weight tolerance)."""
    from oracle import knn as KNN, wls as W
    delta = points[idx] - queries[:, None, :]
    for a in range(g.dim):
        if g.periodic(a):
            L = g.length(a)
            da = delta[..., a]
            delta[..., a] = np.where(da > L / 2, da - L, np.where(da < -L / 2, da + L, da))
    d2 = KNN.squared_distance(delta)
    hs = W.support_radius(d2.max(axis=1), idx.shape[1], g.dim, support_factor)
    w = W.gaussian_weight(d2, hs[:, None], eps)
    q = W.basis(delta / hs[:, None, None])
    C = np.einsum("qk,qki,qkj->qij", w, q, q)
    return np.linalg.cond(C)


def test_vertex_rows_match_oracle(env, vproblems):
    """Rows at the vertex unknowns (K nearest nodes, bit-exact columns) and at the nodes (the
    vertex block, bit-exact lattice columns); weights within the kappa bound."""
    pc, torch, dev = env
    ulp = np.finfo(np.float64).eps
    for prob, opl, _ in vproblems:
        plan = _vplan(pc, prob, "fp64")
        g = opl.grid
        col, D = plan.rows(prob.dim + 1)
        assert np.array_equal(col, opl.pt_col), (prob.bc_lo, prob.n)
        kap = _row_kappa(prob.nodes.T, V.pressure_points(g), opl.pt_col, g)
        assert np.all(np.abs(D - opl.pt_D) <= 64 * ulp * kap[None, :, None] * np.abs(opl.pt_D).max(axis=2, keepdims=True))
        col, D = plan.rows(prob.dim)
        assert np.array_equal(col, opl.node_col), (prob.bc_lo, prob.n)
        kap = _row_kappa(V.lattice_points(g), prob.nodes.T, opl.node_col, g)
        assert np.all(np.abs(D - opl.node_D) <= 64 * ulp * kap[None, :, None] * np.abs(opl.node_D).max(axis=2, keepdims=True))
        plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_vertex_project_matches_oracle(env, vproblems, precision, tol):
    """One pass on the vertex grid against the oracle: p at the unknowns, u and f at the nodes;
    the statistics' removed mean; the CUDA-graph replay (no statistics) bitwise equal."""
    pc, torch, dev = env
    for prob, _, ref in vproblems:
        plan = _vplan(pc, prob, precision)
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev)
        p, uo, fo, st = plan.project(u, f, stats=True)
        for name, got, want in (("p", p, ref["p"]), ("u", uo, ref["u"]), ("f", fo, ref["f"])):
            e = rel(got.cpu().numpy(), want)
            assert e <= tol, (prob.bc_lo, prob.n, precision, name, e)
        assert abs(st["removed_mean"] - ref["removed"]) <= 1e-10 * (1 + abs(ref["removed"]))
        p2, u2, f2, _ = plan.project(u, f)
        p3, u3, f3, _ = plan.project(u, f)
        assert torch.equal(p2, p3) and torch.equal(u2, u3) and torch.equal(f2, f3)
        assert rel(p2.cpu().numpy(), ref["p"]) <= tol
        plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_vertex_project_ib_matches_oracle(env, vproblems, precision, tol):
    """The IB-force iteration on the vertex grid (device loop graph): a fixed number of passes
    and the 1e-3 rule of §2.3, against the oracle's iteration."""
    pc, torch, dev = env
    for prob, opl, _ in vproblems[:2] + vproblems[3:]:
        plan = _vplan(pc, prob, precision)
        u = torch.as_tensor(prob.u_star, device=dev)
        ref = V.project_ib(opl, prob.dt, prob.u_star, tol=0.0, max_iters=3)
        p, uo, fo, info = plan.project_ib(u, tol=0.0, max_iters=3)
        assert info["iterations"] == 3
        for name, got, want in (("p", p, ref["p"]), ("u", uo, ref["u"]), ("f", fo, ref["f"])):
            e = rel(got.cpu().numpy(), want)
            assert e <= tol, (prob.bc_lo, precision, name, e)
        ref = V.project_ib(opl, prob.dt, prob.u_star, tol=1e-3, max_iters=50)
        p, uo, fo, info = plan.project_ib(u, tol=1e-3, max_iters=50)
        assert info["iterations"] == ref["iterations"], (info["iterations"], ref["iterations"])
        assert rel(fo.cpu().numpy(), ref["f"]) <= tol, rel(fo.cpu().numpy(), ref["f"])
        plan.close()


def test_vertex_project_host_arrays_and_clone(env, vproblems):
    """Host (pinned) arrays through the staged path, and a clone's workspace, give the device
    result bit for bit."""
    pc, torch, dev = env
    prob, _, ref = vproblems[0]
    plan = _vplan(pc, prob, "mixed")
    u = torch.as_tensor(prob.u_star, device=dev)
    f = torch.as_tensor(prob.f_ib, device=dev)
    p1, u1, f1, _ = plan.project(u, f)
    hu = torch.as_tensor(prob.u_star).pin_memory()
    hf = torch.as_tensor(prob.f_ib).pin_memory()
    outs = (torch.empty(plan.shape, dtype=torch.float64).pin_memory(),
            torch.empty(prob.u_star.shape, dtype=torch.float64).pin_memory(),
            torch.empty(prob.u_star.shape, dtype=torch.float64).pin_memory())
    p2, u2, f2, _ = plan.project(hu, hf, out=outs)
    torch.cuda.synchronize()
    assert np.array_equal(p2.numpy(), p1.cpu().numpy())
    assert np.array_equal(u2.numpy(), u1.cpu().numpy()) and np.array_equal(f2.numpy(), f1.cpu().numpy())
    c = plan.clone()
    p3, u3, f3, _ = c.project(u, f)
    assert torch.equal(p3, p1) and torch.equal(u3, u1) and torch.equal(f3, f1)
    c.close()
    plan.close()


def test_vertex_project_rhs_mask_matches_oracle(env, vproblems):
    pc, torch, dev = env
    prob, opl, _ = vproblems[2]
    plan = _vplan(pc, prob, "mixed")
    mask = (np.random.default_rng(3).random(plan.shape) > 0.25).astype(np.uint8)
    plan.set_rhs_mask(mask)
    ref = V.project(opl, prob.dt, prob.u_star, prob.f_ib, rhs_mask=mask)
    p, uo, fo, _ = plan.project(torch.as_tensor(prob.u_star, device=dev), torch.as_tensor(prob.f_ib, device=dev))
    for name, got, want in (("p", p, ref["p"]), ("u", uo, ref["u"]), ("f", fo, ref["f"])):
        assert rel(got.cpu().numpy(), want) <= 1e-10, name
    plan.close()


def test_vertex_plan_refuses_faces(env):
    pc, torch, dev = env
    prob = wl.generic(dim=2, n=(16, 16), seed=1)
    with pytest.raises(pc.PcError) as e:
        pc.Plan(prob, div_mode="faces", grid_type="vertices")
    assert e.value.status == 2


def test_solve_graph_equals_direct(env):
    """pc_solve_poisson with device arrays replays a cached graph; with graphs off it launches
    directly. Both give the same bits, on vertex and cell grid-only plans, and a second call
    with other arrays captures its own graph."""
    pc, torch, dev = env
    lib = pc.load()
    for grid_type, n, lo, hi in (("vertices", (24, 20), ("I", "W"), ("D", "W")), ("cells", (32, 16), ("P", "W"), ("P", "D"))):
        h = (0.05, 0.07)
        plan = pc.GridPlan(2, n, h, lo, hi, grid_type=grid_type, precision="mixed")
        rng = np.random.default_rng(11)
        s1 = torch.as_tensor(rng.normal(size=plan.shape), device=dev)
        s2 = torch.as_tensor(rng.normal(size=plan.shape), device=dev)
        out = torch.empty(plan.shape, dtype=torch.float64, device=dev)
        g1 = plan.solve_poisson(s1, p_out=out)[0].clone()   # captured for (s1, out)
        out.zero_()
        g1b = plan.solve_poisson(s1, p_out=out)[0].clone()  # the same key: a replay
        g2, _ = plan.solve_poisson(s2)           # another argument set
        assert lib.pc_set_graphs(plan.handle, 0) == 0
        d1, _ = plan.solve_poisson(s1)
        d2, _ = plan.solve_poisson(s2)
        torch.cuda.synchronize()
        assert torch.equal(g1, d1) and torch.equal(g1b, d1) and torch.equal(g2, d2), grid_type
        plan.close()
