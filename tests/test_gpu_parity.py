"""GPU parity of libpc against the CPU oracle, through the C ABI.

Tolerances (relative L2 = ||x - x_ref|| / ||x_ref||):
  FP64 path    1e-12 on p, u, f (the stated FP64 target); KNN column sets bit-exact; WLS weights
               within 64 eps kappa(C) of the row scale (Cholesky against LU: each solve is
               accurate to about kappa(C) eps, kappa ~1e3 inside, up to ~1e5 at 3D walls).
  mixed path   1e-10 after refinement (the stated mixed target).
  FP32 path    unrefined; reported, bounded by 1e-5.
Sizes span several tiles and ragged tails (column tiles of 4-32 lines over widths that are not
multiples of the tile), every boundary pairing, obstacles with boundary/virtual nodes, 2D and 3D.
"""
import itertools

import numpy as np
import pytest

from oracle import grid as G
from oracle import poisson as P
from oracle import projection as PR
from paper_2304_14690_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


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


CASES = [
    dict(dim=2, n=(24, 20), bc_lo=("P", "P"), bc_hi=("P", "P")),
    dict(dim=2, n=(24, 20), bc_lo=("W", "W"), bc_hi=("W", "W"), obstacles=[("circle", (0.7, 0.6), 0.2)]),
    dict(dim=2, n=(32, 16), bc_lo=("I", "W"), bc_hi=("D", "W"), obstacles=[("circle", (0.8, 0.5), 0.15)]),
    dict(dim=2, n=(16, 24), bc_lo=("P", "D"), bc_hi=("P", "D")),
    dict(dim=2, n=(20, 40), bc_lo=("I", "P"), bc_hi=("I", "P")),
    dict(dim=2, n=(48, 30), bc_lo=("D", "I"), bc_hi=("W", "W")),
    dict(dim=3, n=(10, 8, 8), bc_lo=("P", "W", "W"), bc_hi=("P", "W", "W")),
    dict(dim=3, n=(8, 8, 10), bc_lo=("W", "W", "I"), bc_hi=("W", "W", "D"),
         obstacles=[("sphere", (0.25, 0.25, 0.3), 0.12)]),
]


@pytest.fixture(scope="module")
def problems():
    out = []
    for i, c in enumerate(CASES):
        p = wl.generic(seed=300 + i, with_force=True, **c)
        plan = PR.build_plan(grid_of(p), p.nodes, p.node_type, K=p.knn)
        out.append((p, plan, PR.project(plan, p.dt, p.u_star, p.f_ib)))
    return out


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


def test_rows_match_oracle(env, problems):
    pc, torch, dev = env
    ulp = np.finfo(np.float64).eps
    for prob, oplan, _ in problems:
        plan = pc.Plan(prob, precision="fp64")
        g = oplan.grid
        pts = prob.nodes.T
        for a in range(prob.dim):
            col, w = plan.rows(a)
            wall = g.face_is_wall(a).ravel()
            assert np.array_equal(col[~wall], oplan.face_col[a][~wall]), (prob.bc_lo, a)
            kap = _row_kappa(pts, g.face_points(a), oplan.face_col[a], g)
            tol = 64 * ulp * kap[:, None] * np.abs(oplan.face_w[a]).max(axis=1, keepdims=True)
            assert np.all(np.abs(w - oplan.face_w[a]) <= tol)
            assert np.all(w[wall] == 0.0)
        col, D = plan.rows(prob.dim)
        assert np.array_equal(col, oplan.node_col)
        kap = _row_kappa(g.cell_points(), pts, oplan.node_col, g)
        tol = 64 * ulp * kap[None, :, None] * np.abs(oplan.node_D).max(axis=2, keepdims=True)
        assert np.all(np.abs(D - oplan.node_D) <= tol)
        plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10), ("fp32", 1e-5)])
def test_project_matches_oracle(env, problems, precision, tol):
    pc, torch, dev = env
    for prob, _, ref in problems:
        plan = pc.Plan(prob, precision=precision)
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev)
        p, uo, fo, st = plan.project(u, f, stats=True)
        for name, got, want in (("p", p, ref["p"]), ("u", uo, ref["u"]), ("f", fo, ref["f"])):
            e = rel(got.cpu().numpy(), want)
            assert e <= tol, (precision, prob.bc_lo, prob.bc_hi, prob.n, name, e)
        assert abs(st["removed_mean"] - ref["removed"]) <= 1e-9 * max(1.0, np.abs(ref["s"]).max())
        ib = prob.node_type != 0
        assert np.all(uo.cpu().numpy()[:, ib] == 0.0)
        if precision != "fp32":
            # corrected face flux is discretely divergence-free (minus the removed mean)
            expect = prob.beta * prob.dt * abs(ref["removed"])
            scale = np.abs(ref["s"]).max() * prob.beta * prob.dt
            assert st["max_div_after"] <= expect + 1e-9 * scale
        plan.close()


KINDS = {"PP": ("P", "P"), "NN": ("W", "W"), "DD": ("D", "D"), "ND": ("I", "D"), "DN": ("D", "W")}


def _poisson_case(kinds, n, seed):
    dim = len(n)
    rng = np.random.default_rng(seed)
    h = tuple(rng.uniform(0.5, 2.0) / n[a] for a in range(dim))
    g = G.Grid(dim, tuple(n), tuple([0.0] * dim), h, tuple(KINDS[k][0] for k in kinds),
               tuple(KINDS[k][1] for k in kinds))
    s = rng.normal(size=n)
    return g, s


def _GridProblem(g):
    """A problem on grid g (jittered nodes, used only for the plan's WLS setup)."""
    return wl.generic(dim=g.dim, n=g.n, h=g.h, lo=g.lo, bc_lo=g.bc_lo, bc_hi=g.bc_hi, seed=7)


@pytest.mark.parametrize("n", [(8, 8), (24, 20), (96, 64), (40, 48), (8, 12, 10), (16, 6, 20)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10), ("fp32", 1e-5)])
def test_poisson_matches_oracle(env, n, precision, tol):
    pc, torch, dev = env
    dim = len(n)
    combos = list(itertools.product(list(KINDS), repeat=dim))
    if dim == 3:
        combos = combos[::7]
    for i, kinds in enumerate(combos):
        g, s = _poisson_case(kinds, n, 1000 + i)
        ref, removed = P.solve(s, g)
        plan = pc.Plan(_GridProblem(g), precision=precision)
        p, st = plan.solve_poisson(torch.as_tensor(s, device=dev), stats=True)
        e = rel(p.cpu().numpy(), ref)
        assert e <= tol, (kinds, n, precision, e)
        plan.close()


def test_host_pointers_match_device(env, problems):
    pc, torch, dev = env
    prob, _, ref = problems[2]
    plan = pc.Plan(prob, precision="mixed")
    u = torch.as_tensor(prob.u_star, device=dev)
    f = torch.as_tensor(prob.f_ib, device=dev)
    p1, u1, f1, _ = plan.project(u, f)
    hu = torch.as_tensor(prob.u_star).pin_memory()
    hf = torch.as_tensor(prob.f_ib).pin_memory()
    outs = (torch.empty(prob.n[: prob.dim], dtype=torch.float64).pin_memory(),
            torch.empty_like(hu).pin_memory(), torch.empty_like(hu).pin_memory())
    p2, u2, f2, _ = plan.project(hu, hf, out=outs)
    assert torch.equal(p1.cpu(), p2) and torch.equal(u1.cpu(), u2) and torch.equal(f1.cpu(), f2)
    plan.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("graphs", [True, False])
def test_host_arrays_pinned_and_pageable(env, problems, precision, graphs):
    """Host arrays, page-locked or pageable, are staged through the plan's device buffers: every
    path gives the bits of the device-array call, the call returns with the results in the host
    arrays, and a repeated call with new input values in the same host arrays is right too."""
    pc, torch, dev = env
    prob, _, _ = problems[2]
    plan = pc.Plan(prob, precision=precision)
    plan.graphs(graphs)
    u = torch.as_tensor(prob.u_star, device=dev)
    f = torch.as_tensor(prob.f_ib, device=dev)
    ref = [t.cpu() for t in plan.project(u, f)[:3]]
    ref2 = [t.cpu() for t in plan.project(u * 0.5, f)[:3]]
    hu = torch.as_tensor(prob.u_star).pin_memory()
    hf = torch.as_tensor(prob.f_ib).pin_memory()
    outs = (torch.empty(prob.n[: prob.dim], dtype=torch.float64).pin_memory(),
            torch.empty_like(hu).pin_memory(), torch.empty_like(hu).pin_memory())
    got = plan.project(hu, hf, out=outs)[:3]
    assert all(torch.equal(a, b) for a, b in zip(got, ref))
    hu.mul_(0.5)
    got = plan.project(hu, hf, out=outs)[:3]
    assert all(torch.equal(a, b) for a, b in zip(got, ref2))
    pu = torch.as_tensor(prob.u_star).clone()            # pageable: staged
    pouts = (torch.empty(prob.n[: prob.dim], dtype=torch.float64), torch.empty_like(pu), torch.empty_like(pu))
    got = plan.project(pu, torch.as_tensor(prob.f_ib).clone(), out=pouts)[:3]
    assert all(torch.equal(a, b) for a, b in zip(got, ref))
    plan.close()


def test_graph_equals_direct(env, problems):
    """The cached CUDA-graph path gives bitwise the same results as direct launches, also after
    the arguments change (new capture) and when they come back (cache hit)."""
    pc, torch, dev = env
    for prob, _, _ in (problems[1], problems[7]):
        plan = pc.Plan(prob, precision="mixed")
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev)
        a = plan.alloc_outputs()
        b = plan.alloc_outputs()
        u2 = u * 2.0
        plan.project(u, f, out=a)                 # captured and replayed
        plan.project(u2, f, out=b)                # other arguments: second graph
        plan.project(u, f, out=a)                 # cache hit
        plan.graphs(False)
        c = plan.alloc_outputs()
        d = plan.alloc_outputs()
        plan.project(u, f, out=c)
        plan.project(u2, f, out=d)
        torch.cuda.synchronize()
        for x, y in zip(a + b, c + d):
            assert torch.equal(x, y)
        plan.close()


def test_batch_equals_single(env, problems):
    """pc_project_batch runs one launch per stage for all problems; every result is bitwise the
    result of a separate pc_project call (mixed and FP32 plans batched, 2D and 3D groups, with and
    without IB force, singular and non-singular; an FP64 plan runs on its own)."""
    pc, torch, dev = env
    plans, args, singles = [], [], []
    extra = [wl.generic(dim=2, n=(64, 96), bc_lo=("P", "P"), bc_hi=("P", "P"), seed=41),
             wl.generic(dim=2, n=(32, 48), bc_lo=("W", "W"), bc_hi=("W", "W"), seed=42,
                        obstacles=[("circle", (1.0, 1.5), 0.3)], with_force=True)]
    probs = [pr for pr, _, _ in problems] + extra
    precisions = ["mixed"] * (len(probs) - 2) + ["fp32", "fp64"]
    for prob, prec in zip(probs, precisions):
        plan = pc.Plan(prob, precision=prec)
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev) if prob.f_ib is not None else None
        p, uo, fo = plan.alloc_outputs()
        plans.append(plan)
        args.append(dict(dt=prob.dt, u_star=u, f_ib=f, p=p, u=uo, f=fo))
        plan.graphs(False)
        singles.append(plan.project(u, f)[:3])
    for rep in range(2):               # second call replays the cached batch graph
        for a in args:
            a["p"].zero_(); a["u"].zero_(); a["f"].zero_()
        pc.project_batch(plans, args)
        torch.cuda.synchronize()
        for a, s in zip(args, singles):
            assert torch.equal(a["p"], s[0]) and torch.equal(a["u"], s[1]) and torch.equal(a["f"], s[2])
    for pl in plans:
        pl.close()


def test_taylor_green_config(env):
    """Periodic 64x64 Taylor-Green workload, FP64 and mixed against the oracle."""
    pc, torch, dev = env
    prob = wl.periodic_taylor_green()
    ref = PR.project(PR.build_plan(grid_of(prob), prob.nodes, prob.node_type, K=12), prob.dt, prob.u_star)
    for precision, tol in (("fp64", 1e-12), ("mixed", 1e-10)):
        plan = pc.Plan(prob, precision=precision)
        p, uo, fo, st = plan.project(torch.as_tensor(prob.u_star, device=dev), stats=True)
        assert rel(p.cpu().numpy(), ref["p"]) <= tol
        assert rel(uo.cpu().numpy(), ref["u"]) <= tol
        assert st["max_div_after"] * min(prob.h) / st["max_abs_u_star"] <= 1e-9
        plan.close()


IB_CASES = [1, 2, 7]     # the cases with obstacles (boundary and virtual nodes)


def _masked(prob, f):
    out = np.zeros_like(f)
    ib = prob.node_type != 0
    out[:, ib] = f[:, ib]
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_project_ib_matches_oracle(env, problems, precision, tol):
    """Fixed number of passes (tol 0): every pass's force feeds the next (§2.3). The force given
    for the first pass is used only at boundary/virtual nodes, so the GPU gets the workload's
    whole field and the oracle its IB entries. The per-pass sums of the stopping rule are
    compared relative to their size (they are differences of nearly equal forces late in the
    iteration, so they carry the forces' error over the relative change)."""
    pc, torch, dev = env
    for k in IB_CASES:
        prob, oplan, _ = problems[k]
        ref = PR.project_ib(oplan, prob.dt, prob.u_star, _masked(prob, prob.f_ib), tol=0.0, max_iters=4)
        assert ref["iterations"] == 4
        plan = pc.Plan(prob, precision=precision)
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev)
        p, uo, fo, info = plan.project_ib(u, f, tol=0.0, max_iters=4)
        assert info["iterations"] == 4 and not info["converged"]
        for name, got, want in (("p", p, ref["p"]), ("u", uo, ref["u"]), ("f", fo, ref["f"])):
            e = rel(got.cpu().numpy(), want)
            assert e <= tol, (precision, k, name, e)
        for (gd, gp), (rd, rp) in zip(info["history"], ref["history"]):
            assert abs(gd - rd) <= 1e-7 * rd and abs(gp - rp) <= 1e-7 * rp, (k, gd, rd, gp, rp)
        plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_project_ib_stops_like_oracle(env, problems, precision):
    """The paper's tolerance 1e-3: the GPU stops after the same pass as the oracle (the case is
    checked to be far from the threshold at every pass, so rounding cannot flip a decision)."""
    pc, torch, dev = env
    for k in IB_CASES:
        prob, oplan, _ = problems[k]
        ref = PR.project_ib(oplan, prob.dt, prob.u_star, tol=1e-3, max_iters=60)
        ratios = [d / p for d, p in ref["history"] if p > 0]
        assert all(abs(r / 1e-3 - 1.0) > 0.01 for r in ratios)
        plan = pc.Plan(prob, precision=precision)
        u = torch.as_tensor(prob.u_star, device=dev)
        p, uo, fo, info = plan.project_ib(u, tol=1e-3, max_iters=60)
        assert info["iterations"] == ref["iterations"] and info["converged"]
        assert info["history"][0][1] == 0.0             # the first pass starts from zero force
        assert rel(fo.cpu().numpy(), ref["f"]) <= 1e-9
        plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_project_ib_equals_repeated_project(env, problems, precision):
    """The incremental passes (IB-node prep, listed faces, IB-node gradient) give bitwise the
    iterates of full pc_project passes fed with the previous force."""
    pc, torch, dev = env
    for k in IB_CASES:
        prob, _, _ = problems[k]
        plan = pc.Plan(prob, precision=precision)
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(_masked(prob, prob.f_ib), device=dev)
        for _ in range(3):
            p, uo, f, _ = plan.project(u, f)
            p, uo, f = p.clone(), uo.clone(), f.clone()
        pi, ui, fi, info = plan.project_ib(u, f_init=torch.as_tensor(_masked(prob, prob.f_ib), device=dev),
                                           tol=0.0, max_iters=3)
        assert info["iterations"] == 3
        assert torch.equal(pi, p) and torch.equal(ui, uo) and torch.equal(fi, f), (precision, k)
        plan.close()


def test_project_ib_without_ib_nodes(env, problems):
    """No boundary/virtual nodes: one pass, converged (no force and no change), equal to
    pc_project."""
    pc, torch, dev = env
    prob, _, _ = problems[0]
    assert not np.any(prob.node_type != 0)
    plan = pc.Plan(prob, precision="mixed")
    u = torch.as_tensor(prob.u_star, device=dev)
    p, uo, fo, _ = plan.project(u)
    p, uo, fo = p.clone(), uo.clone(), fo.clone()
    pi, ui, fi, info = plan.project_ib(u, tol=1e-3)
    assert info["iterations"] == 1 and info["converged"] and info["history"] == [(0.0, 0.0)]
    assert torch.equal(pi, p) and torch.equal(ui, uo) and torch.equal(fi, fo)
    with pytest.raises(pc.PcError):
        plan.project_ib(u.cpu(), tol=1e-3)              # device pointers only
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_project_ib_graph_equals_host_loop(env, problems, precision):
    """The loop graph (while node, device-side stopping rule) and the host-driven loop run the
    same passes: same pass count and history, bitwise outputs; a replay of the cached graph with
    new input values gives the host loop's result too; max_iters bounds the graph's loop."""
    pc, torch, dev = env
    for k in IB_CASES:
        prob, _, _ = problems[k]
        plan = pc.Plan(prob, precision=precision)
        u = torch.as_tensor(prob.u_star, device=dev)
        outs = plan.alloc_outputs()
        res = {}
        for mode in (False, True):
            plan.graphs(mode)
            for scale in (1.0, 0.5):
                u.copy_(torch.as_tensor(prob.u_star, device=dev) * scale)
                p, uo, fo, info = plan.project_ib(u, tol=1e-3, max_iters=60, out=outs)
                res[mode, scale] = ([t.clone() for t in (p, uo, fo)], info)
        for scale in (1.0, 0.5):
            (a, ia), (b, ib_) = res[False, scale], res[True, scale]
            assert ia["iterations"] == ib_["iterations"] and ia["history"] == ib_["history"], (k, scale)
            assert all(torch.equal(x, y) for x, y in zip(a, b)), (precision, k, scale)
        for m in (1, 2):
            _, _, _, info = plan.project_ib(u, tol=0.0, max_iters=m, out=outs)
            assert info["iterations"] == m and not info["converged"]
        plan.close()


@pytest.mark.parametrize("n", [(8, 8), (24, 20), (96, 64), (8, 12, 10)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_poisson_spectral_matches_oracle(env, n, precision, tol):
    """Pseudo-spectral eigenvalues (§2.3): every boundary pairing against the oracle's
    expansion with the same eigenvalues."""
    pc, torch, dev = env
    dim = len(n)
    combos = list(itertools.product(list(KINDS), repeat=dim))
    if dim == 3:
        combos = combos[::7]
    for i, kinds in enumerate(combos):
        g, s = _poisson_case(kinds, n, 2000 + i)
        ref, _ = P.solve(s, g, eigenvalues="spectral")
        plan = pc.Plan(_GridProblem(g), precision=precision, eigenvalues="spectral")
        p, _ = plan.solve_poisson(torch.as_tensor(s, device=dev))
        e = rel(p.cpu().numpy(), ref)
        assert e <= tol, (kinds, n, precision, e)
        plan.close()


def test_project_spectral_matches_oracle(env, problems):
    """Whole projection with the pseudo-spectral solve (FP64 plans), and the mixed precision
    refused (its refinement residual is that of the finite-difference operator)."""
    pc, torch, dev = env
    for prob, oplan, _ in problems:
        ref = PR.project(oplan, prob.dt, prob.u_star, prob.f_ib, eigenvalues="spectral")
        plan = pc.Plan(prob, precision="fp64", eigenvalues="spectral")
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev)
        p, uo, fo, st = plan.project(u, f, stats=True)
        for name, got, want in (("p", p, ref["p"]), ("u", uo, ref["u"]), ("f", fo, ref["f"])):
            e = rel(got.cpu().numpy(), want)
            assert e <= 1e-12, (prob.bc_lo, prob.bc_hi, prob.n, name, e)
        assert st["residual_norm"] == [0.0]
        plan.close()
    with pytest.raises(pc.PcError):
        pc.Plan(problems[0][0], precision="mixed", eigenvalues="spectral")


def _mask_for(prob, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(tuple(prob.n[:prob.dim])) > 0.3).astype(np.uint8)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_project_rhs_mask_matches_oracle(env, problems, precision, tol):
    """§3.5 RHS mask: the source is zeroed outside the flow domain; single projections, the
    IB iteration and a batch against the oracle (and the batch bitwise equal to single calls);
    max_div_after is taken inside the mask; clearing the mask restores the unmasked result."""
    pc, torch, dev = env
    for k, (prob, oplan, ref0) in enumerate(problems):
        mask = _mask_for(prob, 50 + k)
        ref = PR.project(oplan, prob.dt, prob.u_star, prob.f_ib, rhs_mask=mask)
        plan = pc.Plan(prob, precision=precision)
        plan.set_rhs_mask(mask)
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev)
        p, uo, fo, st = plan.project(u, f, stats=True)
        for name, got, want in (("p", p, ref["p"]), ("u", uo, ref["u"]), ("f", fo, ref["f"])):
            e = rel(got.cpu().numpy(), want)
            assert e <= tol, (precision, k, name, e)
        expect = prob.beta * prob.dt * abs(ref["removed"])
        scale = np.abs(ref["s"]).max() * prob.beta * prob.dt
        assert st["max_div_after"] <= expect + 1e-9 * scale
        # graph replay (no stats) and a batch of this plan with a clone give the same bits
        p1, u1, f1, _ = plan.project(u, f)
        p1, u1, f1 = p1.clone(), u1.clone(), f1.clone()
        if precision == "mixed":
            outs = plan.alloc_outputs()
            pc.project_batch([plan], [dict(dt=prob.dt, u_star=u, f_ib=f, p=outs[0], u=outs[1], f=outs[2])])
            torch.cuda.synchronize()
            assert all(torch.equal(a, b) for a, b in zip(outs, (p1, u1, f1)))
        assert rel(p1.cpu().numpy(), ref["p"]) <= tol
        if np.any(prob.node_type != 0):
            rib = PR.project_ib(oplan, prob.dt, prob.u_star, tol=0.0, max_iters=3, rhs_mask=mask)
            pi, ui, fi, _ = plan.project_ib(u, tol=0.0, max_iters=3)
            for name, got, want in (("p", pi, rib["p"]), ("u", ui, rib["u"]), ("f", fi, rib["f"])):
                assert rel(got.cpu().numpy(), want) <= tol, (precision, k, "ib", name)
        plan.set_rhs_mask(None)
        p2, _, _, _ = plan.project(u, f)
        assert rel(p2.cpu().numpy(), ref0["p"]) <= tol
        plan.close()


def test_direct_divergence_rows_match_oracle(env, problems):
    """Cell-centre derivative rows of the direct divergence: KNN columns bit-exact, weights
    within the kappa bound of the WLS normal matrix (as the face and node rows)."""
    pc, torch, dev = env
    ulp = np.finfo(np.float64).eps
    for prob, oplan, _ in problems:
        plan = pc.Plan(prob, precision="fp64", div_mode="wls_direct")
        col, D = plan.rows(prob.dim + 1)
        ccol, cD = PR.cell_rows(oplan)
        assert np.array_equal(col, ccol), (prob.bc_lo, prob.n)
        kap = _row_kappa(prob.nodes.T, oplan.grid.cell_points(), ccol, oplan.grid)
        tol = 64 * ulp * kap[None, :, None] * np.abs(cD).max(axis=2, keepdims=True)
        assert np.all(np.abs(D - cD) <= tol)
        plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_project_direct_divergence_matches_oracle(env, problems, precision, tol):
    """The paper's direct WLS divergence at the cell centres: single projections and the IB
    iteration against the oracle, and a batch entry (run one by one) bitwise equal to a single
    call."""
    pc, torch, dev = env
    for k, (prob, oplan, _) in enumerate(problems):
        ref = PR.project(oplan, prob.dt, prob.u_star, prob.f_ib, div_mode="wls_direct")
        plan = pc.Plan(prob, precision=precision, div_mode="wls_direct")
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev)
        p, uo, fo, st = plan.project(u, f, stats=True)
        for name, got, want in (("p", p, ref["p"]), ("u", uo, ref["u"]), ("f", fo, ref["f"])):
            e = rel(got.cpu().numpy(), want)
            assert e <= tol, (precision, k, name, e)
        assert abs(st["removed_mean"] - ref["removed"]) <= 1e-9 * max(1.0, np.abs(ref["s"]).max())
        assert st["max_div_after"] == 0.0
        p1 = plan.project(u, f)[0].clone()
        outs = plan.alloc_outputs()
        pc.project_batch([plan], [dict(dt=prob.dt, u_star=u, f_ib=f, p=outs[0], u=outs[1], f=outs[2])])
        torch.cuda.synchronize()
        assert torch.equal(outs[0], p1)
        if np.any(prob.node_type != 0):
            rib = PR.project_ib(oplan, prob.dt, prob.u_star, tol=0.0, max_iters=3, div_mode="wls_direct")
            pi, ui, fi, info = plan.project_ib(u, tol=0.0, max_iters=3)
            assert info["iterations"] == 3
            for name, got, want in (("p", pi, rib["p"]), ("u", ui, rib["u"]), ("f", fi, rib["f"])):
                assert rel(got.cpu().numpy(), want) <= tol, (precision, k, "ib", name)
        plan.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_schedule_knobs(env, problems, precision):
    """The transform schedule: every slot count gives the oracle's result within tolerance
    (results change only by rounding between schedules), the CTA target changes nothing at all
    (each line is transformed the same way in any tile), a batch call agrees bitwise with the
    single call under any schedule, and bad values are refused."""
    pc, torch, dev = env
    tol = 1e-12 if precision == "fp64" else 1e-10
    for k in (1, 6):
        prob, _, ref = problems[k]
        plan = pc.Plan(prob, precision=precision)
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(prob.f_ib, device=dev)
        for slots in ((2, 4, 8, 16) if precision == "fp64" else (0, 1, 2, 4, 8, 16)):
            for a in range(prob.dim):
                plan.set_slots(a, slots)
            base = None
            for ctas in (1, 2, 4, 8):
                for a in range(prob.dim):
                    plan.set_ctas(a, ctas)
                got = [t.clone() for t in plan.project(u, f)[:3]]
                if base is None:
                    base = got
                    assert rel(got[0].cpu().numpy(), ref["p"]) <= tol, (k, slots)
                else:
                    assert all(torch.equal(x, y) for x, y in zip(got, base)), (k, slots, ctas)
            if precision == "mixed":
                outs = plan.alloc_outputs()
                pc.project_batch([plan], [dict(dt=prob.dt, u_star=u, f_ib=f, p=outs[0], u=outs[1], f=outs[2])])
                torch.cuda.synchronize()
                assert all(torch.equal(x, y) for x, y in zip(outs, base)), (k, slots)
        assert plan.ctas() == [8] * prob.dim
        for bad in (0, 3, 16):
            with pytest.raises(pc.PcError):
                plan.set_ctas(0, bad)
        plan.close()


def test_non_finite_input_reported(env, problems):
    """Device-detected non-finite data come back as a status, and the plan stays usable: a NaN in
    u* makes a projection with statistics return PC_ERR_INVALID_ARG and the IB iteration
    PC_ERR_NOT_CONVERGED; the next call with finite data is right."""
    pc, torch, dev = env
    prob, _, ref = problems[1]
    plan = pc.Plan(prob, precision="mixed")
    u = torch.as_tensor(prob.u_star, device=dev)
    f = torch.as_tensor(prob.f_ib, device=dev)
    bad = u.clone()
    bad[0, 5] = float("nan")
    with pytest.raises(pc.PcError) as e:
        plan.project(bad, f, stats=True)
    assert e.value.status == 1
    with pytest.raises(pc.PcError) as e:
        plan.project_ib(bad, tol=1e-3, max_iters=5)
    assert e.value.status == 7
    p, uo, fo, st = plan.project(u, f, stats=True)
    assert rel(p.cpu().numpy(), ref["p"]) <= 1e-10
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_fp32_velocity_storage(env, precision, tol):
    """Velocity arrays stored in FP32 (as the 3D workload has them): projections, the IB
    iteration and the direct divergence against the oracle run on the same FP32 values promoted
    to FP64. p is computed in full precision from the FP32 input (tol); u and f are stored in
    FP32, so they agree to FP32 rounding."""
    pc, torch, dev = env
    f32 = 2.0 ** -23
    for k in IB_CASES:
        c = CASES[k]
        prob = wl.generic(seed=300 + k, with_force=True, dtype=np.float32, **c)
        oplan = PR.build_plan(grid_of(prob), prob.nodes, prob.node_type, K=prob.knn)
        u64 = prob.u_star.astype(np.float64)
        fm = _masked(prob, prob.f_ib.astype(np.float64))
        u = torch.as_tensor(prob.u_star, device=dev)
        f = torch.as_tensor(_masked(prob, prob.f_ib), device=dev)
        for div_mode in ("faces", "wls_direct"):
            plan = pc.Plan(prob, precision=precision, div_mode=div_mode)
            ref = PR.project(oplan, prob.dt, u64, fm, div_mode=div_mode)
            p, uo, fo, _ = plan.project(u, f)
            assert uo.dtype == torch.float32
            assert rel(p.cpu().numpy(), ref["p"]) <= tol, (precision, k, div_mode)
            assert rel(uo.cpu().numpy(), ref["u"]) <= f32 and rel(fo.cpu().numpy(), ref["f"]) <= f32
            rib = PR.project_ib(oplan, prob.dt, u64, fm, tol=0.0, max_iters=3, div_mode=div_mode)
            pi, ui, fi, info = plan.project_ib(u, f_init=f, tol=0.0, max_iters=3)
            assert info["iterations"] == 3
            # the force iterates are stored in FP32 between passes: FP32-level agreement
            assert rel(pi.cpu().numpy(), rib["p"]) <= 1e-5, (precision, k, div_mode)
            assert rel(fi.cpu().numpy(), rib["f"]) <= 1e-5 and rel(ui.cpu().numpy(), rib["u"]) <= 1e-5
            plan.close()
