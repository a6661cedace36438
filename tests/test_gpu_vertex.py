"""Grid-only plans against the oracle: the Poisson solve on the vertex ("regular") pressure grid
of §2.3 (the grid of the §3.2 results) for every boundary pairing, and on the cell-centred grid
without nodes. The vertex solve goes through the symmetric extension to a periodic cell grid on
the device; the oracle expands in the DCT-I / DST-I / quarter-wave eigenvectors directly."""
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
