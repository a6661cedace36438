"""The allocation-free Poisson solve (pc_solve_poisson_static) against the plan-based one.

Callers that cannot allocate device memory (memory pools that own the device, host callbacks,
start-up-sized deployments) use pc_solve_poisson_static, whose workspace is a fixed device array
inside the library. This checks, through the C ABI, that two calls in a row on different grids
give the same pressure as pc_solve_poisson with a plan, within the FP64 tolerance of the other
parity tests (relative L2 <= 1e-12), and that the size limit is reported. The file is named to
be collected last; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2304_14690_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CASES = [
    dict(dim=2, n=(96, 64), h=(1 / 64, 1 / 48), bc_lo=("I", "W"), bc_hi=("D", "W")),
    dict(dim=2, n=(64, 40), h=(0.05, 0.02), bc_lo=("P", "W"), bc_hi=("P", "W")),
    dict(dim=3, n=(16, 12, 20), h=(0.1, 0.2, 0.05), bc_lo=("W", "P", "D"), bc_hi=("W", "P", "D")),
    # singular problems: the 3D all-wall box (mean gauge) and the corner gauge, whose constant is
    # taken by the gauge kernels from the workspace's statistics
    dict(dim=3, n=(16, 12, 10), h=(0.1, 0.2, 0.05), bc_lo=("W", "W", "W"), bc_hi=("W", "W", "W")),
    dict(dim=2, n=(64, 40), h=(0.05, 0.02), bc_lo=("P", "W"), bc_hi=("P", "W"), gauge=1),
    dict(dim=3, n=(16, 12, 10), h=(0.1, 0.2, 0.05), bc_lo=("W", "P", "I"), bc_hi=("W", "P", "W"), gauge=1),
]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_solve_matches_plan_solve():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    results = []
    for c in CASES:
        prob = wl.generic(seed=11, **{k: v for k, v in c.items() if k != "gauge"})
        plan = pc.Plan(prob, precision="fp64", gauge=c.get("gauge", 0))
        s = torch.as_tensor(rng.normal(size=prob.n[: prob.dim]), device=dev)
        ref, _ = plan.solve_poisson(s)
        results.append((c, s, ref.cpu().numpy()))
        plan.close()
    # two calls in a row (and a third that repeats the first grid after the second); the
    # singular cases also check that each call starts from clean statistics and counters
    for c, s, ref in results[:2] + results[:1] + results[2:] + results[3:]:
        p = torch.empty_like(s)
        pc.solve_poisson_static(c["dim"], c["n"], c["h"], c["bc_lo"], c["bc_hi"], s, p, gauge=c.get("gauge", 0))
        torch.cuda.synchronize()
        assert rel(p.cpu().numpy(), ref) <= 1e-12, c
        if c.get("gauge", 0) == 1:
            assert p.flatten()[0].item() == 0.0


def test_static_solve_rejects_arrays_of_another_device():
    """s and p_out must be memory of the current device: the workspace is per device."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU to place the arrays elsewhere")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc
    s = torch.zeros((16, 16), dtype=torch.float64, device="cuda:1")
    with torch.cuda.device(0):
        with pytest.raises(pc.PcError) as e:
            pc.solve_poisson_static(2, (16, 16), (1.0, 1.0), ("W", "W"), ("W", "W"), s, torch.empty_like(s))
    assert e.value.status == 1


def test_static_solve_rejects_large_grid():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc
    s = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")
    with pytest.raises(pc.PcError) as e:
        pc.solve_poisson_static(2, (1024, 1024), (1.0, 1.0), ("W", "W"), ("W", "W"), s, torch.empty_like(s))
    assert e.value.status == 5 and "static workspace limit" in str(e.value)
