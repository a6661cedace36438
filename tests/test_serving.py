"""Serving loop on the GPU: continuous batching of a Poisson-arrival trace over a small geometry
pool (2D and 3D, obstacles). Every request's result is the same alone and in the mix: the
outputs of the served request equal a single pc_project call on the same plan with the same
u* (bitwise when plans stay resident; within 1e-12 when a tight budget forces evictions and
rebuilds)."""
import numpy as np
import pytest

from paper_2304_14690_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_14690_gb300 import pc, serving
    return pc, serving, torch


@pytest.fixture(scope="module")
def pool():
    return wl.serving_pool(count=8, seed=77, sizes_2d=(64, 96, 128), sizes_3d=(16, 24))


def _alone(server, torch, gid, scale):
    plan = server.cache.plans[gid][0][0].plan        # the root instance
    u = torch.mul(server.base_u[gid], scale)
    p, uo, fo, _ = plan.project(u)
    torch.cuda.synchronize()
    return p.cpu(), uo.cpu(), fo.cpu()


def test_results_same_alone_and_in_mix(env, pool):
    pc, serving, torch = env
    trace = wl.serving_trace(count=120, rate=20000.0, pool_size=len(pool), seed=5)
    srv = serving.Server(pool, budget_bytes=40 << 30, keep_outputs=True)
    reqs = srv.run(trace)
    assert all(np.isfinite(r.done) and r.done >= r.arrival for r in reqs)
    sizes = np.bincount([r.batch for r in reqs])
    assert sizes.max() > 1                       # requests were batched together
    assert srv.cache.evictions == 0
    for r in reqs:
        got = srv.outputs[r.rid]
        ref = _alone(srv, torch, r.geometry, r.scale)
        for a, b in zip(got, ref):
            assert torch.equal(a, b), r
    s = serving.summarize(reqs, pool)
    assert s["requests"] == len(reqs) and s["latency_ms"]["p99"] >= s["latency_ms"]["p50"]
    srv.close()


def test_tight_budget_evicts_and_rebuilds(env, pool):
    pc, serving, torch = env
    sizes = []
    for prob in pool:
        plan = pc.Plan(prob, precision="mixed")
        sizes.append(plan.nbytes() + prob.u_star.nbytes)
        plan.close()
    io = max(prob.num_cells * 8 + 3 * prob.u_star.nbytes for prob in pool)
    budget = sum(sorted(sizes)[-3:]) + 2 * io       # about three plans resident at a time
    trace = wl.serving_trace(count=60, rate=20000.0, pool_size=len(pool), seed=6)
    srv = serving.Server(pool, budget_bytes=budget, keep_outputs=True)
    reqs = srv.run(trace)
    assert srv.cache.evictions > 0
    assert srv.cache.used + srv.io_used <= budget
    for r in reqs:
        got = srv.outputs[r.rid]
        gid = r.geometry
        plan = pc.Plan(pool[gid], precision="mixed")
        u = torch.mul(torch.as_tensor(pool[gid].u_star, device="cuda"), r.scale)
        ref = plan.project(u)[:3]
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            b = b.cpu()
            assert float(torch.linalg.vector_norm((a - b).double())) <= 1e-12 * float(torch.linalg.vector_norm(b.double()))
        plan.close()
    srv.close()


def test_clone_shares_rows_and_matches(env, pool):
    """A clone computes bitwise what its root computes, alone and in one batch with the root
    (two workspaces, one set of rows); the root cannot be destroyed while the clone lives."""
    pc, serving, torch = env
    prob = pool[0]
    root = pc.Plan(prob, precision="mixed")
    twin = root.clone()
    assert twin.nbytes() < root.nbytes()
    u = torch.as_tensor(prob.u_star, device="cuda")
    a = [t.cpu() for t in root.project(u)[:3]]
    b = [t.cpu() for t in twin.project(u)[:3]]
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    outs = [root.alloc_outputs(), twin.alloc_outputs()]
    u2 = u * 0.5
    args = [dict(dt=prob.dt, u_star=u, p=outs[0][0], u=outs[0][1], f=outs[0][2]),
            dict(dt=prob.dt, u_star=u2, p=outs[1][0], u=outs[1][1], f=outs[1][2])]
    bat = pc.Batcher(0)
    bat.launch([root, twin], args)
    torch.cuda.synchronize()
    single = [t.cpu() for t in root.project(u2)[:3]]
    assert all(torch.equal(x.cpu(), y) for x, y in zip(outs[0], a))
    assert all(torch.equal(x.cpu(), y) for x, y in zip(outs[1], single))
    with pytest.raises(pc.PcError):
        root.close()
    twin.close()
    root.close()
    bat.close()


def test_overload_is_shed_and_latency_bounded(env, pool):
    """Offered far above capacity, with a bounded queue and a deadline: arrivals that find the
    queue full are refused, waiting requests past the deadline are dropped, every other request
    is served within deadline + the time of the batches ahead of it, and served results still
    equal single calls."""
    pc, serving, torch = env
    trace = wl.serving_trace(count=400, rate=2.0e6, pool_size=len(pool), seed=9)
    srv = serving.Server(pool, budget_bytes=40 << 30, keep_outputs=True, max_queue=16, deadline_s=0.002,
                         max_batch=8)
    srv.warm(range(len(pool)))
    reqs = srv.run(trace)
    s = serving.summarize(reqs, pool)
    assert s["shed"]["queue"] > 0                # the burst overflowed the queue
    assert s["served"] + s["shed"]["queue"] + s["shed"]["deadline"] == len(reqs)
    assert 0 < s["served"] < len(reqs)
    served = [r for r in reqs if not r.shed]
    assert all(np.isfinite(r.done) and r.launched - r.arrival <= 0.002 + 0.02 for r in served)
    assert all(r.rid not in srv.outputs for r in reqs if r.shed)
    for r in served[:20]:
        ref = _alone(srv, torch, r.geometry, r.scale)
        for a, b in zip(srv.outputs[r.rid], ref):
            assert torch.equal(a, b), r
    srv.close()
