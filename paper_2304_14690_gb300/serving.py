"""Request loop for pressure-correction projections: continuous batching under a device-memory
budget.

Requests for projections on different grids arrive over time. The server:
  - keeps plans (WLS rows, transform tables, workspace) resident in an LRU cache bounded by a
    byte budget, and builds a missing plan when its first request is admitted (a cold build,
    counted in that request's latency);
  - admits pending requests in arrival order as memory allows, skipping those whose plan is
    already in flight (a plan holds the workspace of one projection at a time);
  - launches every admitted set as one batch through the batch executor (one launch per
    pipeline stage for all its problems) on a free stream, so that while batches run on the
    device the next one is assembled from the requests that arrived meanwhile and launched as
    soon as an in-flight slot frees: batches overlap on the device;
  - records each request's completion from a CUDA event recorded behind its batch;
  - bounds latency under overload: an arrival that finds max_queue requests already waiting is
    refused at once (backpressure), and a waiting request not launched within deadline_s of its
    arrival is dropped (load shedding). Shed requests are counted and never computed.
A request's result does not depend on the batch it rides in: the batched kernels keep the
single-call decomposition, so results equal those of a pc_project call on the same plan.
"""
import collections
import dataclasses
import heapq
import math
import time

import numpy as np

from . import pc


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    geometry: int           # index into the geometry pool
    scale: float            # u* = scale x the geometry's field
    launched: float = math.nan
    done: float = math.nan
    cold: bool = False      # its plan was built when it was admitted
    batch: int = -1
    shed: str = ""          # "queue" (refused on arrival) or "deadline" (dropped while waiting)

    @property
    def latency(self):
        return self.done - self.arrival


class PlanCache:
    """Resident plans per geometry, least recently used first, within a byte budget. A geometry
    holds its plan (the root) and up to max_instances - 1 clones, extra workspaces on the same
    rows, so that several of its requests can run at once. Geometries with an instance in flight
    are never evicted.

    make_plan(gid, budget_bytes) returns an object with nbytes(), clone() and close(), or raises
    pc.PcError with status PC_ERR_BUDGET when it would not fit. clone_bytes(gid) estimates the
    device bytes of one more instance (a clone is made only into free budget, never by
    evicting)."""

    def __init__(self, budget_bytes, make_plan, extra_bytes=lambda gid: 0, max_instances=1,
                 clone_bytes=lambda gid: 0, clone_headroom=0):
        self.budget = int(budget_bytes)
        self.make_plan = make_plan
        self.extra_bytes = extra_bytes          # per-geometry device bytes held beside the plan
        self.clone_bytes = clone_bytes
        self.clone_headroom = clone_headroom     # budget clones leave free (for request buffers)
        self.max_instances = max_instances
        self.plans = collections.OrderedDict()  # gid -> [instances (root first), bytes]
        self.used = 0
        self.builds = 0
        self.clones = 0
        self.evictions = 0

    def resident(self, gid):
        return gid in self.plans

    def _evict_one(self, keep):
        for gid in self.plans:
            if gid not in keep:
                insts, b = self.plans.pop(gid)
                for inst in reversed(insts):     # clones before their root
                    inst.close()
                self.used -= b
                self.evictions += 1
                return True
        return False

    def get(self, gid, keep, reserve=0):
        """The root plan of gid (built if absent, evicting idle geometries as needed) and whether
        it was built now; None when it cannot fit beside `keep` and `reserve` bytes."""
        if gid in self.plans:
            self.plans.move_to_end(gid)
            return self.plans[gid][0][0], False
        extra = self.extra_bytes(gid)
        while True:
            free = self.budget - self.used - reserve - extra
            plan = None
            if free > 0:
                try:
                    plan = self.make_plan(gid, free)
                except pc.PcError as e:
                    if e.status != pc.PC_ERR_BUDGET:
                        raise
            if plan is not None:
                b = plan.nbytes() + extra
                self.plans[gid] = [[plan], b]
                self.used += b
                self.builds += 1
                return plan, True
            if not self._evict_one(keep | {gid}):
                return None

    def acquire(self, gid, busy, keep, reserve=0):
        """An instance of gid that is not in `busy` (built or cloned as needed) and whether the
        plan was built now; None when there is none."""
        got = self.get(gid, keep, reserve)
        if got is None:
            return None
        _, cold = got
        insts = self.plans[gid][0]
        for inst in insts:
            if id(inst) not in busy:
                return inst, cold
        if len(insts) >= self.max_instances:
            return None
        need = self.clone_bytes(gid)
        if self.used + reserve + need + self.clone_headroom > self.budget:
            return None
        inst = insts[0].clone()
        b = inst.nbytes()
        insts.append(inst)
        self.plans[gid][1] += b
        self.used += b
        self.clones += 1
        return inst, cold

    def make_room(self, nbytes, keep):
        """Evict idle geometries until nbytes more fit in the budget; False when they cannot."""
        while self.used + nbytes > self.budget:
            if not self._evict_one(keep):
                return False
        return True

    def close(self):
        for insts, _ in self.plans.values():
            for inst in reversed(insts):
                inst.close()
        self.plans.clear()
        self.used = 0


@dataclasses.dataclass
class _Batch:
    reqs: list
    gids: set
    instances: set            # id() of the plan instances in flight
    stream_index: int
    end: object
    io_bytes: int
    outputs: list
    begin: object = None


class Server:
    """Continuous-batching request loop over a pool of geometries (workloads.Problem)."""

    def __init__(self, geometries, budget_bytes, precision="mixed", refine=4, max_batch=64,
                 max_inflight=4, max_instances=4, clone_headroom=8 << 30, device=0,
                 keep_outputs=False, batched=True, tune=False, refine_tol=1e-13, max_queue=None,
                 deadline_s=None):
        import torch
        self.torch = torch
        self.geoms = geometries
        self.precision = precision
        self.refine = refine
        self.refine_tol = refine_tol
        self.max_batch = max_batch if batched else 1
        self.max_inflight = max_inflight
        self.device = torch.device("cuda", device)
        self.keep_outputs = keep_outputs  # True: every request's outputs; a set: those request ids
        self.max_queue = max_queue        # waiting requests beyond which arrivals are refused
        self.deadline_s = deadline_s      # a request not launched this long after arrival is dropped
        self.batched = batched
        self.tune = tune
        self.base_u = {}
        self.cache = PlanCache(budget_bytes, self._make_plan, self._field_bytes,
                               max_instances=max_instances if batched else 1,
                               clone_bytes=self._clone_bytes, clone_headroom=clone_headroom)
        self.io_used = 0
        self.outputs = {}
        self.batcher = pc.Batcher(device, slots=max_inflight + 2) if batched else None

    def warm(self, gids):
        """Build the plans of gids ahead of the requests (as far as the budget allows); returns
        how many are resident."""
        for gid in gids:
            if self.cache.get(gid, set()) is None:
                break
        return sum(1 for g in gids if self.cache.resident(g))

    def _field_bytes(self, gid):
        return self.geoms[gid].u_star.nbytes

    def _clone_bytes(self, gid):
        # a clone's workspace: face fluxes, cell arrays, node copies (+10% for scratch)
        p = self.geoms[gid]
        faces = sum(p.num_cells // p.n[a] * (p.n[a] + (0 if p.bc_lo[a] == "P" else 1)) for a in range(p.dim))
        return int(1.1 * (faces * 8 + p.num_cells * 52 + p.dim * p.num_nodes * 8))

    def _make_plan(self, gid, budget):
        prob = self.geoms[gid]
        plan = pc.Plan(prob, precision=self.precision, refine_iters=self.refine, refine_tol=self.refine_tol,
                       device=self.device.index, budget_bytes=int(budget))
        if self.tune:
            plan.autotune()
        self.base_u[gid] = self.torch.as_tensor(prob.u_star, device=self.device)
        return _OwnedPlan(plan, self.base_u, gid)

    def _io_bytes(self, gid):
        p = self.geoms[gid]
        return p.num_cells * 8 + 3 * p.u_star.nbytes        # p; u*, u, f

    def _assemble(self, queues, inflight):
        """Requests for the next batch: oldest request first across the geometries' queues,
        each on a free instance of its geometry's plan, as memory allows."""
        busy, busy_g = set(), set()
        for b in inflight:
            busy |= b.instances
            busy_g |= b.gids
        heap = [(q[0].arrival, gid) for gid, q in queues.items() if q]
        heapq.heapify(heap)
        batch, taken_g = [], set()
        while heap and len(batch) < self.max_batch:
            _, gid = heapq.heappop(heap)
            q = queues[gid]
            io = self._io_bytes(gid)
            keep = busy_g | taken_g
            got = self.cache.acquire(gid, busy, keep, reserve=self.io_used + io)
            if got is None:
                continue
            if self.cache.used + self.io_used + io > self.cache.budget:
                # buffers of batches in flight free memory soon: wait for them rather than evict
                if inflight or batch or not self.cache.make_room(self.io_used + io, keep | {gid}):
                    continue
            inst, cold = got
            r = q.popleft()
            r.cold = cold
            busy.add(id(inst))
            taken_g.add(gid)
            self.io_used += io
            batch.append((r, inst, io))
            if q:
                heapq.heappush(heap, (q[0].arrival, gid))
        return batch

    def _launch(self, batch, stream_index, streams, now, nbatch):
        torch = self.torch
        st = streams[stream_index]
        plans, args, outs, io = [], [], [], 0
        with torch.cuda.stream(st):
            begin = torch.cuda.Event(enable_timing=True)
            begin.record(st)
            for r, inst, b in batch:
                prob = self.geoms[r.geometry]
                u = torch.mul(self.base_u[r.geometry], r.scale)
                p_out = torch.empty(prob.n[: prob.dim], dtype=torch.float64, device=self.device)
                u_out = torch.empty_like(u)
                f_out = torch.empty_like(u)
                plans.append(inst.plan)
                args.append(dict(dt=prob.dt, u_star=u, p=p_out, u=u_out, f=f_out))
                outs.append((r.rid, p_out, u_out, f_out, u))
                r.launched = now
                r.batch = nbatch
                io += b
            if self.batched:
                self.batcher.launch(plans, args, stream=st)
            else:
                for pl, a in zip(plans, args):
                    pl.project(a["u_star"], out=(a["p"], a["u"], a["f"]), stream=st)
            end = torch.cuda.Event(enable_timing=True)
            end.record(st)
        return _Batch([r for r, _, _ in batch], {r.geometry for r, _, _ in batch},
                      {id(inst) for _, inst, _ in batch}, stream_index, end, io, outs, begin)

    def run(self, trace):
        """Serve (arrival, geometry, scale) requests in real time; returns the requests with
        their launch and completion times."""
        torch = self.torch
        reqs = [Request(i, a, g, s) for i, (a, g, s) in enumerate(trace)]
        streams = [torch.cuda.Stream(self.device) for _ in range(self.max_inflight)]
        start = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        start.record(streams[0])
        queues = collections.defaultdict(collections.deque)
        waiting = 0
        inflight = []
        i = ndone = nbatch = 0
        self.host_s = 0.0          # host time assembling and launching batches
        self.gpu_s = 0.0           # sum of batch durations on the device (overlaps counted twice)
        self.shed = 0
        while ndone < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                if self.max_queue is not None and waiting >= self.max_queue:
                    reqs[i].shed = "queue"           # backpressure: refused on arrival
                    ndone += 1
                    self.shed += 1
                else:
                    queues[reqs[i].geometry].append(reqs[i])
                    waiting += 1
                i += 1
            if self.deadline_s is not None and waiting:
                for q in queues.values():
                    while q and now - q[0].arrival > self.deadline_s:
                        q.popleft().shed = "deadline"    # load shedding: dropped while waiting
                        waiting -= 1
                        ndone += 1
                        self.shed += 1
            for b in list(inflight):
                if b.end.query():
                    t_done = start.elapsed_time(b.end) * 1e-3
                    self.gpu_s += b.begin.elapsed_time(b.end) * 1e-3
                    for r in b.reqs:
                        r.done = t_done
                    if self.keep_outputs:
                        for rid, p_out, u_out, f_out, _ in b.outputs:
                            if self.keep_outputs is True or rid in self.keep_outputs:
                                self.outputs[rid] = (p_out.cpu(), u_out.cpu(), f_out.cpu())
                    self.io_used -= b.io_bytes
                    inflight.remove(b)
                    ndone += len(b.reqs)
            launched = False
            if len(inflight) < self.max_inflight and waiting:
                th = time.perf_counter()
                batch = self._assemble(queues, inflight)
                if batch:
                    used = {b.stream_index for b in inflight}
                    si = next(k for k in range(self.max_inflight) if k not in used)
                    inflight.append(self._launch(batch, si, streams, time.perf_counter() - t0, nbatch))
                    waiting -= len(batch)
                    nbatch += 1
                    launched = True
                self.host_s += time.perf_counter() - th
            if not launched:
                if not inflight and not waiting and i < len(reqs):
                    time.sleep(max(0.0, reqs[i].arrival - (time.perf_counter() - t0) - 50e-6))
                else:
                    time.sleep(20e-6)
        torch.cuda.synchronize(self.device)
        self.batches = nbatch
        return reqs

    def close(self):
        self.cache.close()
        if self.batcher is not None:
            self.batcher.close()


class _OwnedPlan:
    """A plan instance; the root also owns the device copy of its geometry's field."""

    def __init__(self, plan, fields, gid, root=True):
        self.plan, self.fields, self.gid, self.root = plan, fields, gid, root

    def nbytes(self):
        return self.plan.nbytes()

    def clone(self):
        return _OwnedPlan(self.plan.clone(), self.fields, self.gid, root=False)

    def close(self):
        self.plan.close()
        if self.root:
            self.fields.pop(self.gid, None)


def summarize(reqs, geoms):
    """Throughput and latency of a served trace (latency over the requests that were served;
    shed requests are counted apart)."""
    served = [r for r in reqs if not r.shed]
    out = {"requests": len(reqs), "served": len(served),
           "shed": {"queue": sum(r.shed == "queue" for r in reqs),
                    "deadline": sum(r.shed == "deadline" for r in reqs)}}
    if not served:
        return out
    lat = np.array([r.latency for r in served]) * 1e3
    cells = sum(geoms[r.geometry].num_cells for r in served)
    t_first = min(r.arrival for r in reqs)
    t_last = max(r.done for r in served)
    out.update({"cells": int(cells), "value": cells / (t_last - t_first), "unit": "grid-points/s",
                "seconds": round(t_last - t_first, 4),
                "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                               "p99": round(float(np.percentile(lat, 99)), 3),
                               "mean": round(float(lat.mean()), 3), "max": round(float(lat.max()), 3)},
                "cold_requests": int(sum(r.cold for r in served))})
    return out
