"""Host logic of the serving loop's plan cache (no GPU): least-recently-used eviction within the
byte budget, plans in flight never evicted, refusal when nothing can be freed."""
import pytest

from paper_2304_14690_gb300 import pc
from paper_2304_14690_gb300.serving import PlanCache


class FakePlan:
    closed = []

    def __init__(self, gid, size):
        self.gid, self.size = gid, size

    def nbytes(self):
        return self.size

    def clone(self):
        return FakePlan(self.gid, 1)

    def close(self):
        FakePlan.closed.append(self.gid)


def make_cache(budget, sizes):
    FakePlan.closed = []

    def make(gid, free):
        if sizes[gid] > free:
            raise pc.PcError(pc.PC_ERR_BUDGET, "too big")
        return FakePlan(gid, sizes[gid])
    return PlanCache(budget, make)


def test_builds_then_hits():
    c = make_cache(100, {0: 40, 1: 40})
    p, cold = c.get(0, set())
    assert cold and p.gid == 0 and c.used == 40
    p2, cold = c.get(0, set())
    assert p2 is p and not cold and c.builds == 1


def test_lru_eviction_respects_budget():
    c = make_cache(100, {0: 40, 1: 40, 2: 40})
    c.get(0, set())
    c.get(1, set())
    c.get(0, set())                       # 0 is now the most recent
    p, cold = c.get(2, set())
    assert cold and FakePlan.closed == [1] and c.used == 80 and c.evictions == 1
    assert c.resident(0) and c.resident(2) and not c.resident(1)


def test_busy_plans_are_kept():
    c = make_cache(100, {0: 40, 1: 40, 2: 40})
    c.get(0, set())
    c.get(1, set())
    assert c.get(2, keep={0, 1}) is None  # both resident plans are in flight
    assert FakePlan.closed == [] and c.used == 80
    p, _ = c.get(2, keep={1})
    assert FakePlan.closed == [0] and c.resident(2)


def test_reserve_counts_against_budget():
    c = make_cache(100, {0: 40, 1: 40})
    c.get(0, set())
    assert c.get(1, keep={0}, reserve=30) is None
    p, _ = c.get(1, keep={0}, reserve=10)
    assert c.used == 80


def test_other_errors_propagate():
    def make(gid, free):
        raise pc.PcError(pc.PC_ERR_WLS_SINGULAR, "bad")
    c = PlanCache(100, make)
    with pytest.raises(pc.PcError):
        c.get(0, set())


def test_make_room_evicts_idle_only():
    c = make_cache(100, {0: 40, 1: 40})
    c.get(0, set())
    c.get(1, set())
    assert not c.make_room(30, keep={0, 1})
    assert c.make_room(30, keep={1}) and FakePlan.closed == [0] and c.used == 40


def test_instances_clone_into_free_budget_only():
    FakePlan.closed = []
    sizes = {0: 40, 1: 40}

    def make(gid, free):
        if sizes[gid] > free:
            raise pc.PcError(pc.PC_ERR_BUDGET, "too big")
        return FakePlan(gid, sizes[gid])
    c = PlanCache(100, make, max_instances=3, clone_bytes=lambda gid: 1)
    a, cold = c.acquire(0, busy=set(), keep=set())
    assert cold and c.used == 40
    b, cold = c.acquire(0, busy={id(a)}, keep={0})          # the root is busy: a clone
    assert b is not a and not cold and c.clones == 1 and c.used == 41
    c3, _ = c.acquire(0, busy={id(a), id(b)}, keep={0})
    assert c.acquire(0, busy={id(a), id(b), id(c3)}, keep={0}) is None   # max_instances
    c.get(1, set())
    assert c.used == 40 + 2 + 40
    big = PlanCache(50, make, max_instances=2, clone_bytes=lambda gid: 20)
    r, _ = big.acquire(0, set(), set())
    assert big.acquire(0, {id(r)}, {0}) is None            # no free budget: no clone, no eviction
    assert FakePlan.closed == []
