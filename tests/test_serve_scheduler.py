"""CPU checks of the serving scheduler (no GPU): every request is launched
once, a launch holds requests of one grid size in arrival order, the HBM
budget and the stream count are never exceeded, and the oldest waiting
request is never overtaken by a later one of another size."""
import random

import pytest

from paper_2405_14513_gb300 import serve


def _drive(trace, sched, seed=0):
    rng = random.Random(seed)
    in_flight, launches, order = [], [], []
    i = 0
    while i < len(trace) or sched.waiting or in_flight:
        # a few arrivals, then launch what may be launched, then finish some
        for _ in range(rng.randint(0, 3)):
            if i < len(trace):
                sched.arrive(trace[i])
                i += 1
        while True:
            oldest = sched.waiting[0] if sched.waiting else None
            nxt = sched.next_launch()
            if nxt is None:
                break
            slot, batch = nxt
            assert batch[0] is oldest, "the oldest waiting request leads the launch"
            assert len({r.ng for r in batch}) == 1 and len(batch) <= sched.max_batch[batch[0].ng]
            assert [r.rid for r in batch] == sorted(r.rid for r in batch)
            assert sched.used() <= sched.budget and sched.in_flight <= sched.streams
            in_flight.append(slot)
            launches.append(batch)
            order.extend(r.rid for r in batch)
        if in_flight and (rng.random() < 0.7 or i >= len(trace)):
            sched.done(in_flight.pop(rng.randrange(len(in_flight))))
        if not in_flight and not sched.waiting and i >= len(trace):
            break
    return launches, order


@pytest.mark.parametrize("streams,budget", [(4, 100), (1, 100), (3, 40)])
def test_every_request_served_once_within_budget(streams, budget):
    trace = serve.make_trace(200, seed=3)
    mb = {64: 16, 128: 8, 256: 4, 512: 1}
    sb = {64: 2, 128: 5, 256: 12, 512: 30}
    sched = serve.Scheduler(mb, sb, budget, streams)
    launches, order = _drive(trace, sched)
    assert sorted(order) == [r.rid for r in trace]
    assert not sched.waiting and sched.in_flight == 0


def test_slot_larger_than_budget_is_refused():
    with pytest.raises(ValueError):
        serve.Scheduler({64: 1}, {64: 10}, 5, 1)


def test_trace_recipe():
    tr = serve.make_trace(300, seed=0)
    assert len(tr) == 300 and all(b.t_arrive > a.t_arrive for a, b in zip(tr, tr[1:]))
    assert all(4 <= r.n_k1 <= 30 and 0 <= r.k1_lo and r.k1_lo + r.n_k1 <= 30 for r in tr)
    assert {r.l_max for r in tr} == {2, 4, 6}
    rate = len(tr) / tr[-1].t_arrive
    assert 15 < rate < 26                      # mean 20 requests/s
    frac = {ng: sum(r.ng == ng for r in tr) / len(tr) for ng in serve.GRIDS}
    assert abs(frac[64] - 0.4) < 0.08 and abs(frac[512] - 0.1) < 0.05
