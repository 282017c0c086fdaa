"""The serving loop's admission policy on the CPU (no device): a discrete-event
simulation drives `serving.Admission` with Poisson arrivals and service times,
and checks the invariants the GPU loop relies on: the memory budget and the
slot count are never exceeded, requests are admitted in arrival order and
never before they arrive, nothing is left behind, and with room to spare every
request is admitted the moment it arrives."""
import heapq

import numpy as np
import pytest

from paper_2111_11924_gb300 import serving as SV


def simulate(reqs, budget, slots, seed):
    """Admit and complete `reqs` (service time proportional to size, with
    jitter); returns the admission log [(time, request, slot)]."""
    rng = np.random.default_rng(seed)
    adm = SV.Admission(reqs, budget, slots)
    finish = []  # (time, slot)
    log, now = [], 0.0
    while not adm.done():
        while finish and finish[0][0] <= now:
            _, slot = heapq.heappop(finish)
            adm.complete(slot)
        for req, slot in adm.admit(now):
            assert adm.used <= budget and len(adm.inflight) <= slots
            assert now >= req.arrival
            log.append((now, req, slot))
            heapq.heappush(finish, (now + req.device_bytes() * 1e-9 * rng.uniform(0.5, 2.0), slot))
        if adm.done():
            break
        # the next event: a completion, or the head's arrival if it is still ahead
        events = ([finish[0][0]] if finish else []) + ([adm.next_arrival()] if adm.next_arrival() > now else [])
        assert events, "stalled with work left"
        now = min(events)
    return log, adm


def requests(count, seed, rate=2000.0, min_bytes=1024, max_bytes=2_000_000):
    return SV.poisson_requests(rate, count, seed, widths=(2048, 3072, 4096), min_bytes=min_bytes,
                               max_bytes=max_bytes)


@pytest.mark.parametrize("budget_x,slots,seed", [(1.0, 4, 1), (3.0, 32, 2), (50.0, 2, 3), (8.0, 16, 4)])
def test_admission_invariants(budget_x, slots, seed):
    """budget_x: the budget in units of the largest request."""
    reqs = requests(300, seed)
    budget = int(budget_x * max(r.device_bytes() for r in reqs))
    log, adm = simulate(reqs, budget, slots, seed)
    assert len(log) == len(reqs) and adm.done() and adm.used == 0
    order = [r.rid for _, r, _ in log]
    assert order == [r.rid for r in sorted(reqs, key=lambda r: r.arrival)]  # arrival order, no overtaking
    assert adm.peak_used <= budget and adm.peak_inflight <= slots
    times = [t for t, _, _ in log]
    assert times == sorted(times)


def test_room_to_spare_admits_on_arrival():
    reqs = requests(200, 7)
    log, adm = simulate(reqs, budget=10**12, slots=len(reqs), seed=7)
    assert all(t == r.arrival for t, r, _ in log)
    assert adm.peak_inflight > 1


def test_one_request_at_a_time_when_the_budget_fits_one():
    reqs = requests(60, 11, min_bytes=150_000, max_bytes=200_000)
    biggest = max(r.device_bytes() for r in reqs)
    assert 2 * min(r.device_bytes() for r in reqs) > biggest  # no two requests fit together
    log, adm = simulate(reqs, budget=biggest, slots=8, seed=11)
    assert adm.peak_inflight == 1 and len(log) == len(reqs)


def test_request_larger_than_the_budget_is_refused():
    reqs = requests(10, 13)
    with pytest.raises(ValueError):
        SV.Admission(reqs, budget_bytes=max(r.device_bytes() for r in reqs) - 1, slots=4)


def test_pack_batch_takes_the_oldest_and_its_kind():
    reqs = requests(40, 21)
    ready = sorted(reqs, key=lambda r: r.arrival)[:25]
    batch = SV.pack_batch(ready)
    head = ready[0]
    assert batch[0] is head
    assert all(r.op == head.op and r.nbits == head.nbits for r in batch)
    assert [r.rid for r in batch] == [r.rid for r in ready if r.op == head.op and r.nbits == head.nbits]
    # a chunk cap keeps the head and skips what does not fit
    cap = SV.num_chunks(head.msg_len, head.nbits)
    assert SV.pack_batch(ready, max_chunks=cap)[0] is head
    small = SV.pack_batch(ready, max_chunks=cap)
    assert sum(SV.num_chunks(r.msg_len, r.nbits) for r in small) <= max(cap, 0) or len(small) == 1
    assert SV.pack_batch([]) == []


def test_batch_layout_keeps_each_requests_key_binding():
    reqs = requests(12, 22, max_bytes=50_000)
    K = 7
    offsets, key_idx = SV.batch_layout(reqs, K)
    counts = [SV.num_chunks(r.msg_len, r.nbits) for r in reqs]
    assert list(np.diff(offsets)) == counts and offsets[0] == 0 and len(key_idx) == offsets[-1]
    for i, (a, b) in enumerate(zip(offsets[:-1], offsets[1:])):
        assert list(key_idx[a:b]) == [t % K for t in range(b - a)]  # chunk t of every request: key t mod K
        for c in (a, b - 1):
            assert SV.request_of_chunk(offsets, c) == i


def test_dispatch_keeps_priority_lanes_for_small_batches():
    """Lanes 0-1 are priority lanes for batches of at most 100 chunks: a small
    head takes one, a large head takes an ordinary lane or waits, and when
    only priority lanes are free the oldest small requests go ahead of a
    large one; without priority lanes any lane takes the head."""
    def req(rid, n, nbits=1024):
        return SV.Request(rid=rid, op="decrypt", nbits=nbits, arrival=rid, msg_len=n * 127, payload=None)

    big, small1, small2 = req(0, 500), req(1, 10), req(2, 20)
    lane, batch = SV.dispatch([small1, big], [0, 1, 2, 3], 2, 100, 1 << 30)
    assert lane in (0, 1) and [r.rid for r in batch] == [1]
    lane, batch = SV.dispatch([big, small1], [0, 1, 2, 3], 2, 100, 1 << 30)
    assert lane in (2, 3) and 0 in [r.rid for r in batch]
    lane, batch = SV.dispatch([big, small1, small2], [0, 1], 2, 100, 1 << 30)
    assert lane in (0, 1) and [r.rid for r in batch] == [1, 2]
    assert SV.dispatch([big], [0, 1], 2, 100, 1 << 30) is None
    lane, batch = SV.dispatch([small1], [2], 2, 100, 1 << 30)  # no priority lane free: an ordinary one
    assert lane == 2 and [r.rid for r in batch] == [1]
    lane, batch = SV.dispatch([big, small1], [0, 1, 2], 0, 100, 1 << 30)
    assert lane == 2 and [r.rid for r in batch] == [0, 1]
