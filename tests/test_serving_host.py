"""Host-side logic of the serving scheduler (no GPU): first-come first-served admission under a memory
budget and a slot limit."""
from paper_2412_12360_b300.serve import admit_count


def test_admission_respects_budget_slots_and_order():
    assert admit_count([10, 10, 10], 0, 0, 25, 8) == 2
    assert admit_count([10, 10, 10], 0, 0, 100, 2) == 2
    assert admit_count([10, 10, 10], 1, 0, 100, 2) == 1
    assert admit_count([30, 5, 5], 0, 0, 25, 8) == 0          # the head blocks smaller requests behind it
    assert admit_count([5, 30, 5], 0, 0, 25, 8) == 1
    assert admit_count([], 0, 0, 100, 8) == 0
    assert admit_count([10], 0, 95, 100, 8) == 0
    assert admit_count([5, 5], 0, 90, 100, 8) == 2


def test_admission_simulated_stream_never_exceeds_budget():
    import random
    rng = random.Random(3)
    budget, slots = 100, 4
    queue = [rng.randint(5, 60) for _ in range(200)]
    inflight = []
    done = 0
    while queue or inflight:
        n = admit_count(queue, len(inflight), sum(inflight), budget, slots)
        inflight += queue[:n]
        del queue[:n]
        assert sum(inflight) <= budget and len(inflight) <= slots
        if inflight:
            inflight.pop(rng.randrange(len(inflight)))
            done += 1
    assert done == 200
