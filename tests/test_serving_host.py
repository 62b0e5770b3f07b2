"""Host-side logic of the serving scheduler (no GPU): first-come first-served admission under a memory
budget and a slot limit, and the grouping of running requests by the bytes a step moves."""
from paper_2412_12360_b300.serve import admit_count, partition, step_bytes


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


def test_partition_keeps_order_budget_and_group_size():
    assert partition([10, 10, 10, 10], 25, 8) == [[0, 1], [2, 3]]
    assert partition([10, 30, 5], 25, 8) == [[0], [1], [2]]        # a request above the budget goes alone
    assert partition([1] * 10, 0, 8) == [list(range(8)), [8, 9]]   # no budget: groups of max_group
    assert partition([5] * 5, 100, 2) == [[0, 1], [2, 3], [4]]
    assert partition([], 10, 8) == []
    import random
    rng = random.Random(4)
    for _ in range(200):
        sizes = [rng.randint(1, 50) for _ in range(rng.randint(1, 12))]
        budget, mg = rng.randint(10, 120), rng.randint(1, 8)
        groups = partition(sizes, budget, mg)
        assert [i for g in groups for i in g] == list(range(len(sizes)))
        for g in groups:
            assert len(g) <= mg and (len(g) == 1 or sum(sizes[i] for i in g) <= budget)


def test_step_bytes_counts_52_bytes_per_cell():
    class Sc:
        n = (64, 32, 16)
    assert step_bytes(Sc()) == 52 * 64 * 32 * 16
