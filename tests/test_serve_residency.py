"""Residency accounting of the server (host logic, no GPU): every resident
molecule is charged the bytes it was admitted with and exactly that is
returned on eviction, so the budget never drifts and a molecule that fits
alone is always admitted once nothing is in flight."""
import random

from paper_2404_09452_gb300.serve import Residency


def test_mixed_sizes_never_drift():
    rng = random.Random(7)
    budget = 1000
    r = Residency(budget)
    sizes = {m: rng.choice([5, 20, 80, 400, 900]) for m in range(30)}
    for _ in range(5000):
        m = rng.randrange(30)
        if r.touch(m):
            continue
        busy = set(rng.sample(sorted(r.bytes), k=min(len(r.bytes), rng.randrange(3))))
        ok, evicted = r.admit(m, sizes[m], busy)
        assert not (set(evicted) & busy)
        assert r.used == sum(r.bytes.values())
        assert r.used <= budget or len(r.bytes) == 1
        if not busy:
            assert ok


def test_big_after_small_and_back():
    """The case that used to stall: a big molecule evicted on behalf of a small
    one must give back all of its bytes."""
    r = Residency(100)
    assert r.admit("big", 90, set())[0]
    assert r.admit("small", 20, set()) == (True, ["big"])
    assert r.used == 20
    assert r.admit("big2", 95, set()) == (True, ["small"])
    assert r.used == 95


def test_busy_blocks_eviction_and_oversize_runs_alone():
    r = Residency(100)
    assert r.admit("a", 60, set())[0]
    assert r.admit("b", 60, {"a"}) == (False, [])
    assert r.admit("huge", 150, set()) == (True, ["a"])
    assert list(r.bytes) == ["huge"] and r.used == 150
