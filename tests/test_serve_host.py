"""Host-side logic of the server, without a GPU: the resident arena's slot ranges (first fit,
a molecule keeps its range while its size is unchanged, least recently used molecules not in
flight are evicted, nothing overlaps, nothing is placed when every holder is in flight)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def slots_cls():
    serve = pytest.importorskip("paper_2401_10462_gb300.serve")
    return serve._ArenaSlots


def _check_disjoint(s):
    spans = sorted((b, b + n) for b, n, _ in s.used.values())
    for (lo0, hi0), (lo1, _) in zip(spans, spans[1:]):
        assert hi0 <= lo1
    assert all(0 <= lo and hi <= s.capacity for lo, hi in spans)


def test_first_fit_reuse_and_lru(slots_cls):
    s = slots_cls(100)
    assert s.lookup("a", 40, set()) == (0, True)
    assert s.lookup("b", 30, set()) == (40, True)
    assert s.lookup("a", 40, set()) == (0, False)          # same size: same range, lists kept
    # no room for 50: the least recently used key not in flight ("b") goes
    assert s.lookup("c", 50, set()) == (40, True)
    assert "b" not in s.used
    # "a" in flight: the only victim is "c"; 60 fits once "c" is gone
    assert s.lookup("d", 60, {"a"}) == (40, True)
    assert "a" in s.used and "c" not in s.used
    # everything in flight and no room: not placed
    assert s.lookup("e", 10, {"a", "d"}) == (-1, False)
    # a new size for a key gives it a new range
    b, fresh = s.lookup("a", 20, {"d"})
    assert fresh and s.used["a"][1] == 20
    _check_disjoint(s)


def test_random_sequence_keeps_ranges_disjoint(slots_cls):
    rng = np.random.default_rng(0)
    s = slots_cls(1000)
    sizes = {}
    for step in range(3000):
        key = int(rng.integers(40))
        n = sizes.setdefault(key, int(rng.integers(1, 300)))
        if rng.random() < 0.02:
            sizes[key] = n = int(rng.integers(1, 300))
        busy = {int(k) for k in rng.choice(40, size=int(rng.integers(0, 4)), replace=False)} - {key}
        held = {k: s.used[k][:2] for k in busy if k in s.used}
        b, fresh = s.lookup(key, n, busy)
        if b >= 0:
            assert s.used[key][:2] == (b, n)
        else:
            assert key not in s.used
        for k, span in held.items():        # molecules in flight keep their ranges
            assert s.used[k][:2] == span
        _check_disjoint(s)
