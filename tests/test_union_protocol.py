"""Interleaving check of the concurrent Rem union (Algorithm 2 with Algorithm 8's
concurrency), step for step as the GPU kernels (rem_unite_g and the tile pass) and the
oracle's PARemSP merger run it: two loads of the parents, then one compare-and-swap that
either links a root or splices a non-root, each from exactly the value read; a failed
compare-and-swap re-reads.  Every interleaving of single memory accesses of a few
concurrent unions is explored (sequential consistency), and the final forest must have
the partition of the initial forest plus the united pairs.

The regression scenario is a lost union seen on GB300 (about 1% of labellings of large
near-critical images): a splice that lowers a parent it did not read (an atomic minimum,
or the paper's unlocked write) detaches a node that another union had just attached to a
root, and no union reconnects that root.  The negative control runs the same scenario
with atomic-minimum splices and must find the lost union, which shows the search reaches
the failing interleaving.
"""
import random

import pytest

# node ids of the scenario: D=0 < O=1 < C=2 < B=3 < A=4 < X=5, X starting as a child of B
SCENARIO_P0 = (0, 1, 2, 3, 4, 3)
SCENARIO_UNIONS = ((4, 3), (4, 0), (4, 2), (4, 1), (5, 4))


def _step(P, st, splice_cas):
    """One memory access of one union.  st = (rx, ry, pc, px, py); returns (P, st or None)."""
    rx, ry, pc, px, py = st
    if pc == 0:  # load p[rx]
        return P, (rx, ry, 1, P[rx], 0)
    if pc == 1:  # load p[ry], decide
        py = P[ry]
        if px == py:
            return P, None
        return P, (rx, ry, 2 if px > py else 3, px, py)
    # pc 2: write p[rx] <- py (root link or splice); pc 3: write p[ry] <- px
    r, old, new = (rx, px, py) if pc == 2 else (ry, py, px)
    Pl = list(P)
    if splice_cas or old == r:  # a root link is always a compare-and-swap
        if Pl[r] != old:
            return P, (rx, ry, 0, 0, 0)
        Pl[r] = new
    else:
        Pl[r] = min(Pl[r], new)
    if old == r:
        return tuple(Pl), None
    return tuple(Pl), ((old, ry, 0, 0, 0) if pc == 2 else (rx, old, 0, 0, 0))


def _roots(P):
    out = []
    for v in range(len(P)):
        for _ in range(len(P) + 1):
            if P[v] == v:
                break
            v = P[v]
        else:
            raise AssertionError("cycle")
        out.append(v)
    return tuple(out)


def _expected(P0, unions):
    par = list(range(len(P0)))

    def f(v):
        while par[v] != v:
            v = par[v]
        return v
    for a, b in list(enumerate(P0)) + list(unions):
        ra, rb = f(a), f(b)
        if ra != rb:
            par[max(ra, rb)] = min(ra, rb)
    return tuple(f(v) for v in range(len(P0)))


def _same_partition(r1, r2):
    m = {}
    return all(m.setdefault(a, b) == b for a, b in zip(r1, r2)) and len(set(r1)) == len(set(r2))


def explore(P0, unions, splice_cas=True, cap=2_000_000):
    """Depth-first search over every interleaving; returns (failing final forest or None,
    number of states)."""
    exp = _expected(P0, unions)
    start = (tuple(P0), tuple((x, y, 0, 0, 0) for x, y in unions))
    seen, stack = set(), [start]
    while stack:
        P, sts = stack.pop()
        if (P, sts) in seen:
            continue
        seen.add((P, sts))
        assert len(seen) <= cap, "state cap"
        live = [i for i, s in enumerate(sts) if s is not None]
        if not live:
            if not _same_partition(_roots(P), exp):
                return P, len(seen)
            continue
        for i in live:
            P2, s2 = _step(P, sts[i], splice_cas)
            stack.append((P2, sts[:i] + (s2,) + sts[i + 1:]))
    return None, len(seen)


def test_regression_scenario_every_interleaving_is_correct():
    bad, n = explore(SCENARIO_P0, SCENARIO_UNIONS)
    assert bad is None, bad
    assert n > 10_000  # the search really branched


def test_negative_control_atomic_min_splice_loses_a_union():
    bad, _ = explore(SCENARIO_P0, SCENARIO_UNIONS, splice_cas=False)
    assert bad is not None
    # node O (1) ends up a root of its own although it was united with A (4)
    assert _roots(bad)[1] != _roots(bad)[4]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_small_forests(seed):
    rng = random.Random(seed)
    for _ in range(40):
        n = rng.randrange(3, 7)
        P0 = list(range(n))
        for v in range(1, n):
            if rng.random() < 0.5:
                P0[v] = rng.randrange(0, v)
        unions = tuple((rng.randrange(n), rng.randrange(n)) for _ in range(rng.randrange(2, 5)))
        bad, _ = explore(tuple(P0), unions)
        assert bad is None, (P0, unions, bad)
