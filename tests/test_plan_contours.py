"""Contours for a fixed budget, cut in gaps of a predicted spectrum: the oracle's `plan_contours`
against cases whose answer is fixed by the rule, and the library's host implementation (C ABI)
against the oracle, bit for bit (the rule is comparisons and midpoints).  No GPU."""
import ctypes as C

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def G():
    from paper_2511_01927_gb300 import build
    build.build()
    import paper_2511_01927_gb300 as G
    G.lib()
    return G


def spectra(seed, count=12):
    rng = np.random.default_rng(seed)
    for k in range(count):
        if k % 3 == 0:
            yield rng.uniform(0.0, 100.0, int(rng.integers(20, 400))), 0.0, 100.0
        elif k % 3 == 1:
            centres = np.sort(rng.uniform(0.0, 100.0, int(rng.integers(2, 9))))
            p = np.concatenate([c + rng.uniform(0.1, 2.0) * rng.standard_normal(int(rng.integers(3, 60)))
                                for c in centres])
            yield p, -5.0, 105.0
        else:   # predictions beyond the interval are ignored
            yield rng.uniform(-20.0, 120.0, int(rng.integers(10, 300))), 0.0, 100.0


def test_two_clusters_cut_in_the_middle_of_the_gap():
    pred = np.r_[np.linspace(1.0, 1.2, 10), np.linspace(3.0, 3.2, 10)]
    (a0, b0, _, _, n0), (a1, b1, _, _, n1) = O.plan_contours(pred, 0.0, 4.0, 2)
    assert (a0, b1) == (0.0, 4.0) and b0 == a1 == 0.5 * (1.2 + 3.0) and n0 == n1 == 10


def test_widest_gap_of_the_middle_half():
    """Even spacing with one wider gap among the middle half: the cut is in it.  A wider gap
    outside the middle half is not taken, so both halves keep a quarter of the predictions."""
    pred = np.r_[np.arange(50.0), np.arange(50.0) + 55.0]          # gap 49 .. 55
    (_, t, _, _, n0), _ = O.plan_contours(pred, -1.0, 110.0, 2)
    assert t == 52.0 and n0 == 50
    edge = np.r_[0.0, 30.0 + np.arange(40.0)]                     # widest gap 0 .. 30 at rank 0
    (_, t, _, _, n0), (_, _, _, _, n1) = O.plan_contours(edge, -1.0, 80.0, 2)
    assert 30.0 < t < 69.0 and min(n0, n1) >= 41 // 4


@pytest.mark.parametrize("budget", [1, 2, 5, 8, 13])
def test_budget_and_tiling(budget):
    for pred, lo, hi in spectra(3):
        out = O.plan_contours(pred, lo, hi, budget, alpha=0.25)
        assert 1 <= len(out) <= budget
        assert out[0][0] == lo and out[-1][1] == hi and all(x[1] == y[0] for x, y in zip(out, out[1:]))
        inside = np.sort(pred[(pred >= lo) & (pred <= hi)])
        assert sum(x[4] for x in out) == inside.size
        for a, b, c, r, n in out:
            assert c == 0.5 * (a + b) and r == 1.25 * 0.5 * (b - a)
        # every cut lies strictly inside a gap between consecutive predictions
        for a, b, _, _, _ in out[:-1]:
            j = np.searchsorted(inside, b)
            assert 0 < j < inside.size and inside[j - 1] < b < inside[j]
        if len(out) < budget:   # stopped early: no piece can be cut
            assert all(x[4] < 2 or np.unique(inside[(inside >= x[0]) & (inside <= x[1])]).size < 2 for x in out)


def test_empty_and_degenerate_predictions():
    assert O.plan_contours(np.zeros(0), 1.0, 2.0, 4) == [(1.0, 2.0, 1.5, 0.5, 0)]
    assert len(O.plan_contours(np.full(30, 1.5), 1.0, 2.0, 4)) == 1


def test_library_matches_oracle_exactly(G):
    for budget in (1, 3, 8, 9):
        for pred, lo, hi in spectra(4, 15):
            a = O.plan_contours(pred, lo, hi, budget, alpha=0.1)
            b = G.gcie_plan_contours(pred, lo, hi, budget, alpha=0.1)
            assert a == b
    assert G.gcie_plan_contours([], 1.0, 2.0, 3) == [(1.0, 2.0, 1.5, 0.5, 0)]


def test_library_rejects_bad_arguments(G):
    pred = np.linspace(0.0, 1.0, 50)
    for args in ((1.0, 0.0, 2), (0.0, 1.0, 0), (0.0, np.inf, 2)):
        with pytest.raises(G.GcieError) as e:
            G.gcie_plan_contours(pred, *args)
        assert e.value.code == 1
    with pytest.raises(G.GcieError):
        G.gcie_plan_contours(pred, 0.0, 1.0, 2, alpha=-0.5)
    with pytest.raises(G.GcieError):
        G.gcie_plan_contours(np.array([0.5, np.nan]), 0.0, 1.0, 2)
    # output capacity below the contour count: the count comes back, nothing is written
    out = (G._binding.Contour * 1)()
    counts = np.zeros(1, dtype=np.int32)
    n = C.c_int32(0)
    rc = G.lib().gcie_plan_contours(pred.ctypes.data, pred.size, 0.0, 1.0, 4, 0.0, C.cast(out, C.c_void_p),
                                    counts.ctypes.data, 1, C.byref(n))
    assert rc == 1 and n.value == 4 and counts[0] == 0
