"""Contour construction from a predicted spectrum (Algorithm 2, Section 4.2): the oracle against
properties the algorithm fixes, and the library's host implementation (C ABI) against the oracle.
No GPU."""
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
    """Seeded predicted spectra: uniform stretches and Gaussian clusters of mixed widths."""
    rng = np.random.default_rng(seed)
    for k in range(count):
        if k % 2 == 0:
            yield rng.uniform(0.0, 100.0, int(rng.integers(30, 400)))
        else:
            centres = np.sort(rng.uniform(0.0, 200.0, int(rng.integers(2, 8))))
            yield np.concatenate([c + rng.uniform(0.1, 2.0) * rng.standard_normal(int(rng.integers(5, 80)))
                                  for c in centres])


def members(pred, lo, hi, last):
    return int(np.sum((pred >= lo) & ((pred <= hi) if last else (pred < hi))))


# --------------------------------------------------------------------------- oracle pins

def test_mirror_clusters_cut_at_the_gap_centre():
    """Two mirror-image clusters: G_k is symmetric about the middle of the gap, so the one split
    of Algorithm 2 lies there and each contour takes one cluster."""
    rng = np.random.default_rng(1)
    d = 0.02 * rng.standard_normal(20)
    pred = np.r_[1.0 + d, 2.0 - d]
    out = O.kde_contours(pred, nmin=10, nmax=30, w=10.0)
    assert len(out) == 2
    # a minimiser found by comparing values of G_k is fixed only to about sqrt(machine eps) of the
    # scale: G_k is flat to second order at its minimum
    assert abs(out[0][1] - 1.5) <= 1e-7 and out[0][4] == out[1][4] == 20


def test_sparsity_kernel_width():
    """Each prediction adds a Gaussian of height 1 and e-folding half-width (b - a) / sqrt(w) to G_k
    (Eq. 6): 1 at the prediction, 1/e that far from it, and the sum of the two for two predictions."""
    a, b, w = 2.0, 6.0, 16.0
    lam = np.array([3.0])
    assert O.kde_sparsity(np.array([3.0]), lam, a, b, w)[0] == 1.0
    e = O.kde_sparsity(np.array([2.0, 4.0]), lam, a, b, w)
    assert np.allclose(e, np.exp(-1.0), rtol=1e-15)
    two = O.kde_sparsity(np.array([4.0]), np.array([3.0, 5.0]), a, b, w)[0]
    assert abs(two - 2 * np.exp(-1.0)) <= 1e-15


def test_wider_gap_is_cut_first():
    """Three equal clusters at 0, 1 and 3: the sparsest point of the whole range lies in the wide
    gap, so one split leaves 40 | 20. With a lower cap the left part [min - eps, t) is split again;
    its kernels are a third of its width wide at w = 10, too wide to resolve the clusters at 0 and 1
    (G_k is lowest at the ends), and at w = 40 the narrow gap is cut."""
    rng = np.random.default_rng(5)
    pred = np.concatenate([c + 0.01 * rng.standard_normal(20) for c in (0.0, 1.0, 3.0)])
    one = O.kde_contours(pred, nmin=10, nmax=50, w=10.0)
    assert [x[4] for x in one] == [40, 20] and 1.5 < one[0][1] < 2.9
    three = O.kde_contours(pred, nmin=10, nmax=30, w=40.0)
    assert [x[4] for x in three] == [20, 20, 20] and 0.1 < three[0][1] < 0.9 and 1.5 < three[1][1] < 2.9


def test_cut_is_a_minimum_of_the_sparsity_function():
    """The split point minimises G_k (Eq. 6) over the predictions' range of the interval (Algorithm 2:
    the sparsest location): no grid cell centre and no point near it has a smaller G_k. With a wide
    kernel over an even spread of predictions G_k falls towards both ends, and the minimum is at the
    last cell next to an end rather than a local minimum in a gap."""
    for pred in spectra(2, 6):
        p = np.sort(pred)
        a, b = p[0], p[-1]
        t = O.kde_cut(p, a, b, 10.0)
        g = lambda x: O.kde_sparsity(np.atleast_1d(x), p, a, b, 10.0)  # noqa: E731
        assert p[0] < t < p[-1]
        h = (p[-1] - p[0]) / O.KDE_GRID
        grid = p[0] + (np.arange(O.KDE_GRID) + 0.5) * h
        gt = g(t)[0]
        assert gt <= np.min(g(grid)) + 1e-12
        i = int(np.argmin(g(grid)))
        near = np.linspace(grid[max(i - 1, 0)], grid[min(i + 1, O.KDE_GRID - 1)], 401)
        assert gt <= np.min(g(near)) + 1e-12


@pytest.mark.parametrize("nmin,nmax", [(10, 50), (5, 20), (0, 30)])
def test_partition_invariants(nmin, nmax):
    """The contours tile [min - eps, max + eps] without gaps, every prediction is in exactly one of
    them, each holds at most nmax, and at least nmin when more than one contour is left."""
    for pred in spectra(3):
        beta, alpha = 0.05, 0.2
        out = O.kde_contours(pred, nmin=nmin, nmax=nmax, w=10.0, alpha=alpha, beta=beta)
        eps = beta * (pred.max() - pred.min())
        assert out[0][0] == pred.min() - eps and out[-1][1] == pred.max() + eps
        for (lo, hi, c, r, n), nxt in zip(out, out[1:] + [None]):
            if nxt is not None:
                assert hi == nxt[0]
            assert n == members(pred, lo, hi, nxt is None)
            assert c == 0.5 * (lo + hi) and r == (1 + alpha) * 0.5 * (hi - lo)
            assert n <= nmax
            if len(out) > 1:
                assert n >= nmin
        assert sum(x[4] for x in out) == pred.size


def test_one_contour_when_everything_fits_and_equal_predictions():
    pred = np.linspace(3.0, 7.0, 40)
    (lo, hi, c, r, n), = O.kde_contours(pred, nmin=10, nmax=40, w=10.0, alpha=0.5, beta=0.1)
    assert (lo, hi, n) == (3.0 - 0.4, 7.0 + 0.4, 40) and r == 1.5 * 0.5 * (hi - lo)
    same = np.full(70, 2.5)
    assert O.kde_contours(same, nmin=10, nmax=50)[0][4] == 70


# --------------------------------------------------------------------------- library vs oracle

def test_library_matches_oracle(G):
    for pred in spectra(4, 16):
        a = O.kde_contours(pred, 10, 50, 10.0, 0.1, 0.02)
        b = G.gcie_kde_contours(pred, 10, 50, 10.0, 0.1, 0.02)
        assert len(a) == len(b)
        assert [x[4] for x in a] == [y[4] for y in b]
        span = pred.max() - pred.min()
        # cut points in wide flat gaps are ill-conditioned in the last digits; the partition of the
        # predictions (the counts) is what must agree exactly
        for x, y in zip(a, b):
            assert abs(x[0] - y[0]) <= 1e-6 * span and abs(x[1] - y[1]) <= 1e-6 * span
            assert abs(x[2] - y[2]) <= 1e-6 * span and abs(x[3] - y[3]) <= 1e-6 * span


def test_library_rejects_bad_arguments(G):
    pred = np.linspace(0.0, 1.0, 100)
    for kw in (dict(nmin=20, nmax=10), dict(w=0.0), dict(alpha=-1.0), dict(nmax=0)):
        with pytest.raises(G.GcieError) as e:
            G.gcie_kde_contours(pred, **kw)
        assert e.value.code == 1
    with pytest.raises(G.GcieError):
        G.gcie_kde_contours(np.array([0.0, np.nan, 1.0]))
    # too small an output array: the count comes back, nothing is written
    lib = G.lib()
    out = (G._binding.Contour * 1)()
    counts = np.zeros(1, dtype=np.int32)
    n = C.c_int32(0)
    rc = lib.gcie_kde_contours(pred.ctypes.data, pred.size, 2, 10, 10.0, 0.0, 0.0, C.cast(out, C.c_void_p),
                               counts.ctypes.data, 1, C.byref(n))
    assert rc == 1 and n.value > 1 and counts[0] == 0
