"""The contour pipeline in the oracle, end to end on CPU: a predicted spectrum (the definition's
eigenvalues plus seeded noise, a stand-in for a trained predictor) -> contours (Algorithm 2, or a
fixed budget cut in gaps) -> the CI solve with the count check -> the definition's set."""
import numpy as np
import pytest

import oracle as O
import pencils as P


@pytest.fixture(scope="module")
def pencil():
    K, M = P.fem2d_p1_lognormal(24)
    lam, X = O.eigpairs_dense(K, M)
    i0, i1 = 10, 70
    lo, hi = 0.5 * (lam[i0 - 1] + lam[i0]), 0.5 * (lam[i1] + lam[i1 + 1])
    return K, M, lam, lo, hi, i0, i1


@pytest.mark.parametrize("layout", ["kde", "planned"])
def test_predicted_contours_give_the_definition(pencil, layout):
    K, M, lam, lo, hi, i0, i1 = pencil
    want = lam[i0:i1 + 1]
    spacing = (want[-1] - want[0]) / (want.size - 1)
    pred = want + np.random.default_rng(3).normal(0.0, 0.1 * spacing, want.size)
    if layout == "kde":
        cts = O.kde_contours(pred, nmin=10, nmax=50, w=10.0)
    else:
        cts = O.plan_contours(pred, lo, hi, 3)
    edges = [lo] + [c[1] for c in cts[:-1]] + [hi]
    contours = [(0.5 * (a + b), 0.5 * (b - a), a, b) for a, b in zip(edges[:-1], edges[1:])]
    V = P.gaussian_block(K.n, 16, 4)
    r = O.ci_solve(K, M, lo, hi, V, contours=contours, nodes=16, moments_m=2, tol=1e-10, judge=True)
    # the oracle has no stop rule for spurious Ritz values, so a contour can end flagged with one
    # still open inside it; the returned set is what must equal the definition
    assert len(r["evals"]) == want.size == O.count_in(K, M, lo, hi)
    assert np.max(np.abs(r["evals"] - want) / want) < 1e-10
    assert np.max(r["resid"]) <= 1e-10
