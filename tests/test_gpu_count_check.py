"""The count check on the CUDA path (through the C ABI) against the oracle and closed forms: the
trace estimate of S_0 (Section 2, CI eigensolvers) and the recovery of a contour whose basis is
too small for the eigenvalues it encloses, by re-splitting at a KDE cut (Algorithm 2).

Tolerances: the trace estimate within 1e-7 relative of the oracle's on the same V (S_0 differs by
the shifted solves' 1e-11 residual); eigenpairs as in the other solve tests (values 1e-10 relative
to the closed form, |x^T M x_ref| > 1 - 1e-9)."""
import numpy as np
import pytest

import oracle as O
import pencils as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2511_01927_gb300 import build
    build.build()
    import paper_2511_01927_gb300 as G
    return G


@pytest.fixture(scope="module")
def ctx(G):
    h = G.gcie_create(0)
    yield h
    G.gcie_destroy(h)


def sines(n, ks, M):
    h = 1.0 / (n + 1)
    X = np.sin(np.outer(np.arange(1, n + 1), ks) * np.pi * h)
    return X / np.sqrt(np.einsum("ij,ij->j", X, M.to_scipy() @ X))


def test_trace_estimate_matches_oracle(G, ctx):
    K, M, spec = P.workload("fem1d-n2000")
    V = P.gaussian_block(K.n, spec["L"], 1)
    r = G.gcie_solve(ctx, K, M, spec["lo"], spec["hi"], nodes=16, moments=2, nuniform=1, V0=V, tol=1e-10, judge=1)
    tr = {}
    ro = O.ci_solve(K, M, spec["lo"], spec["hi"], V, ncontours=1, nodes=16, moments_m=2, tol=1e-10, trace=tr,
                    judge=True)
    assert r["resplits"] == ro["resplits"] == 0
    est, se = O.trace_estimate(V, tr["contours"][0]["S"][0])
    assert abs(r["count_estimate"][0] - est) <= 1e-7 * abs(est)
    assert abs(ro["estimates"][0] - est) == 0.0
    assert len(r["evals"]) == spec["count"]
    # without the check the estimate is still formed (the stall rule uses it), from the same solves
    plain = G.gcie_solve(ctx, K, M, spec["lo"], spec["hi"], nodes=16, moments=2, nuniform=1, V0=V, tol=1e-10)
    assert abs(plain["count_estimate"][0] - r["count_estimate"][0]) <= 1e-12 * abs(est)
    assert plain["resplits"] == 0
    assert plain["contours"] == [(0.5 * (spec["lo"] + spec["hi"]), 0.5 * (spec["hi"] - spec["lo"]), spec["lo"],
                                  spec["hi"])]


def test_judged_solve_recovers_a_saturated_contour(G, ctx):
    """24 eigenvalues in one contour with a 12-column basis (L = 6, m = 2): the check re-splits it
    until every piece fits, and all 24 come back at the closed-form values and vectors."""
    n = 300
    K, M = P.fem1d(n)
    lam = P.fem1d_eigenvalue(np.arange(1, 40), n)
    lo, hi = 0.5 * (lam[4] + lam[5]), 0.5 * (lam[28] + lam[29])
    V = P.gaussian_block(n, 6, 3)
    plain = G.gcie_solve(ctx, K, M, lo, hi, nodes=16, moments=2, nuniform=1, V0=V, tol=1e-10, allow_noconv=True)
    assert len(plain["evals"]) < 24
    r = G.gcie_solve(ctx, K, M, lo, hi, nodes=16, moments=2, nuniform=1, V0=V, tol=1e-10, judge=1, max_resplit=4)
    assert r["rc"] == 0 and r["resplits"] >= 1 and all(s == 0 for s in r["status"])
    assert len(r["evals"]) == 24
    want = lam[5:29]
    assert np.max(np.abs(r["evals"] - want) / want) < 1e-10
    assert np.max(r["resid"]) <= 1e-10
    dots = np.abs(np.einsum("ij,ij->j", r["evecs"], M.to_scipy() @ sines(n, np.arange(6, 30), M)))
    assert np.min(dots) > 1 - 1e-9
    cts = r["contours"]
    assert len(cts) == r["resplits"] + 1 == len(r["count_estimate"]) == len(r["status"])
    assert cts[0][2] == lo and cts[-1][3] == hi and all(a[3] == b[2] for a, b in zip(cts, cts[1:]))
    assert set(r["contour_of"].tolist()) <= set(range(len(cts)))
    for (c, R, s, e), est in zip(cts, r["count_estimate"]):
        assert abs(est - np.sum((lam >= s) & (lam <= e))) < 4.0
    # the oracle with the same check returns the same set
    ro = O.ci_solve(K, M, lo, hi, V, ncontours=1, nodes=16, moments_m=2, tol=1e-10, judge=True, max_resplit=4)
    assert np.max(np.abs(np.sort(ro["evals"]) - r["evals"]) / want) < 1e-10


def test_judge_rejects_bad_options(G, ctx):
    K, M = P.fem1d(50)
    for kw in (dict(judge=2), dict(max_resplit=-1), dict(max_resplit=17)):
        with pytest.raises(G.GcieError) as e:
            G.gcie_solve(ctx, K, M, 1.0, 100.0, L=8, **kw)
        assert e.value.code == 1


def test_judge_reports_a_miss_left_at_the_last_level(G, ctx):
    """The saturated contour with no re-split allowed: the check fails, the contour keeps what it
    found and the solve reports GCIE_ENOCONV for it."""
    n = 300
    K, M = P.fem1d(n)
    lam = P.fem1d_eigenvalue(np.arange(1, 40), n)
    lo, hi = 0.5 * (lam[4] + lam[5]), 0.5 * (lam[28] + lam[29])
    V = P.gaussian_block(n, 6, 3)
    r = G.gcie_solve(ctx, K, M, lo, hi, nodes=16, moments=2, nuniform=1, V0=V, tol=1e-10, judge=1, max_resplit=0,
                     allow_noconv=True)
    assert r["rc"] == 5 and r["status"] == [5] and r["resplits"] == 0
    assert len(r["evals"]) < 24 and r["count_estimate"][0] > len(r["evals"]) + 1.5


def test_stalled_contour_is_flagged(G, ctx):
    """A contour that stops on the stall rule before the FEAST cap reports GCIE_ENOCONV unless the count
    check agrees that the unconverged Ritz values are spurious.  Here the basis (L = 8, one moment) is far
    smaller than the 50 eigenvalues the contour encloses: no Ritz pair converges, the stall rule ends
    the contour early, and every Ritz value lies on the diameter (no spare direction), so the check
    flags it even with the judge off.  Whatever pairs it returns are eigenpairs of the definition."""
    K, M, spec = P.workload("fem2d-p1-40")
    V = P.gaussian_block(K.n, 8, 3)
    r = G.gcie_solve(ctx, K, M, spec["lo"], spec["hi"], nodes=16, moments=1, nuniform=1, V0=V, L=8, max_outer=20,
                     allow_noconv=True)
    assert r["rc"] == 5 and r["status"] == [5]
    assert r["iters"][0] < 20                      # stopped by the stall rule, not by the cap
    assert np.isfinite(r["count_estimate"][0])
    if len(r["evals"]):
        lam, _ = O.eigpairs_dense(K, M, spec["lo"], spec["hi"])
        assert np.max(r["resid"]) <= 1e-10
        assert np.all(np.min(np.abs(r["evals"][:, None] - lam[None, :]), axis=1) <= 1e-10 * np.abs(r["evals"]))
