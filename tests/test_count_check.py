"""Count check of a contour in the oracle: the stochastic trace estimate of the enclosed eigenvalue
count from S_0 (Section 2, CI eigensolvers; Eq. quadrature_appendix), the Ritz-count rule, and
the re-split of a contour that misses eigenvalues at a KDE cut (Algorithm 2).  No GPU."""
import numpy as np
import pytest

import oracle as O
import pencils as P


def fem1d_modes(n):
    """Closed-form eigenpairs of the 1D linear FEM pencil: lambda_k from `fem1d_eigenvalue`, nodal
    values of sin(k pi x) as eigenvectors (exact for this pencil), M-normalised."""
    K, M = P.fem1d(n)
    k = np.arange(1, n + 1)
    lam = P.fem1d_eigenvalue(k, n)
    x = np.arange(1, n + 1) / (n + 1)
    X = np.sin(np.pi * np.outer(x, k))
    Ms = M.to_scipy()
    X /= np.sqrt(np.einsum("ij,ij->j", X, Ms @ X))
    return K, M, lam, X


def trapezoid_filter(lam, c, R, N):
    """The scalar the N-node trapezoid rule on |z - c| = R (nodes at theta_j = 2 pi (j - 1/2) / N)
    applies to an eigencomponent at lam: summing the geometric series of 1 / (1 - x e^{-i theta_j})
    over the nodes leaves 1 / (1 + x^N), x = (lam - c) / R, for |x| < 1 and |x| > 1 alike."""
    x = (np.asarray(lam) - c) / R
    return 1.0 / (1.0 + x ** N)


def s0_of(K, M, V, c, R, N):
    z, w = O.trapezoid_nodes(c, R, N)
    Ks, Ms = K.to_scipy(), M.to_scipy()
    bw = O.bandwidth(Ks, Ms)
    X = [O.ShiftedSolver(Ks, Ms, zj, bw).solve(Ms @ V) for zj in z]
    return O.moments(X, z, w, c, R, 1)[0]


def test_filter_closed_form_at_the_centre_and_far_away():
    assert trapezoid_filter(0.0, 0.0, 1.0, 16) == 1.0
    assert trapezoid_filter(1.0, 0.0, 1.0, 16) == 0.5
    assert trapezoid_filter(3.0, 0.0, 1.0, 16) < 1e-7


def test_trace_estimate_is_the_filtered_projector_trace():
    """est = mean_l v_l^T S_0[:, l] with S_0 = sum_i rho(lam_i) x_i x_i^T M V: the oracle's
    quadrature, solves and moment sum against the closed-form modes and filter."""
    n, N = 120, 16
    K, M, lam, X = fem1d_modes(n)
    V = P.gaussian_block(n, 6, 11)
    a, b = 0.5 * (lam[9] + lam[10]), 0.5 * (lam[19] + lam[20])   # modes 11..20 inside
    c, R = 0.5 * (a + b), 0.5 * (b - a)
    est, se = O.trace_estimate(V, s0_of(K, M, V, c, R, N))
    rho = trapezoid_filter(lam, c, R, N)
    Ms = M.to_scipy()
    PV = X @ (rho[:, None] * (X.T @ (Ms @ V)))
    want = np.mean(np.einsum("il,il->l", V, PV))
    assert abs(est - want) <= 1e-9 * max(1.0, abs(want))
    assert se > 0
    # the filter's sum over the spectrum is the enclosed count, 10 modes, up to the leakage of the
    # two neighbours half a gap outside the circle
    assert abs(rho.sum() - 10.0) < 1.0


def test_trace_estimate_is_unbiased_with_the_stated_error():
    """Many columns: the estimate lies within 4 standard errors of tr P = sum rho(lam_i), and the
    standard error matches the Gaussian quadratic form's variance 2 ||(A + A^T)/2||_F^2 / L."""
    n, N, L = 60, 16, 4000
    K, M, lam, X = fem1d_modes(n)
    V = P.gaussian_block(n, L, 12)
    c, R = 0.5 * (lam[3] + lam[14]), 0.5 * (lam[14] - lam[3]) + 0.1 * (lam[15] - lam[14])
    est, se = O.trace_estimate(V, s0_of(K, M, V, c, R, N))
    rho = trapezoid_filter(lam, c, R, N)
    A = X @ np.diag(rho) @ X.T @ M.to_scipy().toarray()
    As = 0.5 * (A + A.T)
    sd = np.sqrt(2.0 * np.sum(As * As) / L)
    assert abs(est - rho.sum()) <= 4 * sd
    assert 0.85 < se / sd < 1.15


def test_count_miss_rules():
    th = np.array([1.0, 2.0, 3.0, 9.0])
    res = np.array([1e-12, 1e-12, 1e-3, 1e-12])
    # 2 converged on [0, 4]; the estimate 3 is within max(1.5, 3 se) of it
    assert not O.count_miss(3.0, 0.1, th, res, 2.0, 2.0, 4, 1e-10)
    # a deficit beyond max(1.5, 3 se)
    assert O.count_miss(3.6, 0.1, th, res, 2.0, 2.0, 4, 1e-10)
    assert not O.count_miss(3.6, 0.6, th, res, 2.0, 2.0, 4, 1e-10)
    # every Ritz value of the basis on the diameter: no spare direction
    assert O.count_miss(2.0, 0.1, th, np.full(4, 1e-12), 5.0, 5.0, 4, 1e-10)


def test_resplit_cuts_the_gap_and_keeps_the_inflation():
    th = np.r_[np.linspace(1.0, 1.2, 8), np.linspace(3.0, 3.3, 8), 7.5]
    (c0, r0, s0, e0), (c1, r1, s1, e1) = O.resplit(th, 2.0, 1.2 * 1.5, 0.5, 3.5)
    assert s0 == 0.5 and e1 == 3.5 and e0 == s1 and 1.2 < e0 < 3.0
    assert r0 == pytest.approx(1.2 * 0.5 * (e0 - s0)) and r1 == pytest.approx(1.2 * 0.5 * (e1 - s1))
    assert c0 == 0.5 * (s0 + e0) and c1 == 0.5 * (s1 + e1)
    # fewer than two distinct Ritz values inside: the midpoint
    (_, _, _, t), _ = O.resplit(np.array([2.0, 9.0]), 2.0, 1.5, 0.5, 3.5)
    assert t == 2.0


def test_judged_solve_recovers_a_saturated_contour():
    """24 eigenvalues inside one contour with a 12-column basis (L = 6, m = 2): without the check
    the contour cannot return them all; with it the contour is re-split until every piece fits,
    and every eigenvalue comes back at the closed-form value."""
    n = 300
    K, M = P.fem1d(n)
    lam = P.fem1d_eigenvalue(np.arange(1, 40), n)
    lo, hi = 0.5 * (lam[4] + lam[5]), 0.5 * (lam[28] + lam[29])   # modes 6..29
    V = P.gaussian_block(n, 6, 3)
    plain = O.ci_solve(K, M, lo, hi, V, ncontours=1, nodes=16, moments_m=2, tol=1e-10, max_outer=10)
    assert len(plain["evals"]) < 24
    r = O.ci_solve(K, M, lo, hi, V, ncontours=1, nodes=16, moments_m=2, tol=1e-10, max_outer=10,
                   judge=True, max_resplit=4)
    assert r["resplits"] >= 1 and all(st == 0 for st in r["status"])
    assert len(r["evals"]) == 24
    assert np.max(np.abs(r["evals"] - lam[5:29]) / lam[5:29]) < 1e-10
    cts = r["contours"]
    assert cts[0][2] == lo and cts[-1][3] == hi
    assert all(a[3] == b[2] for a, b in zip(cts, cts[1:]))
    assert len(r["estimates"]) == len(cts)
    # each final piece's estimate is within its own count check
    for (c, R, s, e), est in zip(cts, r["estimates"]):
        inside = np.sum((lam >= s) & (lam <= e))
        assert abs(est - inside) < 4.0


def test_resplit_keeps_a_quarter_on_each_side_of_a_widening_spectrum():
    """On eigenvalues whose gaps widen (1D Laplacian, lambda_k ~ k^2) the plain argmin of G_k sits
    in the widest gap at the top; the re-split searches between the quartiles instead."""
    lam = P.fem1d_eigenvalue(np.arange(1, 25), 300)
    s, e = 0.5 * lam[0], lam[-1] + 1.0
    (_, _, _, t), _ = O.resplit(lam, 0.5 * (s + e), 0.5 * (e - s), s, e)
    below = int(np.sum(lam < t))
    assert 6 <= below <= 18 and lam[6] <= t <= lam[17]
    plain = O.kde_cut(lam, s, e, 10.0)
    assert np.sum(lam < plain) > 18


# --------------------------------------------------------------------------- library vs oracle (host)

@pytest.fixture(scope="module")
def G():
    from paper_2511_01927_gb300 import build
    build.build()
    import paper_2511_01927_gb300 as G
    G.lib()
    return G


def test_library_count_miss_matches_oracle(G):
    rng = np.random.default_rng(21)
    for _ in range(300):
        q = int(rng.integers(1, 40))
        th = rng.uniform(0.0, 10.0, q)
        res = 10.0 ** rng.uniform(-14, -4, q)
        c, r = rng.uniform(2.0, 8.0), rng.uniform(0.5, 4.0)
        est, se = rng.uniform(0.0, 30.0), rng.uniform(0.0, 3.0)
        rank = int(rng.integers(1, 45))
        assert G.gcie_count_miss(est, se, th, res, c, r, rank, 1e-10) == O.count_miss(est, se, th, res, c, r, rank, 1e-10)


def test_library_resplit_matches_oracle(G):
    rng = np.random.default_rng(22)
    for k in range(40):
        s, e = 0.0, float(rng.uniform(5.0, 50.0))
        if k % 3 == 0:
            th = rng.uniform(s - 2.0, e + 2.0, int(rng.integers(0, 40)))
        elif k % 3 == 1:
            th = np.concatenate([x + 0.1 * rng.standard_normal(6) for x in rng.uniform(s, e, 4)])
        else:
            th = np.full(5, 0.5 * e)
        infl = 1.0 + float(rng.uniform(0.0, 0.3))
        c, R = 0.5 * (s + e), infl * 0.5 * (e - s)
        a = O.resplit(th, c, R, s, e)
        b = G.gcie_resplit(th, c, R, s, e)
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=0, atol=1e-9 * e)
    with pytest.raises(G.GcieError):
        G.gcie_resplit([1.0], 1.0, 0.5, 2.0, 1.0)
