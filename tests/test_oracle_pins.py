"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks one oracle function against something other than itself: a closed form,
an identity, an invariant, brute force, or a library routine on a special case.  The targets
are chosen so that a plausible slip (wrong sign of a weight, dropped factor 2, wrong node angle,
transposed operand, missing M in the right-hand side) fails at least one test; the
`test_*_detects_*` tests plant such slips in a copy of the oracle's arithmetic and check that
the pin rejects them.
"""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

import oracle as O
import pencils as P


# --------------------------------------------------------------------------- helpers

def fem1d_exact(n, ks):
    """Closed-form eigenpairs of the 1D linear-FEM pencil: lambda_k and x_i = sin(k pi i h),
    M-normalised, largest entry positive."""
    K, M = P.fem1d(n)
    lam = P.fem1d_eigenvalue(np.asarray(ks), n)
    h = 1.0 / (n + 1)
    i = np.arange(1, n + 1)
    X = np.sin(np.outer(i, np.asarray(ks)) * np.pi * h)
    Ms = M.to_scipy()
    X = X / np.sqrt(np.einsum("ij,ij->j", X, Ms @ X))
    return K, M, lam, O.fix_sign(X)


# --------------------------------------------------------------------------- Jacobi

def test_jacobi_tridiagonal_closed_form():
    n = 40
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    w, V = O.jacobi_eigh(A)
    exact = 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    assert np.max(np.abs(w - np.sort(exact))) < 1e-13
    assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-13
    assert np.max(np.abs(A @ V - V * w)) < 1e-13


def test_jacobi_prescribed_spectrum():
    rng = np.random.default_rng(5)
    n = 30
    Qh, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = np.concatenate([np.linspace(-3, 7, n - 4), [1.0, 1.0, 1.0, 100.0]])  # triple eigenvalue
    A = Qh @ np.diag(d) @ Qh.T
    w, V = O.jacobi_eigh(0.5 * (A + A.T))
    assert np.max(np.abs(w - np.sort(d))) < 1e-12
    assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-13


# --------------------------------------------------------------------------- definition

def test_dense_definition_fem1d_closed_form():
    n = 120
    K, M, lam, X = fem1d_exact(n, np.arange(1, n + 1))
    w, Z = O.eigpairs_dense(K, M)
    # backward-stable bound: absolute error ~ eps * lambda_max (plus the closed form's own rounding)
    assert np.max(np.abs(w - lam) / (1e-13 * lam[-1] + 1e-12 * lam)) < 1
    # eigenvectors (simple eigenvalues): equal up to sign (the largest-entry sign rule ties for
    # sin modes, whose extreme entries come in +/- pairs)
    dots = np.abs(np.einsum("ij,ij->j", Z, M.to_scipy() @ X))
    assert np.max(np.abs(dots - 1)) < 1e-10


def test_dense_definition_q1_kronecker_closed_form():
    nc = 9
    K, M = P.fem_q1(nc, 2)
    w, Z = O.eigpairs_dense(K, M)
    l1 = P.fem1d_eigenvalue(np.arange(1, nc), nc - 1)
    exact = np.sort((l1[:, None] + l1[None, :]).ravel())
    assert np.max(np.abs(w - exact) / exact) < 1e-12
    Ms = M.to_scipy()
    assert np.max(np.abs(Z.T @ (Ms @ Z) - np.eye(K.n))) < 1e-11


def test_dense_definition_matches_library_on_random_field():
    K, M = P.fem2d_p1_lognormal(14)
    w, Z = O.eigpairs_dense(K, M)
    ref = sl.eigh(K.to_scipy().toarray(), M.to_scipy().toarray(), eigvals_only=True)
    assert np.max(np.abs(w - ref) / np.abs(ref)) < 1e-11


# --------------------------------------------------------------------------- counting

@pytest.mark.parametrize("sigma_k", [1, 7, 31, 90])
def test_inertia_sturm_fem1d(sigma_k):
    n = 150
    K, M = P.fem1d(n)
    lam = P.fem1d_eigenvalue(np.arange(1, n + 1), n)
    sigma = 0.5 * (lam[sigma_k - 1] + lam[sigma_k])  # between lambda_k and lambda_{k+1}
    assert O.inertia_count(K, M, sigma) == sigma_k


def test_inertia_q1_3d_kronecker_count():
    nc = 8
    K, M = P.fem_q1(nc, 3)
    l1 = P.fem1d_eigenvalue(np.arange(1, nc), nc - 1)
    exact = np.sort((l1[:, None, None] + l1[None, :, None] + l1[None, None, :]).ravel())
    u = np.unique(np.round(exact, 8))
    for j in (3, 10, 40):
        sigma = 0.5 * (u[j] + u[j + 1])
        assert O.inertia_count(K, M, sigma) == int(np.sum(exact < sigma))


def test_inertia_random_field_vs_dense():
    K, M = P.fem2d_p1_lognormal(16)
    w = sl.eigh(K.to_scipy().toarray(), M.to_scipy().toarray(), eigvals_only=True)
    for j in (0, 5, 50, 120):
        sigma = 0.5 * (w[j] + w[j + 1])
        assert O.inertia_count(K, M, sigma) == j + 1


# --------------------------------------------------------------------------- shifted solves

def test_band_lu_against_library_dense_solve():
    K, M = P.fem2d_p1_lognormal(12)
    z = 300.0 + 45.0j
    rng = np.random.default_rng(3)
    B = rng.standard_normal((K.n, 5)) + 1j * rng.standard_normal((K.n, 5))
    X = O.ShiftedSolver(K, M, z).solve(B)
    A = z * M.to_scipy().toarray() - K.to_scipy().toarray()
    ref = np.linalg.solve(A, B)
    assert np.max(np.abs(X - ref)) / np.max(np.abs(ref)) < 1e-12
    assert np.max(np.abs(A @ X - B)) / np.max(np.abs(B)) < 1e-12


def test_band_lu_pivoting_needed():
    # a zero leading diagonal entry: elimination without row interchanges would fail
    n = 6
    A = np.diag(np.full(n, 2.0 + 0j)) + np.diag(np.full(n - 1, 1.0 + 1j), 1) + np.diag(np.full(n - 1, -1.0), -1)
    A[0, 0] = 0.0
    Ks = sp.csr_matrix(-A.real)
    Ms = sp.csr_matrix(np.zeros((n, n)))
    # (z M - K) with z = 0 and K = -A gives A exactly (complex part via a second real matrix)
    solver = O.ShiftedSolver(Ks, Ms, 0.0)
    solver_ab = np.zeros_like(solver.ab)
    kl = solver.kl
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + kl + 1)):
            solver_ab[i, j - i + kl] = A[i, j]
    ipiv = np.zeros(n, dtype=np.int64)
    info = O._L().oracle_zband_lu_factor(n, kl, kl, O._ptr(solver_ab), O._ptr(ipiv))
    assert info == 0 and ipiv[0] != 0
    solver.ab, solver.ipiv = solver_ab, ipiv
    b = np.arange(1, n + 1).astype(complex)
    x = solver.solve(b)[:, 0]
    assert np.max(np.abs(A @ x - b)) < 1e-13


def test_shifted_apply_closed_form_modes():
    """Closed form on the 1D pencil: the sine modes x_k(i) = sin(k pi i h) satisfy K x_k = lambda_k M x_k
    and M x_k = (h/6)(4 + 2 cos(k pi h)) x_k, so (z M - K) x_k = (z - lambda_k)(h/6)(4 + 2 cos(k pi h)) x_k
    for every complex z.  A block of complex combinations of modes pins the sign of the operator
    (z M - K, not K - z M), that z enters unconjugated, and that P is not conjugated."""
    n = 30
    K, M = P.fem1d(n)
    h = 1.0 / (n + 1)
    ks = np.array([1, 4, 9, 17])
    X = np.sin(np.outer(np.arange(1, n + 1), ks) * np.pi * h)
    lam = P.fem1d_eigenvalue(ks, n)
    mu = (h / 6.0) * (4.0 + 2.0 * np.cos(ks * np.pi * h))
    rng = np.random.default_rng(1)
    A = rng.standard_normal((ks.size, 3)) + 1j * rng.standard_normal((ks.size, 3))
    Pm = X @ A
    for z in (2.0 - 7.0j, -3.0 + 1e3j, 5e3 + 0.5j):
        Q = O.shifted_apply(K, M, z, Pm)
        expect = X @ (((z - lam) * mu)[:, None] * A)
        assert np.max(np.abs(Q - expect)) <= 1e-10 * np.max(np.abs(expect))


def test_norm1_hand_values():
    """||K||_1 of the 1D stiffness tridiag(-1, 2, -1)/h is 4/h = 4(n + 1) (interior columns), of the
    mass (h/6) tridiag(1, 4, 1) it is h; on a non-symmetric 2 x 2 it is the largest column sum (8),
    not the largest row sum (6)."""
    n = 30
    K, M = P.fem1d(n)
    assert abs(O.norm1(K) - 4.0 * (n + 1)) <= 1e-12 * 4.0 * (n + 1)
    assert abs(O.norm1(M) - 1.0 / (n + 1)) <= 1e-15
    import scipy.sparse as sps
    assert O.norm1(sps.csr_matrix(np.array([[1.0, -5.0], [2.0, 3.0]]))) == 8.0


# --------------------------------------------------------------------------- nodes, weights, moments

def _filter_setup(N=16):
    n = 60
    K, M = P.fem1d(n)
    lam = P.fem1d_eigenvalue(np.arange(1, n + 1), n)
    c, R = 0.5 * (lam[9] + lam[20]), 0.5 * (lam[20] - lam[9])
    rng = np.random.default_rng(7)
    V = rng.standard_normal((n, 4))
    _, _, _, X = fem1d_exact(n, np.arange(1, n + 1))
    return K, M, lam, X, c, R, V


def _closed_form_moment(lam, X, M, V, c, R, N, k):
    """Trapezoid filter: S_k = X diag(x^k / (1 + x^N)) X^T M V, x = (lambda - c)/R, 0 <= k < N."""
    x = (lam - c) / R
    return X @ ((x ** k / (1 + x ** N))[:, None] * (X.T @ (M.to_scipy() @ V)))


@pytest.mark.parametrize("N", [8, 16, 32])
def test_moments_match_trapezoid_filter_closed_form(N):
    K, M, lam, X, c, R, V = _filter_setup(N)
    z, w = O.trapezoid_nodes(c, R, N)
    B = M.to_scipy() @ V
    Xs = [O.ShiftedSolver(K, M, zj).solve(B) for zj in z]
    S = O.moments(Xs, z, w, c, R, 3)
    for k in range(3):
        ref = _closed_form_moment(lam, X, M, V, c, R, N, k)
        assert np.max(np.abs(S[k] - ref)) / np.max(np.abs(ref)) < 1e-11, k


def test_conjugate_symmetry_full_circle():
    K, M, lam, X, c, R, V = _filter_setup()
    N = 16
    th = 2 * np.pi * (np.arange(1, N + 1) - 0.5) / N
    zf = c + R * np.exp(1j * th)
    wf = R * np.exp(1j * th) / N
    B = M.to_scipy() @ V
    full = sum(wj * ((zj - c) / R) * O.ShiftedSolver(K, M, zj).solve(B) for zj, wj in zip(zf, wf))
    z, w = O.trapezoid_nodes(c, R, N)
    half = O.moments([O.ShiftedSolver(K, M, zj).solve(B) for zj in z], z, w, c, R, 2)[1]
    assert np.max(np.abs(full.imag)) < 1e-12 * np.max(np.abs(full.real))
    assert np.max(np.abs(full.real - half)) < 1e-12 * np.max(np.abs(half))


def test_filter_pin_detects_wrong_weight_or_angle():
    """Plant slips in the node/weight rule and check the closed-form pin rejects each."""
    K, M, lam, X, c, R, V = _filter_setup()
    N = 16
    B = M.to_scipy() @ V
    ref = _closed_form_moment(lam, X, M, V, c, R, N, 1)
    j = np.arange(1, N // 2 + 1)
    variants = {
        "angle without half shift": 2 * np.pi * j / N,
        "conjugated weight": None,
    }
    for name, th in variants.items():
        if th is None:
            z, w = O.trapezoid_nodes(c, R, N)
            w = np.conj(w)
        else:
            e = np.exp(1j * th)
            z, w = c + R * e, R * e / N
        Xs = [O.ShiftedSolver(K, M, zj).solve(B) for zj in z]
        S1 = O.moments(Xs, z, w, c, R, 2)[1]
        assert np.max(np.abs(S1 - ref)) / np.max(np.abs(ref)) > 1e-3, name
    # missing mass matrix on the right-hand side
    z, w = O.trapezoid_nodes(c, R, N)
    Xs = [O.ShiftedSolver(K, M, zj).solve(V) for zj in z]
    S1 = O.moments(Xs, z, w, c, R, 2)[1]
    assert np.max(np.abs(S1 - ref)) / np.max(np.abs(ref)) > 1e-3


# --------------------------------------------------------------------------- basis, projection, residual

def test_m_orthonormalize_invariants_and_rank_truncation():
    K, M = P.fem2d_p1_lognormal(10)
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((K.n, 8))
    Y = np.concatenate([Y, Y[:, :3] @ rng.standard_normal((3, 2))], axis=1)  # rank 8 of 10
    Q = O.m_orthonormalize(Y, M)
    Ms = M.to_scipy()
    assert Q.shape[1] == 8
    assert np.max(np.abs(Q.T @ (Ms @ Q) - np.eye(8))) < 1e-12
    # same span: Y is reproduced by its M-projection onto Q
    Yp = Q @ (Q.T @ (Ms @ Y))
    assert np.max(np.abs(Yp - Y)) < 1e-10 * np.max(np.abs(Y))


def test_rayleigh_ritz_exact_subspace():
    n = 80
    K, M, lam, X = fem1d_exact(n, np.arange(1, n + 1))
    rng = np.random.default_rng(4)
    sub = X[:, [3, 4, 9, 30]] @ rng.standard_normal((4, 4))  # mixes of 4 eigenvectors
    Q = O.m_orthonormalize(sub, M)
    theta, Z = O.rayleigh_ritz(K, M, Q)
    assert np.max(np.abs(theta - lam[[3, 4, 9, 30]]) / lam[[3, 4, 9, 30]]) < 1e-12
    res = O.residuals(K, M, theta, Z)
    assert np.max(res) < 1e-13


def test_residual_definition_scaling():
    n = 50
    K, M, lam, X = fem1d_exact(n, [3])
    r_exact = O.residuals(K, M, lam, X)[0]
    assert r_exact < 1e-14
    # scaling the vector does not change the relative residual; a wrong value raises it
    assert abs(O.residuals(K, M, lam, 7.0 * X)[0] - r_exact) < 1e-14
    r_bad = O.residuals(K, M, lam * (1 + 1e-6), X)[0]
    Ms, Ks = M.to_scipy(), K.to_scipy()
    # ||K||_1 = 4 (n + 1) for the 1D stiffness (hand value, see test_norm1_hand_values)
    expect = np.linalg.norm(lam[0] * 1e-6 * (Ms @ X[:, 0])) / (4.0 * (n + 1) * np.linalg.norm(X[:, 0]))
    assert abs(r_bad - expect) < 1e-3 * expect


def test_merge_dedup():
    n = 40
    K, M, lam, X = fem1d_exact(n, [2, 5, 6])
    theta = np.array([lam[1], lam[0], lam[1] * (1 + 1e-12), lam[2]])
    Z = np.stack([X[:, 1], X[:, 0], -X[:, 1], X[:, 2]], axis=1)
    res = np.array([1e-12, 1e-13, 1e-14, 1e-13])
    cid = np.array([0, 0, 1, 1], dtype=np.int32)
    t, Zk, r, c = O.merge_dedup(theta, Z, res, cid, M)
    assert len(t) == 3 and np.all(np.diff(t) > 0)
    assert r[1] == 1e-14 and c[1] == 1   # the duplicate with the smaller residual wins


# --------------------------------------------------------------------------- whole CI method

def test_ci_solve_fem1d_closed_form():
    K, M, spec = P.workload("fem1d-n2000")
    V = P.gaussian_block(K.n, spec["L"], 1)
    r = O.ci_solve(K, M, spec["lo"], spec["hi"], V, ncontours=1, nodes=16, moments_m=2, tol=1e-10)
    lam = P.fem1d_eigenvalue(np.arange(spec["first"], spec["last"] + 1), K.n)
    assert len(r["evals"]) == spec["count"] == 51
    assert np.max(np.abs(r["evals"] - lam) / lam) < 1e-10
    assert np.max(r["resid"]) <= 1e-10
    assert O.count_in(K, M, spec["lo"], spec["hi"]) == 51
    # eigenvectors against sin(k pi x) closed form
    _, _, _, X = fem1d_exact(K.n, np.arange(spec["first"], spec["last"] + 1))
    dots = np.abs(np.einsum("ij,ij->j", r["evecs"], M.to_scipy() @ X))
    assert np.min(dots) > 1 - 1e-10


def test_ci_solve_random_field_vs_definition_and_split_invariance():
    K, M = P.fem2d_p1_lognormal(24)
    wd, Zd = O.eigpairs_dense(K, M)
    lo, hi = 0.5 * (wd[9] + wd[10]), 0.5 * (wd[49] + wd[50])
    V = P.gaussian_block(K.n, 24, 11)
    out = []
    for nct in (2, 3):
        r = O.ci_solve(K, M, lo, hi, V, ncontours=nct, nodes=16, moments_m=2, tol=1e-10)
        assert len(r["evals"]) == 40 == O.count_in(K, M, lo, hi)
        assert np.max(np.abs(r["evals"] - wd[10:50]) / wd[10:50]) < 1e-10
        assert np.max(r["resid"]) <= 1e-10
        dots = np.abs(np.einsum("ij,ij->j", r["evecs"], M.to_scipy() @ Zd[:, 10:50]))
        assert np.min(dots) > 1 - 1e-8
        out.append(r["evals"])
    assert np.max(np.abs(out[0] - out[1]) / out[0]) < 1e-10


def test_ci_solve_multiplicity_q1_kronecker():
    nc = 12
    K, M = P.fem_q1(nc, 2)
    l1 = P.fem1d_eigenvalue(np.arange(1, nc), nc - 1)
    exact = np.sort((l1[:, None] + l1[None, :]).ravel())
    lo, hi = 0.5 * (exact[2] + exact[3]), 0.5 * (exact[21] + exact[22])
    assert exact[2] < exact[3] and exact[21] < exact[22]
    V = P.gaussian_block(K.n, 16, 3)
    r = O.ci_solve(K, M, lo, hi, V, ncontours=2, nodes=16, moments_m=2, tol=1e-10)
    ref = exact[(exact > lo) & (exact < hi)]
    assert len(r["evals"]) == len(ref) == O.count_in(K, M, lo, hi)
    assert np.max(np.abs(r["evals"] - ref) / ref) < 1e-10
