"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step and end to end.

Tolerances:
  * FP32 shifted SpMM: per element, 2^-21 * ((|z| |M| + |K|) |P|)_i  (a few FP32 roundings of every
    product and sum that forms the element);
  * FP64 kernels: the same bound with 2^-49;
  * shifted solves: the residual ||D^-1/2 (B - (zM - K) X)|| / ||D^-1/2 B|| <= 2 lin_tol (D = diag K,
    the library's stopping test), computed here in FP64 by the oracle's operator, and the LU
    solution's forward error;
  * eigenpairs: values within 1e-10 relative of the oracle / closed form, residual <= 1e-10,
    counts equal to the oracle's inertia count exactly.
"""
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


@pytest.fixture(scope="module")
def small2d(G, ctx):
    K, M, spec = P.workload("fem2d-p1-40")
    pen = G.gcie_pencil_create(ctx, K, M)
    yield K, M, spec, pen
    G.gcie_pencil_destroy(pen)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def spmm_bound(K, M, z, Pb):
    Ks, Ms = abs(K.to_scipy()), abs(M.to_scipy())
    return abs(z) * (Ms @ np.abs(Pb)) + Ks @ np.abs(Pb)


# --------------------------------------------------------------------------- a4: shifted SpMM

@pytest.mark.parametrize("ncol", [2, 6, 64])
def test_shifted_spmm_f32(G, ctx, small2d, ncol):
    K, M, spec, pen = small2d
    rng = np.random.default_rng(ncol)
    z = np.array([100 + 30j, 250 + 5j, 40 + 80j])
    Pb = (rng.standard_normal((3, K.n, ncol)) + 1j * rng.standard_normal((3, K.n, ncol))).astype(np.complex64)
    dP = dev(Pb)
    dQ = torch.zeros_like(dP)
    G.gcie_shifted_spmm_f32(ctx, pen, z, ncol, dP, dQ)
    Q = host(dQ)
    for s in range(3):
        ref = O.shifted_apply(K, M, z[s], Pb[s].astype(np.complex128))
        bound = 2.0 ** -21 * spmm_bound(K, M, z[s], Pb[s].astype(np.complex128))
        assert np.all(np.abs(Q[s] - ref) <= bound + 1e-30), s


@pytest.mark.parametrize("ncol", [1, 5, 32])
def test_shifted_spmm_f64(G, ctx, small2d, ncol):
    K, M, spec, pen = small2d
    rng = np.random.default_rng(100 + ncol)
    z = np.array([10 - 3j, 300 + 120j])
    Pb = rng.standard_normal((2, K.n, ncol)) + 1j * rng.standard_normal((2, K.n, ncol))
    dP = dev(Pb)
    dQ = torch.zeros_like(dP)
    G.gcie_shifted_spmm_f64(ctx, pen, z, ncol, dP, dQ)
    Q = host(dQ)
    for s in range(2):
        ref = O.shifted_apply(K, M, z[s], Pb[s])
        assert np.all(np.abs(Q[s] - ref) <= 2.0 ** -49 * spmm_bound(K, M, z[s], Pb[s]) + 1e-300), s


# --------------------------------------------------------------------------- a4-a6: shifted solves

@pytest.mark.parametrize("precision,precond", [(0, 3), (1, 3), (0, 2), (1, 2), (0, 0), (1, 0)])
def test_shifted_solve_matches_lu(G, ctx, small2d, precision, precond):
    K, M, spec, pen = small2d
    lo, hi = spec["lo"], spec["hi"]
    c, R = 0.5 * (lo + hi), 0.5 * (hi - lo)
    z, w = O.trapezoid_nodes(c, R, 16)
    z = z[[0, 3, 7]]
    ncol = 6
    V = P.gaussian_block(K.n, ncol, 5)
    B = M.to_scipy() @ V
    dB = dev(B)
    dX = torch.zeros((len(z), K.n, ncol), dtype=torch.complex128, device="cuda")
    lin_tol = 1e-11
    iters, rc = G.gcie_shifted_solve(ctx, pen, z, ncol, dB, dX, lin_tol=lin_tol, precision=precision, precond=precond)
    X = host(dX)
    assert iters > 0
    if precond == 3:
        assert iters <= 12          # FP32 band LDL^T factors: a few preconditioned iterations
    elif precond == 2:
        assert iters < 1500         # multigrid cycle
    # the stopping test is on the symmetrically scaled system D^-1/2 (zM - K) D^-1/2 with D = diag(K)
    dsc = 1.0 / np.sqrt(K.to_scipy().diagonal())
    for s, zs in enumerate(z):
        res = B - O.shifted_apply(K, M, zs, X[s])
        rel = np.linalg.norm(dsc[:, None] * res, axis=0) / np.linalg.norm(dsc[:, None] * B, axis=0)
        assert np.max(rel) <= 2 * lin_tol, (s, rel)
        Xr = O.ShiftedSolver(K, M, zs).solve(B)
        err = np.linalg.norm(X[s] - Xr, axis=0) / np.linalg.norm(Xr, axis=0)
        assert np.max(err) < 1e-7, (s, err)


@pytest.mark.parametrize("sc,kind", [(sc, k) for k in ("ws", "plain", "tc") for sc in (8, 16, 32)] + [(4, "plain")])
def test_band_sweep_variants(G, ctx, small2d, sc, kind, monkeypatch):
    """Every column-per-CTA variant of the band sweeps gives the same converged solves (ragged
    column groups: 38 columns do not fill the last group of 4, 8, 16 or 32): warp-specialised (ws),
    solve-then-apply (plain), and with the block updates on the tensor cores (tc, forced at this narrow
    band: b = 40)."""
    monkeypatch.setenv("GCIE_BAND_SC", str(sc))
    monkeypatch.setenv("GCIE_SWEEP_TC", "1" if kind == "tc" else "0")
    monkeypatch.setenv("GCIE_BAND_WS", "1" if kind == "ws" else "0")
    K, M, spec, pen = small2d
    lo, hi = spec["lo"], spec["hi"]
    z, _ = O.trapezoid_nodes(0.5 * (lo + hi), 0.5 * (hi - lo), 16)
    z = z[[1, 6]]
    ncol = 38
    V = P.gaussian_block(K.n, ncol, 11)
    B = M.to_scipy() @ V
    dX = torch.zeros((len(z), K.n, ncol), dtype=torch.complex128, device="cuda")
    iters, rc = G.gcie_shifted_solve(ctx, pen, z, ncol, dev(B), dX, lin_tol=1e-11, precision=0, precond=3)
    X = host(dX)
    assert 0 < iters <= 12
    for s, zs in enumerate(z):
        Xr = O.ShiftedSolver(K, M, zs).solve(B)
        err = np.linalg.norm(X[s] - Xr, axis=0) / np.linalg.norm(Xr, axis=0)
        assert np.max(err) < 1e-7, (sc, s, err)


def test_band_sweep_wait_timeout_reports_and_recovers(G, small2d, monkeypatch):
    """The bounded wait of the warp-specialised band sweeps (the others copy with cp.async and have no
    wait that can run out): with the bulk copy of one factor block never issued (test switch), the
    waiting threads give up after about a second, the other waits then return at once and the CTA
    finishes, the call returns GCIE_ETIMEOUT, and the context stays usable for the next solve."""
    monkeypatch.setenv("GCIE_BAND_WS", "1")
    K, M, spec, _ = small2d
    ctx2 = G.gcie_create(0)
    try:
        pen = G.gcie_pencil_create(ctx2, K, M)
        z = np.array([0.5 * (spec["lo"] + spec["hi"]) + 20j])
        B = M.to_scipy() @ P.gaussian_block(K.n, 8, 3)
        dX = torch.zeros((1, K.n, 8), dtype=torch.complex128, device="cuda")
        monkeypatch.setenv("GCIE_TEST_STOP_COPY", "3")
        with pytest.raises(G.GcieError) as e:
            G.gcie_shifted_solve(ctx2, pen, z, 8, dev(B), dX, lin_tol=1e-11, precision=0, precond=3)
        assert e.value.code == 7
        monkeypatch.delenv("GCIE_TEST_STOP_COPY")
        iters, rc = G.gcie_shifted_solve(ctx2, pen, z, 8, dev(B), dX, lin_tol=1e-11, precision=0, precond=3)
        Xr = O.ShiftedSolver(K, M, z[0]).solve(B)
        assert rc == 0 and np.max(np.abs(host(dX)[0] - Xr)) <= 1e-7 * np.max(np.abs(Xr))
        G.gcie_pencil_destroy(pen)
    finally:
        G.gcie_destroy(ctx2)


def test_shifted_solve_initial_guess_and_zero_rhs(G, ctx, small2d):
    K, M, spec, pen = small2d
    z = np.array([200 + 20j])
    V = P.gaussian_block(K.n, 4, 8)
    V[:, 1] = 0.0                                   # a zero right-hand side: x = 0 exactly
    B = M.to_scipy() @ V
    Xr = O.ShiftedSolver(K, M, z[0]).solve(B)
    dX = dev(Xr[None].copy())                       # exact initial guess
    iters, rc = G.gcie_shifted_solve(ctx, pen, z, 4, dev(B), dX, x0=True, lin_tol=1e-11)
    X = host(dX)
    assert iters <= 1 and np.all(X[0][:, 1] == 0)
    assert np.max(np.abs(X[0] - Xr)) <= 1e-10 * np.max(np.abs(Xr))


# --------------------------------------------------------------------------- a7: moments

def test_moments_match_oracle(G, ctx, small2d):
    K, M, spec, pen = small2d
    c, R = 200.0, 60.0
    z, w = O.trapezoid_nodes(c, R, 16)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((8, K.n, 6)) + 1j * rng.standard_normal((8, K.n, 6))
    dS = torch.zeros((K.n, 3 * 6), dtype=torch.float64, device="cuda")
    G.gcie_moments(ctx, K.n, z, w, c, R, 3, 6, dev(X), dS)
    S = host(dS)
    ref = O.moments(list(X), z, w, c, R, 3)
    for k in range(3):
        assert np.max(np.abs(S[:, 6 * k:6 * k + 6] - ref[k])) <= 1e-13 * np.max(np.abs(ref[k])), k


# --------------------------------------------------------------------------- a8-a11: dense steps

@pytest.mark.parametrize("p", [1, 7, 50, 128])
def test_jacobi_matches_oracle(G, ctx, p):
    rng = np.random.default_rng(p)
    Qh, _ = np.linalg.qr(rng.standard_normal((p, p)))
    d = rng.standard_normal(p) * 10
    if p >= 7:
        d[:3] = 2.0                                  # a triple eigenvalue
    A = Qh @ np.diag(d) @ Qh.T
    A = 0.5 * (A + A.T)
    dA, dw, dV = dev(A.copy()), torch.zeros(p, dtype=torch.float64, device="cuda"), torch.zeros((p, p), dtype=torch.float64, device="cuda")
    G.gcie_jacobi_eig(ctx, p, dA, dw, dV)
    w, V = host(dw), host(dV)
    wo, _ = O.jacobi_eigh(A)
    nA = np.linalg.norm(A)
    assert np.max(np.abs(w - wo)) <= 1e-13 * nA
    assert np.max(np.abs(A @ V - V * w)) <= 1e-13 * nA
    assert np.max(np.abs(V.T @ V - np.eye(p))) <= 1e-13


def test_m_orthonormalize_matches_oracle_span(G, ctx, small2d):
    K, M, spec, pen = small2d
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((K.n, 16))
    Y[:, 14] = Y[:, 0] - 2 * Y[:, 3]
    Y[:, 15] = 0.0
    dQ = torch.zeros_like(dev(Y))
    rank = G.gcie_m_orthonormalize(ctx, pen, 16, dev(Y), 1e-14, dQ)
    Q = host(dQ)[:, :rank]
    Qo = O.m_orthonormalize(Y, M)
    Ms = M.to_scipy()
    assert rank == Qo.shape[1] == 14
    assert np.max(np.abs(Q.T @ (Ms @ Q) - np.eye(rank))) <= 1e-12
    # same subspace: M-orthogonal projectors agree
    Pg = Q @ (Q.T @ (Ms @ Y))
    Po = Qo @ (Qo.T @ (Ms @ Y))
    assert np.max(np.abs(Pg - Po)) <= 1e-10 * np.max(np.abs(Y))


def test_rayleigh_ritz_matches_oracle(G, ctx):
    n = 300
    K, M = P.fem1d(n)
    lam = P.fem1d_eigenvalue(np.arange(1, n + 1), n)
    h = 1.0 / (n + 1)
    X = np.sin(np.outer(np.arange(1, n + 1), np.arange(1, 13)) * np.pi * h)
    rng = np.random.default_rng(2)
    Y = X @ rng.standard_normal((12, 12)) + 1e-3 * rng.standard_normal((n, 12))
    Q = O.m_orthonormalize(Y, M)
    th_o, Z_o = O.rayleigh_ritz(K, M, Q)
    res_o = O.residuals(K, M, th_o, Z_o)
    pen = G.gcie_pencil_create(ctx, K, M)
    try:
        dZ = torch.zeros((n, Q.shape[1]), dtype=torch.float64, device="cuda")
        th, res = G.gcie_rayleigh_ritz(ctx, pen, Q.shape[1], dev(Q), dZ)
        Z = host(dZ)
    finally:
        G.gcie_pencil_destroy(pen)
    assert np.max(np.abs(th - th_o) / np.abs(th_o)) <= 1e-12
    assert np.max(np.abs(res - res_o)) <= 1e-12 + 1e-6 * np.max(res_o)
    dots = np.abs(np.einsum("ij,ij->j", Z, M.to_scipy() @ Z_o))
    assert np.min(dots) > 1 - 1e-9


# --------------------------------------------------------------------------- whole path

def _check_against(r, ref_vals, K, M, ref_vecs=None, tol=1e-10):
    assert len(r["evals"]) == len(ref_vals)
    assert np.max(np.abs(r["evals"] - ref_vals) / np.abs(ref_vals)) <= tol
    assert np.max(r["resid"]) <= 1e-10
    # the library's residuals are the definition's, recomputed here in FP64
    assert np.max(np.abs(O.residuals(K, M, r["evals"], r["evecs"]) - r["resid"])) <= 1e-12
    Ms = M.to_scipy()
    G = r["evecs"].T @ (Ms @ r["evecs"])
    assert np.max(np.abs(G - np.eye(len(ref_vals)))) <= 1e-9
    if ref_vecs is not None:
        dots = np.abs(np.einsum("ij,ij->j", r["evecs"], Ms @ ref_vecs))
        assert np.min(dots) > 1 - 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_fem1d_closed_form(G, ctx, precision):
    K, M, spec = P.workload("fem1d-n2000")
    V = P.gaussian_block(K.n, spec["L"], 1)
    r = G.gcie_solve(ctx, K, M, spec["lo"], spec["hi"], nodes=16, moments=2, nuniform=1, V0=V,
                     precision=precision, tol=1e-10)
    ks = np.arange(spec["first"], spec["last"] + 1)
    lam = P.fem1d_eigenvalue(ks, K.n)
    h = 1.0 / (K.n + 1)
    X = np.sin(np.outer(np.arange(1, K.n + 1), ks) * np.pi * h)
    X /= np.sqrt(np.einsum("ij,ij->j", X, M.to_scipy() @ X))
    assert len(r["evals"]) == spec["count"] == O.count_in(K, M, spec["lo"], spec["hi"])
    _check_against(r, lam, K, M, X)


def test_solve_fem3d_q1_octants_matches_definition(G, ctx):
    """Reduced member of the 3D Q1 octant-coefficient family (27-point stencil, n = 9^3 = 729,
    bandwidth 91): the returned set is the definition's, eigenvalues 12..51 of the dense solve."""
    K, M = P.fem_q1(10, 3, P.octant_coefficients(3, 4), P.octant_coefficients(3, 5))
    lam, X = O.eigpairs_dense(K, M)
    i0, i1 = 12, 51
    lo, hi = 0.5 * (lam[i0 - 1] + lam[i0]), 0.5 * (lam[i1] + lam[i1 + 1])
    V = P.gaussian_block(K.n, 32, 4)
    r = G.gcie_solve(ctx, K, M, lo, hi, nodes=16, moments=2, nuniform=2, V0=V, tol=1e-10)
    assert len(r["evals"]) == i1 - i0 + 1 == O.count_in(K, M, lo, hi)
    _check_against(r, lam[i0:i1 + 1], K, M, X[:, i0:i1 + 1])


def test_solve_fem2d_matches_oracle_ci(G, ctx, small2d):
    K, M, spec, pen = small2d
    V = P.gaussian_block(K.n, 32, 2)
    r = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nodes=16, moments=2, nuniform=2, V0=V)
    ro = O.ci_solve(K, M, spec["lo"], spec["hi"], V, ncontours=2, nodes=16, moments_m=2, tol=1e-10)
    assert len(r["evals"]) == spec["count"] == len(ro["evals"])
    _check_against(r, ro["evals"], K, M, ro["evecs"])


@pytest.mark.parametrize("lin_tol_first,lin_tol", [(1e-6, 1e-11), (1e-3, 1e-11), (1e-6, 1e-8)])
def test_solve_loose_inner_tolerance(G, ctx, small2d, lin_tol_first, lin_tol):
    """Looser inner tolerance in the first FEAST iteration (Appendix A.3.3: the subspace iteration needs the
    filtered basis, not exact solves), lin_tol in the later ones: the pairs still meet tol (a contour whose
    pairs do not is iterated again), they match the oracle's CI solve; the contours never take fewer FEAST
    iterations than with the tight default."""
    K, M, spec, pen = small2d
    V = P.gaussian_block(K.n, 32, 2)
    ro = O.ci_solve(K, M, spec["lo"], spec["hi"], V, ncontours=2, nodes=16, moments_m=2, tol=1e-10)
    tight = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nodes=16, moments=2, nuniform=2, V0=V)
    loose = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nodes=16, moments=2, nuniform=2, V0=V,
                                lin_tol_first=lin_tol_first, lin_tol=lin_tol)
    assert len(loose["evals"]) == spec["count"] == len(ro["evals"])
    _check_against(loose, ro["evals"], K, M, ro["evecs"])
    assert loose["outer_iters"] >= tight["outer_iters"]
    with pytest.raises(G.GcieError):
        G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nuniform=2, lin_tol_first=1e-13)


@pytest.mark.parametrize("lin_tol", [1e-6, 1e-4])
def test_solve_loose_everywhere_is_flagged_or_right(G, ctx, small2d, lin_tol):
    """A loose inner tolerance in every FEAST iteration can stall the iteration above tol; the solve then says
    so (GCIE_ENOCONV) and what it returns is still right: every returned pair meets tol and is one of the
    oracle's (no pair is ever returned inexact)."""
    K, M, spec, pen = small2d
    V = P.gaussian_block(K.n, 32, 2)
    ro = O.ci_solve(K, M, spec["lo"], spec["hi"], V, ncontours=2, nodes=16, moments_m=2, tol=1e-10)
    r = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nodes=16, moments=2, nuniform=2, V0=V,
                            lin_tol=lin_tol, allow_noconv=True)
    assert r["rc"] in (0, 5)
    if r["rc"] == 0:
        _check_against(r, ro["evals"], K, M, ro["evecs"])
    assert len(r["evals"]) <= len(ro["evals"])
    if len(r["evals"]):
        assert np.max(r["resid"]) <= 1e-10
        near = np.min(np.abs(r["evals"][:, None] - ro["evals"][None, :]) / np.abs(ro["evals"][None, :]), axis=1)
        assert np.max(near) <= 1e-10


def test_solve_fem2d_32_nodes_matches_oracle(G, ctx, small2d):
    """The paper's N_q = 32 trapezoid nodes per circle (Section 4.2): 16 shifted systems per
    contour in one batch, same set and values as the oracle with 32 nodes."""
    K, M, spec, pen = small2d
    V = P.gaussian_block(K.n, 32, 5)
    r = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nodes=32, moments=2, nuniform=2, V0=V)
    ro = O.ci_solve(K, M, spec["lo"], spec["hi"], V, ncontours=2, nodes=32, moments_m=2, tol=1e-10)
    assert len(r["evals"]) == spec["count"] == len(ro["evals"])
    _check_against(r, ro["evals"], K, M, ro["evecs"])


def test_solve_split_invariance_and_boundaries(G, ctx, small2d):
    K, M, spec, pen = small2d
    V = P.gaussian_block(K.n, 32, 7)
    a = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nuniform=1, V0=V, L=32)
    b = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nuniform=3, V0=V, L=32)
    assert len(a["evals"]) == len(b["evals"]) == spec["count"]
    assert np.max(np.abs(a["evals"] - b["evals"]) / a["evals"]) <= 1e-10
    assert set(b["contour_of"].tolist()) <= {0, 1, 2}


def test_solve_empty_interval(G, ctx, small2d):
    K, M, spec, pen = small2d
    lo = spec["lo"]                     # gap midpoint: nothing within gap_lo of it
    r = G.gcie_solve_pencil(ctx, pen, lo - 0.25 * spec["gap_lo"], lo + 0.25 * spec["gap_lo"], L=8)
    assert len(r["evals"]) == 0 and r["rc"] == 0


def test_expected_count_mismatch(G, ctx, small2d):
    K, M, spec, pen = small2d
    with pytest.raises(G.GcieError) as e:
        G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], L=32, nuniform=2, expected_count=spec["count"] + 1)
    assert e.value.code == 8


def test_invalid_inputs(G, ctx):
    import copy
    K, M = P.fem1d(50)
    bad = copy.deepcopy(K)
    bad.val = bad.val.copy()
    bad.val[1] *= 1.5                               # breaks symmetry
    with pytest.raises(G.GcieError) as e:
        G.gcie_solve(ctx, bad, M, 1.0, 100.0)
    assert e.value.code == 2
    Mz = copy.deepcopy(M)
    Mz.val = Mz.val.copy()
    Mz.val[0] = 0.0                                 # zero diagonal of M
    with pytest.raises(G.GcieError) as e:
        G.gcie_solve(ctx, K, Mz, 1.0, 100.0)
    assert e.value.code == 3
    with pytest.raises(G.GcieError) as e:
        G.gcie_solve(ctx, K, M, 100.0, 1.0)         # lo >= hi
    assert e.value.code == 1
    unsorted = copy.deepcopy(K)
    unsorted.col = unsorted.col.copy()
    unsorted.col[[1, 2]] = unsorted.col[[2, 1]]
    with pytest.raises(G.GcieError) as e:
        G.gcie_solve(ctx, unsorted, M, 1.0, 100.0)
    assert e.value.code == 1
    with pytest.raises(G.GcieError) as e:
        G.gcie_solve(ctx, K, M, 1.0, 100.0, nodes=7)
    assert e.value.code == 1


def test_solve_batch_of_uneven_pencils(G, ctx, small2d):
    """Independent pencils of different kinds and sizes in one call: each result is the one a
    single solve gives, and each set is the definition's (closed form / inertia count)."""
    K2, M2, spec2, _ = small2d
    items = []
    for n in (300, 700):
        K, M = P.fem1d(n)
        lam = P.fem1d_eigenvalue(np.arange(1, 30), n)
        items.append((K, M, 0.5 * (lam[2] + lam[3]), 0.5 * (lam[19] + lam[20]), lam[3:20]))
    items.append((K2, M2, spec2["lo"], spec2["hi"], None))
    outs = G.gcie_solve_batch(ctx, [(K, M, lo, hi) for K, M, lo, hi, _ in items], L=32, nuniform=2, seed=9)
    assert len(outs) == 3 and all(o["rc"] == 0 for o in outs)
    for (K, M, lo, hi, want), o in zip(items, outs):
        one = G.gcie_solve(ctx, K, M, lo, hi, L=32, nuniform=2, seed=9)
        assert len(o["evals"]) == len(one["evals"]) == O.count_in(K, M, lo, hi)
        assert np.max(np.abs(o["evals"] - one["evals"]) / np.abs(one["evals"])) <= 1e-12
        if want is not None:
            assert np.max(np.abs(o["evals"] - want) / want) < 1e-10
        assert np.max(o["resid"]) <= 1e-10
    with pytest.raises(G.GcieError):
        G.gcie_solve_batch(ctx, [(K2, M2, 1.0, 0.5)])


def test_solve_batch_concurrent_equals_sequential(G, ctx):
    """The batch scheduler (several pencils in flight on their own streams) returns, pencil by pencil, the
    result of solving them one after another, and each set is the definition's (inertia count)."""
    import pencils as PP
    batch = PP.serving_batch(5, 17)
    items = []
    for K, M, lo, hi, kind in batch:
        if K.n > 60000:                              # keep the oracle inertia counts quick
            continue
        items.append((K, M, lo, hi))
    a = G.gcie_solve_batch(ctx, items, L=32, nuniform=4, batch_streams=1, seed=3, allow_noconv=True)
    b = G.gcie_solve_batch(ctx, items, L=32, nuniform=4, batch_streams=4, seed=3, allow_noconv=True)
    for (K, M, lo, hi), x, y in zip(items, a, b):
        assert len(x["evals"]) == len(y["evals"]) == O.count_in(K, M, lo, hi)
        assert np.array_equal(x["evals"], y["evals"])
        assert np.max(y["resid"]) <= 1e-10
