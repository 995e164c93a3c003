"""Parity of the band-preconditioned path at the bench workload's bandwidth (b = 500).

The 2D P1 strip of 12 x 500 cells (n = 5489) has the bandwidth of the 500 x 500 pencil, so these tests
reach the code paths that smaller parity pencils do not:

  * the factorization's trailing update split in 128-row items over both CTAs of the cluster (4 row
    items per column group at b = 500);
  * the sweeps' window of b + 16 rows and the backward strip of ceil(b / 8) factor pieces;
  * the COCG sweeps' band-sized row chunks (taken once (n / b) x shifts >= 2 x SMs, here with 32 shifts);
  * every column-per-CTA variant (8, 16, 32) of the band sweeps on 64 columns;
  * the factorization with its trailing update on the tensor cores (4 x 128-row tiles at b = 500, split
    TF32) and on CUDA cores;
  * the sweeps with the window in tensor memory and the block updates as MMAs, and on CUDA cores.

Tolerances are those of tests/test_gpu_parity.py: the stopping test's scaled residual <= 2 lin_tol on
every column of every shift, forward error < 1e-7 against the oracle's banded LU, eigenpairs within
1e-10 of the oracle's CI solve with residuals <= 1e-10, counts equal to the inertia count.
"""
import numpy as np
import pytest

import oracle as O
import pencils as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LIN_TOL = 1e-11
NCOL = 64
CHECK_LU = (0, 5, 11)          # shifts also compared column by column with the oracle's LU


@pytest.fixture(scope="module")
def G():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2511_01927_gb300 import build
    build.build()
    import paper_2511_01927_gb300 as G
    return G


@pytest.fixture(scope="module")
def strip(G):
    K, M, spec = P.workload("fem2d-p1-strip")
    assert O.bandwidth(K, M) == 500
    ctx = G.gcie_create(0)
    pen = G.gcie_pencil_create(ctx, K, M)
    # the 16 upper-half nodes of the workload's two contours (N = 32 per circle: 32 shifts)
    z = []
    for c, R, _, _ in O.uniform_contours(spec["lo"], spec["hi"], 2):
        z.extend(O.trapezoid_nodes(c, R, 32)[0])
    z = np.array(z)
    B = M.to_scipy() @ P.gaussian_block(K.n, NCOL, 21)
    ref = O.node_map(lambda zs: O.ShiftedSolver(K, M, zs, 500).solve(B), z[list(CHECK_LU)])
    yield K, M, spec, ctx, pen, z, B, dict(zip(CHECK_LU, ref))
    G.gcie_pencil_destroy(pen)
    G.gcie_destroy(ctx)


@pytest.mark.parametrize("sc,factor_tc,sweep_tc,ws", [(8, 1, 1, 0), (16, 1, 1, 0), (32, 1, 1, 0), (8, 0, 0, 1),
                                                      (32, 0, 0, 1), (8, 1, 0, 1), (16, 1, 0, 1), (32, 1, 0, 1),
                                                      (32, 1, 0, 0), (8, 1, 0, 0), (4, 1, 0, 0)])
def test_strip_band_solves_match_lu(G, strip, sc, factor_tc, sweep_tc, ws, monkeypatch):
    """factor_tc / sweep_tc: the factorization's trailing update and the sweeps' block updates on the
    tensor cores (1, split TF32) or on CUDA cores (0); ws: the CUDA-core sweeps warp-specialised (1) or
    solve-then-apply (0).  All give FP32-quality preconditioners, so the iteration bound and the parity
    are the same."""
    monkeypatch.setenv("GCIE_BAND_SC", str(sc))
    monkeypatch.setenv("GCIE_FACTOR_TC", str(factor_tc))
    monkeypatch.setenv("GCIE_SWEEP_TC", str(sweep_tc))
    monkeypatch.setenv("GCIE_BAND_WS", str(ws))
    K, M, spec, ctx, pen, z, B, ref = strip
    dX = torch.zeros((len(z), K.n, NCOL), dtype=torch.complex128, device="cuda")
    iters, rc = G.gcie_shifted_solve(ctx, pen, z, NCOL, torch.from_numpy(B).cuda(), dX, lin_tol=LIN_TOL,
                                     precision=0, precond=3)
    torch.cuda.synchronize()
    X = dX.cpu().numpy()
    assert rc == 0 and 0 < iters <= 12, iters
    dsc = 1.0 / np.sqrt(K.to_scipy().diagonal())
    bn = np.linalg.norm(dsc[:, None] * B, axis=0)
    for s, zs in enumerate(z):
        res = B - O.shifted_apply(K, M, zs, X[s])
        rel = np.linalg.norm(dsc[:, None] * res, axis=0) / bn
        assert np.max(rel) <= 2 * LIN_TOL, (sc, s, np.max(rel))
    for s, Xr in ref.items():
        err = np.linalg.norm(X[s] - Xr, axis=0) / np.linalg.norm(Xr, axis=0)
        assert np.max(err) < 1e-7, (sc, s, np.max(err))


def test_strip_shifted_spmm_band_chunks(G, strip):
    """The fused SpMM at 32 shifts and 64 columns on the b = 500 strip against the definition, per
    element within the FP32 bound of the step parity test."""
    K, M, spec, ctx, pen, z, B, ref = strip
    rng = np.random.default_rng(5)
    Pb = (rng.standard_normal((len(z), K.n, NCOL)) + 1j * rng.standard_normal((len(z), K.n, NCOL))).astype(np.complex64)
    dP = torch.from_numpy(Pb).cuda()
    dQ = torch.zeros_like(dP)
    G.gcie_shifted_spmm_f32(ctx, pen, z, NCOL, dP, dQ)
    torch.cuda.synchronize()
    Q = dQ.cpu().numpy()
    Ks, Ms = abs(K.to_scipy()), abs(M.to_scipy())
    for s in range(len(z)):
        Ps = Pb[s].astype(np.complex128)
        ref_q = O.shifted_apply(K, M, z[s], Ps)
        bound = 2.0 ** -21 * (abs(z[s]) * (Ms @ np.abs(Ps)) + Ks @ np.abs(Ps))
        assert np.all(np.abs(Q[s] - ref_q) <= bound + 1e-30), s


def test_strip_solve_matches_oracle_ci(G, strip):
    """The whole solve at b = 500 (two contours, 16 nodes, L = 32, 2 moments) against the oracle's CI
    solve of the same V: the same 40 eigenpairs, the inertia count of the interval."""
    K, M, spec, ctx, pen, z, B, ref = strip
    V = P.gaussian_block(K.n, 32, 2)
    r = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], nodes=16, moments=2, nuniform=2, V0=V, L=32,
                            precond=3)
    ro = O.ci_solve(K, M, spec["lo"], spec["hi"], V, ncontours=2, nodes=16, moments_m=2, tol=1e-10)
    assert len(r["evals"]) == len(ro["evals"]) == spec["count"] == O.count_in(K, M, spec["lo"], spec["hi"])
    assert np.max(np.abs(r["evals"] - ro["evals"]) / np.abs(ro["evals"])) <= 1e-10
    assert np.max(r["resid"]) <= 1e-10
    assert np.max(np.abs(O.residuals(K, M, r["evals"], r["evecs"]) - r["resid"])) <= 1e-12
    Ms = M.to_scipy()
    dots = np.abs(np.einsum("ij,ij->j", r["evecs"], Ms @ ro["evecs"]))
    assert np.min(dots) > 1 - 1e-9


@pytest.fixture(scope="module")
def wide_strip(G):
    """An 8 x 700 strip (n = 4893, bandwidth 700): above the tensor-core factorization's limit (512), so the
    CUDA-core factorization runs; its sweep windows only fit the narrower column groups."""
    K, M = P.fem2d_p1_strip(8, 700)
    assert O.bandwidth(K, M) == 700
    ctx = G.gcie_create(0)
    pen = G.gcie_pencil_create(ctx, K, M)
    import scipy.linalg as sla
    lam = sla.eigh(O.as_scipy(K).toarray(), O.as_scipy(M).toarray(), eigvals_only=True, subset_by_index=[0, 59])
    z = np.array(O.trapezoid_nodes(0.5 * (lam[10] + lam[40]), 0.5 * (lam[40] - lam[10]), 8)[0][[0, 2]])
    B = M.to_scipy() @ P.gaussian_block(K.n, 16, 5)
    ref = O.node_map(lambda zs: O.ShiftedSolver(K, M, zs, 700).solve(B), z)
    yield K, M, ctx, pen, z, B, ref
    G.gcie_pencil_destroy(pen)
    G.gcie_destroy(ctx)


@pytest.mark.parametrize("sc,ws", [(4, 0), (8, 0), (8, 1)])
def test_wide_band_solves_match_lu(G, wide_strip, sc, ws, monkeypatch):
    """Band solves at bandwidth 700 with every sweep variant whose window fits shared memory there."""
    monkeypatch.setenv("GCIE_BAND_SC", str(sc))
    monkeypatch.setenv("GCIE_BAND_WS", str(ws))
    K, M, ctx, pen, z, B, ref = wide_strip
    dX = torch.zeros((len(z), K.n, 16), dtype=torch.complex128, device="cuda")
    iters, rc = G.gcie_shifted_solve(ctx, pen, z, 16, torch.from_numpy(B).cuda(), dX, lin_tol=LIN_TOL,
                                     precision=0, precond=3)
    X = dX.cpu().numpy()
    assert rc == 0 and 0 < iters <= 12, iters
    for s, Xr in enumerate(ref):
        err = np.linalg.norm(X[s] - Xr, axis=0) / np.linalg.norm(Xr, axis=0)
        assert np.max(err) < 1e-7, (sc, ws, s, np.max(err))
