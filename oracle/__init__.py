"""Plain FP64 CPU oracle for the contour-integral (CI) generalized eigensolver.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA path (the GPU library never
loads `liboracle.so`, and nothing here imports `paper_2511_01927_gb300`).

What it computes (paper: arXiv 2511.01927, "Learning-Guided Integration Contours Construction
for Fast Large-Scale Generalized Eigensolvers"):

* the definition of the result, Eq. GEP (Section 3.1) restricted to the target range of
  Algorithm 1: every eigenpair (lambda, x) of A x = lambda B x with lambda in [lo, hi]
  (`eigpairs_dense`, `inertia_count`);
* the CI method step by step in the paper's order (`ci_solve`): contours from the partition of
  the range (Section 4.2 circle rule), trapezoid nodes on each circle (Section 4.2 N_q-point
  trapezoid rule; Eq. quadrature_appendix), the shifted solves (z_j B - A) X_j = B V at every
  node (Algorithm 1), the moment sums S_k (Appendix A.3.3, moment-based methods), orthonormal
  basis, projection, reduced GEP, Ritz recovery and "keep lambda in I_k" (Algorithm 1), the
  subspace iteration of FEAST (Appendix A.3.3, U_{i+1} = orth(P_k U_i)) until the residual
  tolerance is met (Section 5.1 / Appendix B.2), and the merge/de-duplication across contours;
* contours for a fixed budget (`plan_contours`): cuts of [lo, hi] in the widest gaps of a predicted
  spectrum, the fullest piece first, until the budget is reached;
* the count check of a contour (`trace_estimate`, `count_miss`, `resplit`): the stochastic trace
  estimate of the enclosed eigenvalue count (Section 2, CI eigensolvers) against the Ritz count,
  and the re-split of a contour that misses eigenvalues at a KDE cut (Algorithm 2).

* the KDE contour construction of Algorithm 2 (`kde_contours`): recursive splits of the predicted
  spectrum's range at the minimiser of the interval sparsity function G_k (Section 4.2), then
  the merge of intervals holding too few predicted eigenvalues.

Readings of points the paper leaves open (node placement, moment scaling, residual norm, basis
orthonormalisation, dedup rule, eigenvector sign, the argmin domain and merge rule of Algorithm 2)
are stated at each function.

Notation: the paper's A, B are K (stiffness, symmetric) and M (mass, SPD) here.
"""
from __future__ import annotations

import concurrent.futures as _cf
import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (strict IEEE double, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_zband_lu_factor.argtypes = [i64, i64, i64, p, p]
        lib.oracle_zband_lu_factor.restype = ctypes.c_int
        lib.oracle_zband_lu_solve.argtypes = [i64, i64, i64, p, p, i64, p]
        lib.oracle_zband_lu_solve.restype = None
        lib.oracle_dband_ldlt_negcount.argtypes = [i64, i64, p, p]
        lib.oracle_dband_ldlt_negcount.restype = i64
        lib.oracle_jacobi_eig.argtypes = [i64, p, p, p, ctypes.c_double, ctypes.c_int]
        lib.oracle_jacobi_eig.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def host_threads() -> int:
    """Host cores this process may run on (its CPU affinity set)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def node_map(fn, items, threads: int | None = None):
    """[fn(x) for x in items], the items on separate host threads.  The quadrature nodes of a contour
    are independent (Algorithm 1 solves them "in parallel"), and the C kernels run without Python's
    lock, so each node's factorization and solves run on a core of their own; the arithmetic of
    each item is exactly that of the serial loop."""
    items = list(items)
    t = min(len(items), threads or host_threads())
    if t <= 1:
        return [fn(x) for x in items]
    with _cf.ThreadPoolExecutor(max_workers=t) as ex:
        return list(ex.map(fn, items))


# ----------------------------------------------------------------------------- matrices

def as_scipy(A):
    """Accept a pencils.Csr-like object (n, rowptr, col, val) or a scipy matrix."""
    if sp.issparse(A):
        return sp.csr_matrix(A)
    return sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))


def bandwidth(*mats) -> int:
    bw = 0
    for A in mats:
        A = sp.coo_matrix(as_scipy(A))
        if A.nnz:
            bw = max(bw, int(np.max(np.abs(A.row.astype(np.int64) - A.col))))
    return bw


def norm1(A) -> float:
    """||A||_1 = max column absolute sum (= ||A||_inf for symmetric A)."""
    A = as_scipy(A)
    return float(np.max(np.asarray(abs(A).sum(axis=0)).ravel()))


# ----------------------------------------------------------------------------- shifted solves

class ShiftedSolver:
    """Factorization of (z M - K) by complex banded Gaussian elimination with partial pivoting;
    `solve(B)` returns X with (z M - K) X = B.  These are the shifted linear systems of
    Eq. quadrature_appendix / Algorithm 1 ("Solve (z_j B - A) X_j = B V")."""

    def __init__(self, K, M, z: complex, bw: int | None = None):
        Ks, Ms = as_scipy(K), as_scipy(M)
        n = Ks.shape[0]
        kl = ku = bandwidth(Ks, Ms) if bw is None else bw
        W = 2 * kl + ku + 1
        A = (complex(z) * Ms.astype(np.complex128) - Ks.astype(np.complex128)).tocoo()
        ab = np.zeros((n, W), dtype=np.complex128)
        ab[A.row, A.col.astype(np.int64) - A.row + kl] += A.data
        self.n, self.kl, self.ku, self.ab = n, kl, ku, ab
        self.ipiv = np.zeros(n, dtype=np.int64)
        info = _L().oracle_zband_lu_factor(n, kl, ku, _ptr(ab), _ptr(self.ipiv))
        if info != 0:
            raise np.linalg.LinAlgError(f"zero pivot in column {info - 1}")

    def solve(self, B: np.ndarray) -> np.ndarray:
        X = np.array(B, dtype=np.complex128, order="C", copy=True)
        if X.ndim == 1:
            X = X[:, None]
        _L().oracle_zband_lu_solve(self.n, self.kl, self.ku, _ptr(self.ab), _ptr(self.ipiv),
                                   X.shape[1], _ptr(X))
        return X


def shifted_apply(K, M, z: complex, P: np.ndarray) -> np.ndarray:
    """Q = (z M - K) P: the operator of the shifted systems applied to a block (plain definition)."""
    Ks, Ms = as_scipy(K), as_scipy(M)
    return complex(z) * (Ms @ P) - Ks @ P


# ----------------------------------------------------------------------------- counting

def inertia_count(K, M, sigma: float) -> int:
    """Number of eigenvalues of K x = lambda M x below sigma, as the number of negative pivots of
    LDL^T(K - sigma M) (Sylvester's law of inertia; the eigenvalue counting the paper cites in
    Sections 2.1 and 3.3).  Banded, no pivoting."""
    Ks, Ms = as_scipy(K), as_scipy(M)
    n = Ks.shape[0]
    bw = bandwidth(Ks, Ms)
    A = sp.tril(Ks - sigma * Ms).tocoo()
    ab = np.zeros((n, bw + 1), dtype=np.float64)
    ab[A.row, A.col.astype(np.int64) - A.row + bw] += A.data
    nz = np.zeros(1, dtype=np.int64)
    return int(_L().oracle_dband_ldlt_negcount(n, bw, _ptr(ab), _ptr(nz)))


def count_in(K, M, lo: float, hi: float) -> int:
    """Eigenvalues in [lo, hi] = #neg(hi) - #neg(lo)."""
    return inertia_count(K, M, hi) - inertia_count(K, M, lo)


# ----------------------------------------------------------------------------- dense symmetric

def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, maxsweep: int = 60):
    """Eigen-decomposition of a dense symmetric matrix by cyclic Jacobi; ascending eigenvalues,
    eigenvectors as columns."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    p = A.shape[0]
    w = np.zeros(p)
    V = np.zeros((p, p))
    if p == 0:
        return w, V
    _L().oracle_jacobi_eig(p, _ptr(A), _ptr(w), _ptr(V), tol, maxsweep)
    order = np.argsort(w, kind="stable")
    return w[order], np.ascontiguousarray(V[:, order])


def fix_sign(Z: np.ndarray) -> np.ndarray:
    """Sign convention for eigenvectors: the entry of largest magnitude is positive."""
    Z = np.array(Z, dtype=np.float64, copy=True)
    if Z.size == 0:
        return Z
    idx = np.argmax(np.abs(Z), axis=0)
    s = np.sign(Z[idx, np.arange(Z.shape[1])])
    s[s == 0] = 1.0
    return Z * s


def eigpairs_dense(K, M, lo: float = -np.inf, hi: float = np.inf):
    """The definition of the result: all eigenpairs of K x = lambda M x with lambda in [lo, hi]
    (Eq. GEP; Algorithm 1 ENSURE), by Cholesky reduction M = L L^T, C = L^-1 K L^-T, Jacobi on C,
    x = L^-T y.  Eigenvectors are M-orthonormal with the `fix_sign` convention.  Dense: small n."""
    Kd = as_scipy(K).toarray()
    Md = as_scipy(M).toarray()
    Lc = np.linalg.cholesky(Md)
    Li = np.linalg.inv(Lc)
    C = Li @ Kd @ Li.T
    C = 0.5 * (C + C.T)
    w, Y = jacobi_eigh(C)
    X = Li.T @ Y
    keep = (w >= lo) & (w <= hi)
    return w[keep], fix_sign(X[:, keep])


# ----------------------------------------------------------------------------- CI method

def uniform_contours(lo: float, hi: float, ncontours: int, alpha: float = 0.0):
    """Equal-width partition of [lo, hi]; each piece I_k = [s, e] becomes the circle with centre
    (s+e)/2 and radius (1+alpha)(e-s)/2 (Section 4.2 circle rule).  Returns a list of
    (c, R, s, e)."""
    edges = np.linspace(lo, hi, ncontours + 1)
    out = []
    for k in range(ncontours):
        s, e = float(edges[k]), float(edges[k + 1])
        out.append((0.5 * (s + e), (1.0 + alpha) * 0.5 * (e - s), s, e))
    return out


def trapezoid_nodes(c: float, R: float, N: int):
    """Upper-half nodes and weights of the N-point trapezoid rule on the circle |z - c| = R
    (Section 4.2; Eq. quadrature_appendix).  Reading: theta_j = 2 pi (j - 1/2) / N, j = 1..N, so
    no node lies on the real axis and nodes come in conjugate pairs; the weight folds in
    dz/(2 pi i): omega_j = R e^{i theta_j} / N.  Only j = 1..N/2 (Im z > 0) are returned; the
    lower half contributes the complex conjugate because K, M are real."""
    if N % 2:
        raise ValueError("N must be even")
    j = np.arange(1, N // 2 + 1)
    th = 2.0 * np.pi * (j - 0.5) / N
    e = np.exp(1j * th)
    return c + R * e, R * e / N


def moments(X_nodes, z, w, c: float, R: float, m: int):
    """Moment sums S_k = (1/2 pi i) oint s^k (z M - K)^-1 M V dz by the trapezoid rule, k = 0..m-1
    (Appendix A.3.3, moment-based methods).  Reading: the power is of the normalised node
    s_j = (z_j - c)/R instead of z_j (same span, better conditioned).  With upper-half nodes:
    S_k = 2 Re sum_j omega_j s_j^k X_j."""
    S = []
    for k in range(m):
        acc = np.zeros(X_nodes[0].shape, dtype=np.complex128)
        for Xj, zj, wj in zip(X_nodes, z, w):
            acc += wj * ((zj - c) / R) ** k * Xj
        S.append(2.0 * acc.real)
    return S


def m_orthonormalize(Y: np.ndarray, M, drop: float = 1e-14):
    """Orthonormal basis of span(Y) in the M inner product ("Orthonormalize Q <- orth(Y)",
    Algorithm 1).  Reading: Gram matrix G = Y^T M Y, G = U diag(sigma) U^T by Jacobi, keep
    sigma_i > drop * max sigma (rank truncation), Q = Y U_k diag(sigma_k)^-1/2."""
    Ms = as_scipy(M)
    G = Y.T @ (Ms @ Y)
    G = 0.5 * (G + G.T)
    sig, U = jacobi_eigh(G)
    if sig.size == 0 or sig[-1] <= 0:
        return Y[:, :0]
    keep = sig > drop * sig[-1]
    return Y @ (U[:, keep] / np.sqrt(sig[keep]))


def rayleigh_ritz(K, M, Q: np.ndarray):
    """Project and solve the reduced GEP (Algorithm 1): A_k = Q^T K Q, B_k = Q^T M Q,
    A_k u = theta B_k u via Cholesky reduction of B_k and Jacobi; Ritz vectors Z = Q U."""
    Ks, Ms = as_scipy(K), as_scipy(M)
    Kh = Q.T @ (Ks @ Q)
    Mh = Q.T @ (Ms @ Q)
    Kh = 0.5 * (Kh + Kh.T)
    Mh = 0.5 * (Mh + Mh.T)
    Lc = np.linalg.cholesky(Mh)
    Li = np.linalg.inv(Lc)
    C = Li @ Kh @ Li.T
    theta, Yc = jacobi_eigh(0.5 * (C + C.T))
    U = Li.T @ Yc
    return theta, Q @ U


def residuals(K, M, theta: np.ndarray, Z: np.ndarray, normK1: float | None = None):
    """Relative residual ||K z - theta M z||_2 / (||K||_1 ||z||_2) per Ritz pair (reading of the
    paper's unspecified "residual tolerance", Section 5.1 / Appendix B.2)."""
    Ks, Ms = as_scipy(K), as_scipy(M)
    if normK1 is None:
        normK1 = norm1(Ks)
    R = Ks @ Z - (Ms @ Z) * theta
    return np.linalg.norm(R, axis=0) / (normK1 * np.linalg.norm(Z, axis=0))


def merge_dedup(theta, Z, res, cid, M, rtol: float = 1e-8):
    """Merge the per-contour results and remove duplicates ("Merge and de-duplicate solutions
    across k", Algorithm 1).  Reading: sort by value; two pairs are the same when
    |theta - theta'| <= rtol max(1, |theta|) and |z^T M z'| > 0.5; the smaller residual wins."""
    Ms = as_scipy(M)
    order = np.argsort(theta, kind="stable")
    theta, Z, res, cid = theta[order], Z[:, order], res[order], cid[order]
    keep = []
    for i in range(len(theta)):
        dup = False
        for k in range(len(keep) - 1, -1, -1):
            j = keep[k]
            if abs(theta[i] - theta[j]) > rtol * max(1.0, abs(theta[i])):
                break
            if abs(Z[:, i] @ (Ms @ Z[:, j])) > 0.5:
                dup = True
                if res[i] < res[j]:
                    keep[k] = i
                break
        if not dup:
            keep.append(i)
    keep = np.array(sorted(keep, key=lambda i: theta[i]), dtype=np.int64)
    return theta[keep], Z[:, keep], res[keep], cid[keep]


def trace_estimate(V: np.ndarray, S0: np.ndarray):
    """Stochastic estimate of how many eigenvalues the contour encloses: the eigenvalue-count
    estimate by stochastic trace estimation that the paper names among the ways CI methods place
    contours (Section 2, CI eigensolvers).  S_0 = P V, P the quadrature's spectral filter (Eq.
    quadrature_appendix); for V with independent N(0, 1) entries E[v^T P v] = tr P, the sum of the
    filter over the spectrum: the enclosed count, up to the filter's leakage next to the circle.
    Reading: one sample per column, est = mean_l v_l^T (S_0)_l, and its standard error
    std_l / sqrt(L) from the same samples.  Returns (est, se)."""
    per = np.einsum("il,il->l", V, S0)
    L = per.size
    se = float(per.std(ddof=1) / np.sqrt(L)) if L > 1 else float("inf")
    return float(per.mean()), se


def count_miss(est: float, se: float, theta, res, c: float, R: float, rank: int, tol: float) -> bool:
    """Count check of a finished contour (the stochastic trace of S_0 and the Ritz count).
    Reading: on the circle's diameter [c - R, c + R] a contour misses eigenvalues when (a) every
    Ritz value of its basis lies there (no spare direction: the basis may be smaller than the
    number of enclosed eigenvalues, which the subspace iteration of Appendix A.3.3 needs it to
    exceed), or (b) the trace estimate exceeds the converged Ritz pairs there by more than
    max(1.5, 3 se)."""
    on = np.abs(np.asarray(theta) - c) <= R
    found = int(np.sum(on & (np.asarray(res) <= tol)))
    return bool(int(np.sum(on)) >= rank or est - found > max(1.5, 3.0 * se))


def resplit(theta, c: float, R: float, s: float, e: float, w: float = 10.0):
    """The two contours that replace one that failed the count check.  I_k = [s, e] is split at
    the minimiser of the KDE sparsity function of its Ritz values in [s, e] (G_k and `kde_cut` of
    Algorithm 2) searched between their lower and upper quartiles: the cut lies in a gap, and each
    half keeps at least a quarter of them (a plain argmin peels the edge of a spectrum whose gaps
    widen, one level per few eigenvalues).  Reading: with k sorted Ritz values the quartiles are
    the (k // 4)-th and (k - 1 - k // 4)-th; with fewer than two distinct values between them, or a
    cut not strictly inside (s, e), the midpoint.  Both halves keep the parent's radius-to-half-width
    ratio (1 + alpha, Section 4.2 circle rule).  Returns two (c, R, s, e)."""
    th = np.asarray(theta, dtype=np.float64)
    pts = np.sort(th[(th >= s) & (th <= e)])
    t = 0.5 * (s + e)
    k = pts.size
    if k >= 2:
        q1, q3 = pts[k // 4], pts[k - 1 - k // 4]
        if q1 < q3:
            tc = kde_cut(pts, s, e, w, within=(q1, q3))
            if s < tc < e:
                t = tc
    infl = R / (0.5 * (e - s))
    return [(0.5 * (s + t), infl * 0.5 * (t - s), s, t), (0.5 * (t + e), infl * 0.5 * (e - t), t, e)]


def plan_contours(pred, lo: float, hi: float, max_contours: int, alpha: float = 0.0):
    """Contours for a fixed budget of contours: [lo, hi] is cut in gaps of the predicted spectrum
    until it has max_contours pieces.  Algorithm 2 stops at N_max predictions per interval, so its
    piece count follows from the spectrum, and its G_k with w = 10 is a third of the interval wide:
    on an even spectrum it sees only the broad shape and cuts near the ends.  A GPU solve whose
    shifted systems all run in one wave wants the count fixed instead, and FEAST converges fastest
    when no eigenvalue lies near a circle, so the cut goes in the widest gap (the argmin of G_k in
    the limit of a narrow kernel).  Reading: while fewer than max_contours pieces exist, the piece
    with the most predictions in [a, b] (leftmost on ties) is cut at the middle of the widest gap
    between consecutive predictions of ranks k // 4 .. k - 1 - k // 4 (k sorted predictions; first
    such gap on ties), so each half keeps a quarter of them; a piece whose widest such gap is empty
    (fewer than two distinct predictions) is not cut and planning stops.  Contour k: c = (a + b)/2,
    r = (1 + alpha)(b - a)/2 (Section 4.2).  Returns a list of (lo, hi, c, r, count), ascending."""
    p = np.sort(np.asarray(pred, dtype=np.float64))

    def inside(a, b):
        return p[(p >= a) & (p <= b)]

    pieces = [(float(lo), float(hi))]
    while len(pieces) < max_contours:
        counts = [inside(a, b).size for a, b in pieces]
        k = int(np.argmax(counts))
        a, b = pieces[k]
        q = inside(a, b)
        m = q.size
        if m < 2:
            break
        i0, i1 = m // 4, m - 1 - m // 4          # gaps q[i] .. q[i + 1] for i0 <= i < i1 (at least one)
        i1 = max(i1, i0 + 1)
        gaps = q[i0 + 1:i1 + 1] - q[i0:i1]
        j = int(np.argmax(gaps))
        if not gaps[j] > 0.0:
            break
        t = 0.5 * (q[i0 + j] + q[i0 + j + 1])
        pieces[k:k + 1] = [(a, t), (t, b)]
    return [(a, b, 0.5 * (a + b), (1.0 + alpha) * 0.5 * (b - a), int(inside(a, b).size)) for a, b in pieces]


def ci_solve(K, M, lo: float, hi: float, V: np.ndarray, *, ncontours: int = 1, nodes: int = 16,
             moments_m: int = 2, tol: float = 1e-10, max_outer: int = 10, alpha: float = 0.0,
             contours=None, trace: dict | None = None, judge: bool = False, max_resplit: int = 3,
             kde_w: float = 10.0, threads: int | None = None):
    """The CI eigensolver of Algorithm 1 with the moment method and FEAST outer iterations.

    For each contour (c, R) enclosing I_k = [s, e]:
      1. nodes/weights of the trapezoid rule (upper half);
      2. iteration 0: Y = [S_0 .. S_{m-1}] from the solves (z_j M - K) X_j = M V;
      3. Q = M-orthonormal basis of Y; Ritz pairs (theta, Z) of (Q^T K Q, Q^T M Q);
      4. residual of each Ritz pair; the pairs with theta in I_k are kept when their residual
         is <= tol;
      5. if some theta in I_k still has residual > tol: next iteration with V <- Z (all Ritz
         vectors), one moment (plain FEAST filter P_k Z), same factorizations; back to 3.
    With `judge`, a finished contour that fails the count check (`count_miss`, on the trace
    estimate of iteration 0's S_0) is replaced, in place, by the two halves of `resplit` (up to
    `max_resplit` levels; at the last level it keeps its pairs and reports non-convergence).
    Then merge/dedup across contours.  V is the random block (n x L) drawn by the caller.
    `trace`, if given, receives per-contour intermediates of iteration 0 (nodes, S, Q, theta).
    `threads`: host threads (default: every core of the affinity set), shared by the contours of a
    level and the nodes of each contour.  `trace` holds the input contours (depth 0) in order.
    Returns dict(evals, evecs, resid, contour_of, outer_iters, status, contours, estimates,
    resplits); contour_of indexes the final contours."""
    Ks, Ms = as_scipy(K), as_scipy(M)
    nK = norm1(Ks)
    if contours is None:
        contours = uniform_contours(lo, hi, ncontours, alpha)
    bw = bandwidth(Ks, Ms)
    cores = threads or host_threads()

    def one_contour(ct, node_threads):
        """Steps 1-5 for one contour; the contours are independent until the merge."""
        c, R, s, e = ct
        z, w = trapezoid_nodes(c, R, nodes)
        solvers = node_map(lambda zj: ShiftedSolver(Ks, Ms, zj, bw), z, node_threads)
        Vk = np.asarray(V, dtype=np.float64)
        m = moments_m
        ok = False
        tr = None
        for it in range(max_outer):
            B = Ms @ Vk
            X = node_map(lambda sv: sv.solve(B), solvers, node_threads)
            S = moments(X, z, w, c, R, m)
            if it == 0:
                est, se = trace_estimate(Vk, S[0])
            Y = np.concatenate(S, axis=1)
            Q = m_orthonormalize(Y, Ms)
            theta, Z = rayleigh_ritz(Ks, Ms, Q)
            res = residuals(Ks, Ms, theta, Z, nK)
            if it == 0:
                tr = dict(z=z, w=w, S=S, Q=Q, theta=theta, res=res)
            inside = (theta >= s) & (theta <= e)
            if not np.any(inside & (res > tol)):
                ok = True
                break
            Vk, m = Z, 1
        return dict(ct=ct, theta=theta, Z=Z, res=res, inside=inside, est=est, se=se, rank=Q.shape[1],
                    iters=it + 1, ok=ok, trace=tr)

    # the contours of a level are solved side by side (each with its share of the host cores), then
    # judged in order; a contour that fails the check is replaced in place by its halves, which the
    # next level solves, so the final contours keep the order of the depth-first splits
    slots = [dict(ct=tuple(ct), depth=0, out=None) for ct in contours]
    resplits = 0
    while True:
        pend = [sl for sl in slots if sl["out"] is None]
        if not pend:
            break
        per = max(1, cores // len(pend))
        outs = node_map(lambda sl: one_contour(sl["ct"], per), pend, min(cores, len(pend)))
        new_slots = []
        for sl in slots:
            if sl["out"] is not None:
                new_slots.append(sl)
                continue
            o = outs[pend.index(sl)]
            c, R, s, e = sl["ct"]
            if trace is not None and sl["depth"] == 0:
                trace.setdefault("contours", []).append(o["trace"])
            if judge and count_miss(o["est"], o["se"], o["theta"], o["res"], c, R, o["rank"], tol):
                if sl["depth"] < max_resplit and e > s:
                    new_slots.extend(dict(ct=tuple(ch), depth=sl["depth"] + 1, out=None)
                                     for ch in resplit(o["theta"], c, R, s, e, kde_w))
                    resplits += 1
                    continue
                o["ok"] = False
            sl["out"] = o
            new_slots.append(sl)
        slots = new_slots
    leaves = [sl["ct"] for sl in slots]
    outs = [sl["out"] for sl in slots]
    ests = [o["est"] for o in outs]
    iters = [o["iters"] for o in outs]
    status = [0 if o["ok"] else 1 for o in outs]
    sels = [o["inside"] & (o["res"] <= tol) for o in outs]
    all_t = [o["theta"][sel] for o, sel in zip(outs, sels)]
    all_z = [o["Z"][:, sel] for o, sel in zip(outs, sels)]
    all_r = [o["res"][sel] for o, sel in zip(outs, sels)]
    cid = [np.full(t.size, k, dtype=np.int32) for k, t in enumerate(all_t)]
    theta = np.concatenate(all_t)
    Z = np.concatenate(all_z, axis=1) if all_z else np.zeros((Ks.shape[0], 0))
    res = np.concatenate(all_r)
    cid = np.concatenate(cid)
    theta, Z, res, cid = merge_dedup(theta, Z, res, cid, Ms)
    # M-normalise and fix the sign of each returned vector
    Zn = Z / np.sqrt(np.einsum("ij,ij->j", Z, Ms @ Z))
    return dict(evals=theta, evecs=fix_sign(Zn), resid=res, contour_of=cid,
                outer_iters=max(iters) if iters else 0, status=status, contours=leaves,
                estimates=np.array(ests), resplits=resplits)


# --------------------------------------------------------------------------- Algorithm 2 (KDE)

KDE_GRID = 1024        # grid points of the first search for the minimiser of G_k
KDE_GOLDEN_STEPS = 100  # golden-section steps of its refinement


def kde_sparsity(t, pts, a: float, b: float, w: float):
    """G_k(t) = sum_j exp(-w (t - lam_j)^2 / (b - a)^2) over the predictions lam_j in I_k = [a, b]
    (Section 4.2, interval sparsity function)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    s = w / (b - a) ** 2
    return np.exp(-s * (t[:, None] - pts[None, :]) ** 2).sum(axis=1)


def kde_cut(pts, a: float, b: float, w: float, within=None) -> float:
    """The split point of Algorithm 2: argmin of G_k.  Reading: the minimum is taken over the open
    range between the interval's smallest and largest predictions (over all of I_k it would always
    be an end point, where the kernels thin out), located by a uniform grid of KDE_GRID cell centres
    (first minimum on ties) and refined by golden-section search between the neighbouring cell
    centres, so the cut lies strictly between the smallest and largest prediction and both halves
    keep at least one.  `within` = (lo, hi) narrows the search range (the re-split of `resplit`)."""
    lo, hi = (float(pts.min()), float(pts.max())) if within is None else (float(within[0]), float(within[1]))
    h = (hi - lo) / KDE_GRID
    grid = lo + (np.arange(KDE_GRID) + 0.5) * h
    i = int(np.argmin(kde_sparsity(grid, pts, a, b, w)))
    ga, gb = grid[max(i - 1, 0)], grid[min(i + 1, KDE_GRID - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    x1, x2 = gb - g * (gb - ga), ga + g * (gb - ga)
    f1, f2 = kde_sparsity(x1, pts, a, b, w)[0], kde_sparsity(x2, pts, a, b, w)[0]
    for _ in range(KDE_GOLDEN_STEPS):
        if f1 <= f2:
            gb, x2, f2 = x2, x1, f1
            x1 = gb - g * (gb - ga)
            f1 = kde_sparsity(x1, pts, a, b, w)[0]
        else:
            ga, x1, f1 = x1, x2, f2
            x2 = ga + g * (gb - ga)
            f2 = kde_sparsity(x2, pts, a, b, w)[0]
    return 0.5 * (ga + gb)


def kde_contours(pred, nmin: int = 10, nmax: int = 50, w: float = 10.0, alpha: float = 0.0,
                 beta: float = 0.0):
    """Algorithm 2 (adaptive contour construction via KDE), in its order:

    1. the initial range I_0 = [min - eps, max + eps], eps = beta (max - min) (Section 4.2);
    2. pop an interval; if it holds at most nmax predictions it is final, else it is split at the
       minimiser of G_k (`kde_cut`) and both halves are pushed;
    3. intervals with fewer than nmin predictions are merged with their nearest neighbour, and a
       merged interval above nmax is split again (Section 4.2, refinement loop).

    Readings: a prediction belongs to [lo, hi) (the last interval also takes hi); an interval whose
    predictions are all equal is not split.  The refinement repeatedly takes the interval with the
    fewest predictions (leftmost on ties) while it holds fewer than nmin, and joins it to the
    neighbour with the nearer centre (left on ties); a joined interval above nmax is split again
    between its two middle predictions (the KDE cut would peel off the edge of a locally uniform
    stretch and recreate the small interval).  The loop ends when no interval is below nmin, one
    interval is left, or after 4 x (number of intervals) joins.  Contours: c = (lo + hi)/2,
    r = (1 + alpha)(hi - lo)/2 (Section 4.2).  Returns a list of (lo, hi, c, r, count), ascending."""
    p = np.sort(np.asarray(pred, dtype=np.float64))
    if p.size == 0:
        raise ValueError("no predicted eigenvalues")
    eps = beta * (p[-1] - p[0])
    A, B = p[0] - eps, p[-1] + eps

    def members(a, b):
        m = (p >= a) & (p < b)
        if b == B:
            m |= p == b
        return p[m]

    def split_all(intervals):
        work, done = list(intervals), []
        while work:
            a, b = work.pop()
            pts = members(a, b)
            if pts.size <= nmax or pts.min() == pts.max():
                done.append((a, b))
                continue
            t = kde_cut(pts, a, b, w)
            work.append((a, t))
            work.append((t, b))
        return sorted(done)

    final = split_all([(A, B)])
    for _ in range(4 * len(final)):
        if len(final) == 1:
            break
        counts = [members(a, b).size for a, b in final]
        k = int(np.argmin(counts))
        if counts[k] >= nmin:
            break
        if k == 0:
            j = 1
        elif k == len(final) - 1:
            j = k - 1
        else:
            ck = 0.5 * (final[k][0] + final[k][1])
            dl = ck - 0.5 * (final[k - 1][0] + final[k - 1][1])
            dr = 0.5 * (final[k + 1][0] + final[k + 1][1]) - ck
            j = k - 1 if dl <= dr else k + 1
        lo_i, hi_i = min(k, j), max(k, j)
        a, b = final[lo_i][0], final[hi_i][1]
        q = members(a, b)
        if q.size > nmax:
            m = q.size // 2
            t = 0.5 * (q[m - 1] + q[m])
            new = [(a, t), (t, b)]
        else:
            new = [(a, b)]
        final = final[:lo_i] + new + final[hi_i + 1:]
    out = final
    return [(a, b, 0.5 * (a + b), (1.0 + alpha) * 0.5 * (b - a), int(members(a, b).size)) for a, b in out]


# --------------------------------------------------------------------------- density predictor (reference forward)
# The learned-contour path (Section 4.1's spectrum predictor stand-in, Algorithm 3 "predict, construct
# contours, solve") runs a small network on the GPU.  This is its plain NumPy forward pass, written from
# the layout the C ABI states: the 64 x 64 x 2 input of block means of log(kappa), log(rho); four 3 x 3
# convolutions with stride 2, zero padding 1 and ReLU (2 -> 16 -> 32 -> 64 -> 64 channels, NHWC); the
# 4 x 4 x 64 features flattened as (y, x, channel) followed by (log lo - 6.5, log hi - 6.5); fc1 1026 -> 512
# with ReLU; fc2 512 -> 256 with softplus.  Weights: one float32 array, W[Cout][3][3][Cin] then b[Cout] per
# convolution, then W1[512][1026], b1, W2[256][512], b2.  With `bf16`, weights and every layer's input are
# rounded to BF16 (round to nearest even), as the GPU path does; sums are formed in FP64.

DENSITY_CONV = ((2, 16), (16, 32), (32, 64), (64, 64))
DENSITY_FEAT = 64 * 4 * 4 + 2
DENSITY_HID = 512
DENSITY_BINS = 256


def bf16_round(x):
    """Round float32 values to the nearest BF16 value (ties to even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def density_unpack(w):
    """The flat weight array as [(W, b), ...] per layer (W of the convolutions as [Cout][3][3][Cin])."""
    w = np.asarray(w, dtype=np.float32).ravel()
    out, pos = [], 0
    shapes = [((co, 3, 3, ci), co) for ci, co in DENSITY_CONV]
    shapes += [((DENSITY_HID, DENSITY_FEAT), DENSITY_HID), ((DENSITY_BINS, DENSITY_HID), DENSITY_BINS)]
    for shp, nb in shapes:
        nw = int(np.prod(shp))
        out.append((w[pos:pos + nw].reshape(shp), w[pos + nw:pos + nw + nb]))
        pos += nw + nb
    if pos != w.size:
        raise ValueError(f"expected {pos} weights, got {w.size}")
    return out


def density_input(kappa, rho):
    """64 x 64 x 2 network input of one member: block means of log(kappa), log(rho) (G x G cell grids)."""
    G = kappa.shape[0]
    s = G // 64
    lk = np.log(np.asarray(kappa, dtype=np.float64)).reshape(64, s, 64, s).mean(axis=(1, 3))
    lr = np.log(np.asarray(rho, dtype=np.float64)).reshape(64, s, 64, s).mean(axis=(1, 3))
    return np.stack([lk, lr], axis=-1)


def density_forward(w, kappa, rho, bounds, bf16: bool = True):
    """Predicted histograms (batch x 256): kappa, rho batch x G x G; bounds batch x 2 (lo, hi)."""
    layers = density_unpack(w)
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    kappa = np.asarray(kappa)
    rho = np.asarray(rho)
    if kappa.ndim == 2:
        kappa, rho = kappa[None], rho[None]
    bounds = np.asarray(bounds, dtype=np.float64).reshape(-1, 2)
    out = []
    for b in range(kappa.shape[0]):
        x = density_input(kappa[b], rho[b]).astype(np.float32)
        for (W, bias), (ci, co) in zip(layers[:4], DENSITY_CONV):
            H = x.shape[0]
            Ho = H // 2
            xp = np.zeros((H + 2, H + 2, ci))
            xp[1:H + 1, 1:H + 1] = rnd(x)
            Wr = rnd(W)
            y = np.zeros((Ho, Ho, co))
            for ky in range(3):
                for kx in range(3):
                    patch = xp[ky:ky + 2 * Ho:2, kx:kx + 2 * Ho:2, :]      # (Ho, Ho, ci): rows 2 oy + ky - 1
                    y += patch @ Wr[:, ky, kx, :].T
            x = np.maximum(y + bias.astype(np.float64), 0.0).astype(np.float32)
        f = np.concatenate([x.reshape(-1), (np.log(bounds[b]) - 6.5).astype(np.float32)])
        (W1, b1), (W2, b2) = layers[4], layers[5]
        h = np.maximum(rnd(W1) @ rnd(f) + b1, 0.0).astype(np.float32)
        z = rnd(W2) @ rnd(h) + b2
        out.append(np.where(z > 20.0, z, np.log1p(np.exp(np.minimum(z, 20.0)))))
    return np.array(out)


def hist_quantiles(hist, lo: float, hi: float):
    """Pseudo-eigenvalues of a histogram over [lo, hi] (counts spread evenly inside each bin): with
    N = round(total), value k (k = 1..N) is where the cumulative count reaches k - 1/2."""
    h = np.asarray(hist, dtype=np.float64)
    N = int(np.floor(h.sum() + 0.5))
    edges = np.linspace(lo, hi, h.size + 1)
    cum = np.concatenate([[0.0], np.cumsum(h)])
    out = []
    for k in range(1, N + 1):
        t = min(k - 0.5, cum[-1])
        j = int(np.searchsorted(cum, t, side="left")) - 1
        j = min(max(j, 0), h.size - 1)
        while h[j] == 0.0 and j < h.size - 1 and cum[j + 1] < t:
            j += 1
        frac = min(1.0, max(0.0, (t - cum[j]) / h[j])) if h[j] > 0 else 1.0
        out.append(edges[j] + frac * (edges[j + 1] - edges[j]))
    return np.array(out)
