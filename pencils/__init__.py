"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module only *generates* inputs: finite-element stiffness/mass pencils (K, M) of the
kinds the paper's workloads come from (scalar elliptic operators with random coefficient
fields, Section 3.1 "From PDE operators to GEPs" and Appendix D/E.3), and the random
right-hand-side block V that the contour-integral method draws (Algorithm 1, "draw a random
block V").  It holds none of the eigensolver's arithmetic, so both the oracle and the CUDA
path can consume it without sharing any part of the method.

All matrices are returned as `Csr` (0-based, sorted column indices, no duplicates, both
triangles stored), values in float64.
"""
from __future__ import annotations

import dataclasses
import json
import os

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Csr", "fem1d", "fem2d_p1", "fem2d_p1_rect", "fem2d_p1_strip", "grf_lognormal", "fem2d_p1_lognormal", "fem_q1",
    "octant_coefficients", "gaussian_block", "fem1d_eigenvalue", "workload", "WORKLOADS", "family_member", "serving_batch",
]


@dataclasses.dataclass
class Csr:
    """Compressed sparse row matrix: row i holds col[rowptr[i]:rowptr[i+1]] / val[...]."""
    n: int
    rowptr: np.ndarray  # int64, n+1
    col: np.ndarray     # int32, nnz
    val: np.ndarray     # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    @staticmethod
    def from_scipy(a, drop_zeros: bool = True) -> "Csr":
        a = sp.csr_matrix(a)
        a.sum_duplicates()
        if drop_zeros:
            a.eliminate_zeros()
        a.sort_indices()
        return Csr(a.shape[0], np.ascontiguousarray(a.indptr, dtype=np.int64),
                   np.ascontiguousarray(a.indices, dtype=np.int32),
                   np.ascontiguousarray(a.data, dtype=np.float64))


# --------------------------------------------------------------------------- 1D

def fem1d(n: int) -> tuple[Csr, Csr]:
    """Linear finite elements for -u'' = lambda u on (0,1), homogeneous Dirichlet, n interior nodes.

    K = tridiag(-1, 2, -1)/h,  M = (h/6) tridiag(1, 4, 1),  h = 1/(n+1).
    """
    h = 1.0 / (n + 1)
    e = np.ones(n)
    K = sp.diags([-e[1:], 2 * e, -e[1:]], [-1, 0, 1]) / h
    M = sp.diags([e[1:], 4 * e, e[1:]], [-1, 0, 1]) * (h / 6.0)
    return Csr.from_scipy(K), Csr.from_scipy(M)


def fem1d_eigenvalue(k, n: int):
    """Closed-form k-th (1-based) eigenvalue of the `fem1d(n)` pencil:
    lambda_k = (6/h^2) (1 - cos(k pi h)) / (2 + cos(k pi h))."""
    h = 1.0 / (n + 1)
    c = np.cos(np.asarray(k, dtype=np.float64) * np.pi * h)
    return 6.0 / (h * h) * (1.0 - c) / (2.0 + c)


# --------------------------------------------------------------------------- 2D P1

def grf_lognormal(nc: int, ell: float, sigma: float, seed: int) -> np.ndarray:
    """exp(g) on the nc x nc cell-centroid grid of the unit square, g a zero-mean Gaussian field
    with squared-exponential covariance sigma^2 exp(-r^2 / (2 ell^2)).

    Sampled by circulant embedding on a 2nc x 2nc periodic grid (spacing 1/nc); negative
    eigenvalues of the embedding are clipped to zero (an approximate embedding, adequate for a
    synthetic coefficient field)."""
    m = 2 * nc
    k = np.arange(m)
    d = np.minimum(k, m - k) / nc
    r2 = d[:, None] ** 2 + d[None, :] ** 2
    cov = sigma * sigma * np.exp(-r2 / (2.0 * ell * ell))
    lam = np.fft.fft2(cov).real
    lam[lam < 0.0] = 0.0
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    g = np.fft.fft2(np.sqrt(lam / (m * m)) * xi).real[:nc, :nc]
    return np.exp(g)


def fem2d_p1(nc: int, kappa=None, rho=None) -> tuple[Csr, Csr]:
    """P1 triangles on the unit square: nc x nc cells, each cut along its (i,j)-(i+1,j+1) diagonal,
    homogeneous Dirichlet; n = (nc-1)^2 interior nodes numbered x-major (index = (i-1)(nc-1) + (j-1)).

    K_ij = sum_e kappa_e int grad phi_i . grad phi_j,  M_ij = sum_e rho_e int phi_i phi_j,
    with kappa, rho constant per cell (both triangles of a cell share the value).  The
    hypotenuse couplings of K vanish exactly for right isosceles triangles, so K has the
    5-point pattern and M the 7-point pattern."""
    return fem2d_p1_rect(nc, nc, kappa, rho)


def fem2d_p1_rect(nci: int, ncj: int, kappa=None, rho=None) -> tuple[Csr, Csr]:
    """The same P1 discretisation on a rectangle of nci x ncj square cells of side h = 1/max(nci, ncj)
    (kappa, rho of shape (nci, ncj)); n = (nci-1)(ncj-1) interior nodes numbered with j fastest
    (index = (i-1)(ncj-1) + (j-1)), so the bandwidth is ncj (the diagonal neighbour (i+1, j+1))."""
    if kappa is None:
        kappa = np.ones((nci, ncj))
    if rho is None:
        rho = np.ones((nci, ncj))
    h = 1.0 / max(nci, ncj)
    Nj = ncj + 1
    I, J = np.meshgrid(np.arange(nci), np.arange(ncj), indexing="ij")
    a = I * Nj + J
    b = (I + 1) * Nj + J
    c = (I + 1) * Nj + (J + 1)
    d = I * Nj + (J + 1)
    # triangle (a, b, c): right angle at b; triangle (a, c, d): right angle at d
    k1 = np.array([[0.5, -0.5, 0.0], [-0.5, 1.0, -0.5], [0.0, -0.5, 0.5]])
    k2 = np.array([[0.5, 0.0, -0.5], [0.0, 0.5, -0.5], [-0.5, -0.5, 1.0]])
    ml = (h * h / 24.0) * (np.ones((3, 3)) + np.eye(3))
    rows, cols, kv, mv = [], [], [], []
    for tri, kl in (((a, b, c), k1), ((a, c, d), k2)):
        for p in range(3):
            for q in range(3):
                rows.append(tri[p].ravel())
                cols.append(tri[q].ravel())
                kv.append((kappa * kl[p, q]).ravel())
                mv.append((rho * ml[p, q]).ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    nt = (nci + 1) * Nj
    K = sp.csr_matrix((np.concatenate(kv), (rows, cols)), shape=(nt, nt))
    M = sp.csr_matrix((np.concatenate(mv), (rows, cols)), shape=(nt, nt))
    ii, jj = np.meshgrid(np.arange(nci + 1), np.arange(Nj), indexing="ij")
    keep = np.nonzero(((ii > 0) & (ii < nci) & (jj > 0) & (jj < ncj)).ravel())[0]
    K = K[keep][:, keep]
    M = M[keep][:, keep]
    return Csr.from_scipy(K), Csr.from_scipy(M)


def fem2d_p1_strip(nci: int, ncj: int, seeds=(2, 3), sigma: float = 1.0, ell: float = 0.1):
    """A strip of the 2D log-normal P1 family: the first nci rows of cells of the ncj x ncj field's
    grid (same covariance, spacing 1/ncj), so its bandwidth is that of the ncj x ncj pencil (ncj)
    while n = (nci - 1)(ncj - 1) stays small."""
    kappa = grf_lognormal(ncj, ell, sigma, seeds[0])[:nci]
    rho = grf_lognormal(ncj, ell, sigma, seeds[1])[:nci]
    return fem2d_p1_rect(nci, ncj, kappa, rho)


def fem2d_p1_lognormal(nc: int, seeds=(2, 3), sigma: float = 1.0, ell: float = 0.1):
    """2D P1 pencil with independent log-normal fields kappa (in K) and rho (in M)."""
    kappa = grf_lognormal(nc, ell, sigma, seeds[0])
    rho = grf_lognormal(nc, ell, sigma, seeds[1])
    return fem2d_p1(nc, kappa, rho)


def serving_batch(count: int = 64, seed: int = 6):
    """The serving workload: `count` independent pencils of uneven size, alternating a 2D P1 pencil with
    log-normal fields (n = (nc - 1)^2 drawn from U[10k, 200k]) and a 3D Q1 pencil with octant coefficients
    (n = (nc - 1)^3 from U[10k, 27k], where its band stays within the shared-memory sweeps).  Each gets an
    interval meant to hold k ~ U[20, 200] eigenvalues, placed with Weyl's law for -div(kappa grad u) =
    lambda rho u (2D: N(lambda) ~ lambda mean(rho / kappa) / (4 pi); 3D: N(lambda) ~ lambda^(3/2)
    mean((rho / kappa)^(3/2)) / (6 pi^2)), from N = 4.5 to N = 4.5 + k.  Returns a list of
    (K, M, lo, hi, kind)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        k = int(rng.integers(20, 201))
        if i % 2 == 0:
            nc = int(round(np.sqrt(rng.uniform(10_000, 200_000)))) + 1
            kappa = grf_lognormal(nc, 0.1, 1.0, 1000 + 2 * i)
            rho = grf_lognormal(nc, 0.1, 1.0, 1001 + 2 * i)
            K, M = fem2d_p1(nc, kappa, rho)
            c = float(np.mean(rho / kappa)) / (4.0 * np.pi)
            lam = lambda N: N / c
            kind = "2d-p1"
        else:
            nc = int(round(rng.uniform(10_000, 27_000) ** (1.0 / 3.0))) + 1
            ck, cm = octant_coefficients(3, 2000 + 2 * i), octant_coefficients(3, 2001 + 2 * i)
            K, M = fem_q1(nc, 3, ck, cm)
            c = float(np.mean((cm / ck) ** 1.5)) / (6.0 * np.pi ** 2)
            lam = lambda N: (N / c) ** (2.0 / 3.0)
            kind = "3d-q1"
        out.append((K, M, lam(4.5), lam(4.5 + k), kind))
    return out


def family_member(seed: int, nc: int = 256):
    """Member `seed` of the learned-contour family: the 2D log-normal P1 pencil on nc x nc cells with the
    fields of seeds (2 seed + 10, 2 seed + 11).  Returns (K, M, kappa, rho), the fields on the cell grid
    (the density predictor's input)."""
    kappa = grf_lognormal(nc, 0.1, 1.0, 2 * seed + 10)
    rho = grf_lognormal(nc, 0.1, 1.0, 2 * seed + 11)
    K, M = fem2d_p1(nc, kappa, rho)
    return K, M, kappa, rho


# --------------------------------------------------------------------------- Q1 (2D/3D)

def _q1_1d(N1: int, h: float, e0: int, e1: int):
    """1D linear-element stiffness and mass assembled over elements e0..e1-1 of a uniform grid."""
    K = sp.lil_matrix((N1, N1))
    M = sp.lil_matrix((N1, N1))
    for e in range(e0, e1):
        K[e, e] += 1.0 / h; K[e + 1, e + 1] += 1.0 / h
        K[e, e + 1] -= 1.0 / h; K[e + 1, e] -= 1.0 / h
        M[e, e] += 2.0 * h / 6.0; M[e + 1, e + 1] += 2.0 * h / 6.0
        M[e, e + 1] += h / 6.0; M[e + 1, e] += h / 6.0
    return K.tocsr(), M.tocsr()


def fem_q1(nc: int, dim: int, coef_k=None, coef_m=None) -> tuple[Csr, Csr]:
    """Q1 (bi/tri-linear) elements on the unit square/cube, nc cells per side, homogeneous
    Dirichlet, coefficients constant on each of the 2^dim half-size sub-boxes ("octants").

    coef_k / coef_m: arrays of shape (2,)*dim (None = all ones).  On each sub-box the element
    matrices are tensor products of 1D ones, so K = sum_box kappa_box sum_d (K1 in dim d) (x)
    (M1 in the other dims) and M = sum_box rho_box (x)_d M1.  With constant coefficients the
    eigenvalues are the sums of 1D `fem1d` eigenvalues.  Node index is x-major."""
    if coef_k is None:
        coef_k = np.ones((2,) * dim)
    if coef_m is None:
        coef_m = np.ones((2,) * dim)
    h = 1.0 / nc
    N1 = nc + 1
    halves = [(0, nc // 2), (nc // 2, nc)]
    parts = {s: _q1_1d(N1, h, *halves[s]) for s in (0, 1)}
    K = None
    M = None
    for box in np.ndindex(*((2,) * dim)):
        k1 = [parts[s][0] for s in box]
        m1 = [parts[s][1] for s in box]
        mm = m1[0]
        for t in range(1, dim):
            mm = sp.kron(mm, m1[t], format="csr")
        kk = None
        for d in range(dim):
            term = k1[0] if d == 0 else m1[0]
            for t in range(1, dim):
                term = sp.kron(term, k1[t] if t == d else m1[t], format="csr")
            kk = term if kk is None else kk + term
        kk = kk * float(coef_k[box])
        mm = mm * float(coef_m[box])
        K = kk if K is None else K + kk
        M = mm if M is None else M + mm
    grids = np.meshgrid(*([np.arange(N1)] * dim), indexing="ij")
    inside = np.ones(grids[0].shape, dtype=bool)
    for g in grids:
        inside &= (g > 0) & (g < nc)
    keep = np.nonzero(inside.ravel())[0]
    K = sp.csr_matrix(K)[keep][:, keep]
    M = sp.csr_matrix(M)[keep][:, keep]
    return Csr.from_scipy(K), Csr.from_scipy(M)


def octant_coefficients(dim: int, seed: int, ratio: float = 1e3) -> np.ndarray:
    """Piecewise-constant coefficients, log-uniform in [1, ratio], one per half-size sub-box."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(0.0, np.log(ratio), size=(2,) * dim))


# --------------------------------------------------------------------------- random block

def gaussian_block(n: int, L: int, seed: int) -> np.ndarray:
    """The random starting block V (n x L, row-major float64), entries N(0, 1)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, L)))


# --------------------------------------------------------------------------- named workloads

_GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")

WORKLOADS = {
    # 1D linear FEM, n = 2000; eigenvalues 10..60 with one contour, 16 nodes, L = 32, 2 moments.
    "fem1d-n2000": dict(kind="fem1d", n=2000, first=10, last=60, contours=1, nodes=16, L=32, moments=2),
    # 2D P1 on a 500 x 500 grid with log-normal fields (sigma 1, correlation length 0.1);
    # eigenvalues 101..400 with 8 equal-width contours, 16 nodes, L = 64, 2 moments.
    "fem2d-p1-500": dict(kind="fem2d", nc=500, seeds=(2, 3), first=101, last=400, contours=8, nodes=16,
                         L=64, moments=2, golden="fem2d_p1_500.json"),
    # Smaller members of the same 2D family (parity sizes the oracle finishes in seconds).
    "fem2d-p1-40": dict(kind="fem2d", nc=40, seeds=(2, 3), first=11, last=60, contours=2, nodes=16,
                        L=32, moments=2, golden="fem2d_p1_40.json"),
    # A reduced member of the 500 x 500 workload (160 x 160 cells, n = 25281, bandwidth 160) with the same
    # solver configuration (8 contours x 16 nodes, L = 64, 2 moments): the oracle's timed whole solve.
    "fem2d-p1-160": dict(kind="fem2d", nc=160, seeds=(2, 3), first=11, last=40, contours=8, nodes=16,
                         L=64, moments=2, golden="fem2d_p1_160.json"),
    # A strip of the 500 x 500 family (12 x 500 cells, n = 11 x 499 = 5489) with the bench workload's
    # bandwidth (500): parity of the band kernels at full bandwidth, eigenvalues 21..60.
    "fem2d-p1-strip": dict(kind="fem2d_strip", nci=12, ncj=500, seeds=(2, 3), first=21, last=60, contours=2,
                           nodes=16, L=32, moments=2, golden="fem2d_p1_strip.json"),
}


def workload(name: str):
    """Return (K, M, spec) for a named workload; spec carries the solver configuration and, where the
    interval endpoints come from a stored inertia computation, lo/hi/count from tests/golden."""
    spec = dict(WORKLOADS[name])
    if spec["kind"] == "fem1d":
        K, M = fem1d(spec["n"])
        lam = fem1d_eigenvalue(np.arange(1, spec["n"] + 1), spec["n"])
        f, l = spec["first"], spec["last"]
        spec["lo"] = 0.5 * (lam[f - 2] + lam[f - 1])
        spec["hi"] = 0.5 * (lam[l - 1] + lam[l])
        spec["count"] = l - f + 1
    elif spec["kind"] in ("fem2d", "fem2d_strip"):
        if spec["kind"] == "fem2d":
            K, M = fem2d_p1_lognormal(spec["nc"], spec["seeds"])
        else:
            K, M = fem2d_p1_strip(spec["nci"], spec["ncj"], spec["seeds"])
        g = spec.get("golden")
        if g and os.path.exists(os.path.join(_GOLDEN, g)):
            with open(os.path.join(_GOLDEN, g)) as fh:
                spec.update(json.load(fh))
    else:
        raise KeyError(name)
    return K, M, spec
