"""ctypes marshalling for libgcie.so (include/gcie.h).  No arithmetic of the method lives here."""
from __future__ import annotations

import ctypes as C
import weakref
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgcie.so")

STATUS = {0: "GCIE_OK", 1: "GCIE_EINVAL", 2: "GCIE_ENOTSYM", 3: "GCIE_ENOTSPD", 4: "GCIE_ENOMEM",
          5: "GCIE_ENOCONV", 6: "GCIE_EBREAKDOWN", 7: "GCIE_ETIMEOUT", 8: "GCIE_ECOUNT", 9: "GCIE_ECUDA",
          10: "GCIE_ECONTEXT"}
MIXED, FP64 = 0, 1

EXPORTED_SYMBOLS = [
    "gcie_create", "gcie_destroy", "gcie_default_opts", "gcie_strerror", "gcie_last_error", "gcie_get_stats",
    "gcie_reset_stats", "gcie_set_profile", "gcie_pencil_create", "gcie_pencil_destroy", "gcie_pencil_n", "gcie_pencil_nnz",
    "gcie_solve", "gcie_solve_pencil", "gcie_solve_batch", "gcie_result_free", "gcie_buffer_free", "gcie_kde_contours", "gcie_plan_contours", "gcie_count_miss", "gcie_resplit", "gcie_trapezoid_nodes", "gcie_shifted_spmm_f32",
    "gcie_shifted_spmm_f64", "gcie_shifted_solve", "gcie_moments", "gcie_m_orthonormalize",
    "gcie_rayleigh_ritz", "gcie_jacobi_eig", "gcie_jacobi_eig_noalloc", "gcie_gemm_tf32x3", "gcie_gemm_bf16",
    "gcie_density_net_create", "gcie_density_net_destroy", "gcie_density_predict", "gcie_hist_quantiles",
    "gcie_fp64_rates",
]
DENSITY_NWEIGHTS = 717520
DENSITY_BINS = 256


class GcieError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} {msg}")


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class Contour(C.Structure):
    _fields_ = [("c", C.c_double), ("r", C.c_double), ("lo", C.c_double), ("hi", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("nodes", C.c_int32), ("L", C.c_int32), ("moments", C.c_int32), ("max_outer", C.c_int32),
                ("max_iters", C.c_int32), ("precision", C.c_int32), ("tol", C.c_double), ("lin_tol", C.c_double),
                ("ncontours", C.c_int32), ("nuniform", C.c_int32), ("contours", C.c_void_p), ("alpha", C.c_double),
                ("h_V0", C.c_void_p), ("seed", C.c_uint64), ("hbm_budget_bytes", C.c_size_t),
                ("expected_count", C.c_int32), ("profile", C.c_int32), ("precond", C.c_int32),
                ("judge", C.c_int32), ("max_resplit", C.c_int32), ("batch_streams", C.c_int32),
                ("lin_tol_first", C.c_double)]


class Result(C.Structure):
    _fields_ = [("n", C.c_int64), ("count", C.c_int32), ("evals", C.POINTER(C.c_double)),
                ("evecs", C.POINTER(C.c_double)), ("resid", C.POINTER(C.c_double)),
                ("contour_of", C.POINTER(C.c_int32)), ("ncontours", C.c_int32),
                ("status_per_contour", C.POINTER(C.c_int32)), ("iters_per_contour", C.POINTER(C.c_int32)),
                ("outer_iters", C.c_int32), ("cocg_iters", C.c_int64), ("norm_k1", C.c_double),
                ("contours", C.POINTER(Contour)), ("count_estimate", C.POINTER(C.c_double)),
                ("resplits", C.c_int32)]


NCLASS = 8
KERNEL_CLASSES = ["spmm_dir", "spmm_upd", "refine", "moment", "dense", "other", "prec", "factor"]


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64 * NCLASS), ("ms", C.c_double * NCLASS), ("bytes", C.c_double * NCLASS),
                ("flops", C.c_double * NCLASS), ("total_launches", C.c_int64)]


_lib = None


def library_path() -> str:
    return _SO


def lib():
    """Load libgcie.so (built in-tree by paper_2511_01927_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO):
        raise RuntimeError(f"libgcie.so not built ({_SO}); run paper_2511_01927_gb300.build.build()")
    L = C.CDLL(_SO)
    vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "gcie_create": (C.c_int, [C.POINTER(vp), C.c_int, vp]),
        "gcie_destroy": (None, [vp]),
        "gcie_default_opts": (None, [C.POINTER(Opts)]),
        "gcie_strerror": (C.c_char_p, [C.c_int]),
        "gcie_last_error": (C.c_char_p, []),
        "gcie_get_stats": (C.c_int, [vp, C.POINTER(Stats)]),
        "gcie_reset_stats": (None, [vp]),
        "gcie_set_profile": (None, [vp, C.c_int]),
        "gcie_pencil_create": (C.c_int, [vp, C.POINTER(Csr), C.POINTER(Csr), C.POINTER(vp)]),
        "gcie_pencil_destroy": (None, [vp]),
        "gcie_pencil_n": (i64, [vp]),
        "gcie_pencil_nnz": (i64, [vp]),
        "gcie_solve": (C.c_int, [vp, C.POINTER(Csr), C.POINTER(Csr), d, d, C.POINTER(Opts), C.POINTER(Result)]),
        "gcie_solve_pencil": (C.c_int, [vp, vp, d, d, C.POINTER(Opts), C.POINTER(Result)]),
        "gcie_solve_batch": (C.c_int, [vp, i32, vp, vp, vp, vp, C.POINTER(Opts), vp]),
        "gcie_result_free": (None, [C.POINTER(Result)]),
        "gcie_buffer_free": (None, [vp]),
        "gcie_trapezoid_nodes": (C.c_int, [d, d, i32, vp, vp]),
        "gcie_kde_contours": (C.c_int, [vp, i32, i32, i32, d, d, d, vp, vp, i32, C.POINTER(i32)]),
        "gcie_plan_contours": (C.c_int, [vp, i32, d, d, i32, d, vp, vp, i32, C.POINTER(i32)]),
        "gcie_count_miss": (C.c_int, [d, d, vp, vp, i32, d, d, i32, d, C.POINTER(i32)]),
        "gcie_resplit": (C.c_int, [vp, i32, C.POINTER(Contour), d, vp]),
        "gcie_shifted_spmm_f32": (C.c_int, [vp, vp, i32, vp, i32, vp, vp]),
        "gcie_shifted_spmm_f64": (C.c_int, [vp, vp, i32, vp, i32, vp, vp]),
        "gcie_shifted_solve": (C.c_int, [vp, vp, i32, vp, i32, vp, vp, i32, d, i32, i32, i32, C.POINTER(i64)]),
        "gcie_moments": (C.c_int, [vp, i64, i32, vp, vp, d, d, i32, i32, vp, vp]),
        "gcie_m_orthonormalize": (C.c_int, [vp, vp, i32, vp, d, vp, C.POINTER(i32)]),
        "gcie_rayleigh_ritz": (C.c_int, [vp, vp, i32, vp, vp, vp, vp]),
        "gcie_jacobi_eig": (C.c_int, [vp, i32, vp, vp, vp]),
        "gcie_jacobi_eig_noalloc": (C.c_int, [vp, i32, vp, vp, vp]),
        "gcie_gemm_tf32x3": (C.c_int, [vp, i32, i32, i32, vp, i32, vp, i32, vp, i32]),
        "gcie_gemm_bf16": (C.c_int, [vp, i32, i32, i32, vp, i32, vp, i32, vp, i32, vp, i32]),
        "gcie_density_net_create": (C.c_int, [vp, vp, i64, C.POINTER(vp)]),
        "gcie_density_net_destroy": (None, [vp]),
        "gcie_density_predict": (C.c_int, [vp, vp, i32, i32, vp, vp, vp, vp]),
        "gcie_hist_quantiles": (C.c_int, [vp, i32, d, d, vp, i32, C.POINTER(i32)]),
        "gcie_fp64_rates": (C.c_int, [vp, C.POINTER(d), C.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int, where: str, allow=()):
    if rc != 0 and rc not in allow:
        raise GcieError(rc, where, lib().gcie_last_error().decode())
    return rc


def _ptr(x) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


# ------------------------------------------------------------------ host structs

class _HostCsr:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, A):
        self.rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(A.col, dtype=np.int32)
        self.val = np.ascontiguousarray(A.val, dtype=np.float64)
        self.s = Csr(int(A.n), int(self.rowptr[-1]), self.rowptr.ctypes.data, self.col.ctypes.data,
                     self.val.ctypes.data)


def csr_struct(A) -> _HostCsr:
    return _HostCsr(A)


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().gcie_default_opts(C.byref(o))
    for k, v in kw.items():
        if k in ("contours", "h_V0"):
            continue
        setattr(o, k, v)
    return o


class _OptsHolder:
    def __init__(self, kw):
        kw = dict(kw)
        self.contours = kw.pop("contours", None)
        V0 = kw.pop("V0", None)
        self.o = default_opts(**kw)
        if self.contours is not None:
            arr = (Contour * len(self.contours))(*[Contour(*map(float, cc)) for cc in self.contours])
            self._carr = arr
            self.o.contours = C.cast(arr, C.c_void_p)
            self.o.ncontours = len(self.contours)
        if V0 is not None:
            self.V0 = np.ascontiguousarray(V0, dtype=np.float64)
            self.o.h_V0 = self.V0.ctypes.data
            self.o.L = self.V0.shape[1]


# ------------------------------------------------------------------ context / pencil

def gcie_create(device: int = 0, stream: int | None = None):
    h = C.c_void_p()
    _check(lib().gcie_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None), "gcie_create")
    return h


def gcie_destroy(ctx):
    lib().gcie_destroy(ctx)


def gcie_get_stats(ctx) -> dict:
    s = Stats()
    _check(lib().gcie_get_stats(ctx, C.byref(s)), "gcie_get_stats")
    return {name: dict(launches=int(s.launches[i]), ms=float(s.ms[i]), bytes=float(s.bytes[i]), flops=float(s.flops[i]))
            for i, name in enumerate(KERNEL_CLASSES)} | {"total_launches": int(s.total_launches)}


def gcie_reset_stats(ctx):
    lib().gcie_reset_stats(ctx)


def gcie_set_profile(ctx, on: bool):
    lib().gcie_set_profile(ctx, int(bool(on)))


def gcie_pencil_create(ctx, K, M):
    hk, hm = _HostCsr(K), _HostCsr(M)
    h = C.c_void_p()
    _check(lib().gcie_pencil_create(ctx, C.byref(hk.s), C.byref(hm.s), C.byref(h)), "gcie_pencil_create")
    return h


def gcie_pencil_destroy(p):
    lib().gcie_pencil_destroy(p)


def _take_evecs(r: Result, n: int, k: int):
    """The eigenvectors as an n x k view of the library's buffer, no copy: the pointer is taken out
    of the result (gcie_result_free then skips it) and freed by gcie_buffer_free when the array is
    garbage collected."""
    if not k:
        return np.zeros((n, 0))
    ptr = C.cast(r.evecs, C.c_void_p).value
    arr = np.ctypeslib.as_array(r.evecs, (k, n))
    r.evecs = C.POINTER(C.c_double)()
    weakref.finalize(arr, lib().gcie_buffer_free, C.c_void_p(ptr))
    return arr.T


def _take_result(r: Result) -> dict:
    n, k = int(r.n), int(r.count)
    out = dict(
        evals=np.ctypeslib.as_array(r.evals, (k,)).copy() if k else np.zeros(0),
        evecs=_take_evecs(r, n, k),
        resid=np.ctypeslib.as_array(r.resid, (k,)).copy() if k else np.zeros(0),
        contour_of=np.ctypeslib.as_array(r.contour_of, (k,)).copy() if k else np.zeros(0, np.int32),
        status=[int(r.status_per_contour[i]) for i in range(r.ncontours)] if r.status_per_contour else [],
        iters=[int(r.iters_per_contour[i]) for i in range(r.ncontours)] if r.iters_per_contour else [],
        outer_iters=int(r.outer_iters), cocg_iters=int(r.cocg_iters), norm_k1=float(r.norm_k1),
        contours=[(r.contours[i].c, r.contours[i].r, r.contours[i].lo, r.contours[i].hi) for i in range(r.ncontours)]
        if r.contours else [],
        count_estimate=np.array([r.count_estimate[i] for i in range(r.ncontours)]) if r.count_estimate else np.zeros(0),
        resplits=int(r.resplits))
    lib().gcie_result_free(C.byref(r))
    return out


def _check_result(rc: int, r: Result, where: str, allow_noconv: bool):
    """Raise for a failed solve, releasing what the library put into the result first."""
    try:
        _check(rc, where, allow=(5,) if allow_noconv else ())
    except GcieError:
        lib().gcie_result_free(C.byref(r))
        raise


def gcie_solve_batch(ctx, pencils, allow_noconv: bool = False, **opts) -> list:
    """Independent pencils [(K, M, lo, hi), ...] with the same options (gcie_opts fields as keywords);
    a list of results as gcie_solve returns them."""
    hs = [(_HostCsr(K), _HostCsr(M)) for K, M, _, _ in pencils]
    npen = len(hs)
    Ks = (Csr * npen)(*[h[0].s for h in hs])
    Ms = (Csr * npen)(*[h[1].s for h in hs])
    lo = np.ascontiguousarray([float(p[2]) for p in pencils], dtype=np.float64)
    hi = np.ascontiguousarray([float(p[3]) for p in pencils], dtype=np.float64)
    oh = _OptsHolder(opts)
    res = (Result * max(npen, 1))()
    rc = lib().gcie_solve_batch(ctx, npen, C.cast(Ks, C.c_void_p), C.cast(Ms, C.c_void_p), lo.ctypes.data,
                                hi.ctypes.data, C.byref(oh.o), C.cast(res, C.c_void_p))
    if rc != 0 and not (allow_noconv and rc == 5):
        for i in range(npen):
            lib().gcie_result_free(C.byref(res[i]))
        _check(rc, "gcie_solve_batch")
    outs = []
    for i in range(npen):
        o = _take_result(res[i])
        o["rc"] = rc
        outs.append(o)
    return outs


def gcie_solve(ctx, K, M, lo: float, hi: float, allow_noconv: bool = False, **opts) -> dict:
    """All eigenpairs in [lo, hi] from host CSR matrices (pencils.Csr-like objects).  Keyword
    options are the gcie_opts fields; `contours` = list of (c, r, lo, hi); `V0` = n x L block."""
    hk, hm = _HostCsr(K), _HostCsr(M)
    oh = _OptsHolder(opts)
    r = Result()
    rc = lib().gcie_solve(ctx, C.byref(hk.s), C.byref(hm.s), float(lo), float(hi), C.byref(oh.o), C.byref(r))
    _check_result(rc, r, "gcie_solve", allow_noconv)
    out = _take_result(r)
    out["rc"] = rc
    return out


def gcie_solve_pencil(ctx, pencil, lo: float, hi: float, allow_noconv: bool = False, **opts) -> dict:
    oh = _OptsHolder(opts)
    r = Result()
    rc = lib().gcie_solve_pencil(ctx, pencil, float(lo), float(hi), C.byref(oh.o), C.byref(r))
    _check_result(rc, r, "gcie_solve_pencil", allow_noconv)
    out = _take_result(r)
    out["rc"] = rc
    return out


# ------------------------------------------------------------------ steps (device buffers)

def gcie_kde_contours(pred, nmin: int = 10, nmax: int = 50, w: float = 10.0, alpha: float = 0.0,
                      beta: float = 0.0) -> list:
    """Contours from predicted eigenvalues (Algorithm 2); a list of (lo, hi, c, r, count)."""
    p = np.ascontiguousarray(np.asarray(pred, dtype=np.float64).ravel())
    n = C.c_int32(0)
    cap = max(1, p.size)
    out = (Contour * cap)()
    counts = np.zeros(cap, dtype=np.int32)
    _check(lib().gcie_kde_contours(p.ctypes.data, int(p.size), int(nmin), int(nmax), float(w), float(alpha),
                                   float(beta), C.cast(out, C.c_void_p), counts.ctypes.data, cap, C.byref(n)),
           "gcie_kde_contours")
    return [(out[i].lo, out[i].hi, out[i].c, out[i].r, int(counts[i])) for i in range(n.value)]


def gcie_plan_contours(pred, lo: float, hi: float, max_contours: int, alpha: float = 0.0) -> list:
    """Contours for a fixed budget, cut in gaps of the predicted spectrum; a list of
    (lo, hi, c, r, count)."""
    p = np.ascontiguousarray(np.asarray(pred, dtype=np.float64).ravel())
    n = C.c_int32(0)
    cap = max(1, int(max_contours))
    out = (Contour * cap)()
    counts = np.zeros(cap, dtype=np.int32)
    _check(lib().gcie_plan_contours(p.ctypes.data if p.size else None, int(p.size), float(lo), float(hi),
                                    int(max_contours), float(alpha), C.cast(out, C.c_void_p), counts.ctypes.data,
                                    cap, C.byref(n)), "gcie_plan_contours")
    return [(out[i].lo, out[i].hi, out[i].c, out[i].r, int(counts[i])) for i in range(n.value)]


def gcie_count_miss(est: float, se: float, theta, res, c: float, r: float, rank: int, tol: float) -> bool:
    """Count check of a finished contour (trace estimate against the Ritz count)."""
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).ravel())
    rs = np.ascontiguousarray(np.asarray(res, dtype=np.float64).ravel())
    if th.size != rs.size:
        raise ValueError("theta and res differ in length")
    miss = C.c_int32(0)
    _check(lib().gcie_count_miss(float(est), float(se), th.ctypes.data, rs.ctypes.data, int(th.size), float(c),
                                 float(r), int(rank), float(tol), C.byref(miss)), "gcie_count_miss")
    return bool(miss.value)


def gcie_resplit(theta, c: float, r: float, lo: float, hi: float, w: float = 10.0) -> list:
    """The two halves (c, r, lo, hi) of a contour that failed the count check."""
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).ravel())
    parent = Contour(float(c), float(r), float(lo), float(hi))
    out = (Contour * 2)()
    _check(lib().gcie_resplit(th.ctypes.data, int(th.size), C.byref(parent), float(w), C.cast(out, C.c_void_p)),
           "gcie_resplit")
    return [(o.c, o.r, o.lo, o.hi) for o in out]


def gcie_trapezoid_nodes(c: float, r: float, N: int):
    z = np.zeros(N // 2, dtype=np.complex128)
    w = np.zeros(N // 2, dtype=np.complex128)
    _check(lib().gcie_trapezoid_nodes(float(c), float(r), int(N), z.ctypes.data, w.ctypes.data), "gcie_trapezoid_nodes")
    return z, w


def _zarr(z):
    return np.ascontiguousarray(np.asarray(z, dtype=np.complex128).ravel())


def gcie_shifted_spmm_f32(ctx, pencil, z, ncol: int, d_P, d_Q):
    zz = _zarr(z)
    _check(lib().gcie_shifted_spmm_f32(ctx, pencil, len(zz), zz.ctypes.data, int(ncol), _ptr(d_P), _ptr(d_Q)),
           "gcie_shifted_spmm_f32")


def gcie_shifted_spmm_f64(ctx, pencil, z, ncol: int, d_P, d_Q):
    zz = _zarr(z)
    _check(lib().gcie_shifted_spmm_f64(ctx, pencil, len(zz), zz.ctypes.data, int(ncol), _ptr(d_P), _ptr(d_Q)),
           "gcie_shifted_spmm_f64")


def gcie_shifted_solve(ctx, pencil, z, ncol: int, d_B, d_X, x0: bool = False, lin_tol: float = 1e-11,
                       max_iters: int = 5000, precision: int = MIXED, precond: int = 1, allow_noconv: bool = False):
    zz = _zarr(z)
    it = C.c_int64(0)
    rc = lib().gcie_shifted_solve(ctx, pencil, len(zz), zz.ctypes.data, int(ncol), _ptr(d_B), _ptr(d_X), int(bool(x0)),
                                  float(lin_tol), int(max_iters), int(precision), int(precond), C.byref(it))
    _check(rc, "gcie_shifted_solve", allow=(5,) if allow_noconv else ())
    return int(it.value), rc


def gcie_moments(ctx, n: int, z, w, c: float, r: float, m: int, ncol: int, d_X, d_S):
    zz, ww = _zarr(z), _zarr(w)
    _check(lib().gcie_moments(ctx, int(n), len(zz), zz.ctypes.data, ww.ctypes.data, float(c), float(r), int(m),
                              int(ncol), _ptr(d_X), _ptr(d_S)), "gcie_moments")


def gcie_m_orthonormalize(ctx, pencil, ncolY: int, d_Y, drop: float, d_Q) -> int:
    rank = C.c_int32(0)
    _check(lib().gcie_m_orthonormalize(ctx, pencil, int(ncolY), _ptr(d_Y), float(drop), _ptr(d_Q), C.byref(rank)),
           "gcie_m_orthonormalize")
    return int(rank.value)


def gcie_rayleigh_ritz(ctx, pencil, q: int, d_Q, d_Z):
    th = np.zeros(q)
    rs = np.zeros(q)
    _check(lib().gcie_rayleigh_ritz(ctx, pencil, int(q), _ptr(d_Q), _ptr(d_Z), th.ctypes.data, rs.ctypes.data),
           "gcie_rayleigh_ritz")
    return th, rs


def gcie_jacobi_eig(ctx, p: int, d_A, d_w, d_V):
    _check(lib().gcie_jacobi_eig(ctx, int(p), _ptr(d_A), _ptr(d_w), _ptr(d_V)), "gcie_jacobi_eig")


def gcie_jacobi_eig_noalloc(stream, p: int, d_A, d_w, d_V):
    """Allocation-free variant (stream: a cudaStream_t handle as int, or None)."""
    _check(lib().gcie_jacobi_eig_noalloc(C.c_void_p(stream) if stream else None, int(p), _ptr(d_A), _ptr(d_w),
                                         _ptr(d_V)), "gcie_jacobi_eig_noalloc")


def gcie_gemm_tf32x3(ctx, M: int, N: int, K: int, d_A, lda: int, d_B, ldb: int, d_D, ldd: int):
    """D = A B^T on the tensor cores, FP32 operands split into TF32 head and tail (device pointers)."""
    _check(lib().gcie_gemm_tf32x3(ctx, int(M), int(N), int(K), _ptr(d_A), int(lda), _ptr(d_B), int(ldb), _ptr(d_D),
                                  int(ldd)), "gcie_gemm_tf32x3")


def gcie_gemm_bf16(ctx, M: int, N: int, K: int, d_A, lda: int, d_B, ldb: int, d_bias, relu: bool, d_D, ldd: int):
    """D = act(A B^T + bias) on the tensor cores, BF16 operands (device tensors of dtype bfloat16)."""
    _check(lib().gcie_gemm_bf16(ctx, int(M), int(N), int(K), _ptr(d_A), int(lda), _ptr(d_B), int(ldb), _ptr(d_bias),
                                int(bool(relu)), _ptr(d_D), int(ldd)), "gcie_gemm_bf16")


def gcie_density_net_create(ctx, weights):
    """Upload the density predictor's weights (float32, the gcie.h order); returns the net handle."""
    w = np.ascontiguousarray(weights, dtype=np.float32).ravel()
    out = C.c_void_p()
    _check(lib().gcie_density_net_create(ctx, w.ctypes.data, int(w.size), C.byref(out)), "gcie_density_net_create")
    return out


def gcie_density_net_destroy(net):
    lib().gcie_density_net_destroy(net)


def gcie_density_predict(ctx, net, kappa, rho, bounds) -> np.ndarray:
    """Predicted eigenvalue histograms (batch x 256) from fields kappa, rho (batch x G x G) and bounds
    (batch x 2: lo, hi)."""
    k = np.ascontiguousarray(kappa, dtype=np.float32)
    r = np.ascontiguousarray(rho, dtype=np.float32)
    if k.ndim == 2:
        k, r = k[None], r[None]
    b = np.ascontiguousarray(bounds, dtype=np.float64).reshape(-1, 2)
    B, G = k.shape[0], k.shape[1]
    hist = np.zeros((B, DENSITY_BINS))
    _check(lib().gcie_density_predict(ctx, net, B, G, k.ctypes.data, r.ctypes.data, b.ctypes.data, hist.ctypes.data),
           "gcie_density_predict")
    return hist


def gcie_hist_quantiles(hist, lo: float, hi: float) -> np.ndarray:
    """Pseudo-eigenvalues of a predicted histogram over [lo, hi]."""
    h = np.ascontiguousarray(hist, dtype=np.float64)
    cap = int(np.floor(h.sum() + 0.5)) + 1
    out = np.zeros(cap)
    nout = C.c_int32(0)
    _check(lib().gcie_hist_quantiles(h.ctypes.data, int(h.size), float(lo), float(hi), out.ctypes.data, cap,
                                     C.byref(nout)), "gcie_hist_quantiles")
    return out[:nout.value].copy()


def gcie_fp64_rates(ctx) -> tuple:
    """Measured FP64 TFLOP/s of the GPU: (CUDA-core FMA, FP64 MMA)."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    _check(lib().gcie_fp64_rates(ctx, C.byref(a), C.byref(b)), "gcie_fp64_rates")
    return float(a.value), float(b.value)
