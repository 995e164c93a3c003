"""Write the stored interval endpoints of the 2D workloads (tests/golden/fem2d_p1_*.json).

The paper prints no worked example, so these files hold only values computed here by the
oracle: for a workload asking for eigenvalues first..last (1-based, ascending), lo and hi are
placed at the midpoints of the spectral gaps (lambda_{first-1}, lambda_first) and
(lambda_last, lambda_{last+1}), each eigenvalue located by multisection on the oracle's
Sylvester-inertia count of LDL^T(K - sigma M).  `count` is the oracle's inertia count of
[lo, hi], and `gap_lo`, `gap_hi` the distances from the endpoints to the nearest eigenvalue.

Usage: python tests/golden/make_golden.py fem2d-p1-40 [fem2d-p1-500 ...]
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

_KM = None


def _init(name):
    global _KM
    import pencils
    K, M, _ = pencils.workload(name)
    _KM = (K, M)


def _count(sigma):
    import oracle
    return oracle.inertia_count(_KM[0], _KM[1], sigma)


def locate(pool, k, a, b, ca, cb, rel=1e-6, ways=8):
    """Bracket lambda_k (count(a) < k <= count(b)) to relative width rel by multisection."""
    while (b - a) > rel * abs(b):
        pts = list(np.linspace(a, b, ways + 1)[1:-1])
        cs = pool.map(_count, pts)
        grid = [(a, ca)] + list(zip(pts, cs)) + [(b, cb)]
        for (x0, c0), (x1, c1) in zip(grid[:-1], grid[1:]):
            if c0 < k <= c1:
                a, ca, b, cb = x0, c0, x1, c1
                break
    return 0.5 * (a + b)


def main(name):
    import pencils
    spec = pencils.WORKLOADS[name]
    first, last = spec["first"], spec["last"]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1), initializer=_init, initargs=(name,)) as pool:
        # a bracket [0, top] holding eigenvalues 1..last+1
        top = 1.0
        while pool.map(_count, [top])[0] < last + 1:
            top *= 2.0
        c_top = pool.map(_count, [top])[0]
        lam = {}
        for k in (first - 1, first, last, last + 1):
            lam[k] = locate(pool, k, 0.0, top, 0, c_top)
        lo = 0.5 * (lam[first - 1] + lam[first])
        hi = 0.5 * (lam[last] + lam[last + 1])
        c_lo, c_hi = pool.map(_count, [lo, hi])
    out = dict(lo=lo, hi=hi, count=int(c_hi - c_lo), below_lo=int(c_lo),
               gap_lo=0.5 * (lam[first] - lam[first - 1]), gap_hi=0.5 * (lam[last + 1] - lam[last]),
               note="written by tests/golden/make_golden.py from oracle.inertia_count")
    assert out["count"] == last - first + 1 and out["below_lo"] == first - 1, out
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), spec["golden"])
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(name, out)


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        main(nm)
