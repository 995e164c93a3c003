"""Host logic of bench.py's predicted-contour modes on CPU: the solve that supplies the prediction
is replaced by a fixed spectrum, the contour construction runs in the library (host-only calls).
Checks that the options tile the target interval, turn the count check on and drop the uniform
split."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def G():
    from paper_2511_01927_gb300 import build
    build.build()
    import paper_2511_01927_gb300 as G
    G.lib()
    return G


class _Solver:
    """The library with the prediction's solve replaced by a fixed, seeded spectrum."""

    def __init__(self, G):
        self.G = G

    def __getattr__(self, name):
        return getattr(self.G, name)

    def gcie_solve_pencil(self, ctx, pen, lo, hi, **opts):
        rng = np.random.default_rng(0)
        return {"evals": np.sort(rng.uniform(lo + 1.0, hi - 1.0, 300))}


@pytest.mark.parametrize("kind", ["kde", "planned"])
def test_predicted_contour_options(G, kind):
    import bench
    spec = {"lo": 427.5, "hi": 1604.5, "contours": 8, "count": 300}
    opts = dict(nodes=16, moments=2, nuniform=8, V0=None, tol=1e-10, expected_count=300)
    o, info = bench.predicted_opts(_Solver(G), None, None, spec, opts, 0.1, kind)
    cts = o["contours"]
    assert o["judge"] == 1 and "nuniform" not in o and o["expected_count"] == 300
    assert cts[0][2] == spec["lo"] and cts[-1][3] == spec["hi"]
    assert all(a[3] == b[2] for a, b in zip(cts, cts[1:]))
    assert all(c == 0.5 * (a + b) and r == 0.5 * (b - a) for c, r, a, b in cts)
    assert sum(info["predicted_counts"]) == 300 and len(info["edges"]) == len(cts) + 1
    if kind == "planned":
        assert len(cts) == spec["contours"]
