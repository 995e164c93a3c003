"""Host-side checks of the C-ABI library (no GPU): it builds, loads, exports every symbol the header
declares, and its host-only helpers agree with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle as O
import pencils as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    from paper_2511_01927_gb300 import build
    build.build()
    import paper_2511_01927_gb300 as G
    G.lib()
    return G


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gcie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gcie_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(G):
    syms = declared_symbols()
    assert len(syms) >= 20
    lib = G.lib()
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(G.EXPORTED_SYMBOLS) == syms


def test_strerror_and_default_opts(G):
    lib = G.lib()
    assert lib.gcie_strerror(0) == b"ok"
    assert lib.gcie_strerror(5) == b"not converged"
    o = G.default_opts()
    assert (o.nodes, o.L, o.moments, o.tol, o.expected_count) == (16, 32, 2, 1e-10, -1)


@pytest.mark.parametrize("N", [2, 8, 16, 32])
def test_trapezoid_nodes_match_oracle(G, N):
    z, w = G.gcie_trapezoid_nodes(3.5, 0.75, N)
    zo, wo = O.trapezoid_nodes(3.5, 0.75, N)
    assert np.max(np.abs(z - zo)) < 1e-15 and np.max(np.abs(w - wo)) < 1e-15
    assert np.all(z.imag > 0)


def test_trapezoid_rejects_odd(G):
    with pytest.raises(G.GcieError):
        G.gcie_trapezoid_nodes(0.0, 1.0, 7)


def test_create_without_gpu_fails_cleanly(G):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(G.GcieError) as e:
        G.gcie_create(0)
    assert e.value.code == 1


def test_generators_deterministic_and_symmetric():
    K1, M1 = P.fem2d_p1_lognormal(20)
    K2, M2 = P.fem2d_p1_lognormal(20)
    assert np.array_equal(K1.val, K2.val) and np.array_equal(M1.val, M2.val)
    for A in (K1, M1):
        S = A.to_scipy()
        assert abs(S - S.T).max() <= 1e-14 * abs(S).max()
    assert np.all(M1.to_scipy().diagonal() > 0)
    V1 = P.gaussian_block(100, 4, 9)
    assert np.array_equal(V1, P.gaussian_block(100, 4, 9))


def test_golden_interval_counts_match_oracle_inertia():
    K, M, spec = P.workload("fem2d-p1-40")
    assert O.count_in(K, M, spec["lo"], spec["hi"]) == spec["count"] == spec["last"] - spec["first"] + 1
    assert O.inertia_count(K, M, spec["lo"]) == spec["first"] - 1


def header_struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in include/gcie.h."""
    src = open(os.path.join(ROOT, "include", "gcie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        for part in decl.split(","):          # "double c, r": one field per declarator
            if part.strip():
                fields.append(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", part)[-1])
    return fields


@pytest.mark.parametrize("cname,pyname", [("gcie_opts", "Opts"), ("gcie_contour", "Contour")])
def test_binding_structs_follow_the_header(G, cname, pyname):
    """The ctypes mirrors of the ABI structs list the header's fields in the header's order."""
    from paper_2511_01927_gb300 import _binding as B
    assert [f[0] for f in getattr(B, pyname)._fields_] == header_struct_fields(cname)
