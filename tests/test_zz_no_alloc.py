"""The allocation-free Jacobi entry point (gcie_jacobi_eig_noalloc) against the regular one.

For callers that cannot allocate device memory (a fixed up-front reservation, or a stream that must
not see cudaMalloc's synchronisation) the library offers a variant whose workspace is a fixed device
array.  This file runs last so that a failure here comes after every other test has run; it also
passes on its own in a fresh process.  Two calls in a row check that the shared workspace carries
nothing from one call to the next.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2511_01927_gb300 import build
    build.build()
    import paper_2511_01927_gb300 as G
    return G


def sym(p, seed):
    rng = np.random.default_rng(seed)
    Qh, _ = np.linalg.qr(rng.standard_normal((p, p)))
    d = np.sort(rng.uniform(-50.0, 50.0, p))
    A = Qh @ np.diag(d) @ Qh.T
    return 0.5 * (A + A.T)


def test_noalloc_matches_regular_entry_twice(G):
    ctx = G.gcie_create(0)
    try:
        stream = torch.cuda.current_stream()
        # calls in a row, different sizes: the whole fixed array (p = 256), a middle size, one element
        for p, seed in ((256, 3), (128, 1), (37, 2), (1, 4)):
            A = sym(p, seed)
            nA = np.linalg.norm(A)
            outs = []
            for which in ("regular", "noalloc"):
                dA = torch.from_numpy(A.copy()).cuda()
                dw = torch.zeros(p, dtype=torch.float64, device="cuda")
                dV = torch.zeros((p, p), dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                if which == "regular":
                    G.gcie_jacobi_eig(ctx, p, dA, dw, dV)
                else:
                    G.gcie_jacobi_eig_noalloc(stream.cuda_stream, p, dA, dw, dV)
                torch.cuda.synchronize()
                outs.append((dw.cpu().numpy(), dV.cpu().numpy()))
            (w0, V0), (w1, V1) = outs
            # same tolerances as the Jacobi parity test: 1e-13 ||A|| on values and eigen-residuals
            assert np.max(np.abs(w1 - w0)) <= 1e-13 * nA
            assert np.max(np.abs(A @ V1 - V1 * w1)) <= 1e-13 * nA
            assert np.max(np.abs(V1.T @ V1 - np.eye(p))) <= 1e-13
            # distinct eigenvalues: vectors agree up to sign
            dots = np.abs(np.einsum("ij,ij->j", V0, V1))
            assert np.min(dots) > 1 - 1e-10
    finally:
        G.gcie_destroy(ctx)


def test_noalloc_rejects_oversize(G):
    dA = torch.zeros((257, 257), dtype=torch.float64, device="cuda")
    dw = torch.zeros(257, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GcieError) as e:
        G.gcie_jacobi_eig_noalloc(None, 257, dA, dw, dA)
    assert e.value.code == 1 and "fixed workspace" in str(e.value)
