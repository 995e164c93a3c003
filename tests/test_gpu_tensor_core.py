"""The tensor-core (tcgen05) products through the C ABI against FP64 products of the same inputs.

Bounds, per element, with S = sum_k |A_ik| |B_jk|:
  * split TF32 (gcie_gemm_tf32x3): |D - A B^T| <= 2^-19 S  (the dropped tail x tail term and the TF32
    rounding of the tails are 2^-22 S each, FP32 accumulation over K adds K-dependent 2^-24 terms);
  * BF16 operands (gcie_gemm_bf16): the reference is the FP64 product of the BF16-rounded operands, so
    only FP32 accumulation differs: |D - ref| <= 2^-20 S.
Shapes cover ragged tiles in M, N and K (not multiples of 128, 64 and the 128-byte K block).
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


@pytest.fixture(scope="module")
def ctx(G):
    h = G.gcie_create(0)
    yield h
    G.gcie_destroy(h)


@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (300, 200, 100), (1, 17, 5), (517, 64, 500)])
def test_gemm_tf32x3_fp32_faithful(G, ctx, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = (rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, (N, 1)))).astype(np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dD = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    G.gcie_gemm_tf32x3(ctx, M, N, K, dA, K, dB, K, dD, N)
    D = dD.cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    S = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    assert np.all(np.abs(D - ref) <= 2.0 ** -19 * S + 1e-30)
    # and plainly better than a single TF32 product would be on these inputs
    assert np.max(np.abs(D - ref) / (S + 1e-30)) < 2.0 ** -16


def _bf16(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t, t.to(torch.float32).numpy().astype(np.float64)


@pytest.mark.parametrize("M,N,K,relu", [(256, 128, 64, 0), (4096, 32, 18, 1), (130, 70, 300, 1)])
def test_gemm_bf16_bias_relu(G, ctx, M, N, K, relu):
    rng = np.random.default_rng(7 * M + K)
    tA, A = _bf16(rng.standard_normal((M, K)))
    tB, B = _bf16(rng.standard_normal((N, K)) / np.sqrt(K))
    bias = rng.standard_normal(N).astype(np.float32)
    dD = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    dbias = torch.from_numpy(bias).cuda()
    G.gcie_gemm_bf16(ctx, M, N, K, tA.cuda(), K, tB.cuda(), K, dbias, relu, dD, N)
    D = dD.cpu().numpy().astype(np.float64)
    ref = A @ B.T + bias
    if relu:
        ref = np.maximum(ref, 0.0)
    S = np.abs(A) @ np.abs(B).T + np.abs(bias)
    assert np.all(np.abs(D - ref) <= 2.0 ** -20 * S + 1e-30)


def test_gemm_rejects_bad_leading_dimension(G, ctx):
    d = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(G.GcieError) as e:
        G.gcie_gemm_tf32x3(ctx, 8, 8, 8, d, 4, d, 8, d, 8)
    assert e.value.code == 1


def test_fp64_rate_probe(G, ctx):
    """The FP64 probe returns positive rates below the nominal FP64 ceiling of the part (a few TFLOP/s)."""
    fma, mma = G.gcie_fp64_rates(ctx)
    assert 0.05 < fma < 100.0 and 0.05 < mma < 100.0
