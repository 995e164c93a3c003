"""The density predictor's GPU inference (im2col kernels + BF16 tensor-core GEMMs, through the C ABI)
against the oracle's NumPy forward pass of the same weights.

  * the hand-built network of tests/test_density_oracle.py: output known in closed form (stride, padding,
    flatten order and bound features), to 1e-5;
  * random weights on random fields (G = 128 and 256, batch 3): the oracle rounds weights and every layer's
    input to BF16 as the GPU path does and sums in FP64, the GPU sums in FP32 on the tensor cores, so an
    intermediate activation can land on the other side of a BF16 rounding boundary: per element
    |gpu - ref| <= 2^-6 max|ref|, and on average within 2^-9 of |ref|;
  * the trained weights (when present) on members of the learned-contour family.
"""
import os

import numpy as np
import pytest

import oracle as O
import pencils as P

from test_density_oracle import delta_inputs, delta_network

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2511_01927_gb300",
                       "density_net.npz")


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


def predict(G, ctx, w, kappa, rho, bounds):
    net = G.gcie_density_net_create(ctx, w)
    try:
        return G.gcie_density_predict(ctx, net, kappa, rho, bounds)
    finally:
        G.gcie_density_net_destroy(net)


def test_density_hand_network(G, ctx):
    kappa, rho, bounds, expect = delta_inputs()
    out = predict(G, ctx, delta_network(), kappa, rho, bounds)
    assert np.max(np.abs(out[0] - expect)) < 1e-5


@pytest.mark.parametrize("grid", [128, 256])
def test_density_random_weights(G, ctx, grid):
    rng = np.random.default_rng(grid)
    w = (rng.standard_normal(717520) * 0.08).astype(np.float32)
    kappa = np.exp(rng.standard_normal((3, grid, grid)))
    rho = np.exp(rng.standard_normal((3, grid, grid)))
    bounds = np.array([[300.0, 900.0], [50.0, 1000.0], [120.0, 250.0]])
    out = predict(G, ctx, w, kappa, rho, bounds)
    ref = O.density_forward(w, kappa, rho, bounds)
    err = np.abs(out - ref)
    assert np.max(err) <= 2.0 ** -6 * np.max(np.abs(ref))
    assert np.mean(err) <= 2.0 ** -9 * np.mean(np.abs(ref))


def test_density_rejects_bad_grid(G, ctx):
    net = G.gcie_density_net_create(ctx, delta_network())
    try:
        with pytest.raises(G.GcieError) as e:
            G.gcie_density_predict(ctx, net, np.ones((1, 96, 96)), np.ones((1, 96, 96)), [[1.0, 2.0]])
        assert e.value.code == 1
    finally:
        G.gcie_density_net_destroy(net)


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained weights")
def test_density_trained_weights_on_family(G, ctx):
    w = np.load(WEIGHTS)["w"]
    kap, rh = [], []
    for seed in (100000, 100001):
        _, _, k, r = P.family_member(seed)
        kap.append(k)
        rh.append(r)
    bounds = np.array([[300.0, 900.0], [300.0, 900.0]])
    out = predict(G, ctx, w, np.array(kap), np.array(rh), bounds)
    ref = O.density_forward(w, np.array(kap), np.array(rh), bounds)
    assert np.max(np.abs(out - ref)) <= 2.0 ** -6 * np.max(np.abs(ref))
    assert np.all(out >= 0.0)
