"""Pins of the oracle's density-predictor forward pass and histogram quantiles (CPU), and the host-only
quantile entry point of the C ABI against the oracle.

The forward pass is pinned by a hand-built network whose output is known in closed form: centre taps that
pick channel 0 through the four stride-2 convolutions (so the output at (y, x) is the input pixel
(16 y, 16 x): a wrong padding offset or stride picks another pixel), an fc1 that reads the 4 x 4 features
in (y, x, channel) order and the two bound features, an fc2 that copies them through softplus.
"""
import numpy as np
import pytest

import oracle as O


def test_bf16_round_ties_to_even():
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, -2.5, 3.0e-3], dtype=np.float32)
    r = O.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2.0 ** -6 and r[3] == 1 + 2.0 ** -7 and r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 2.0 ** -8 * 3.0e-3      # half a unit in the last of 7 stored bits


def test_density_input_block_means():
    G = 128
    rng = np.random.default_rng(0)
    a = rng.uniform(-1, 1, (64, 64))
    kappa = np.exp(np.kron(a, np.ones((2, 2))))
    rho = np.exp(2.0 * np.ones((G, G)))
    x = O.density_input(kappa, rho)
    assert x.shape == (64, 64, 2)
    assert np.max(np.abs(x[..., 0] - a)) < 1e-12 and np.max(np.abs(x[..., 1] - 2.0)) < 1e-12


def delta_network():
    """Weights of the hand-built network (ABI order)."""
    parts = []
    for ci, co in O.DENSITY_CONV:
        W = np.zeros((co, 3, 3, ci), np.float32)
        W[0, 1, 1, 0] = 1.0                      # output channel 0 = input channel 0 at pixel (2 oy, 2 ox)
        parts += [W.ravel(), np.zeros(co, np.float32)]
    W1 = np.zeros((O.DENSITY_HID, O.DENSITY_FEAT), np.float32)
    for y in range(4):
        for x in range(4):
            W1[4 * y + x, 64 * (4 * y + x)] = 1.0   # feature (y, x, channel 0)
    W1[20, 1024] = 1.0                          # log lo - 6.5
    W1[21, 1025] = 1.0                          # log hi - 6.5
    W2 = np.zeros((O.DENSITY_BINS, O.DENSITY_HID), np.float32)
    for j in list(range(16)) + [20, 21]:
        W2[j, j] = 1.0
    parts += [W1.ravel(), np.zeros(O.DENSITY_HID, np.float32), W2.ravel(), np.zeros(O.DENSITY_BINS, np.float32)]
    return np.concatenate(parts)


def delta_inputs():
    yy, xx = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
    p = 0.25 + ((yy * 64 + xx) % 7) / 4.0       # exact in BF16
    kappa = np.exp(p)[None]
    rho = np.ones((1, 64, 64))
    bounds = np.array([[np.exp(7.5), np.exp(8.25)]])
    expect = np.full(O.DENSITY_BINS, np.log(2.0))
    sp = lambda v: np.log1p(np.exp(v))
    for y in range(4):
        for x in range(4):
            expect[4 * y + x] = sp(p[16 * y, 16 * x])
    expect[20], expect[21] = sp(1.0), sp(1.75)
    return kappa, rho, bounds, expect


def test_density_forward_hand_network():
    w = delta_network()
    assert w.size == 717520
    kappa, rho, bounds, expect = delta_inputs()
    out = O.density_forward(w, kappa, rho, bounds)
    assert out.shape == (1, 256)
    assert np.max(np.abs(out[0] - expect)) < 1e-6


def test_density_forward_matches_library_convolution():
    """Cross-check with torch's conv2d / linear on random weights (a second, library implementation)."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(3)
    w = (rng.standard_normal(717520) * 0.05).astype(np.float32)
    kappa = np.exp(rng.standard_normal((2, 128, 128)))
    rho = np.exp(rng.standard_normal((2, 128, 128)))
    bounds = np.array([[300.0, 900.0], [50.0, 1000.0]])
    ref = O.density_forward(w, kappa, rho, bounds, bf16=False)
    layers = O.density_unpack(w)
    outs = []
    for b in range(2):
        x = torch.tensor(O.density_input(kappa[b], rho[b]), dtype=torch.float64).permute(2, 0, 1)[None]
        for W, bias in layers[:4]:
            Wt = torch.tensor(W, dtype=torch.float64).permute(0, 3, 1, 2)
            x = F.relu(F.conv2d(x, Wt, torch.tensor(bias, dtype=torch.float64), stride=2, padding=1))
        f = torch.cat([x[0].permute(1, 2, 0).reshape(-1), torch.tensor(np.log(bounds[b]) - 6.5)])
        (W1, b1), (W2, b2) = layers[4], layers[5]
        h = F.relu(torch.tensor(W1, dtype=torch.float64) @ f + torch.tensor(b1, dtype=torch.float64))
        z = torch.tensor(W2, dtype=torch.float64) @ h + torch.tensor(b2, dtype=torch.float64)
        outs.append(F.softplus(z).numpy())
    assert np.max(np.abs(np.array(outs) - ref)) < 1e-5 * max(1.0, np.max(np.abs(ref)))


def test_hist_quantiles_closed_forms():
    # a flat histogram of 4 per bin over [0, 8] with 8 bins: 32 values at (k - 1/2) / 4
    q = O.hist_quantiles(np.full(8, 4.0), 0.0, 8.0)
    assert np.allclose(q, (np.arange(1, 33) - 0.5) / 4.0, rtol=0, atol=1e-12)
    # one occupied bin: values spread evenly inside it; empty bins are skipped
    q = O.hist_quantiles(np.array([0.0, 0.0, 2.0, 0.0]), 10.0, 14.0)
    assert np.allclose(q, [12.25, 12.75])
    # the count is the rounded total
    assert O.hist_quantiles(np.array([0.2, 0.2]), 0.0, 1.0).size == 0
    assert O.hist_quantiles(np.array([0.3, 0.3]), 0.0, 1.0).size == 1


def test_hist_quantiles_abi_matches_oracle():
    from paper_2511_01927_gb300 import build
    build.build()
    import paper_2511_01927_gb300 as G
    rng = np.random.default_rng(11)
    for _ in range(100):
        h = rng.uniform(0, 3, int(rng.integers(1, 300)))
        h[rng.random(h.size) < 0.3] = 0.0
        a, b = O.hist_quantiles(h, 100.0, 900.0), G.gcie_hist_quantiles(h, 100.0, 900.0)
        assert a.size == b.size and np.max(np.abs(a - b), initial=0.0) <= 1e-9
