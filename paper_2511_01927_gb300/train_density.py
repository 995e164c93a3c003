"""Train the density predictor of the learned-contour path on pencils this library solves.

    python -m paper_2511_01927_gb300.train_density data  --members 2000 --out DIR   # solve the training family
    python -m paper_2511_01927_gb300.train_density train --data DIR --out WEIGHTS.npz [--epochs 60]

Family: `pencils.family_member(seed)`, the 2D log-normal P1 pencil on 256 x 256 cells (n = 65025).  For
every member the solver (8 uniform contours x 16 nodes, L = 64, 2 moments, the count check on) returns
the eigenvalues in [L0, L1] = [50, 1000]; the network input is the 64 x 64 block mean of log(kappa) and
log(rho).  Training samples random sub-intervals [lo, hi] of [L0, L1] (width at least a fifth of it) per
member and epoch; the target is the 256-bin histogram of the member's eigenvalues over [lo, hi], the loss
the Poisson negative log-likelihood of the predicted counts (softplus output).  The weights are written in
the C ABI's order (gcie.h, GCIE_DENSITY_NWEIGHTS float32 values) for gcie_density_net_create.  This is the
paper's recipe (Section 4.1: a predictor trained on spectra of the same operator family computed by a
solver) with a small convolutional network in place of its neural operator; PyTorch serves only here,
for training.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import pencils as P  # noqa: E402

L0, L1 = 50.0, 1000.0
CONV = ((2, 16), (16, 32), (32, 64), (64, 64))
FEAT, HID, BINS = 64 * 4 * 4 + 2, 512, 256


def net_input(kappa, rho):
    """64 x 64 x 2 block means of log(kappa), log(rho) (the input the GPU kernel forms)."""
    s = kappa.shape[0] // 64
    lk = np.log(kappa).reshape(64, s, 64, s).mean(axis=(1, 3))
    lr = np.log(rho).reshape(64, s, 64, s).mean(axis=(1, 3))
    return np.stack([lk, lr], axis=-1).astype(np.float32)


def make_data(members: int, first: int, out: str):
    import paper_2511_01927_gb300 as G

    os.makedirs(out, exist_ok=True)
    ctx = G.gcie_create(0)
    xs, evs, info = [], [], []
    t0 = time.time()

    def member(seed):
        K, M, kappa, rho = P.family_member(seed)
        return seed, K, M, net_input(kappa, rho)

    with cf.ThreadPoolExecutor(4) as ex:
        for seed, K, M, x in ex.map(member, range(first, first + members)):
            r = G.gcie_solve(ctx, K, M, L0, L1, nuniform=8, nodes=16, L=64, moments=2, judge=1, allow_noconv=True,
                             V0=P.gaussian_block(K.n, 64, seed + 1))
            xs.append(x.astype(np.float16))
            evs.append(np.asarray(r["evals"]))
            info.append((seed, int(r["rc"]), len(r["evals"]), int(r["resplits"])))
            if len(xs) % 100 == 0:
                print(f"{len(xs)} members, {time.time() - t0:.0f} s", flush=True)
    G.gcie_destroy(ctx)
    lens = np.array([e.size for e in evs])
    np.savez_compressed(os.path.join(out, f"family_{first}_{members}.npz"), x=np.array(xs), lens=lens,
                        evals=np.concatenate(evs), info=np.array(info))
    print(json.dumps({"members": members, "first": first, "seconds": time.time() - t0,
                      "count_min": int(lens.min()), "count_max": int(lens.max()),
                      "noconv": int(sum(1 for i in info if i[1] != 0))}))


def build_model(torch):
    nn = torch.nn

    class DensityNet(nn.Module):
        def __init__(self):
            super().__init__()
            self.convs = nn.ModuleList([nn.Conv2d(ci, co, 3, stride=2, padding=1) for ci, co in CONV])
            self.fc1 = nn.Linear(FEAT, HID)
            self.fc2 = nn.Linear(HID, BINS)

        def forward(self, x, u):              # x: B x 2 x 64 x 64 (NCHW), u: B x 2
            for cv in self.convs:
                x = torch.relu(cv(x))
            f = torch.cat([x.permute(0, 2, 3, 1).reshape(x.shape[0], -1), u], dim=1)   # (y, x, channel)
            return nn.functional.softplus(self.fc2(torch.relu(self.fc1(f))))

    return DensityNet()


def export(model) -> np.ndarray:
    """Weights in the C ABI's order: W[Cout][3][3][Cin], b per convolution; W1, b1; W2, b2."""
    parts = []
    for cv in model.convs:
        parts += [cv.weight.detach().permute(0, 2, 3, 1).cpu().numpy().ravel(), cv.bias.detach().cpu().numpy()]
    for fc in (model.fc1, model.fc2):
        parts += [fc.weight.detach().cpu().numpy().ravel(), fc.bias.detach().cpu().numpy()]
    return np.concatenate(parts).astype(np.float32)


def load_family(paths):
    xs, evs = [], []
    for p in paths:
        d = np.load(p)
        offs = np.concatenate([[0], np.cumsum(d["lens"])])
        xs.append(d["x"].astype(np.float32))
        evs += [d["evals"][offs[i]:offs[i + 1]] for i in range(d["lens"].size)]
    return np.concatenate(xs), evs


def histograms(evs, lo, hi):
    h = np.zeros((lo.size, BINS), np.float32)
    for i, e in enumerate(evs):
        sel = e[(e >= lo[i]) & (e <= hi[i])]
        h[i] = np.histogram(sel, bins=BINS, range=(lo[i], hi[i]))[0]
    return h


def random_intervals(rng, m):
    """m intervals [lo, hi] inside [L0, L1], at least a fifth of it wide."""
    lo = rng.uniform(L0, L0 + 0.7 * (L1 - L0), m)
    hi = lo + rng.uniform(0.2 * (L1 - L0), L1 - lo)
    return lo, hi


def train(data_dir: str, out: str, epochs: int, seed: int = 0):
    import torch

    paths = sorted(os.path.join(data_dir, f) for f in os.listdir(data_dir) if f.startswith("family_"))
    x, evs = load_family(paths)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    torch.manual_seed(seed)
    model = build_model(torch).to(dev)
    opt = torch.optim.Adam(model.parameters(), lr=1e-3)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, epochs)
    xt = torch.tensor(x, device=dev).permute(0, 3, 1, 2).contiguous()
    nval = max(1, x.shape[0] // 20)
    tr_idx, va_idx = np.arange(nval, x.shape[0]), np.arange(nval)
    rng = np.random.default_rng(seed)
    vlo, vhi = random_intervals(np.random.default_rng(99), nval)
    vh = torch.tensor(histograms([evs[i] for i in va_idx], vlo, vhi), device=dev)
    vu = torch.tensor(np.stack([np.log(vlo) - 6.5, np.log(vhi) - 6.5], 1), dtype=torch.float32, device=dev)
    t0 = time.time()
    for ep in range(epochs):
        model.train()
        for rep in range(4):                               # four random intervals per member and epoch
            perm = rng.permutation(tr_idx)
            lo, hi = random_intervals(rng, perm.size)
            ht = torch.tensor(histograms([evs[i] for i in perm], lo, hi), device=dev)
            ut = torch.tensor(np.stack([np.log(lo) - 6.5, np.log(hi) - 6.5], 1), dtype=torch.float32, device=dev)
            for b0 in range(0, perm.size, 64):
                sl = slice(b0, b0 + 64)
                pred = model(xt[perm[sl]], ut[sl])
                loss = torch.nn.functional.poisson_nll_loss(pred, ht[sl], log_input=False, full=False).mean()
                opt.zero_grad()
                loss.backward()
                opt.step()
        sched.step()
        model.eval()
        with torch.no_grad():
            pv = model(xt[va_idx], vu)
            cnt_err = (pv.sum(1) - vh.sum(1)).abs() / vh.sum(1).clamp(min=1)
            vloss = torch.nn.functional.poisson_nll_loss(pv, vh, log_input=False).item()
        print(f"epoch {ep + 1}: val poisson {vloss:.4f}, count error {cnt_err.mean().item():.4f}, {time.time() - t0:.0f} s",
              flush=True)
    w = export(model.cpu())
    np.savez(out, w=w, l0=L0, l1=L1, members=x.shape[0], val_count_error=float(cnt_err.mean()), epochs=epochs)
    print(json.dumps({"weights": out, "n": int(w.size), "val_count_error": float(cnt_err.mean())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["data", "train"])
    ap.add_argument("--members", type=int, default=2000)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--out", required=True)
    ap.add_argument("--data")
    ap.add_argument("--epochs", type=int, default=60)
    a = ap.parse_args()
    if a.what == "data":
        make_data(a.members, a.first, a.out)
    else:
        train(a.data, a.out, a.epochs)


if __name__ == "__main__":
    main()
