"""Benchmark: converged eigenpairs per second of the contour-integral eigensolver on the 2D P1-FEM
pencil of a 500 x 500 grid (n = 249001, log-normal coefficient fields in K and M), eigenvalues
101..400 (300 pairs) with 8 uniform contours x 16 trapezoid nodes, L = 64, 2 moments, FP32 COCG with
FP64 refinement, residual tolerance 1e-10.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
                    [--contours uniform|kde|planned [--pred-noise S]] [--precision mixed|fp64]

One step = one complete solve (ingested pencil resident on the GPU; every step repeats the shifted
solves, moments, basis, Rayleigh-Ritz and merge).  `--contours kde` times the same workload with
contours from Algorithm 2 instead, `--contours planned` with as many contours as the uniform layout
cut in the widest gaps (gcie_plan_contours): the predicted spectrum is the solver's own eigenvalues
of an untimed uniform solve plus seeded Gaussian noise of S mean spacings (a stand-in for a trained
predictor, at its best), the solve runs with the count check on.  `--precision fp64` runs the COCG
recurrences, SpMM and refinement in FP64 (the band factors stay FP32): the in-box FP64 comparator.
The timed steps run without per-launch events; one extra profiled step after them gives the
per-kernel times of the roofline.  The CPU baseline is the oracle's whole solve of a reduced member
(160 x 160) on the host cores.  Prints one JSON line on rank 0.  Under torchrun each rank solves its
own replica of the workload (independent problems, no collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pencils as P  # noqa: E402

METRIC = "converged eigenpairs/s at residual<=1e-10 (uniform contours)"
METRIC_KDE = "converged eigenpairs/s at residual<=1e-10 (KDE contours from a perturbed spectrum)"
METRIC_PLANNED = "converged eigenpairs/s at residual<=1e-10 (gap-planned contours from a perturbed spectrum)"
METRICS = {"uniform": METRIC, "kde": METRIC_KDE, "planned": METRIC_PLANNED}
UNIT = "eigenpairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fem2d-p1-500")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--contours", default="uniform", choices=["uniform", "kde", "planned", "learned"])
    ap.add_argument("--seeds", type=int, default=200,
                    help="with --contours learned: held-out members of the 256 x 256 family to solve")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="shifted solves: FP32 COCG with FP64 refinement (mixed) or FP64 COCG (fp64); both "
                         "with the FP32 band factors as preconditioner")
    ap.add_argument("--lin-tol", type=float, default=1e-11,
                    help="shifted-solve tolerance (scaled residual) of the FEAST iterations after the first")
    ap.add_argument("--lin-tol-first", type=float, default=1e-6,
                    help="looser shifted-solve tolerance of every contour's first FEAST iteration, --lin-tol in the "
                         "later ones (0: --lin-tol throughout); the eigenpair test ||Kx - lambda Mx|| / (||K||_1 ||x||) "
                         "<= 1e-10 applies either way, and a contour whose pairs miss it is iterated again")
    ap.add_argument("--pred-noise", type=float, default=0.1,
                    help="with --contours kde|planned: noise of the predicted spectrum in mean eigenvalue spacings")
    ap.add_argument("--profile-case", type=int, default=0, metavar="NODES",
                    help="run only a small shifted solve (NODES nodes of the first contour, L columns, band "
                         "preconditioner, 4 iterations) for kernel profiling, then exit")
    return ap.parse_args()


def profile_case(args):
    """A reduced launch of the hot kernels for ncu: the shifted solves of a few nodes of the workload
    (same pencil, bandwidth and column count as the full solve, fewer nodes)."""
    import torch
    import paper_2511_01927_gb300 as G

    K, M, spec = P.workload(args.workload)
    V = P.gaussian_block(K.n, spec["L"], 1)
    B = torch.from_numpy(M.to_scipy() @ V).cuda()
    c = spec["lo"] + 0.5 * (spec["hi"] - spec["lo"]) / spec["contours"]
    r = 0.5 * (spec["hi"] - spec["lo"]) / spec["contours"]
    z, _ = G.gcie_trapezoid_nodes(c, r, spec["nodes"])
    z = z[:args.profile_case]
    ctx = G.gcie_create(0, torch.cuda.current_stream().cuda_stream)
    pen = G.gcie_pencil_create(ctx, K, M)
    X = torch.zeros((len(z), K.n, spec["L"]), dtype=torch.complex128, device="cuda")
    it, rc = G.gcie_shifted_solve(ctx, pen, z, spec["L"], B, X, lin_tol=1e-11, max_iters=4, precond=3,
                                  allow_noconv=True)
    torch.cuda.synchronize()
    G.gcie_pencil_destroy(pen)
    G.gcie_destroy(ctx)
    print(json.dumps({"profile_case": args.workload, "nodes": len(z), "iters": it, "rc": rc}))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------- our path
def solver_opts(spec, V, precision="mixed"):
    return dict(nodes=spec["nodes"], moments=spec["moments"], nuniform=spec["contours"], V0=V, tol=1e-10,
                lin_tol=1e-11, expected_count=spec["count"], precision=0 if precision == "mixed" else 1)


def run_ours(args, rank, world):
    import torch
    import paper_2511_01927_gb300 as G

    torch.cuda.set_device(0 if world == 1 else int(os.environ.get("LOCAL_RANK", rank)))
    dev = torch.cuda.current_device()
    K, M, spec = P.workload(args.workload)
    if "count" not in spec:
        raise SystemExit(f"workload {args.workload}: no stored interval (tests/golden)")
    V = P.gaussian_block(K.n, spec["L"], 1)
    stream = torch.cuda.current_stream()
    ctx = G.gcie_create(dev, stream.cuda_stream)
    pen = G.gcie_pencil_create(ctx, K, M)
    opts = solver_opts(spec, V, args.precision)
    opts["lin_tol"] = args.lin_tol
    if args.lin_tol_first > 0:
        opts["lin_tol_first"] = args.lin_tol_first
    kde = None
    if args.contours != "uniform":
        opts, kde = predicted_opts(G, ctx, pen, spec, opts, args.pred_noise, args.contours)

    def step(profile):
        return G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], profile=int(profile), **opts)

    for _ in range(args.warmup):
        step(False)
    fp64 = G.gcie_fp64_rates(ctx)          # FP64 peaks of this GPU (CUDA-core FMA, FP64 MMA), measured
    # timed region: device events on the library's stream (torch's current stream), max over ranks
    G.gcie_reset_stats(ctx)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    count = 0
    last = None
    for _ in range(args.steps):
        last = step(False)
        count += len(last["evals"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = int(G.gcie_get_stats(ctx)["total_launches"])
    # one more step, after the timed region, with every launch timed by CUDA events on the library's
    # stream: the per-kernel-class times of the roofline (the timed steps run without those events)
    G.gcie_reset_stats(ctx)
    step(True)
    stats = G.gcie_get_stats(ctx)
    if world > 1:
        ms, count = reduce_over_ranks(ms, count, "cuda")
    resid_max = float(np.max(last["resid"])) if len(last["resid"]) else None

    # end to end through the public host-buffer call: CSR and V0 from pinned host memory in, the
    # eigenpairs out, every step
    e2e = e2e_measure(G, ctx, K, M, spec, opts, args.steps)
    G.gcie_pencil_destroy(pen)
    G.gcie_destroy(ctx)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return dict(ms=ms, count=count, stats=stats, clocks=clk, last=last, resid_max=resid_max, spec=spec, K=K, e2e=e2e,
                kde=kde, launches=launches, sms=sms, fp64=fp64)


def predicted_opts(G, ctx, pen, spec, opts, noise, kind):
    """Options for a solve on contours from a predicted spectrum: the eigenvalues of one untimed
    uniform solve plus N(0, (noise x mean spacing)^2), seed 7.  kind "kde": Algorithm 2 with the
    paper's parameters (N_min = 10, N_max = 50, w = 10), outer ends moved to the target interval's;
    kind "planned": gcie_plan_contours with the uniform layout's number of contours.  The count
    check is on."""
    ref = G.gcie_solve_pencil(ctx, pen, spec["lo"], spec["hi"], **opts)
    lam = np.sort(ref["evals"])
    spacing = (lam[-1] - lam[0]) / max(len(lam) - 1, 1)
    pred = lam + np.random.default_rng(7).normal(0.0, noise * spacing, lam.size)
    if kind == "kde":
        cts = G.gcie_kde_contours(pred, nmin=10, nmax=50, w=10.0)
        info = {"nmin": 10, "nmax": 50, "w": 10.0}
    else:
        cts = G.gcie_plan_contours(pred, spec["lo"], spec["hi"], spec["contours"])
        info = {"max_contours": spec["contours"]}
    edges = [spec["lo"]] + [c[1] for c in cts[:-1]] + [spec["hi"]]
    contours = [(0.5 * (a + b), 0.5 * (b - a), a, b) for a, b in zip(edges[:-1], edges[1:])]
    o = {k: v for k, v in opts.items() if k != "nuniform"}
    o.update(contours=contours, judge=1)
    info.update(noise_spacings=noise, edges=[float(e) for e in edges], predicted_counts=[int(c[4]) for c in cts])
    return o, info


def source_digest(text):
    """sha256 of a CUDA source with its // comments and blank lines removed, so that edits to
    comments alone do not mark a capture as stale."""
    lines = []
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code.strip():
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def traffic_per_flop():
    """DRAM bytes per algorithmic flop of the band sweeps from the committed ncu summary, or None when
    the kernel source has changed since that capture."""
    rec = {}
    try:
        with open(os.path.join(ROOT, "profiles", "band_solve_traffic.txt")) as fh:
            for line in fh:
                if "=" in line and not line.startswith("#"):
                    k, v = line.strip().split("=", 1)
                    rec[k] = v
        with open(os.path.join(ROOT, rec["source"])) as fh:
            sha = source_digest(fh.read())
    except (OSError, KeyError):
        return None
    return float(rec["dram_bytes_per_flop"]) if sha == rec.get("sha256") else None


def reduce_over_ranks(ms, count, device):
    """Whole-job figures of a replicas run: the slowest rank's time and the eigenpairs of all ranks
    (value = total count / max time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, count], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), int(tsum[1])


def pinned(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t.numpy()


def e2e_measure(G, ctx, K, M, spec, opts, steps):
    import torch

    Kp = P.Csr(K.n, pinned(K.rowptr), pinned(K.col), pinned(K.val))
    Mp = P.Csr(M.n, pinned(M.rowptr), pinned(M.col), pinned(M.val))
    o = dict(opts)
    o["V0"] = pinned(opts["V0"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cnt = 0
    res = None
    for _ in range(steps):
        res = G.gcie_solve(ctx, Kp, Mp, spec["lo"], spec["hi"], **o)
        cnt += len(res["evals"])
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    h2d = sum(a.nbytes for a in (Kp.rowptr, Kp.col, Kp.val, Mp.rowptr, Mp.col, Mp.val, o["V0"]))
    d2h = res["evecs"].nbytes + res["evals"].nbytes + res["resid"].nbytes + res["contour_of"].nbytes
    return {"value": cnt / sec, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


# ----------------------------------------------------------------------------- batched serving
def run_serving(args):
    """64 independent pencils of uneven size (pencils.serving_batch: alternating 2D P1, n 10k-200k, and 3D
    Q1, n 10k-27k, intervals of about 20-200 eigenvalues), solved by one gcie_solve_batch call from host
    CSR buffers (ingest, solve, eigenpairs out): `--steps` timed calls with 4 pencils in flight
    (batch_streams = 4, the library's scheduler), then one call with the pencils one after another
    (batch_streams = 1) on the same inputs; counts must agree pencil by pencil.  4 uniform contours x 16
    nodes, L = 64, 2 moments."""
    import torch
    import paper_2511_01927_gb300 as G

    batch = P.serving_batch(64, 6)
    items = [(K, M, lo, hi) for K, M, lo, hi, _ in batch]
    ctx = G.gcie_create(0)
    opts = dict(nuniform=4, nodes=16, L=64, moments=2, tol=1e-10, lin_tol=args.lin_tol,
                lin_tol_first=args.lin_tol_first)

    def run(streams):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = G.gcie_solve_batch(ctx, items, allow_noconv=True, batch_streams=streams, **opts)
        torch.cuda.synchronize()
        return outs, time.perf_counter() - t0

    for _ in range(max(1, args.warmup)):
        run(4)
    G.gcie_reset_stats(ctx)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    secs, pairs, outs = 0.0, 0, None
    for _ in range(args.steps):
        outs, s = run(4)
        secs += s
        pairs += sum(len(o["evals"]) for o in outs)
    clk = clocks.stop()
    launches = int(G.gcie_get_stats(ctx)["total_launches"])
    seq, s1 = run(1)
    counts = [len(o["evals"]) for o in outs]
    agree = all(len(a["evals"]) == c for a, c in zip(seq, counts))
    worst = max(float(np.max(o["resid"])) for o in outs if len(o["resid"]))
    G.gcie_destroy(ctx)
    value = pairs / secs
    out = {"metric": "converged eigenpairs/s at residual<=1e-10, batched serving", "value": value, "unit": UNIT,
           "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c32+f64", "data": "synthetic",
           "config": {"workload": "serving: 64 pencils, 2D P1 n 10k-200k / 3D Q1 n 10k-27k, 20-200 eigenvalues each",
                      "n_total": int(sum(K.n for K, _, _, _ in items)), "pairs_per_step": int(sum(counts)),
                      "contours": 4, "nodes": 16, "L": 64, "moments": 2, "batch_streams": 4, "lin_tol": args.lin_tol,
                      "lin_tol_first": args.lin_tol_first,
                      "max_resid": worst,
                      "status_not_ok": int(sum(1 for o in outs if o["rc"] != 0))},
           "sequential": {"value": sum(counts) / s1, "seconds": s1, "counts_agree": agree},
           "speedup_over_sequential": value / (sum(counts) / s1),
           "gpu_launches": launches, "clocks": clk,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(sum(K.val.nbytes + K.col.nbytes + K.rowptr.nbytes
                                                                              + M.val.nbytes + M.col.nbytes + M.rowptr.nbytes
                                                                              for K, M, _, _ in items)),
                   "d2h_bytes_per_step": int(sum(o["evecs"].nbytes + o["evals"].nbytes for o in outs))}}
    print(json.dumps(out))


# ----------------------------------------------------------------------------- learned contours
LEARNED_LO, LEARNED_HI = 300.0, 900.0      # target interval of the learned-contour comparison
LEARNED_FIRST = 100000                     # held-out members (training used seeds 0..1999)


def run_learned(args):
    """Learned vs uniform contours on held-out members of the 256 x 256 log-normal family (the density
    predictor's family), target interval [300, 900], 8 contours x 16 nodes, L = 64, 2 moments.  Per member:
      uniform: 8 equal-width contours;
      learned: GPU prediction of the interval's eigenvalue histogram from the coefficient fields, its
               quantiles as the predicted spectrum, 8 contours cut in its gaps (gcie_plan_contours), the
               judged solve (count check on);
      kde:     the same prediction through Algorithm 2 (N_min 10, N_max 50, w 10), judged solve.
    Each arm is timed wall-clock around its calls (prediction and planning included), the stream drained
    on both sides; the ingested pencil and V are shared.  Counts of the arms must agree on every member."""
    import torch
    import paper_2511_01927_gb300 as G

    w = np.load(os.path.join(ROOT, "paper_2511_01927_gb300", "density_net.npz"))["w"]
    ctx = G.gcie_create(0, torch.cuda.current_stream().cuda_stream)
    net = G.gcie_density_net_create(ctx, w)
    lo, hi = LEARNED_LO, LEARNED_HI
    common = dict(nodes=16, L=64, moments=2, tol=1e-10, lin_tol=args.lin_tol, lin_tol_first=args.lin_tol_first)
    # uniform_fp64: the in-box comparator of the learned mixed-precision solve (FP64 COCG recurrences, SpMM and
    # residuals, the same FP32 band factors, tight inner tolerance throughout)
    arms = ("uniform", "learned", "kde", "uniform_fp64")
    tot = {a: 0.0 for a in arms}
    pairs = {a: 0 for a in arms}
    passes = {a: [] for a in arms}
    resplits = {a: 0 for a in arms}
    agree, pred_err, ncont = 0, [], {"learned": [], "kde": []}

    def solve(arm, pen, K, kappa, rho, V):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if arm == "uniform":
            r = G.gcie_solve_pencil(ctx, pen, lo, hi, nuniform=8, V0=V, allow_noconv=True, **common)
            pc = None
        elif arm == "uniform_fp64":
            r = G.gcie_solve_pencil(ctx, pen, lo, hi, nuniform=8, V0=V, allow_noconv=True,
                                    **(common | dict(precision=1, lin_tol=1e-11, lin_tol_first=0.0)))
            pc = None
        else:
            hist = G.gcie_density_predict(ctx, net, kappa[None], rho[None], [[lo, hi]])[0]
            pred = G.gcie_hist_quantiles(hist, lo, hi)
            if arm == "learned":
                cts = G.gcie_plan_contours(pred, lo, hi, 8)
            else:
                cts = G.gcie_kde_contours(pred, nmin=10, nmax=50, w=10.0)
            edges = [lo] + [c[1] for c in cts[:-1]] + [hi]
            contours = [(0.5 * (a + b), 0.5 * (b - a), a, b) for a, b in zip(edges[:-1], edges[1:])]
            r = G.gcie_solve_pencil(ctx, pen, lo, hi, contours=contours, judge=1, V0=V, allow_noconv=True, **common)
            pc = (float(hist.sum()), len(contours))
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0, pc

    members = list(range(LEARNED_FIRST, LEARNED_FIRST + args.seeds))
    # warm-up: every arm once on the first member (not counted)
    K, M, kappa, rho = P.family_member(members[0])
    pen = G.gcie_pencil_create(ctx, K, M)
    for arm in arms:
        solve(arm, pen, K, kappa, rho, P.gaussian_block(K.n, 64, 1))
    G.gcie_pencil_destroy(pen)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for seed in members:
        K, M, kappa, rho = P.family_member(seed)
        pen = G.gcie_pencil_create(ctx, K, M)
        V = P.gaussian_block(K.n, 64, seed)
        counts = {}
        for arm in arms:
            r, sec, pc = solve(arm, pen, K, kappa, rho, V)
            tot[arm] += sec
            pairs[arm] += len(r["evals"])
            counts[arm] = len(r["evals"])
            passes[arm].append(max(r["iters"]))
            resplits[arm] += r["resplits"]
            if pc is not None:
                ncont[arm].append(pc[1])
                if arm == "learned":
                    pred_err.append(abs(pc[0] - len(r["evals"])) / max(1, len(r["evals"])))
        agree += len(set(counts.values())) == 1
        G.gcie_pencil_destroy(pen)
    clk = clocks.stop()
    G.gcie_density_net_destroy(net)
    G.gcie_destroy(ctx)
    val = {a: pairs[a] / tot[a] for a in arms}
    out = {"metric": "converged eigenpairs/s at residual<=1e-10, learned vs uniform contours", "value": val["learned"],
           "unit": UNIT, "n_gpus": 1, "steps": len(members), "warmup": 1, "ms_per_step": 1e3 * tot["learned"] / len(members),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c32+f64", "data": "synthetic",
           "config": {"workload": "fem2d-p1-256 family, held-out members " + f"{members[0]}..{members[-1]}",
                      "n": 65025, "interval": [lo, hi], "contours": 8, "nodes": 16, "L": 64, "moments": 2, "tol": 1e-10,
                      "predictor": "density net (BF16, tcgen05), trained on members 0..1999 solved by this library",
                      "lin_tol": args.lin_tol, "lin_tol_first": args.lin_tol_first},
           "arms": {a: {"value": val[a], "seconds": tot[a], "pairs": pairs[a],
                        "mean_feast_passes": float(np.mean(passes[a])), "resplits": resplits[a]} for a in arms},
           "learned_over_uniform": val["learned"] / val["uniform"], "kde_over_uniform": val["kde"] / val["uniform"],
           "learned_over_uniform_fp64": val["learned"] / val["uniform_fp64"],
           "count_agreement": agree / len(members),
           "predicted_count_rel_error": float(np.mean(pred_err)),
           "kde_contours_mean": float(np.mean(ncont["kde"])), "clocks": clk}
    print(json.dumps(out))


# ----------------------------------------------------------------------------- CPU oracle baseline
REDUCED = "fem2d-p1-160"   # the reduced member of the 500 x 500 workload the oracle solves whole


def oracle_solve(contour_index=None):
    """The oracle's whole CI solve (every step of Algorithm 1 with FEAST, dense steps included) of the
    reduced member of the workload's family: 160 x 160 cells (n = 25281, bandwidth 160), eigenvalues
    11..40, the workload's solver configuration (8 uniform contours x 16 nodes, L = 64, 2 moments), on
    the host cores (contours and nodes on separate threads).  contour_index: only that contour (the
    reference arm's bounded step).  Returns (pairs, seconds, threads, sample description)."""
    import oracle as O

    K, M, spec = P.workload(REDUCED)
    V = P.gaussian_block(K.n, spec["L"], 1)
    cts = O.uniform_contours(spec["lo"], spec["hi"], spec["contours"])
    if contour_index is not None:
        cts = [cts[contour_index % len(cts)]]
    cores = O.host_threads()
    t0 = time.perf_counter()
    r = O.ci_solve(K, M, spec["lo"], spec["hi"], V, contours=cts, nodes=spec["nodes"], moments_m=spec["moments"],
                   tol=1e-10, threads=cores)
    sec = time.perf_counter() - t0
    used = min(cores, len(cts) * spec["nodes"] // 2)
    what = "whole solve" if contour_index is None else f"contour {contour_index % spec['contours']} of 8"
    sample = (f"oracle CI solve ({what}) of the reduced member {REDUCED}: n = {K.n}, bandwidth "
              f"{O.bandwidth(K, M)}, eigenvalues 11..40, 8 uniform contours x 16 nodes, L = 64, 2 moments, banded LU "
              f"per node, dense steps included, {used} host threads; {len(r['evals'])} pairs in {sec:.1f} s")
    return len(r["evals"]), sec, used, sample


def workload_config(args, spec, n):
    """The config keys both arms report: the workload and the solver configuration it is run with."""
    return {"workload": args.workload, "n": int(n), "pairs_per_step": spec["count"], "contours": spec["contours"],
            "nodes": spec["nodes"], "L": spec["L"], "moments": spec["moments"], "tol": 1e-10,
            "l2": "inputs larger than L2 (16 GB block)", "contour_layout": args.contours}


# ----------------------------------------------------------------------------- main
def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    if args.contours == "learned":
        run_learned(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        if rank != 0:
            return
        K, M, spec = P.workload(args.workload)
        # each step: the oracle's solve of one contour of the reduced member (a bounded sample, a few
        # seconds), the contours taken in turn; value = pairs / seconds over the timed steps
        for w in range(args.warmup):
            oracle_solve(w)
        pairs, secs, used = 0, 0.0, 1
        for k in range(args.steps):
            n_k, s_k, used, _ = oracle_solve(k)
            pairs += n_k
            secs += s_k
        value = pairs / secs
        sample = (f"oracle CI solve of one of the 8 contours per step (taken in turn) of the reduced member {REDUCED} "
                  f"(n = 25281, bandwidth 160, eigenvalues 11..40, 16 nodes, L = 64, 2 moments, dense steps "
                  f"included): {pairs} pairs in {secs:.1f} s over {args.steps} steps, {used} host threads")
        out = {"impl": "reference", "metric": METRICS[args.contours], "value": value, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": workload_config(args, spec, K.n),
               "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
               "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    r = run_ours(args, rank, world)
    if rank != 0:
        return
    spec, stats = r["spec"], r["stats"]
    ms_step = r["ms"] / args.steps
    value = r["count"] / (r["ms"] / 1e3)
    metric = METRICS[args.contours]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    # dominant kernel class of the timed region
    classes = {k: v for k, v in stats.items() if isinstance(v, dict)}
    dom = max(classes, key=lambda k: classes[k]["ms"])
    d = classes[dom]
    launches = max(d["launches"], 1)
    sm_mhz = r["clocks"].get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # FP32 CUDA-core peak: SMs (from the device) x 128 FMA lanes x 2 flops x the maximum SM clock
    alu_peak = r["sms"] * 128 * 2 * sm_mhz * 1e6 / 1e12
    if dom in ("prec", "factor"):
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
        bpf = traffic_per_flop() if dom == "prec" else None
        roof = {"kernel_class": dom, "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak,
                "traffic": None if bpf is None else bpf * d["flops"] / launches,
                "per_launch_ms": d["ms"] / launches, "launches": d["launches"],
                "peak_derivation": f"{r['sms']} SMs x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz",
                "timing": "CUDA events per launch in one profiled step after the timed region"}
    else:
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        roof = {"kernel_class": dom, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "per_launch_ms": d["ms"] / launches, "launches": d["launches"],
                "timing": "CUDA events per launch in one profiled step after the timed region"}
    spmm_ms = stats["spmm_dir"]["ms"] + stats["spmm_upd"]["ms"]
    spmm_gbs = (stats["spmm_dir"]["bytes"] + stats["spmm_upd"]["bytes"]) / max(spmm_ms, 1e-9) / 1e6
    out = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c32+f64" if args.precision == "mixed" else "c128 (c64 band factors)",
           "data": "synthetic",
           "config": workload_config(args, spec, r["K"].n) | {
                      "max_resid": r["resid_max"], "outer_iters": r["last"]["outer_iters"],
                      "feast_iters_per_contour": r["last"]["iters"], "cocg_iters": r["last"]["cocg_iters"],
                      "precision": args.precision, "lin_tol": args.lin_tol}
                      | ({"lin_tol_first": args.lin_tol_first} if args.lin_tol_first > 0 else {}),
           "roofline": roof,
           "spmm_hbm": {"achieved": spmm_gbs, "peak": hbm_peak, "frac": spmm_gbs / hbm_peak, "unit": "GB/s",
                        "nameplate_frac": spmm_gbs / 8000.0},
           "kernel_ms": {k: round(v["ms"], 2) for k, v in classes.items()},
           "fp64_peaks_measured": {"fma_tflops": r["fp64"][0], "mma_tflops": r["fp64"][1]},
           "gpu_launches": r["launches"],
           "clocks": r["clocks"], "e2e": r["e2e"]}
    if r["kde"] is not None:
        out["config"]["predicted_contours"] = r["kde"] | {"resplits": r["last"]["resplits"],
                                           "count_estimate": [round(float(x), 2) for x in r["last"]["count_estimate"]]}
    if not args.no_cpu_baseline and world == 1 or (world > 1 and rank == 0 and not args.no_cpu_baseline):
        pairs, sec, used, sample = oracle_solve()
        out["cpu_baseline"] = {"value": pairs / sec, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
