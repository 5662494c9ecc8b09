#!/usr/bin/env python
"""Benchmark of k-NN graph construction (Wang et al., arXiv:1307.7852) on GB300.

One step = one whole graph build (T random divisions, leaf graphs, merge, R
propagation rounds) over a synthetic point set resident in HBM.  Default
workload: 1,000,000 SIFT-like points (d = 128, integer values 0..255 from a
1,024-centre Gaussian mixture), k = 20, T = 8, leaf size 256, 2 rounds.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is whole-job points/s (n x ranks / max-over-
ranks seconds per step), measured with CUDA events on the build's stream;
``e2e`` is the same metric through the host-buffer C ABI call with the
host<->device copies inside the timed region.  Under torchrun every rank builds
an independent replica (the method is not sharded: "replicas only").
``--impl reference`` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: generator args and method parameters
    "sift1m": dict(gen="sift_like", n=1_000_000, d=128, centers=1024, k=20, T=8, g=256, R=2,
                   desc="1M x 128 SIFT-like integer mixture (1,024 centres, std 20), k=20, T=8, g=256, R=2"),
    "sift400k": dict(gen="sift_like", n=400_000, d=128, centers=410, k=20, T=8, g=256, R=2,
                     desc="400k x 128 SIFT-like integer mixture (410 centres), k=20, T=8, g=256, R=2 (profiling size)"),
    "sift10k": dict(gen="sift_like", n=10_000, d=128, centers=64, k=10, T=4, g=64, R=1,
                    desc="10k x 128 SIFT-like integer mixture (64 centres), k=10, T=4, g=64, R=1"),
    "gist1m": dict(gen="gist_like", n=1_000_000, d=960, centers=256, k=10, T=8, g=512, R=1,
                   desc="1M x 960 GIST-like normalised mixture (256 centres), k=10, T=8, g=512, R=1"),
}
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2}
PROPAGATION = {"first_order": 0, "best_first": 1, "pairwise": 2}
# Small cases of the workloads for DRAM-traffic captures (ncu): the same
# method parameters and data law, fewer points (inputs still larger than L2).
PROFILE_CASE = {"sift1m": dict(n=400_000, centers=410), "gist1m": dict(n=60_000, centers=256),
                "sift400k": dict(n=400_000, centers=410)}
# kernels whose DRAM bytes are recorded, and the unit each is scaled by
TRAFFIC_KERNELS = {"propagate_kernel": "point-round", "leaf_tc_kernel": "point-tree",
                   "leaf_rescore_staged_kernel": "point-tree", "gather_quant_kernel": "point-tree",
                   "merge_kernel": "point", "project_bytes_tma_kernel": "point-tree-level",
                   "project_kernel": "point-level"}
METRIC = "points/sec to build the k-NN graph (recall@k reported on a 10k-point sample)"


def make_data(w, seed):
    from paper_1307_7852_gb300 import synthetic
    if w["gen"] == "sift_like":
        return synthetic.sift_like(w["n"], w["d"], centers=w["centers"], seed=seed)
    if w["gen"] == "gist_like":
        return synthetic.gist_like(w["n"], w["d"], centers=w["centers"], seed=seed)
    raise ValueError(w["gen"])


# ------------------------------------------------------------ multi-rank
def aggregate(elapsed_s: float, points_per_rank: int, world: int, dist=None, device=None):
    """Max over ranks of the timed seconds, and whole-job points/s
    (world x points_per_rank / that time).  Every rank returns the same."""
    el = float(elapsed_s)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([el], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    return el, points_per_rank * world / el


# ------------------------------------------------------------ DRAM traffic
def source_hash() -> str:
    """Hash of the CUDA sources: a recorded traffic figure holds only for the
    kernels it was measured on."""
    import glob
    import hashlib
    hh = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1307_7852_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                    glob.glob(os.path.join(csrc, "*.h"))):
        with open(f, "rb") as fh:
            hh.update(os.path.basename(f).encode())
            hh.update(fh.read())
    return hh.hexdigest()[:16]


def traffic_path(workload, precision):
    return os.path.join(ROOT, "profiles", f"dram_traffic_{workload}_{precision}.json")


def load_traffic(workload, precision):
    """Per-unit DRAM bytes of the kernels, from a capture of the current
    sources (None when the sources changed since or nothing was captured)."""
    try:
        with open(traffic_path(workload, precision)) as f:
            rec = json.load(f)
    except Exception:
        return None
    return rec if rec.get("source_hash") == source_hash() else None


def traffic_from_csv(args, w):
    """Writes the per-unit DRAM bytes of an ncu launch list (--metrics
    dram__bytes_read.sum,dram__bytes_write.sum, --csv) of `bench.py
    --profile-case` to profiles/dram_traffic_<workload>_<precision>.json."""
    import csv
    case = dict(n=w["n"], centers=w["centers"]) if args.traffic_full else PROFILE_CASE[args.workload]
    n, T, R = case["n"], w["T"], w["R"]
    # launches in order; a build starts with init_perm_kernel, and only the
    # last build's launches count (a full-size run also holds its warm-up)
    launches = {}
    order = []
    with open(args.traffic_from) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        name = row.get("Kernel Name", "")
        base = name.split("(")[0].split("<")[0].split("::")[-1].strip().split()[-1] if name.strip() else ""
        key = row["ID"]
        if key not in launches:
            launches[key] = {"kernel": base, "bytes": 0.0}
            order.append(key)
        unit = row.get("Metric Unit", "byte").lower()
        scale = {"byte": 1, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9}.get(unit, 1)
        if row["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            launches[key]["bytes"] += float(row["Metric Value"].replace(",", "")) * scale
    starts = [i for i, key in enumerate(order) if launches[key]["kernel"] == "init_perm_kernel"]
    if starts:
        order = order[starts[-1]:]
    order = [key for key in order if launches[key]["kernel"] in TRAFFIC_KERNELS]
    per = {}
    for key in order:
        per.setdefault(launches[key]["kernel"], []).append(launches[key]["bytes"])
    out = {}
    for kname, vals in per.items():
        unit = TRAFFIC_KERNELS[kname]
        if unit == "point-round":
            out[kname] = {"unit": unit, "bytes_per_unit": [v / n for v in vals]}
        elif unit == "point-tree":
            out[kname] = {"unit": unit, "bytes_per_unit": sum(vals) / (n * T)}
        elif unit == "point":
            out[kname] = {"unit": unit, "bytes_per_unit": sum(vals) / n}
        else:
            out[kname] = {"unit": "point-build", "bytes_per_unit": sum(vals) / n}
    if not args.traffic_hash:
        raise SystemExit("--traffic-from needs --traffic-hash: the source_hash the profiled run printed")
    rec = {"workload": args.workload, "precision": args.precision, "source_hash": args.traffic_hash,
           "case": {"n": n, **{k_: w[k_] for k_ in ("d", "k", "T", "g", "R")}, "centers": case["centers"]},
           "command": args.traffic_command or "", "per_unit": out}
    if args.traffic_full:
        # a full-size capture of some kernels (-k) refines the record of the
        # profiling case for those kernels
        try:
            with open(traffic_path(args.workload, args.precision)) as f:
                old = json.load(f)
        except Exception:
            old = None
        if old and old.get("source_hash") == args.traffic_hash:
            for kname in out:
                old["per_unit"][kname] = dict(out[kname], n=n, command=args.traffic_command or "")
            old.setdefault("full_size", [])
            old["full_size"] = sorted(set(old["full_size"]) | set(out))
            rec = old
    with open(traffic_path(args.workload, args.precision), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))
    return 0


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            P = json.load(f)
        return float(P["hbm_gbs"]), float(P["bf16_tflops"]), float(P.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 2070.0, "fallback"


def unique_candidates(ids: np.ndarray, sample: np.ndarray) -> float:
    """Mean number of candidates a first-order round scores per point: the
    distinct ids of the neighbours' lists that are not p and not already in
    p's list."""
    tot = 0
    for p in sample:
        own = ids[p]
        own = own[own >= 0]
        c = ids[own].ravel()
        c = c[(c >= 0) & (c != p)]
        c = np.setdiff1d(np.unique(c), own, assume_unique=False)
        tot += c.size
    return tot / max(1, len(sample))


def distance_errors(X, q, gi, gd, precision, cosine):
    """Relative errors of the graph's FP32 distances on a sample of rows
    against FP64 distances of the same pairs (plain NumPy), and, for the
    reduced-precision paths, of the candidate distance between the quantised
    rows (BF16 round to nearest even; E4M3 with a per-row scale max|x|/448)
    -- the error the FP32 rescoring removes."""
    Xf = np.asarray(X, dtype=np.float64)
    if cosine:
        nrm = np.linalg.norm(Xf, axis=1, keepdims=True)
        Xf = Xf / np.where(nrm > 0, nrm, 1.0)
    a = np.repeat(q, gi.shape[1])
    b = gi.ravel()
    ok = b >= 0
    a, b, g = a[ok], b[ok], gd.ravel()[ok].astype(np.float64)
    exact = np.empty(len(a))
    for s0 in range(0, len(a), 65536):
        dd = Xf[a[s0:s0 + 65536]] - Xf[b[s0:s0 + 65536]]
        exact[s0:s0 + 65536] = np.einsum("ij,ij->i", dd, dd)
    if cosine:
        exact *= 0.5
    pos = exact > 0
    rel = np.abs(g[pos] - exact[pos]) / exact[pos]

    def summary(r):
        return {"max": float(r.max()) if len(r) else 0.0, "p50": float(np.percentile(r, 50)) if len(r) else 0.0,
                "p99": float(np.percentile(r, 99)) if len(r) else 0.0,
                "p99.9": float(np.percentile(r, 99.9)) if len(r) else 0.0,
                "hist_log10": {str(e): int(np.sum((r >= 10.0 ** e) & (r < 10.0 ** (e + 1)))) for e in range(-9, 0)},
                "zero": int(np.sum(r == 0))}
    out = {"pairs": int(len(a)), "graph_fp32": summary(rel), "reference": "FP64 squared distance of the same pairs"}
    if precision != "fp32" and not cosine:
        import torch
        sel = np.nonzero(pos)[0][:200000]
        rows = np.unique(np.concatenate([a[sel], b[sel]]))
        Xt = torch.from_numpy(np.asarray(X, dtype=np.float32)[rows])
        if precision == "bf16":
            Q = Xt.to(torch.bfloat16).to(torch.float64).numpy()
        else:
            sc = Xt.abs().amax(dim=1, keepdim=True) / 448.0
            sc = torch.where(sc > 0, sc, torch.ones_like(sc))
            Q = ((Xt / sc).to(torch.float8_e4m3fn).to(torch.float64) * sc.to(torch.float64)).numpy()
        pos_of = {int(r): i for i, r in enumerate(rows)}
        ia = np.array([pos_of[int(v)] for v in a[sel]])
        ib = np.array([pos_of[int(v)] for v in b[sel]])
        dq = np.einsum("ij,ij->i", Q[ia] - Q[ib], Q[ia] - Q[ib])
        out[f"candidate_{precision}"] = summary(np.abs(dq - exact[sel]) / exact[sel])
    return out


# ---------------------------------------------------------- batched sets
def run_batched(args):
    """256 independent Gaussian-mixture sets (n log-uniform in [2k, 200k], d in
    {64, 128, 256}, 16-256 centres), k=10, T=6, leaf size 128, 1 round: one
    recorded graph launch for all sets vs one knng_build per set."""
    import torch
    import paper_1307_7852_gb300 as knng
    from paper_1307_7852_gb300 import synthetic
    sets = synthetic.batched_sets(args.batch_sets, seed=args.data_seed)
    dev = torch.device("cuda", 0)
    Xs = [torch.from_numpy(X).to(dev) for X in sets]
    ntot = sum(X.shape[0] for X in sets)
    k, T, g, R = 10, 6, 128, 1
    prec = PRECISIONS[args.precision]
    h = knng.Handle(0)
    outs = [(torch.empty((X.shape[0], k), dtype=torch.int32, device=dev),
             torch.empty((X.shape[0], k), dtype=torch.float32, device=dev)) for X in Xs]
    stream = torch.cuda.current_stream(dev)
    # tile shapes of the tensor-core leaf kernel from the autotuner, one per
    # dimension (tuned on the largest set of that dimension)
    tiles = {}
    if prec != 0:
        for dd in sorted(set(int(X.shape[1]) for X in Xs)):
            big = max((X for X in Xs if X.shape[1] == dd), key=lambda X: X.shape[0])
            tiles[dd] = knng.knng_autotune(big, k, T, g, args.seed, precision=prec, h=h)

    def batched():
        knng.knng_build_batched(Xs, k, T, g, R, args.seed, prec, 2, outs=outs, h=h)

    def separate():
        for X, (oi, od) in zip(Xs, outs):
            knng.knng_build(X, k, T, g, R, args.seed, prec, 2, ids=oi, dists=od, h=h)

    res = {}
    legs = (("batched", batched),) if args.no_separate else (("separate", separate), ("batched", batched))
    for name, fn in legs:
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        l0 = knng.knng_launch_counter()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            t0.record(stream)
            for _ in range(args.steps):
                fn()
            t1.record(stream)
            torch.cuda.synchronize()
        res[name] = {"ms_per_step": t0.elapsed_time(t1) / args.steps,
                     "launches_per_step": (knng.knng_launch_counter() - l0) / args.steps,
                     "clocks": clk.summary()}
    sec = res["batched"]["ms_per_step"] / 1e3
    line = {
        "metric": "points/sec to build the k-NN graphs of 256 independent sets", "value": ntot / sec,
        "unit": "points/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16+f32", "fp8": "e4m3+f32"}[args.precision], "data": "synthetic",
        "config": {"workload": "batched256", "sets": len(sets), "points": ntot,
                   "dims": sorted(set(int(X.shape[1]) for X in sets)), "k": k, "T": T, "leaf_size": g,
                   "rounds": R, "precision": args.precision},
        "gpu_launches": int(res["batched"]["launches_per_step"] * args.steps),
        "separate": None if args.no_separate else {
            "value": ntot / (res["separate"]["ms_per_step"] / 1e3), "ms_per_step": res["separate"]["ms_per_step"],
            "launches_per_step": res["separate"]["launches_per_step"]},
        "speedup_vs_separate": None if args.no_separate else
        res["separate"]["ms_per_step"] / res["batched"]["ms_per_step"],
        "autotuned_tiles": {str(dd): {"stages": t[0], "rows_per_group": t[1], "leaf_ms": t[2]}
                            for dd, t in tiles.items()},
        "clocks": res["batched"]["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- learned splits
def run_learned(args):
    """10M x 96 FP16 points (4,096-centre normalised mixture, std 0.05), k=20,
    leaf size 256, 1 round.  The split-feature network (96 -> 256 -> 16) is
    trained on the k-NN graph the method builds for a 1M-point subsample;
    then learned splits with T=4 are timed against random directions with T=8
    (and T=4), recall against exact brute force on a sample."""
    import torch
    import paper_1307_7852_gb300 as knng
    from paper_1307_7852_gb300 import synthetic
    n = args.learned_n
    X = synthetic.sphere_f16(n, 96, centers=4096, std=0.05, seed=args.data_seed)
    dev = torch.device("cuda", 0)
    Xd = torch.from_numpy(X).to(dev)
    k, g, R = 20, 256, 1
    prec = PRECISIONS[args.precision]
    h = knng.Handle(0)
    stream = torch.cuda.current_stream(dev)
    # training graph: random directions, T=8, on a 1M subsample
    nsub = min(n, 1_000_000)
    sub = Xd[:nsub]
    t0 = time.perf_counter()
    gi, _ = knng.knng_build(sub, k, 8, g, 1, args.seed + 7, prec, 2, h=h)
    net = knng.Mlp(96, 256, 16, seed=args.seed)
    loss0 = net.train(sub, gi, 1, batch_edges=4096, lr=2e-3, seed=1)
    loss = net.train(sub, gi, args.train_steps, batch_edges=4096, lr=2e-3, seed=2)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    ids = torch.empty((n, k), dtype=torch.int32, device=dev)
    dists = torch.empty((n, k), dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            a.record(stream)
            for _ in range(args.steps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps, clk.summary()

    q = synthetic.sample_ids(n, args.recall_sample, args.seed + 1)
    qd = torch.from_numpy(q).to(dev)
    ei, _ = knng.knng_exact_knn(Xd, qd, k, h=h)
    e_ids = ei.cpu().numpy()

    def recall():
        got = ids[qd.long()].cpu().numpy()
        return float(np.mean([len(set(got[r]) & set(e_ids[r])) / k for r in range(len(q))]))

    res = {}
    l0 = knng.knng_launch_counter()
    # headline: per-level learned features (random directions where a
    # feature is flat in the node), T=4
    ms, clk = timed(lambda: knng.knng_build_learned(net, Xd, k, 4, g, R, args.seed, prec, 2, ids=ids, dists=dists,
                                                    h=h, partitioner=knng.PART_FEATURES))
    launches = (knng.knng_launch_counter() - l0) // (args.steps + args.warmup)
    res["learned_T4"] = {"ms_per_step": ms, "recall": recall(), "splits": "per-level learned features"}
    for name, part in (("learned_features_pca_T4", knng.PART_FEATURES_PCA),
                       ("learned_embedding_random_T4", knng.PART_RANDOM), ("learned_embedding_pca_T4", knng.PART_PCA)):
        ms_l, _ = timed(lambda: knng.knng_build_learned(net, Xd, k, 4, g, R, args.seed, prec, 2, ids=ids,
                                                        dists=dists, h=h, partitioner=part))
        res[name] = {"ms_per_step": ms_l, "recall": recall()}
    for T in (8, 6, 5, 4):
        ms_r, _ = timed(lambda: knng.knng_build(Xd, k, T, g, R, args.seed, prec, 2, ids=ids, dists=dists, h=h))
        res[f"random_T{T}"] = {"ms_per_step": ms_r, "recall": recall()}
    ms_p, _ = timed(lambda: knng.knng_build(Xd, k, 4, g, R, args.seed, prec, 2, ids=ids, dists=dists, h=h,
                                            partitioner=knng.PART_PCA))
    res["pca_T4"] = {"ms_per_step": ms_p, "recall": recall()}
    for v in res.values():
        v["points_per_s"] = n / (v["ms_per_step"] / 1e3)
    line = {
        "metric": "points/sec to build the k-NN graph with learned splits (T=4) vs random (T=8)",
        "value": res["learned_T4"]["points_per_s"], "unit": "points/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["learned_T4"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16+f32", "fp8": "e4m3+f32"}[args.precision], "data": "synthetic",
        "config": {"workload": "learned10m", "n": n, "d": 96, "input": "f16", "k": k, "leaf_size": g, "rounds": R,
                   "precision": args.precision, "network": "96-256-16 GELU, FP32 weights, BF16 inference",
                   "train": {"subsample": nsub, "graph": "random T=8 R=1", "steps": args.train_steps,
                             "batch_edges": 4096, "loss_first": loss0, "loss_last": loss, "seconds": train_s}},
        "gpu_launches": int(launches * args.steps),
        "results": res, "recall_sample": int(len(q)), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ reference arm
def run_reference(args, w, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    X = make_data(w, seed=args.data_seed)
    ns = args.ref_sample
    Xs = np.ascontiguousarray(X[:ns])
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.build_graph(Xs, w["k"], w["T"], w["g"], w["R"], args.seed)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    sec = statistics.mean(times)
    val = ns / sec
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_points": ns, **{k: w[k] for k in ("d", "k", "T", "g", "R")}},
        "cpu_baseline": {"value": val, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {ns} points of the {args.workload} workload, whole method"},
        "e2e": {"value": val, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- ours
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched256", "learned10m"], default="sift1m")
    ap.add_argument("--learned-n", type=int, default=10_000_000)
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--batch-sets", type=int, default=256)
    ap.add_argument("--no-separate", action="store_true", help="batched256: time the batched launch only")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="bf16")
    ap.add_argument("--seed", type=int, default=12345)
    ap.add_argument("--data-seed", type=int, default=2013)
    ap.add_argument("--recall-sample", type=int, default=10000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=300000)
    ap.add_argument("--ref-sample", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-recall", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="timed builds only (for profiler runs)")
    ap.add_argument("--trees", type=int, default=None, help="override T of the workload")
    ap.add_argument("--rounds", type=int, default=None, help="override R of the workload")
    ap.add_argument("--propagation", choices=sorted(PROPAGATION), default="first_order")
    ap.add_argument("--budget", type=int, default=0, help="best-first visit budget")
    ap.add_argument("--r-stop", type=float, default=0.0, help="> 0: divisions until r_m < r_stop (at most T)")
    ap.add_argument("--metric-kind", choices=["l2", "cosine"], default="l2")
    ap.add_argument("--partitioner", choices=["random", "pca"], default="random")
    ap.add_argument("--profile-case", action="store_true",
                    help="one build of the workload's small profiling case (for an ncu launch list), then exit")
    ap.add_argument("--traffic-from", default=None,
                    help="ncu --csv launch list of --profile-case with dram__bytes_{read,write}.sum: record the "
                         "kernels' DRAM bytes per unit under profiles/ and exit")
    ap.add_argument("--traffic-command", default=None, help="the ncu command line, recorded with the traffic")
    ap.add_argument("--traffic-full", action="store_true",
                    help="--traffic-from holds a capture of the full workload (not of --profile-case)")
    ap.add_argument("--traffic-hash", default=None,
                    help="source_hash printed by the profiled --profile-case run (the kernels the counts belong to)")
    args = ap.parse_args()
    if args.workload in ("batched256", "learned10m"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the whole method "
                              "on the sift1m workload only"}))
            return 0
        return run_batched(args) if args.workload == "batched256" else run_learned(args)
    w = dict(WORKLOADS[args.workload])
    if args.trees is not None:
        w["T"] = args.trees
    if args.rounds is not None:
        w["R"] = args.rounds
    if (args.trees, args.rounds) != (None, None) or args.propagation != "first_order" or args.r_stop > 0 \
            or args.metric_kind != "l2" or args.partitioner != "random":
        w["desc"] += f" [T={w['T']}, R={w['R']}, {args.propagation}" + \
            (f", budget {args.budget}" if args.propagation == "best_first" else "") + \
            (f", r_stop {args.r_stop}" if args.r_stop > 0 else "") + f", {args.metric_kind}, {args.partitioner}]"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, w, rank)
    if args.traffic_from:
        return traffic_from_csv(args, w)
    if args.profile_case:
        import torch
        import paper_1307_7852_gb300 as knng
        case = PROFILE_CASE[args.workload]
        wc = dict(w, n=case["n"], centers=case["centers"])
        Xc = torch.from_numpy(make_data(wc, seed=args.data_seed)).cuda()
        knng.knng_build(Xc, w["k"], w["T"], w["g"], w["R"], args.seed, PRECISIONS[args.precision], 2)
        torch.cuda.synchronize()
        print(f"source_hash={source_hash()}", flush=True)
        return 0

    import torch
    import paper_1307_7852_gb300 as knng
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    # CPU oracle work runs before the first CUDA call (no fork after CUDA init)
    X = make_data(w, seed=args.data_seed + rank)
    n, d, k, T, g, R = w["n"], w["d"], w["k"], w["T"], w["g"], w["R"]
    prec = PRECISIONS[args.precision]
    Xd = torch.from_numpy(X).to(dev)
    ids = torch.empty((n, k), dtype=torch.int32, device=dev)
    dists = torch.empty((n, k), dtype=torch.float32, device=dev)
    h = knng.Handle(local)
    stream = torch.cuda.current_stream(dev)
    nev = 4 + R
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(args.steps)]
    for row in ev:  # torch creates the CUDA event on first record
        for e_ in row:
            e_.record(stream)

    opts = dict(metric=1 if args.metric_kind == "cosine" else 0, propagation=PROPAGATION[args.propagation],
                budget=args.budget, r_stop=args.r_stop, partitioner=1 if args.partitioner == "pca" else 0)

    def step(events=None):
        if events is not None:
            knng.knng_set_stage_events(events, h)
        knng.knng_build(Xd, k, T, g, R, args.seed, prec, 2, ids=ids, dists=dists, h=h, **opts)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = knng.knng_launch_counter()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        t_start.record(stream)
        for s in range(args.steps):
            step(ev[s])
        t_end.record(stream)
        torch.cuda.synchronize()
    knng.knng_set_stage_events(None, h)
    launches = knng.knng_launch_counter() - l0
    div_used, div_rates = knng.knng_divisions_used(h)
    el, _ = aggregate(t_start.elapsed_time(t_end) / 1e3, n, world, dist, dev)
    sec = el / args.steps
    value = n * world / sec
    names = ["partition", "leaf_knn", "merge"] + [f"propagate_r{r}" for r in range(R)]
    stage_ms = {nm: statistics.mean(ev[s][i].elapsed_time(ev[s][i + 1]) for s in range(args.steps))
                for i, nm in enumerate(names)}

    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16+f32", "fp8": "e4m3+f32"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "n": n, "d": d, "k": k, "T": T,
                   "leaf_size": g, "rounds": R, "precision": args.precision, "seed": args.seed,
                   "propagation": args.propagation, "budget": args.budget, "r_stop": args.r_stop,
                   "metric": args.metric_kind, "partitioner": args.partitioner,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2 (X = {X.nbytes / 2**20:.0f} MiB > 126 MiB)"},
        "stage_ms": {k_: round(v, 4) for k_, v in stage_ms.items()},
        "gpu_launches": launches,
        "divisions_used": div_used,
        "clocks": clk.summary(),
    }

    if not args.no_extras and rank == 0:
        hbm, bf16, sm_mhz, src = peaks()
        off = knng.knng_leaf_offsets(n, g)
        m = np.diff(off).astype(np.float64)
        depth = knng.knng_split_levels(n, g)
        # bytes per row entry the gathers read: float rows holding only bytes
        # (d <= 256) are read from their exact byte copy
        byte_rows = X.dtype == np.float32 and d <= 256 and args.metric_kind == "l2" and bool(
            np.all((X >= 0) & (X <= 255) & (X == np.rint(X))))
        s_el = 1 if byte_rows else X.itemsize
        traffic = load_traffic(args.workload if args.workload != "sift400k" else "sift1m", args.precision)
        tr = (traffic or {}).get("per_unit", {})
        plain = args.propagation == "first_order" and args.partitioner == "random" and args.metric_kind == "l2"
        roof = {}
        # ---- propagation: what the build's rounds read, counted on the device
        # (one more, untimed build with the read counters on), next to the
        # plain first-order count k^2*4 + u*d*s + k*8 per point ("survey
        # bytes"; u measured on a sample of the graphs the rounds start from)
        if R > 0 and args.propagation == "first_order":
            cnt = torch.zeros(2 * R, dtype=torch.int64, device=dev)
            knng.knng_set_propagation_counters(cnt, h)
            step()
            torch.cuda.synchronize()
            knng.knng_set_propagation_counters(None, h)
            counts = cnt.cpu().numpy().reshape(R, 2)
            perm = knng.knng_partition(Xd, T, g, args.seed, h=h)
            li, ld_ = knng.knng_leaf_knn(Xd, T, g, perm, k, prec, 2, h=h)
            cur_i, cur_d = knng.knng_merge(li, ld_, h=h)
            del perm, li, ld_
            rng = np.random.default_rng(7)
            samp = rng.choice(n, size=min(n, 20000), replace=False)
            u = []
            for r in range(R):
                u.append(unique_candidates(cur_i.cpu().numpy(), samp))
                if r + 1 < R:
                    cur_i, cur_d = knng.knng_propagate(Xd, cur_i, cur_d, 1, h=h)
            del cur_i, cur_d
            t_prop = [stage_ms[f"propagate_r{r}"] / 1e3 for r in range(R)]
            survey = [n * (k * k * 4 + u[r] * d * s_el + k * 8) for r in range(R)]
            # rows scored and list slots loaded, plus every point's own list,
            # row and output
            scored = [int(counts[r, 0]) * d * s_el + int(counts[r, 1]) * 4 + n * (2 * k * 8 + d * s_el)
                      for r in range(R)]
            dram = None
            if traffic and plain and "propagate_kernel" in tr:
                per = tr["propagate_kernel"]["bytes_per_unit"]
                if len(per) == R:
                    dram = [b * n for b in per]
            ach = sum(scored) / sum(t_prop) / 1e9
            roof["propagate"] = {
                "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": statistics.mean(dram) if dram else None,
                "scored_bytes": statistics.mean(scored), "survey_bytes": statistics.mean(survey),
                "dram_bytes": statistics.mean(dram) if dram else None,
                "survey_achieved": sum(survey) / sum(t_prop) / 1e9,
                "rows_scored_per_point": [float(counts[r, 0]) / n for r in range(R)],
                "list_slots_per_point": [float(counts[r, 1]) / n for r in range(R)],
                "unique_candidates_per_point": u, "ms": sum(t_prop) * 1e3 / R,
                "basis": "achieved = scored_bytes (rows scored and list slots loaded, counted on the device, "
                         "+ each point's list, row and output) per launch / launch time; rows that L2 serves "
                         "(points run in leaf order) count here but not in dram_bytes, so frac may pass 1"}
            if dram:
                roof["propagate"]["dram_gbs"] = sum(dram) / sum(t_prop) / 1e9
                roof["propagate"]["dram_frac"] = sum(dram) / sum(t_prop) / 1e9 / hbm
        # ---- leaf graphs: Gram flops of the distinct pairs (tensor pipe or
        # FP32 ALU), and the bytes the stage reads and writes
        gram_flops = T * float(np.sum(2.0 * d * m * (m - 1) / 2.0))
        t_leaf = stage_ms["leaf_knn"] / 1e3
        leaf_dram = None
        if traffic and plain:
            leaf_dram = sum(tr[kn]["bytes_per_unit"] * n * T for kn in
                            ("leaf_tc_kernel", "leaf_rescore_staged_kernel", "gather_quant_kernel") if kn in tr)
        ach = gram_flops / t_leaf / 1e12
        if prec == 0:
            alu = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
            roof["leaf_knn"] = {"bound": "alu", "achieved": ach, "peak": alu, "unit": "TFLOP/s", "frac": ach / alu,
                                "traffic": leaf_dram, "algorithmic_flops_per_launch": gram_flops}
        else:
            roof["leaf_knn"] = {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                                "frac": ach / bf16, "traffic": leaf_dram, "algorithmic_flops_per_launch": gram_flops}
        if leaf_dram:
            roof["leaf_knn"]["dram_gbs"] = leaf_dram / t_leaf / 1e9
            roof["leaf_knn"]["dram_frac"] = leaf_dram / t_leaf / 1e9 / hbm
        # ---- merge: (T + 1) k 8 bytes per point (algorithmic), DRAM measured
        merge_bytes = n * (T + 1) * k * 8
        ach = merge_bytes / (stage_ms["merge"] / 1e3) / 1e9
        mdram = tr["merge_kernel"]["bytes_per_unit"] * n if (traffic and plain and "merge_kernel" in tr) else None
        roof["merge"] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "traffic": mdram, "algorithmic_bytes_per_launch": merge_bytes}
        # ---- partition: depth * n * d * s per tree plus 16 bytes of keys and
        # permutation per point and level ("survey bytes"); the rows the kernels
        # read: byte rows once per tree and level (node-major), float rows
        # once per level for all trees (point-major)
        part_survey = T * depth * (n * d * s_el + 16 * n)
        rows_read = depth * n * d * s_el * (T if byte_rows else 1)
        part_read = rows_read + T * depth * 16 * n
        t_part = stage_ms["partition"] / 1e3
        # DRAM bytes of the projection kernels (the select and scatter
        # kernels are not in the record)
        pdram = None
        if traffic and plain:
            pk = [tr[kn]["bytes_per_unit"] * n for kn in ("project_kernel", "project_bytes_tma_kernel") if kn in tr]
            pdram = sum(pk) if pk else None
        roof["partition"] = {"bound": "hbm", "achieved": part_read / t_part / 1e9, "peak": hbm, "unit": "GB/s",
                             "frac": part_read / t_part / 1e9 / hbm, "traffic": pdram,
                             "read_bytes": part_read, "survey_bytes": part_survey,
                             "survey_achieved": part_survey / t_part / 1e9, "levels": depth}
        if traffic:
            roof["dram_capture"] = {"source_hash": traffic["source_hash"], "case": traffic["case"],
                                    "command": traffic.get("command", "")}
        # the kernel that takes the most time in a step carries the headline
        # roofline object (its figures are per launch)
        stage_of = {"leaf_knn": stage_ms["leaf_knn"], "merge": stage_ms["merge"],
                    "partition": stage_ms["partition"]}
        if "propagate" in roof:
            stage_of["propagate"] = sum(stage_ms[f"propagate_r{r}"] for r in range(R))
        dom = max(stage_of, key=stage_of.get)
        line["roofline"] = dict(roof[dom], kernel=dom, peak_source=src)
        line["roofline_all"] = roof

        # ---- recall on a sample against exact brute force (GPU, same FP32 distance)
        if not args.no_recall:
            from paper_1307_7852_gb300 import synthetic
            q = synthetic.sample_ids(n, args.recall_sample, args.seed + 1)
            qd = torch.from_numpy(q).to(dev)
            ei, ed = knng.knng_exact_knn(Xd, qd, k, h=h)
            got_i = ids[qd.long()]
            got_d = dists[qd.long()]
            kth = ed[:, -1:]
            tie = (got_d <= kth).sum(1).float().mean().item() / k
            gi = got_i.cpu().numpy()
            eii = ei.cpu().numpy()
            idset = float(np.mean([len(set(gi[r]) & set(eii[r])) / k for r in range(len(q))]))
            line["recall"] = {"tie_tolerant": tie, "id_set": idset, "sample": int(len(q)),
                              "reference": "exact brute force over all n (GPU, FP32 distances)"}
            line["distance_error"] = distance_errors(X, q, gi, got_d.cpu().numpy(), args.precision,
                                                     args.metric_kind == "cosine")

        # ---- end to end through the host-buffer C ABI call
        if not args.no_e2e:
            Xp = torch.from_numpy(X).pin_memory()
            oi = torch.empty((n, k), dtype=torch.int32).pin_memory()
            od = torch.empty((n, k), dtype=torch.float32).pin_memory()
            Xn, oin, odn = Xp.numpy(), oi.numpy(), od.numpy()
            knng.knng_build_host(Xn, k, T, g, R, args.seed, prec, 2, ids=oin, dists=odn, device=local, h=h, **opts)
            tt = []
            for _ in range(args.e2e_steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                knng.knng_build_host(Xn, k, T, g, R, args.seed, prec, 2, ids=oin, dists=odn, device=local, h=h,
                                     **opts)
                tt.append(time.perf_counter() - t0)
            e2e_sec = statistics.mean(tt)
            line["e2e"] = {"value": n / e2e_sec, "unit": "points/s", "h2d_bytes_per_step": int(X.nbytes),
                           "d2h_bytes_per_step": int(n * k * 8), "ms_per_step": e2e_sec * 1e3,
                           "api": "knng_build_host (pinned host buffers)"}

    # ---- the CPU oracle on a bounded sample (rank 0, N = 1 only)
    if not args.no_extras and not args.no_cpu_baseline and rank == 0 and world == 1 and args.partitioner == "random":
        import oracle
        # about 15 s of oracle work: fewer points for wider rows
        ns = min(args.cpu_sample * 128 // max(d, 128), n)
        Xs = np.ascontiguousarray(X[:ns])
        t0 = time.perf_counter()
        oracle.build_graph(Xs, k, T, g, R, args.seed, metric=opts["metric"], prop=opts["propagation"],
                           budget=opts["budget"], r_stop=opts["r_stop"])  # (random partitioner only)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ns / dt, "unit": "points/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"first {ns} points of the workload, whole method "
                                                            f"({dt:.1f} s)"}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
