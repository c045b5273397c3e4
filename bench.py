#!/usr/bin/env python
"""GRNND build benchmark on one GB300 (or N independent replicas under torchrun).

A step is one whole build (Alg 3: rnd_init, T1 x T2 rounds of rnd_join + rev_merge,
reverse sampling, final prune, export, search entry) of the SIFT-shaped synthetic
workload: n = 1,000,000 points of d = 128, S = 32, R = 64, T1 = 4, T2 = 15, rho = 0.6,
seeded, integer values in [0, 255].  `value` = points/s with the points resident in
HBM; `e2e` = the same through grnnd_build with pinned host input and the graph read
back to pinned host memory.  Recall@10 at beam 64 over 10,000 held-out queries is
measured after the timed region.

`--impl reference` times the FP64 CPU oracle (the correctness reference) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "build points/s at recall@10>=0.95 (BF16 vs FP32, 1 GB300); p50/p99 build latency"
WORKLOAD = dict(workload="SIFT1M-shaped synthetic build: n=1,000,000, d=128, 1000-cluster mixture, "
                         "integers in [0,255]; S=32, R=64, T1=4, T2=15, rho=0.6; 10,000 queries, k=10, beam 64",
                n=1_000_000, d=128, S=32, R=64, T1=4, T2=15, rho=0.6, nq=10_000, k=10, beam=64)
# ncu DRAM bytes (read + write) per unit of the join -- one round, i.e. its warp and team
# launches -- for the workload above: DRAM bytes per algorithmic byte of the join, measured by
# an ncu capture of rounds 1 and 2 of a 600,000-point build of the same generator (BF16 rows
# of 173 MB, larger than L2; 0.8135 = 7.962 GB / 9.787 GB), times the full workload's
# algorithmic bytes per round (2.2025e9); reported only while the join kernels' code is
# unchanged since that capture.
TRAFFIC = {"kernel": "rnd_join", "form": "bf16", "n": 1_000_000, "bytes_per_launch": 0.8135 * 2.2025e9,
           "source_sha256": "96bf15c3714c04b97486ad8f711a3b0c68672b25a39073616d44eaedf014b20d"}


CACHE_BYTES = 16 << 30  # grnnd_set_memory_cache for the timed builds of our arm


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"], help="points (default: the full workload)")
    ap.add_argument("--nq", type=int, default=WORKLOAD["nq"])
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-recall", action="store_true")
    ap.add_argument("--no-gist", action="store_true",
                    help="skip the GIST-shaped 1M x 960 line (BF16 and FP32 build, recall by beam) of a full-size run")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--forms", default="fp32,bf16", help="comma list of fp32, bf16, fp8 (the last one is the headline)")
    ap.add_argument("--report", choices=["precision", "ablation", "batched", "serve", "rounds"], default=None,
                    help="precision: per-form distance error against FP64 and recall loss on a "
                         "GIST-shaped (d=960, continuous) or DEEP-shaped (d=96, IP) set of --n points")
    ap.add_argument("--shape", choices=["gist", "deep"], default="gist")
    ap.add_argument("--serve-seconds", type=float, default=30.0, help="serve report: length of the arrival stream")
    ap.add_argument("--rounds", type=int, default=2, help="rounds report: rounds of the first outer iteration")
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.index = ids[local_rank] if local_rank < len(ids) and ids[local_rank].strip().isdigit() else str(local_rank)
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", self.index, "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9 and p[1].replace(".", "").isdigit():
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()) if rows else None,
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------------------

CPU_SAMPLE = 50_000  # points of the oracle's bounded sample (both the CPU baseline and the reference arm)


def oracle_build_rate(X, n_sample: int, threads: int = 1):
    """The FP64 oracle's build of the first n_sample points: orc_build itself (threads = 1),
    or the same steps of the oracle with its per-vertex prunes and per-target merges split
    over `threads` host threads (oracle/grnnd_oracle_mt.c; the same graph, tested)."""
    from oracle import oracle as O
    O.build()
    Xs = X[:n_sample]
    w = WORKLOAD
    t = time.perf_counter()
    if threads == 1:
        O.build_graph(Xs, w["S"], w["R"], w["T1"], w["T2"], w["rho"], 0)
    else:
        O.build_graph_mt(Xs, w["S"], w["R"], w["T1"], w["T2"], w["rho"], 0, threads=threads)
    dt = time.perf_counter() - t
    return n_sample / dt, dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2510_02774_gb300 import synth
    X = synth.sift_like(args.n, 0, seed=args.seed)
    n_s = min(CPU_SAMPLE, args.n)
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_build_rate(X, n_s, cores)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_build_rate(X, n_s, cores)
        times.append(dt)
    tot = sum(times)
    value = n_s * args.steps / tot
    sample = (f"oracle build of the first {n_s} points of the same {args.n}-point dataset per step "
              f"(S=32, R=64, T1=4, T2=15), FP64, the oracle's per-vertex prunes and per-target merges "
              f"over {cores} host threads (its initialisation single-threaded)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**{k: v for k, v in WORKLOAD.items()}, "n": args.n, "sample_points": n_s},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------

KERNELS_PER_GROUP = {"scan": 2, "entry": 6}
JOIN_KERNELS = ("rnd_join_warp", "rnd_join_team", "rnd_join")


def _pct(xs, p):
    q = sorted(xs)
    return q[min(len(q) - 1, int(round(p * (len(q) - 1))))]


def _source_sha():
    """sha256 of the code of the join kernels that the traffic figure was taken on (the warp
    and team joins of pool_kernels.cu, with common.cuh and kernels.cuh): comments and blank
    lines removed, so the figure follows the code, not its commentary."""
    import re
    csrc = os.path.join(ROOT, "paper_2510_02774_gb300", "csrc")
    with open(os.path.join(csrc, "pool_kernels.cu")) as f:
        text = f.read()
    a = text.index("// rnd_join for pools of at most 32 entries")
    b = text.index("// rev_merge: exclusive scan")
    parts = [text[a:b]]
    for h in ("common.cuh", "kernels.cuh"):
        with open(os.path.join(csrc, h)) as f:
            parts.append(f.read())
    lines = [re.sub(r"\s*//.*$", "", ln).rstrip() for ln in "\n".join(parts).splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def join_algorithmic_bytes(rows, n, proposals, fired, rechecks, d, elem):
    """Algorithmic bytes of the join over some rounds: rows gathered (elem bytes per
    dimension), pool degrees read once per round, every entry proposed (kept in place or
    written) once, each redirect written (target + key) and counted, and the FP32 rows of
    every re-decided pair (three rows: the pair and the row it is decided against)."""
    return rows * d * elem + n * 4 + proposals * 8 + fired * (12 + 4) + rechecks * 3 * d * 4


def gist_line(seed):
    """The same metric on the precision workload at full size: GIST-shaped 1M x 960 (continuous,
    per-dimension scales spanning 100x), BF16 and FP32 forms, one warm-up and one timed build
    each (CUDA events around the build call, points resident on the device), and recall@10
    of 1000 held-out queries against exact k-NN at beams 64, 80, 96 and 128 (the smallest
    beam reaching 0.95 is reported: at beam 64 this workload stays just below it)."""
    import numpy as np
    import torch
    from paper_2510_02774_gb300 import grnnd, synth
    n, nq, k = 1_000_000, 1000, 10
    kw = dict(S=32, R=64, T1=4, T2=15, rho=0.6, seed=seed)
    X, Q = synth.gist_like(n, nq, seed=seed)
    d = X.shape[1]
    Xd = torch.from_numpy(X).cuda()
    Qt = torch.from_numpy(Q).cuda()
    Xp, _ = grnnd.device_points(X)
    Qp, _ = grnnd.device_points(Q)
    del X
    gt = grnnd.brute_knn(Xp, d, Qp, k)[0].cpu().numpy()
    del Xp
    out = {"workload": f"GIST1M-shaped synthetic: n={n}, d={d}, 500-cluster mixture, per-dimension scales "
                       f"log-uniform in [0.1, 10]; S 32, R 64, T1 4, T2 15; {nq} held-out queries, k={k}",
           "forms": {}}
    for name, prec in (("bf16", grnnd.BF16), ("fp32", grnnd.FP32)):
        grnnd.build(Xd, precision=prec, **kw)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        g = grnnd.build(Xd, precision=prec, **kw)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        by_beam = {}
        for bm in (64, 80, 96, 128):
            found = g.search(Qt, k, bm).cpu().numpy()
            by_beam[bm] = float(np.mean([len(set(a.tolist()) & set(b.tolist())) / k for a, b in zip(found, gt)]))
            if by_beam[bm] >= 0.95:
                break
        out["forms"][name] = {"build_ms": ms, "points_per_s": n / (ms / 1e3), "recall@10_by_beam": by_beam,
                              "smallest_beam_recall_0.95": min((b for b, r in by_beam.items() if r >= 0.95),
                                                               default=None)}
        del g
    out["bf16_speedup_vs_fp32"] = out["forms"]["fp32"]["build_ms"] / out["forms"]["bf16"]["build_ms"]
    return out


def run_precision_report(args):
    """Each form's distance error against FP64 and its recall loss, on continuous data.

    Builds the graph of the same points with the FP32, BF16 and FP8 forms, then:
      * recall@10 of a beam-64 search of 1000 held-out queries against exact k-NN (GPU brute
        force); the BF16 form's loss is FP32 recall - BF16 recall;
      * the recorded distance of every edge against the FP64 distance recomputed on the host
        (relative error |d_rec - d_64| / max(d_64, tiny)), and how many prune decisions the
        BF16 form re-took in FP32."""
    import numpy as np
    import torch
    from paper_2510_02774_gb300 import build as B
    B.build()
    from paper_2510_02774_gb300 import grnnd, synth
    n, nq, k, beam = args.n, 1000, 10, 64
    if args.shape == "gist":
        X, Q = synth.gist_like(n, nq, seed=args.seed)
        metric, kw = grnnd.L2SQ, dict(S=32, R=64, T1=4, T2=15, rho=0.6, seed=args.seed)
        shape = f"GIST1M-shaped synthetic: n={n}, d=960, 500-cluster mixture, per-dimension scales log-uniform in [0.1, 10]; S 32, R 64, T1 4, T2 15"
    else:
        X, Q = synth.deep_like(n, nq, seed=args.seed)
        metric, kw = grnnd.IP, dict(S=16, R=32, T1=3, T2=10, rho=0.6, seed=args.seed)
        shape = f"DEEP-shaped synthetic: n={n}, d=96, unit vectors, 50-cluster vMF-like mixture, inner product; S 16, R 32, T1 3, T2 10"
    d = X.shape[1]
    Xd = torch.from_numpy(X).cuda()
    Xp, _ = grnnd.device_points(X)
    Qp, _ = grnnd.device_points(Q)
    gt, _ = grnnd.brute_knn(Xp, d, Qp, k, metric=metric)
    gt = gt.cpu().numpy()
    X64 = X.astype(np.float64) if n <= 200_000 else X  # rows are widened per chunk on large sets
    out = {"report": "precision", "workload": shape, "queries": nq, "k": k, "beam": beam, "forms": {}}
    for name, prec in (("fp32", grnnd.FP32), ("bf16", grnnd.BF16), ("fp8", grnnd.FP8)):
        g = grnnd.build(Xd, precision=prec, metric=metric, **kw)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        g2 = grnnd.build(Xd, precision=prec, metric=metric, **kw)
        t1.record()
        torch.cuda.synchronize()
        Qt = torch.from_numpy(Q).cuda()

        def recall_at(bm):
            found = g2.search(Qt, k, bm).cpu().numpy()
            return float(np.mean([len(set(a.tolist()) & set(b.tolist())) / k for a, b in zip(found, gt)]))

        rec = recall_at(beam)
        # the smallest candidate list of these that reaches recall@10 >= 0.95
        beams = {bm: (rec if bm == beam else recall_at(bm)) for bm in (48, 64, 80, 96, 128, 192, 256)}
        min_beam = min((bm for bm, r in beams.items() if r >= 0.95), default=None)
        ids, dist, deg = g2.to_numpy()
        mask = np.arange(ids.shape[1])[None, :] < deg[:, None]
        rows = np.nonzero(mask)[0]
        cols = ids[mask].astype(np.int64)
        rec_d = dist[mask].astype(np.float64)
        if len(rows) > 2_000_000:  # a seeded sample of the edges on large sets
            pick = np.random.default_rng(1).choice(len(rows), 2_000_000, replace=False)
            rows, cols, rec_d = rows[pick], cols[pick], rec_d[pick]
        d64 = np.empty(len(rows))
        for a in range(0, len(rows), 1 << 16):  # FP64 recomputation in chunks
            xa = X64[rows[a:a + (1 << 16)]].astype(np.float64)
            xb = X64[cols[a:a + (1 << 16)]].astype(np.float64)
            d64[a:a + (1 << 16)] = ((xa - xb) ** 2).sum(1) if metric == grnnd.L2SQ else 1.0 - (xa * xb).sum(1)
        rel = np.abs(rec_d - d64) / np.maximum(np.abs(d64), 1e-30)
        st = g2.stats()
        out["forms"][name] = {"build_ms": t0.elapsed_time(t1), "recall@10": rec, "edges": int(deg.sum()),
                              "recall@10_by_beam": beams, "smallest_beam_recall_0.95": min_beam,
                              "dist_rel_err_max": float(rel.max()), "dist_rel_err_mean": float(rel.mean()),
                              "dist_rel_err_p99": float(np.quantile(rel, 0.99)),
                              "rechecks": int(st["rechecks"]), "pair_distances": int(st["pair_distances"])}
        del g, g2
    for q in ("bf16", "fp8"):
        out[q + "_recall_loss"] = out["forms"]["fp32"]["recall@10"] - out["forms"][q]["recall@10"]
        out[q + "_speedup_vs_fp32"] = out["forms"]["fp32"]["build_ms"] / out["forms"][q]["build_ms"]
    print(json.dumps(out), flush=True)




def run_rounds_report(args):
    """The first --rounds rounds of the bench workload's build (BF16 form) through the step
    calls, one JSON line per round with its counters and the join's algorithmic bytes: the
    reference figures for a DRAM capture of the same rounds' join launches."""
    import torch
    from paper_2510_02774_gb300 import build as B
    B.build()
    from paper_2510_02774_gb300 import grnnd, synth
    w = WORKLOAD
    n, d = args.n, w["d"]
    X = synth.sift_like(n, 0, seed=args.seed)
    Xd, _ = grnnd.device_points(X)
    qp = grnnd.quantize(Xd, d, grnnd.BF16)
    keys, deg = grnnd.pool_init(Xd, d, w["S"], w["R"], args.seed)
    ws = grnnd.workspace(n, w["R"])
    for t2 in range(1, args.rounds + 1):
        st = torch.zeros(8, dtype=torch.int64, device="cuda")
        keys, deg = grnnd.join_round(Xd, d, keys, deg, args.seed, 1, t2, ws=ws, stats=st, inplace=True,
                                     precision=grnnd.BF16, qpoints=qp)
        grnnd.workspace_status(ws, n, w["R"])
        s = st.cpu().tolist()
        algo = join_algorithmic_bytes(s[1], n, s[4], s[3], 0, d, 2)
        print(json.dumps({"report": "rounds", "n": n, "t1": 1, "t2": t2, "vertices_with_new": s[0],
                          "rows_gathered": s[1], "pair_distances": s[2], "pairs_fired": s[3], "proposals": s[4],
                          "join_algorithmic_bytes": algo}), flush=True)


def run_ablation_report(args):
    """Sec 4.3-style ablations on the SIFT-shaped set (--n points, BF16 form): pair-visit order
    (ascending / descending / random), reverse-sampling ratio rho, the T1 x T2 split, and the
    search beam (queries per second against recall@10).  One JSON line per setting."""
    import numpy as np
    import torch
    from paper_2510_02774_gb300 import build as B
    B.build()
    from paper_2510_02774_gb300 import grnnd, synth
    n, nq, k = args.n, 10000, 10
    X, Q = synth.sift_like(n, nq, seed=args.seed)
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    Xp, _ = grnnd.device_points(X)
    Qp, _ = grnnd.device_points(Q)
    gt = grnnd.brute_knn(Xp, X.shape[1], Qp, k)[0].cpu().numpy()
    base = dict(S=32, R=64, T1=4, T2=15, rho=0.6, seed=args.seed, order=grnnd.ORDER_RANDOM)

    def recall(found):
        return float(np.mean([len(set(a.tolist()) & set(b.tolist())) / k for a, b in zip(found, gt)]))

    def run(tag, **over):
        kw = dict(base, **over)
        grnnd.build(Xd, precision=grnnd.BF16, **kw)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g = grnnd.build(Xd, precision=grnnd.BF16, **kw)
        e1.record()
        torch.cuda.synchronize()
        ids, dist, deg = g.to_numpy()
        line = {"report": "ablation", "sweep": tag, "n": n, **{k2: v for k2, v in kw.items() if k2 != "seed"},
                "build_ms": e0.elapsed_time(e1), "points_per_s": n / (e0.elapsed_time(e1) / 1e3),
                "recall@10_beam64": recall(g.search(Qd, k, 64).cpu().numpy()),
                "mean_degree": float(deg.mean())}
        print(json.dumps(line), flush=True)
        return g

    for name, o in (("ascending", grnnd.ORDER_ASC), ("descending", grnnd.ORDER_DESC), ("random", grnnd.ORDER_RANDOM)):
        run("order:" + name, order=o)
    for rho in (0.0, 0.3, 0.6, 0.9, 1.0):
        run("rho", rho=rho)
    for t1, t2 in ((1, 60), (2, 30), (3, 20), (4, 15), (6, 10), (10, 6)):
        run("T1xT2", T1=t1, T2=t2)
    g = run("beam-graph")
    for beam in (10, 16, 24, 32, 48, 64, 96, 128, 192, 256):
        g.search(Qd, k, beam)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        found = g.search(Qd, k, beam)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"report": "ablation", "sweep": "search_beam", "n": n, "queries": nq, "beam": beam,
                          "qps": nq / (ms / 1e3), "recall@10": recall(found.cpu().numpy())}), flush=True)


def run_batched_report(args):
    """The batched form: 512 independent builds of n log-uniform in [1k, 50k] DEEP-shaped
    unit vectors (d = 96, a 50-cluster mixture per build, inner product, BF16 tiles; S 16,
    R 32, T1 3, T2 10) in one grnnd_build_batch pass, against the same builds one
    grnnd_build_ex call after another.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_2510_02774_gb300 import build as B
    B.build()
    from paper_2510_02774_gb300 import grnnd, synth
    nbuild = 512
    g = np.random.default_rng(args.seed)
    sizes = np.exp(g.uniform(np.log(1000), np.log(50000), nbuild)).astype(np.int64)
    parts = [synth.deep_like(int(m), 0, seed=1000 + b) for b, m in enumerate(sizes)]
    X = torch.from_numpy(np.concatenate(parts)).cuda()
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    total = int(off[-1])
    kw = dict(S=16, R=32, T1=3, T2=10, rho=0.6, seed=args.seed, metric=grnnd.IP, precision=grnnd.BF16)
    del parts
    # warm-up of both paths
    grnnd.build_batch(X[: int(off[8])], off[:9], **kw)
    grnnd.build(X[: int(off[1])], **kw)
    torch.cuda.synchronize()

    def timed(fn, reps):
        ts = []
        out = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t = time.perf_counter()
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append((e0.elapsed_time(e1), (time.perf_counter() - t) * 1e3))
            if reps > 1:
                del out
                out = None
        return ts, out

    # the autotuner on a batch of 64 of the builds, then the whole batched pass with its choice
    tune = grnnd.autotune(X[: int(off[64])], offsets=off[:65], **kw)
    tb0, _ = timed(lambda: grnnd.build_batch(X, off, **kw), max(3, args.steps))
    tb, _ = timed(lambda: grnnd.build_batch(X, off, tuning=tune, **kw), max(3, args.steps))
    ts, _ = timed(lambda: [grnnd.build(X[int(off[b]):int(off[b + 1])], **kw) for b in range(nbuild)], 1)
    # the same results both ways (a sample of builds)
    gs = grnnd.build_batch(X, off, **kw)
    same = True
    for b in (0, 1, nbuild // 2, nbuild - 1):
        one = grnnd.build(X[int(off[b]):int(off[b + 1])], **kw)
        same &= bool((gs[b].to_numpy()[0] == one.to_numpy()[0]).all()) and gs[b].entry == one.entry
    bms = sorted(t[1] for t in tb)
    # the pool-capacity autotuner on the largest build's generator (its rows plus 500 held-out
    # queries): the fastest R of 16, 24, 32 whose graph reaches recall@10 >= 0.95 at beam 64,
    # then the batched pass with that capacity
    bmax = int(np.argmax(sizes))
    Xs, Qs = synth.deep_like(int(sizes[bmax]), 500, seed=1000 + bmax)
    kwp = {k2: v for k2, v in kw.items() if k2 != "R"}
    R_pool, rec_pool, ms_pool = grnnd.autotune_pool(np.concatenate([Xs, Qs]), 500, [16, 24, 32],
                                                    recall_target=0.95, k=10, beam=64, tuning=tune, **kwp)
    tp, _ = timed(lambda: grnnd.build_batch(X, off, tuning=tune, **{**kw, "R": R_pool, "S": min(16, R_pool)}),
                  max(3, args.steps))
    grnnd.profile_begin()
    grnnd.build_batch(X, off, tuning=tune, **kw)  # not captured while profiling
    torch.cuda.synchronize()
    kern = {k2: round(v[1], 2) for k2, v in sorted(grnnd.profile_end().items(), key=lambda kv: -kv[1][1])}
    line = {"report": "batched", "workload": "512 builds, n log-uniform in [1000, 50000], DEEP-shaped d=96 unit "
                                              "vectors (50-cluster mixture per build), IP, BF16; S 16, R 32, T1 3, T2 10",
            "builds": nbuild, "points": total, "min_n": int(sizes.min()), "max_n": int(sizes.max()),
            "batched_ms_p50": bms[len(bms) // 2], "batched_points_per_s": total / (bms[len(bms) // 2] / 1e3),
            "batched_builds_per_s": nbuild / (bms[len(bms) // 2] / 1e3),
            "sequential_ms": ts[0][1], "sequential_points_per_s": total / (ts[0][1] / 1e3),
            "speedup": ts[0][1] / bms[len(bms) // 2], "same_graphs_sampled": same,
            "tuning": tune.as_dict(), "batched_default_tuning_ms_p50": sorted(t[1] for t in tb0)[len(tb0) // 2],
            "pool_autotune": {"sample_n": int(sizes[bmax]), "queries": 500, "candidates": [16, 24, 32],
                              "recall_target": 0.95, "R": R_pool, "recall@10": rec_pool, "sample_build_ms": ms_pool,
                              "batched_ms_p50": sorted(t[1] for t in tp)[len(tp) // 2]},
            "kernels_ms_profiled_pass": kern}
    print(json.dumps(line), flush=True)


def run_serve_report(args):
    """Serving loop (grnnd_server_*): a Poisson stream of requests at 20 per second, each a
    build (n log-uniform in [5k, 500k], d 128 SIFT-shaped L2 with S 32, R 64, T1 4, T2 15, or
    d 96 DEEP-shaped inner product with S 16, R 32, T1 3, T2 10; BF16 tiles with FP32
    re-decisions) or a search of 1..1024 queries (k 10, beam 64) against a resident index,
    admitted under a 150 GB HBM budget on 4 slots.  Points and queries come from pinned host
    memory (slices of two seeded 2M-point sets).  Reports p50/p99 latency per kind (submit to
    done, the server's clock), then a burst of the stream's builds all submitted at once
    against the same builds run one after another through grnnd_build_ex (FP32, the plain
    per-request path, and BF16).  One JSON line."""
    import numpy as np
    import torch
    from paper_2510_02774_gb300 import build as B
    B.build()
    from paper_2510_02774_gb300 import grnnd, synth
    rng = np.random.default_rng(args.seed)
    base = {128: synth.sift_like(2_000_000, 20000, seed=args.seed + 1),
            96: synth.deep_like(2_000_000, 20000, seed=args.seed + 2)}
    base = {d: (torch.from_numpy(X).pin_memory(), torch.from_numpy(Q).pin_memory()) for d, (X, Q) in base.items()}
    cfg = {128: dict(S=32, R=64, T1=4, T2=15, rho=0.6, metric=grnnd.L2SQ),
           96: dict(S=16, R=32, T1=3, T2=10, rho=0.6, metric=grnnd.IP)}
    # the request stream: arrival times and contents, drawn up front
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / 20.0)
        if t > args.serve_seconds:
            break
        if not reqs or rng.random() < 0.5:
            n = int(np.exp(rng.uniform(np.log(5000), np.log(500000))))
            d = int(rng.choice([96, 128]))
            o = int(rng.integers(0, 2_000_000 - n))
            reqs.append(("build", t, d, o, n))
        else:
            nq = int(rng.integers(1, 1025))
            reqs.append(("search", t, None, int(rng.integers(0, 20000 - nq)), nq))
    budget = 150 << 30
    srv = grnnd.Server(slots=4, hbm_budget=budget)
    # warm-up (kernel set-up, pool growth): one build of each shape, then released
    for d in (96, 128):
        srv.release(srv.wait(srv.submit_build(base[d][0][:20000], precision=grnnd.BF16, seed=1, **cfg[d]))["index"])
    ids, built, kinds = [], [], []
    t0 = time.perf_counter()
    for kind, ta, d, o, n in reqs:
        delay = ta - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        if kind == "build":
            rid = srv.submit_build(base[d][0][o:o + n], precision=grnnd.BF16, seed=len(built), **cfg[d])
            built.append((rid, d))
        else:
            idx, dq = built[int(rng.integers(0, len(built)))]
            rid = srv.submit_search(idx, base[dq][1][o:o + n], 10, 64)
        ids.append(rid)
        kinds.append(kind)
    infos = [srv.wait(r) for r in ids]
    wall = time.perf_counter() - t0
    st = srv.status()
    lat = {k: sorted(1e3 * (i["t_done"] - i["t_submit"]) for i in infos if i["kind"] == k) for k in ("build", "search")}
    pts = sum(i["units"] for i in infos if i["kind"] == "build")
    nq_tot = sum(i["units"] for i in infos if i["kind"] == "search")
    sb = [i["batch"] for i in infos if i["kind"] == "search"]
    for rid, _ in built:
        srv.release(rid)
    # burst: the stream's builds all at once, against the same builds one after another
    bl = [(d, o, n) for kind, _, d, o, n in reqs if kind == "build"]
    t1 = time.perf_counter()
    bids = [srv.submit_build(base[d][0][o:o + n], precision=grnnd.BF16, seed=i, **cfg[d]) for i, (d, o, n) in enumerate(bl)]
    for r in bids:
        srv.wait(r)
    burst = time.perf_counter() - t1
    for r in bids:
        srv.release(r)
    # search burst: 2,000 search requests (1..1024 queries each) submitted at once against one
    # resident 500k-point index: waiting searches of the same index are served together
    # (continuous batching); against the same searches one after another through grnnd_search
    idx = srv.wait(srv.submit_build(base[128][0][:500000], precision=grnnd.BF16, seed=7, **cfg[128]))["index"]
    qreq = []
    for _ in range(2000):
        nq = int(rng.integers(1, 1025))
        qreq.append((int(rng.integers(0, 20000 - nq)), nq))
    t3 = time.perf_counter()
    sids = [srv.submit_search(idx, base[128][1][o:o + nq], 10, 64) for o, nq in qreq]
    sinfo = [srv.wait(r) for r in sids]
    sburst = time.perf_counter() - t3
    srv.release(idx)
    srv.close()
    gref = grnnd.build(base[128][0][:500000].numpy(), precision=grnnd.BF16, seed=7, **cfg[128])
    qnp = base[128][1].numpy()
    t4 = time.perf_counter()
    same = True
    for (o, nq), inf in zip(qreq, sinfo):
        same &= bool((gref.search(qnp[o:o + nq], 10, 64) == inf["out"]).all())
    sseq = time.perf_counter() - t4
    del gref
    qtot = sum(nq for _, nq in qreq)
    slat = sorted(1e3 * (i["t_done"] - i["t_submit"]) for i in sinfo)
    sbat = [i["batch"] for i in sinfo]
    seq = {}
    for name, prec in (("fp32", grnnd.FP32), ("bf16", grnnd.BF16)):
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for i, (d, o, n) in enumerate(bl):
            g = grnnd.build(base[d][0][o:o + n], precision=prec, seed=i, **cfg[d])
            del g
        torch.cuda.synchronize()
        seq[name] = time.perf_counter() - t2
    bp = sum(n for _, _, n in bl)

    def pct(xs, q):
        return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))] if xs else None

    line = {"report": "serve",
            "workload": "Poisson stream, 20 requests/s for %.0f s: builds (n log-uniform [5k, 500k]; d 128 SIFT-shaped "
                        "L2 S32 R64 T1 4 T2 15, or d 96 DEEP-shaped IP S16 R32 T1 3 T2 10; BF16) and searches "
                        "(1..1024 queries, k 10, beam 64) on resident indices; 150 GB budget, 4 slots" % args.serve_seconds,
            "requests": len(infos), "builds": len(lat["build"]), "searches": len(lat["search"]),
            "build_latency_ms": {"p50": pct(lat["build"], 0.5), "p99": pct(lat["build"], 0.99)},
            "search_latency_ms": {"p50": pct(lat["search"], 0.5), "p99": pct(lat["search"], 0.99)},
            "stream_points_per_s": pts / wall, "stream_queries_per_s": nq_tot / wall, "stream_wall_s": wall,
            "search_batch_mean": float(np.mean(sb)) if sb else None, "search_batch_max": max(sb) if sb else None,
            "peak_bytes": st["peak_bytes"],
            "search_burst": {"requests": len(qreq), "queries": qtot, "server_s": sburst,
                             "server_queries_per_s": qtot / sburst, "batch_mean": float(np.mean(sbat)),
                             "batch_max": max(sbat), "latency_ms": {"p50": pct(slat, 0.5), "p99": pct(slat, 0.99)},
                             "sequential_s": sseq, "sequential_queries_per_s": qtot / sseq,
                             "results_equal_to_sequential": same},
            "burst": {"builds": len(bl), "points": bp, "server_bf16_s": burst, "server_points_per_s": bp / burst,
                      "sequential_fp32_s": seq["fp32"], "sequential_fp32_points_per_s": bp / seq["fp32"],
                      "sequential_bf16_s": seq["bf16"], "sequential_bf16_points_per_s": bp / seq["bf16"],
                      "speedup_vs_sequential_fp32": seq["fp32"] / burst}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    rank, world, local = _dist()
    if args.report == "precision":
        run_precision_report(args)
        return
    if args.report == "ablation":
        run_ablation_report(args)
        return
    if args.report == "batched":
        run_batched_report(args)
        return
    if args.report == "serve":
        run_serve_report(args)
        return
    if args.report == "rounds":
        run_rounds_report(args)
        return
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2510_02774_gb300 import build as B
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_2510_02774_gb300 import grnnd, synth
    grnnd.lib()
    # builds keep their freed device memory for the next build (a caching allocator; the
    # graphs are the same with or without it)
    grnnd.set_memory_cache(CACHE_BYTES)

    w = WORKLOAD
    n, d = args.n, w["d"]
    X, Q = synth.sift_like(n, args.nq, seed=args.seed + rank)   # each replica builds its own dataset
    Xd = torch.from_numpy(X).cuda()
    kw = dict(S=w["S"], R=w["R"], T1=w["T1"], T2=w["T2"], rho=w["rho"], seed=args.seed)
    stream = torch.cuda.current_stream()

    def timed_form(precision: int):
        """W untimed builds, then K timed builds bracketed by barrier + synchronize; CUDA
        events on the build stream; events around the join's launches (the roofline's kernel)
        and clocks sampled meanwhile.  Then K more builds, not timed, with events around every
        launch, for the per-kernel breakdown and the launch count (an event pair costs about
        2 us of stream time per launch: timing every kernel would slow the timed builds)."""
        for _ in range(args.warmup):
            g = grnnd.build(Xd, precision=precision, **kw)
            del g
        torch.cuda.synchronize()
        clocks = Clocks(local)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        grnnd.profile_begin(only=JOIN_KERNELS)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        g = None
        e0.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            g = grnnd.build(Xd, precision=precision, **kw)
            ev[i][1].record(stream)
            stats.append(g.stats())
            if i + 1 < args.steps:
                del g
        e1.record(stream)
        torch.cuda.synchronize()
        kern = grnnd.profile_end()
        clk = clocks.stop()
        if dist:
            dist.barrier()
        total = e0.elapsed_time(e1)
        t_max = torch.tensor([total], dtype=torch.float64, device="cuda")
        if dist:
            dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        grnnd.profile_begin()
        for _ in range(args.steps):
            g2 = grnnd.build(Xd, precision=precision, **kw)
            del g2
        torch.cuda.synchronize()
        kern_all = grnnd.profile_end()
        return dict(total_ms=float(t_max.item()), step_ms=step_ms, stats=stats, kern=kern, kern_all=kern_all,
                    clocks=clk, graph=g)

    forms = {}
    names = [f.strip() for f in args.forms.split(",") if f.strip()]
    for name in names:
        forms[name] = timed_form({"fp32": grnnd.FP32, "bf16": grnnd.BF16, "fp8": grnnd.FP8}[name])
    head_name = names[-1]
    head = forms[head_name]
    total_ms, step_ms, stats, kern, kern_all, clk, g = (head["total_ms"], head["step_ms"], head["stats"], head["kern"],
                                                       head["kern_all"], head["clocks"], head["graph"])
    value = n * world * args.steps / (total_ms / 1e3)

    # ---- recall@10 at beam 64 on the last graph of each form (not timed) --------------
    recall = {}
    if not args.no_recall and args.nq > 0:
        Xp, _ = grnnd.device_points(X)
        Qp, _ = grnnd.device_points(Q)
        gt, _ = grnnd.brute_knn(Xp, d, Qp, w["k"])
        gt_np = gt.cpu().numpy()
        Qt = torch.from_numpy(Q).cuda()
        for name, f in forms.items():
            found = f["graph"].search(Qt, w["k"], w["beam"]).cpu().numpy()
            recall[name] = float(np.mean([len(set(a.tolist()) & set(b.tolist())) / w["k"]
                                          for a, b in zip(found, gt_np)]))
        del Xp, Qp
    for f in forms.values():
        f["graph"] = None
    del g

    # ---- e2e: public API with pinned host input and the graph read back ----------------
    e2e_steps = args.e2e_steps or args.steps
    Xh = torch.from_numpy(X).pin_memory()
    ids_h = torch.empty((n, w["R"]), dtype=torch.int32).pin_memory()
    deg_h = torch.empty(n, dtype=torch.int32).pin_memory()
    import ctypes
    L = grnnd.lib()

    def e2e_step():
        p = grnnd.params(precision={"fp32": grnnd.FP32, "bf16": grnnd.BF16, "fp8": grnnd.FP8}[head_name], **kw)
        h = ctypes.c_void_p()
        grnnd._check(L.grnnd_build_ex(ctypes.c_void_p(Xh.data_ptr()), n, d, ctypes.byref(p), ctypes.byref(h)))
        grnnd._check(L.grnnd_graph_copy(h, ctypes.c_void_p(ids_h.data_ptr()), None, ctypes.c_void_p(deg_h.data_ptr())))
        L.grnnd_free(h)

    e2e_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_ms = []
    t = time.perf_counter()
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        e2e_step()  # returns after the graph's read-back has completed
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t
    t_e = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t_e, op=dist.ReduceOp.MAX)
    e2e_value = n * world * e2e_steps / float(t_e.item())

    # ---- roofline of the dominant kernel ------------------------------------------------
    # rnd_join runs as two launches per round on disjoint vertex sets (pools of up to 32
    # entries: one warp per vertex; 33..64 entries: a two-warp team, or batched CTAs for
    # FP32 rows longer than 128): their sum is the round's join, measured as one unit.
    # (the join's time from the timed builds; the other kernels' from the profiled ones)
    join = [k for k in JOIN_KERNELS if k in kern]
    groups = {k: v for k, v in kern_all.items() if k not in JOIN_KERNELS}
    if join:
        groups["rnd_join"] = (sum(kern[k][0] for k in join), sum(kern[k][1] for k in join))
    dom_name, (dom_launches, dom_ms) = max(groups.items(), key=lambda kv: kv[1][1])
    agg = {k: sum(s[k] for s in stats) for k in stats[0]}
    rounds = agg["rounds"]
    elem = {"fp32": 4, "bf16": 2, "fp8": 1}[head_name]
    units = dom_launches
    if dom_name == "rnd_join":
        # rows gathered (elem bytes per dimension); pool keys read once; survivors written;
        # redirects out (target + key); FP32 rows of the rechecked pairs
        algo = (join_algorithmic_bytes(agg["rows_gathered"], n, agg["proposals"], agg["pairs_fired"],
                                       agg["rechecks"], d, elem) + (rounds - 1) * n * 4)
        units = rounds
    elif dom_name == "select":
        algo = agg["merged"] * 8 + agg["proposals"] * 8 * 2
    else:
        algo = None
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        hbm_peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        hbm_peak, peak_src = 6800.0, "fallback"
    roof = None
    if algo is not None:
        achieved = algo / (dom_ms / 1e3) / 1e9
        traffic = None
        if (TRAFFIC["kernel"] == dom_name and TRAFFIC["form"] == head_name and TRAFFIC["n"] == n
                and TRAFFIC["source_sha256"] == _source_sha()):
            traffic = TRAFFIC["bytes_per_launch"]
        roof = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_source": peak_src, "traffic": traffic,
                "algorithmic_bytes_per_launch": algo / units,
                "avg_launch_ms": dom_ms / units, "launches": dom_launches,
                "per_round_launches": {k: kern[k][0] // max(1, rounds) for k in join} if dom_name == "rnd_join" else None}
    launches = sum(v[0] * KERNELS_PER_GROUP.get(k, 1) for k, v in kern_all.items())

    # ---- CPU baseline (oracle) on a bounded sample --------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_s = min(CPU_SAMPLE, n)
        cores = host_cores()
        rate, dt = oracle_build_rate(X, n_s, cores)        # all host cores
        rate1, dt1 = oracle_build_rate(X, n_s, 1)          # orc_build as it stands, one core
        cpu = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
               "sample": (f"first {n_s} points of the same dataset, same S/R/T1/T2/rho, FP64; the oracle's "
                          f"per-vertex prunes and per-target merges over {cores} host threads "
                          f"(initialisation single-threaded), {dt:.1f} s"),
               "single_thread": {"value": rate1, "unit": "points/s", "cores": 1, "seconds": dt1}}

    # ---- the same metric on the precision workload (GIST-shaped 1M x 960) ----------------
    gist = None
    if rank == 0 and world == 1 and n == WORKLOAD["n"] and not args.no_gist:
        del Xd
        try:
            gist = gist_line(args.seed)
        except Exception as ex:  # reported in the line; the headline above stands
            gist = {"error": f"{type(ex).__name__}: {ex}"}

    if rank == 0:
        p99 = _pct(step_ms, 0.99)
        line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3"}[head_name], "data": "synthetic",
                "config": {**{k: v for k, v in WORKLOAD.items()}, "n": n, "nq": args.nq,
                           "precision": {"bf16": "bf16 dist_tile (tensor cores, FP32 accumulate, FP32 re-decision)",
                                         "fp8": "fp8-e4m3 dist_tile, per-row scales (tensor cores, FP32 accumulate, "
                                                "FP32 re-decision)",
                                         "fp32": "fp32 dist_tile (CUDA cores)"}[head_name],
                           "l2": "inputs larger than L2 (512 MB of points per replica)",
                           "allocator": f"library memory cache of {CACHE_BYTES >> 30} GiB (grnnd_set_memory_cache)",
                           "parallelism": f"{world} independent replica(s)"},
                "p50_ms": statistics.median(step_ms), "p99_ms": p99, "recall@10": recall.get(head_name),
                "beam": w["beam"],
                "forms": {k: {"value": n * world * args.steps / (f["total_ms"] / 1e3),
                              "ms_per_step": f["total_ms"] / args.steps,
                              "p50_ms": statistics.median(f["step_ms"]), "p99_ms": _pct(f["step_ms"], 0.99),
                              "recall@10": recall.get(k),
                              "kernels_ms": {kk: round(vv[1], 3) for kk, vv in
                                             sorted(f["kern_all"].items(), key=lambda kv: -kv[1][1])},
                              "join_ms_timed": {kk: round(vv[1], 3) for kk, vv in f["kern"].items()}}
                          for k, f in forms.items()},
                "bf16_speedup_vs_fp32": (forms["fp32"]["total_ms"] / forms["bf16"]["total_ms"]
                                         if "fp32" in forms and "bf16" in forms else None),
                "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": n * d * 4,
                        "d2h_bytes_per_step": n * w["R"] * 4 + n * 4,
                        "p50_ms": statistics.median(e2e_ms), "p99_ms": _pct(e2e_ms, 0.99)},
                "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
                "kernels_ms": {k: round(v[1], 3) for k, v in sorted(kern_all.items(), key=lambda kv: -kv[1][1])},
                "kernels_ms_source": (f"{args.steps} further builds with events around every launch "
                                      "(not the timed builds, whose events bracket only the join)"),
                "join_ms_timed": {k: round(v[1], 3) for k, v in kern.items()},
                "build_stats": {k: v / args.steps for k, v in agg.items()},
                "gist1m": gist}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
