#!/usr/bin/env python
"""AdANNS-IVF search throughput on GB300.

One step = one batched AdANNS-IVF search (prep -> cluster mapping at d_c ->
probe inversion -> list scan at d_s with fused top-k -> cross-list merge) of
the whole query batch of the ImageNet-shaped workload (N = 1,281,167 x 2048
database, B = 50,000 queries, nlist = 1024) against a resident index.

Default arm: the CUDA library.  `--impl reference`: the FP64 CPU oracle on the
host cores, each step a bounded sample of the same workload.

Prints one JSON line (rank 0).  Run with torchrun for N > 1 GPUs: each rank
searches its own full query batch against its own replica of the index
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthdata  # noqa: E402

CACHE = os.path.join(ROOT, "_cache")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="adanns", choices=["adanns", "reference"])
    p.add_argument("--workload", default="imagenet")
    p.add_argument("--n", type=int, default=None, help="database rows (default: workload N)")
    p.add_argument("--b", type=int, default=None, help="queries per step (default: workload B)")
    p.add_argument("--d_c", type=int, default=32)
    p.add_argument("--d_s", type=int, default=512)
    p.add_argument("--nprobe", type=int, default=16)
    p.add_argument("--k", type=int, default=100)
    p.add_argument("--nlist", type=int, default=1024)
    p.add_argument("--niter", type=int, default=20)
    p.add_argument("--seed", type=int, default=42)
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target CPU time of the oracle baseline sample")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle legs")
    p.add_argument("--skip-gpu-build", action="store_true",
                   help="do not time the GPU k-means build (profiling runs)")
    p.add_argument("--mode", default="bf16", choices=["f32", "bf16", "fp8"],
                   help="headline path: FP32 scan, or BF16 / FP8 tensor-core scan + FP32 rerank of 4k")
    p.add_argument("--compare", nargs="*", default=["f32", "fp8"],
                   help="other paths timed beside the headline")
    p.add_argument("--serve-seconds", type=float, default=8.0,
                   help="length of each serving run (0 disables the serving phase)")
    p.add_argument("--serve-rate", type=float, default=20000.0,
                   help="mean offered load of the serving runs, queries/s")
    p.add_argument("--serve-rate-small", type=float, default=200000.0,
                   help="query rate of the small-request serving load (above what one "
                        "request per launch sustains, so requests queue and share batches)")
    p.add_argument("--quiet", action="store_true")
    p.add_argument("--accuracy-sweep", action="store_true",
                   help="recall and distance error of every tier vs the FP64 oracle per "
                        "(d_c, d_s, nprobe) on a query sample, instead of the timed run")
    p.add_argument("--sweep-queries", type=int, default=500)
    p.add_argument("--flat-opq", action="store_true",
                   help="exhaustive AdANNS-OPQ byte-budget sweep on the ImageNet-shaped data")
    p.add_argument("--ivfopq", action="store_true",
                   help="IVF-OPQ on the NQ-shaped workload (build, QPS per (d_s, M, nprobe), "
                        "recall@10 against exact search on a query sample) instead of the timed run")
    p.add_argument("--gt-queries", type=int, default=100)
    p.add_argument("--graph", action="store_true",
                   help="AdANNS-DiskANN graph shortlist + rerank on the ImageNet-shaped data")
    p.add_argument("--no-largest", action="store_true",
                   help="skip the largest grid point (d_c = 64, d_s = 2048, nprobe = 32)")
    p.add_argument("--option", action="append", default=[], metavar="NAME=VALUE",
                   help="set a library run-time option first (e.g. SCAN_FILTER=1); recorded in "
                        "the config")
    return p.parse_args()


def log(*a):
    if os.environ.get("RANK", "0") == "0":
        print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self) -> dict:
        rows = [r.split(",") for r in (getattr(self, "out", "") or "").splitlines() if r.strip()]
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle index (cached)
def oracle_index(data, args, N):
    import oracle
    key = f"{args.workload}-{N}-{args.d_c}-{args.nlist}-{args.niter}-{args.seed}"
    path = os.path.join(CACHE, "oracle_ivf_" + hashlib.sha1(key.encode()).hexdigest()[:12] + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        off, ids = oracle.lists_from_assignment(z["assign"], args.nlist)
        return {"centroids": z["centroids"], "assign": z["assign"], "list_off": off,
                "list_ids": ids, "metric": oracle.METRIC_L2_PREFIXNORM,
                "objectives": z["objectives"].tolist(), "build_s": float(z["build_s"])}
    t = time.time()
    train_n = min(N, 256 * args.nlist)
    o = oracle.build_ivf(data["db"], args.d_c, args.nlist, args.niter, train_n, args.seed)
    o["build_s"] = time.time() - t
    os.makedirs(CACHE, exist_ok=True)
    np.savez(path + ".tmp.npz", centroids=o["centroids"], assign=o["assign"],
             objectives=np.array(o["objectives"]), build_s=o["build_s"])
    os.replace(path + ".tmp.npz", path)
    return o


def workload_config(args, N, B):
    scan = {"f32": "FP32 scan", "bf16": "BF16 tensor-core scan + FP32 rerank of 4k",
            "fp8": "FP8-E4M3 tensor-core scan + FP32 rerank of 4k"}[args.mode]
    return {"workload": f"AdANNS-IVF {args.workload}-shaped: N={N:,} d=2048 B={B:,} "
                        f"nlist={args.nlist} d_c={args.d_c} d_s={args.d_s} nprobe={args.nprobe} "
                        f"k={args.k}, {scan}", "mode": args.mode,
            "N": N, "B": B, "d": 2048, "nlist": args.nlist, "d_c": args.d_c, "d_s": args.d_s,
            "nprobe": args.nprobe, "k": args.k, "metric": "L2 on prefix-normalised MR prefixes",
            "l2": "inputs larger than L2 (scanned lists exceed 129 MB)",
            "index": "k-means index built by the FP64 oracle, imported to the GPU"}


def oracle_sample_size(oidx, data, args, target_s):
    """Queries the oracle searches in about target_s seconds (calibrated)."""
    import oracle
    q = data["queries"]
    t = time.time()
    n0 = 8
    oracle.search_ivf(data["db"], oidx, q[:n0], args.d_c, args.d_s, args.nprobe, args.k)
    per = max((time.time() - t) / n0, 1e-5)
    return int(max(8, min(len(q), target_s / per)))


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    w = synthdata.WORKLOADS[args.workload]
    N = args.n or w.N
    B = args.b or w.B
    data = synthdata.make(args.workload, n=N, b=B)
    oidx = oracle_index(data, args, N)
    per_step_s = max(2.0, args.cpu_seconds / max(1, args.steps))
    S = oracle_sample_size(oidx, data, args, per_step_s)
    q = data["queries"][:S]
    for _ in range(args.warmup):
        oracle.search_ivf(data["db"], oidx, q, args.d_c, args.d_s, args.nprobe, args.k)
    t = time.time()
    for _ in range(args.steps):
        oracle.search_ivf(data["db"], oidx, q, args.d_c, args.d_s, args.nprobe, args.k)
    el = time.time() - t
    qps = S * args.steps / el
    cores = os.cpu_count()
    print(json.dumps({
        "impl": "reference", "metric": "QPS at recall@10 vs oracle", "value": qps,
        "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args, N, B),
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{S} queries per step (of {B}), FP64 oracle, {cores} threads"},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- DRAM traffic records
KERNEL_SOURCES = {"mma_scan_kernel": ["mma_scan.cu"],
                  "rerank_chunks_kernel": ["rerank_lists.cu"],
                  "scan_f32_kernel": ["scan_f32.cu"],
                  "dist_f32_kernel": ["stream_f32.cu"],
                  "adc_dist_kernel": ["opq.cu"]}


def kernel_source_hash(kernel):
    """sha1 (first 16 hex digits) of the source files that define `kernel`."""
    h = hashlib.sha1()
    for name in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_2305_19435_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel, mode, workload_key):
    """DRAM bytes (read + write) per launch of `kernel` from a committed ncu
    summary under profiles/ (a line `traffic-record: kernel=... mode=...
    workload=... src_sha1=... bytes_per_launch=...`), used only when it was
    captured on this workload from the current source of the kernel; else
    None, so a stale capture is never reported."""
    import glob
    want = kernel_source_hash(kernel)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                line = line.strip().strip("`")
                if not line.startswith("traffic-record:"):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                if (kv.get("kernel") == kernel and kv.get("mode") == mode
                        and kv.get("workload") == workload_key and kv.get("src_sha1") == want):
                    return float(kv["bytes_per_launch"])
    return None


# ---------------------------------------------------------------- GPU arm
MODES = {"f32": (1, 0), "bf16": (2, 4), "fp8": (4, 4)}   # storage code, rerank multiple of k


def mode_rerank(mode, k):
    return MODES[mode][1] * k


def timed(P, torch, step, steps, stream):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = P.launch_count()
    P.profile_enable(True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = (P.launch_count() - l0) // steps
    prof = P.profile_read()
    host = P.profile_read_host()
    cnt = P.profile_read_counters()
    P.profile_enable(False)
    prof["_host_us"] = (sum(host.values()) / steps, 1)
    timed.counters = {k2: v / steps for k2, v in cnt.items()}   # work counters per step
    return ev0.elapsed_time(ev1) / steps, launches, prof


def serving_phase(P, torch, data, db_dev, args, B):
    """Poisson request streams over two resident indices (d_c = 16 and 64) with
    per-request budgets, each once with every request on the mixed-precision
    path and once on the FP32 path: request sizes uniform in [1, 4096] at the
    offered rate, and small interactive requests (uniform in [1, 64]) at ten
    times that rate, more requests than one launch per request sustains, so they
    queue and share batches."""
    from paper_2305_19435_gb300.serving import Budget, NativeServer, poisson_stream
    idx = {}
    for d_c in (16, 64):
        g = P.build_ivf(db_dev, d_c, args.nlist, args.niter, min(db_dev.shape[0], 256 * args.nlist),
                        args.seed)
        # re-lay the same lists with a BF16 tier for the mixed-precision requests
        off, ids = g.lists()
        assign = torch.empty(db_dev.shape[0], dtype=torch.int32, device="cuda")
        sizes = (off[1:] - off[:-1]).to(torch.int64)
        assign[ids.long()] = torch.repeat_interleave(
            torch.arange(g.nlist, device="cuda", dtype=torch.int32), sizes)
        idx[d_c] = P.index_create(db_dev, g.centroids(), assign, storage=1 | P.STORE_BF16)
        g.free()
    grans = [m for m in P.GRANULARITIES if 64 <= m <= db_dev.shape[1]]
    qh = torch.from_numpy(data["queries"]).pin_memory()
    loads = {"sizes_1_4096": (4096, args.serve_seconds, args.serve_rate),
             "sizes_1_64": (64, min(args.serve_seconds, 2.0), args.serve_rate_small)}
    out = {}
    for load, (max_rows, seconds, rate) in loads.items():
        out[load] = {}
        for mode in ("bf16", "f32"):
            rng = np.random.default_rng(args.seed)   # same budgets and slices for both paths
            arrivals = poisson_stream(rate, seconds, seed=args.seed + 5, max_rows=max_rows)
            srv = NativeServer(idx, streams=3, max_batch=8192, mem_budget=24 << 30).start()
            reqs = []
            t0 = time.perf_counter()
            for (t, n, _) in arrivals:
                d_c = int(rng.choice([16, 64]))
                d_s = int(rng.choice(grans))
                nprobe = int(rng.integers(1, 129))
                k = int(rng.choice([10, 100]))
                b = Budget(d_c, d_s, nprobe, k, P.STORE_BF16, 4 * k) if mode == "bf16" else \
                    Budget(d_c, d_s, nprobe, k)
                lo = int(rng.integers(0, B - n + 1))
                while time.perf_counter() - t0 < t:
                    time.sleep(2e-4)
                reqs.append(srv.submit(qh[lo:lo + n], b, index_key=d_c))
            for r in reqs:
                r.wait(600)
            st = srv.stats()
            srv.stop()
            st["errors"] = sum(1 for r in reqs if r.error is not None)
            st["offered_qps"] = rate
            out[load][mode] = st
    for g in idx.values():
        g.status()
        g.free()
    return {"workload": "Poisson arrivals; budgets d_c in "
                        "{16, 64}, d_s in G within [64, 2048], nprobe U[1, 128], k in {10, 100}; "
                        "bf16 = BF16 tensor-core scan + FP32 rerank of 4k, f32 = exact FP32 "
                        "scan; the native server packs requests whose budgets share a pass",
            "loads": {key: f"request sizes U[1, {v[0]}], mean {v[2]:.0f} queries/s for "
                           f"{v[1]:.0f} s" for key, v in loads.items()},
            **out}


def scan_hbm_phase(P, torch, idx, q, oidx, args, hbm_peak, modes):
    """The list scans where they are memory-bound: a serving-sized batch
    (2,048 queries) with one probe, so almost every probed list is read for a
    single query.  Achieved bandwidth = unique bytes of the probed lists at d_s
    (stored values + per-member ids or scales) / the scan kernel's time."""
    Bq, nprobe, k = 2048, 1, 10
    qq = q[:Bq]
    _, _, probes = P.search_ivf(idx, qq, args.d_c, args.d_s, nprobe, k, return_probes=True)
    probed = np.unique(probes.cpu().numpy())
    sizes = np.diff(oidx["list_off"])[probed].astype(np.int64)
    out = {"workload": f"{Bq} queries, nprobe={nprobe}, k={k}, {len(probed)} distinct lists "
                       f"({int(sizes.sum()):,} members)"}
    for d_s in (512, 2048):
        for mode in modes:
            code, mult = MODES[mode]
            rr = mult * k
            epb = {"f32": 16, "bf16": 64, "fp8": 128}[mode]
            e = {"f32": 4, "bf16": 2, "fp8": 1}[mode]
            dpad = (d_s + epb - 1) // epb * epb if mode != "f32" else d_s
            per_member = dpad * e + (8 if mode == "f32" else 4)
            step = lambda: P.search_ivf(idx, qq, args.d_c, d_s, nprobe, k, storage=code,
                                        rerank_k=rr)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            ms, _, prof = timed(P, torch, step, 10, torch.cuda.current_stream())
            stage = "scan" if mode == "f32" else "mma"
            t = prof.get(stage, (0.0, 1))[0] / 10
            gbs = int(sizes.sum()) * per_member / (t / 1e3) / 1e9 if t else None
            f32_kernel = ("dist_f32_kernel (streaming scan)"
                          if P.get_option(P.OPT_FP32_STREAM) else "scan_f32_kernel")
            out[f"{mode}_ds{d_s}"] = {"kernel": f32_kernel if mode == "f32" else "mma_scan_kernel",
                                      "kernel_ms": t, "step_ms": ms, "achieved_gbs": gbs,
                                      "frac_of_hbm": gbs / hbm_peak if gbs else None}
    return out


def largest_point_phase(P, torch, data, idx, oidx, q, args, N, B, modes, peaks):
    """The largest point of the ImageNet-shaped grid (d_c = 64, d_s = 2048,
    nprobe = 32, k = 100) on an index clustered at d_c = 64, every mode timed
    over the full batch, recall@10 against the oracle on a query sample."""
    import oracle
    d_c, d_s, nprobe, k = 64, 2048, 32, args.k
    steps = max(3, args.steps // 2)
    _, _, probes = P.search_ivf(idx, q, d_c, d_s, nprobe, k, return_probes=True)
    pairs = int(np.diff(oidx["list_off"])[probes.cpu().numpy()].sum())
    S = min(200, B)
    ref = oracle.search_ivf(data["db"], oidx, data["queries"][:S], d_c, d_s, nprobe, k)
    out = {"workload": f"AdANNS-IVF {args.workload}-shaped: N={N:,} d=2048 B={B:,} "
                       f"nlist={args.nlist} d_c={d_c} d_s={d_s} nprobe={nprobe} k={k} "
                       "(largest point of the grid)", "pairs_per_step": pairs,
           "recall_sample": S}
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    for mode in modes:
        code, mult = MODES[mode]
        ids = torch.empty(B, k, dtype=torch.int64, device="cuda")
        dd = torch.empty(B, k, dtype=torch.float32, device="cuda")

        def step(ids=ids, dd=dd, code=code, rr=mult * k):
            P.search_ivf(idx, q, d_c, d_s, nprobe, k, storage=code, rerank_k=rr, out=(ids, dd))

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        ms, launches, prof = timed(P, torch, step, steps, torch.cuda.current_stream())
        sm = {k2: v[0] / steps for k2, v in prof.items()}
        gi = ids[:S].cpu().numpy()
        rec = float(np.mean([len(set(a[:10].tolist()) & set(b[:10].tolist())) / 10.0
                             for a, b in zip(gi, ref["ids"])]))
        row = {"qps": B / (ms / 1e3), "ms_per_step": ms, "stages_ms": sm,
               "recall_at_10_vs_oracle": rec, "gpu_launches": launches}
        if mode != "f32" and sm.get("mma"):
            peak = bf16_peak * (2.0 if mode == "fp8" else 1.0)
            ach = 2.0 * pairs * d_s / (sm["mma"] / 1e3) / 1e12
            row["mma_tflops"] = ach
            row["mma_frac_of_peak"] = ach / peak
        elif mode == "f32" and sm.get("scan"):
            row["scan_tflops"] = 4.0 * pairs * d_s / (sm["scan"] / 1e3) / 1e12
        out[mode] = row
        log(json.dumps({"largest_point": mode, **row}))
    return out


def accuracy_sweep(args):
    """Recall@10 / recall@100 and relative distance error of the FP32, BF16 and
    FP8 paths against the FP64 oracle, for every (d_c, d_s, nprobe) of the
    ImageNet-shaped grid, on the first `sweep_queries` queries."""
    import torch
    import oracle
    import paper_2305_19435_gb300 as P
    P.build()
    w = synthdata.WORKLOADS[args.workload]
    N = args.n or w.N
    data = synthdata.make(args.workload, n=N, b=max(args.sweep_queries, 8))
    qs = data["queries"][:args.sweep_queries]
    db_dev = torch.from_numpy(data["db"]).cuda()
    q_dev = torch.from_numpy(qs).cuda()
    k = args.k
    rows = []
    for d_c in (16, 32, 64):
        a2 = argparse.Namespace(**{**vars(args), "d_c": d_c})
        oidx = oracle_index(data, a2, N)
        idx = P.index_create(db_dev, torch.from_numpy(oidx["centroids"]).cuda(),
                             torch.from_numpy(oidx["assign"].astype(np.int32)).cuda(),
                             storage=1 | P.STORE_BF16 | P.STORE_FP8)
        for d_s in (64, 128, 256, 512, 1024, 2048):
            for nprobe in (1, 4, 16, 32):
                ref = oracle.search_ivf(data["db"], oidx, qs, d_c, d_s, nprobe, k)
                row = {"d_c": d_c, "d_s": d_s, "nprobe": nprobe}
                for mode, (code, mult) in MODES.items():
                    gi, gd = P.search_ivf(idx, q_dev, d_c, d_s, nprobe, k, storage=code,
                                          rerank_k=mult * k)
                    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
                    r10 = float(np.mean([len(set(a[:10]) & set(b[:10])) / 10.0
                                         for a, b in zip(gi, ref["ids"])]))
                    r100 = float(np.mean([len(set(a) & set(b)) / float(k)
                                          for a, b in zip(gi, ref["ids"])]))
                    errs = []
                    for a, da, b, db_ in zip(gi, gd, ref["ids"], ref["dist"]):
                        m = dict(zip(b.tolist(), db_.tolist()))
                        for i, d in zip(a.tolist(), da.tolist()):
                            if i in m and m[i] > 0:
                                errs.append(abs(d - m[i]) / m[i])
                    errs = np.array(errs) if errs else np.zeros(1)
                    row[mode] = {"recall10": r10, "recall100": r100,
                                 "max_rel_err": float(errs.max()), "mean_rel_err": float(errs.mean())}
                rows.append(row)
                log(json.dumps(row))
        idx.free()
    print(json.dumps({"accuracy_sweep": rows, "queries": len(qs), "k": k,
                      "rerank_k": {m: MODES[m][1] * k for m in MODES},
                      "workload": f"{args.workload}-shaped, N={N:,}"}))


def exact_topk_prefixnorm(db, q, d_s, k, chunk=1 << 20):
    """Exact k nearest by squared L2 on normalised d_s prefixes (numpy, FP32
    matrix products over database chunks): the ground truth for recall."""
    Q = q[:, :d_s].astype(np.float32)
    qn = np.linalg.norm(Q, axis=1, keepdims=True)
    Q = np.where(qn > 0, Q / np.maximum(qn, 1e-30), 0).astype(np.float32)
    q2 = (Q * Q).sum(1, keepdims=True)
    best_d = np.full((len(Q), k), np.inf, dtype=np.float32)
    best_i = np.full((len(Q), k), -1, dtype=np.int64)
    for c0 in range(0, db.shape[0], chunk):
        X = db[c0:c0 + chunk, :d_s]
        xn = np.linalg.norm(X, axis=1)
        X = np.where(xn[:, None] > 0, X / np.maximum(xn, 1e-30)[:, None], 0).astype(np.float32)
        x2 = (xn > 0).astype(np.float32)[None, :]
        d = q2 + x2 - 2.0 * (Q @ X.T)
        ids = np.arange(c0, c0 + X.shape[0])[None, :].repeat(len(Q), 0)
        cd = np.concatenate([best_d, d], 1)
        ci = np.concatenate([best_i, ids], 1)
        o = np.argpartition(cd, k - 1, axis=1)[:, :k]
        best_d = np.take_along_axis(cd, o, 1)
        best_i = np.take_along_axis(ci, o, 1)
    return best_i


def ivfopq_bench(args):
    """AdANNS-IVF-OPQ on the NQ-shaped workload: coarse k-means at d_c = 64
    over 4,096 lists, OPQ codes of the d_s prefix, ADC scan of the probed lists
    (optionally an exact FP32 rerank of the top 4k)."""
    import torch
    import paper_2305_19435_gb300 as P
    P.build()
    w = synthdata.WORKLOADS["nq"]
    N = args.n or w.N
    B = args.b or w.B
    t0 = time.time()
    data = synthdata.make("nq", n=N, b=B)
    log(f"data {time.time() - t0:.1f}s")
    db_dev = torch.from_numpy(data["db"]).cuda()
    q = torch.from_numpy(data["queries"]).cuda()
    nlist = 4096 if N >= 4096 * 64 else max(64, N // 512)
    torch.cuda.synchronize()
    tb = time.time()
    g = P.build_ivf(db_dev, 64, nlist, args.niter, min(N, 256 * nlist), args.seed)
    torch.cuda.synchronize()
    ivf_build_s = time.time() - tb
    log(f"ivf build {ivf_build_s:.1f}s")
    S = min(args.gt_queries, B)
    st = torch.cuda.current_stream()
    rows = []
    for d_s, M in ((192, 16), (384, 32), (768, 64)):
        tb = time.time()
        P.build_opq(g, db_dev, d_s, M, 10, 4, 20, min(N, 65536), args.seed + 7)
        torch.cuda.synchronize()
        opq_build_s = time.time() - tb
        gt = exact_topk_prefixnorm(data["db"], data["queries"][:S], d_s, 10)
        # the IVF part alone: exact FP32 distances inside the same probed lists
        ivf_only = {}
        for nprobe in (8, 32, 128):
            fi, _ = P.search_ivf(g, q[:S], 64, d_s, nprobe, 10)
            fi = fi.cpu().numpy()
            ivf_only[nprobe] = float(np.mean([len(set(a.tolist()) & set(b.tolist())) / 10.0
                                              for a, b in zip(fi, gt)]))
        for nprobe in (8, 32, 128):
            for rr in (0, 4 * args.k):
                ids = torch.empty(B, args.k, dtype=torch.int64, device="cuda")
                dd = torch.empty(B, args.k, dtype=torch.float32, device="cuda")

                def step(nprobe=nprobe, rr=rr, ids=ids, dd=dd):
                    P.search_ivfopq(g, q, 64, nprobe, args.k, rerank_k=rr, out=(ids, dd))

                for _ in range(3):
                    step()
                torch.cuda.synchronize()
                ms, launches, prof = timed(P, torch, step, args.steps, st)
                gi = ids[:S].cpu().numpy()
                rec = float(np.mean([len(set(a[:10].tolist()) & set(b.tolist())) / 10.0
                                     for a, b in zip(gi, gt)]))
                row = {"d_s": d_s, "M": M, "nprobe": nprobe, "rerank_k": rr,
                       "qps": B / (ms / 1e3), "ms_per_step": ms,
                       "stages_ms": {k2: v[0] / args.steps for k2, v in prof.items()},
                       "recall10_vs_exact": rec,
                       "ivf_fp32_recall10_vs_exact": ivf_only[nprobe],
                       "opq_build_s": opq_build_s,
                       "gpu_launches": launches}
                rows.append(row)
                log(json.dumps(row))
    g.free()
    print(json.dumps({"ivfopq": rows, "workload": f"NQ-shaped IVF-OPQ: N={N:,} d=768 B={B:,} "
                                                 f"nlist={nlist} d_c=64 k={args.k}",
                      "ivf_build_s": ivf_build_s, "recall_sample": S,
                      "recall_reference": "exact top-10 by L2 on normalised d_s prefixes "
                                          "(numpy over the whole database)"}))


def flat_opq_bench(args):
    """Exhaustive AdANNS-OPQ at byte budgets 8-64 (Sec. 4.2; the exact-search
    OPQ table of the appendix): OPQ on the d_s prefix of the ImageNet-shaped
    database, ADC over all N codes for every query (a one-list index), recall@10
    against exact search at the same d_s."""
    import torch
    import paper_2305_19435_gb300 as P
    P.build()
    w = synthdata.WORKLOADS["imagenet"]
    N = args.n or w.N
    B = args.b or 10_000
    data = synthdata.make("imagenet", n=N, b=B)
    db_dev = torch.from_numpy(data["db"]).cuda()
    q = torch.from_numpy(data["queries"]).cuda()
    g = P.flat_index(db_dev)
    S = min(args.gt_queries, B)
    st = torch.cuda.current_stream()
    rows = []
    for d_s in (128, 512, 2048):
        gt = exact_topk_prefixnorm(data["db"], data["queries"][:S], d_s, 10)
        for M, opq_iters in ((8, 5), (16, 5), (32, 5), (64, 5), (32, 0)):
            if d_s // M > 64:  # the builder's sub-vector limit
                continue
            tb = time.time()
            P.build_opq(g, db_dev, d_s, M, opq_iters, 4, 20, min(N, 65536), args.seed + 7)
            torch.cuda.synchronize()
            build_s = time.time() - tb
            ids = torch.empty(B, 10, dtype=torch.int64, device="cuda")
            dd = torch.empty(B, 10, dtype=torch.float32, device="cuda")

            def step(ids=ids, dd=dd):
                P.search_ivfopq(g, q, 8, 1, 10, out=(ids, dd))

            for _ in range(2):
                step()
            torch.cuda.synchronize()
            ms, launches, prof = timed(P, torch, step, args.steps, st)
            gi = ids[:S].cpu().numpy()
            rec = float(np.mean([len(set(a.tolist()) & set(b.tolist())) / 10.0
                                 for a, b in zip(gi, gt)]))
            adc_ms = prof.get("adc", (0.0, 1))[0] / args.steps
            row = {"d_s": d_s, "bytes": M, "rotation": "OPQ" if opq_iters else "PQ (identity)",
                   "qps": B / (ms / 1e3), "ms_per_step": ms,
                   "lookups_per_s": B * N * M / (adc_ms / 1e3) if adc_ms else None,
                   "stages_ms": {k2: v[0] / args.steps for k2, v in prof.items()},
                   "recall10_vs_exact": rec, "build_s": build_s, "gpu_launches": launches}
            rows.append(row)
            log(json.dumps(row))
    g.free()
    print(json.dumps({"flat_opq": rows,
                      "workload": f"exhaustive AdANNS-OPQ, ImageNet-shaped: N={N:,} d=2048 B={B:,} "
                                  f"k=10 (one list, every code scanned per query)",
                      "recall_sample": S,
                      "recall_reference": "exact top-10 by L2 on normalised d_s prefixes "
                                          "(numpy over the whole database)"}))


def graph_bench(args):
    """AdANNS-DiskANN on the ImageNet-shaped workload (Sec. 4.3): a graph formed
    at the low-d MR (d_g = 16), best-first shortlist at d_g, exact rerank with
    the high-d MR; QPS and recall@10 against exact search at the rerank's d_s."""
    import torch
    import paper_2305_19435_gb300 as P
    P.build()
    w = synthdata.WORKLOADS["imagenet"]
    N = args.n or w.N
    B = args.b or 10_000
    data = synthdata.make("imagenet", n=N, b=B)
    db_dev = torch.from_numpy(data["db"]).cuda()
    q = torch.from_numpy(data["queries"]).cuda()
    torch.cuda.synchronize()
    tb = time.time()
    g = P.graph_build(db_dev, 16, 64, 32, 1.2)
    torch.cuda.synchronize()
    build_s = time.time() - tb
    log(f"graph build {build_s:.1f}s")
    del db_dev
    torch.cuda.empty_cache()
    S = min(args.gt_queries, B)
    st = torch.cuda.current_stream()
    rows = []
    for d_s in (512, 2048):
        gt = exact_topk_prefixnorm(data["db"], data["queries"][:S], d_s, 10)
        for L, kr in ((32, 32), (64, 40), (128, 100), (256, 200)):
            ids = torch.empty(B, 10, dtype=torch.int64, device="cuda")

            def step(L=L, kr=kr):
                P.graph_search(g, q, L, d_s, 10, kr)

            for _ in range(2):
                step()
            torch.cuda.synchronize()
            ms, launches, prof = timed(P, torch, step, args.steps, st)
            gi, _ = P.graph_search(g, q[:S], L, d_s, 10, kr)
            gi = gi.cpu().numpy()
            rec = float(np.mean([len(set(a.tolist()) & set(b.tolist())) / 10.0
                                 for a, b in zip(gi, gt)]))
            row = {"d_g": 16, "d_s": d_s, "L": L, "rerank_k": kr, "qps": B / (ms / 1e3),
                   "ms_per_step": ms, "stages_ms": {k2: v[0] / args.steps for k2, v in prof.items()},
                   "recall10_vs_exact": rec, "gpu_launches": launches}
            rows.append(row)
            log(json.dumps(row))
    g.free()
    print(json.dumps({"graph": rows, "build_s": build_s,
                      "workload": f"AdANNS-DiskANN, ImageNet-shaped: N={N:,} d=2048 B={B:,} k=10, "
                                  "graph at d_g=16 (K=64 candidates, R=32, alpha=1.2)",
                      "recall_sample": S,
                      "recall_reference": "exact top-10 by L2 on normalised d_s prefixes "
                                          "(numpy over the whole database)"}))


def main():
    args = parse()
    if getattr(args, "graph", False):
        graph_bench(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.accuracy_sweep:
        accuracy_sweep(args)
        return
    if args.ivfopq:
        ivfopq_bench(args)
        return
    if args.flat_opq:
        flat_opq_bench(args)
        return
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        if world > 1:
            t = torch.tensor([v], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            v = float(t.item())
        return v

    import paper_2305_19435_gb300 as P
    if rank == 0:
        P.build()
    barrier()
    P.build()
    props = torch.cuda.get_device_properties(local)
    options = {}
    for kv in args.option:
        name, val = kv.split("=", 1)
        P.set_option(getattr(P, "OPT_" + name.upper()), int(val))
        options[name.upper()] = int(val)

    w = synthdata.WORKLOADS[args.workload]
    N = args.n or w.N
    B = args.b or w.B
    t0 = time.time()
    data = synthdata.make(args.workload, n=N, b=B)
    log(f"data {time.time() - t0:.1f}s")
    if rank == 0:
        oidx = oracle_index(data, args, N)
    barrier()
    if rank != 0:
        oidx = oracle_index(data, args, N)
    log(f"oracle index ready ({oidx.get('build_s', 0):.1f}s build)")
    modes = [args.mode] + [m for m in args.compare if m != args.mode]
    storage = 1
    for m in modes:
        storage |= MODES[m][0]
    db_dev = torch.from_numpy(data["db"]).cuda()
    tb = time.time()
    idx = P.index_create(db_dev, torch.from_numpy(oidx["centroids"]).cuda(),
                         torch.from_numpy(oidx["assign"].astype(np.int32)).cuda(), storage=storage)
    torch.cuda.synchronize()
    layout_s = time.time() - tb
    gpu_build_s = None
    if not args.skip_gpu_build:
        tb = time.time()
        gidx = P.build_ivf(db_dev, args.d_c, args.nlist, args.niter, min(N, 256 * args.nlist),
                           args.seed)
        torch.cuda.synchronize()
        gpu_build_s = time.time() - tb
        gidx.free()
    big = None
    if not args.no_largest:
        a64 = argparse.Namespace(**{**vars(args), "d_c": 64})
        oidx64 = oracle_index(data, a64, N)
        idx64 = P.index_create(db_dev, torch.from_numpy(oidx64["centroids"]).cuda(),
                               torch.from_numpy(oidx64["assign"].astype(np.int32)).cuda(),
                               storage=storage)
        big = (idx64, oidx64)
    serving = None
    if args.serve_seconds > 0 and world == 1:
        serving = serving_phase(P, torch, data, db_dev, args, B)
        log(f"serving {serving}")
    del db_dev
    torch.cuda.empty_cache()

    qh = torch.from_numpy(data["queries"]).pin_memory()
    q = qh.cuda()
    st = torch.cuda.current_stream()
    results = {}
    for mode in modes:
        ids = torch.empty(B, args.k, dtype=torch.int64, device="cuda")
        dd = torch.empty(B, args.k, dtype=torch.float32, device="cuda")
        code, rr = MODES[mode][0], mode_rerank(mode, args.k)

        def step(ids=ids, dd=dd, code=code, rr=rr):
            P.search_ivf(idx, q, args.d_c, args.d_s, args.nprobe, args.k, storage=code,
                         rerank_k=rr, out=(ids, dd))

        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        barrier()
        if mode == args.mode:
            with Clocks(local) as clk:
                ms, launches, prof = timed(P, torch, step, args.steps, st)
            clocks = clk.summary()
        else:
            ms, launches, prof = timed(P, torch, step, args.steps, st)
        barrier()
        ms = max_over_ranks(ms)
        results[mode] = {"ms": ms, "qps": world * B / (ms / 1000.0), "launches": launches,
                         "stages_ms": {k2: v[0] / args.steps for k2, v in prof.items()},
                         "counters": dict(timed.counters),
                         "ids": ids, "step": step}
    idx.status()  # raises if a device-side check or a pipeline wait failed during the runs
    main_r = results[args.mode]
    # the headline step replayed from a captured CUDA graph
    code, rr = MODES[args.mode][0], mode_rerank(args.mode, args.k)
    plan = P.Plan(idx, q, args.d_c, args.d_s, args.nprobe, args.k, storage=code, rerank_k=rr)
    for _ in range(3):
        plan.launch()
    g_ms, _, _ = timed(P, torch, plan.launch, args.steps, st)
    plan.free()
    graph_ms = max_over_ranks(g_ms)

    # end to end through the public API: pinned host queries in, results out
    code, rr = MODES[args.mode][0], mode_rerank(args.mode, args.k)
    ih = torch.empty(B, args.k, dtype=torch.int64).pin_memory()
    dh = torch.empty(B, args.k, dtype=torch.float32).pin_memory()
    ids_e = torch.empty(B, args.k, dtype=torch.int64, device="cuda")
    dd_e = torch.empty(B, args.k, dtype=torch.float32, device="cuda")

    def e2e_serial_step():
        # copy in, search, copy out, one after the other on one stream
        qd = qh.cuda(non_blocking=True)
        P.search_ivf(idx, qd, args.d_c, args.d_s, args.nprobe, args.k, storage=code, rerank_k=rr,
                     out=(ids_e, dd_e))
        ih.copy_(ids_e, non_blocking=True)
        dh.copy_(dd_e, non_blocking=True)

    def e2e_step():
        # the host-buffer call: slices whose copies overlap the neighbouring searches
        P.search_ivf_host(idx, qh, args.d_c, args.d_s, args.nprobe, args.k, storage=code,
                          rerank_k=rr, out=(ih, dh))

    def time_e2e(step):
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            step()
        e1.record(st)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / args.steps)

    e2e_serial_ms = time_e2e(e2e_serial_step)
    e2e_ms = time_e2e(e2e_step)

    # work accounting from the probe lists of the timed batch
    _, _, probes = P.search_ivf(idx, q, args.d_c, args.d_s, args.nprobe, args.k, return_probes=True)
    probes = probes.cpu().numpy()
    sizes = np.diff(oidx["list_off"])
    pairs = int(sizes[probes].sum())
    probed = np.unique(probes)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_count = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    ffma_peak = sm_count * 128 * 2 * sm_max * 1e6 / 1e12
    wl_key = (f"{args.workload}-N{N}-B{B}-nlist{args.nlist}-dc{args.d_c}-ds{args.d_s}"
              f"-np{args.nprobe}-k{args.k}")

    def traffic(mode, kern):
        return traffic_record({"mma": "mma_scan_kernel", "rerank": "rerank_chunks_kernel"}[kern],
                              mode, wl_key)

    rooflines = {}
    for mode, r in results.items():
        sm = r["stages_ms"]
        if mode == "f32":
            t = sm.get("scan", 0.0)
            ach = 4.0 * pairs * args.d_s / (t / 1e3) / 1e12
            rooflines[mode] = {"kernel": "scan_f32_kernel (list scan)", "bound": "alu",
                               "achieved": ach, "peak": ffma_peak, "unit": "TFLOP/s",
                               "frac": ach / ffma_peak,
                               "traffic": traffic_record("scan_f32_kernel", "f32", wl_key),
                               "kernel_ms": t,
                               "peak_source": f"derived FP32 FFMA peak: {sm_count} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz"}
        else:
            t = sm.get("mma", 0.0)
            epb = 64 if mode == "bf16" else 128
            dpad = (args.d_s + epb - 1) // epb * epb
            ach = 2.0 * pairs * dpad / (t / 1e3) / 1e12
            peak = bf16_peak * (2.0 if mode == "fp8" else 1.0)
            rooflines[mode] = {"kernel": "mma_scan_kernel (tensor-core list scan)", "bound": "tensor",
                               "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                               "traffic": traffic(mode, "mma"), "kernel_ms": t,
                               "peak_source": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"
                               + (" x 2 (nominal fp8/bf16 ratio)" if mode == "fp8" else "")}
            # exact rerank: every database row it re-scores and every query row is
            # needed once (N + B rows of d_s FP32 bound the unique bytes); each
            # re-scored pair also gathers one query row (from L2)
            rr_t = sm.get("rr_pairs", sm.get("rerank", 0.0))
            rr_pairs = r["counters"].get("rerank_pairs", 0)
            rr_bytes = (N + B) * args.d_s * 4
            rooflines[mode]["rerank"] = {
                "kernel": "rerank_chunks_kernel (exact FP32 rerank of the pruned shortlist)",
                "bound": "hbm", "achieved": rr_bytes / (rr_t / 1e3) / 1e9 if rr_t else None,
                "peak": hbm_peak, "unit": "GB/s", "kernel_ms": rr_t,
                "traffic": traffic(mode, "rerank"),
                "pairs": rr_pairs, "shortlist_slots": r["counters"].get("shortlist_slots", 0),
                "gathered_query_gb": rr_pairs * args.d_s * 4 / 1e9,
                "note": "algorithmic bytes = (N + B) x d_s x 4: each database and query row "
                        "once; the query rows are gathered once per pair from L2"}
    scan_hbm = scan_hbm_phase(P, torch, idx, q, oidx, args, hbm_peak, list(results))
    largest = None
    if big is not None:
        largest = largest_point_phase(P, torch, data, big[0], big[1], q, args, N, B,
                                      list(results), peaks)
        big[0].status()
        big[0].free()
    main_roof = dict(rooflines[args.mode])
    # the dominant kernel of the step (largest stage) carries the headline roofline
    main_stages = main_r["stages_ms"]
    kern_stages = {k2: v for k2, v in main_stages.items() if k2 not in ("rerank", "_host_us")}
    dom = max(kern_stages, key=kern_stages.get) if kern_stages else None
    if args.mode != "f32" and dom == "rr_pairs":
        rrd = main_roof.pop("rerank")
        main_roof = {**rrd, "frac": (rrd["achieved"] or 0) / hbm_peak,
                     "peak_source": "measured STREAM-style copy (MEASURED_PEAKS.json)",
                     "mma": {k2: v for k2, v in rooflines[args.mode].items() if k2 != "rerank"}}

    cfg = workload_config(args, N, B)
    if options:
        cfg["options"] = options
    out = {"metric": "QPS at recall@10 vs oracle", "value": main_r["qps"], "unit": "queries/s",
           "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
           "ms_per_step": main_r["ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": {"f32": "f32", "bf16": "bf16", "fp8": "fp8e4m3"}[args.mode],
           "data": "synthetic (seeded Matryoshka-like Gaussian mixture)", "config": cfg,
           "clocks": clocks, "gpu_launches": int(main_r["launches"]), "roofline": main_roof,
           "stages_ms": main_r["stages_ms"],
           "modes": {m: {"qps": r["qps"], "ms_per_step": r["ms"], "stages_ms": r["stages_ms"],
                         "work_per_step": r["counters"], "roofline": rooflines[m]}
                     for m, r in results.items()},
           "graph_replay": {"ms_per_step": graph_ms, "qps": world * B / (graph_ms / 1000.0)},
           "serving": serving,
           "scan_hbm_regime": scan_hbm,
           "largest_point": largest,
           "p50_ms": (serving or {}).get("sizes_1_4096", {}).get(args.mode, {}).get("p50_ms"),
           "p99_ms": (serving or {}).get("sizes_1_4096", {}).get(args.mode, {}).get("p99_ms"),
           "gpu_build_s": gpu_build_s, "index_layout_s": layout_s, "pairs_per_step": pairs,
           "unique_lists_per_step": int(len(probed)),
           "e2e": {"value": world * B / (e2e_ms / 1000.0), "unit": "queries/s",
                   # the prefix of each query row the search reads from host memory
                   "h2d_bytes_per_step": int(B * max(args.d_c, args.d_s) * 4),
                   "d2h_bytes_per_step": int(ih.numel() * 8 + dh.numel() * 4),
                   "call": "adanns_search_ivf_host on page-locked host buffers: the GPU reads "
                           "each query's first max(d_c, d_s) coordinates and writes the results "
                           "in place over the host link, no staging copy",
                   "serial_copies_qps": world * B / (e2e_serial_ms / 1000.0),
                   "serial_copies_h2d_bytes_per_step": int(qh.numel() * 4)}}

    if rank == 0 and not args.no_cpu:
        import oracle
        S = oracle_sample_size(oidx, data, args, args.cpu_seconds)
        t = time.time()
        ref = oracle.search_ivf(data["db"], oidx, data["queries"][:S], args.d_c, args.d_s,
                                args.nprobe, args.k)
        el = time.time() - t
        for mode, r in results.items():
            r["step"]()
            torch.cuda.synchronize()
            gi = r["ids"][:S].cpu().numpy()
            rec = float(np.mean([len(set(a[:10].tolist()) & set(b[:10].tolist())) / 10.0
                                 for a, b in zip(gi, ref["ids"])]))
            out["modes"][mode]["recall_at_10_vs_oracle"] = rec
        out["recall_at_10_vs_oracle"] = out["modes"][args.mode]["recall_at_10_vs_oracle"]
        out["recall_sample"] = S
        out["cpu_baseline"] = {"value": S / el, "unit": "queries/s", "cores": os.cpu_count(),
                               "kind": "oracle",
                               "sample": f"first {S} of {B} queries, same index and config, "
                                         f"FP64 oracle with {os.cpu_count()} threads"}
    if rank == 0:
        print(json.dumps(out))
    idx.free()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
