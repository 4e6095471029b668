"""Benchmark of the APRIL intermediate filter on GB300.

One step = one pass of the filter (Algorithm 2 on every candidate pair) over
the paper-scale workload: 200k + 200k synthetic star polygons on a 2^16 grid,
~2.7M MBR-join candidate pairs (seeded; the synthetic stand-in for the
paper's TIGER/OSM joins).  The A/F sets are built and uploaded once (the
paper precomputes approximations); the timed region runs the filter kernels
on pairs and sets already resident in HBM.  L2 is flushed between timed
steps.

Output: one JSON line (rank 0).  `value` is pairs/s of the selected mode
(default: batched); the line also carries the plain one-pair-per-thread
kernel's pairs/s on the same pairs, the end-to-end number through the
host-buffer entry point, the HBM roofline of the dominant kernel, and the
oracle's CPU throughput on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode batched|warp|plain]
  python bench.py --impl reference ...   # the oracle (CPU) on the same workload
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "APRIL filter pairs/s & HBM GB/s (batched vs plain); serving p50/p99 latency"
CONFIG_NAMES = {1: "tiny-plain-1k", 2: "paper-scale-200k", 3: "skewed-pareto-200k"}
PAIR_ID_BYTES = 8       # r and s ids
DESC_BYTES = 32         # two 16-byte object descriptors
VERDICT_BYTES = 1
IV_BYTES = 8            # one interval = two uint32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4])
    ap.add_argument("--mode", default="batched", choices=["batched", "warp", "plain", "packed"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tuning (profiling runs)")
    ap.add_argument("--tune", default=None,
                    help="T,G,W,CW[,JO]: fixed batched tuning instead of the autotuner (JO: join order 0 or 1)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--serving-requests", type=int, default=120)
    ap.add_argument("--no-selection", action="store_true", help="skip the selection-query measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the within / mixed-granularity measurement")
    ap.add_argument("--no-construction", action="store_true", help="skip the GPU construction measurement")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha() -> str:
    """Hash of the kernel sources a profile was taken on."""
    h = hashlib.sha256()
    for f in ("filter.cu", "join_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2307_01716_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def kernel_traffic(kernel: str, workload: str, tune):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources with the same tuning."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    sha = kernel_source_sha()
    key = None if tune is None else [tune["cta_threshold"], tune["group_lanes"], tune["group_window"],
                                     tune["cta_window"], tune.get("join_order", 0)]
    for e in json.load(open(p)):
        if (e.get("kernel") == kernel and e.get("workload") == workload and e.get("src_sha") == sha
                and e.get("tune") == key):
            return e.get("dram_bytes_per_launch")
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"april_clocks_{os.getpid()}.csv")

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, device_index: int = 0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_fn(w):
    """f(pr, ps) -> the oracle's verdicts for workload w (partitioned
    workloads: each pair on its routed partition's grid, the grids computed
    once)."""
    import oracle
    if not w.partitions:
        g = oracle.Grid(w.order)
        return lambda pr, ps: oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, pr, ps, g)
    grids = oracle.partition_areas(w.R.mbr, w.S.mbr, w.partitions, w.order)

    def f(pr, ps):
        part = oracle.route_pairs(w.R.mbr, w.S.mbr, pr, ps, w.partitions)
        out = np.zeros(len(pr), dtype=np.uint8)
        for p in np.unique(part):
            sel = np.nonzero(part == p)[0]
            out[sel] = oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, pr[sel], ps[sel], grids[int(p)])
        return out
    return f


def cpu_baseline(w, seconds: float, seed: int = 1234):
    """The oracle, as it stands, on a bounded random sample of the pairs."""
    f = oracle_fn(w)
    rng = np.random.default_rng(seed)
    done = 0
    t0 = time.perf_counter()
    batch = 200
    while time.perf_counter() - t0 < seconds:
        idx = np.sort(rng.choice(len(w.pr), batch, replace=False))
        f(w.pr[idx], w.ps[idx])
        done += batch
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} random pairs of the {len(w.pr)} (seeded), cell-set oracle, single thread, "
                      f"{dt:.1f} s"}


def _event_times(torch, stream, flush, run, steps, warmup):
    """CUDA-event times (ms) of `run` on `stream`, L2 flushed before each step."""
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record(stream)
        run()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def selection_bench(ctx, A, torch, dev, stream, flush, R, dR, steps, warmup):
    """Selection queries (Sec. 4.3.1): 1000 county-like query polygons over the
    200k data polygons of config 2 (R side), the data lists and the MBR index
    resident.  Timed: april_select (MBR candidates on the GPU, the count read
    back, the batched filter) with the query lists already on the device; and
    end to end from host query polygons (host construction of the query
    lists, upload, april_select, verdicts back to the host)."""
    from synth import selection
    s = selection.make(1.0, 1000)
    g = A.global_grid(s.order)
    if R is None:
        R = A.april_build_sets(s.R.xy, s.R.off, g)
        dR = A.april_upload(R, dev)
    dI = A.april_index_upload(A.april_index_build(R), dev)
    t0 = time.perf_counter()
    Q = A.april_build_sets(s.Q.xy, s.Q.off, g)
    build_s = time.perf_counter() - t0
    dQ = A.april_upload(Q, dev)
    off = torch.empty(s.Q.n + 1, dtype=torch.int32, device=dev)
    sc0 = torch.empty(ctx.select_scratch_bytes(0), dtype=torch.uint8, device=dev)
    n = ctx.april_select(dI, dR, dQ, 0, None, None, None, off, sc0, stream)
    d_r = torch.empty(n, dtype=torch.int32, device=dev)
    d_q = torch.empty(n, dtype=torch.int32, device=dev)
    d_v = torch.empty(n, dtype=torch.uint8, device=dev)
    scratch = torch.empty(ctx.select_scratch_bytes(n), dtype=torch.uint8, device=dev)

    # the filter's tuning for these pairs (small data polygons against large
    # queries), picked by the autotuner on the candidate pairs
    ctx.april_select(dI, dR, dQ, n, d_r, d_q, d_v, off, scratch, stream)
    stream.synchronize()
    sc_tune = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device=dev)
    tuned = ctx.april_autotune(dR, dQ, d_r, d_q, n, d_v, sc_tune, stream).as_dict()
    del sc_tune

    def run():
        ctx.april_select(dI, dR, dQ, n, d_r, d_q, d_v, off, scratch, stream)
    t = _event_times(torch, stream, flush, run, steps, warmup)
    ctx.april_sync_status(stream)
    r = d_r.cpu().numpy().view(np.uint32)
    q = d_q.cpu().numpy().view(np.uint32)
    v = d_v.cpu().numpy()
    t0 = time.perf_counter()
    hv, _ = A.april_host_filter(R, Q, r, q)
    host_all = time.perf_counter() - t0
    k1 = min(n, 20_000)
    t0 = time.perf_counter()
    A.april_host_filter(R, Q, r[:k1], q[:k1], n_threads=1)
    host_one = time.perf_counter() - t0
    if not np.array_equal(v, hv):
        raise SystemExit("selection verdicts differ from Algorithm 2 on the host")
    # end to end: host polygons in, host verdicts out
    e2e = []
    h_v = torch.empty(n, dtype=torch.uint8).pin_memory()
    for k in range(max(2, steps // 3)):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Qk = A.april_build_sets(s.Q.xy, s.Q.off, g)
        dQk = A.april_upload(Qk, dev, stream)
        ctx.april_select(dI, dR, dQk, n, d_r, d_q, d_v, off, scratch, stream)
        h_v.copy_(d_v, non_blocking=True)
        stream.synchronize()
        e2e.append(time.perf_counter() - t0)
    # end to end with the query lists built on the GPU: pinned host polygons
    # copied in, construction, selection, verdicts back
    h_xy = torch.from_numpy(np.ascontiguousarray(s.Q.xy, dtype=np.int32)).pin_memory()
    h_off = torch.from_numpy(np.ascontiguousarray(s.Q.off, dtype=np.int64)).pin_memory()
    d_xy = torch.empty_like(h_xy, device=dev)
    d_off = torch.empty_like(h_off, device=dev)
    d_xy.copy_(h_xy)
    d_off.copy_(h_off)
    _, binfo = ctx.april_build_sets_device(d_xy, d_off, g, stream=stream)
    bwork = torch.empty(int(binfo.work_bytes), dtype=torch.uint8, device=dev)
    bimage = torch.empty(int(binfo.image_bytes), dtype=torch.uint8, device=dev)
    e2e_dev = []
    for k in range(max(3, steps)):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_xy.copy_(h_xy, non_blocking=True)
        d_off.copy_(h_off, non_blocking=True)
        dQk, _ = ctx.april_build_sets_device(d_xy, d_off, g, work=bwork, image=bimage, stream=stream)
        ctx.april_select(dI, dR, dQk, n, d_r, d_q, d_v, off, scratch, stream)
        h_v.copy_(d_v, non_blocking=True)
        stream.synchronize()
        e2e_dev.append(time.perf_counter() - t0)
    if not np.array_equal(h_v.numpy(), hv):
        raise SystemExit("selection with GPU-built query lists differs")
    ms = statistics.mean(t)
    e2e_dev_ms = statistics.mean(e2e_dev[1:]) * 1e3
    return {"workload": s.name, "queries": int(s.Q.n), "candidate_pairs": int(n), "ms_per_batch": ms,
            "filter_tune": tuned,
            "e2e_gpu_construction": {"ms_per_batch": e2e_dev_ms, "queries_per_s": s.Q.n / (e2e_dev_ms * 1e-3),
                                     "h2d_bytes": int(h_xy.numel() * 4 + h_off.numel() * 8), "d2h_bytes": int(n),
                                     "path": "pinned query polygons to the GPU + april_build_sets_device + "
                                             "april_select + verdicts to host"},
            "queries_per_s": s.Q.n / (ms * 1e-3), "pairs_per_s": n / (ms * 1e-3),
            "query_list_build_ms_host": build_s * 1e3,
            "e2e": {"ms_per_batch": statistics.mean(e2e) * 1e3,
                    "queries_per_s": s.Q.n / statistics.mean(e2e),
                    "path": "host query construction + upload + april_select + verdicts to host"},
            "cpu_alg2": {"threads_1_pairs_per_s": k1 / host_one, "threads_all_pairs_per_s": n / host_all,
                         "threads": os.cpu_count()},
            "verdict_mix": (np.bincount(v, minlength=3)[:3] / max(n, 1)).round(4).tolist()}


def construction_bench(ctx, A, torch, dev, stream, flush, w, S, dS, host_v, steps, warmup):
    """Construction of the R side (200k polygons of config 2) on the GPU
    (april_build_sets_device, polygons already in device memory) against the
    host builder on all host cores; parity through the filter: the
    GPU-built R with the host-built S gives the same verdicts."""
    g = A.global_grid(w.order)
    d_xy = torch.from_numpy(np.ascontiguousarray(w.R.xy, dtype=np.int32)).to(dev)
    d_off = torch.from_numpy(np.ascontiguousarray(w.R.off, dtype=np.int64)).to(dev)
    dR, info = ctx.april_build_sets_device(d_xy, d_off, g, stream=stream)
    work = torch.empty(int(info.work_bytes), dtype=torch.uint8, device=dev)
    image = dR.buf

    def run():
        ctx.april_build_sets_device(d_xy, d_off, g, work=work, image=image, stream=stream)
    t = _event_times(torch, stream, flush, run, steps, warmup)
    n = len(w.pr)
    d_r = torch.from_numpy(w.pr.view(np.int32)).to(dev)
    d_s = torch.from_numpy(w.ps.view(np.int32)).to(dev)
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device=dev)
    dR2, _ = ctx.april_build_sets_device(d_xy, d_off, g, work=work, image=image, stream=stream)
    ctx.april_filter_pairs(dR2, dS, d_r, d_s, n, out, A.MODE_BATCHED, scratch, stream)
    ctx.april_sync_status(stream)
    if not np.array_equal(out.cpu().numpy(), host_v):
        raise SystemExit("GPU-built sets filter to other verdicts")
    t0 = time.perf_counter()
    A.april_build_sets(w.R.xy, w.R.off, g)
    host_s = time.perf_counter() - t0
    ms = statistics.mean(t)
    return {"polygons": int(w.R.n), "ms_gpu": ms, "polygons_per_s_gpu": w.R.n / (ms * 1e-3),
            "touched_cells": int(info.touched_cells), "work_bytes": int(info.work_bytes),
            "image_bytes": int(info.image_bytes), "ms_host_all_cores": host_s * 1e3, "host_threads": os.cpu_count(),
            "speedup": host_s * 1e3 / ms,
            "timed": "april_build_sets_device (count, one size read-back, build), polygons resident on the GPU"}


def variants_bench(ctx, A, torch, dev, stream, flush, w, R, S, dR, dS, steps, warmup):
    """The filter variants on the same candidate pairs: within (Sec. 4.3.2,
    both sets at N) and different granularity (Sec. 5.3, S at N-2)."""
    n = len(w.pr)
    d_r = torch.from_numpy(w.pr.view(np.int32)).to(dev)
    d_s = torch.from_numpy(w.ps.view(np.int32)).to(dev)
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    scratch = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, n), dtype=torch.uint8, device=dev)
    S2 = A.april_build_sets(w.S.xy, w.S.off, A.global_grid(w.order - 2))
    dS2 = A.april_upload(S2, dev)
    res = {}
    for name, sets, dsets, pred in (("within", S, dS, A.PREDICATE_WITHIN),
                                    (f"intersects_r{w.order}_s{w.order - 2}", S2, dS2, A.PREDICATE_INTERSECTS)):
        def run():
            ctx.april_filter_pairs_ex(dR, dsets, d_r, d_s, n, out, pred, scratch, stream)
        t = _event_times(torch, stream, flush, run, steps, warmup)
        ctx.april_sync_status(stream)
        hv, _ = A.april_host_filter_ex(R, sets, w.pr, w.ps, pred)
        if not np.array_equal(out.cpu().numpy(), hv):
            raise SystemExit(f"variant {name}: verdicts differ from the host execution")
        ms = statistics.mean(t)
        res[name] = {"pairs_per_s": n / (ms * 1e-3), "ms_per_step": ms,
                     "verdict_mix": (np.bincount(hv, minlength=3)[:3] / n).round(4).tolist()}
    return res


def serving_bench(ctx_cls, A, torch, dev, n_requests: int, budget_gb: float = 40.0):
    """Config 5: 300k + 300k polygons (config-3 generator, 2^16 grid) resident
    in HBM; requests are query windows of 1k-2M candidate pairs (log-uniform)
    arriving as a Poisson stream.  Continuous batching (8 stream slots, a 40 GB
    arena) against one request per launch, at 50% and 80% of the measured
    one-request-per-launch capacity."""
    from synth import configs, serving
    w = configs.make(5)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    dR, dS = A.april_upload(R, dev), A.april_upload(S, dev)
    ctx = ctx_cls(dev.index or 0)
    maker = serving.RequestMaker(w.R.mbr, w.S.mbr, w.pr, w.ps)
    reqs = maker.requests(seed=11, count=n_requests, rate=0.0)
    bufs = [(torch.from_numpy(q.pr.view(np.int32).copy()).pin_memory(),
             torch.from_numpy(q.ps.view(np.int32).copy()).pin_memory(),
             torch.empty(len(q.pr), dtype=torch.uint8).pin_memory()) for q in reqs]
    sizes = np.array([len(q.pr) for q in reqs])
    arena = torch.empty(int(budget_gb * (1 << 30)), dtype=torch.uint8, device=dev)

    def run(max_inflight, arrivals):
        srv = A.Server(ctx, dR, dS, arena, max_inflight)
        try:
            for b in bufs[:4]:  # warm-up
                srv.april_wait(srv.april_submit(*b))
            t0 = time.perf_counter()
            tickets = []
            for b, at in zip(bufs, arrivals):
                while time.perf_counter() - t0 < at:
                    pass
                tickets.append(srv.april_submit(*b))
            stats = [srv.april_wait(t, 600000) for t in tickets]
            info = srv.info()
        finally:
            srv.close()
        lat = np.array([(st.done_ns - st.submit_ns) / 1e6 for st in stats])
        span = (max(st.done_ns for st in stats) - min(st.submit_ns for st in stats)) / 1e9
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "pairs_per_s": float(sizes.sum() / span),
                "requests_per_s": float(len(reqs) / span), "max_concurrent": int(info.max_concurrent),
                "arena_peak_gb": info.arena_peak_bytes / (1 << 30)}

    # capacity: all requests offered at once, one per launch
    cap = run(1, np.zeros(len(reqs)))
    capacity = cap["requests_per_s"]
    out = {"workload": w.name, "candidates": int(len(w.pr)), "requests": len(reqs),
           "request_pairs_mean": float(sizes.mean()), "request_pairs_p50": float(np.median(sizes)),
           "budget_gb": budget_gb, "capacity_one_per_launch_req_s": capacity, "rates": {}}
    rng = np.random.default_rng(77)
    gaps = rng.exponential(1.0, len(reqs))
    for frac in (0.5, 0.8):
        lam = frac * capacity
        arrivals = np.cumsum(gaps) / lam
        out["rates"][f"{frac:.0%}"] = {"rate_req_s": lam, "continuous": run(8, arrivals),
                                       "one_per_launch": run(1, arrivals)}
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from synth import configs
    w = configs.make(args.config)
    f = oracle_fn(w)
    rng = np.random.default_rng(99)
    per_step = 300
    times = []
    for step in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(len(w.pr), per_step, replace=False))
        t0 = time.perf_counter()
        f(w.pr[idx], w.ps[idx])
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = per_step * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": w.name, "pairs": int(len(w.pr)),
                                              "sample_pairs_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} random pairs per step of {len(w.pr)}"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from synth import configs
    from paper_2307_01716_gb300 import april as A

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = configs.make(args.config)
    if w.partitions:
        R, S = A.april_build_partitioned_sets(w.R.xy, w.R.off, w.S.xy, w.S.off, w.partitions, w.order)
    else:
        grid = A.global_grid(w.order)
        R = A.april_build_sets(w.R.xy, w.R.off, grid)
        S = A.april_build_sets(w.S.xy, w.S.off, grid)
    if args.mode == "packed" or w.partitions:
        R.compress()
        S.compress()
    dR, dS = A.april_upload(R, dev), A.april_upload(S, dev)
    ctx = A.Context(local)
    n = len(w.pr)
    d_r = torch.from_numpy(w.pr.view(np.int32)).to(dev)
    d_s = torch.from_numpy(w.ps.view(np.int32)).to(dev)
    out = torch.empty(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    # algorithmic bytes: the intervals sequential Algorithm 2 reads, per pair;
    # the same host run (all cores) is the CPU Algorithm 2 leg
    t0 = time.perf_counter()
    host_v, consumed = A.april_host_filter(R, S, w.pr, w.ps)
    host_all_s = time.perf_counter() - t0
    b_seq = float(IV_BYTES * consumed.sum() + n * (PAIR_ID_BYTES + DESC_BYTES + VERDICT_BYTES))
    # the kernels start every join at the first interval that can meet the
    # other list; the bytes they must read are those of that reading
    host_v2, consumed2 = A.april_host_filter(R, S, w.pr, w.ps, searched=True)
    if not np.array_equal(host_v, host_v2):
        raise SystemExit("the searched host execution disagrees with Algorithm 2")
    b_alg = float(IV_BYTES * consumed2.sum() + n * (PAIR_ID_BYTES + DESC_BYTES + VERDICT_BYTES))
    b_full = None
    if not w.partitions:  # no early exit: AA, AF and FA read every list in full
        a_r, f_r = R.lengths()
        a_s, f_s = S.lengths()
        iv = (2 * a_r[w.pr].astype(np.uint64) + 2 * a_s[w.ps] + f_r[w.pr] + f_s[w.ps]).sum()
        b_full = float(IV_BYTES * iv + n * (PAIR_ID_BYTES + DESC_BYTES + VERDICT_BYTES))
    k1 = min(n, 100_000)
    t0 = time.perf_counter()
    A.april_host_filter(R, S, w.pr[:k1], w.ps[:k1], n_threads=1)
    host_one_s = time.perf_counter() - t0
    cpu_alg2 = {"kind": "Algorithm 2 merge joins (AA, AF, FA, early exit) over the same lists, host C++",
                "threads_1": {"pairs_per_s": k1 / host_one_s, "sample": f"first {k1} pairs"},
                "threads_all": {"pairs_per_s": n / host_all_s, "threads": os.cpu_count(), "sample": "all pairs"},
                "cpu": os.uname().machine}

    mode_ids = dict(A.MODES, packed=A.MODE_BATCHED_PACKED)

    def make_runner(mode_name):
        m = mode_ids[mode_name]
        sb = ctx.scratch_bytes(m, n)
        scratch = torch.empty(max(sb, 256), dtype=torch.uint8, device=dev) if sb else None

        def run():
            ctx.april_filter_pairs(dR, dS, d_r, d_s, n, out, m, scratch, stream)
        return run

    def time_mode(mode_name, steps, warmup):
        run = make_runner(mode_name)
        for _ in range(warmup):
            run()
        ctx.april_sync_status(stream)
        if not np.array_equal(out.cpu().numpy(), host_v):
            raise SystemExit(f"mode {mode_name}: verdicts differ from Algorithm 2 on the host")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        for k in range(steps):
            flush.fill_(k & 0xFF)
            evs[k][0].record(stream)
            run()
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
        ctx.april_sync_status(stream)
        return [a.elapsed_time(b) for a, b in evs]

    mode = args.mode
    tune = None
    if mode in ("batched", "packed") and args.tune:
        vals = [int(x) for x in args.tune.split(",")]
        T, G, W, CW = vals[:4]
        ctx.set_tune(A.april_tune(T, G, W, CW, 0, 0.0, vals[4] if len(vals) > 4 else 0))
        tune = ctx.get_tune().as_dict()
    elif mode in ("batched", "packed") and not args.no_autotune:
        # the project's autotuner picks the CTA threshold and first warp window
        m = A.MODE_BATCHED
        scratch = torch.empty(ctx.scratch_bytes(m, n), dtype=torch.uint8, device=dev)
        tune = ctx.april_autotune(dR, dS, d_r, d_s, n, out, scratch, stream).as_dict()
        del scratch
    clocks = Clocks()
    clocks.start()
    t_main = time_mode(mode, args.steps, args.warmup)
    if w.partitions:  # partitioned sets run only in the batched modes
        t_plain = None
        t_warp = None
        t_other = time_mode("packed" if mode == "batched" else "batched", args.steps, args.warmup)
    else:
        t_plain = time_mode("plain", max(3, args.steps // 2), args.warmup) if mode != "plain" else t_main
        t_warp = time_mode("warp", args.steps, args.warmup) if mode == "batched" else None
        t_other = None

    from paper_2307_01716_gb300 import dist as D
    ms = statistics.mean(t_main)
    ms_max = D.max_over_ranks(ms, ws, device=dev)
    value = ws * n / (ms_max * 1e-3)
    plain_ms = statistics.mean(t_plain) if t_plain else None

    # end to end through the host-buffer entry point (pinned host pairs in,
    # host verdicts out, copies inside the timed region)
    m = mode_ids[mode]
    work = torch.empty(ctx.host_work_bytes(m, n), dtype=torch.uint8, device=dev)
    h_r = torch.from_numpy(w.pr.view(np.int32)).pin_memory()
    h_s = torch.from_numpy(w.ps.view(np.int32)).pin_memory()
    h_v = torch.empty(n, dtype=torch.uint8).pin_memory()
    for _ in range(args.warmup):
        ctx.april_filter_pairs_host(dR, dS, h_r, h_s, n, h_v, m, work, stream)
    e2e_t = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.april_filter_pairs_host(dR, dS, h_r, h_s, n, h_v, m, work, stream)
        e2e_t.append(time.perf_counter() - t0)
    clk = clocks.stop(local)
    if not np.array_equal(h_v.numpy(), host_v):
        raise SystemExit("end-to-end verdicts differ")
    e2e_s = statistics.mean(e2e_t)

    peak, peak_kind = peaks()
    achieved = b_alg / (ms * 1e-3) / 1e9
    kernel_name = {"plain": "k_plain", "warp": "k_warp", "batched": "k_persistent", "packed": "k_persistent"}[mode]
    traffic = kernel_traffic(kernel_name, w.name, tune)
    # batched: binning + persistent kernel (+ routing for partitioned sets)
    launches = {"plain": 1, "warp": 1, "batched": 2, "packed": 2}[mode] + (1 if w.partitions else 0)

    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "polygons_per_side": int(w.R.n), "grid_order": w.order,
                   "pairs": n, "mode": mode, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": (f"dp{ws}: every rank filters its own full batch of pairs against its own "
                                  "resident sets; no collective on the data path") if ws > 1 else "single GPU"},
        "plain": None if plain_ms is None else {"pairs_per_s": n / (plain_ms * 1e-3), "ms_per_step": plain_ms,
                                                "speedup_of_mode": plain_ms / ms},
        "other_batched_mode": None if t_other is None else {
            "mode": "packed" if mode == "batched" else "batched",
            "pairs_per_s": n / (statistics.mean(t_other) * 1e-3), "ms_per_step": statistics.mean(t_other)},
        "sets": {"raw_list_bytes_per_side": [int(R.info().raw_list_bytes), int(S.info().raw_list_bytes)],
                 "packed_list_bytes_per_side": [int(R.info().packed_list_bytes), int(S.info().packed_list_bytes)],
                 "entries_per_side": [int(R.info().n_entries), int(S.info().n_entries)]},
        "warp": None if t_warp is None else {"pairs_per_s": n / (statistics.mean(t_warp) * 1e-3),
                                             "ms_per_step": statistics.mean(t_warp)},
        "useful_GBps": achieved,
        "algorithmic_bytes_per_step": b_alg,
        "algorithmic_bytes_model": ("search-start merge: per pair 8 B ids + 32 B descriptors + 1 B verdict + 8 B per "
                                    "interval the joins read from the searched start, plus the search probes"),
        "sequential_alg2_bytes_per_step": b_seq,
        "full_scan_bytes_per_step": b_full,
        "dram_over_algorithmic": None if traffic is None else traffic / b_alg,
        "cpu_alg2": cpu_alg2,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kernel_name,
                     "peak_kind": f"{peak_kind} copy bandwidth (burst)"},
        "e2e": {"value": n / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": n},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "tune": tune,
        "verdict_mix": (np.bincount(host_v, minlength=3)[:3] / n).round(4).tolist(),
    }
    if rank == 0 and not args.no_variants and not w.partitions:
        line["variants"] = variants_bench(ctx, A, torch, dev, stream, flush, w, R, S, dR, dS, args.steps,
                                          args.warmup)
    if rank == 0 and not args.no_construction and not w.partitions:
        line["construction"] = construction_bench(ctx, A, torch, dev, stream, flush, w, S, dS, host_v, args.steps,
                                                  args.warmup)
    if rank == 0 and not args.no_selection:
        same = args.config == 2 and not w.partitions
        line["selection"] = selection_bench(ctx, A, torch, dev, stream, flush, R if same else None,
                                            dR if same else None, args.steps, args.warmup)
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_bench(A.Context, A, torch, dev, args.serving_requests)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
        line["cpu_baseline"]["cpu"] = os.uname().machine
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()  # the other ranks wait for rank 0's serving and CPU legs
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
