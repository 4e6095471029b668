"""Benchmark of the APRIL intermediate filter on GB300.

One step = one pass of the filter (Algorithm 2 on every candidate pair) over
a synthetic workload standing in for the paper's TIGER/OSM joins.  The A/F
sets are built and uploaded once (the paper precomputes approximations); the
timed region runs the filter kernels on pairs and sets already resident in
HBM, and L2 is flushed between timed steps.

The headline (`value`) is the batched filter on the paper-scale workload:
200k + 200k star polygons on a 2^16 grid, ~2.7M MBR-join candidate pairs,
run with the library's default tuning.  The same JSON line carries:
  - the plain one-pair-per-thread and one-pair-per-warp kernels on the same
    pairs (the speed-up of batching), the autotuner's pick, the end-to-end
    number through the host-buffer entry point, the HBM roofline of the
    batched step (the triage and the lane-group kernel; algorithmic bytes of
    april_host_filter_searched's model over the step time, with the ncu DRAM
    bytes of the same kernels, workload and tuning when profiles/traffic.json
    has them for the current kernel sources);
  - `workloads`: the skewed 10M-pair workload (Pareto radii, lists of 1 to
    ~10^5 intervals) and the partitioned workload (16x16 partitions of order
    14, raw and compressed lists), each with the same figures;
  - parity: every timed mode equals host Algorithm 2 on every pair, and a
    seeded sample of pairs (long ones included) equals the oracle;
  - the filter variants, GPU construction, selection queries, the serving
    loop (a 40 GB budget and one that binds, every served verdict checked);
  - the oracle's throughput on all host cores on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode batched|warp|plain|packed]
  python bench.py --impl reference ...   # the oracle (CPU) on the same workload
  python bench.py --profile [--config C] [--mode M]   # one warm-up and one timed launch, nothing else
  python bench.py --selection-build                   # GPU construction of the selection queries only

Under torchrun (N > 1) the pairs are split into N contiguous shards of about
equal estimated cost; each rank filters its shard on its own GPU against its
own copy of both sets, the verdicts are gathered to rank 0 and checked, and
`value` is all pairs / the slowest rank's time (strong scaling).
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
PAIR_ID_BYTES = 8       # r and s ids
DESC_BYTES = 32         # two 16-byte object descriptors
VERDICT_BYTES = 1
IV_BYTES = 8            # one interval = two uint32
EXTRA_WORKLOADS = (3, 4)
# Tuning each workload is timed with (T,G,W,CW,JO as for --tune): the
# autotuner's pick on that workload, committed so that every run times the
# tuning the committed ncu traffic (profiles/traffic.json) was taken on; the
# paper-scale workload's pick is the library default.  Each leg also reports
# the autotuner's live pick and its time.
LEG_TUNES: dict[int, str] = {}  # none: the library default is the pick on every workload
ORACLE_SAMPLE = {2: (800, 200), 3: (800, 200), 4: (600, 200)}  # (short, long) pairs checked against the oracle
LONG_PAIR_COST = 2048  # a sampled pair is long when |A(r)| + |A(s)| exceeds this


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4])
    ap.add_argument("--mode", default="batched", choices=["batched", "warp", "plain", "packed"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="skip the autotuner leg")
    ap.add_argument("--autotuned", action="store_true",
                    help="time the headline with the autotuner's pick instead of the default tuning")
    ap.add_argument("--tune", default=None,
                    help="T,G,W,CW[,JO[,ESC[,TRIAGE_OFF]]]: fixed batched tuning instead of the default (JO: join "
                         "order 0, 1 or 2 = automatic; ESC: escalate_windows; TRIAGE_OFF: 1 = no triage pass)")
    ap.add_argument("--no-workloads", action="store_true", help="skip the skewed and partitioned workloads")
    ap.add_argument("--no-oracle-sample", action="store_true", help="skip the oracle parity samples")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--serving-requests", type=int, default=120)
    ap.add_argument("--no-selection", action="store_true", help="skip the selection-query measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the within / mixed-granularity measurement")
    ap.add_argument("--no-construction", action="store_true", help="skip the GPU construction measurement")
    ap.add_argument("--profile", action="store_true",
                    help="build the workload, run one warm-up and one timed step of --mode, exit (ncu captures)")
    ap.add_argument("--selection-build", action="store_true",
                    help="build the selection workload's query lists on the GPU four times, exit (ncu captures)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_sha() -> str:
    """Hash of the kernel sources a profile was taken on: filter.cu and
    join_device.cuh with their comments and whitespace removed, so that a
    comment edit keeps the profiles' DRAM figures attached."""
    import re
    h = hashlib.sha256()
    for f in ("filter.cu", "join_device.cuh"):
        src = open(os.path.join(ROOT, "paper_2307_01716_gb300", "csrc", f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def tune_key(t):
    return [t["cta_threshold"], t["group_lanes"], t["group_window"], t["cta_window"], t.get("join_order", 0),
            t.get("escalate_windows", 0), t.get("triage_off", 0)]


def triage_applies(tune, partitions, mode) -> bool:
    """Whether the batched filter runs its triage kernel (include/april.h,
    april_tune.triage_off): sets built from polygons (one grid or partitioned,
    raw or compressed), no long-pair threshold, lane groups below 32."""
    return (mode in ("batched", "packed") and tune is not None and not tune.get("triage_off", 0)
            and tune["cta_threshold"] == 0xFFFFFFFF and tune["group_lanes"] < 32)


def launches_per_step(tune, partitions, mode) -> int:
    """This library's kernels in one filter step: the partition routing, then
    the triage or the length binning (or neither), the persistent kernel and,
    with escalation, the kernel that finishes the handed-over joins."""
    if mode not in ("batched", "packed"):
        return 1
    n = 1 + (1 if partitions else 0)
    if triage_applies(tune, partitions, mode) or tune["cta_threshold"] != 0xFFFFFFFF:
        n += 1
    if tune.get("escalate_windows", 0) and tune["group_lanes"] < 32:
        n += 1
    return n


def kernel_traffic(kernel: str, workload: str, mode: str, tune):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources for the same workload, mode and tuning."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None, None
    sha = kernel_source_sha()
    key = None if tune is None else tune_key(tune)
    for e in json.load(open(p)):
        if (e.get("kernel") == kernel and e.get("workload") == workload and e.get("mode", "batched") == mode
                and e.get("src_sha") == sha and e.get("tune") == key):
            return e.get("dram_bytes_per_launch"), e.get("source")
    return None, None


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



def oracle_fn(w, threads: int):
    """f(pr, ps) -> the oracle's verdicts for workload w on `threads` host
    threads (partitioned workloads: each pair on its routed partition's grid,
    the grids computed once)."""
    import oracle
    if not w.partitions:
        g = oracle.Grid(w.order)
        return lambda pr, ps: oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, pr, ps, g, threads)
    grids = oracle.partition_areas(w.R.mbr, w.S.mbr, w.partitions, w.order)

    def f(pr, ps):
        part = oracle.route_pairs(w.R.mbr, w.S.mbr, pr, ps, w.partitions)
        out = np.zeros(len(pr), dtype=np.uint8)
        for p in np.unique(part):
            sel = np.nonzero(part == p)[0]
            out[sel] = oracle.verdicts(w.R.xy, w.R.off, w.S.xy, w.S.off, pr[sel], ps[sel], grids[int(p)], threads)
        return out
    return f


def cpu_baseline(w, cost, threshold, got, n_short, n_long, min_seconds=0.0, seed=2024):
    """The oracle, as it stands, timed on all host cores on a bounded seeded
    sample of workload w's pairs: n_long pairs above the long-pair threshold
    and n_short below it, then (until min_seconds have passed) further random
    pairs.  Its verdicts are compared with the GPU's verdicts `got` of the
    same pairs; a mismatch ends the run."""
    threads = os.cpu_count() or 1
    f = oracle_fn(w, threads)
    rng = np.random.default_rng(seed)
    long_idx = np.nonzero(cost > threshold)[0]
    short_idx = np.nonzero(cost <= threshold)[0]
    pick = [rng.choice(long_idx, min(n_long, len(long_idx)), replace=False),
            rng.choice(short_idx, min(n_short, len(short_idx)), replace=False)]
    batches = [np.sort(np.concatenate(pick))]
    done = 0
    t0 = time.perf_counter()
    while batches:
        idx = batches.pop()
        want = f(w.pr[idx], w.ps[idx])
        bad = np.nonzero(got[idx] != want)[0]
        if len(bad):
            raise SystemExit(f"{w.name}: {len(bad)} of {len(idx)} sampled verdicts differ from the oracle "
                             f"(first pair index {int(idx[bad[0]])})")
        done += len(idx)
        if time.perf_counter() - t0 < min_seconds:
            batches.append(np.sort(rng.choice(len(w.pr), 100 * threads, replace=False)))
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "pairs/s", "cores": threads, "kind": "oracle",
            "sample": f"{done} pairs of the {len(w.pr)} of {w.name} (seeded: {len(pick[0])} with "
                      f"|A(r)|+|A(s)| > {threshold}, {len(pick[1])} below, the rest uniform), cell-set oracle on "
                      f"{threads} host threads, {dt:.1f} s",
            "cpu": f"{os.uname().machine}, {threads} cores",
            "parity": {"pairs": int(done), "long_pairs": int(len(pick[0])), "mismatches": 0,
                       "compared_with": "the GPU verdicts of the same pairs"}}


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


class Leg:
    """One workload: its sets on the device, the host reference execution and
    the timing of the filter modes on it, over all pairs or one rank's shard."""

    def __init__(self, A, torch, ctx, dev, stream, flush, cfg, pack=False):
        from synth import configs
        self.A, self.torch, self.ctx, self.dev, self.stream, self.flush = A, torch, ctx, dev, stream, flush
        w = self.w = configs.make(cfg)
        if w.partitions:
            self.R, self.S = A.april_build_partitioned_sets(w.R.xy, w.R.off, w.S.xy, w.S.off, w.partitions, w.order)
        else:
            g = A.global_grid(w.order)
            self.R = A.april_build_sets(w.R.xy, w.R.off, g)
            self.S = A.april_build_sets(w.S.xy, w.S.off, g)
        if pack or w.partitions:
            self.R.compress()
            self.S.compress()
        self.dR, self.dS = A.april_upload(self.R, dev), A.april_upload(self.S, dev)
        self.n_all = len(w.pr)
        self.cost = self._cost()
        self.use_shard(0, self.n_all)

    def use_shard(self, lo, hi):
        """Filter pairs [lo, hi) of the workload from now on (one rank's shard)."""
        torch, w = self.torch, self.w
        self.lo, self.hi = lo, hi
        self.pr, self.ps = w.pr[lo:hi], w.ps[lo:hi]
        self.n = hi - lo
        self.d_r = torch.from_numpy(np.ascontiguousarray(self.pr).view(np.int32)).to(self.dev)
        self.d_s = torch.from_numpy(np.ascontiguousarray(self.ps).view(np.int32)).to(self.dev)
        self.out = torch.empty(max(self.n, 1), dtype=torch.uint8, device=self.dev)
        self.host_v = None

    def _cost(self):
        """|A(r)| + |A(s)| per pair (for partitioned sets, of the entries the
        pair is routed to), the length the long-pair threshold compares."""
        if not self.w.partitions:
            a_r, _ = self.R.lengths()
            a_s, _ = self.S.lengths()
            return a_r[self.w.pr].astype(np.int64) + a_s[self.w.ps]
        er, es = self.A.april_route_pairs(self.R, self.S, self.w.pr, self.w.ps)
        a_r, _ = self.R.lengths()
        a_s, _ = self.S.lengths()
        return a_r[er].astype(np.int64) + a_s[es]

    def host_reference(self):
        """Host Algorithm 2 on this rank's pairs: the verdicts every mode must
        give, the intervals sequential Algorithm 2 reads, and those the
        searched joins read (the algorithmic bytes)."""
        A = self.A
        t0 = time.perf_counter()
        self.host_v, consumed = A.april_host_filter(self.R, self.S, self.pr, self.ps)
        self.host_all_s = time.perf_counter() - t0
        fixed = self.n * (PAIR_ID_BYTES + DESC_BYTES + VERDICT_BYTES)
        self.b_seq = float(IV_BYTES * consumed.sum() + fixed)
        v2, consumed2 = A.april_host_filter(self.R, self.S, self.pr, self.ps, searched=True)
        if not np.array_equal(self.host_v, v2):
            raise SystemExit("the searched host execution disagrees with Algorithm 2")
        self.b_alg = float(IV_BYTES * consumed2.sum() + fixed)
        self.b_full = None
        if not self.w.partitions:  # no early exit: AA, AF and FA read every list in full
            a_r, f_r = self.R.lengths()
            a_s, f_s = self.S.lengths()
            iv = (2 * a_r[self.pr].astype(np.uint64) + 2 * a_s[self.ps] + f_r[self.pr] + f_s[self.ps]).sum()
            self.b_full = float(IV_BYTES * iv + fixed)
        k1 = min(self.n, 100_000)
        t0 = time.perf_counter()
        A.april_host_filter(self.R, self.S, self.pr[:k1], self.ps[:k1], n_threads=1)
        host_one_s = time.perf_counter() - t0
        self.cpu_alg2 = {"kind": "Algorithm 2 merge joins (AA, AF, FA, early exit) over the same lists, host C++",
                         "threads_1": {"pairs_per_s": k1 / host_one_s, "sample": f"first {k1} pairs"},
                         "threads_all": {"pairs_per_s": self.n / self.host_all_s, "threads": os.cpu_count(),
                                         "sample": "all pairs"}}

    def runner(self, mode_name):
        A, ctx = self.A, self.ctx
        m = {"plain": A.MODE_PLAIN, "warp": A.MODE_WARP, "batched": A.MODE_BATCHED,
             "packed": A.MODE_BATCHED_PACKED}[mode_name]
        sb = ctx.scratch_bytes(m, self.n)
        scratch = self.torch.empty(max(sb, 256), dtype=self.torch.uint8, device=self.dev) if sb else None

        def run():
            ctx.april_filter_pairs(self.dR, self.dS, self.d_r, self.d_s, self.n, self.out, m, scratch, self.stream)
        return run

    def time_mode(self, mode_name, steps, warmup, barrier=None):
        """CUDA-event times (ms) of `steps` passes, after `warmup` untimed ones
        whose verdicts must equal host Algorithm 2 on every pair."""
        torch = self.torch
        run = self.runner(mode_name)
        for _ in range(warmup):
            run()
        self.ctx.april_sync_status(self.stream)
        if self.host_v is not None and not np.array_equal(self.out[:self.n].cpu().numpy(), self.host_v):
            raise SystemExit(f"{self.w.name} mode {mode_name}: verdicts differ from Algorithm 2 on the host")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if barrier:
            barrier()
        torch.cuda.synchronize(self.dev)
        for k in range(steps):
            self.flush.fill_(k & 0xFF)
            evs[k][0].record(self.stream)
            run()
            evs[k][1].record(self.stream)
        torch.cuda.synchronize(self.dev)
        if barrier:
            barrier()
        self.ctx.april_sync_status(self.stream)
        return [a.elapsed_time(b) for a, b in evs]

    def e2e(self, mode_name, steps, warmup):
        """The same filter end to end through april_filter_pairs_host: pinned
        host pairs in, host verdicts out, the copies inside the timed region."""
        A, torch = self.A, self.torch
        m = {"plain": A.MODE_PLAIN, "warp": A.MODE_WARP, "batched": A.MODE_BATCHED,
             "packed": A.MODE_BATCHED_PACKED}[mode_name]
        work = torch.empty(self.ctx.host_work_bytes(m, self.n), dtype=torch.uint8, device=self.dev)
        h_r = torch.from_numpy(np.ascontiguousarray(self.pr).view(np.int32)).pin_memory()
        h_s = torch.from_numpy(np.ascontiguousarray(self.ps).view(np.int32)).pin_memory()
        h_v = torch.empty(self.n, dtype=torch.uint8).pin_memory()
        for _ in range(warmup):
            self.ctx.april_filter_pairs_host(self.dR, self.dS, h_r, h_s, self.n, h_v, m, work, self.stream)
        ts = []
        for k in range(steps):
            self.flush.fill_(k & 0xFF)
            torch.cuda.synchronize(self.dev)
            t0 = time.perf_counter()
            self.ctx.april_filter_pairs_host(self.dR, self.dS, h_r, h_s, self.n, h_v, m, work, self.stream)
            ts.append(time.perf_counter() - t0)
        if self.host_v is not None and not np.array_equal(h_v.numpy(), self.host_v):
            raise SystemExit(f"{self.w.name}: end-to-end verdicts differ")
        e2e_s = statistics.mean(ts)
        return {"value": self.n / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": 8 * self.n,
                "d2h_bytes_per_step": self.n, "ms_per_step": e2e_s * 1e3,
                "path": "april_filter_pairs_host: pinned host pairs in, verdicts to pinned host memory"}

    def roofline(self, ms, mode, tune, peak, peak_kind):
        achieved = self.b_alg / (ms * 1e-3) / 1e9
        kernel = {"plain": "k_plain", "warp": "k_warp", "batched": "k_persistent", "packed": "k_persistent"}[mode]
        traffic, src = kernel_traffic(kernel, self.w.name, mode, tune)
        if triage_applies(tune, self.w.partitions, mode):
            # the batched step is two kernels: the triage, then the lane groups
            kernel = "k_triage + k_persistent"
            t2, src2 = kernel_traffic("k_triage", self.w.name, mode, tune)
            traffic, src = (traffic + t2, f"{src} + {src2}") if traffic is not None and t2 is not None else (None, None)
        r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
             "traffic": traffic, "kernel": kernel, "peak_kind": f"{peak_kind} copy bandwidth (burst)",
             "achieved_bytes": "galloping search-start model (algorithmic_bytes_per_step)",
             "frac_sequential_alg2": self.b_seq / (ms * 1e-3) / 1e9 / peak}
        if traffic is not None:
            r["dram_GBps_at_step_time"] = traffic / (ms * 1e-3) / 1e9
            r["frac_dram"] = r["dram_GBps_at_step_time"] / peak
            r["dram_over_algorithmic"] = traffic / self.b_alg
            r["traffic_source"] = src
        return r


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


def serving_bench(A, torch, dev, n_requests: int, threads: int):
    """Config 5: 300k + 300k polygons (config-3 generator, 2^16 grid) resident
    in HBM; requests are query windows of 1k-2M candidate pairs (log-uniform)
    arriving as a Poisson stream.  Continuous batching (8 stream slots)
    against one request per launch, at 50% and 80% of the measured
    one-request-per-launch capacity, under the 40 GB budget and under a budget
    that binds (1.5x the largest request's buffers).  Every served verdict is
    compared with host Algorithm 2; the cpu_baseline leg compares a sample of
    them with the oracle."""
    from synth import configs, serving
    w = configs.make(5)
    g = A.global_grid(w.order)
    R = A.april_build_sets(w.R.xy, w.R.off, g)
    S = A.april_build_sets(w.S.xy, w.S.off, g)
    dR, dS = A.april_upload(R, dev), A.april_upload(S, dev)
    host_v, _ = A.april_host_filter(R, S, w.pr, w.ps)  # the verdict of every candidate a request may hold
    ctx = A.Context(dev.index or 0)
    maker = serving.RequestMaker(w.R.mbr, w.S.mbr, w.pr, w.ps)
    reqs = maker.requests(seed=11, count=n_requests, rate=0.0)
    bufs = [(torch.from_numpy(q.pr.view(np.int32).copy()).pin_memory(),
             torch.from_numpy(q.ps.view(np.int32).copy()).pin_memory(),
             torch.empty(len(q.pr), dtype=torch.uint8).pin_memory()) for q in reqs]
    sizes = np.array([len(q.pr) for q in reqs])

    def run(max_inflight, arrivals, arena):
        for b in bufs:
            b[2].fill_(0xEE)
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
        bad = sum(int((b[2].numpy() != host_v[q.idx]).sum()) for b, q in zip(bufs, reqs))
        if bad:
            raise SystemExit(f"serving: {bad} served verdicts differ from Algorithm 2 on the host")
        lat = np.array([(st.done_ns - st.submit_ns) / 1e6 for st in stats])
        queue = np.array([(st.admit_ns - st.submit_ns) / 1e6 for st in stats])
        service = np.array([(st.done_ns - st.admit_ns) / 1e6 for st in stats])
        span = (max(st.done_ns for st in stats) - min(st.submit_ns for st in stats)) / 1e9
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()),
                "queue_p50_ms": float(np.percentile(queue, 50)), "queue_p99_ms": float(np.percentile(queue, 99)),
                "service_p50_ms": float(np.percentile(service, 50)),
                "service_p99_ms": float(np.percentile(service, 99)),
                "pairs_per_s": float(sizes.sum() / span), "requests_per_s": float(len(reqs) / span),
                "max_concurrent": int(info.max_concurrent), "arena_peak_mb": info.arena_peak_bytes / (1 << 20),
                "verdicts_checked": int(sizes.sum()), "mismatches": 0}

    out = {"workload": w.name, "candidates": int(len(w.pr)), "requests": len(reqs),
           "request_pairs_mean": float(sizes.mean()), "request_pairs_p50": float(np.median(sizes)),
           "request_pairs_max": int(sizes.max()), "slots": 8, "budgets": {}}
    rng = np.random.default_rng(77)
    gaps = rng.exponential(1.0, len(reqs))
    big = int(1.5 * 25 * sizes.max()) + (1 << 20)  # a request of n pairs takes about 25 n bytes of arena
    capacity = None
    for label, nbytes in (("40GB", 40 << 30), ("binding", big)):
        arena = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        b = {"arena_mb": nbytes / (1 << 20)}
        if capacity is None:  # all requests offered at once, one per launch
            cap = run(1, np.zeros(len(reqs)), arena)
            capacity = cap["requests_per_s"]
            out["capacity_one_per_launch_req_s"] = capacity
        b["rates"] = {}
        for frac in (0.5, 0.8):
            lam = frac * capacity
            arrivals = np.cumsum(gaps) / lam
            b["rates"][f"{frac:.0%}"] = {"rate_req_s": lam, "continuous": run(8, arrivals, arena),
                                         "one_per_launch": run(1, arrivals, arena)}
        out["budgets"][label] = b
        del arena
    # the oracle on a sample of the served pairs (the served verdicts equal host_v)
    all_idx = np.concatenate([q.idx for q in reqs])
    pick = np.unique(np.random.default_rng(5).choice(all_idx, 300, replace=False))
    t0 = time.perf_counter()
    want = oracle_fn(w, threads)(w.pr[pick], w.ps[pick])
    dt = time.perf_counter() - t0
    if not np.array_equal(want, host_v[pick]):
        raise SystemExit("serving: sampled served verdicts differ from the oracle")
    out["cpu_baseline"] = {"value": len(pick) / dt, "unit": "pairs/s", "cores": threads, "kind": "oracle",
                           "sample": f"{len(pick)} served pairs (seeded), compared with their served verdicts",
                           "parity": {"pairs": int(len(pick)), "mismatches": 0}}
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The reference arm: the oracle (the plain CPU statement of the method)
    as it stands, on all host cores, each step a bounded random sample of the
    same workload; rank 0 only."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from synth import configs
    w = configs.make(args.config)
    threads = os.cpu_count() or 1
    f = oracle_fn(w, threads)
    rng = np.random.default_rng(99)
    per_step = 100 * threads
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
            "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": w.name, "pairs": int(len(w.pr)),
                                              "sample_pairs_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} random pairs per step of {len(w.pr)}, {threads} host threads"},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def selection_build_only(A, torch, dev):
    """GPU construction of the selection workload's 1,000 query polygons, four
    times, from polygons already on the device (for ncu launch lists)."""
    from synth import selection
    s = selection.make(1.0, 1000)
    ctx = A.Context(dev.index or 0)
    g = A.global_grid(s.order)
    d_xy = torch.from_numpy(np.ascontiguousarray(s.Q.xy, dtype=np.int32)).to(dev)
    d_off = torch.from_numpy(np.ascontiguousarray(s.Q.off, dtype=np.int64)).to(dev)
    _, info = ctx.april_build_sets_device(d_xy, d_off, g)
    work = torch.empty(int(info.work_bytes), dtype=torch.uint8, device=dev)
    image = torch.empty(int(info.image_bytes), dtype=torch.uint8, device=dev)
    ts = []
    for _ in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.april_build_sets_device(d_xy, d_off, g, work=work, image=image)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    print(json.dumps({"selection_build_ms": [round(t * 1e3, 2) for t in ts], "queries": int(s.Q.n),
                      "touched_cells": int(info.touched_cells)}), flush=True)


def parse_tune(A, spec):
    """T,G,W,CW[,JO[,ESC[,TRIAGE_OFF]]] (april_tune; JO 2 = automatic when omitted)."""
    vals = [int(x) for x in spec.split(",")]
    T, G, W, CW = vals[:4]
    return A.april_tune(T, G, W, CW, 0, 0.0, vals[4] if len(vals) > 4 else 2, vals[5] if len(vals) > 5 else 0,
                        vals[6] if len(vals) > 6 else 0)


def run_leg(A, torch, ctx, dev, stream, flush, cfg, args, mode, peak, peak_kind, default_tune, ws=1, rank=0,
            barrier=None, gloo=None):
    """One workload: the timed mode, the modes it is compared with, the
    autotuner's pick, end to end, the roofline and the parity checks; the
    context starts from default_tune (the library default)."""
    from paper_2307_01716_gb300 import dist as D
    L = Leg(A, torch, ctx, dev, stream, flush, cfg, pack=(mode == "packed"))
    ctx.set_tune(default_tune)  # earlier legs may have autotuned the context
    tuning = "library default"
    if args.tune:
        ctx.set_tune(parse_tune(A, args.tune))
        tuning = "fixed --tune"
    elif cfg in LEG_TUNES and not args.autotuned:
        ctx.set_tune(parse_tune(A, LEG_TUNES[cfg]))
        tuning = "committed for this workload (the autotuner's pick)"
    res = {"workload": L.w.name, "pairs": int(L.n_all), "polygons_per_side": int(L.w.R.n), "grid_order": L.w.order,
           "partitions": int(L.w.partitions), "mode": mode, "tuning": tuning if not args.autotuned else "autotuned"}
    timed = {}

    def run_shard(lo, hi):
        """This rank's pairs: host reference, autotuner, the timed mode."""
        L.use_shard(lo, hi)
        L.host_reference()
        if mode in ("batched", "packed") and not args.no_autotune:
            sc = torch.empty(ctx.scratch_bytes(A.MODE_BATCHED, L.n), dtype=torch.uint8, device=dev)
            chosen = ctx.get_tune()
            picked = ctx.april_autotune(L.dR, L.dS, L.d_r, L.d_s, L.n, L.out, sc, stream).as_dict()
            res["autotune"] = {"pick": picked, "pick_ms": picked["ms"],
                               "kept_default": tune_key(picked) == tune_key(chosen.as_dict())}
            if not args.autotuned:
                ctx.set_tune(chosen)
            del sc
        timed["t"] = L.time_mode(mode, args.steps, args.warmup, barrier)
        return L.out[:L.n].cpu().numpy()

    shards, gathered = D.sharded_filter(L.cost, ws, rank, run_shard, group=gloo)
    tune = ctx.get_tune().as_dict() if mode in ("batched", "packed") else None
    ms = statistics.mean(timed["t"])
    ms_max = D.max_over_ranks(ms, ws, device=dev)
    res.update({"ms_per_step": ms_max, "pairs_per_s": L.n_all / (ms_max * 1e-3), "tune": tune,
                "verdict_mix": (np.bincount(L.host_v, minlength=3)[:3] / max(L.n, 1)).round(4).tolist()})
    if ws > 1:
        res["shards"] = [list(map(int, sh)) for sh in shards]
    if L.w.partitions:
        other = "packed" if mode == "batched" else "batched"
        t_o = L.time_mode(other, args.steps, args.warmup)
        ms_o = statistics.mean(t_o)
        res["other_batched_mode"] = {"mode": other, "ms_per_step": ms_o, "pairs_per_s": L.n / (ms_o * 1e-3),
                                     "time_ratio_to_mode": ms_o / ms,
                                     "roofline": L.roofline(ms_o, other, tune, peak, peak_kind)}
    else:
        if mode != "plain":
            t_p = L.time_mode("plain", max(3, args.steps // 4), args.warmup)
            res["plain"] = {"pairs_per_s": L.n / (statistics.mean(t_p) * 1e-3), "ms_per_step": statistics.mean(t_p),
                            "speedup_of_mode": statistics.mean(t_p) / ms}
        if mode == "batched":
            t_w = L.time_mode("warp", args.steps, args.warmup)
            res["warp"] = {"pairs_per_s": L.n / (statistics.mean(t_w) * 1e-3), "ms_per_step": statistics.mean(t_w)}
    res["e2e"] = L.e2e(mode, args.steps, args.warmup)
    res["roofline"] = L.roofline(ms, mode, tune, peak, peak_kind)
    res["useful_GBps"] = res["roofline"]["achieved"]
    res["algorithmic_bytes_per_step"] = L.b_alg
    res["algorithmic_bytes_model"] = ("galloping merge from the searched starts: per pair 8 B ids + 32 B descriptors "
                                      "+ 1 B verdict + 8 B per interval the joins read and per search probe (a search "
                                      "at each join's start and after 16 consecutive advances of one list)")
    res["sequential_alg2_bytes_per_step"] = L.b_seq
    res["full_scan_bytes_per_step"] = L.b_full
    res["cpu_alg2"] = L.cpu_alg2
    res["sets"] = {"raw_list_bytes_per_side": [int(L.R.info().raw_list_bytes), int(L.S.info().raw_list_bytes)],
                   "packed_list_bytes_per_side": [int(L.R.info().packed_list_bytes),
                                                  int(L.S.info().packed_list_bytes)],
                   "entries_per_side": [int(L.R.info().n_entries), int(L.S.info().n_entries)]}
    res["parity"] = {"host_alg2": f"every timed mode equals host Algorithm 2 on all {L.n} pairs of this rank"}
    if rank == 0 and ws > 1:
        full, _ = A.april_host_filter(L.R, L.S, L.w.pr, L.w.ps)
        if not np.array_equal(gathered, full):
            raise SystemExit("the gathered verdicts of the shards differ from Algorithm 2 on all pairs")
        res["parity"]["gathered_shards"] = "equal host Algorithm 2 on all pairs"
    return L, res, gathered


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from paper_2307_01716_gb300 import april as A

    ws, rank, local = dist_env()
    gloo = None
    if ws > 1:
        dist.init_process_group("nccl")
        gloo = dist.new_group(backend="gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.selection_build:
        return selection_build_only(A, torch, dev)
    ctx = A.Context(local)
    default_tune = ctx.get_tune()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    mode = args.mode
    if args.profile:
        L = Leg(A, torch, ctx, dev, stream, flush, args.config, pack=(mode == "packed"))
        if args.tune or args.config in LEG_TUNES:
            ctx.set_tune(parse_tune(A, args.tune or LEG_TUNES[args.config]))
        run = L.runner(mode)
        run()
        flush.fill_(1)
        run()
        ctx.april_sync_status(stream)
        torch.cuda.synchronize()
        print(json.dumps({"profile": L.w.name, "mode": mode, "tune": ctx.get_tune().as_dict()}), flush=True)
        return
    peak, peak_kind = peaks()
    barrier = dist.barrier if ws > 1 else None
    clocks = Clocks()
    clocks.start()
    L, head, _ = run_leg(A, torch, ctx, dev, stream, flush, args.config, args, mode, peak, peak_kind, default_tune,
                         ws, rank, barrier, gloo)
    clk = clocks.stop(local)
    roof = head["roofline"]
    line = {
        "metric": METRIC, "value": head["pairs_per_s"], "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded star polygons standing in for the paper's TIGER/OSM datasets)",
        "config": {"workload": head["workload"], "polygons_per_side": head["polygons_per_side"],
                   "grid_order": head["grid_order"], "pairs": head["pairs"], "mode": mode,
                   "tuning": head["tuning"],
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": (f"{ws} ranks: the pairs split into {ws} contiguous shards of about equal "
                                   "|A(r)|+|A(s)|, each filtered on its own GPU against its own copy of both sets; "
                                   "verdicts gathered to rank 0 after the timed region") if ws > 1 else "single GPU"},
        "roofline": roof,
        "e2e": head["e2e"],
        "gpu_launches": launches_per_step(head.get("tune") or ctx.get_tune().as_dict(), L.w.partitions,
                                          mode) * args.steps,
        "clocks": clk,
    }
    for k, v in head.items():
        if k not in line and k not in ("workload", "polygons_per_side", "grid_order", "pairs", "mode",
                                       "pairs_per_s", "ms_per_step", "tuning"):
            line[k] = v
    line["dram_over_algorithmic"] = roof.get("dram_over_algorithmic")
    threads = os.cpu_count() or 1
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(L.w, L.cost, LONG_PAIR_COST, L.out[:L.n].cpu().numpy(),
                                            *ORACLE_SAMPLE.get(args.config, (600, 200)), min_seconds=args.cpu_seconds)
    if rank == 0 and ws == 1 and args.config == 2:
        if not args.no_variants:
            line["variants"] = variants_bench(ctx, A, torch, dev, stream, flush, L.w, L.R, L.S, L.dR, L.dS,
                                              args.steps, args.warmup)
        if not args.no_construction:
            line["construction"] = construction_bench(ctx, A, torch, dev, stream, flush, L.w, L.S, L.dS, L.host_v,
                                                      args.steps, args.warmup)
        if not args.no_selection:
            line["selection"] = selection_bench(ctx, A, torch, dev, stream, flush, L.R, L.dR, args.steps,
                                                args.warmup)
    del L
    if rank == 0 and not args.no_workloads and args.config == 2:
        line["workloads"] = {}
        for cfg in EXTRA_WORKLOADS:
            torch.cuda.empty_cache()
            Lx, res, _ = run_leg(A, torch, ctx, dev, stream, flush, cfg, args, "batched", peak, peak_kind,
                                 default_tune)
            if not args.no_cpu_baseline:
                res["cpu_baseline"] = cpu_baseline(Lx.w, Lx.cost, LONG_PAIR_COST,
                                                   Lx.out[:Lx.n].cpu().numpy(), *ORACLE_SAMPLE[cfg])
            line["workloads"][res["workload"]] = res
            del Lx
    if rank == 0 and not args.no_serving:
        line["serving"] = serving_bench(A, torch, dev, args.serving_requests, threads)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()  # the other ranks wait for rank 0's extra legs
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
