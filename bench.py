#!/usr/bin/env python
"""Benchmark of the GB300 ensemble transfer-entropy hot path.

One step = one pass of the whole hot path (embedding gather, max-norm kNN search, marginal
range counts, digamma sum, surrogate p-values) over one batch of synthetic input.  The default
workload is the largest single-GPU configuration, the large-ensemble surrogate test: 4000
trials of a logistic-map source driving an AR(1) target, d = 5, tau = 1, u = 5, window 3
(N = 12,000 points in an 11-D joint space), 200 analysis time points x (1 original + 200
trial-shuffled surrogates) = 40,200 estimates, k = 4.

Printed (rank 0, one JSON line): combined max-norm pair evaluations per second (both passes,
ordered pairs i != j) over all ranks, TE estimates per second, the end-to-end rate through the
public API with host buffers, per-instance launches against one batched launch on the same GPU,
the roofline of the search kernels against the FP32 ALU peak (operations actually issued), the
SM clocks seen, and the CPU oracle timed on a bounded sample of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c5]
                    [--scaling strong|weak]
Under torchrun (N > 1) the ranks share the workload by default (strong scaling): each takes a
cost-balanced share of the analysis time points (with all of their surrogates) and the results
are all-gathered once per step, the only exchange; value = the workload's pair evaluations /
max-over-ranks time. --scaling weak has every rank run the whole workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "max-norm pair evals/s & TE estimates/s (incl. surrogates), batched vs per-launch"
FLUSH_BYTES = 256 << 20          # > 129 MB L2: written between timed steps
FALLBACK_SM_MHZ = 2070.0
ALU_LANES_PER_SM = 128           # FP32 lanes per SM (4 SMSPs x 32)
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "{kernel}_traffic.json")

WORKLOADS = {
    "c3": dict(cid=3, kw={}, desc="C3 surrogate test: AR(2) X->Y, 400 trials, d=3, tau=1, u=5, W=3 "
               "(N=1200, D=7), 50 time points x (1+1000 surrogates) = 50,050 estimates, k=4"),
    "c3-small": dict(cid=3, kw=dict(n_t=4, S=200), desc="C3 shapes, 4 time points x (1+200)"),
    "c1": dict(cid=1, kw={}, desc="C1 stationary AR(2): N=1000, D=5, 1 estimate, k=4"),
    "c2": dict(cid=2, kw={}, desc="C2 non-stationary AR(2): N=1500, D=7, 100 time points, k=4"),
    "c4": dict(cid=4, kw={}, desc="C4 uneven MEG-like batch: 20 pink-noise pairs x 30 t, N 50..10000, D 3..11"),
    "c5": dict(cid=5, kw={}, desc="C5 large ensemble: N=12000, D=11, 200 t x (1+200) = 40,200 estimates"),
    "c5-small": dict(cid=5, kw=dict(n_t=2, S=20), desc="C5 shapes, 2 time points x (1+20)"),
    "c5-4t": dict(cid=5, kw=dict(n_t=4), desc="C5 shapes, 4 time points x (1+200) = 804 estimates"),
    "ar1-scan": dict(cid=None, kw={}, desc="AR(1) unidirectional scenario (Table 1): 50 trials x 3000 samples, "
                     "d=1, windows of 300 (N=15000, D=3) at 0.2/0.5/0.8/1.1 s, delay scan u=1..20, "
                     "500 surrogates each = 40,080 estimates, k=4"),
    "lorenz-scan": dict(cid="lorenz", kw={}, desc="Lorenz X->Y (Eq. 11, Fig. 6): 150 repetitions x 3000 samples, "
                        "d=4, tau=3, windows of 250 (N=37500, D=9) at 200/1600/2750, delay scan u=35..55, "
                        "50 surrogates each = 3,213 estimates, k=4"),
    "paper-chunk": dict(cid="chunk", kw={}, desc="the paper's benchmark chunk (performance test): 16 estimates "
                        "of 30094 points x 17-D (d=8, coupled Lorenz data), k=4"),
}

# The paper's timing of its benchmark chunk (kNN search in 17-D + range search, 30094 points) on a
# GTX Titan: 24.1 s / 50 per chunk, i.e. about 3.6e9 ordered pair evaluations per second over both
# searches; another machine's number, context for the paper-chunk workload only.
PAPER_CHUNK_TITAN_PAIR_RATE = 2 * 30094 * 30093 / 0.51


def load_workload(spec):
    from paper_1401_4068_gb300 import inputs as I
    if spec["cid"] is None:
        return I.ar1_analysis("unidirectional", S=500)
    if spec["cid"] == "lorenz":
        return I.lorenz_analysis(S=50)
    if spec["cid"] == "chunk":
        return I.paper_chunk(chunks=16)
    return I.config(spec["cid"], **spec["kw"])


def scan_range(w):
    return (w.extra["u_lo"], w.extra["u_hi"]) if "u_lo" in w.extra else None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _scan_factor(w):
    sr = scan_range(w)
    return 1 if sr is None else sr[1] - sr[0] + 1


def pair_evals(w):
    """Ordered pairs i != j of ONE pass, summed over the estimates of one step (a delay scan
    repeats every listed estimate once per scanned delay)."""
    return _scan_factor(w) * sum(w.n_points(i) * (w.n_points(i) - 1) for i in w.instances)


def lane_ops(w):
    """Algorithmic FP32 operations of both passes: D subtractions + D abs-max per ordered pair."""
    return 2 * _scan_factor(w) * sum(w.n_points(i) * (w.n_points(i) - 1) * 2 * w.joint_dim(i)
                                     for i in w.instances)


# the translation units that hold each search kernel (file-name prefixes under csrc/)
KERNEL_UNITS = {"lane_kernel": ("te_lanes",), "batched_kernel": ("te_batched_d", "te_batched_mix"),
                "bundle_kernel": ("te_bundle.cu",)}


def kernel_source_hash(kernel: str) -> str:
    """Hash of the device code a search kernel is built from: its translation units and every
    project header they include, directly or not (a change elsewhere leaves it unchanged)."""
    csrc = os.path.join(ROOT, "paper_1401_4068_gb300", "csrc")
    inc = os.path.join(ROOT, "include")
    todo = sorted(f for f in os.listdir(csrc)
                  if f.endswith(".cu") and f.startswith(KERNEL_UNITS[kernel]))
    seen = {}
    while todo:
        f = todo.pop()
        if f in seen:
            continue
        path = next((os.path.join(d, f) for d in (csrc, inc) if os.path.exists(os.path.join(d, f))), None)
        if path is None:
            continue
        with open(path, "rb") as fh:
            seen[f] = fh.read()
        todo += re.findall(r'^\s*#include\s+"([^"]+)"', seen[f].decode(), flags=re.M)
    h = hashlib.sha256()
    for f in sorted(seen):
        h.update(f.encode() + seen[f])
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def traffic_per_launch(w, kernel):
    """DRAM bytes of one launch of `kernel` from the committed ncu summary (a capture of the same
    instance shape, scaled by the number of estimates, since every estimate stages the same
    points), or None when absent, taken on another instance shape, or taken on different kernel
    sources."""
    try:
        with open(PROFILE_TRAFFIC.format(kernel=kernel)) as f:
            prof = json.load(f)
    except (OSError, ValueError):
        return None
    if kernel not in KERNEL_UNITS or prof.get("kernel_src_hash") != kernel_source_hash(kernel):
        return None
    shape = sorted({(w.n_points(i), w.joint_dim(i)) for i in w.instances})
    if [list(x) for x in shape] != prof.get("instance_shapes"):
        return None
    return prof["dram_bytes"] / prof["estimates"] * len(w.instances)


LARGE_N = 8192          # above this, the oracle is timed on sampled query points of an estimate
LARGE_N_QUERIES = 64    # query points per estimate


def run_oracle_sample(w, idx, threads):
    """Time the oracle on the estimates idx; returns (pair evaluations, seconds, estimates). An
    estimate with more than LARGE_N points is timed on LARGE_N_QUERIES seeded query points (the
    oracle's per-point kNN and counts over all N points): its pair evaluations and its share of
    an estimate are counted accordingly."""
    import oracle  # CPU baseline only
    import numpy as np
    insts = [w.instances[i] for i in idx]
    small = [it for it in insts if w.n_points(it) <= LARGE_N]
    large = [it for it in insts if w.n_points(it) > LARGE_N]
    pe, est, dt = 0, 0.0, 0.0
    if small:
        t0 = time.perf_counter()
        oracle.te_batch(w.series, small, w.k, n_threads=threads)
        dt += time.perf_counter() - t0
        pe += sum(w.n_points(i) * (w.n_points(i) - 1) for i in small) * 2
        est += len(small)
    for j, it in enumerate(large):
        s = w.series[it.series]
        perm = None if it.perm < 0 else s.perms[it.perm]
        pts = oracle.embed(s.src, s.tgt, s.d, s.tau, s.u, it.t_start, it.window, perm)
        N = pts.shape[0]
        q = np.random.default_rng(300 + j).choice(N, LARGE_N_QUERIES, replace=False)
        t0 = time.perf_counter()
        oracle.points_at(pts, s.d, s.d, w.k, q, n_threads=threads)
        dt += time.perf_counter() - t0
        pe += 2 * LARGE_N_QUERIES * (N - 1)
        est += LARGE_N_QUERIES / N
    return pe, dt, est


def cpu_baseline(w, seconds: float):
    """Oracle as it stands on the host cores, on a bounded sample sized to ~`seconds`."""
    import oracle
    from paper_1401_4068_gb300 import inputs as I
    threads = oracle.default_threads()
    n = max(threads, 8)
    idx = I.sample_instances(w, n, seed=11)
    pe, dt, m = run_oracle_sample(w, idx, threads)
    for seed in (12, 13):  # resample, sized from the last sample's rate, until it fills the budget
        if dt >= 0.8 * seconds or n >= len(w.instances):
            break
        n = min(len(w.instances), max(n + 1, int(n * min(64.0, seconds / max(dt, 1e-3)))))
        idx = I.sample_instances(w, n, seed=seed)
        pe, dt, m = run_oracle_sample(w, idx, threads)
    return {"value": pe / dt, "unit": "pair-evals/s", "cores": threads, "kind": "oracle",
            "seconds": round(dt, 2), "te_estimates_per_s": m / dt,
            "sample": f"{m:.4g} of {len(w.instances)} estimates (cost-stratified, seeded; estimates over "
                      f"{LARGE_N} points on {LARGE_N_QUERIES} sampled query points each), both passes"}


# ---------------------------------------------------------------------------------- ours
PATH_KERNELS = ("lane_kernel", "bundle_kernel", "batched_kernel")  # te_last_paths order
SHARING = {"none": 0, "auto": 1, "bundles": 2, "lanes": 3}  # te_set_sharing modes


def make_runner(te, torch, h, w, dev, units=None):
    """The hot path on this rank: the whole workload, or (sharded) the units listed — analysis
    starts of a surrogate test or delay scan, instances of a te_estimate batch. Returns (step,
    outs, rows): step(series, outs) runs the library on this rank's share; rows(outs) packs its
    results as float64 rows, one per unit (for the gather of a sharded run)."""
    scan = scan_range(w)
    surrogate = w.S > 0 and w.t_starts is not None
    if scan or surrogate:
        ts = list(w.t_starts[0]) if units is None else [w.t_starts[0][u] for u in units]
        nt = len(ts)
        if scan:
            n_u = scan[1] - scan[0] + 1
            outs = {"te": torch.empty((n_u, nt), dtype=torch.float64, device=dev),
                    "p": torch.empty((n_u, nt), dtype=torch.float64, device=dev),
                    "u_best": torch.empty(nt, dtype=torch.int32, device=dev)}

            def step(series_dev, o):
                return te.te_delay_scan(h, series_dev[0], ts, w.window, scan[0], scan[1], w.S, w.k, out=o)

            def rows(o):
                return torch.cat([o["te"].t(), o["p"].t(), o["u_best"].to(torch.float64).view(-1, 1)], dim=1)
        else:
            outs = {"te_orig": torch.empty((1, nt), dtype=torch.float64, device=dev),
                    "te_surr": torch.empty((1, nt, w.S), dtype=torch.float64, device=dev),
                    "p": torch.empty((1, nt), dtype=torch.float64, device=dev)}

            def step(series_dev, o):
                return te.te_surrogate_test(h, series_dev, ts, w.window, w.S, w.k, out=o)

            def rows(o):
                return torch.cat([o["te_orig"].view(-1, 1), o["p"].view(-1, 1), o["te_surr"].view(nt, w.S)], dim=1)
        return step, outs, rows
    insts = list(w.instances) if units is None else [w.instances[u] for u in units]
    arr = te.instance_array(insts)  # host descriptors, built once like the device series
    outs = torch.empty(len(insts), dtype=torch.float64, device=dev)

    def step(series_dev, o):
        return te.te_estimate(h, series_dev, arr, w.k, te=o)

    def rows(o):
        return o.view(-1, 1)
    return step, outs, rows


def bench_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1401_4068_gb300 import build
    from paper_1401_4068_gb300 import inputs as I
    from paper_1401_4068_gb300 import sharding
    from paper_1401_4068_gb300 import te

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    # one rank (re)builds the library if it is stale; the others wait and then find it current
    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    build.build()
    spec = WORKLOADS[args.workload]
    w = load_workload(spec)
    scan = scan_range(w)
    surrogate = w.S > 0 and w.t_starts is not None
    h = te.Handle(local)
    ds = te.to_device(w.series, dev)
    te.te_set_profiling(h, True)
    te.te_set_search(h, not args.exhaustive)
    share = te.SHARE_NONE if args.no_sharing else SHARING[args.sharing]
    te.te_set_sharing(h, share)

    # strong scaling (default with several ranks): each rank takes a cost-balanced share of the
    # units and the per-unit results are all-gathered; weak: every rank runs the whole workload
    sharded = ws > 1 and args.scaling == "strong"
    units = parts = None
    if sharded:
        if scan or surrogate:
            parts = sharding.balance(sharding.time_point_costs(w), ws)
            n_units = len(w.t_starts[0])
        else:
            parts = sharding.shard(w, ws)
            n_units = len(w.instances)
        units = parts[rank]
    step_local, outs, rows = make_runner(te, torch, h, w, dev, units)
    if sharded and not units:
        raise SystemExit(f"rank {rank} has no work: fewer units than ranks")

    def step(series_dev, o):
        step_local(series_dev, o)
        if sharded:
            return sharding.gather_rows(rows(o), parts, n_units)
        return None

    tuned = None
    if args.shape:
        tuned = tuple(int(v) for v in args.shape.lower().split("x"))
        te.te_set_launch_config(h, tuned[0], tuned[1])
    elif not args.no_autotune:
        tuned = te.te_autotune(h, ds, w.instances if units is None or scan or surrogate else
                               [w.instances[u] for u in units], w.k)

    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        step(ds, outs)
    torch.cuda.synchronize()
    te.te_sync_status(h)

    def barrier():
        if ws > 1:
            dist.barrier()

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid else None)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kernel_ms = []
    launches = 0
    for a, b in ev:
        flush.zero_()
        a.record()
        step(ds, outs)
        b.record()
        launches += te.te_last_launch_count(h)
        kernel_ms.append(te.te_last_kernel_ms(h))
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    exec_pairs, exec_ops, swept = te.te_last_work(h)
    alu_ops, bundles = te.te_last_alu_ops(h)
    paths = te.te_last_paths(h)
    (pass_pairs, pass_cycles) = te.te_last_pass_work(h)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    te.te_sync_status(h)

    # units of work: the whole workload once per step (sharded), or once per rank (replicated)
    copies = 1 if sharded else ws
    pe_step = 2 * pair_evals(w)
    n_est = len(w.instances) * _scan_factor(w)
    value = copies * pe_step * args.steps / (total_ms / 1e3)
    te_rate = copies * n_est * args.steps / (total_ms / 1e3)
    # this rank's share of the pair evaluations (for its own device-side counters)
    if sharded and (scan or surrogate):
        pe_rank = pe_step * len(units) / len(w.t_starts[0])
    elif sharded:
        pe_rank = 2 * _scan_factor(w) * sum(w.n_points(w.instances[u]) * (w.n_points(w.instances[u]) - 1)
                                            for u in units)
    else:
        pe_rank = pe_step

    # ---- the two passes: the step time split by the warps' SM cycles in each pass (device clock,
    # counted by the sweep); the algorithmic work is N (N - 1) pairs per pass
    passes = None
    if swept and sum(pass_cycles) > 0:
        per_pass = pe_rank / 2
        passes = {"time_split": "step time x share of the warps' SM cycles spent in the pass (clock64 on "
                                "the device; pass 2 includes the digamma terms)"}
        for name, pp, cyc in (("pass1_knn", pass_pairs[0], pass_cycles[0]),
                              ("pass2_counts", pass_pairs[1], pass_cycles[1])):
            cyc_frac = cyc / sum(pass_cycles)
            passes[name] = {"cycle_share": round(cyc_frac, 4),
                            "pair_evals_per_s": copies * (pe_step / 2) * args.steps / (total_ms * cyc_frac / 1e3),
                            "pair_evals_executed_per_step": pp,
                            "executed_vs_algorithmic": round(pp / max(1.0, per_pass), 4)}

    # ---- roofline of the search kernels (CUDA events the library records around them on the
    # launching stream, live): `frac` counts the FP32 subtract / abs-max operations the kernels
    # actually issued; the kernel named is the one that ran most of the estimates
    kms = statistics.mean(kernel_ms)
    kernel = PATH_KERNELS[max(range(3), key=lambda i: (paths[i], -i))]
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or FALLBACK_SM_MHZ)
    n_sm = props.multi_processor_count
    peak = n_sm * ALU_LANES_PER_SM * sm_max * 1e6 / 1e12
    achieved = alu_ops / (kms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4),
            "peak_source": f"{n_sm} SMs x {ALU_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz "
                           f"({'MEASURED_PEAKS.json sm_max_mhz' if peaks.get('sm_max_mhz') else 'fallback clock'})",
            "op": "FP32 subtract / abs-max operations the search kernels issued (target parts computed "
                  "once for the estimates that share them; references skipped by the exact shared "
                  "bound not evaluated)",
            "kernel": kernel, "kernel_ms": round(kms, 4),
            "traffic": traffic_per_launch(w, kernel) if not sharded else None,
            "alu_ops_executed": alu_ops,
            # 2 D operations per (query, reference, estimate) pair the kernels decided: the
            # algorithmic unit, which counts shared and skipped operations as if executed
            "frac_2d_per_decided_pair": round(exec_ops / (kms / 1e3) / 1e12 / peak, 4)}
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = round(achieved / (n_sm * ALU_LANES_PER_SM * clocks["sm_mhz"] * 1e6 / 1e12), 4)

    # ---- end to end through the public API: pinned host inputs in, results out, every step
    host = []
    for s in w.series:
        hs = {"src": torch.from_numpy(np.ascontiguousarray(s.src)).pin_memory(),
              "tgt": torch.from_numpy(np.ascontiguousarray(s.tgt)).pin_memory(),
              "perms": None if s.perms is None else torch.from_numpy(np.ascontiguousarray(s.perms)).pin_memory()}
        host.append(hs)
    h2d = sum(v.numel() * v.element_size() for hs in host for v in hs.values() if v is not None)
    res_dev = step(ds, outs)
    if res_dev is not None:
        out_host = torch.empty(res_dev.shape, dtype=res_dev.dtype).pin_memory()
    elif isinstance(outs, dict):
        out_host = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in outs.items()}
    else:
        out_host = torch.empty(outs.shape, dtype=outs.dtype).pin_memory()
    d2h = (sum(v.numel() * v.element_size() for v in out_host.values()) if isinstance(out_host, dict)
           else out_host.numel() * out_host.element_size())

    def e2e_step():
        for s, hs in zip(ds, host):
            s.src.copy_(hs["src"], non_blocking=True)
            s.tgt.copy_(hs["tgt"], non_blocking=True)
            if hs["perms"] is not None:
                s.perms.copy_(hs["perms"], non_blocking=True)
        r = step(ds, outs)
        if r is not None:
            out_host.copy_(r, non_blocking=True)
        elif isinstance(outs, dict):
            for k in outs:
                out_host[k].copy_(outs[k], non_blocking=True)
        else:
            out_host.copy_(outs, non_blocking=True)

    e2e_steps = max(3, args.steps // 2)
    e2e_step()
    torch.cuda.synchronize()
    barrier()
    eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    for a, b in eev:
        flush.zero_()
        a.record()
        e2e_step()
        b.record()
    torch.cuda.synchronize()
    barrier()
    e2e_ms = sum(a.elapsed_time(b) for a, b in eev)
    if ws > 1:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = {"value": copies * pe_step * e2e_steps / (e2e_ms / 1e3), "unit": "pair-evals/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "te_estimates_per_s": copies * n_est * e2e_steps / (e2e_ms / 1e3),
           "ms_per_step": e2e_ms / e2e_steps}

    # ---- per-instance launches against one batched launch on a sub-batch, same GPU and stream:
    # (a) one launch per estimate of the unshared persistent kernel, (b) one launch of the same
    # kernel for the whole sub-batch (the like-for-like ratio: same kernel, same staging), (c) the
    # default batched path (target parts shared)
    per = None
    if not args.no_per_launch and ws == 1:
        if surrogate:
            per_t = lane_ops(w) // len(w.t_starts[0])
            n_t_sub = max(1, min(len(w.t_starts[0]), args.per_launch_instances // ((w.S + 1) * _scan_factor(w))))
            n_t_sub = max(1, min(n_t_sub, int(2.0e12 // max(1, per_t))))
            wsub = I.Workload(w.name, w.series, w.instances[: n_t_sub * (w.S + 1)], w.k,
                              [w.t_starts[0][:n_t_sub]], w.window, w.S, extra=dict(w.extra))
            if scan:  # a few delays of the first window keep the unbatched run short
                n_u_sub = max(1, min(_scan_factor(w), args.per_launch_instances // (w.S + 1)))
                wsub.extra = dict(u_lo=scan[0], u_hi=scan[0] + n_u_sub - 1)
        else:
            wsub = I.Workload(w.name, w.series, w.instances[: args.per_launch_instances], w.k)
        sub_step, sub_outs, _ = make_runner(te, torch, h, wsub, dev)
        arms = (("per_instance_launch", True, te.SHARE_NONE), ("batched_same_kernel", False, te.SHARE_NONE),
                ("batched_default", False, share))
        pe_sub = 2 * pair_evals(wsub)
        n_sub = len(wsub.instances) * _scan_factor(wsub)
        per = {"instances": n_sub}
        for name, per_inst, mode in arms:
            te.te_set_batching(h, per_inst)
            te.te_set_sharing(h, mode)
            sub_step(ds, sub_outs)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record()
            sub_step(ds, sub_outs)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            pth = te.te_last_paths(h)
            per[name] = {"value": pe_sub / (ms / 1e3), "unit": "pair-evals/s", "te_estimates_per_s": n_sub / (ms / 1e3),
                         "ms": round(ms, 3), "kernel_launches": te.te_last_launch_count(h),
                         "kernel_path": {k: v for k, v in zip(PATH_KERNELS, pth) if v},
                         "launch": "one per estimate" if per_inst else "one persistent launch (CUDA graph)"}
        te.te_set_batching(h, False)
        te.te_set_sharing(h, share)
        per["batched_vs_per_launch"] = round(per["per_instance_launch"]["ms"] / per["batched_same_kernel"]["ms"], 2)
        per["default_vs_per_launch"] = round(per["per_instance_launch"]["ms"] / per["batched_default"]["ms"], 2)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)

    line = {
        "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "dtype": "f32", "data": "synthetic",
        "vs_baseline": (round(value / PAPER_CHUNK_TITAN_PAIR_RATE, 2) if args.workload == "paper-chunk" else None),
        "config": {"workload": spec["desc"], "estimates_per_step": n_est,
                   "pair_evals_per_step": pe_step, "k": w.k,
                   "l2": "256 MiB buffer written between timed steps (inputs smaller than L2)",
                   "per_rank": ("a cost-balanced share of the analysis starts / estimates per rank, results "
                                "all-gathered (strong scaling)") if sharded else
                               ("every rank runs the full workload (weak scaling)" if ws > 1 else "one GPU"),
                   "launch_shape": None if tuned is None else {"threads": tuned[0], "queries_per_thread": tuned[1],
                                                               "chosen_by": "--shape" if args.shape else "te_autotune"}},
        "te_estimates_per_s": te_rate,
        "search": {"mode": "sorted sweep" if swept else "exhaustive",
                   "paths": {k: v for k, v in zip(PATH_KERNELS, paths)},
                   "pair_evals_executed_per_step": exec_pairs,
                   "executed_vs_algorithmic": round(exec_pairs / max(1, pe_rank), 4),
                   "passes": passes,
                   "target_part_sharing": {"bundles": bundles, "alu_ops_executed_per_step": alu_ops,
                                           "alu_ops_vs_2D_per_pair": round(alu_ops / max(1, exec_ops), 4)}},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "per_launch": per,
        "batched_vs_per_launch": None if per is None else per["batched_vs_per_launch"],
        "impl": "ours",
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------- reference
def bench_reference(args):
    """The oracle (plain C, host threads) on the host cores: the reference arm of this tier."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1401_4068_gb300 import inputs as I
    spec = WORKLOADS[args.workload]
    w = load_workload(spec)
    threads = oracle.default_threads()
    per_step = max(threads, args.reference_instances)
    if max(w.n_points(i) for i in w.instances) > LARGE_N:
        per_step = 4  # sampled query points of a few large estimates per step
    for s in range(args.warmup):
        run_oracle_sample(w, I.sample_instances(w, threads, seed=100 + s), threads)
    pe_tot, dt_tot, n_tot = 0, 0.0, 0
    for s in range(args.steps):
        pe, dt, m = run_oracle_sample(w, I.sample_instances(w, per_step, seed=200 + s), threads)
        pe_tot += pe
        dt_tot += dt
        n_tot += m
    value = pe_tot / dt_tot
    sample = (f"{per_step} cost-stratified estimates of {len(w.instances)} per step (estimates over {LARGE_N} "
              f"points on {LARGE_N_QUERIES} sampled query points each), both passes")
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt_tot * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": spec["desc"], "estimates_per_step": per_step, "k": w.k},
        "impl": "reference",
        "te_estimates_per_s": n_tot / dt_tot,
        "cpu_baseline": {"value": value, "unit": "pair-evals/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "pair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c5")
    ap.add_argument("--scaling", choices=["strong", "weak"], default="strong",
                    help="with several ranks: shard the workload (strong) or replicate it (weak)")
    ap.add_argument("--per-launch-instances", type=int, default=2002)
    ap.add_argument("--no-per-launch", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--exhaustive", action="store_true", help="exhaustive search instead of the sorted sweep")
    ap.add_argument("--no-sharing", action="store_true", help="no target-part sharing across estimates")
    ap.add_argument("--sharing", choices=sorted(SHARING), default="auto",
                    help="target-part sharing: auto (lanes for large groups, bundles for small), lanes, bundles, none")
    ap.add_argument("--shape", default=None, help="fixed launch shape THREADSxQPT instead of autotuning")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-instances", type=int, default=32)
    args = ap.parse_args()
    if args.impl == "ours":
        args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
