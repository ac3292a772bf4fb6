"""Throughput of aggregation over dominated points on GB300.

Default workload (one step = one forward pass of the whole pipeline):
m = 2, |D| = |Q| = 2^24, float32 coordinates uniform in [0, 1) with 25% of
the points quantised to a 2^-16 grid (ties), float32 weights N(0, 1),
F = sum.  value = queries per second (whole job: all ranks' queries / the
slowest rank's time).  The line also carries:
  roofline      the dominant HBM-bound kernel (the points' radix pass: the
                records of this workload never reach HBM) against the
                measured HBM copy bandwidth; largest_kinds lists the kernel
                kinds by device time (the shared-memory level kernels k_top
                and k_group among them);
  cpu_baseline  the CPU oracle on bounded samples: its sort-and-scan (the
                paper's pipeline in list form, one thread) and its brute force
                (all host cores);
  e2e           the same metric through domagg_forward_host (host buffers,
                copies inside the timed region);
  fwd_bwd       forward + backward (the autograd step) on the same workload;
  m3            forward on the m = 3 workload (|D| = |Q| = 2^21, Gaussian
                mixture int32 coordinates, int64 weights).
``--impl reference`` times the CPU oracle's sort-and-scan alone, step by
step, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s for dominance-sum at m=2,3 (n=2^24); fwd+bwd; % of HBM roofline"
WORKLOAD = "m2_nD2^24_nQ2^24_f32coords_25pct_tied_f32w_sum"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=2**24, help="|D| = |Q| of the m=2 workload")
    ap.add_argument("--n3", type=int, default=2**21, help="|D| = |Q| of the m=3 workload")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU time of the baseline sample")
    ap.add_argument("--no-extras", action="store_true", help="skip fwd_bwd, m3, batch, e2e and the CPU baseline")
    ap.add_argument("--batch-k", type=int, default=4096, help="instances of the batch workload")
    ap.add_argument("--only-batch", action="store_true", help="print the batch line alone (e.g. --batch-k 4096)")
    ap.add_argument("--only-m3", action="store_true", help="print the m = 3 line alone (e.g. --n3 524288)")
    ap.add_argument("--no-autotune", action="store_true", help="planned batch without the launch-shape autotuner")
    ap.add_argument("--variant", default="improved", choices=["improved", "wavelet"],
                    help="formulation of the timed m=2 step: the Sec. 5 record pipeline (default) or the "
                         "level-wise passes")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def profiled_traffic(bytes_per_launch: float, source: str = "k_radix.cuh",
                     profile: str = "k_onesweep_points_m2_n2e24.md"):
    """DRAM bytes of one launch of the dominant HBM-bound kernel (a radix
    pass, or a level-wise pass): the committed ncu summary's measured DRAM
    bytes per algorithmic byte, times this run's algorithmic bytes per
    launch; None if the kernel source changed since that capture."""
    import hashlib
    src = os.path.join(ROOT, "paper_2305_16751_gb300", "csrc", source)
    prof = os.path.join(ROOT, "profiles", profile)
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        fields = dict(ln.split(":", 1) for ln in open(prof) if ln.startswith(("kernel_source", "traffic_per")))
    except (OSError, ValueError):
        return None
    if fields.get("kernel_source_sha256_16", "").strip() != digest:
        return None
    return float(fields["traffic_per_algorithmic_byte"]) * bytes_per_launch


def kind_roofline(kinds: dict, kind: str, peak: float, peak_src: str, kernel: str):
    """Roofline object of one kernel kind from the library's per-launch
    timing (CUDA events on the launching stream): its algorithmic bytes per
    launch over its average launch time, against the measured HBM peak."""
    k = kinds.get(kind, {"ms": 0.0, "bytes": 0.0, "launches": 0})
    n = max(k["launches"], 1)
    achieved = k["bytes"] / max(k["ms"], 1e-9) / 1e6
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "peak_source": peak_src, "kernel": kernel, "launch_ms": k["ms"] / n,
            "bytes_per_launch": k["bytes"] / n}


def step_model(n_points: int, records: int, n_queries: int, ms: float, peak: float, m: int = 2):
    """The whole step against the per-query byte model of the hot-path scope
    (what the pipeline must move at minimum): m = 2, 4-byte keys and
    payloads, 8-bit digits: 170 B per point, 72 B per record, 4 B per query;
    m = 3, 8-byte keys, four 11-bit passes: 176 B per record."""
    b = 170.0 * n_points + 72.0 * records + 4.0 * n_queries if m == 2 else 176.0 * records
    return {"bytes": b, "ms": ms, "achieved_gbs": b / (ms * 1e6), "frac": b / (ms * 1e6) / peak}


def _sortscan_sample(p, n: int):
    """The first n data points and n queries of the workload (the same
    distribution at a size the CPU oracle completes)."""
    return p.D[:n], p.Q[:n], (None if p.w is None else p.w[:n])


def cpu_baseline(p, seconds: float):
    """The oracle as it stands on the host cores, on bounded samples of the
    workload.  Headline: the paper's algorithm in list form (oracle_sortscan:
    dense ranks, the flat map, one lexicographic sort, the segmented scans;
    sequential, one thread) on the first n data points and n queries, n
    doubled until one run takes about a third of `seconds`.  Beside it the
    brute-force definition (OpenMP, all host cores) on a random sample of
    queries against all data points."""
    import numpy as np

    import oracle
    n, spent, T = 1 << 12, 0.0, 0
    while True:
        D, Q, w = _sortscan_sample(p, n)
        t0 = time.perf_counter()
        _, T = oracle.sortscan(D, Q, w, p.op)
        spent = max(time.perf_counter() - t0, 1e-6)
        if spent >= seconds / 3 or 2 * n > min(p.Q.shape[0], 1 << 19):
            break
        n *= 2
    line = {"value": n / spent, "unit": "queries/s", "cores": 1, "kind": "oracle",
            "sample": f"sort-and-scan oracle (the paper's pipeline in list form, one thread) on the first {n} "
                      f"data points and {n} queries of the workload ({T} flat-map records), {spent:.2f} s",
            "seconds": spent, "n": n}
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(0)
    k = min(p.Q.shape[0], 64)
    for _ in range(4):  # grow the sample until one run takes at least a third of the target
        qi = rng.choice(p.Q.shape[0], size=k, replace=False)
        t0 = time.perf_counter()
        oracle.brute(p.D, p.Q[qi], p.w, p.op, threads=threads)
        bt = max(time.perf_counter() - t0, 1e-3)
        if bt >= seconds / 3 or k == p.Q.shape[0]:
            break
        k = int(min(p.Q.shape[0], max(k + 1, k * seconds / 3 / bt)))
    line["all_cores"] = {"value": k / bt, "unit": "queries/s", "cores": threads, "kind": "oracle",
                         "sample": f"brute-force definition (OpenMP) on {k} random queries of the workload, each "
                                   f"against all {p.D.shape[0]} data points, {bt:.2f} s"}
    return line


REFERENCE_N = 1 << 16  # per side: one sort-and-scan step of about a second on one host core


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle's sort-and-scan (the paper's
    algorithm in list form, sequential) timed step by step on a bounded sample
    of the workload -- the first REFERENCE_N data points and queries --
    since the full 2^24 workload would need tens of GB of records and many
    minutes per step on the host."""
    if rank != 0:
        return
    import oracle
    from paper_2305_16751_gb300 import workloads
    p = workloads.tied_floats(n=args.n)
    n = min(REFERENCE_N, args.n)
    D, Q, w = _sortscan_sample(p, n)
    times, T = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, T = oracle.sortscan(D, Q, w, p.op)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    v = n / sec
    sample = (f"sort-and-scan oracle (one thread) on the first {n} data points and {n} queries of the "
              f"{WORKLOAD} workload ({T} flat-map records) per step")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "m": 2, "op": "sum", "sample": sample},
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batch(args, dev, stream, torch, domagg, workloads):
    """k instances of the batch workload (m in {2, 3}, |D| = |Q| log-uniform
    in [256, 2^18], int32 coordinates uniform in [0, 2^31), float32 weights,
    F = sum) in one domagg_batch call, against a loop of domagg_forward calls
    over the same instances, and as a planned batch replayed from a CUDA
    graph."""
    probs = workloads.batch_instances(k=args.batch_k)
    inst = [(torch.from_numpy(p.D).to(dev), torch.from_numpy(p.Q).to(dev), torch.from_numpy(p.w).to(dev))
            for p in probs]
    nq = sum(p.Q.shape[0] for p in probs)
    npts = sum(p.Q.shape[0] + p.D.shape[0] for p in probs)
    tb = timed_steps(lambda: domagg.batch(inst, "sum"), 2, 1, stream, torch)
    b_ms = statistics.mean(tb)
    # one more call with the library's per-kind timing, and each half of the
    # batch (the m = 2 and the m = 3 instances) on its own
    h = domagg.handle(dev.index or 0)
    domagg.domagg_timing_enable(h, True)
    domagg.domagg_timing_read(h)
    domagg.batch(inst, "sum")
    kb = domagg.domagg_timing_read(h)
    domagg.domagg_timing_enable(h, False)
    by_m = {}
    for m in (2, 3):
        part = [t for t in inst if t[0].shape[1] == m]
        if part:
            by_m[f"m{m}_instances"] = {"instances": len(part), "points": sum(t[0].shape[0] + t[1].shape[0] for t in part),
                                       "ms": statistics.mean(timed_steps(lambda: domagg.batch(part, "sum"), 2, 1,
                                                                         stream, torch))}

    def loop():
        for D, Q, w in inst:
            domagg.forward(D, Q, w, "sum")

    tl = timed_steps(loop, 1, 1, stream, torch)
    l_ms = statistics.mean(tl)
    # the planned batch captured once in a CUDA graph, then replayed
    plan = domagg.BatchPlan(inst, "sum", headroom=0.05)
    tuned_ms = None if args.no_autotune else plan.autotune()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.run()
    tg = timed_steps(graph.replay, 3, 1, stream, torch)
    plan.status()
    g_ms = statistics.mean(tg)
    plan_gb = plan.workspace_bytes() / 1e9
    plan.close()
    return {"value": nq / (b_ms / 1e3), "unit": "queries/s", "ms_per_step": b_ms, "instances": len(probs),
            "points": npts, "queries": nq, "per_instance_loop": {"value": nq / (l_ms / 1e3), "ms_per_step": l_ms},
            "graph_replay": {"value": nq / (g_ms / 1e3), "ms_per_step": g_ms, "plan_workspace_gb": plan_gb,
                             "autotuned_ms": tuned_ms},
            "phase_ms": {k: round(v["ms"], 3) for k, v in kb.items() if v["ms"] > 0}, "by_m": by_m,
            "workload": f"{len(probs)} instances, m in {{2,3}} 50/50, |D|=|Q| log-uniform [256, 2^18], "
                        "int32 coords U[0,2^31), f32 w, sum"}


def bench_variants(args, dev, stream, torch, domagg, workloads):
    """The widened rows: the basic (unimproved) variant of Sec. 4 against the
    Sec. 5 pipeline on the same m = 2 problem, ECDF counting (D = Q, every
    coordinate non-strict) at m = 3, and MIN."""
    import numpy as np
    res = {}
    rng = np.random.default_rng(2305167517)
    n = args.n // 16
    D = torch.from_numpy((rng.integers(0, 1 << 24, size=(n, 2)) * 2.0**-24).astype(np.float32)).to(dev)
    Q = torch.from_numpy((rng.integers(0, 1 << 24, size=(n, 2)) * 2.0**-24).astype(np.float32)).to(dev)
    w = torch.from_numpy(rng.integers(-1000, 1001, size=n).astype(np.int64)).to(dev)
    for name, variant in (("improved", "improved"), ("basic", "basic")):
        t = timed_steps(lambda: domagg.forward(D, Q, w, "sum", variant=variant), 3, 2, stream, torch)
        ms = statistics.mean(t)
        res[f"m2_{name}"] = {"value": n / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
                             "records": domagg.stats(dev.index or 0)["n_records"]}
    res["m2_workload"] = f"|D|=|Q|={n}, float32 U[0,1) on the 2^-24 grid, int64 sum"
    del D, Q, w
    p = workloads.ecdf_samples(n=args.n // 16, m=3)
    X = torch.from_numpy(p.D).to(dev)
    t = timed_steps(lambda: domagg.forward(X, X, None, "count", nonstrict=7), 3, 2, stream, torch)
    ms = statistics.mean(t)
    res["ecdf_m3"] = {"value": X.shape[0] / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
                      "records": domagg.stats(dev.index or 0)["n_records"],
                      "workload": f"D=Q={X.shape[0]} points, m=3, N(0,1) on a 2^-8 grid, count, all coordinates <="}
    del X
    pm = workloads.tied_floats(n=args.n, weights="i32")
    Dm, Qm, wm = (torch.from_numpy(a).to(dev) for a in (pm.D, pm.Q, pm.w))
    om = torch.empty(Qm.shape[0], dtype=torch.int32, device=dev)
    t = timed_steps(lambda: domagg.forward(Dm, Qm, wm, "min", out=om), 3, 2, stream, torch)
    ms = statistics.mean(t)
    res["min_m2"] = {"value": Qm.shape[0] / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
                     "workload": "tied_floats 2^24, int32 weights, min"}
    return res


def _pow2(n: int) -> str:
    return f"2^{n.bit_length() - 1}" if n > 0 and n & (n - 1) == 0 else str(n)


def bench_m3(args, dev, stream, torch, domagg, workloads):
    """The m = 3 workload (Gaussian-mixture int32 coordinates, int64 sum):
    forward steps, then one call with the library's per-kind timing; its
    roofline is the records radix pass (64-bit and 32-bit key classes)."""
    peak, peak_src = peaks()
    h = domagg.handle(dev.index or 0)
    p3 = workloads.gaussian_mixture_i32(n=args.n3)
    D3, Q3, w3 = (torch.from_numpy(a).to(dev) for a in (p3.D, p3.Q, p3.w))
    o3 = torch.empty(p3.Q.shape[0], dtype=torch.int64, device=dev)
    t3 = timed_steps(lambda: domagg.forward(D3, Q3, w3, "sum", out=o3), max(3, args.steps // 2), 2, stream, torch)
    m3_ms = statistics.mean(t3)
    st3 = domagg.stats(dev.index or 0)
    domagg.domagg_timing_enable(h, True)
    domagg.domagg_timing_read(h)
    domagg.forward(D3, Q3, w3, "sum", out=o3)
    k3 = domagg.domagg_timing_read(h)
    domagg.domagg_timing_enable(h, False)
    roof = kind_roofline(k3, "sort_records", peak, peak_src,
                         "k_onesweep (records radix pass, 64-bit and 32-bit key classes)")
    if args.n3 == 2**21:  # the profile's workload: its DRAM bytes per algorithmic byte
        roof["traffic"] = profiled_traffic(roof["bytes_per_launch"], "k_radix.cuh", "k_onesweep_records_m3_n2e21.md")
    return {"value": p3.Q.shape[0] / (m3_ms / 1e3), "unit": "queries/s", "ms_per_step": m3_ms,
            "workload": f"m3_nD{_pow2(args.n3)}_nQ{_pow2(args.n3)}_gmm_i32coords_i64w_sum", "records": st3["n_records"],
            "record_passes": st3["record_passes"], "phase_ms": {k: v["ms"] for k, v in k3.items()},
            "roofline": roof,
            "step_model": step_model(2 * args.n3, st3["n_records"], args.n3, m3_ms, peak, m=3)}


def bench_wavelet(args, D, Q, w, out, dev, stream, torch, domagg):
    """The level-wise formulation (variant "wavelet") on the headline
    workload: no flat-map records, two rank levels per pass over 16-byte
    points.  Its roofline: the passes' algorithmic bytes (16 B read + 16 B
    written per point and pass; the first pass gathers ranks and weights, the
    last writes outputs) over their summed device time."""
    def step():
        domagg.forward(D, Q, w, "sum", out=out, variant="wavelet")

    t = timed_steps(step, max(3, args.steps // 2), 3, stream, torch)
    ms = statistics.mean(t)
    st = domagg.stats(dev.index or 0)
    h = domagg.handle(dev.index or 0)
    domagg.domagg_timing_enable(h, True)
    domagg.domagg_timing_read(h)
    step()
    kinds = domagg.domagg_timing_read(h)
    domagg.domagg_timing_enable(h, False)
    wv = kinds.get("wavelet", {"ms": 0.0, "bytes": 0.0, "launches": 1})
    peak, peak_src = peaks()
    achieved = wv["bytes"] / max(wv["ms"], 1e-9) / 1e6
    return {"value": Q.shape[0] / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
            "workload": WORKLOAD, "passes": st["record_passes"], "rank_bits": st["rank_bits"][0],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": profiled_traffic(wv["bytes"] / max(wv["launches"], 1), "k_wavelet.cuh",
                                                     "k_wavelet_pass_m2_n2e22.md"),
                         "peak_source": peak_src, "kernel": "k_wavelet_pass (all passes)",
                         "launch_ms": wv["ms"] / max(wv["launches"], 1),
                         "bytes_per_launch": wv["bytes"] / max(wv["launches"], 1)},
            "phase_ms": {k: v["ms"] for k, v in kinds.items() if v["ms"] > 0}}


def job_throughput(local_ms: float, units_per_rank: int, world: int, device=None):
    """Whole-job throughput: every rank's units over the slowest rank's time
    (max over ranks of the timed region).  Returns (units/s, max ms)."""
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return world * units_per_rank / (ms / 1e3), ms


def timed_steps(fn, steps, warmup, stream, torch):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.only_batch or args.only_m3:
        import torch
        from paper_2305_16751_gb300 import domagg, workloads
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        if args.only_batch:
            print(json.dumps({"batch": bench_batch(args, dev, stream, torch, domagg, workloads)}), flush=True)
        else:
            print(json.dumps({"m3": bench_m3(args, dev, stream, torch, domagg, workloads)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import numpy as np
    import torch

    from paper_2305_16751_gb300 import domagg, workloads

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    p = workloads.tied_floats(n=args.n)
    D = torch.from_numpy(p.D).to(dev)
    Q = torch.from_numpy(p.Q).to(dev)
    w = torch.from_numpy(p.w).to(dev)
    out = torch.empty(p.Q.shape[0], dtype=torch.float32, device=dev)
    h = domagg.handle(local)

    if world > 1:
        # the forward split over the ranks: each rank its shard of the flat
        # map, one all-gather of the (float-float) partials, the join
        from paper_2305_16751_gb300 import shards

        def step():
            shards.forward_distributed(D, Q, w, "sum")
    else:
        def step():
            domagg.forward(D, Q, w, "sum", out=out, variant=args.variant)

    # timed region: forward steps, with per-launch events inside the library
    step()
    torch.cuda.synchronize()
    domagg.domagg_timing_enable(h, True)
    domagg.domagg_timing_read(h)  # reset
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        times = timed_steps(step, args.steps, args.warmup, stream, torch)
    kinds = domagg.domagg_timing_read(h)
    domagg.domagg_timing_enable(h, False)
    # one job answers the |Q| queries per step, split over the ranks (strong scaling)
    value, total_ms = job_throughput(sum(times), p.Q.shape[0] * args.steps / world, world, dev)
    ms = total_ms / args.steps
    st = domagg.stats(local)
    # kinds were logged over warmup + steps calls
    calls = args.warmup + args.steps
    launches = sum(v["launches"] for k, v in kinds.items() if k not in ("h2d", "d2h")) // calls * args.steps
    peak, peak_src = peaks()
    dom_kind = "wavelet" if args.variant == "wavelet" else "sort_points"
    dom = kinds.get(dom_kind, {"ms": 0.0, "bytes": 0.0, "launches": 1})
    achieved = dom["bytes"] / max(dom["ms"], 1e-9) / 1e6  # GB/s
    phase_ms = {k: v["ms"] / calls for k, v in kinds.items()}

    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "m": 2, "op": "sum", "weights": "f32",
                       "parallelism": f"flat map sharded over {world} GPUs, one all-gather of the partials"
                       if world > 1 else "1 GPU",
                       "records": st["n_records"], "records_in_shared_memory": st["n_records_shared"],
                       "record_passes": st["record_passes"],
                       "l2": f"inputs ({(p.D.nbytes + p.Q.nbytes + p.w.nbytes) >> 20} MB) and the library's "
                             f"workspace ({st['workspace_bytes'] >> 20} MB) exceed the 129 MB L2; no flush"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": profiled_traffic(dom["bytes"] / max(dom["launches"], 1),
                                                     *(("k_wavelet.cuh", "k_wavelet_pass_m2_n2e22.md")
                                                       if args.variant == "wavelet" else ())),
                         "peak_source": peak_src,
                         "kernel": "k_wavelet_pass (level-wise pass)" if args.variant == "wavelet"
                         else "k_onesweep (point radix pass: first coordinate and last coordinate)",
                         "launch_ms": dom["ms"] / max(dom["launches"], 1),
                         "bytes_per_launch": dom["bytes"] / max(dom["launches"], 1)},
            "gpu_launches": launches,
            "phase_ms": phase_ms,
            "largest_kinds": sorted(((k, round(v, 4)) for k, v in phase_ms.items() if k not in ("h2d", "d2h")),
                                    key=lambda kv: -kv[1])[:4],
            "step_model": step_model(2 * args.n, st["n_records"], args.n, ms, peak)}
    clocks = clk.summary()
    line["clocks"] = clocks

    if not args.no_extras and rank == 0:
        # forward + backward (the autograd step) on the same workload
        wg = w.clone().requires_grad_(True)
        grad_out = torch.randn(p.Q.shape[0], device=dev, generator=torch.Generator(dev).manual_seed(0))

        def fb():
            o = domagg.dominance_sum(D, Q, wg)
            o.backward(grad_out)

        tfb = timed_steps(fb, max(3, args.steps // 2), 2, stream, torch)
        fb_ms = statistics.mean(tfb)
        domagg.domagg_timing_enable(h, True)
        domagg.domagg_timing_read(h)
        fb()
        kfb = domagg.domagg_timing_read(h)
        domagg.domagg_timing_enable(h, False)
        dom_fb = max((k for k in kfb if k not in ("h2d", "d2h", "small")), key=lambda k: kfb[k]["ms"])
        line["fwd_bwd"] = {"value": p.Q.shape[0] / (fb_ms / 1e3), "unit": "queries/s", "ms_per_step": fb_ms,
                           "roofline": kind_roofline(kfb, "sort_points", peak, peak_src,
                                                     "k_onesweep (point radix pass), forward and backward"),
                           "largest_kind": dom_fb,
                           "phase_ms": {k: v["ms"] for k, v in kfb.items() if v["ms"] > 0}}

        def fbw():
            o = domagg.dominance_sum(D, Q, wg, 0, "wavelet")
            o.backward(grad_out)

        tfbw = timed_steps(fbw, max(3, args.steps // 2), 2, stream, torch)
        fbw_ms = statistics.mean(tfbw)
        line["fwd_bwd_wavelet"] = {"value": p.Q.shape[0] / (fbw_ms / 1e3), "unit": "queries/s",
                                   "ms_per_step": fbw_ms, "variant": "level-wise formulation"}
        del wg
        line["m3"] = bench_m3(args, dev, stream, torch, domagg, workloads)
        line["wavelet"] = bench_wavelet(args, D, Q, w, out, dev, stream, torch, domagg)
        line["variants"] = bench_variants(args, dev, stream, torch, domagg, workloads)
        line["batch"] = bench_batch(args, dev, stream, torch, domagg, workloads)
        # end to end through the host-buffer entry point
        Dh = torch.from_numpy(p.D).pin_memory()
        Qh = torch.from_numpy(p.Q).pin_memory()
        wh = torch.from_numpy(p.w).pin_memory()
        for _ in range(2):
            domagg.forward_host(Dh, Qh, wh, "sum", device=local)
        te = []
        for _ in range(max(3, args.steps // 2)):
            t0 = time.perf_counter()
            domagg.forward_host(Dh, Qh, wh, "sum", device=local)
            te.append(time.perf_counter() - t0)
        e2e_s = statistics.mean(te)
        line["e2e"] = {"value": world * p.Q.shape[0] / e2e_s, "unit": "queries/s",
                       "h2d_bytes_per_step": int(p.D.nbytes + p.Q.nbytes + p.w.nbytes),
                       "d2h_bytes_per_step": int(p.Q.shape[0] * 4), "ms_per_step": e2e_s * 1e3}
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
