"""Benchmark of the FastSimilarityGraph hot path on GB300.

One step = the whole path of Algorithm 2 on one synthetic point set resident
in HBM: tree rebuild (fsg_tree_update), then fsg_build_graph (bin-pass KDE,
degrees, descent of all n*L samples, leaf finish with weights, SET edge list).

Workload: Gaussian mixture, n = 100,000, d = 10, 10 equal-weight unit blobs
with centres uniform in [-10,10]^10, sigma = 1.5 (gamma = 1/(2 sigma^2)),
L = 64 samples per point, Philox seed 0.

Printed (one JSON line, rank 0): sampled edges/s = n*L / step time (device,
CUDA events, L2 flushed between steps by writing a 512 MB buffer), the e2e
figure through the host-buffer entry point (copies inside the timed region),
the roofline of the dominant kernel (bin pass, ALU bound) and the oracle's
CPU throughput on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sampled graph edges/s & Gkernel-evals/s vs plain FP32 GPU path; p50/p99 latency"
UNIT = "sampled edges/s"
OUTPUTS = ("edge list (src, dst, FP32 weight) and FP64 degrees written every step; the optional per-sample "
           "neighbour and flag arrays are not requested")
WORKLOAD = dict(workload="gaussian_mixture n=100000 d=10 k=10 box=10 sigma=1.5 L=64 seed=0", n=100_000, d=10,
                sigma=1.5, L=64, seed=0, edges="SET", self_term="EXCLUDE", l2="flushed (512 MB write) between steps",
                outputs=OUTPUTS)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
MUFU_EX2_PER_SM = 16


def alu_peak_evals(d: int, mhz: float = SM_MAX_MHZ, ops: int = 0) -> float:
    """ALU bound of the bin pass, in kernel evaluations/s: per evaluation the
    FP32 pipe executes d subtractions, d multiply-adds, one scale and one
    accumulate per row the value is added to (2d+2 lane operations, 2d+3 when
    each value serves two rows) and the MUFU one ex2."""
    fp32 = SM_COUNT * FP32_LANES_PER_SM * mhz * 1e6 / (ops or 2 * d + 2)
    mufu = SM_COUNT * MUFU_EX2_PER_SM * mhz * 1e6
    return min(fp32, mufu)


DIGITS = dict(workload="digit_like n=70000 d=784 (10 prototypes, 8-bit) sigma=median/2 L=64 seed=0", n=70_000,
              d=784, sigma=None, L=64, seed=0, edges="SET", self_term="EXCLUDE",
              l2="flushed (512 MB write) between steps", outputs=OUTPUTS)


def make_points(rank: int = 0):
    from paper_2310_13870_gb300 import inputs
    if WORKLOAD["d"] == 784:
        X = inputs.digit_like(n=WORKLOAD["n"], seed=WORKLOAD["seed"] + rank)
        if WORKLOAD["sigma"] is None:
            WORKLOAD["sigma"] = inputs.median_pair_distance(X, m=4096, seed=0) / 2
        return X
    return inputs.gaussian_mixture(n=WORKLOAD["n"], d=WORKLOAD["d"], seed=WORKLOAD["seed"] + rank)


def set_size(n: int):
    """Smaller instance of the same workload (used for profiler captures)."""
    WORKLOAD["n"] = n
    WORKLOAD["workload"] = WORKLOAD["workload"].replace("n=100000", f"n={n}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"fsg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, device=None) -> float:
    """The slowest rank's value (timings are reported as the max over ranks);
    x itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput of `world` independent replicas that each process
    `units_per_rank` units in a step of `ms` milliseconds (the slowest rank's)."""
    return world * units_per_rank / (ms * 1e-3)


def cpu_oracle_throughput(X, n_queries: int, L: int, sigma: float, seed: int, keep: dict = None):
    """The oracle (as it stands) on a bounded sample: the descent of every
    sample of n_queries points plus their degrees, on all host cores.
    Returns (sampled edges/s, seconds, threads); `keep` receives the sampled
    query indices and their FP64 degrees."""
    import oracle as ora
    gam = ora.gamma(sigma)
    q = np.arange(n_queries, dtype=np.int64) * (X.shape[0] // n_queries)
    t0 = time.perf_counter()
    ora.sample(X, gam, L, seed, queries=q)
    deg = ora.degrees(X, gam, queries=q)
    dt = time.perf_counter() - t0
    if keep is not None:
        keep["q"], keep["deg"] = q, deg
    return n_queries * L / dt, dt, ora.num_threads()


def kde_error(deg_gpu, ref) -> dict:
    """Relative error of GPU degrees against the oracle's FP64 degrees."""
    q, want = ref["q"], ref["deg"]
    rel = np.abs(np.asarray(deg_gpu)[q] - want) / want
    return {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()), "queries": int(q.size),
            "kind": "degrees (Eq. 1 over all points) vs the FP64 oracle"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as ora
    ora.build()
    X = make_points(0)
    L, sigma, seed = WORKLOAD["L"], WORKLOAD["sigma"], WORKLOAD["seed"]
    nq = args.ref_queries
    vals = []
    for s in range(args.warmup + args.steps):
        v, dt, threads = cpu_oracle_throughput(X, nq, L, sigma, seed)
        if s >= args.warmup:
            vals.append((v, dt))
    value = statistics.mean(v for v, _ in vals)
    ms = statistics.mean(dt for _, dt in vals) * 1e3
    sample = f"{nq} query points of the n=100000 workload per step (all {L} samples + degrees), extrapolated per edge"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism="oracle on host cores"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_steps(step, steps, stream, flush):
    """CUDA-event times (ms) of `steps` calls of step() on `stream`, with the
    L2 flushed before each."""
    import torch
    out = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def tensor_peak():
    """Measured sustained BF16 tensor peak (TFLOP/s) and where it came from."""
    pf = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pf):
        with open(pf) as f:
            return json.load(f).get("bf16_tflops_sustained", 1700.0), "measured cuBLAS BF16 sustained"
    return 1700.0, "fallback"


def sub_digits(fsg, stream, flush, steps):
    """Digit-image workload (n = 70,000, d = 784, L = 64, sigma = median/2) on
    the exact 8-bit tensor-core path: throughput, bin-pass roofline against
    the tensor peak, degree error against the FP64 oracle on 256 points."""
    import torch
    import oracle as ora
    from paper_2310_13870_gb300 import inputs
    n, d, L, seed = 70_000, 784, 64, 0
    X = inputs.digit_like(n=n, seed=0)
    sigma = inputs.median_pair_distance(X, m=4096, seed=0) / 2
    p = fsg.params(sigma)
    with torch.cuda.stream(stream):
        pts = torch.from_numpy(X).cuda()
        tree = fsg.fsg_build_tree(pts, stream=stream)
        bufs = fsg.GraphBuffers(n, L, with_aux=False)
        bufs.deg = torch.empty(n, dtype=torch.float64, device="cuda")

    # launch shapes picked by the library's autotuner (untimed), as for the headline workload
    fsg.fsg_autotune(tree, p, L, seed, reps=3, stream=stream)

    def step():
        fsg.fsg_tree_update(tree, pts, stream=stream)
        fsg.fsg_build_graph(tree, p, L, seed, bufs=bufs, stream=stream)

    for _ in range(3):
        step()
    fsg.fsg_profile(tree, True)
    kde = []
    ms = []
    for _ in range(steps):
        ms += timed_steps(step, 1, stream, flush)
        kde.append(fsg.fsg_profile_read(tree)[0]["kde_bins"])
    fsg.fsg_profile(tree, False)
    assert fsg.fsg_sync(tree, stream=stream) == 0
    st = fsg.stats_dict(bufs)
    t = statistics.mean(ms)
    peak, basis = tensor_peak()
    pairs = fsg.fsg_bin_pass_evals(tree, p)  # executed (query, point) pairs: each pair once off the diagonal
    achieved = 2.0 * pairs * d / (statistics.mean(kde) * 1e-3) / 1e12
    q = np.random.Generator(np.random.PCG64(21)).choice(n, size=256, replace=False)
    want = ora.degrees(X, ora.gamma(sigma), queries=q)
    rel = np.abs(bufs.deg.cpu().numpy()[q] - want) / want
    # the same input in split precision (three-part BF16 operands, six
    # products per coordinate, the FP32-data form at d > 64)
    ps = fsg.params(sigma, precision=fsg.FSG_PREC_SPLIT_BF16)
    fsg.fsg_autotune(tree, ps, L, seed, reps=3, stream=stream)  # its own launch shapes (untimed)

    def step_split():
        fsg.fsg_tree_update(tree, pts, stream=stream)
        fsg.fsg_build_graph(tree, ps, L, seed, bufs=bufs, stream=stream)

    for _ in range(3):
        step_split()
    fsg.fsg_profile(tree, True)
    skde, sms = [], []
    for _ in range(steps):
        sms += timed_steps(step_split, 1, stream, flush)
        skde.append(fsg.fsg_profile_read(tree)[0]["kde_bins"])
    fsg.fsg_profile(tree, False)
    assert fsg.fsg_sync(tree, stream=stream) == 0
    sst = fsg.stats_dict(bufs)
    srel = np.abs(bufs.deg.cpu().numpy()[q] - want) / want
    dpad = 64 * ((d + 63) // 64)
    spairs = sst["n_bin_evals"]
    sflops = 12.0 * dpad * spairs  # six BF16 products over the padded coordinates, per executed pair
    sach = sflops / (statistics.mean(skde) * 1e-3) / 1e12
    st_split = {"precision": "split: three-part BF16 operands, six tcgen05 products per coordinate (FP32 data form)",
                "value": n * L / (statistics.mean(sms) * 1e-3), "unit": UNIT, "ms_per_step": statistics.mean(sms),
                "flagged_samples": sst["n_flagged"], "flag_eps": 2.0 ** -10,
                "roofline": {"bound": "tensor", "kernel": "kde_bins_tc_kernel (symmetric, split operands)",
                             "achieved": sach, "peak": peak, "unit": "TFLOP/s", "frac": sach / peak,
                             "kde_bins_ms": statistics.mean(skde), "executed_pairs": int(spairs),
                             "flops_per_launch": sflops, "peak_basis": basis},
                "kde_error": {"max_rel": float(srel.max()), "mean_rel": float(srel.mean()), "queries": int(q.size),
                              "kind": "degrees vs the FP64 oracle"}}
    tree.close()
    return {"workload": "digit_like n=70000 d=784 (10 prototypes, 8-bit) sigma=median/2 L=64 seed=0",
            "precision": "exact 8-bit tcgen05 bin pass (BF16 products of k/255 data, FP32 accumulate)",
            "value": n * L / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "steps": steps,
            "flagged_samples": st["n_flagged"], "edges_per_step": int(bufs.m.item()),
            "roofline": {"bound": "tensor", "kernel": "kde_bins_tc_kernel (symmetric)", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "kde_bins_ms": statistics.mean(kde),
                         "executed_pairs": int(pairs), "flops_per_launch": 2.0 * pairs * d,
                         "algorithmic_pairs": n * n, "peak_basis": basis},
            "kde_error": {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()), "queries": int(q.size),
                          "kind": "degrees (Eq. 1 over all points) vs the FP64 oracle"},
            "split_precision": st_split}


def sub_seg_batch(fsg, stream, flush, steps):
    """64 segmentation-shaped images (h 160..321, w = min(481, 1.5 h), d = 5,
    sigma = 0.05, L = 48) as one batch replayed from a CUDA graph: throughput,
    executed bin-pass evaluations per second of the whole step against the
    d = 5 FP32 bound, degree error on 64 points of four images."""
    import torch
    import oracle as ora
    from paper_2310_13870_gb300 import inputs
    imgs = inputs.segmentation_batch(count=64)
    L, sigma = 48, 0.05
    with torch.cuda.stream(stream):
        sets = [(torch.from_numpy(X).cuda(), fsg.params(sigma), L, 1000 + i) for i, X in enumerate(imgs)]
        batch = fsg.Batch(sets, streams=4, capture=True, stream=stream)
    for _ in range(3):
        batch.run(stream=stream)
    stream.synchronize()
    ms = timed_steps(lambda: batch.run(stream=stream), steps, stream, flush)
    t = statistics.mean(ms)
    n_tot = sum(int(X.shape[0]) for X in imgs)
    bin_evals = 0
    for (pts, p, _, _) in sets:
        tr = fsg.fsg_build_tree(pts, stream=stream)
        bin_evals += fsg.fsg_bin_pass_evals(tr, p)
        tr.close()
    peak = alu_peak_evals(5, ops=2 * 5 + 3) / 1e9
    achieved = bin_evals / (t * 1e-3) / 1e9
    errs = []
    for k in (0, 21, 42, 63):
        X = imgs[k]
        q = np.random.Generator(np.random.PCG64(50 + k)).choice(X.shape[0], size=64, replace=False)
        want = ora.degrees(X, ora.gamma(sigma), queries=q)
        errs.append(np.abs(batch.bufs[k].deg.cpu().numpy()[q] - want) / want)
    rel = np.concatenate(errs)
    flagged = sum(int(b.stats[1].item()) for b in batch.bufs)
    batch.close()
    # the packed bin pass's share of the batch, from the committed ncu launch
    # list of this workload: its own rate (the graph's kernels have no events)
    share = None
    sfile = os.path.join(ROOT, "profiles", "launches_segbatch_64img_d5_L48.md")
    if os.path.exists(sfile):
        with open(sfile) as fh:
            for line in fh:
                if line.startswith("packed_share:"):
                    share = float(line.split(":")[1])
    kernel = None
    if share:
        kach = bin_evals / (share * t * 1e-3) / 1e9
        kernel = {"packed_share": share, "kernel_ms_estimate": share * t, "achieved": kach, "frac": kach / peak,
                  "note": "share of the packed bin pass in the ncu launch list (profiles/), times this step"}
    return {"workload": "segmentation batch: 64 images h 160..321, w=min(481,1.5h), d=5, sigma=0.05, L=48",
            "points": n_tot, "value": n_tot * L / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "steps": steps,
            "flagged_samples": flagged, "parallelism": "4 streams, CUDA graph",
            "roofline": {"bound": "alu", "kernel": "kde_bins_sym_packed_kernel<5> (one launch over 64 images)",
                         "achieved": achieved, "peak": peak, "unit": "Gkernel-evals/s (executed, per step time)",
                         "frac": achieved / peak, "executed_bin_evals": int(bin_evals),
                         "note": "step time includes every other phase: a lower bound of the bin pass's rate",
                         "kernel_estimate": kernel},
            "kde_error": {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()), "queries": int(rel.size),
                          "kind": "degrees vs the FP64 oracle (64 points of images 0, 21, 42, 63)"}}


def sub_serving(fsg, requests, rate, slots=8, admission=0):
    """Serving: `requests` graph-build requests (Poisson arrivals at `rate`/s,
    n log-uniform in [1e3, 2e5], d in {2, 10, 64}, mixture data, sigma = 1.5,
    L = 32) through the library's server: p50/p99 latency and edges/s; the
    degree error of three of the trace's requests run through the same
    kernels alone (results in the mix equal the results alone)."""
    import torch
    import oracle as ora
    from paper_2310_13870_gb300 import inputs
    L, sigma, warm = 32, 1.5, 20
    reqs = inputs.serving_requests(count=requests + warm, rate_hz=rate)
    pools = {d: torch.from_numpy(inputs.gaussian_mixture(n=200_000, d=d, seed=d)).pin_memory().numpy()
             for d in (2, 10, 64)}
    ring = [tuple(torch.empty(200_000 * L, dtype=dt).pin_memory().numpy()
                  for dt in (torch.int32, torch.int32, torch.float32)) for _ in range(24)]
    free_ring = list(range(len(ring)))
    server = fsg.Server(hbm_budget_bytes=120 << 30, max_slots=slots, admission=admission)
    p = fsg.params(sigma)
    owner, lat, done = {}, [], [0]

    def collect(wait_ms=0):
        for rec, _ in server.poll(wait_ms=wait_ms):
            slot, n_r, timed = owner.pop(rec["id"])
            free_ring.append(slot)
            if rec["status"] != fsg.FSG_OK:
                raise RuntimeError(f"request failed: {rec}")
            if timed:
                lat.append(rec["latency_ms"])
                done[0] += n_r * L

    def submit(r, timed):
        while not free_ring:
            collect(wait_ms=1)
        slot = free_ring.pop()
        rid = server.submit(pools[r.d][: r.n], p, L, r.seed, out=ring[slot])
        owner[rid] = (slot, r.n, timed)

    for r in reqs[:warm]:
        submit(r, False)
    while owner:
        collect(wait_ms=5)
    timed_reqs = reqs[warm:]
    base = timed_reqs[0].arrival_s
    t0 = time.perf_counter()
    for r in timed_reqs:
        due = t0 + (r.arrival_s - base)
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            collect(wait_ms=0)
            if due - now > 0.002:
                time.sleep(0.001)
        submit(r, True)
        collect(wait_ms=0)
    while owner:
        collect(wait_ms=5)
    wall = time.perf_counter() - t0
    server.close()
    errs = []
    for d in (2, 10, 64):
        r = min((r for r in timed_reqs if r.d == d), key=lambda r: r.n)
        X = pools[d][: r.n]
        tree = fsg.fsg_build_tree(torch.from_numpy(np.ascontiguousarray(X)).cuda())
        deg = fsg.fsg_degrees(tree, p).cpu().numpy()
        tree.close()
        q = np.random.Generator(np.random.PCG64(60 + d)).choice(r.n, size=min(64, r.n), replace=False)
        want = ora.degrees(X, ora.gamma(sigma), queries=q)
        errs.append(np.abs(deg[q] - want) / want)
    rel = np.concatenate(errs)
    lat.sort()
    pct = lambda a, x: a[min(len(a) - 1, int(x * len(a)))]
    return {"workload": f"serving: {len(timed_reqs)} requests, Poisson {rate}/s, n log-uniform [1e3, 2e5], "
                        f"d in {{2,10,64}}, mixture data, sigma=1.5, L=32, SET edges, HBM budget 120 GB, {slots} slots",
            "value": done[0] / wall, "unit": UNIT, "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
            "max_ms": lat[-1], "wall_s": wall, "offered_s": timed_reqs[-1].arrival_s - base,
            "kde_error": {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()), "queries": int(rel.size),
                          "kind": "degrees vs the FP64 oracle (the smallest request of each d, run alone)"}}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2310_13870_gb300 import fsg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if not os.path.exists(fsg.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    fsg.load()
    X = make_points(rank)
    n, d, L, sigma, seed = WORKLOAD["n"], WORKLOAD["d"], WORKLOAD["L"], WORKLOAD["sigma"], WORKLOAD["seed"]
    stream = torch.cuda.Stream()
    split = args.precision == "split"
    if args.kde_eps > 0 and not split:
        raise SystemExit("--kde-eps needs --precision split (the approximate bin pass is the split form's)")
    if args.resolve and split:
        raise SystemExit("--resolve takes the FP32 fused path (not --precision split)")
    p = fsg.params(sigma, precision=fsg.FSG_PREC_SPLIT_BF16 if split else fsg.FSG_PREC_AUTO, kde_eps=args.kde_eps,
                   resolve=args.resolve)
    # split form at d <= 64: the spatial tree order (its tiles are centred),
    # computed on the GPU in every step (fsg_tree_update); d > 64 needs none
    order = fsg.FSG_ORDER_SPATIAL if split and d <= 64 else fsg.FSG_ORDER_IDENTITY
    with torch.cuda.stream(stream):
        pts = torch.from_numpy(X).cuda()
        tree = fsg.fsg_build_tree(pts, stream=stream, order=order)
        bufs = fsg.GraphBuffers(n, L, with_aux=False)
        bufs.deg = torch.empty(n, dtype=torch.float64, device="cuda")
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    tuning = None
    if not args.no_tune:  # launch shapes picked by the library's autotuner (untimed)
        tuning = fsg.fsg_autotune(tree, p, L, seed, reps=3, stream=stream)

    def step():
        fsg.fsg_tree_update(tree, pts, stream=stream)
        fsg.fsg_build_graph(tree, p, L, seed, bufs=bufs, stream=stream)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    fsg.fsg_sync(tree, stream=stream)
    fsg.fsg_profile(tree, True)
    _, launches0 = fsg.fsg_profile_read(tree)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)  # let the sampler start before the timed region
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, kde_ms, phase_tot = [], [], {}
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ph, _ = fsg.fsg_profile_read(tree)
        kde_ms.append(ph["kde_bins"])
        for k, v in ph.items():
            phase_tot[k] = phase_tot.get(k, 0.0) + v
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    _, launches1 = fsg.fsg_profile_read(tree)
    fsg.fsg_profile(tree, False)
    assert fsg.fsg_sync(tree, stream=stream) == 0
    ms = statistics.mean(step_ms)
    st = fsg.stats_dict(bufs)
    m = int(bufs.m.item())
    deg_main = bufs.deg.cpu().numpy()  # the timed path's degrees (the comparison runs below reuse bufs)
    ms = max_over_ranks(ms, device="cuda")
    value = replica_throughput(n * L, world, ms)
    evals_per_step = st["n_evals"]
    gevals = world * evals_per_step / (ms * 1e-3) / 1e9

    # roofline of the dominant kernel (bin pass)
    kde_avg = statistics.mean(kde_ms)
    on_tc = WORKLOAD["workload"].startswith("digit") or split
    if on_tc:  # tensor-core GEMM (8-bit data): flops 2 n^2 d of the dot products;
        # split form: six BF16 products per coordinate over 64 padded coordinates,
        # for the pairs it executes (tile pairs whose values are all zero are skipped)
        pairs = st["n_bin_evals"] if split else fsg.fsg_bin_pass_evals(tree, p)
        # coordinates the split form's MMAs run: K-steps of 16 (d <= 64), K chunks of 64 (d > 64)
        kpad = 16 * ((d + 15) // 16) if d <= 64 else 64 * ((d + 63) // 64)
        achieved = (12.0 * pairs * kpad if split else 2.0 * pairs * d) / (kde_avg * 1e-3) / 1e12
        peaks = {}
        pf = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pf):
            with open(pf) as f:
                peaks = json.load(f)
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        roof = {"bound": "tensor", "kernel": "kde_bins_split_kernel" if split and d <= 64 else "kde_bins_tc_kernel",
                "achieved": achieved, "peak": peak,
                **({"executed_pairs": int(pairs), "skipped_fraction": 1.0 - pairs / (n * n)} if split and d <= 64
                   else {"executed_pairs": int(pairs), "note": "symmetric pass: each pair once off the diagonal"}
                   if split else {}),
                "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_basis": "measured cuBLAS BF16 sustained (MEASURED_PEAKS.json)" if peaks else "fallback"}
        if split:
            # the split form's other bound: one ex2 per executed pair on the
            # MUFU units (16 per SM per clock); with few K-steps (small d) it
            # needs more time than the tensor work and is the binding unit
            mufu_peak = 152 * 16 * 2.07  # G ex2/s at 2,070 MHz
            t_tensor = 12.0 * pairs * kpad / (peak * 1e12)
            t_mufu = pairs / (mufu_peak * 1e9)
            if t_mufu > t_tensor:
                ach = pairs / (kde_avg * 1e-3) / 1e9
                roof = {"bound": "alu", "kernel": "kde_bins_split_kernel", "achieved": ach, "peak": mufu_peak,
                        "executed_pairs": int(pairs), "skipped_fraction": 1.0 - pairs / (n * n),
                        "unit": "G ex2/s (one per executed pair)", "frac": ach / mufu_peak,
                        "peak_basis": "152 SMs x 16 ex2/clk (MUFU) x 2070 MHz",
                        "tensor_frac": achieved / peak}
    else:
        # executed evaluations of the bin pass; the symmetric kernel adds each
        # value to two rows (2d+3 FP32 lane operations), the plain one to one (2d+2)
        bin_evals = fsg.fsg_bin_pass_evals(tree, p)
        sym = bin_evals < n * n
        ops = 2 * d + (3 if sym else 2)  # generic d > 16 pass: the same count per executed evaluation
        achieved = bin_evals / (kde_avg * 1e-3) / 1e9
        peak = alu_peak_evals(d, ops=ops) / 1e9
        kname = (f"kde_bins_{'sym_' if sym else ''}kernel<{d}>" if d <= 16 else
                 f"kde_bins_generic{'_sym' if sym else ''}_kernel")
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved,
                "peak": peak, "unit": "Gkernel-evals/s (executed)", "frac": achieved / peak,
                "units_per_launch": bin_evals, "algorithmic_evals_per_launch": n * n,
                "algorithmic_gevals_per_s": n * n / (kde_avg * 1e-3) / 1e9,
                "peak_basis": f"{SM_COUNT} SMs x min({FP32_LANES_PER_SM} FP32 lanes/{ops} lane-ops per evaluation, "
                              f"{MUFU_EX2_PER_SM} ex2) x {SM_MAX_MHZ:.0f} MHz"}
    # DRAM bytes per launch of the dominant kernel, from the committed ncu
    # summary of this workload at full size (null for other workloads)
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "kde_bins_sym_traffic_gmm_n100000_d10.md")
    if os.path.exists(tfile) and not split and d == 10 and n == 100_000 and not WORKLOAD["workload"].startswith("digit"):
        with open(tfile) as f:
            for line in f:
                if line.startswith("bytes_per_launch:"):
                    traffic = int(line.split(":")[1])

    # the plain FP32 exact GPU path (levelwise schedule) on the same input, same clocks regime
    def run_plain(schedule):
        pl = fsg.params(sigma, schedule=schedule)
        fsg.fsg_build_graph(tree, pl, L, seed, bufs=bufs, stream=stream)  # warm-up
        stream.synchronize()
        pms = []
        for _ in range(args.plain_steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fsg.fsg_tree_update(tree, pts, stream=stream)
            fsg.fsg_build_graph(tree, pl, L, seed, bufs=bufs, stream=stream)
            e1.record(stream)
            e1.synchronize()
            pms.append(e0.elapsed_time(e1))
        assert fsg.fsg_sync(tree, stream=stream) == 0
        pst = fsg.stats_dict(bufs)
        pt = statistics.mean(pms)
        return {"value": n * L / (pt * 1e-3), "unit": UNIT, "ms_per_step": pt, "steps": args.plain_steps,
                "evals_per_step": pst["n_evals"], "gkernel_evals_per_s": pst["n_evals"] / (pt * 1e-3) / 1e9,
                "flagged_samples": pst["n_flagged"], "speedup_of_fused": (n * L / (ms * 1e-3)) / (n * L / (pt * 1e-3))}

    plain = carried = None
    if args.plain_steps > 0 and not split:
        plain = dict(schedule="levelwise (Algorithm 1 per level, FP32 direct differences, no bin pass)",
                     **run_plain(fsg.FSG_SCHED_LEVELWISE))
        carried = dict(schedule="carried denominator (left half per level, g_R = g_node - g_L)",
                       **run_plain(fsg.FSG_SCHED_CARRIED))

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e and not split:  # the host entry point builds its own (identity-order) tree
        cap = n * L
        hsrc = torch.empty(cap, dtype=torch.int32).pin_memory().numpy()
        hdst = torch.empty(cap, dtype=torch.int32).pin_memory().numpy()
        hw = torch.empty(cap, dtype=torch.float32).pin_memory().numpy()
        hX = torch.from_numpy(X).pin_memory().numpy()
        times, mm = [], 0
        for r in range(2 + args.e2e_steps):
            t0 = time.perf_counter()
            s_, d_, w_ = fsg.fsg_build_graph_host(hX, p, L, seed, out=(hsrc, hdst, hw), stream=stream)
            dt = time.perf_counter() - t0
            mm = len(s_)
            if r >= 2:
                times.append(dt)
        e2e_s = statistics.mean(times)
        e2e_s = max_over_ranks(e2e_s, device="cuda")
        e2e = {"value": replica_throughput(n * L, world, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": int(X.nbytes),
               "d2h_bytes_per_step": int(8 + mm * 12), "ms_per_step": e2e_s * 1e3}

    def run_approx(eps, ref):
        # the approximate KDE (tree-pruned split bin pass) on the same input in
        # the spatial tree order, computed on the GPU inside every timed step
        pa = fsg.params(sigma, precision=fsg.FSG_PREC_SPLIT_BF16, kde_eps=eps)
        with torch.cuda.stream(stream):
            t2 = fsg.fsg_build_tree(pts, stream=stream, order=fsg.FSG_ORDER_SPATIAL)
        fsg.fsg_build_graph(t2, pa, L, seed, bufs=bufs, stream=stream)  # warm-up
        fsg.fsg_build_graph(t2, pa, L, seed, bufs=bufs, stream=stream)
        ams, bin_ms = [], []
        fsg.fsg_profile(t2, True)
        for _ in range(max(3, args.plain_steps)):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fsg.fsg_tree_update(t2, pts, stream=stream)
            fsg.fsg_build_graph(t2, pa, L, seed, bufs=bufs, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ams.append(e0.elapsed_time(e1))
            bin_ms.append(fsg.fsg_profile_read(t2)[0]["kde_bins"])
        fsg.fsg_profile(t2, False)
        assert fsg.fsg_sync(t2, stream=stream) == 0
        ast = fsg.stats_dict(bufs)
        t2.close()
        at = statistics.mean(ams)
        return {"precision": f"approximate KDE: split form, kde_eps = {eps:.3g}, spatial tree order (GPU, in the step)",
                "value": n * L / (at * 1e-3), "unit": UNIT, "ms_per_step": at, "bin_pass_ms": statistics.mean(bin_ms),
                "executed_pairs": int(ast["n_bin_evals"]), "skipped_fraction": 1.0 - ast["n_bin_evals"] / (n * n),
                "flagged_samples": ast["n_flagged"], "kde_error": kde_error(bufs.deg.cpu().numpy(), ref)}

    def run_family(fam, ofam, nq=1024):
        # the same input and path under another kernel of Sec. 2.1 (same sigma)
        import oracle as ora
        pf = fsg.params(sigma, kernel=fam)
        fsg.fsg_build_graph(tree, pf, L, seed, bufs=bufs, stream=stream)  # warm-up
        fms = []
        for _ in range(max(3, args.plain_steps)):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fsg.fsg_tree_update(tree, pts, stream=stream)
            fsg.fsg_build_graph(tree, pf, L, seed, bufs=bufs, stream=stream)
            e1.record(stream)
            e1.synchronize()
            fms.append(e0.elapsed_time(e1))
        assert fsg.fsg_sync(tree, stream=stream) == 0
        fst = fsg.stats_dict(bufs)
        q = np.random.Generator(np.random.PCG64(7)).choice(n, size=min(nq, n), replace=False)
        want = ora.degrees(X, ora.scale(sigma, ofam), queries=q, kernel=ofam)
        got = bufs.deg.cpu().numpy()[q]
        rel = np.abs(got - want) / want
        ft = statistics.mean(fms)
        return {"value": n * L / (ft * 1e-3), "unit": UNIT, "ms_per_step": ft, "flagged_samples": fst["n_flagged"],
                "kde_error": {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()), "queries": int(q.size),
                              "kind": "degrees vs the FP64 oracle of the same kernel"}}

    def run_resolve():
        # the same input and path with the high-precision re-decision of the
        # flagged samples (and FP64 weights): step time, the re-decision's
        # own time, samples re-decided and still flagged
        out = {}
        for name, pr in (("resolve", fsg.params(sigma, resolve=True)),
                         ("resolve_f64_weights", fsg.params(sigma, resolve=True, weight_f64=True))):
            b2 = fsg.GraphBuffers(n, L, with_aux=False, weight_f64=bool(pr.weight_f64))
            fsg.fsg_build_graph(tree, pr, L, seed, bufs=b2, stream=stream)  # warm-up
            fsg.fsg_profile(tree, True)
            rms, rph = [], []
            for _ in range(max(3, args.plain_steps)):
                rms += timed_steps(lambda: (fsg.fsg_tree_update(tree, pts, stream=stream),
                                            fsg.fsg_build_graph(tree, pr, L, seed, bufs=b2, stream=stream)),
                                   1, stream, flush)
                rph.append(fsg.fsg_profile_read(tree)[0]["resolve"])
            fsg.fsg_profile(tree, False)
            assert fsg.fsg_sync(tree, stream=stream) == 0
            rst = fsg.stats_dict(b2)
            rt = statistics.mean(rms)
            out[name] = {"value": n * L / (rt * 1e-3), "unit": UNIT, "ms_per_step": rt,
                         "resolve_ms": statistics.mean(rph), "added_ms": rt - ms,
                         "resolved_samples": rst["n_resolved"], "flagged_after": rst["n_flagged"],
                         "flagged_without": st["n_flagged"]}
        return out

    cpu = None
    err = split_cmp = approx_cmp = families = subs = resolved = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ref = {}
        v, dt, threads = cpu_oracle_throughput(X, args.cpu_queries, L, sigma, seed, keep=ref)
        err = kde_error(deg_main, ref)
        if not split and not on_tc and d <= 64 and args.plain_steps > 0:
            # the split-precision path on the same tree and input, beside the FP32 path
            ps = fsg.params(sigma, precision=fsg.FSG_PREC_SPLIT_BF16)
            fsg.fsg_build_graph(tree, ps, L, seed, bufs=bufs, stream=stream)  # warm-up
            sms = []
            for _ in range(max(3, args.plain_steps)):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fsg.fsg_tree_update(tree, pts, stream=stream)
                fsg.fsg_build_graph(tree, ps, L, seed, bufs=bufs, stream=stream)
                e1.record(stream)
                e1.synchronize()
                sms.append(e0.elapsed_time(e1))
            assert fsg.fsg_sync(tree, stream=stream) == 0
            sst = fsg.stats_dict(bufs)
            st_ms = statistics.mean(sms)
            split_cmp = {"precision": "split (three-part BF16 tcgen05 bin pass, identity tree order)",
                         "value": n * L / (st_ms * 1e-3), "unit": UNIT, "ms_per_step": st_ms,
                         "flagged_samples": sst["n_flagged"], "flag_eps": 2.0 ** -10,
                         "kde_error": kde_error(bufs.deg.cpu().numpy(), ref)}
            approx_cmp = run_approx(2.0 ** -20, ref)
            families = {name: run_family(fam, ofam) for name, fam, ofam in
                        (("laplacian", fsg.FSG_KERNEL_LAPLACIAN, 1), ("exponential", fsg.FSG_KERNEL_EXPONENTIAL, 2))}
        if not split and not on_tc and d <= 16:
            resolved = run_resolve()
        if not args.no_sub and WORKLOAD["workload"].startswith("gaussian_mixture") and not split and n == 100_000:
            # the other workloads, each measured the same way (value, roofline, error vs the oracle)
            subs = {"digits": sub_digits(fsg, stream, flush, 5),
                    "seg_batch": sub_seg_batch(fsg, stream, flush, 3),
                    "serving": sub_serving(fsg, args.sub_requests, args.rate, args.slots)}
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{args.cpu_queries} of the {n} query points (all {L} samples each + their degrees), "
                         f"{dt:.1f} s, extrapolated per sampled edge"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16x3 split, f32 accumulate" if split else "f32", "data": "synthetic",
                "config": dict(WORKLOAD, parallelism=f"replicas x{world} (independent point sets)",
                               **({"precision": "split (spatial tree order, GPU, in the step)" if d <= 64 else
                                   "split (three-part BF16 operands, identity tree order)"} if split else {}),
                               **({"kde_eps": args.kde_eps} if args.kde_eps > 0 else {}),
                               **({"resolve": True} if args.resolve else {})),
                "gkernel_evals_per_s": gevals, "evals_per_step": evals_per_step, "edges_per_step": m,
                "flagged_samples": st["n_flagged"], "items": st["n_items"],
                "phase_ms": {k: v / args.steps for k, v in phase_tot.items() if v > 0},
                "kde_error": err, "split_precision": split_cmp, "approximate_kde": approx_cmp,
                "kernel_families": families, "workloads": subs, "high_precision": resolved,
                "roofline": dict(roof, traffic=traffic), "plain_fp32_gpu": plain, "carried_fp32_gpu": carried,
                "tuning": tuning,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": int(launches1 - launches0)}
        print(json.dumps(line), flush=True)
    tree.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_seg_batch(args):
    """64 segmentation-shaped images (heights 160..321, w = min(481, 1.5 h),
    (r,g,b,x,y) features, sigma = 0.05, L = 48) built as one batch: every
    image's whole Algorithm 2 on 4 streams, replayed from a CUDA graph."""
    import torch

    from paper_2310_13870_gb300 import fsg, inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if not os.path.exists(fsg.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    fsg.load()
    count = args.images
    imgs = inputs.segmentation_batch(count=count)
    L, sigma = 48, 0.05
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sets = [(torch.from_numpy(X).cuda(), fsg.params(sigma), L, 1000 + i) for i, X in enumerate(imgs)]
        batch = fsg.Batch(sets, streams=4, capture=True, stream=stream)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        batch.run(stream=stream)
    stream.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.5)
    ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run(stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    n_tot = sum(int(X.shape[0]) for X in imgs)
    edges = sum(int(b.m.item()) for b in batch.bufs)
    evals = sum(int(b.stats[4].item()) for b in batch.bufs)
    flagged = sum(int(b.stats[1].item()) for b in batch.bufs)
    t = statistics.mean(ms)
    plain = None
    if args.plain_steps > 0:  # the same images through the plain FP32 levelwise schedule, one timed run
        batch.close()
        with torch.cuda.stream(stream):
            psets = [(X, fsg.params(sigma, schedule=fsg.FSG_SCHED_LEVELWISE), L, seed) for X, _, L, seed in sets]
            pbatch = fsg.Batch(psets, streams=4, capture=False, stream=stream)
        pbatch.run(stream=stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pbatch.run(stream=stream)
        e1.record(stream)
        e1.synchronize()
        pt = e0.elapsed_time(e1)
        pevals = sum(int(b.stats[4].item()) for b in pbatch.bufs)
        plain = {"schedule": "levelwise (Algorithm 1 per level, FP32 direct differences, no bin pass)",
                 "value": n_tot * L / (pt * 1e-3), "unit": UNIT, "ms_per_step": pt, "steps": 1,
                 "evals_per_step": pevals, "flagged_samples": sum(int(b.stats[1].item()) for b in pbatch.bufs),
                 "speedup_of_fused": pt / t}
        pbatch.close()
        batch = None
    line = {"metric": METRIC, "value": n_tot * L / (t * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"segmentation batch: {count} images h 160..321, w=min(481,1.5h), d=5, "
                                   f"sigma=0.05, L=48, SET edges", "points": n_tot,
                       "l2": "flushed (512 MB write) between steps", "parallelism": "4 streams, CUDA graph"},
            "gkernel_evals_per_s": evals / (t * 1e-3) / 1e9, "edges_per_step": edges, "clocks": clk,
            "flagged_samples": flagged, "plain_fp32_gpu": plain,
            "p50_ms": statistics.median(ms), "p99_ms": sorted(ms)[min(len(ms) - 1, int(0.99 * len(ms)))]}
    print(json.dumps(line), flush=True)
    if batch is not None:
        batch.close()
    return 0


def run_serving(args):
    """Serving: Poisson arrivals (args.rate per second) of graph-build requests
    with n log-uniform in [1e3, 2e5], d uniform on {2, 10, 64}, Gaussian-mixture
    data (unit blobs, centres in [-10,10]^d), sigma = 1.5, L = 32, through the
    library's server (HBM budget 120 GB, 8 slots).  Points come from one
    pinned 200,000-point pool per d (a request uses the first n rows with its
    own seed); edges land in a ring of pinned host buffers."""
    import torch

    from paper_2310_13870_gb300 import fsg, inputs
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if not os.path.exists(fsg.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    fsg.load()
    L, sigma = 32, 1.5
    reqs = inputs.serving_requests(count=args.requests + args.warmup, rate_hz=args.rate)
    pools = {d: torch.from_numpy(inputs.gaussian_mixture(n=200_000, d=d, seed=d)).pin_memory().numpy()
             for d in (2, 10, 64)}
    ring = [tuple(torch.empty(200_000 * L, dtype=dt).pin_memory().numpy() for dt in (torch.int32, torch.int32,
                                                                                       torch.float32))
            for _ in range(24)]
    free_ring = list(range(len(ring)))
    admission = {"arrival": fsg.FSG_ADMIT_ARRIVAL, "ratio": fsg.FSG_ADMIT_RESPONSE_RATIO}[args.admission]
    server = fsg.Server(hbm_budget_bytes=120 << 30, max_slots=args.slots, admission=admission)
    p = fsg.params(sigma)
    # --precision split: the d = 64 requests take the split form (bin pass and
    # leaf phase on the tensor cores, spatial tree order computed on the GPU)
    p_large = fsg.params(sigma, precision=fsg.FSG_PREC_SPLIT_BF16) if args.precision == "split" else p
    owner = {}
    lat, qms, edges_done = [], [], 0
    sampled_done = 0

    def collect(wait_ms=0):
        nonlocal edges_done, sampled_done
        for rec, _ in server.poll(wait_ms=wait_ms):
            slot, n_r, timed = owner.pop(rec["id"])
            free_ring.append(slot)
            if rec["status"] != fsg.FSG_OK:
                raise RuntimeError(f"request failed: {rec}")
            if timed:
                lat.append(rec["latency_ms"])
                qms.append(rec["queue_ms"])
                edges_done += rec["n_edges"]
                sampled_done += n_r * L

    def submit(r, timed):
        while not free_ring:
            collect(wait_ms=1)
        slot = free_ring.pop()
        X = pools[r.d][: r.n]
        rid = server.submit(X, p_large if r.d > 16 else p, L, r.seed, out=ring[slot])
        owner[rid] = (slot, r.n, timed)

    for r in reqs[: args.warmup]:  # warm-up: untimed
        submit(r, False)
    while owner:
        collect(wait_ms=5)
    timed_reqs = reqs[args.warmup:]
    base = timed_reqs[0].arrival_s
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.5)
    t0 = time.perf_counter()
    for r in timed_reqs:
        due = t0 + (r.arrival_s - base)
        while True:
            now = time.perf_counter()
            if now >= due:
                break
            collect(wait_ms=0)
            if due - now > 0.002:
                time.sleep(0.001)
        submit(r, True)
        collect(wait_ms=0)
    while owner:
        collect(wait_ms=5)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    server.close()
    plain = None
    if args.plain_requests > 0:
        # closed loop: the first K timed requests submitted at once, fused vs plain schedule
        def burst(schedule):
            srv = fsg.Server(hbm_budget_bytes=120 << 30, max_slots=args.slots, admission=admission)
            pp = fsg.params(sigma, schedule=schedule)
            sub = timed_reqs[: args.plain_requests]
            t0b = time.perf_counter()
            ids = [srv.submit(pools[r.d][: r.n], pp, L, r.seed) for r in sub]
            done = 0
            while done < len(ids):
                for rec, _ in srv.poll(wait_ms=5):
                    if rec["status"] != fsg.FSG_OK:
                        raise RuntimeError(f"request failed: {rec}")
                    done += 1
            wall_b = time.perf_counter() - t0b
            srv.close()
            return sum(r.n for r in sub) * L / wall_b, wall_b
        vf, wf = burst(fsg.FSG_SCHED_FUSED)
        vp, wp = burst(fsg.FSG_SCHED_LEVELWISE)
        plain = {"schedule": "levelwise (Algorithm 1 per level, FP32 direct differences, no bin pass)",
                 "requests": args.plain_requests, "mode": "closed loop, all submitted at once",
                 "fused_value": vf, "fused_wall_s": wf, "value": vp, "wall_s": wp, "unit": UNIT,
                 "speedup_of_fused": vf / vp}
    lat_sorted = sorted(lat)
    pct = lambda a, q: a[min(len(a) - 1, int(q * len(a)))]
    line = {"metric": METRIC, "value": sampled_done / wall, "unit": UNIT, "n_gpus": 1, "steps": len(timed_reqs),
            "warmup": args.warmup, "ms_per_step": wall * 1e3 / len(timed_reqs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving: {len(timed_reqs)} requests, Poisson {args.rate}/s, n log-uniform "
                                   f"[1e3, 2e5], d in {{2,10,64}}, mixture data, sigma=1.5, L=32, SET edges",
                       "hbm_budget_gb": 120, "slots": args.slots,
                       "parallelism": f"continuous admission, {args.slots} slots",
                       "precision": "d = 64 in split precision" if args.precision == "split" else "FP32 / auto",
                       "admission": {"arrival": "arrival order",
                                     "ratio": "highest response ratio next"}[args.admission]},
            "p50_ms": pct(lat_sorted, 0.5), "p99_ms": pct(lat_sorted, 0.99), "max_ms": lat_sorted[-1],
            "p50_queue_ms": pct(sorted(qms), 0.5), "edges": edges_done, "wall_s": wall,
            "offered_s": timed_reqs[-1].arrival_s - base, "clocks": clk, "plain_fp32_gpu": plain}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-queries", type=int, default=0, help="oracle sample size (default 16384; 512 at d=784)")
    ap.add_argument("--ref-queries", type=int, default=1024)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in launch-shape heuristics")
    ap.add_argument("--no-sub", action="store_true", help="skip the digit, segmentation-batch and serving entries")
    ap.add_argument("--sub-requests", type=int, default=1000, help="serving entry: length of the trace")
    ap.add_argument("--plain-steps", type=int, default=2, help="timed steps of the plain FP32 levelwise path")
    ap.add_argument("--n", type=int, default=0, help="smaller point count (profiler captures only)")
    ap.add_argument("--d", type=int, default=0, help="other dimension of the mixture workload (kernel studies)")
    ap.add_argument("--workload", choices=["gmm", "digits", "seg-batch", "serving"], default="gmm")
    ap.add_argument("--requests", type=int, default=10_000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--images", type=int, default=64)
    ap.add_argument("--plain-requests", type=int, default=40, help="serving: closed-loop burst for the plain path")
    ap.add_argument("--admission", choices=["arrival", "ratio"], default="arrival", help="serving: admission order")
    ap.add_argument("--slots", type=int, default=8, help="serving: requests in flight at once")
    ap.add_argument("--resolve", action="store_true",
                    help="the headline step with the high-precision re-decision of flagged samples")
    ap.add_argument("--kde-eps", type=float, default=0.0,
                    help="approximate KDE (tree-pruned split bin pass) with this relative error bound")
    ap.add_argument("--precision", choices=["auto", "split"], default="auto",
                    help="split-precision tensor-core bin pass (d <= 64: centred tiles on a spatial tree order; "
                         "d > 64, e.g. --workload digits: three-part operands)")
    args = ap.parse_args()
    if args.n:
        set_size(args.n)
    if args.d and args.workload == "gmm":
        WORKLOAD["workload"] = WORKLOAD["workload"].replace(f"d={WORKLOAD['d']}", f"d={args.d}")
        WORKLOAD["d"] = args.d
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "seg-batch":
        return run_seg_batch(args)
    if args.workload == "serving":
        return run_serving(args)
    if not args.cpu_queries:  # about 10 s of oracle work on 16 host cores
        args.cpu_queries = 512 if args.workload == "digits" else 16384
    if args.workload == "digits":
        WORKLOAD.clear()
        WORKLOAD.update(DIGITS)
        if args.n:
            WORKLOAD["n"] = args.n
            WORKLOAD["workload"] = WORKLOAD["workload"].replace("n=70000", f"n={args.n}")
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
