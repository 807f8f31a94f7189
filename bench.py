#!/usr/bin/env python3
"""Throughput of the buffered Frequent Directions update on GB300.

One step streams the whole synthetic matrix of the workload through the
sketch (fd_reset, fd_append of every row, fd_sketch into device memory) and
reports rows per second. Prints one JSON line (rank 0).

Workloads (seeded synthetic inputs shaped like the paper's Random Noisy data,
A = S D U + F / zeta, D from 1 to 0.1 over m signal dimensions):
  c1  (default) n = 200,000, d = 2,000, m = 50, zeta = 10, FP32 rows, FD with
      ell = 100, split-precision BF16x3 tensor-core path
  c0  n = 10,000, d = 500, m = 30, ell = 50 (small case)
Every option can be overridden (--ell, --variant, --prec, --n ...).

--impl reference times the FP64 oracle (the plain CPU restatement of the
method) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "c1": dict(n=200_000, d=2000, m=50, zeta=10.0, seed=1, ell=100, variant="fd", alpha=1.0,
               prec="bf16x3", name="random-noisy n=200000 d=2000 k=50 zeta=10 fp32 rows"),
    "c0": dict(n=10_000, d=500, m=30, zeta=10.0, seed=0, ell=50, variant="fd", alpha=1.0,
               prec="fp32", name="random-noisy n=10000 d=500 m=30 zeta=10"),
    "c4": dict(count=10_000, d=512, ell=32, rate=5e6, seconds=10.0, warm=1.0, seed=4,
               variant="fd", alpha=1.0, prec="fp32", n=None,
               name="serving: 10000 live sketches d=512 ell=32, Poisson row blocks of "
                    "log-uniform size 1..4096, sparse non-negative rows (2%), 5M rows/s offered"),
    "c3": dict(count=4096, seed=3, variant="fd", alpha=1.0, prec="fp32", ell=None, n=None,
               name="batched: 4096 random-noisy streams, d in U{64..1024}, ell in U{16..64}, "
                    "n in U{1000..50000}, k = ell/2, bf16 rows"),
}
FP32_LANES_PER_SM = 128
METRIC_SINGLE = "FD rows/s (sketch update, whole stream per step)"
METRIC_BATCH = "FD rows/s (batched sketch update, every stream per step)"
METRIC_SERVE = "serving append latency p99 (ms) and rows/s"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant
# kernel from one full ncu capture, reported as roofline "traffic" only for
# the configuration it was taken on; None once that kernel changes.
# Single stream: bytes per eigensolve launch, keyed by (ell, prec, variant,
# buffer rows); profiles/eig_gram_rotate_c1_ell100_full.md.
EIG_TRAFFIC = {(100, "bf16x3", "fd", 200): 553728}
# Batched: DRAM bytes per byte of input rows, from a 64-sketch launch of the
# same generator (1,863,630,000 B for 1,817,569,744 B of rows), scaled by the
# rows a launch reads; profiles/batch_kernel_c3_64sketch_full.md.
BATCH_TRAFFIC_PER_INPUT_BYTE = 1863630000 / 1817569744


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c1", choices=sorted(WORKLOADS))
    ap.add_argument("--ell", type=int)
    ap.add_argument("--variant", choices=["fd", "pfd", "ss", "isvd", "fastpfd"])
    ap.add_argument("--buffer-rows", type=int,
                    help="single stream: rows held before a reduction (default 2*ell; ell for fastpfd)")
    ap.add_argument("--alpha", type=float)
    ap.add_argument("--prec", choices=["fp32", "bf16x3", "fp64"])
    ap.add_argument("--n", type=int)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison")
    ap.add_argument("--cpu-sample-rows", type=int, default=0)
    ap.add_argument("--count", type=int, help="batched workload: number of sketches")
    ap.add_argument("--shards", type=int, default=16,
                    help="single stream: also time P contiguous shards sketched concurrently "
                         "and merged pairwise (0 = skip)")
    return ap.parse_args()


def config(args):
    w = dict(WORKLOADS[args.workload])
    if args.workload in ("c3", "c4"):
        for k in ("variant", "alpha"):
            if getattr(args, k) is not None:
                w[k] = getattr(args, k)
        return w
    for k in ("ell", "variant", "alpha", "prec", "n"):
        v = getattr(args, k)
        if v is not None:
            w[k] = v
    if w["variant"] in ("pfd", "fastpfd") and args.alpha is None:
        w["alpha"] = 0.2
    w["buffer_rows"] = args.buffer_rows
    return w


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of every rank's x (the timed step is as slow as the slowest
    rank); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_batch_seed(w, rank: int) -> int:
    """Seed of a rank's batched streams: every rank draws its own sketches
    (sharding by sketch, no data-path collective)."""
    return w["seed"] + 1000 * rank


def mass_account(st: dict) -> dict:
    """Bookkeeping of one sketch from its fd_stats (the latest fd_sketch's
    totals): ||A||_F^2 - removed - ||B||_F^2 is zero in exact arithmetic, and
    Lemma 1 (Sec. 3.1) bounds cov-err by Delta / ||A||_F^2."""
    a2 = float(st["norm_a2"])
    removed = float(st["sketch_removed"])
    b2 = float(st["sketch_norm_b2"])
    delta = float(st["sketch_sum_delta"])
    return {"norm_a2": a2, "removed": removed, "norm_b2": b2, "sum_delta": delta,
            "gap_rel": (a2 - removed - b2) / a2 if a2 > 0 else 0.0,
            "lemma1_bound": delta / a2 if a2 > 0 else 0.0}


def mass_trajectory(sk, A, out, points: int = 8) -> list:
    """mass_account at evenly spaced points of the stream A (rows appended in
    chunks, each point read through the non-destructive sketch call): whether
    ||A||_F^2 - removed - ||B||_F^2 grows steadily or in jumps."""
    n = int(A.shape[0])
    marks = sorted({max(1, int(round(n * (k + 1) / points))) for k in range(points)})
    sk.reset()
    done, res = 0, []
    for mk in marks:
        sk.append(A[done:mk])
        done = mk
        sk.sketch(out=out)
        acc = mass_account(sk.stats())
        res.append({"rows": mk, "gap_rel": acc["gap_rel"], "lemma1_bound": acc["lemma1_bound"]})
    return res


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_rows(w, rank, rows=None):
    from paper_1501_06561_gb300 import workloads
    n = w["n"] if rows is None else rows
    import numpy as np
    return workloads.random_noisy(n, w["d"], m=w["m"], zeta=w["zeta"], seed=w["seed"] + 1000 * rank,
                                  dtype=np.float32, row_stop=n)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_baseline(w, rows_sample):
    """The FP64 oracle as it stands, on the host cores, on the first rows."""
    import numpy as np
    from oracle import fd_sketch
    from paper_1501_06561_gb300 import workloads
    A = workloads.random_noisy(rows_sample, w["d"], m=w["m"], zeta=w["zeta"], seed=w["seed"],
                               dtype=np.float32, row_stop=rows_sample)
    t0 = time.perf_counter()
    fd_sketch(A, w["ell"], w["variant"], w["alpha"], buffer_rows=w.get("buffer_rows"))
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([x.get("num_threads", 1) for x in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return {"value": rows_sample / dt, "unit": "rows/s", "cores": int(cores), "kind": "oracle",
            "sample": f"first {rows_sample} rows of the workload stream ({dt:.1f} s of CPU work)"}


def run_reference_batch(args, w):
    """Oracle on a sample of the batched workload's streams (host-drawn with
    the same recipe), timed per step; rows/s over the sampled streams."""
    import numpy as np
    from oracle import fd_sketch
    from paper_1501_06561_gb300 import workloads
    specs = workloads.batch_specs(args.count or w["count"], seed=w["seed"])
    order = sorted(range(len(specs)), key=lambda i: specs[i]["d"] * specs[i]["ell"])
    pick = [order[0], order[len(order) // 4], order[len(order) // 2]]
    data = [workloads.random_noisy(specs[i]["n"], specs[i]["d"], m=max(1, specs[i]["ell"] // 2),
                                   seed=specs[i]["seed"], dtype="bf16") for i in pick]
    rows = sum(a.shape[0] for a in data)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for i, a in zip(pick, data):
            fd_sketch(a, specs[i]["ell"], w["variant"], w["alpha"])
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    return rows, t, f"{len(pick)} streams of the batch (ids {pick}, {rows} rows) per step"


def run_reference_serve(args, w):
    """Oracle on a sample of the serving workload: a few sketches, each fed
    sparse non-negative rows drawn as the request blocks are."""
    from oracle import FDOracle
    from paper_1501_06561_gb300 import workloads
    nsk, per = 4, 4096
    data = [workloads.sparse_nonneg_rows(per, w["d"], seed=w["seed"], stream=k) for k in range(nsk)]
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for a in data:
            o = FDOracle(w["d"], w["ell"], w["variant"], w["alpha"])
            o.append(a)
            o.sketch()
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    return nsk * per, sum(times) / len(times), f"{nsk} sketches x {per} rows per step"


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload in ("c3", "c4"):
        rows, t, sample = (run_reference_batch(args, w) if args.workload == "c3"
                           else run_reference_serve(args, w))
        try:
            from threadpoolctl import threadpool_info
            cores = max([x.get("num_threads", 1) for x in threadpool_info()] + [1])
        except Exception:
            cores = os.cpu_count() or 1
        val = rows / t
        print(json.dumps({"impl": "reference",
                          "metric": METRIC_BATCH if args.workload == "c3" else METRIC_SERVE,
                          "value": val,
                          "unit": "rows/s", "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": t * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f64", "data": "synthetic",
                          "config": {"workload": w["name"], "sample": sample},
                          "cpu_baseline": {"kind": "oracle", "cores": int(cores), "value": val,
                                           "unit": "rows/s", "sample": sample},
                          "e2e": {"value": val, "unit": "rows/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    rows = args.cpu_sample_rows or default_sample_rows(w)
    times = []
    import numpy as np
    from oracle import fd_sketch
    from paper_1501_06561_gb300 import workloads
    A = workloads.random_noisy(rows, w["d"], m=w["m"], zeta=w["zeta"], seed=w["seed"],
                               dtype=np.float32, row_stop=rows)
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        fd_sketch(A, w["ell"], w["variant"], w["alpha"], buffer_rows=w.get("buffer_rows"))
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    try:
        from threadpoolctl import threadpool_info
        cores = max([x.get("num_threads", 1) for x in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    val = rows / t
    line = {"impl": "reference", "metric": METRIC_SINGLE, "value": val, "unit": "rows/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "ell": w["ell"], "variant": w["variant"],
                       "alpha": w["alpha"],
                       "buffer_rows": w.get("buffer_rows") or (w["ell"] if w["variant"] == "fastpfd"
                                                               else 2 * w["ell"]),
                       "sample_rows": rows},
            "cpu_baseline": {"kind": "oracle", "cores": int(cores), "value": val, "unit": "rows/s",
                             "sample": f"first {rows} rows of the workload stream per step"},
            "e2e": {"value": val, "unit": "rows/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def default_sample_rows(w):
    # about 10-30 s of oracle work: the oracle's SVD of a 2*ell x d buffer per
    # ell+1 rows dominates
    per_red = 8e-10 * (2 * w["ell"]) ** 2 * w["d"]  # seconds per reduction (SVD of 2 ell x d)
    reds = max(20, int(15.0 / max(per_red, 1e-5)))
    return int(min(w["n"], 2 * w["ell"] + reds * (w["ell"] + 1)))


def batch_reductions(n, ell):
    L = 2 * ell
    return 0 if n < L else 1 + (n - L) // (ell + 1)


def run_batch(args, w):
    """Batched workload: every stream through fd_batch_append (one persistent
    launch) and fd_batch_sketch_all (one launch) per step."""
    import numpy as np
    import torch
    from paper_1501_06561_gb300 import fd, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fd.load()
    count = args.count or w["count"]
    specs = workloads.batch_specs(count, seed=rank_batch_seed(w, rank))
    flat, views = workloads.batch_streams_device(specs)
    ds = [sp["d"] for sp in specs]
    ells = [sp["ell"] for sp in specs]
    b = fd.FDBatch(ds, ells, w["variant"], w["alpha"], w["prec"])
    blocks = {i: flat[off:off + n * d].view(n, d) for i, (off, n, d) in enumerate(views)}
    prep = b.prepare(blocks)
    offs, tot = b.offsets()
    out = torch.empty(tot, device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()
    rows = int(sum(sp["n"] for sp in specs))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    ka = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]

    def step(i=None):
        b.reset()
        if i is not None:
            ka[2 * i].record(stream)
        b.append_prepared(prep)
        if i is not None:
            ka[2 * i + 1].record(stream)
        b.sketch_all(out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_kernel = sum(ka[2 * i].elapsed_time(ka[2 * i + 1]) for i in range(args.steps)) / args.steps
    ms = max_over_ranks(ms, world)
    value = rows * world / (ms / 1e3)

    # end to end: host rows (a bounded copy of the device streams would not fit the
    # host for 10^8 rows, so the e2e leg copies every stream from pinned host memory
    # into the device buffer inside the timed region)
    e2e = None
    if not args.no_e2e:
        host = torch.empty(flat.numel(), dtype=flat.dtype, pin_memory=True)
        host.copy_(flat)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            flat.copy_(host, non_blocking=True)
            step()
            hout = out.to("cpu")
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / max(1, args.steps)
        e2e = {"value": rows * world / dt, "unit": "rows/s",
               "h2d_bytes_per_step": int(flat.numel() * flat.element_size()),
               "d2h_bytes_per_step": int(hout.numel() * 4)}
        del host

    # the plain FP32 single-sketch path (K7) against the batched kernel on the
    # same sample: the first P sketches, one fd_create handle each, appended
    # on 16 CUDA streams (host wall clock around the appends and a sync), and
    # one FDBatch launch over the same P sketches (CUDA events)
    plain = None
    if not args.no_plain and rank == 0 and args.workload == "c3":
        P = min(64, count)
        sub_rows = int(sum(specs[i]["n"] for i in range(P)))
        streams = [torch.cuda.Stream() for _ in range(16)]
        hs = [fd.FDSketch(ds[i], ells[i], w["variant"], w["alpha"], "fp32", stream=streams[i % 16])
              for i in range(P)]
        for rep in range(2):  # the first pass warms up
            for h in hs:
                h.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i in range(P):
                hs[i].append(blocks[i])
            torch.cuda.synchronize()
            dt_plain = time.perf_counter() - t0
        for h in hs:
            h.close()
        bs = fd.FDBatch(ds[:P], ells[:P], w["variant"], w["alpha"], w["prec"])
        prep_s = bs.prepare({i: blocks[i] for i in range(P)})
        eb0 = torch.cuda.Event(enable_timing=True)
        eb1 = torch.cuda.Event(enable_timing=True)
        for rep in range(2):
            bs.reset()
            eb0.record(stream)
            bs.append_prepared(prep_s)
            eb1.record(stream)
            torch.cuda.synchronize()
        dt_batch = eb0.elapsed_time(eb1) / 1e3
        bs.close()
        plain = {"value": sub_rows / dt_plain, "unit": "rows/s",
                 "batched_same_sample": sub_rows / dt_batch,
                 "sample": f"first {P} sketches ({sub_rows} rows)",
                 "how": "one fd_create FP32 handle per sketch on 16 CUDA streams, host wall clock; "
                        "batched: one persistent launch over the same sketches, CUDA events"}

    if rank != 0:
        b.close()
        return 0
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flops = 0.0
    for sp in specs:
        L = 2 * sp["ell"]
        r = batch_reductions(sp["n"], sp["ell"])
        flops += r * (9.0 * L ** 3 + 2.0 * L * L * sp["d"] + 2.0 * (sp["ell"] - 1) * L * sp["d"])
    achieved = flops / (ms_kernel / 1e3) / 1e12
    in_bytes = int(flat.numel() * flat.element_size())
    traffic = (int(BATCH_TRAFFIC_PER_INPUT_BYTE * in_bytes)
               if BATCH_TRAFFIC_PER_INPUT_BYTE and args.workload == "c3" else None)
    roofline = {"bound": "alu", "kernel": "batch_kernel (persistent: ingest, Gram, tridiagonal "
                "eigensolve, shrink, rotate per sketch)", "achieved": achieved, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": achieved / alu_peak, "traffic": traffic,
                "traffic_source": "ncu capture of 64 sketches, scaled by input bytes",
                "peak_source": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                "algorithmic_flops_per_launch": flops, "avg_launch_us": ms_kernel * 1e3,
                "hbm_bytes_per_launch": int(flat.numel() * flat.element_size())}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_batch(specs, flat, views, w)
    line = {
        "metric": METRIC_BATCH,
        "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16 rows), f64 shrink",
        "data": "synthetic",
        "config": {"workload": w["name"], "sketches": count, "rows_per_step": rows,
                   "reductions_per_step": int(sum(batch_reductions(sp["n"], sp["ell"])
                                                  for sp in specs)),
                   "input_bytes": int(flat.numel() * flat.element_size()),
                   "l2": "input larger than L2 (no flush needed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "plain_fp32": plain,
        "roofline": roofline, "gpu_launches": 2 * args.steps, "clocks": clk, "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    b.close()
    return 0


def cpu_baseline_batch(specs, flat, views, w, budget_s=20.0):
    """The oracle on a stratified sample of the batch's streams (smallest and
    largest d*ell first), until about budget_s seconds of CPU work."""
    import numpy as np
    import torch
    from oracle import fd_sketch
    order = sorted(range(len(specs)), key=lambda i: specs[i]["d"] * specs[i]["ell"])
    pick = [order[0], order[-1], order[len(order) // 2], order[len(order) // 4],
            order[3 * len(order) // 4]]
    rows, t = 0, 0.0
    used = []
    for i in pick:
        off, n, d = views[i]
        A = flat[off:off + n * d].view(n, d).float().cpu().numpy()
        t0 = time.perf_counter()
        fd_sketch(A, specs[i]["ell"], w["variant"], w["alpha"])
        t += time.perf_counter() - t0
        rows += n
        used.append(i)
        if t > budget_s:
            break
    try:
        from threadpoolctl import threadpool_info
        cores = max([x.get("num_threads", 1) for x in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return {"value": rows / t, "unit": "rows/s", "cores": int(cores), "kind": "oracle",
            "sample": f"{len(used)} of the batch's streams (ids {used}, {rows} rows, {t:.1f} s)"}


def run_serve(args, w):
    """Serving workload: an open-loop Poisson generator submits row blocks to
    the continuous-batching server; reports achieved rows/s and the p50/p99
    latency from submit to completion."""
    import numpy as np
    from paper_1501_06561_gb300 import fd, workloads
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    fd.load()
    count = args.count or w["count"]
    rng = np.random.default_rng(w["seed"] + rank)
    pool = workloads.sparse_nonneg_rows(1 << 19, d=w["d"], seed=w["seed"] + rank)
    mean_rows = (4096 - 1) / np.log(4096)
    req_rate = w["rate"] / mean_rows
    srv = fd.FDServer(count, w["d"], w["ell"], w["variant"], w["alpha"],
                      budget_bytes=1 << 30, streams=4)
    total = w["warm"] + w["seconds"]
    t_start = time.perf_counter()
    t_next = t_start
    pos = 0
    backlog = []
    submitted_rows = 0
    warm_tickets = set()
    while True:
        now = time.perf_counter()
        if now - t_start > total:
            break
        while t_next <= now:
            n = int(min(4096, max(1, np.exp(rng.uniform(0, np.log(4096))))))
            sid = int(rng.integers(0, count))
            if pos + n > pool.shape[0]:
                pos = 0
            backlog.append((sid, pos, n, t_next))
            pos += n
            t_next += rng.exponential(1.0 / req_rate)
        keep = []
        for sid, p0, n, ta in backlog:
            t = srv.submit(sid, pool[p0:p0 + n])
            if t is None:
                keep.append((sid, p0, n, ta))
                continue
            submitted_rows += n
            if ta - t_start < w["warm"]:
                warm_tickets.add(t)
        backlog = keep
    t_end = time.perf_counter()
    srv.drain()
    t_drain = time.perf_counter()
    done = srv.poll(1 << 22)
    lat = np.array([l for t, l in done if t not in warm_tickets]) * 1e3
    c = srv.counters()
    srv.close()
    if rank != 0:
        return 0
    rows_done = c["rows_done"]
    line = {"metric": METRIC_SERVE, "value": rows_done / (t_drain - t_start),
            "unit": "rows/s", "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": (t_drain - t_start) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32, f64 shrink", "data": "synthetic",
            "config": {"workload": w["name"], "sketches": count, "offered_rows_per_s": w["rate"],
                       "seconds": w["seconds"], "warm_s": w["warm"]},
            "latency_ms": {"p50": float(np.percentile(lat, 50)) if lat.size else None,
                           "p99": float(np.percentile(lat, 99)) if lat.size else None,
                           "requests": int(lat.size)},
            "server": c, "backlog_left": len(backlog),
            "e2e": {"value": rows_done / (t_drain - t_start), "unit": "rows/s",
                    "h2d_bytes_per_step": int(submitted_rows * w["d"] * 4),
                    "d2h_bytes_per_step": 0},
            "gpu_launches": c["launches"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    w = config(args)
    if args.impl == "reference":
        return run_reference(args, w)
    if args.workload == "c3":
        return run_batch(args, w)
    if args.workload == "c4":
        return run_serve(args, w)
    import numpy as np
    import torch
    from paper_1501_06561_gb300 import fd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fd.load()

    A_host = make_rows(w, rank)
    A = torch.from_numpy(A_host).cuda()
    B = torch.empty(w["ell"], w["d"], device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sk = fd.FDSketch(w["d"], w["ell"], w["variant"], w["alpha"], w["prec"],
                     buffer_rows=w.get("buffer_rows"))

    def step(s, src):
        s.reset()
        s.append(src)
        s.sketch(out=B)

    for _ in range(args.warmup):
        step(sk, A)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0.record(stream)
    ev[0].record(stream)
    for i in range(args.steps):
        step(sk, A)
        ev[i + 1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    per_step = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps))
    step_ms = {"median": per_step[len(per_step) // 2] if len(per_step) % 2
               else 0.5 * (per_step[len(per_step) // 2 - 1] + per_step[len(per_step) // 2]),
               "min": per_step[0], "max": per_step[-1]}
    clk = clocks.stop()
    # per-kernel device times from one more step, outside the timed region
    # (the events bracketing every launch would otherwise be timed too)
    sk.profile(True)
    step(sk, A)
    ktimes = sk.kernel_times()
    sk.profile(False)
    ms = max_over_ranks(ms, world)
    value = w["n"] * world / (ms / 1e3)
    st = sk.stats()
    launches = sum(c for c, _ in ktimes.values()) * args.steps
    # accuracy of this run: cov-err of the sketch against the whole stream
    cov = sk.cov_err(A)
    # bookkeeping along the stream (untimed; its own pass over the rows)
    try:
        trajectory = mass_trajectory(sk, A, B)
    except Exception as ex:  # a diagnostic: never cost the result line
        trajectory = {"error": f"{type(ex).__name__}: {ex}"}

    # end to end through host buffers (pinned staging and copies inside)
    e2e = None
    if not args.no_e2e:
        Bh = np.empty((w["ell"], w["d"]), dtype=np.float32)
        sk.reset()
        sk.append(A_host[: 4 * w["ell"]])
        sk.sketch()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            sk.reset()
            sk.append(A_host)
            Bh = sk.sketch(dtype=np.float32)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / max(1, args.steps)
        e2e = {"value": w["n"] * world / dt, "unit": "rows/s",
               "h2d_bytes_per_step": int(A_host.nbytes), "d2h_bytes_per_step": int(Bh.nbytes)}

    # plain FP32 CUDA-core update on the same stream, for the matched-error comparison
    plain = None
    if not args.no_plain and w["prec"] != "fp32":
        sp = fd.FDSketch(w["d"], w["ell"], w["variant"], w["alpha"], "fp32",
                         buffer_rows=w.get("buffer_rows"))
        step(sp, A)
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        step(sp, A)
        q1.record(stream)
        torch.cuda.synchronize()
        pms = q0.elapsed_time(q1)
        pce = sp.cov_err(A)
        # matched error: |cov-err(mixed) - cov-err(plain)| <= 1e-5 absolute
        plain = {"value": w["n"] / (pms / 1e3), "unit": "rows/s", "cov_err": pce,
                 "cov_err_delta": abs(cov - pce), "matched_within_1e-5": abs(cov - pce) <= 1e-5,
                 "mass_account": mass_account(sp.stats())}
        sp.close()

    # sharded: P contiguous shards, one handle and CUDA stream each (their
    # reductions run concurrently on different SMs), then fd_merge pairwise.
    # A different FD run from the sequential stream, reported beside it.
    sharded = None
    if args.shards and args.shards > 1 and rank == 0:
        P = args.shards
        cuts = [w["n"] * i // P for i in range(P + 1)]
        streams = [torch.cuda.Stream() for _ in range(P)]
        shs = [fd.FDSketch(w["d"], w["ell"], w["variant"], w["alpha"], w["prec"], stream=st,
                           buffer_rows=w.get("buffer_rows"))
               for st in streams]

        def sharded_run():
            for h, a, b in zip(shs, cuts[:-1], cuts[1:]):
                h.reset()
                h.append(A[a:b])
            root = fd.merge_tree(shs)
            root.sketch(out=B)
            return root

        sharded_run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = max(1, args.steps)
        for _ in range(reps):
            root = sharded_run()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        sharded = {"shards": P, "value": w["n"] / dt, "unit": "rows/s",
                   "cov_err": root.cov_err(A),
                   "timing": "host wall clock around the whole run (appends, merges, sketch)",
                   "note": "contiguous shards sketched concurrently, merged pairwise with fd_merge"}
        for h in shs:
            h.close()

    if rank != 0:
        sk.close()
        return 0
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FP32 FMA
    n_eig, ms_eig = ktimes["eig"]
    L = w.get("buffer_rows") or (w["ell"] if w["variant"] == "fastpfd" else 2 * w["ell"])
    eig_flops = 9.0 * L ** 3  # textbook dense symmetric eigensolve with vectors
    achieved = (eig_flops / (ms_eig / max(n_eig, 1) / 1e3)) / 1e12 if n_eig else None
    sm_peak = alu_peak / nsm
    roofline = {"bound": "alu", "kernel": "eigensolve + shrink (one CTA per reduction)",
                "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": (achieved / alu_peak) if achieved else None,
                "traffic": EIG_TRAFFIC.get((w["ell"], w["prec"], w["variant"], L)),
                "traffic_source": "ncu capture, DRAM bytes per eigensolve launch",
                "peak_source": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                "algorithmic_flops_per_launch": eig_flops,
                "avg_launch_us": (ms_eig / n_eig * 1e3) if n_eig else None,
                # the reductions of one stream form a serial chain, so each
                # eigensolve runs on one SM: its share of the chip's peak
                "per_sm": {"peak": sm_peak,
                           "frac": (achieved / sm_peak) if achieved else None}}
    kshare = {k: {"launches": c, "ms_per_step": m,
                  "share": (m / sum(x for _, x in ktimes.values())) if ktimes else None}
              for k, (c, m) in ktimes.items()}
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        cpu = cpu_baseline(w, args.cpu_sample_rows or default_sample_rows(w))
    line = {
        "metric": METRIC_SINGLE,
        "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16x3": "bf16x3 (fp32 accumulate), fp32 eig refined with the original Gram, "
                            "f64 shrink",
                  "fp32": "f32, fp32 eig refined with the original Gram, f64 shrink",
                  "fp64": "f64"}[w["prec"]],
        "data": "synthetic",
        "config": {"workload": w["name"], "ell": w["ell"], "variant": w["variant"],
                   "alpha": w["alpha"], "prec": w["prec"], "rows_per_step": w["n"],
                   "buffer_rows": w.get("buffer_rows") or (w["ell"] if w["variant"] == "fastpfd"
                                                           else 2 * w["ell"]),
                   "input_bytes": int(A_host.nbytes),
                   "l2": "input larger than L2 (no flush needed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "cov_err": cov, "mass_account": mass_account(st), "mass_trajectory": trajectory,
        "reductions_per_step": st["reductions"],
        "eig_fallbacks_per_step": st.get("eig_fallbacks"),
        "step_ms": step_ms,
        "plain_fp32": plain, "sharded": sharded,
        "roofline": roofline, "kernels": kshare,
        "gpu_launches": int(launches + 2 * args.steps),
        "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    sk.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
