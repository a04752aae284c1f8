#!/usr/bin/env python
"""Benchmark of the randomized minimal-norm solver on one GB300.

Workload (the precision workload): m = 2048, n = 262144, A = U diag(sigma) V^*
stored complex64 (4.3 GB), sigma log-spaced from 1 to 1e-5, complex Gaussian b,
eps = 1e-10, l = 4m; mixed precision, with the plain FP64 form timed on the same
inputs beside it. A step is one whole solve of the hot path, Steps 1-5:
minnorm_sketch (SRFT sketch, pivoted QR, P R^{-1}) + minnorm_solve
(preconditioned CG inside the exact-residual refinement) with A and b resident
in HBM. A (4.3 GB) is larger than L2 (129 MB), so no flush is needed between
steps. `--workload c2` runs the plain-method workload instead (512 x 65536
complex128, sigma 1..1e-6, eps 1e-12).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference      # the CPU oracle (Steps 1-5 in FP64)

Under torchrun each rank solves its own system (independent replicas, weak
scaling; the solver has no exchange step) and rank 0 prints one JSON line.
"""
import argparse
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

METRIC = "solves/s at <=1e-10 rel. error (mixed vs plain FP64 GPU); CG matvec HBM GB/s"
# the precision workload (the one the metric is quoted on) and the plain-method workload
WORKLOADS = {
    "c3": dict(m=2048, n=262144, exponent=5, dtype="c64", eps=1e-10, seed=1003,
               name="2048x262144 complex64 (4.3 GB), sigma 1..1e-5, complex Gaussian b, eps 1e-10, l = 4m "
                    "(precision workload)"),
    "c2": dict(m=512, n=65536, exponent=6, dtype="c128", eps=1e-12, seed=1002,
               name="512x65536 complex128 (512 MiB), sigma 1..1e-6, complex Gaussian b, eps 1e-12, l = 4m "
                    "(plain-method workload)"),
}
W = WORKLOADS["c3"]
WORKLOAD_NAME = W["name"]
# O1 (the oracle's dense pivoted-QR solve, ~8 m^2 n flops on the host) is run for the error
# report only up to this many entries of A; above it the oracle's O2 solve (Steps 1-5, FP64)
# of the cpu_baseline sample is the comparison
O1_MAX_ENTRIES = 512 * 65536
# a budget for the reference arm's timed whole O2 solves (seconds of host time)
REFERENCE_BUDGET_S = 240.0
FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s
# DRAM bytes (read + write) per launch of a kernel class, keyed by (workload, class), from one ncu
# capture of the current kernels: on the plain-method workload class 3 = qrp_reg_kernel<16>
# (16.91 + 2.77 MB) + prinv_kernel<1> (2.14 MB + 0.5 KB); Y (16 MiB) stays in L2 through the QR,
# so traffic is one read of Y.
PROFILED_TRAFFIC = {("c2", 3): 21.82e6}
# class 0: the CG's A^* w pass, or both products in one pass over A (mixed precision, 512 < m <= 4096)
KERNEL_CLASSES = {0: "cg_product", 1: "cg_forward_product", 2: "exact_residual", 3: "pivoted_qr",
                  4: "srft_sketch", 5: "cg_fused", 6: "qrp_triangle", 7: "r_inverse"}
# the blocked QR of tall sketches (l > 2048) does its trailing updates as FP64-accurate products on
# the tensor cores: 43 (adjoint) and 34 (update) BF16 slice-pair products per FP64 multiply-add,
# the two products carrying equal flops, so its FP64-equivalent peak is the BF16 peak / 38.5
OZAKI_MEAN_PAIRS = 38.5
REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle error check and CPU baseline")
    ap.add_argument("--m", type=int, default=0, help="rows (profiling runs of a smaller case)")
    ap.add_argument("--n", type=int, default=0, help="columns (profiling runs of a smaller case)")
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "batch", "block", "products", "paper"],
                    help="c3: the benchmark line (precision workload); c2: the plain-method workload "
                         "(512x65536 complex128); batch / block: the batching and block right-hand-side "
                         "workloads, measured on their own (one line each, not the benchmark line); products: "
                         "the block-CG products alone (tensor cores), 4096x131072 complex64, 32 columns; paper: "
                         "the shapes of the paper's Tables 1-4 with its b, 10 T-seeds each")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 4:
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            try:
                bits = int(r[3], 16)
            except ValueError:
                continue
            for b, name in REASON_BITS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("MINNORM_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def replica_seed(rank, w=None):
    """Seed of the system rank `rank` solves: every replica gets its own A and b."""
    return (w or W)["seed"] + 100 * rank


def aggregate_value(world, steps, ms_max):
    """Whole-job solves/s: every rank solved `steps` systems; the job took the slowest rank's time."""
    return world * steps / (ms_max / 1000.0)


def batch_cost(m, n):
    """Relative cost of one system of the batch: its QR (~m^2 l, l = 4m) and its passes over A (~m n
    each, a number of them proportional to m for the refinement's fixed-point passes): m^3 + m^2 n."""
    return float(m) ** 3 + float(m) ** 2 * n


def partition_batch(shapes, world):
    """Shards of the batch's independent systems over `world` GPUs, balanced by cost: systems in
    decreasing cost, each to the least-loaded rank (ties to the lower rank). Returns, per rank, the
    sorted indices of its systems; no system is shared and no exchange is needed."""
    order = sorted(range(len(shapes)), key=lambda i: (-batch_cost(*shapes[i]), i))
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += batch_cost(*shapes[i])
    return [sorted(p) for p in parts]


def reduce_max(pg, value, device):
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg, device):
    if pg is not None:
        import torch
        pg.barrier(device_ids=[device.index]) if device.type == "cuda" else pg.barrier()


def run_oracle_solve(A, b, seed=1, exponent=None):
    """The oracle's Steps 1-5 (FP64, literal), one solve: returns (seconds, x)."""
    import oracle
    m, n = A.shape
    l = 4 * m
    kappa = 10.0 ** (W["exponent"] if exponent is None else exponent)
    if A.dtype != np.complex128:
        A = A.astype(np.complex128)       # the stored values, exactly
    delta = (1e-14 * kappa) ** 2 * m / n       # the paper's Step 4 request (Section 7)
    P = oracle.draw_params(n, l, seed)
    t0 = time.perf_counter()
    out = oracle.minnorm_randomized(P, A, b, delta, maxit=500)
    return time.perf_counter() - t0, out["x"]


def reference_arm(args):
    """The oracle's O2 (Steps 1-5 literally, FP64, all host cores) on the benchmark workload's
    inputs. A step is one whole solve. One solve of the precision workload takes about a minute
    on the host, so the arm times at most `--steps` solves within REFERENCE_BUDGET_S (at least
    one) after at most one warm-up solve (the oracle has no compilation or cache to warm), and
    prints the numbers it actually ran."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import synth
    w = WORKLOADS["c2" if args.workload == "c2" else "c3"]
    s = synth.make_system(w["m"], w["n"], w["exponent"], w["seed"], dtype=w["dtype"])
    warm = min(max(0, args.warmup), 1)
    for _ in range(warm):
        run_oracle_solve(s.A, s.b, exponent=w["exponent"])
    times = []
    while len(times) < max(1, args.steps) and (not times or sum(times) + times[-1] <= REFERENCE_BUDGET_S):
        times.append(run_oracle_solve(s.A, s.b, exponent=w["exponent"])[0])
    total = sum(times)
    value = len(times) / total
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": len(times), "steps_requested": args.steps, "warmup": warm, "warmup_requested": args.warmup,
        "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "m": w["m"], "n": w["n"], "l": 4 * w["m"],
                                        "eps": w["eps"], "storage": w["dtype"]},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": "%d whole solves (Steps 1-5, FP64, oracle O2) of the workload, %.1f s (at most "
                                   "%d requested, within a %.0f s budget)" % (len(times), total, args.steps,
                                                                              REFERENCE_BUDGET_S)},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def class_amount(k, m, n, l, launches):
    """Algorithmic work of `launches` timed regions of kernel class k for an m x n system (mixed
    precision, complex64 products): (amount, unit, bound)."""
    if k in (0, 1, 5):     # one complex64 pass over A per CG product / fused iteration
        return launches * 8.0 * m * n, "GB/s", "hbm"
    if k == 2:             # x = A^* y and b - A x over the 16-byte fixed-point A
        return launches * 2 * 16.0 * m * n, "GB/s", "alu"
    if k == 3:             # the QR of Y: FP64 (l <= 2048) or blocked with tensor-core products
        return launches * 8.0 * m * m * (l - m / 3.0), "TFLOP/s", "tensor" if l > 2048 else "alu"
    if k == 6:             # the pivoted QR of the m x m triangle
        return launches * 16.0 * m ** 3 / 3.0, "TFLOP/s", "alu"
    if k == 7:             # P R^-1: by blocks with tensor-core updates for the blocked QR's sketches
        return launches * 8.0 * m ** 3 / 6.0, "TFLOP/s", "tensor" if l > 2048 and m >= 256 else "alu"
    return launches * (8.0 * m * n + 16.0 * l * m), "GB/s", "hbm"   # sketch: read A once, write Y


def cg_pass_time(stats, cg_iters):
    """Milliseconds per pass over A of the CG and passes per iteration, from the kernel classes'
    (launches, ms) and the CG iterations the solves report: the fused solve (class 5) and the one-pass
    product (class 0 alone) read A once per iteration, the two-pass form (classes 0 and 1) twice. The
    two-pass and one-pass forms enqueue their iterations in chunks, and the launches after the CG's test
    has fired return at once: the iterations, not the launches, count the passes (those launches' few
    microseconds stay in the time, so the figure is conservative)."""
    one_pass = stats[5][0] > 0 or (stats[0][0] > 0 and stats[1][0] == 0)
    if stats[5][0] > 0:
        ms = stats[5][1] / max(1, cg_iters)
    elif one_pass:
        ms = stats[0][1] / max(1, cg_iters)
    else:
        ms = (stats[0][1] + stats[1][1]) / max(1, 2 * cg_iters)
    return ms, (1 if one_pass else 2)


def side_roofline(shapes, stats_of, pk):
    """Roofline of the dominant kernel class over the last step: stats_of(i, k) -> (launches, ms)
    for system i; shapes: (m, n) per system."""
    totals = {}
    for k in KERNEL_CLASSES:
        amount, ms, unit, bound = 0.0, 0.0, None, None
        for i, (m, n) in enumerate(shapes):
            nl, t = stats_of(i, k)
            a, unit, bound = class_amount(k, m, n, min(4 * m, n), nl)
            amount += a
            ms += t
        totals[k] = (amount, ms, unit, bound)
    dom = max(totals, key=lambda k: totals[k][1])
    amount, ms, unit, bound = totals[dom]
    if ms <= 0:
        return None
    if unit == "GB/s":
        achieved = amount / (ms / 1000.0) / 1e9
        peak, src = pk["hbm_gbs"], "measured HBM copy"
        if dom == 2:   # integer-ALU bound: report the bytes rate against HBM for scale
            src = "measured HBM copy (the pass is integer-ALU bound)"
    elif bound == "tensor":
        achieved = amount / (ms / 1000.0) / 1e12
        peak = pk["bf16_tflops"] / OZAKI_MEAN_PAIRS
        src = "FP64-equivalent: measured BF16 peak / %.1f slice pairs" % OZAKI_MEAN_PAIRS
    else:
        achieved = amount / (ms / 1000.0) / 1e12
        peak, src = FP64_NOMINAL_TFLOPS, "FP64 from unit counts and clock"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": None, "kernel": KERNEL_CLASSES[dom], "peak_source": src,
            "ms_by_class": {KERNEL_CLASSES[k]: round(v[1], 3) for k, v in totals.items()}}


def side_workload(args):
    """The batching workload (256 systems, m uniform in [32, 512], n = m k, k uniform in [8, 64],
    complex64, sigma 1..1e-4, eps 1e-10) or the block right-hand-side workload (4096 x 131072
    complex64, sigma 1..1e-6, 64 complex Gaussian right-hand sides, eps 1e-10), built on the GPU.
    A step is the whole workload: every system's Steps 1-5, or one sketch + all 64 solves."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_0905_4745_gb300 import minnorm as mn
    import synth
    # batch under torchrun: the 256 systems are sharded over the ranks by cost (no exchange);
    # the block workload runs on rank 0 alone
    rank, world, local, pg = dist_setup(args.gpus) if args.workload == "batch" else (0, 1, 0, None)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    steps, warmup = max(1, args.steps), max(1, args.warmup)
    if args.workload == "batch":
        all_shapes = synth.batch_shapes(256, seed=4000)
        mine = partition_batch(all_shapes, world)[rank]
        shapes = [all_shapes[i] for i in mine]
        systems = [synth.make_system(m, n, exponent=4, seed=4000 + i, dtype="c64", device=str(dev))
                   for i, (m, n) in zip(mine, shapes)]
        batch = mn.minnorm_batch_create([m for m, _ in shapes], [n for _, n in shapes], mn.C64, mn.MIXED,
                                        seed=4000, flags=mn.FLAG_TIMING, stream=stream)
        xs = [torch.empty(n, dtype=torch.complex128, device=dev) for _, n in shapes]
        As, bs = [q.A for q in systems], [q.b for q in systems]

        def step():
            return mn.minnorm_batch_solve(batch, As, bs, 1e-10, xs)

        def stats_of(i, k):
            return mn.minnorm_batch_kernel_stats(batch, i, k)
        units, name = len(all_shapes), ("batching: 256 systems, m in [32, 512], n = m k, k in [8, 64], complex64, "
                                        "sigma 1..1e-4, eps 1e-10 (mixed)")
        stat_shapes = shapes
        hbm = sum(m * n * 8 for m, n in all_shapes)
    else:
        w = synth.WORKLOADS["c5_blockrhs_4096x131072"]
        m, n, k = w["m"], w["n"], w["nrhs"]
        q = synth.make_system(m, n, w["exponent"], w["seed"], dtype="c64", nrhs=k, device="cuda:0")
        plan = mn.minnorm_plan_create(m, n, 0, mn.C64, mn.MIXED, seed=5, flags=mn.FLAG_TIMING, stream=stream)
        B = q.b.T.contiguous().T
        X = torch.empty((k, n), dtype=torch.complex128, device=dev).T

        def step():
            mn.minnorm_sketch(plan, q.A)
            return mn.minnorm_solve_many(plan, q.A, B, w["eps"], X)

        def stats_of(i, kk):
            return mn.minnorm_kernel_stats(plan, kk)
        units, name = k, "block right-hand sides: 4096x131072 complex64, sigma 1..1e-6, 64 RHS, eps 1e-10 (mixed)"
        stat_shapes = [(m, n)]
        hbm = m * n * 8
    for _ in range(warmup):
        step()
    launches0 = mn.minnorm_launch_count()
    barrier(pg, dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ck = Clocks(local)
    ck.__enter__()
    e0.record(stream)
    statuses = []
    for _ in range(steps):
        st, infos = step()
        statuses.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    ck.__exit__()
    barrier(pg, dev)
    ms = reduce_max(pg, e0.elapsed_time(e1), dev)
    worst = reduce_max(pg, max(i["err_bound"] for i in infos), dev)
    status = int(reduce_max(pg, float(max(statuses)), dev))
    if rank != 0:
        pg.destroy_process_group()
        return 0
    pk, _ = peaks()
    roof = side_roofline(stat_shapes, stats_of, pk)
    cpu = None
    if not args.no_oracle:
        if args.workload == "batch":
            total, count = 0.0, 0
            while count < len(systems) and (total < 10.0 or count == 0):     # systems in index order, ~10 s
                A_np = systems[count].A.cpu().numpy().astype(np.complex128)
                secs, _ = run_oracle_solve(A_np, systems[count].b.cpu().numpy(), seed=4000 + mine[count])
                total += secs
                count += 1
            cpu = {"value": count / total, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "the first %d systems of rank 0's share of the batch (Steps 1-5, FP64, oracle O2), "
                             "%.1f s" % (count, total)}
        else:
            cpu = {"value": None, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "none: one oracle solve of this workload exceeds the bounded sample "
                             "(its pivoted QR of 16384 x 4096 alone is ~2e12 flops on the host)"}
    if pg is not None:
        pg.destroy_process_group()
    print(json.dumps({"metric": "solves/s (%s workload)" % args.workload, "value": units * steps / (ms / 1000.0),
                      "unit": "solves/s", "n_gpus": world, "steps": steps, "warmup": warmup,
                      "scaling": "strong" if args.workload == "batch" else None,
                      "ms_per_step": ms / steps, "higher_is_better": True, "dtype": "c64 products + f64 QR/R + "
                      "fixed-point residual", "data": "synthetic", "config": {"workload": name, "A_bytes": hbm},
                      "status": mn.STATUS_NAMES[status], "worst_err_bound": worst, "roofline": roof,
                      "cpu_baseline": cpu, "gpu_launches": mn.minnorm_launch_count() - launches0,
                      "clocks": ck.summary()}), flush=True)
    return 0


def products_workload(args):
    """Q = A^* W and T = A Q of the block CG (minnorm_block_products: tensor cores, split BF16) on a
    seeded 4096 x 131072 complex64 A (4.3 GB, larger than L2) and 32 columns; a step is one call
    (both products, the W and Q conversions and the final synchronisation)."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_0905_4745_gb300 import minnorm as mn
    m, n = 4096, 131072
    gen = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(m, n, dtype=torch.complex64, device="cuda", generator=gen)
    Wm = torch.randn(m, 32, dtype=torch.complex128, device="cuda", generator=gen)
    Q = torch.empty(n, 32, dtype=torch.complex128, device="cuda")
    T = torch.empty(m, 32, dtype=torch.complex128, device="cuda")
    plan = mn.minnorm_plan_create(m, n, 0, mn.C64, mn.MIXED, seed=1)
    steps, warmup = max(1, args.steps), max(1, args.warmup)
    for _ in range(warmup):
        mn.minnorm_block_products(plan, A, Wm, Q, T)
    torch.cuda.synchronize()
    launches0 = mn.minnorm_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ck = Clocks(0)
    ck.__enter__()
    e0.record()
    for _ in range(steps):
        mn.minnorm_block_products(plan, A, Wm, Q, T)
    e1.record()
    torch.cuda.synchronize()
    ck.__exit__()
    mn.minnorm_plan_destroy(plan)
    ms = e0.elapsed_time(e1) / steps
    pk, kind = peaks()
    gbs = 2 * 8.0 * m * n / (ms / 1000.0) / 1e9    # two passes over A per call
    print(json.dumps({"metric": "block-CG products (Q = A^* W and T = A Q, 32 columns)", "value": 1000.0 / ms,
                      "unit": "calls/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
                      "higher_is_better": True, "dtype": "bf16 x3 split -> f32 (tensor cores)", "data": "synthetic",
                      "config": {"workload": "4096x131072 complex64 (4.3 GB), 32 right-hand sides", "m": m, "n": n},
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                   "frac": gbs / pk["hbm_gbs"], "traffic": None, "peak_source": kind,
                                   "bytes_per_step": 2 * 8 * m * n},
                      "gpu_launches": mn.minnorm_launch_count() - launches0, "clocks": ck.summary()}), flush=True)
    return 0


# Tables 1-4 of the paper (Section 7): m, n, the randomized solve's mean time t_r (seconds, one
# 1.86 GHz Core Duo core, FP64 Fortran 77) and its worst kappa-normalised error eps_r over 10 trials
PAPER_TABLES = [(128, 16384, 2.4, 1.6e-15), (256, 16384, 5.6, 1.7e-15), (512, 16384, 20.0, 2.9e-15),
                (256, 4096, 2.0, 3.1e-15), (256, 8192, 3.2, 2.7e-15), (256, 32768, 16.0, 1.6e-15)]


def paper_workload(args):
    """The paper's own experiments (Section 7) as a second benchmark: A = U Sigma V^* with kappa =
    1e6, b = A p for p = m^{-1/2} sum eps_j v_j, l = 4m, complex128 storage, every shape of Tables 1-4
    solved with 10 SRFT seeds (mixed precision, eps 1e-12). Reports per shape the mean time of
    Steps 1-5 (plan creation excluded) and the worst ||x - p|| / ||p|| and ||x - p|| / (kappa ||p||)
    beside the paper's t_r and eps_r."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_0905_4745_gb300 import minnorm as mn
    import synth
    kappa, eps, trials = 1e6, 1e-12, 10
    rows = []
    stream = torch.cuda.current_stream()
    launches0 = mn.minnorm_launch_count()
    for idx, (m, n, t_paper, e_paper) in enumerate(PAPER_TABLES):
        s = synth.make_system(m, n, 6, 7000 + idx, rhs="paper", device="cuda:0")
        x = torch.empty(n, dtype=torch.complex128, device="cuda:0")
        pn = float(torch.linalg.norm(s.p))
        total_ms, worst, statuses = 0.0, 0.0, []
        for tseed in range(1, trials + 1):
            plan = mn.minnorm_plan_create(m, n, 0, mn.C128, mn.MIXED, seed=tseed, stream=stream)
            try:
                mn.minnorm_sketch(plan, s.A)        # warm the plan's first use (tuning, caches)
                mn.minnorm_solve(plan, s.A, s.b, eps, x, allow=(mn.OK, mn.EFLOOR, mn.ENOCONV))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                mn.minnorm_sketch(plan, s.A)
                st, _ = mn.minnorm_solve(plan, s.A, s.b, eps, x, allow=(mn.OK, mn.EFLOOR, mn.ENOCONV))
                e1.record(stream)
                torch.cuda.synchronize()
                total_ms += e0.elapsed_time(e1)
                statuses.append(st)
                worst = max(worst, float(torch.linalg.norm(x - s.p)) / pn)
            finally:
                mn.minnorm_plan_destroy(plan)
        rows.append({"m": m, "n": n, "l": 4 * m, "ms_mean": total_ms / trials,
                     "solves_per_s": 1000.0 * trials / total_ms, "rel_err_worst": worst,
                     "eps_r_worst": worst / kappa, "status": mn.STATUS_NAMES[max(statuses)],
                     "paper_t_r_s": t_paper, "paper_eps_r": e_paper})
        del s
    total = sum(r["ms_mean"] for r in rows)
    print(json.dumps({"metric": "solves/s on the paper's Tables 1-4 shapes (kappa 1e6, the paper's b, 10 SRFT "
                               "seeds each; worst error)", "value": 1000.0 * len(rows) / total, "unit": "solves/s",
                      "higher_is_better": True, "dtype": "c64 products + f64 QR/R + fixed-point residual",
                      "data": "synthetic", "config": {"workload": "paper Tables 1-4 shapes, complex128, l = 4m, "
                                                                  "eps 1e-12 (mixed)"},
                      "shapes": rows, "gpu_launches": mn.minnorm_launch_count() - launches0}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "products":
        return products_workload(args)
    if args.workload == "paper":
        return paper_workload(args)
    if args.workload not in ("c3", "c2"):
        return side_workload(args)
    w = WORKLOADS[args.workload]
    import torch
    rank, world, local, pg = dist_setup(args.gpus)
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    import __graft_entry__ as g
    if rank == 0:
        g.build()
    barrier(pg, device)
    g.build()
    from paper_0905_4745_gb300 import minnorm as mn
    import synth

    m, n, eps = args.m or w["m"], args.n or w["n"], w["eps"]
    full = (m, n) == (w["m"], w["n"])
    c64 = w["dtype"] == "c64"
    # inputs built on the GPU from the seeded draws (the 4.3 GB workload takes ~40 s; no host cache)
    s = synth.make_system(m, n, w["exponent"], replica_seed(rank, w), dtype=w["dtype"], device=str(device))
    A, b = s.A, s.b
    del s
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    prec_main = mn.MIXED if args.precision == "mixed" else mn.FP64
    dt = mn.C64 if c64 else mn.C128
    plans = {}
    for name, prec in (("main", prec_main), ("other", mn.FP64 if prec_main == mn.MIXED else mn.MIXED)):
        plans[name] = mn.minnorm_plan_create(m, n, 0, dt, prec, seed=1, flags=mn.FLAG_TIMING, stream=stream)
    x = torch.empty(n, dtype=torch.complex128, device=device)

    def step(plan):
        mn.minnorm_sketch(plan, A)
        st, info = mn.minnorm_solve(plan, A, b, eps, x, allow=(mn.OK, mn.EFLOOR, mn.ENOCONV))
        return st, info

    def timed(plan, steps, warmup, clocks=False):
        for _ in range(warmup):
            step(plan)
        stats = {k: [0, 0.0] for k in KERNEL_CLASSES}
        infos = []
        launches0 = mn.minnorm_launch_count()
        barrier(pg, device)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ck = Clocks(local if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
        if clocks:
            ck.__enter__()
        e0.record(stream)
        for _ in range(steps):
            st, info = step(plan)
            infos.append((st, info))
            for k in KERNEL_CLASSES:
                nl, ms = mn.minnorm_kernel_stats(plan, k)
                stats[k][0] += nl
                stats[k][1] += ms
        e1.record(stream)
        torch.cuda.synchronize()
        if clocks:
            ck.__exit__()
        barrier(pg, device)
        ms = e0.elapsed_time(e1)
        return ms, stats, infos, mn.minnorm_launch_count() - launches0, (ck.summary() if clocks else None)

    ms_main, stats, infos, launches, clk = timed(plans["main"], args.steps, args.warmup, clocks=True)
    xc, xs, ck, _ = mn.minnorm_plan_tuning(plans["main"])
    ms_max = reduce_max(pg, ms_main, device)
    value = aggregate_value(world, args.steps, ms_max)
    x_main = x.clone()
    last_st, last_info = infos[-1]
    ms_other, stats_other, infos_other, _, _ = timed(plans["other"], max(3, args.steps // 2), 2)
    ms_other = reduce_max(pg, ms_other, device)
    other_value = aggregate_value(world, max(3, args.steps // 2), ms_other)
    x_other = x.clone()

    # end to end through the public API with host buffers (pinned): H2D of A and b, D2H of x
    A_h = A.cpu().pin_memory()
    b_h = b.cpu().pin_memory()
    x_h = torch.empty(n, dtype=torch.complex128).pin_memory()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(2):
        mn.minnorm_solve_host(plans["main"], A_h, b_h, eps, x_h, allow=(mn.OK, mn.EFLOOR, mn.ENOCONV))
    barrier(pg, device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    e2e_walls = []
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        mn.minnorm_solve_host(plans["main"], A_h, b_h, eps, x_h, allow=(mn.OK, mn.EFLOOR, mn.ENOCONV))
        e2e_walls.append(round(1000 * (time.perf_counter() - t1), 2))
    f1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    e2e_ms = max(f0.elapsed_time(f1), 1000 * wall)
    e2e_ms = reduce_max(pg, e2e_ms, device)
    e2e_value = aggregate_value(world, e2e_steps, e2e_ms)

    for p in plans.values():
        mn.minnorm_plan_destroy(p)

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return 0

    # roofline of the dominant kernel class over the timed region
    pk, pk_kind = peaks()
    dom = max(KERNEL_CLASSES, key=lambda k: stats[k][1])
    l = 4 * m
    per_launch_ms = stats[dom][1] / max(1, stats[dom][0])
    mixed = prec_main == mn.MIXED
    esz = 8 if (mixed or c64) else 16      # bytes per entry of the A the CG products stream
    if dom in (0, 1, 5):
        # per CG iteration (k = 5 counts iterations): one pass over A in the fused kernel
        bytes_per = m * n * esz
        achieved = bytes_per / (per_launch_ms / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s"}
    elif dom == 2:
        flops = 2 * m * n * 50          # two passes, ~50 FP64 flops per complex element (TwoProd/TwoSum)
        achieved = flops / (per_launch_ms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s"}
    elif dom in (3, 6, 7):
        flops, _, bound = class_amount(dom, m, n, l, 1)
        achieved = flops / (per_launch_ms / 1000.0) / 1e12
        peak = pk["bf16_tflops"] / OZAKI_MEAN_PAIRS if bound == "tensor" else FP64_NOMINAL_TFLOPS
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s"}
    else:
        bytes_per = m * n * esz + 16 * l * m
        achieved = bytes_per / (per_launch_ms / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = PROFILED_TRAFFIC.get((args.workload, dom)) if full else None
    roof["kernel"] = KERNEL_CLASSES[dom]
    roof["peak_source"] = (pk_kind if roof["unit"] == "GB/s" else
                           "FP64-equivalent: %s BF16 peak / %.1f slice pairs" % (pk_kind, OZAKI_MEAN_PAIRS)
                           if roof["bound"] == "tensor" else
                           "derived, not measured: FP64 from unit counts and clock, 152 SMs x 2 DFMA/clk x 2 "
                           "x 2.07 GHz (recipe table 1.25 TFLOP/s)")
    # CG matvec bandwidth (the metric's second half)
    # Per pass, over the CG iterations the solves report: the two-pass form enqueues its iterations
    # in chunks and the launches after the CG's test has fired return at once, so the launch count
    # overstates the passes (their few microseconds stay in the time: a conservative figure).
    cg_iters = sum(i["cg_iters"] for _, i in infos if i)
    cg_ms, cg_passes = cg_pass_time(stats, cg_iters)
    cg_gbs = m * n * esz / (cg_ms / 1000.0) / 1e9 if cg_ms > 0 else None
    cg_roof = None
    if cg_gbs:
        # one pass over A per CG iteration (algorithmic bytes), launch overhead included
        cg_roof = {"bound": "hbm", "achieved": cg_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                   "frac": cg_gbs / pk["hbm_gbs"], "bytes_per_pass": m * n * esz, "passes_per_iteration": cg_passes,
                   "traffic": PROFILED_TRAFFIC.get((args.workload, 5 if stats[5][0] > 0 else 0)) if full else None,
                   "peak_source": pk_kind}
    breakdown = {KERNEL_CLASSES[k]: {"launches": v[0], "ms_total": v[1]} for k, v in stats.items()}

    err_main = err_other = None
    err_kind = None
    cpu = None
    cert = None
    if not args.no_oracle:
        import oracle
        A_np, b_np = A_h.numpy(), b_h.numpy()     # the pinned host copies of the e2e leg
        total, count, x_o2 = 0.0, 0, None
        while count < 8 and (total < 10.0 or count == 0):      # a bounded sample: ~10 s, at least one solve
            secs, xo = run_oracle_solve(A_np, b_np, seed=1 + count, exponent=w["exponent"])
            x_o2 = xo if x_o2 is None else x_o2
            total += secs
            count += 1
        cpu = {"value": count / total, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d whole solve(s) (Steps 1-5, FP64, oracle O2) of the workload, %.1f s" % (count, total)}
        if m * n <= O1_MAX_ENTRIES:
            # O1: the dense pivoted-QR minimal-norm solution with double-double refinement
            p_ref = oracle.minnorm_direct(A_np, b_np, steps=5)["p"]
            err_kind = "||x - p|| / ||p||, p from the oracle's O1 (dense pivoted QR + double-double refinement)"
        else:
            # O1 would take many minutes on the host: the oracle's own O2 solve is the reference
            # (FP64 throughout, its error near kappa * 2^-53 dominates the difference)
            p_ref = x_o2
            err_kind = ("||x - x_O2|| / ||x_O2||, x_O2 from the oracle's O2 solve (Steps 1-5 in FP64, no "
                        "refinement: its own error is of order kappa * 2^-53)")
        nref = np.linalg.norm(p_ref)
        xm, xo = x_main.cpu().numpy(), x_other.cpu().numpy()
        err_main = float(np.linalg.norm(xm - p_ref) / nref)
        err_other = float(np.linalg.norm(xo - p_ref) / nref)
        # a rigorous bound of ||x - p|| / ||x|| computed by the oracle alone (its own FP64 sketch
        # and QR of A, and the double-double residual b - A x)
        bounds, cdelta = oracle.error_certificate(A_np, np.stack([b_np, b_np], 1), np.stack([xm, xo], 1),
                                                  seed=17)
        cert = {"main": float(bounds[0]), "other": float(bounds[1]), "delta": cdelta,
                "how": "oracle.error_certificate: ||R^{-*} (b - A x)|| / ((1 - delta) ||x||) with the oracle's "
                       "FP64 sketch of A (seed 17), a LAPACK QR of it and a double-double residual"}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 products + f64 QR/R + fixed-point residual" if mixed else "f64 + fixed-point residual",
        "data": "synthetic",
        "config": {"workload": w["name"] if full else
                   "%dx%d %s (profiling case, not the benchmark workload)" % (m, n, w["dtype"]),
                   "m": m, "n": n, "l": l, "eps": eps,
                   "precision": "mixed" if mixed else "fp64", "storage": "complex64" if c64 else "complex128",
                   "l2": "no flush: A (%.2f GB) exceeds L2 (129 MB)" % (m * n * (8 if c64 else 16) / 1e9),
                   "replicas": world},
        "rel_err_vs_oracle": err_main, "rel_err_kind": err_kind, "err_certificate_oracle": cert,
        "err_bound": last_info["err_bound"],
        "status": mn.STATUS_NAMES[last_st],
        "solve_info": last_info,
        "plain_fp64" if mixed else "mixed": {"value": other_value, "unit": "solves/s",
                                             "ms_per_step": ms_other / max(3, args.steps // 2),
                                             "rel_err_vs_oracle": err_other,
                                             "err_bound": infos_other[-1][1]["err_bound"]},
        "cg_matvec_gbs": cg_gbs,
        "cg_matvec_roofline": cg_roof,
        "roofline": roof,
        "kernel_breakdown": breakdown,
        "cpu_baseline": cpu,
        "tuning": {"exact_residual": {"column_chunks": xc, "row_splits": xs},
                   "cg_fused": {"l2_keep_pct": ck},
                   "how": "fastest of the candidates timed on the plan's first residual / inner solve"},
        "e2e": {"value": e2e_value, "unit": "solves/s", "step_wall_ms": e2e_walls, "h2d_bytes_per_step": m * n * (8 if c64 else 16) + m * 16,
                "d2h_bytes_per_step": n * 16},
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
