"""Benchmark: RBT + GENP solve throughput on one GB300 (or N replicas).

One step = one whole ``rbt_solve`` of the precision workload: n = 40003
(not a multiple of 4, so every butterfly layer is truncated), depth 2 on both
sides, A = D_r G D_c with G i.i.d. N(0,1) and diagonal scalings 10^U(-1.5,1.5),
one right-hand side, the factorization in the chosen working precision and
double-precision iterative refinement to a backward error <= 1e-13 (double
refactorization if refinement stalls).  A and b are resident in HBM when the
timed region starts (A is 12.8 GB, far above the 129 MB L2, so no flush is
needed); X is resident when it ends.

value = (2 n^3 / 3) / (seconds per step), in TFLOP/s (Sec. 6 counts the
solve's flops this way).  Under torchrun every rank solves its own system of
the same size (independent replicas, weak scaling).

The same JSON line also carries (rank 0):
  * the FP64 path on the same system (the comparison of the metric);
  * end to end: the same solve from pinned host buffers through the C ABI
    (rbt_solve_host: A and b read from host memory, x written back, all
    inside the timed region);
  * the other configurations, each timed with CUDA events over several
    repetitions, a 99% confidence interval and sampled clocks: n = 1003,
    d = 2; n = 20001, d = 3 with A[0,0] = 0 (and Parker's formulation on the
    identity-padded system); 2048 batched systems (FP64 and float factors
    refined in double, one persistent launch replayed from a CUDA graph);
    the differentiation of X = solve(A, B) at n = 8197 with 32 right-hand
    sides;
  * the CPU baseline: the cache-blocked OpenMP FP64 solver of oracle/ on
    every host core at n = 10000 of the same matrix family, and the plain
    oracle on one core at n = 2000.

--impl reference times the CPU oracle (plain FP64 C, one core) on a bounded
sample of the same workload (a smaller n, same matrix family) instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RBT+GENP solve TFLOP/s (2n³/3), mixed+IR vs FP64 at backward err ≤1e-13"
ORACLE_SAMPLE_N = 2000


def ci99(xs):
    """99% confidence interval of the mean of xs (Student t, len(xs) - 1 degrees of freedom)."""
    if len(xs) < 2:
        return None
    from scipy import stats
    m = statistics.fmean(xs)
    h = stats.t.ppf(0.995, len(xs) - 1) * statistics.stdev(xs) / len(xs) ** 0.5
    return [float(m - h), float(m + h)]


def flops(n):
    return 2.0 * n ** 3 / 3.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="precision", choices=["precision", "batched", "autograd", "sweep"],
                   help="precision: the headline solve (default); batched / autograd: the batching and "
                        "differentiation configurations, one JSON line each; sweep: the structure-"
                        "sensitivity study over sizes (no refinement)")
    p.add_argument("--sweep-lo", type=int, default=20480)
    p.add_argument("--sweep-hi", type=int, default=22528)
    p.add_argument("--sweep-step", type=int, default=4)
    p.add_argument("--sweep-tile", type=int, default=512, help="n_b of the tiled reference size")
    p.add_argument("--sweep-paired", action="store_true",
                   help="also solve every size with Parker's structure (the non-tiled rule) for a paired ratio")
    p.add_argument("--n", type=int, default=40003)
    p.add_argument("--depth", type=int, default=2)
    p.add_argument("--prec", default="auto")
    p.add_argument("--nb", type=int, default=0)
    p.add_argument("--kind", default="scaled", choices=["scaled", "rotation"],
                   help="butterflies: the scaled form (default) or the orthogonal rotation form")
    p.add_argument("--align", type=int, default=1, help="reference size: 1 = non-tiled, n_b = tiled")
    p.add_argument("--no-fp64", action="store_true", help="skip the one-step FP64 comparison solve")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-n", type=int, default=10000, help="order of the CPU baseline's sample")
    p.add_argument("--no-configs", action="store_true",
                   help="skip the timed sub-objects of the other configurations (n = 1003; n = 20001, d = 3; "
                        "2048 batched systems; the n = 8197 differentiation)")
    return p.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    from paper_2312_09376_gb300 import replicas
    return replicas.env()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def timed(fn, reps, warmup, index, stream=None, min_ms=0.0):
    """Time `fn` on the device: `warmup` untimed calls, then at least `reps`
    timed calls (more while the timed calls sum to less than min_ms), one
    CUDA event before the first and one after each, with nvidia-smi clocks
    sampled over the timed calls.  Returns (record, outputs of the timed calls)."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    clocks = Clocks(index)
    clocks.start()
    marks = [torch.cuda.Event(enable_timing=True)]
    marks[0].record(s)
    outs = []
    t0 = time.perf_counter()
    while len(outs) < reps or (time.perf_counter() - t0) * 1e3 < min_ms:
        outs.append(fn())
        e = torch.cuda.Event(enable_timing=True)
        e.record(s)
        marks.append(e)
    torch.cuda.synchronize()
    clk = clocks.stop()
    each = [marks[i].elapsed_time(marks[i + 1]) for i in range(len(outs))]
    return {"reps": len(each), "mean_ms": statistics.fmean(each), "ci99_ms": ci99(each), "each_ms": each,
            "clocks": clk}, outs


def _cpulist(text):
    out = []
    for part in text.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            out.extend(range(int(a), int(b) + 1))
        elif part:
            out.append(int(part))
    return out


def gpu_local_cpus(index):
    """(NUMA node, its CPUs) nearest to CUDA device `index`, from sysfs; (None, None) if unknown."""
    try:
        import torch
        p = torch.cuda.get_device_properties(index)
        bus = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        node = int(open("/sys/bus/pci/devices/%s/numa_node" % bus).read())
        if node < 0:
            return None, None
        cpus = [c for c in _cpulist(open("/sys/devices/system/node/node%d/cpulist" % node).read())
                if c in os.sched_getaffinity(0)]
        return (node, cpus) if cpus else (None, None)
    except Exception:
        return None, None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def update_bytes(n, nb, es):
    """Algorithmic DRAM bytes of all trailing updates: C read and written once
    (2 es per entry) plus both operands read once."""
    tot = 0.0
    k = 0
    while k < n:
        kb = min(nb, n - k)
        rest = n - k - kb
        tot += 2.0 * es * rest * rest + es * kb * 2.0 * rest
        k += kb
    return tot


def traffic_ratio(kernel):
    """Measured DRAM bytes per algorithmic byte of `kernel` from the committed
    ncu summary, or None when absent or when the kernel source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    except OSError:
        return None
    for f in lines:
        if f[0] != kernel:
            continue
        src = os.path.join(ROOT, f[2])
        try:
            sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:len(f[1])]
        except OSError:
            return None
        if sha != f[1]:
            return None
        return float(f[3]) / float(f[4])
    return None


def oz_update_bytes(n, outer=512, inner=64, es=8):
    """Algorithmic DRAM bytes of the updates of the two-level sliced
    factorization: per update call, C read and written once plus both
    double-float operands read once (the digit slices in between are the
    kernel's own traffic)."""
    def one(M, N, K):
        return 2.0 * es * M * N + es * K * (M + N) if M > 0 and N > 0 else 0.0
    tot = 0.0
    for k in range(0, n, outer):
        kb = min(outer, n - k)
        for j in range(k, k + kb, inner):
            jb = min(inner, k + kb - j)
            r0 = j + jb
            tot += one(n - r0, k + kb - r0, jb) + one(k + kb - r0, n - k - kb, jb)
        tot += one(n - k - kb, n - k - kb, kb)
    return tot


def update_flops(n, nb):
    """Algorithmic flops of all GENP trailing updates: sum_k 2 (n-k-kb)^2 kb."""
    tot = 0.0
    k = 0
    while k < n:
        kb = min(nb, n - k)
        rest = n - k - kb
        tot += 2.0 * rest * rest * kb
        k += kb
    return tot


# ------------------------------------------------------------ CPU oracle arm

def oracle_sample(n=ORACLE_SAMPLE_N, steps=1):
    """Time the CPU oracle's full RBT solve on an n x n sample of the workload."""
    import numpy as np  # noqa: F401

    import oracle
    from paper_2312_09376_gb300 import inputs
    A, _, _ = inputs.scaled_gaussian(n)
    B = inputs.rhs(n, 1)
    oracle.build()
    times, berrs = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        X, st, b0, berr, it = oracle.rbt_solve(A, B, 2, seed=1, refine_max=30, tol=1e-13)
        times.append(time.perf_counter() - t0)
        berrs.append(berr)
    return times, berrs


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    steps = max(1, args.steps)
    warm = max(0, args.warmup)
    oracle_sample(ORACLE_SAMPLE_N, warm) if warm else None
    times, berrs = oracle_sample(ORACLE_SAMPLE_N, steps)
    t = sum(times) / len(times)
    val = flops(ORACLE_SAMPLE_N) / t / 1e12
    sample = "full RBT+GENP solve with FP64 refinement, n=%d (same matrix family, d=2), single thread" % ORACLE_SAMPLE_N
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "rbt_genp_solve_precision", "n": args.n, "d": args.depth, "nrhs": 1,
                       "matrix": "D_r G D_c, 10^U(-1.5,1.5)", "oracle_sample_n": ORACLE_SAMPLE_N},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "berr": max(berrs)}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm

def pick_prec(args):
    """Fastest working precision whose refinement converges on this workload:
    float, TF32 and BF16 factors stall at n = 40003 (growth after a depth-2
    transform times their unit roundoff exceeds one); double-float does not,
    and its sliced tensor-core update is the fastest form of it: seven digits
    (df64tc7, 28 digit products, four refinement steps) beat eight (df64tc,
    36 products, two steps) by about 10% per solve at equal backward error."""
    return DEFAULT_PREC if args.prec == "auto" else args.prec


DEFAULT_PREC = "df64tc7"
# digit products of one sliced double-float multiply-add: S digits per entry,
# the products of weight p + q <= S + 1 (S (S + 1) / 2 of them)
DIGIT_PRODUCTS = {"df64tc": 36, "df64tc7": 28}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2312_09376_gb300 import _lib, inputs, replicas

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    _lib.load()
    n, d = args.n, args.depth
    prec = pick_prec(args)

    # synthetic input: A = D_r G D_c, b ~ N(0,1), generated on the device (seeded per rank)
    A, B = inputs.device_system(n, scaled=True, seed=replicas.system_seed(rank), device=dev)
    X = torch.empty_like(B)
    opts = _lib.make_opts(depth=d, seed=1, prec=prec, refine_max=30, tol=1e-13, fallback=True, nb=args.nb,
                          align=args.align, kind=args.kind)
    work = torch.empty(_lib.rbt_solve_workspace(opts, n, 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        return _lib.rbt_solve(opts, n, A, B, X, work)

    infos = []
    for _ in range(max(3, args.warmup)):
        infos.append(step()[1])
    torch.cuda.synchronize()

    # timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    _lib.rbt_prof_reset()
    _lib.rbt_prof_enable(True)
    l0 = _lib.rbt_kernel_launches()
    # one event before the first step and one after each step: the first and
    # last bracket the K steps, the ones between give each step's time
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = marks[0], marks[-1]
    e0.record(stream)
    for i in range(args.steps):
        infos.append(step()[1])
        marks[i + 1].record(stream)
    torch.cuda.synchronize()
    step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)]
    launches = _lib.rbt_kernel_launches() - l0
    _lib.rbt_prof_enable(False)
    clk = clocks.stop()
    prof = {k: _lib.rbt_prof_read(k) for k in _lib.PROF_CLASSES}
    ms = replicas.max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    if dist:
        dist.barrier()
    timed_infos = infos[-args.steps:]

    # the float working-copy pass (float arithmetic, HBM-bound) at this size, timed alone
    Uc = _lib.colmajor(n, d, device=dev)
    Vc = _lib.colmajor(n, d, device=dev)
    _lib.rbt_generate(n, d, 1, Uc, Vc)
    F = _lib.colmajor(n, n, dtype=torch.float32, device=dev)
    for _ in range(3):
        _lib.rbt_apply_2sided_wp(n, d, Uc, Vc, A, F, "f32")
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    reps = 10
    g0.record(stream)
    for _ in range(reps):
        _lib.rbt_apply_2sided_wp(n, d, Uc, Vc, A, F, "f32")
    g1.record(stream)
    torch.cuda.synchronize()
    f32_pass_ms = g0.elapsed_time(g1) / reps
    del F
    torch.cuda.empty_cache()

    # end to end: host buffers through the C-ABI (rbt_solve_host: A and b read
    # from pinned host memory, x written back, inside the timed region).  The
    # pinned host buffers are allocated and first touched from the CPUs of the
    # GPU's own NUMA node, so that their pages sit next to the GPU.
    node, near = gpu_local_cpus(local)
    saved_aff = os.sched_getaffinity(0)
    if near:
        os.sched_setaffinity(0, near)
    A_host = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    A_host.copy_(A.T)                           # same bytes (column-major) as the device copy
    B_host = B.cpu().pin_memory()
    X_host = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hwork = torch.empty(_lib.rbt_solve_host_workspace(opts, n, 1), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    # the copy engine's rate for the same buffer (the path rbt_solve_host does
    # not take for pinned memory), for context: A's own bytes copied over it
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    A.T.copy_(A_host, non_blocking=True)
    c1.record(stream)
    torch.cuda.synchronize()
    ce_gbs = 8.0 * n * n / (c0.elapsed_time(c1) * 1e-3) / 1e9
    _lib.rbt_solve_host(opts, n, A_host.T, B_host, X_host, hwork)   # untimed first call
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    e2e_each = []
    f0.record(stream)
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        _lib.rbt_solve_host(opts, n, A_host.T, B_host, X_host, hwork)   # synchronizes before returning
        e2e_each.append((time.perf_counter() - t0) * 1e3)
    f1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = replicas.max_over_ranks(f0.elapsed_time(f1) / args.e2e_steps, dist, dev)
    e2e_same = bool(torch.equal(X_host, X.cpu()))
    os.sched_setaffinity(0, saved_aff)
    del A_host, hwork
    torch.cuda.empty_cache()

    # one FP64 solve of the same system (the comparison path), not part of the value
    fp64 = None
    if not args.no_fp64 and rank == 0:
        o64 = _lib.make_opts(depth=d, seed=1, prec="f64", refine_max=30, tol=1e-13, fallback=False)
        w64 = torch.empty(_lib.rbt_solve_workspace(o64, n, 1), dtype=torch.uint8, device=dev)
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        X64 = torch.empty_like(X)
        _, i64 = _lib.rbt_solve(o64, n, A, B, X64, w64)
        h1.record(stream)
        torch.cuda.synchronize()
        t64 = h0.elapsed_time(h1)
        fp64 = {"ms_per_step": t64, "value": flops(n) / (t64 * 1e-3) / 1e12, "berr": i64["berr"],
                "iters": i64["iters"], "speedup_of_mixed": t64 / ms}
        del w64

    # the other configurations of the benchmark: timed sub-objects (rank 0)
    configs = None
    if not args.no_configs and rank == 0:
        del A, B, X, work
        torch.cuda.empty_cache()
        configs = {"small_n1003_d2": config_small(local),
                   "large_n20001_d3_zero_corner": config_large_zero_corner(local),
                   "batched_2048": config_batched(local),
                   "autograd_n8197_32rhs": config_autograd(local)}
        torch.cuda.empty_cache()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peaks, peak_src = measured_peaks()
    nb = args.nb or (64 if prec in ("f64", "df64") else 128)
    upd_ms, upd_n = prof["update"]
    # df64tc: 512-column panels factored in 64-column steps, every update of
    # both levels on the sliced kernel, so the update class does all the
    # flops of 64-column blocking
    upd_flops = update_flops(n, nb if prec not in DIGIT_PRODUCTS else 64) * args.steps
    if prec in ("tf32", "bf16") or prec in DIGIT_PRODUCTS:
        # the burst figure: a true ceiling for a kernel timed over its own launches
        peak = peaks.get("bf16_tflops", 1900.0) * (0.5 if prec == "tf32" else 1.0)
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": peak,
                "peak_source": "%s bf16 burst%s" % (peak_src, " x 1/2 (tf32 nominal ratio)" if prec == "tf32" else "")}
    elif prec == "df64":
        # plain-ALU bound: a double-float multiply-add costs 12 FP32 operations
        # (lazy accumulation form), so its peak is 152 SMs x 128 FP32 lanes x
        # clock / 12 multiply-adds, 2 flops each
        mhz = (clk or {}).get("sm_mhz", 1900.0)
        peak = 152 * 128 * mhz * 1e6 / 12 * 2 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
                "peak_source": "152 SMs x 128 FP32 lanes x %.0f MHz (sampled) / 12 FP32 ops per double-float FMA x 2" % mhz}
    elif prec == "f64":
        mhz = (clk or {}).get("sm_mhz", 1900.0)
        peak = 152 * 2 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
                "peak_source": "152 SMs x 2 FP64 FMA/clk (probe-measured issue rate) x 2 x %.0f MHz" % mhz}
    else:
        # plain-ALU bound: 152 SMs x 128 FP32 FMA lanes x 2 flops x clock (under-load median)
        mhz = (clk or {}).get("sm_mhz", 1900.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz (sampled SM clock)" % mhz}
    # achieved counts the method's own flops (the GENP updates' multiply-adds)
    achieved = upd_flops / (upd_ms * 1e-3) / 1e12 if upd_ms > 0 else None
    if prec in DIGIT_PRODUCTS and achieved:
        # what the tensor pipe executes: every double-float multiply-add is
        # DIGIT_PRODUCTS[prec] exact BF16 digit products
        ex = DIGIT_PRODUCTS[prec] * achieved
        roof["executed"] = {"achieved": ex, "unit": "TFLOP/s", "frac": ex / peak,
                            "frac_of_sustained": ex / peaks.get("bf16_tflops_sustained", 1700.0),
                            "digit_products_per_multiply_add": DIGIT_PRODUCTS[prec],
                            "note": "BF16 digit-product flops the tensor pipe executes; frac <= 1 by construction "
                                    "of the burst peak, the sustained one is a cuBLAS loop under the power cap"}
        fp64_peak = 152 * 2 * 2 * (clk or {}).get("sm_mhz", 2070.0) * 1e6 / 1e12
        roof["vs_fp64_pipe_peak"] = achieved / fp64_peak
        roof["note"] = ("achieved = the method's flops (sum of 2 rest^2 64 over the trailing updates) over the "
                        "update kernel's own launches; the BF16 pipe executes %d times that" % DIGIT_PRODUCTS[prec])
    # df64: the persistent 128 x 128 kernel takes every update of at least 2048 x 2048
    # (all but the last few percent of the flops)
    kname = {"df64": "gemm_sub_df64_pipe_kernel", "tf32": "tc_update_kernel", "bf16": "tc_update_kernel",
             "df64tc": "oz_update_kernel<8>", "df64tc7": "oz_update_kernel<7>"}.get(prec, "gemm_sub_kernel")
    es = {"df64": 8, "f64": 8, "df64tc": 8, "df64tc7": 8}.get(prec, 4)
    ratio = traffic_ratio(kname)
    alg_bytes = oz_update_bytes(n) if prec in DIGIT_PRODUCTS else update_bytes(n, nb, es)
    alg_per_launch = alg_bytes * args.steps / max(upd_n, 1)
    roof.update({"kernel": "genp trailing update (%s)" % kname, "achieved": achieved,
                 "frac": (achieved / roof["peak"]) if achieved else None,
                 "traffic": ratio * alg_per_launch if ratio else None,
                 "algorithmic_bytes_per_launch": alg_per_launch,
                 "launches": upd_n, "avg_launch_ms": upd_ms / max(upd_n, 1)})
    tr_ms, tr_n = prof["transform"]
    wbytes = {"f64": 8, "df64": 8, "df64tc": 8, "df64tc7": 8}.get(prec, 4)
    tbytes = (8.0 + wbytes) * n * n
    transform = {"kernel": "fused two-sided transform (A -> working copy) inside the solve", "launches": tr_n,
                 "ms_per_launch": tr_ms / max(tr_n, 1), "algorithmic_bytes": tbytes,
                 "achieved_gbs": tbytes / (tr_ms / max(tr_n, 1) * 1e-3) / 1e9 if tr_ms > 0 else None,
                 "peak_gbs": peaks.get("hbm_gbs"),
                 "bound": "hbm", "frac": (tbytes / (tr_ms / max(tr_n, 1) * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6793.1))
                 if tr_ms > 0 else None,
                 "note": ("double-float arithmetic on the FP32 pipes (HBM-bound)" if es == 8 and prec != "f64"
                          else "double arithmetic (FP64-pipe bound on this GPU)" if prec == "f64"
                          else "float arithmetic from the double input (HBM-bound)")}
    tr_ratio = traffic_ratio("fused2_wp_kernel<2,df64>") if es == 8 and prec != "f64" else None
    transform["traffic"] = tr_ratio * tbytes if tr_ratio else None
    f32_bytes = 12.0 * n * n
    f32_pass = {"kernel": "fused2_wp_kernel<2,float>: all layers in one pass, A double in, float copy out",
                "bound": "hbm", "ms_per_launch": f32_pass_ms, "algorithmic_bytes": f32_bytes,
                "achieved": f32_bytes / (f32_pass_ms * 1e-3) / 1e9, "unit": "GB/s", "peak": peaks.get("hbm_gbs"),
                "frac": f32_bytes / (f32_pass_ms * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6746.3),
                "traffic": (traffic_ratio("fused2_wp_kernel<2,float>") or 0.0) * f32_bytes or None}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_tier_b(args.cpu_n)
        times, berrs = oracle_sample(ORACLE_SAMPLE_N, 1)
        cpu["oracle_tier_a"] = {"value": flops(ORACLE_SAMPLE_N) / times[0] / 1e12, "unit": "TFLOP/s", "cores": 1,
                                "sample": "the plain oracle's solve at n=%d, single thread, %.1f s"
                                          % (ORACLE_SAMPLE_N, times[0])}
    value = replicas.aggregate_tflops(world, flops(n), ms)
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "%s+f64" % prec, "data": "synthetic",
        "config": {"workload": "rbt_genp_solve_precision", "n": n, "d": d, "nrhs": 1,
                   "matrix": "D_r G D_c, G~N(0,1), D=10^U(-1.5,1.5)", "prec": prec, "nb": nb if prec not in DIGIT_PRODUCTS else "512/64",
                   "refine": "FP64 IR to berr<=1e-13, %s on stall" % ("eight-digit then FP64 refactor"
                                                                        if prec == "df64tc7" else "FP64 refactor"),
                   "l2": "inputs 12.8 GB >> L2, no flush",
                   "parallelism": "replicas" if world > 1 else "single", "kind": args.kind, "align": args.align},
        "step_ms": {"each": step_ms, "ci99": ci99(step_ms)},
        "berr": max(i["berr"] for i in timed_infos), "iters": [i["iters"] for i in timed_infos],
        "fell_back": [i["fell_back"] for i in timed_infos],
        "roofline": roof, "transform": transform, "transform_f32_pass": f32_pass,
        "breakdown_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "e2e": {"value": replicas.aggregate_tflops(world, flops(n), ms_e2e), "unit": "TFLOP/s",
                "h2d_bytes_per_step": 8 * n * n + 8 * n, "d2h_bytes_per_step": 8 * n, "ms_per_step": ms_e2e,
                "each_ms": e2e_each, "api": "rbt_solve_host (pinned host A, b, x)",
                "same_x_as_device_run": e2e_same, "copy_engine_h2d_gbs": ce_gbs, "host_numa_node": node,
                "copy_overhead_ms": ms_e2e - ms},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
        "fp64_path": fp64,
        "configs": configs,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------- the other configurations

def _solve_record(rec, infos, n):
    """Timing record of a solve plus its throughput and outcome."""
    rec = dict(rec)
    rec["tflops"] = flops(n) / (rec["mean_ms"] * 1e-3) / 1e12
    rec["berr"] = max(float(i["berr"]) for i in infos)
    rec["iters"] = sorted({int(i["iters"]) for i in infos})
    rec["fell_back"] = sorted({int(i["fell_back"]) for i in infos})
    rec["status"] = sorted({int(i["status"]) for i in infos})
    return rec


def config_small(local, reps=4):
    """Plain method, single system: n = 1003 (not a multiple of 4), d = 2,
    A and b i.i.d. N(0,1), FP64 and the sliced double-float paths (eight and
    seven digits)."""
    import torch

    from paper_2312_09376_gb300 import _lib, inputs
    n = 1003
    Ad, Bd = _lib.to_device(inputs.gaussian(n)), _lib.to_device(inputs.rhs(n, 1))
    out = {"n": n, "d": 2, "matrix": "N(0,1)"}
    for prec in ("f64", "df64tc", "df64tc7"):
        opts = _lib.make_opts(depth=2, seed=1, prec=prec, refine_max=30, tol=1e-13, fallback=True)
        X = _lib.colmajor(n, 1)
        work = torch.empty(_lib.rbt_solve_workspace(opts, n, 1), dtype=torch.uint8, device="cuda")
        rec, outs = timed(lambda: _lib.rbt_solve(opts, n, Ad, Bd, X, work)[1], reps, 3, local, min_ms=500.0)
        out[prec] = _solve_record(rec, outs, n)
    return out


def config_large_zero_corner(local, reps=4, fp64_reps=4):
    """Plain method, large system: n = 20001, d = 3, A i.i.d. N(0,1) with
    A[0,0] = 0 (plain GENP stops at its first pivot), one right-hand side;
    the generalized RBT in FP64 and on the sliced double-float path, and
    Parker's formulation (the identity-padded matrix of order 20008, the next
    multiple of 2^d, where the generalized transform is Parker's) on the
    sliced path."""
    import torch

    from paper_2312_09376_gb300 import _lib
    n, d = 20001, 3
    m = 8 * ((n + 7) // 8)
    g = torch.Generator(device="cuda").manual_seed(7)
    Ap = torch.zeros((m, m), dtype=torch.float64, device="cuda").T      # column-major, lda = m
    Ap[:n, :n].T.copy_(torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64))
    Ap[0, 0] = 0.0
    idx = torch.arange(n, m, device="cuda")
    Ap[idx, idx] = 1.0                                                 # [[A, 0], [0, I]]
    bp = torch.zeros(m, dtype=torch.float64, device="cuda")
    bp[:n] = torch.randn(n, generator=g, device="cuda", dtype=torch.float64)
    A, b = Ap[:n, :n], bp[:n].clone()
    out = {"n": n, "d": d, "matrix": "N(0,1), A[0,0] = 0", "parker_order": m}
    for tag, prec, nn, AA, bb, r, w in (("f64", "f64", n, A, b, fp64_reps, 1), ("df64tc", "df64tc", n, A, b, reps, 2),
                                        ("parker_df64tc", "df64tc", m, Ap, bp, reps, 2),
                                        ("df64tc7", "df64tc7", n, A, b, reps, 2)):
        opts = _lib.make_opts(depth=d, seed=1, prec=prec, refine_max=30, tol=1e-13, fallback=True)
        X = torch.empty(nn, dtype=torch.float64, device="cuda")
        work = torch.empty(_lib.rbt_solve_workspace(opts, nn, 1), dtype=torch.uint8, device="cuda")
        rec, outs = timed(lambda: _lib.rbt_solve(opts, nn, AA, bb, X, work)[1], r, w, local)
        out[tag] = _solve_record(rec, outs, nn)
        del work
    out["speedup_df64tc_vs_f64"] = out["f64"]["mean_ms"] / out["df64tc"]["mean_ms"]
    out["speedup_df64tc7_vs_f64"] = out["f64"]["mean_ms"] / out["df64tc7"]["mean_ms"]
    out["generalized_vs_parker_time"] = out["parker_df64tc"]["mean_ms"] / out["df64tc"]["mean_ms"]
    return out


def config_batched(local, reps=5, warmup=3):
    """2048 systems, n ~ U[48, 700], 1-8 right-hand sides, d = 2, each with its
    own butterflies: one persistent launch captured in a CUDA graph and
    replayed, autotuned; GFLOP/s counts sum 2 n^3 / 3 per batch."""
    import numpy as np
    import torch

    from paper_2312_09376_gb300 import _lib, inputs
    ns = inputs.batch_sizes(2048, 48, 700, seed=11)
    rs = inputs.batch_nrhs(2048, 1, 8, seed=12)
    g = torch.Generator(device="cuda").manual_seed(3)
    Ad = [torch.randn(int(n), int(n), generator=g, device="cuda", dtype=torch.float64).T for n in ns]
    Bd = [torch.randn(int(r), int(n), generator=g, device="cuda", dtype=torch.float64).T for n, r in zip(ns, rs)]
    flop = float(sum(2.0 * int(n) ** 3 / 3 for n in ns))
    out = {"systems": len(ns), "n_range": [int(ns.min()), int(ns.max())], "rhs_range": [int(rs.min()), int(rs.max())],
           "d": 2, "flops_per_batch": flop}
    for prec in ("f64", "f32"):
        opts = _lib.make_opts(depth=2, seed=1000, prec=prec, refine_max=30, tol=1e-13)
        Xd = [_lib.colmajor(b.shape[0], b.shape[1]) for b in Bd]
        plan = _lib.rbt_solve_batched_plan(opts, Ad, Bd, Xd)
        variant, _ = _lib.rbt_solve_batched_autotune(plan)
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            _lib.rbt_solve_batched_run(plan, stream=s)
        rec, _ = timed(graph.replay, reps, warmup, local)
        info = plan.infos_host()
        rec.update({"gflops": flop / rec["mean_ms"] / 1e6, "variant": variant,
                    "solved": float((info["status"] == 0).mean()),
                    "fell_back": float((info["fell_back"] > 0).mean()),
                    "redone_in_double_float": float((info["fell_back"] == 1).mean()),
                    "redone_in_double": float((info["fell_back"] == 2).mean()),
                    "max_berr": float(np.max(info["berr"]))})
        out["fp32_ir" if prec == "f32" else "fp64"] = rec
        del plan, Xd, graph
    out["speedup_fp32_ir_vs_fp64"] = out["fp64"]["mean_ms"] / out["fp32_ir"]["mean_ms"]
    return out


def config_autograd(local, reps=4, warmup=1):
    """X = solve(A, B), n = 8197, 32 right-hand sides, d = 2, loss sum(W * X):
    forward (rbt_solve) and backward (adjoint solve + grad_A) on the device."""
    import torch

    from paper_2312_09376_gb300 import autograd as ag
    n, k = 8197, 32
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(n, n, generator=g, device="cuda", dtype=torch.float64).T
    B = torch.randn(k, n, generator=g, device="cuda", dtype=torch.float64).T
    W = torch.randn(n, k, generator=g, device="cuda", dtype=torch.float64)
    out = {"n": n, "nrhs": k, "d": 2}
    for prec in ("f64", "df64tc", "df64tc7"):
        state = {}

        def fwd():
            Ar = A.detach().clone().requires_grad_(True)
            Br = B.detach().clone().requires_grad_(True)
            X = ag.solve(Ar, Br, depth=2, seed=1, prec=prec)
            state["loss"] = (W * X).sum()
            state["grads"] = (Ar, Br)

        def bwd():
            state["loss"].backward()

        f_ms, b_ms, clk = [], [], []
        for it in range(warmup + reps):
            torch.cuda.synchronize()
            rf, _ = timed(fwd, 1, 0, local)
            rb, _ = timed(bwd, 1, 0, local)
            if it >= warmup:
                f_ms.append(rf["mean_ms"])
                b_ms.append(rb["mean_ms"])
                clk += [c for c in (rf["clocks"], rb["clocks"]) if c]
        tot = [a + b for a, b in zip(f_ms, b_ms)]
        out[prec] = {"forward_ms": statistics.fmean(f_ms), "backward_ms": statistics.fmean(b_ms),
                     "total_ms": statistics.fmean(tot), "ci99_total_ms": ci99(tot), "each_total_ms": tot,
                     "forward_tflops": flops(n) / (statistics.fmean(f_ms) * 1e-3) / 1e12,
                     "clocks": {"sm_mhz": statistics.median([c["sm_mhz"] for c in clk]),
                                "sm_max_mhz": max(c["sm_max_mhz"] for c in clk),
                                "reasons": sorted({r for c in clk for r in c["reasons"]})} if clk else None}
    return out


def cpu_baseline_tier_b(n_max=10000, budget_s=20.0):
    """The tier-b CPU baseline (oracle/rbt_cpu_blocked.c: cache-blocked OpenMP
    FP64, the same method) on every host core, on an n x n sample of the
    precision workload's matrix family: one solve, and more while the total
    stays within budget_s."""
    import oracle
    from paper_2312_09376_gb300 import inputs
    n = n_max
    A, _, _ = inputs.scaled_gaussian(n)
    B = inputs.rhs(n, 1)
    cores = oracle.cpu_set_threads(os.cpu_count() or 1)
    runs = []
    t_start = time.perf_counter()
    while True:
        X, st, b0, berr, it, tf, tt = oracle.cpu_rbt_solve(A, B, 2, 1, refine_max=30, tol=1e-13)
        runs.append((tt, berr, it))
        if time.perf_counter() - t_start + tt > budget_s or len(runs) >= 3:
            break
    t = statistics.fmean(r[0] for r in runs)
    return {"value": flops(n) / t / 1e12, "unit": "TFLOP/s", "cores": cores, "nproc": os.cpu_count(),
            "kind": "oracle", "tier": "b: cache-blocked OpenMP FP64 (oracle/rbt_cpu_blocked.c), same method",
            "sample": "full RBT+GENP solve with FP64 refinement at n=%d (D_r G D_c family, d=2, one RHS), "
                      "%d run(s), %.1f s each" % (n, len(runs), t),
            "berr": max(r[1] for r in runs), "iters": [r[2] for r in runs]}


def run_batched(args):
    import torch

    from paper_2312_09376_gb300 import _lib
    torch.cuda.set_device(0)
    _lib.load()
    r = config_batched(0, reps=max(1, args.steps), warmup=max(1, args.warmup))
    for prec in ("fp64", "fp32_ir"):
        rec = r[prec]
        print(json.dumps({"workload": "batched", "metric": "batched RBT solve GFLOP/s (sum 2n^3/3)",
                          "value": rec["gflops"], "unit": "GFLOP/s", "ms_per_batch": rec["mean_ms"], "prec": prec,
                          **{k: v for k, v in rec.items() if k not in ("gflops",)}}), flush=True)
    return 0


def run_autograd(args):
    import torch

    from paper_2312_09376_gb300 import _lib
    torch.cuda.set_device(0)
    _lib.load()
    r = config_autograd(0, reps=max(1, args.steps), warmup=max(1, args.warmup))
    for prec in ("f64", "df64tc", "df64tc7"):
        rec = r[prec]
        print(json.dumps({"workload": "autograd", "metric": "solve forward + backward ms, n=8197, 32 RHS",
                          "value": rec["total_ms"], "unit": "ms", "higher_is_better": False, "prec": prec, **rec}),
              flush=True)
    return 0


def run_sweep(args):
    """Structure-sensitivity sweep (the size study of Sec. 6.2) with N(0,1)
    matrices standing in for the paper's gallery matrices: every multiple of
    sweep-step in [sweep-lo, sweep-hi], d = 2, the tiled reference size with
    n_b = sweep-tile, no refinement; the first backward error per size, the
    sizes with Parker's structure (multiples of 4 n_b) against the rest."""
    import time

    import torch

    from paper_2312_09376_gb300 import _lib, solve, sweep
    torch.cuda.set_device(0)
    _lib.load()
    prec = "df64tc" if args.prec == "auto" else args.prec
    d, tile = args.depth, args.sweep_tile
    ns = sweep.sizes(args.sweep_lo, args.sweep_hi, args.sweep_step)
    results, codes, paired = [], {}, []
    g = torch.Generator(device="cuda")
    t0 = time.perf_counter()
    for n in ns:
        g.manual_seed(n)
        A = torch.randn(n, n, generator=g, device="cuda", dtype=torch.float64).T
        b = torch.randn(n, 1, generator=g, device="cuda", dtype=torch.float64)
        _, info = solve(A, b, depth=d, seed=1, prec=prec, refine_max=0, fallback=False, align=tile)
        results.append((n, float(info["berr_unrefined"])))
        codes[info["code"]] = codes.get(info["code"], 0) + 1
        if args.sweep_paired and sweep.is_parker(n, d, 1):
            _, pinfo = solve(A, b, depth=d, seed=1, prec=prec, refine_max=0, fallback=False, align=1)
            paired.append((n, results[-1][1], float(pinfo["berr_unrefined"])))
        del A, b
    torch.cuda.synchronize()
    out = sweep.summarize(results, d, tile)
    if paired:
        out["paired"] = sweep.summarize_paired(paired)
    print(json.dumps({"workload": "sweep", "metric": "non-Parker sizes with a first backward error below both "
                      "Parker sizes'", "value": out["below_all_parker"], "unit": "fraction", "prec": prec,
                      "depth": d, "tile": tile, "sizes": len(ns), "lo": ns[0], "hi": ns[-1],
                      "step": args.sweep_step, "status_counts": {str(k): v for k, v in codes.items()},
                      "seconds": time.perf_counter() - t0, "data": "synthetic N(0,1), seed = n", **out}),
          flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "autograd":
        return run_autograd(args)
    if args.workload == "sweep":
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
