"""Benchmark of the truncated-product library on GB300.

One step = one low, one high and one full product of the same two n-bit
operands (uniform random uint64 limbs from a seeded PCG64), n = 2^24 by
default: the single-product configuration at n = 2^24 bits. The headline value
is the truncated-product throughput, operand bits per second over the low and
high products (2 n bits / (t_lo + t_hi)); the full product gives the
t_trunc / t_full ratios. Each product is timed with CUDA events on its stream,
with the L2 flushed (256 MB written) between products. Before timing, the plans
(b, N) and the FFT layouts are tuned (tm_autotune_plan, tm_autotune).

Further keys of the JSON line: the FP64 roofline of the FFT passes against the
FP64 FMA rate measured in the same run (tm_probe_dfma); end to end from
page-locked host memory (e2e); squares / kept operands / data-dependent digit
size; Barrett division; the CPU oracle on the host cores (cpu_baseline); in
"detail": single products at n = 2^16 and 2^20 (sizes), n = 2^28 (large), the
4096-product batch against per-product launches (batched), and a served stream of
4000 requests against per-product launches (served); and last, "summary": every
configuration's headline figures in a few hundred bytes. --served runs the
20000-request served stream alone; --paper-params adds the paper's Table 2
parameters (uncertified).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]
Multi-GPU (torchrun, one rank per GPU): replicas, each rank multiplies its own
operands; value = bits of all ranks / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "truncated-product Gbit/s (lo/hi), t_trunc/t_full on GB300, batched p50/p99 ms"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of all FFT pass launches of one
# product, from one ncu capture (each launch alone, cold caches) of the plans and layouts in
# the keys, built from FFT pass source with this digest (fft_source_digest). roofline.traffic
# reports their sum only while the timed plans, layouts and that source are these;
# otherwise null.
FFT_DRAM_CAPTURE = {
    "fft_source_sha256": "4aa18ddfe1420121ba775214995c707e644f7caa4326c284cf93ec7436388be1",
    "bytes": {("lo", 8, 2097152, "1024:0:0"): 151417600,
              ("hi", 8, 2293760, "1024:0:0"): 165634048,
              ("full", 12, 2949120, "1024:0:0"): 170144256},
}

# Sections of csrc/kernels.cu that the FFT pass kernels compile from (shared constants and
# helpers, the digit extraction of the split on load, the passes themselves), each from
# its header line to the next section's header line.
FFT_SECTIONS = (("// ------------------------------------------------------------ constants",
                 "// -------------------------------------------------------- table kernels"),
                ("// ------------------------------------------------------------ digits",
                 "// ----------------------------------------------------- digit norms"),
                ("// ------------------------------------------------------------ FFT pass",
                 "// ------------------------------------------------ twist + pointwise product"))


def fft_source_digest():
    """SHA-256 of the FFT pass kernels' source: csrc/kernels.cuh and the FFT_SECTIONS
    of csrc/kernels.cu (None if a section header is missing)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1703_00640_gb300", "csrc")
    with open(os.path.join(csrc, "kernels.cu")) as f:
        cu = f.read()
    with open(os.path.join(csrc, "kernels.cuh")) as f:
        h = hashlib.sha256(f.read().encode())
    for start, end in FFT_SECTIONS:
        i = cu.find(start)
        j = cu.find(end, i + 1)
        if i < 0 or j < 0:
            return None
        h.update(cu[i:j].encode())
    return h.hexdigest()


def fft_traffic(plans, layouts, kinds):
    """The captured DRAM bytes of one step's FFT passes, or None when the capture does
    not describe this run (another plan, layout or FFT pass source)."""
    if fft_source_digest() != FFT_DRAM_CAPTURE["fft_source_sha256"]:
        return None
    keys = [(k, plans[k]["b"], plans[k]["N"],
             ":".join(str(layouts[k][x]) for x in ("points", "split", "passes"))) for k in kinds]
    if not all(key in FFT_DRAM_CAPTURE["bytes"] for key in keys):
        return None
    return sum(FFT_DRAM_CAPTURE["bytes"][key] for key in keys)


UNIT = "Gbit/s"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 nominal: 152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz
L2_FLUSH_BYTES = 256 << 20


def workload_config(n, world=1):
    """The config of the headline workload, shared by both arms of the bench."""
    return {"workload": f"single low + high product (full product for the ratio), n = {n} "
                        "bits, uniform random uint64 limbs (seeded PCG64)",
            "n_bits": n, "l2": "flushed (256 MB write) before every product",
            "parallelism": f"replicas x{world}"}


def sig(x, d=4):
    """x rounded to d significant digits (None stays None)."""
    if x is None:
        return None
    if isinstance(x, float):
        return float(f"{x:.{d}g}")
    return x


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--n", "--n-bits", dest="n", type=int, default=1 << 24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--served", action="store_true",
                    help="run the served-stream configuration instead of the default")
    ap.add_argument("--served-count", type=int, default=20000,
                    help="requests of the served stream under --served")
    ap.add_argument("--served-quick-count", type=int, default=4000,
                    help="requests of the served stream inside the default run")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the served stream inside the default run")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="run the batched configuration alone (graph launches)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the square / kept-operand timings")
    ap.add_argument("--no-division", action="store_true",
                    help="skip the division timings")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the planner's plans and the default FFT layouts (no "
                         "tm_autotune_plan / tm_autotune before timing)")
    ap.add_argument("--plan", action="append", default=[], metavar="KIND:B:N",
                    help="fix the plan of a product kind at the bench size with "
                         "tm_plan_set (e.g. hi:8:2359296), instead of tuning it")
    ap.add_argument("--layout", action="append", default=[], metavar="KIND:POINTS:SPLIT:PASSES",
                    help="fix the FFT pass layout of a product kind at the bench size with "
                         "tm_set_layout (as the line's plans report it), instead of tuning it")
    ap.add_argument("--large-bits", type=int, default=1 << 28,
                    help="operand size of the large single-product section")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large single-product section")
    ap.add_argument("--large-only", action="store_true",
                    help="run the large single-product section alone")
    ap.add_argument("--large-kinds", default="lo,hi,full",
                    help="products of the large section (comma list of lo, hi, full)")
    ap.add_argument("--paper-params", action="store_true",
                    help="also time the products with the paper's Table 2 parameters "
                         "(uncertified; not part of the default run)")
    ap.add_argument("--no-sizes", action="store_true",
                    help="skip the single products at n = 2^16 and 2^20")
    return ap.parse_args()


def max_over_ranks(values, dist, device):
    """Element-wise maximum of a list of floats over all ranks (every rank gets it)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_throughput(n, steps, world, t_lo_ms, t_hi_ms):
    """Gbit/s of low + high products over all replicas: each of `world` ranks ran
    `steps` low and high products of n bits; the slowest rank's times count."""
    return 2 * n * steps * world / ((t_lo_ms + t_hi_ms) * 1e-3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


# ------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, which, time.time())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        """Samples taken inside [start, end]; when the region is shorter than the
        sampling interval, the samples within 0.25 s of it."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "start", 0.0), getattr(self, "end", 1e30)
        inside = [l for t, l in self.lines if t0 <= t <= t1]
        if not inside:
            inside = [l for t, l in self.lines if t0 - 0.25 <= t <= t1 + 0.25]
        for line in inside:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ reference arm

def oracle_products(n, seeds, par_depth):
    """Times the oracle's low and high products (its C Karatsuba full product plus
    truncation by definition) on the host; returns seconds per (lo, hi) pair."""
    import workloads
    from oracle import bigmul
    times = []
    for seed in seeds:
        u, v = workloads.pattern_limbs("random", n, seed=seed)
        t0 = time.perf_counter()
        bigmul.mul_lo(u, v, n, par_depth=par_depth)
        bigmul.mul_hi_floor(u, v, n, par_depth=par_depth)
        times.append(time.perf_counter() - t0)
    return times


def threads_for(par_depth):
    return 3 ** par_depth if par_depth > 0 else 1


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    n = args.n
    ncpu = os.cpu_count() or 1
    depth = 0
    while threads_for(depth + 1) <= ncpu and depth < 3:
        depth += 1
    oracle_products(n, range(1000, 1000 + args.warmup), depth)
    t = oracle_products(n, range(2000, 2000 + args.steps), depth)
    total = sum(t)
    value = 2 * n * args.steps / total / 1e9
    threads = min(threads_for(depth), ncpu)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(n, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncpu, "threads": threads,
                         "kind": "oracle",
                         "sample": f"{args.steps} steps of one low + one high product at n={n} "
                                   "(C Karatsuba full product + truncation by definition), "
                                   f"{threads} threads on {ncpu} host cores"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ batched configuration

def run_batched(pkg, torch, np, count, steps, warmup, stream, seed, compare=True):
    """count products, n log-uniform in [2^12, 2^20] bits, half low / half high,
    uniform random operands: one graph launch (tm_batch_launch) per step against
    `count` individual tm_mul launches per step, both timed with CUDA events
    (compare=False: the graph launches alone)."""
    import workloads
    sizes = workloads.log_uniform_sizes(count, 12, 20, seed=seed)
    items = []
    for i, n in enumerate(sizes):
        n = int(n)
        kind = "lo" if i % 2 == 0 else "hi"
        u, v = workloads.pattern_limbs("random", n, seed=10000 * seed + i)
        du = torch.from_numpy(u.view(np.int64)).cuda()
        dv = torch.from_numpy(v.view(np.int64)).cuda()
        out = torch.empty(pkg.out_limbs(kind, n), dtype=torch.int64, device="cuda")
        items.append((kind, n, out, du, dv))
    batch = pkg.Batch(items, stream=stream)
    ref = [torch.empty_like(it[2]) for it in items]
    for _ in range(max(1, warmup)):
        batch.launch(stream)
        if compare:
            for it, r in zip(items, ref):
                pkg.mul(it[0], it[3], it[4], it[1], out=r, stream=stream, report=False)
    torch.cuda.synchronize()
    same = all(torch.equal(it[2], r) for it, r in zip(items, ref)) if compare else None
    g_ms, p_ms = [], []
    for _ in range(steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        batch.launch(stream)
        e1.record(stream)
        if compare:
            for it, r in zip(items, ref):
                pkg.mul(it[0], it[3], it[4], it[1], out=r, stream=stream, report=False)
        e2.record(stream)
        e2.synchronize()
        g_ms.append(e0.elapsed_time(e1))
        p_ms.append(e1.elapsed_time(e2))
    st = batch.status(stream)
    pkg.stream_status(stream)
    batch.close()
    bits = float(sum(int(n) for n in sizes))
    med_g, med_p = float(np.median(g_ms)), float(np.median(p_ms))
    if not compare:
        med_p = float("nan")
    return {
        "products": count, "n_bits": "log-uniform in [2^12, 2^20]", "kinds": "50/50 low/high",
        "graph_launch_ms": {"p50": med_g, "p99": float(np.percentile(g_ms, 99))},
        "per_product_launches_ms": {"p50": med_p, "p99": float(np.percentile(p_ms, 99))},
        "products_per_s": count / (med_g * 1e-3),
        "gbit_s": bits / (med_g * 1e-3) / 1e9,
        "speedup_vs_per_product_launches": med_p / med_g,
        "bit_exact_vs_single": bool(same) if compare else None, "status": st["rc"],
        "margin": st["margin"],
    }


# ------------------------------------------------------------ served configuration

def served_requests(pkg, torch, np, count, seed, k=1 << 24):
    """count requests, n log-uniform in [2^10, 2^k]; 40% high products of x with
    the top n bits of a fixed k-bit Barrett-shaped reciprocal, 30% random low,
    30% random high."""
    import workloads
    _, R = workloads.barrett_reciprocal(k, seed)
    sizes = workloads.log_uniform_sizes(count, 10, 24, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    cls = rng.uniform(size=count)
    reqs = []
    for i, n in enumerate(sizes):
        n = int(n)
        u, v = workloads.pattern_limbs("random", n, seed=seed * 100000 + i)
        if cls[i] < 0.4:
            kind, v = "hi", workloads.top_bits(R, k, n)
        else:
            kind = "lo" if cls[i] < 0.7 else "hi"
        du = torch.from_numpy(u.view(np.int64)).cuda()
        dv = torch.from_numpy(np.ascontiguousarray(v).view(np.int64)).cuda()
        out = torch.empty(pkg.out_limbs(kind, n), dtype=torch.int64, device="cuda")
        reqs.append((kind, n, out, du, dv))
    return reqs


def serve(pkg, reqs, arrivals, budget, slots):
    """Request loop: submits each request at its arrival time (host clock),
    polls progress, and records completion latencies."""
    import time as _t
    srv = pkg.Server(budget, slots)
    order = sorted(range(len(reqs)), key=lambda i: arrivals[i])
    t_of, lat = {}, {}
    j = 0
    t0 = _t.perf_counter()
    while len(lat) < len(reqs):
        now = _t.perf_counter() - t0
        while j < len(order) and arrivals[order[j]] <= now:
            i = order[j]
            kind, n, out, u, v = reqs[i]
            t_of[srv.submit(kind, out, u, v, n)] = i
            j += 1
        for t, st in srv.progress():
            if st != 0:
                raise RuntimeError(f"request {t_of[t]} failed with status {st}")
            lat[t_of[t]] = (_t.perf_counter() - t0) - arrivals[t_of[t]]
    total = _t.perf_counter() - t0
    srv.close()
    return total, [lat[i] for i in range(len(reqs))]


def served_section(pkg, torch, np, count, seed, budget=2 << 30, slots=8):
    """The served stream: `count` requests (served_requests) through the request
    loop, first all at once (saturated capacity), then with Poisson arrivals at 0.5x
    and 0.8x that capacity (latency p50 / p99 from arrival to completion); next to
    it the same requests as plain per-product launches (tm_mul, one stream, all at
    once), and a sample of results against the same products alone."""
    reqs = served_requests(pkg, torch, np, count, seed=seed)
    bits = float(sum(r[1] for r in reqs))
    serve(pkg, reqs, [0.0] * count, budget, slots)           # plans and tables of every size
    total_s, lat_s = serve(pkg, reqs, [0.0] * count, budget, slots)
    rate_sat = count / total_s
    loads = {}
    for frac in (0.5, 0.8):
        arr = np.asarray(__import__("workloads").poisson_arrivals(count, frac * rate_sat, seed=9))
        arr -= arr[0]
        total, lat = serve(pkg, reqs, list(arr), budget, slots)
        loads[f"{frac}x"] = {"rate_per_s": frac * rate_sat, "wall_s": total,
                             "throughput_per_s": count / total,
                             "gbit_s": bits / total / 1e9,
                             "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                            "p99": 1e3 * float(np.percentile(lat, 99))}}
    # baseline: the same request mix as individual tm_mul launches on one stream
    s = torch.cuda.Stream()
    refs = [torch.empty_like(r[2]) for r in reqs]
    for (kind, n, out, u, v), o in zip(reqs, refs):           # warm
        pkg.mul(kind, u, v, n, out=o, stream=s, report=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for (kind, n, out, u, v), o in zip(reqs, refs):
        pkg.mul(kind, u, v, n, out=o, stream=s, report=False)
    torch.cuda.synchronize()
    t_pp = time.perf_counter() - t0
    assert pkg.stream_status(s)["rc"] == 0
    same = all(torch.equal(r[2], o) for r, o in zip(reqs, refs))
    return {"requests": count, "budget_mib": budget >> 20, "slots": slots,
            "saturated": {"wall_s": total_s, "throughput_per_s": rate_sat,
                          "gbit_s": bits / total_s / 1e9,
                          "latency_ms": {"p50": 1e3 * float(np.percentile(lat_s, 50)),
                                         "p99": 1e3 * float(np.percentile(lat_s, 99))}},
            "loads": loads,
            "per_product_launches": {"wall_s": t_pp, "throughput_per_s": count / t_pp,
                                     "gbit_s": bits / t_pp / 1e9},
            "bit_exact_vs_per_product": same}


SERVED_WORKLOAD = ("served stream: {count} requests, Poisson arrivals, n log-uniform in "
                   "[2^10, 2^24] bits, 40% high products with the top n bits of a fixed "
                   "2^24-bit Barrett reciprocal, 30% low, 30% high; device-memory budget "
                   "2048 MiB, 8 slots")


def run_served(args):
    import numpy as np
    import torch
    import paper_1703_00640_gb300 as pkg
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    pkg.build()
    pkg.load()
    res = served_section(pkg, torch, np, args.served_count, seed=5 + rank)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC,
            "config": {"workload": SERVED_WORKLOAD.format(count=args.served_count)},
            "unit": UNIT, "value": res["saturated"]["gbit_s"], "higher_is_better": True,
            "served": res, "n_gpus": world, "dtype": "f64", "data": "synthetic"}), flush=True)


# ------------------------------------------------------------ CUDA arm

def summary_of(n, t_lo, t_hi, t_full, steps, e2e_val, achieved, dfma_peak, sizes, large,
               batched, served):
    """Every configuration's headline figures in a few hundred bytes."""
    out = {f"n={n}": {"lo_gbit_s": sig(n * steps / (t_lo * 1e-3) / 1e9),
                      "hi_gbit_s": sig(n * steps / (t_hi * 1e-3) / 1e9),
                      "t_lo/full": sig(t_lo / t_full), "t_hi/full": sig(t_hi / t_full),
                      "e2e_gbit_s": sig(e2e_val)},
           "fft_tflops": sig(achieved), "dfma_peak_tflops": sig(dfma_peak)}
    for key, row in (sizes or {}).items():
        out[f"n={key}"] = {"lo_us": sig(1e3 * row["lo"]["ms"]), "hi_us": sig(1e3 * row["hi"]["ms"]),
                           "full_us": sig(1e3 * row["full"]["ms"]),
                           "t_lo/full": sig(row["t_lo_over_full"]),
                           "t_hi/full": sig(row["t_hi_over_full"])}
    if large:
        r = {"lo_ms": sig(large["lo"]["ms"]) if "lo" in large else None,
             "hi_ms": sig(large["hi"]["ms"]) if "hi" in large else None,
             "full_ms": sig(large["full"]["ms"]) if "full" in large else None}
        for k in ("lo", "hi"):
            if k in large and "t_over_full" in large[k]:
                r[f"t_{k}/full"] = sig(large[k]["t_over_full"])
        if "lo" in large:
            r["fft_tflops_lo"] = sig(large["lo"]["fft_fp64_tflops"])
        out[f"n={large['n_bits']}"] = r
    if batched:
        out["batch"] = {"products": batched["products"],
                        "graph_ms": sig(batched["graph_launch_ms"]["p50"]),
                        "per_product_launches_ms": sig(batched["per_product_launches_ms"]["p50"]),
                        "products_per_s": sig(batched["products_per_s"]),
                        "gbit_s": sig(batched["gbit_s"])}
    if served:
        out["served"] = {"requests": served["requests"],
                         "saturated_req_per_s": sig(served["saturated"]["throughput_per_s"]),
                         "per_product_launch_req_per_s":
                             sig(served["per_product_launches"]["throughput_per_s"]),
                         "p50_p99_ms_0.5x": [sig(served["loads"]["0.5x"]["latency_ms"]["p50"]),
                                             sig(served["loads"]["0.5x"]["latency_ms"]["p99"])],
                         "p50_p99_ms_0.8x": [sig(served["loads"]["0.8x"]["latency_ms"]["p50"]),
                                             sig(served["loads"]["0.8x"]["latency_ms"]["p99"])]}
    return out


def run_cuda(args):
    import numpy as np
    import torch
    import paper_1703_00640_gb300 as pkg
    import workloads

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    pkg.build()
    pkg.load()
    n = args.n
    nl = (n + 63) // 64
    u_np, v_np = workloads.pattern_limbs("random", n, seed=100 + rank)
    u = torch.from_numpy(u_np.view(np.int64)).cuda()
    v = torch.from_numpy(v_np.view(np.int64)).cuda()
    stream = torch.cuda.current_stream()
    kinds = ["lo", "hi", "full"]
    outs = {k: torch.empty(pkg.out_limbs(k, n), dtype=torch.int64, device="cuda") for k in kinds}
    plans = {k: pkg.plan(k, n) for k in kinds}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # the plan (b, N) among the certified candidates, then the FFT pass layout of
    # its length, picked by measurement (tm_autotune_plan, tm_autotune)
    tuned = None
    fixed = {}
    for spec in args.plan:
        k, b, N = spec.split(":")
        pkg.plan_set(k, n, int(b), int(N))
        fixed[k] = {"b": int(b), "N": int(N)}
    fixed_layouts = {}
    for spec in args.layout:
        k, pts, split, passes = spec.split(":")
        fixed_layouts[k] = {"points": int(pts), "split": int(split), "passes": int(passes)}
    if not args.no_autotune:
        tuned = {"plans": {k: pkg.autotune_plan(k, n, stream=stream)
                           for k in kinds if k not in fixed}}
        tuned["layouts"] = {k: pkg.autotune(k, n, stream=stream)
                            for k in kinds if k not in fixed_layouts}
    for k, lay in fixed_layouts.items():       # after the plans: the layout of their length
        pkg.set_layout(k, n, lay["points"], lay["split"], lay["passes"])
    if fixed:
        tuned = dict(tuned or {}, fixed_plans=fixed)
    plans = {k: pkg.plan(k, n) for k in kinds}
    layouts = {k: (fixed_layouts[k] if k in fixed_layouts else
                   {x: tuned["layouts"][k][x] for x in ("points", "split", "passes")}
                   if tuned and k in tuned.get("layouts", {}) else
                   {"points": 1024, "split": 0, "passes": 0}) for k in kinds}

    # correctness gate on the bench workload (sampled against the oracle's low product)
    _, rep = pkg.mul("lo", u, v, n, out=outs["lo"])
    margin = {"lo": rep["margin"]}
    for k in ("hi", "full"):
        _, rep = pkg.mul(k, u, v, n, out=outs[k])
        margin[k] = rep["margin"]

    def one_step(record):
        """One low, one high and one full product (tm_mul), L2 flushed before each;
        CUDA events on the stream bracket every product."""
        ev = {}
        for k in kinds:
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pkg.mul(k, u, v, n, out=outs[k], stream=stream, report=False)
            b.record(stream)
            ev[k] = (a, b)
        if record is not None:
            record.append(ev)

    def phase_step(record):
        """The same products through tm_mul_events, which records events between the
        phases (they break the programmatic overlap at the phase boundaries, so these
        times explain the breakdown, not the headline)."""
        ev = {}
        for k in kinds:
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(pkg.NPHASES + 1)]
            for x in e:          # torch creates the CUDA event on its first record
                x.record(stream)
            pkg.mul_events(k, u, v, n, e, out=outs[k], stream=stream)
            ev[k] = e
        record.append(ev)

    # the FP64 pipe's peak on this GPU, measured outside the timed region
    # (tm_probe_dfma: independent FMAs on every SM, CUDA events, best of 5)
    probe = []
    for _ in range(6):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fl = pkg.probe_dfma(4096, stream=stream)
        b.record(stream)
        b.synchronize()
        probe.append(fl / (a.elapsed_time(b) * 1e-3) / 1e12)
    dfma_peak = max(probe[1:])

    for _ in range(args.warmup):
        one_step(None)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    recs = []
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)                 # let the sampler start
        clk.mark("start")
        t0 = time.perf_counter()
        for _ in range(args.steps):
            one_step(recs)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk.mark("end")
        time.sleep(0.3)
    st = pkg.stream_status(stream)
    # per-product device times
    per = {k: [ev[k][0].elapsed_time(ev[k][1]) for ev in recs] for k in kinds}
    t_lo, t_hi, t_full = (sum(per[k]) for k in kinds)
    dev_total = t_lo + t_hi + t_full
    if dist:
        t_lo, t_hi, t_full, dev_total = max_over_ranks([t_lo, t_hi, t_full, dev_total], dist,
                                                       "cuda")
    value = replica_throughput(n, args.steps, world, t_lo, t_hi)
    # per-phase device times (outside the timed region)
    phase_recs = []
    nphase_steps = max(5, min(args.steps, 50))
    for _ in range(nphase_steps):
        phase_step(phase_recs)
    torch.cuda.synchronize()
    phase = {k: [[] for _ in range(pkg.NPHASES)] for k in kinds}
    for ev in phase_recs:
        for k in kinds:
            e = ev[k]
            for i in range(pkg.NPHASES):
                phase[k][i].append(e[i].elapsed_time(e[i + 1]))

    # roofline of the dominant kernel (the FFT passes): 3 real transforms of length
    # N per product at the conventional 2.5 N log2 N flops each
    fft_flops, fft_ms, fft_launches = 0.0, 0.0, 0
    for k in kinds:
        N = plans[k]["N"]
        fft_flops += nphase_steps * 3 * 2.5 * N * np.log2(N)
        fft_ms += sum(phase[k][1]) + sum(phase[k][3])
        fft_launches += nphase_steps * 2 * plans[k]["fft_passes"]
    achieved = fft_flops / (fft_ms * 1e-3) / 1e12
    traffic = fft_traffic(plans, layouts, kinds)
    # per two-operand product: 1 forward map (both operands; the full product's first
    # forward pass forms its split itself), fwd_streams x passes forward FFT launches
    # (u and v on two streams, or both in one launch per pass), twist, passes inverse
    # launches, back map, 3 carry kernels
    launches = args.steps * sum((plans[k]["fwd_streams"] + 1) * plans[k]["fft_passes"] +
                                (5 if k == "full" else 6) for k in kinds)

    # end to end through tm_mul_host with page-locked host buffers: every call moves
    # the operands host -> device and the product device -> host (the kernels read and
    # write the mapped host buffers over NVLink-C2C), then waits for the stream
    hu = torch.from_numpy(u_np.view(np.int64)).pin_memory()
    hv = torch.from_numpy(v_np.view(np.int64)).pin_memory()
    hout = {k: torch.empty(pkg.out_limbs(k, n), dtype=torch.int64).pin_memory() for k in kinds}
    e2e_t = []
    e2e_stream = torch.cuda.Stream()
    for it in range(args.warmup + args.steps):
        t1 = time.perf_counter()
        for k in ("lo", "hi"):
            pkg.mul_host(k, hu, hv, n, out=hout[k], stream=e2e_stream)
        if it >= args.warmup:
            e2e_t.append(time.perf_counter() - t1)
    e2e_val = 2 * n * len(e2e_t) * world / sum(e2e_t) / 1e9
    assert np.array_equal(hout["lo"].numpy(), outs["lo"].cpu().numpy())

    # squares (u == v) and kept operand transforms: one forward map and one forward
    # FFT per product instead of two; per-product device time, L2 flushed before each
    def timed(fn, reps):
        ts = []
        for i in range(args.warmup + reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            if i >= args.warmup:
                ts.append((a, b))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ts)

    variants = None
    if not args.no_variants:
        reps = max(5, min(args.steps, 20))
        variants = {"square_ms": {}, "kept_operand_ms": {}, "two_operand_ms": {},
                    "adaptive_ms": {}, "adaptive_b": {}}
        for k in kinds:
            variants["adaptive_ms"][k] = timed(
                lambda: pkg.mul_adaptive(k, u, v, n, out=outs[k], report=False), reps)
            _, arep = pkg.mul_adaptive(k, u, v, n, out=outs[k])
            variants["adaptive_b"][k] = [arep["b"], arep["N"]]
            variants["two_operand_ms"][k] = timed(
                lambda: pkg.mul(k, u, v, n, out=outs[k], report=False), reps)
            variants["square_ms"][k] = timed(
                lambda: pkg.mul(k, u, u, n, out=outs[k], report=False), reps)
            op = pkg.Operand(k, v, n)
            variants["kept_operand_ms"][k] = timed(
                lambda: op.mul(u, out=outs[k], report=False), reps)
            ref, _ = pkg.mul(k, u, v, n)
            got, _ = op.mul(u)
            assert torch.equal(ref, got)
            op.close()
        st2 = pkg.stream_status(stream)
        assert st2["rc"] == 0, st2

    # division by a fixed n-bit divisor (Barrett, kept transforms of R and m) and the
    # Newton reciprocal; per call, L2 flushed before each division
    division = None
    if not args.no_division:
        k = n
        m_np = workloads.random_limbs(k, 500 + rank)
        m_np[(k - 1) // 64] |= np.uint64(1 << ((k - 1) % 64))
        dm = torch.from_numpy(m_np.view(np.int64)).cuda()
        x_np = workloads.random_limbs(2 * k, 600 + rank)
        dx = torch.from_numpy(x_np.view(np.int64)).cuda()
        rts = []
        for i in range(3):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            R = pkg.reciprocal(dm, k)
            rts.append(time.perf_counter() - t1)
        bar = pkg.Barrett(dm, k)
        assert torch.equal(bar.reciprocal(), R)
        dq = torch.empty((k + 64) // 64, dtype=torch.int64, device="cuda")
        dr = torch.empty((k + 63) // 64, dtype=torch.int64, device="cuda")
        reps = max(5, min(args.steps, 20))
        div_ms = timed(lambda: bar.divrem(dx, q=dq, r=dr, report=False), reps)
        _, _, drep = bar.divrem(dx, q=dq, r=dr)
        assert drep["status"] == 0, drep
        bar.close()
        division = {"k_bits": k, "divrem_ms": div_ms, "reciprocal_ms": 1e3 * min(rts),
                    "note": "x of 2k bits by a fixed k-bit m: one high (n = k+1) and one "
                            "low (n = k+3) product against kept transforms plus the limb "
                            "corrections; reciprocal by Newton iteration, host-timed "
                            "(it waits for the stream)"}

    sizes = None
    if not args.no_sizes:
        sizes = run_sizes(pkg, torch, np, workloads, (1 << 16, 1 << 20),
                          max(5, min(args.steps, 50)), args.warmup, stream, flush, seed=16 + rank,
                          tune=not args.no_autotune)

    paper_params = None
    if args.paper_params:
        paper_params = run_paper_params(pkg, torch, np, workloads, max(3, min(args.steps, 7)),
                                        args.warmup, stream, flush, seed=2017 + rank)
        pkg.release()                   # the rows' plan tables (about 50 GB)

    large = None
    if not args.no_large:
        large = run_large(pkg, torch, np, workloads, args.large_bits,
                          max(3, min(args.steps, 10)), args.warmup, stream, flush,
                          seed=28 + rank)

    batched = None
    if not args.no_batched:
        batched = run_batched(pkg, torch, np, args.batch_count, max(3, min(args.steps, 10)),
                              args.warmup, stream, seed=4 + rank)

    served = None
    if not args.no_served:
        served = served_section(pkg, torch, np, args.served_quick_count, seed=5 + rank)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline:
        ts = oracle_products(n, range(3000, 3001), 0)
        cpu = {"value": 2 * n / sum(ts) / 1e9, "unit": UNIT, "cores": os.cpu_count() or 1,
               "threads": 1, "kind": "oracle",
               "sample": f"one low + one high product at n={n} bits (C Karatsuba full "
                         "product + truncation by definition), 1 thread"}
    phases = {k: {pkg.PHASES[i]: round(statistics.median(phase[k][i]), 4)
                  for i in range(pkg.NPHASES)} for k in kinds}
    ms = {k: {"p50": sig(statistics.median(per[k])), "p99": sig(float(np.percentile(per[k], 99)))}
          for k in kinds}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(n, world),
        "roofline": {"bound": "alu", "kernel": "k_fft_pass", "achieved": sig(achieved),
                     "peak": sig(dfma_peak), "unit": "TFLOP/s", "frac": sig(achieved / dfma_peak),
                     "traffic": traffic,
                     "note": "FP64-bound FFT passes: 2.5 N log2 N flops per real transform, 3 "
                             "per product, over their device time (phase events); peak = FP64 "
                             "FMA rate measured in this run (tm_probe_dfma); nominal FP64 1.25; "
                             "traffic = DRAM bytes of one step's FFT passes (one low, high and "
                             "full product) from an ncu capture of these plans and layouts "
                             "(cold caches), null when they differ"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": UNIT,
                "h2d_bytes_per_step": 2 * 2 * nl * 8,
                "d2h_bytes_per_step": (pkg.out_limbs("lo", n) + pkg.out_limbs("hi", n)) * 8},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s_timed": wall,
        "ms": ms, "phases_ms_median": phases,
        "plans": {k: {x: plans[k][x] for x in ("b", "N", "lam_fwd", "lam_bwd", "fft_passes")}
                  | {"e_max": sig(plans[k]["e_max"]), "margin": sig(margin[k]),
                     "layout": ":".join(str(layouts[k][x]) for x in ("points", "split", "passes"))}
                  for k in kinds},
        "status_after_timed_region": st["rc"],
        "square_and_kept_operand": variants, "division": division,
        "paper_parameters": paper_params,
    }
    line["summary"] = summary_of(n, t_lo, t_hi, t_full, args.steps, e2e_val, achieved, dfma_peak,
                                 sizes, large, batched, served)
    line["detail"] = {"sizes": sizes, "large": large, "batched": batched, "served": served}
    # the compact summary last: the end of the line carries every configuration
    line["summary"] = line.pop("summary")
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _as_int(t) -> int:
    """A device or host tensor of little-endian uint64 limbs (stored as int64) as an int."""
    return int.from_bytes(t.cpu().numpy().tobytes(), "little")


def run_large(pkg, torch, np, workloads, n, reps, warmup, stream, flush, seed,
              kinds=("lo", "hi", "full")):
    """Single low, high and full products at a large n (2^28 bits by default: 32 MiB
    operands, transforms of 2-3 x 10^7 complex points, far above L2, so the FFT
    passes stream through HBM). Per kind: device time (CUDA events, L2 flushed),
    Gbit/s, the FFT phases' algorithmic HBM bytes (passes x read + write x 16 B per
    complex point, three transforms) over their time, their FP64 rate in the
    conventional 5 M log2 M count, the largest rounding distance (margin) against
    the bound e_max, and the data-dependent digit size's time. The low product is
    checked against the full product's low n bits and the high product against the
    two admissible values floor(uv / 2^n) and floor(uv / 2^n) + 1."""
    u_np, v_np = workloads.pattern_limbs("random", n, seed=seed)
    u = torch.from_numpy(u_np.view(np.int64)).cuda()
    v = torch.from_numpy(v_np.view(np.int64)).cuda()
    kinds = list(kinds)
    outs = {k: torch.empty(pkg.out_limbs(k, n), dtype=torch.int64, device="cuda") for k in kinds}
    reps_margin = {}
    for k in kinds:
        _, rep = pkg.mul(k, u, v, n, out=outs[k], stream=stream)
        assert rep["status"] == 0, rep
        reps_margin[k] = rep
    checks = {}
    if "full" in kinds:
        full = _as_int(outs["full"])
        if "lo" in kinds:      # a mask, not %: Python's division is quadratic in the size
            checks["lo_equals_full_low_bits"] = _as_int(outs["lo"]) == full & ((1 << n) - 1)
        if "hi" in kinds:
            w = _as_int(outs["hi"])
            checks["hi_admissible"] = w in (full >> n, (full >> n) + 1)

    def timed(fn):
        ev = []
        for i in range(warmup + reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            if i >= warmup:
                ev.append((a, b))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)

    res = {}
    for k in kinds:
        ms = timed(lambda: pkg.mul(k, u, v, n, out=outs[k], stream=stream, report=False))
        ph = [[] for _ in range(pkg.NPHASES)]
        for _ in range(reps):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(pkg.NPHASES + 1)]
            for x in e:
                x.record(stream)
            pkg.mul_events(k, u, v, n, e, out=outs[k], stream=stream)
            torch.cuda.synchronize()
            for i in range(pkg.NPHASES):
                ph[i].append(e[i].elapsed_time(e[i + 1]))
        phases = {pkg.PHASES[i]: round(statistics.median(ph[i]), 4) for i in range(pkg.NPHASES)}
        rep = reps_margin[k]
        M = rep["N"] // 2
        fft_ms = phases["fwd_fft"] + phases["inv_fft"]
        fft_bytes = 3 * rep["fft_passes"] * 2 * 16 * M
        ams = timed(lambda: pkg.mul_adaptive(k, u, v, n, out=outs[k], stream=stream,
                                             report=False))
        _, arep = pkg.mul_adaptive(k, u, v, n, out=outs[k], stream=stream)
        assert arep["status"] == 0, arep
        res[k] = {"ms": ms, "gbit_s": n / (ms * 1e-3) / 1e9,
                  "plan": {x: rep[x] for x in ("b", "N", "lam_fwd", "lam_bwd", "fft_passes")},
                  "margin": rep["margin"], "e_max": rep["e_max"],
                  "phases_ms": phases,
                  "fft_hbm_gb_s": fft_bytes / (fft_ms * 1e-3) / 1e9,
                  "fft_fp64_tflops": 3 * 5.0 * M * np.log2(M) / (fft_ms * 1e-3) / 1e12,
                  "adaptive": {"ms": ams, "b": arep["b"], "N": arep["N"],
                               "margin": arep["margin"], "e_max": arep["e_max"]}}
    for k in ("lo", "hi"):
        if k in kinds and "full" in kinds:
            res[k]["t_over_full"] = res[k]["ms"] / res["full"]["ms"]
            res[k]["adaptive"]["t_over_full"] = (res[k]["adaptive"]["ms"] /
                                                 res["full"]["adaptive"]["ms"])
    return {"n_bits": n, "operands": "uniform random uint64 limbs (seeded PCG64)",
            "l2": "flushed (256 MB write) before every product", "reps": reps,
            **checks, **res}


def run_sizes(pkg, torch, np, workloads, sizes, reps, warmup, stream, flush, seed,
              tune=True):
    """Single products at the smaller configuration sizes (n = 2^16 and 2^20): per kind
    the device time (CUDA events, L2 flushed, median), Gbit/s, the t_lo / t_full and
    t_hi / t_full ratios, the plan (tuned with tm_autotune_plan unless tune is off),
    and the margin on uniformly random operands and on all-ones operands (the largest
    coefficients the digit size admits)."""
    out = {}
    for n in sizes:
        if tune:
            for k in ("lo", "hi", "full"):
                pkg.autotune_plan(k, n, stream=stream)
        u_np, v_np = workloads.pattern_limbs("random", n, seed=seed)
        one_np, _ = workloads.pattern_limbs("ones", n)
        u = torch.from_numpy(u_np.view(np.int64)).cuda()
        v = torch.from_numpy(v_np.view(np.int64)).cuda()
        ones = torch.from_numpy(one_np.view(np.int64)).cuda()
        row = {}
        for k in ("lo", "hi", "full"):
            o = torch.empty(pkg.out_limbs(k, n), dtype=torch.int64, device="cuda")
            _, rep = pkg.mul(k, u, v, n, out=o, stream=stream)
            _, rep1 = pkg.mul(k, ones, ones, n, out=o, stream=stream)
            ev = []
            for i in range(warmup + reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pkg.mul(k, u, v, n, out=o, stream=stream, report=False)
                e1.record(stream)
                if i >= warmup:
                    ev.append((e0, e1))
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(c) for a, c in ev)
            row[k] = {"ms": ms, "gbit_s": n / (ms * 1e-3) / 1e9, "b": rep["b"], "N": rep["N"],
                      "margin_random": rep["margin"], "margin_all_ones": rep1["margin"],
                      "e_max": rep["e_max"], "status": max(rep["status"], rep1["status"],
                                                           key=abs)}
        row["t_lo_over_full"] = row["lo"]["ms"] / row["full"]["ms"]
        row["t_hi_over_full"] = row["hi"]["ms"] / row["full"]["ms"]
        out[str(n)] = row
    return out


def table2_rows():
    """The paper's Table 2 (Section 5): n, N and b of the truncated products, lambda,
    the full product's cyclic length 2N and b (rows with n < 2^31)."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "table2_params.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(x) for x in line.split()))
    return rows


def run_paper_params(pkg, torch, np, workloads, reps, warmup, stream, flush, seed,
                     certified_max_bits=1 << 28):
    """Every Table 2 row (n < 2^31): low and high products with the paper's (N, b) and
    the full product with its (2N, b) through tm_mul_params (b chosen by experiment, not
    certified: the acceptance limit is 3/8), next to the certified plans of tm_mul at
    the same n for n <= certified_max_bits (above, their map tables alone take 50-80
    GB). Per row: device times (CUDA events, L2 flushed, median), the
    ratios t_lo / t_full and t_hi / t_full in both settings, margins and statuses;
    the low product is checked against the full product's low bits and the high
    product against the admissible values."""
    out_rows = []
    for n, N, b, lam, L, bf in table2_rows():
        u_np, v_np = workloads.pattern_limbs("random", n, seed=seed)
        u = torch.from_numpy(u_np.view(np.int64)).cuda()
        v = torch.from_numpy(v_np.view(np.int64)).cuda()
        outs = {k: torch.empty(pkg.out_limbs(k, n), dtype=torch.int64, device="cuda")
                for k in ("lo", "hi", "full")}
        row = {"n_bits": n, "paper": {}, "certified": {}}
        prm = {"lo": (b, N), "hi": (b, N), "full": (bf, L)}
        for k in ("lo", "hi", "full"):
            _, rep = pkg.mul_params(k, u, v, n, b=prm[k][0], N=prm[k][1], out=outs[k],
                                    stream=stream, check=False)
            res = {"b": rep["b"], "N": rep["N"], "lam": rep["lam_fwd"], "status": rep["status"],
                   "margin": rep["margin"], "e_max": rep["e_max"]}
            ev = []
            for i in range(warmup + reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pkg.mul_params(k, u, v, n, b=prm[k][0], N=prm[k][1], out=outs[k],
                               stream=stream, report=False, check=False)
                e1.record(stream)
                if i >= warmup:
                    ev.append((e0, e1))
            torch.cuda.synchronize()
            res["ms"] = statistics.median(a.elapsed_time(c) for a, c in ev)
            row["paper"][k] = res
        full = _as_int(outs["full"])
        row["lo_equals_full_low_bits"] = _as_int(outs["lo"]) == full & ((1 << n) - 1)
        row["hi_admissible"] = _as_int(outs["hi"]) in (full >> n, (full >> n) + 1)
        del full
        for k in (("lo", "hi", "full") if n <= certified_max_bits else ()):
            o = torch.empty_like(outs[k])
            _, rep = pkg.mul(k, u, v, n, out=o, stream=stream)
            ev = []
            for i in range(warmup + reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pkg.mul(k, u, v, n, out=o, stream=stream, report=False)
                e1.record(stream)
                if i >= warmup:
                    ev.append((e0, e1))
            torch.cuda.synchronize()
            row["certified"][k] = {"b": rep["b"], "N": rep["N"], "margin": rep["margin"],
                                   "ms": statistics.median(a.elapsed_time(c) for a, c in ev)}
        if not row["certified"]:
            row["certified"] = None
        for setting in ("paper", "certified"):
            r = row[setting]
            if r is None:
                continue
            r["t_lo_over_full"] = r["lo"]["ms"] / r["full"]["ms"]
            r["t_hi_over_full"] = r["hi"]["ms"] / r["full"]["ms"]
            r["trunc_gbit_s"] = 2 * n / ((r["lo"]["ms"] + r["hi"]["ms"]) * 1e-3) / 1e9
        out_rows.append(row)
    return {"source": "Table 2 of the paper (Section 5)", "acceptance_limit": 0.375,
            "operands": "uniform random uint64 limbs (seeded PCG64)", "reps": reps,
            "rows": out_rows}


def run_large_only(args):
    """The large single-product section alone: one JSON line."""
    import numpy as np
    import torch
    import paper_1703_00640_gb300 as pkg
    import workloads
    pkg.build()
    pkg.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    kinds = [k for k in args.large_kinds.split(",") if k]
    res = run_large(pkg, torch, np, workloads, args.large_bits, max(3, min(args.steps, 10)),
                    args.warmup, stream, flush, seed=28, kinds=kinds)
    trunc = [res[k]["ms"] for k in ("lo", "hi") if k in kinds]
    value = len(trunc) * args.large_bits / (sum(trunc) * 1e-3) / 1e9 if trunc else None
    print(json.dumps({"metric": METRIC, "unit": UNIT, "value": value,
                      "large": res, "n_gpus": 1, "dtype": "f64", "data": "synthetic"}),
          flush=True)


def run_batched_only(args):
    """The batched configuration alone (graph launches, no per-product comparison):
    one JSON line, for profiling the batch."""
    import numpy as np
    import torch
    import paper_1703_00640_gb300 as pkg
    pkg.build()
    pkg.load()
    stream = torch.cuda.current_stream()
    res = run_batched(pkg, torch, np, args.batch_count, args.steps, args.warmup, stream, seed=4,
                      compare=False)
    print(json.dumps({"metric": METRIC, "unit": UNIT, "value": res["gbit_s"],
                      "batched": res, "n_gpus": 1, "dtype": "f64", "data": "synthetic"}),
          flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.served:
        run_served(args)
    elif args.batched_only:
        run_batched_only(args)
    elif args.large_only:
        run_large_only(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
