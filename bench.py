#!/usr/bin/env python3
"""Benchmark of the exhaustive epistasis search on GB300.

One step = one full ``fc_search`` (sweep with prefix tables, AND/POPC
counting, FP32 mutual information and per-warp top lists -> block and grid
merge -> FP64 rescoring of the candidates -> final ordering -> results to
the host) over the order-3 workload: 1,000 SNPs x 4,000 samples
(2,000 cases / 2,000 controls), top 100, synthetic HWE genotypes with a
planted 3-SNP interaction.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead (bounded samples of the same workload on the host cores).
Multi-GPU (torchrun): every rank searches its own data set (independent
problems, weak scaling); only the step times are reduced (max over ranks).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("k-SNP combinations/sec and sample-combinations/sec at order 2/3/4; "
          "% of popc roofline")
UNIT = "combinations/s"
POPC_PER_CLK_PER_SM = 16          # 32-bit POPC issue rate per SM per clock
DEFAULT_SM_MAX_MHZ = 2070.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="C2", choices=["C1", "C2", "C3", "C4", "C5", "P5", "P6", "T4", "T5", "T6"])
    p.add_argument("--c5-datasets", type=int, default=64)
    p.add_argument("--c5-replicates", type=int, default=20)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target duration of the CPU-baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--shard", action="store_true",
                   help="with several ranks: shard one search by rank range (strong scaling) instead of "
                        "one data set per rank (weak scaling)")
    p.add_argument("--snps", type=int, default=None,
                   help="keep only the workload's first N SNPs (smaller cases for profiler captures)")
    p.add_argument("--range", default=None, metavar="S/P",
                   help="search only rank range S of P equal ranges (the share of one of P GPUs); "
                        "default for T4, T5 and T6: 63/64")
    return p.parse_args()


class NvtxRange:
    """An NVTX range around the timed steps, so that a profiler can select
    the launches inside it; a no-op where NVTX is unavailable."""

    def __init__(self, name):
        self.name = name
        self.on = False

    def __enter__(self):
        try:
            import torch
            torch.cuda.nvtx.range_push(self.name)
            self.on = True
        except Exception:
            pass
        return self

    def __exit__(self, *exc):
        if self.on:
            import torch
            torch.cuda.nvtx.range_pop()
        return False


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def init_group(world):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def max_over_ranks(dist, value):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def aggregate(dist, world, units_per_rank, steps, local_total_ms):
    """Whole-job throughput: every rank processed ``units_per_rank`` per step;
    the job's time is the slowest rank's (max over ranks)."""
    total_ms = max_over_ranks(dist, local_total_ms)
    return world * units_per_rank * steps / (total_ms / 1e3), total_ms / steps


def workload_title(name):
    from synth.genotypes import CONFIG_TITLES
    return CONFIG_TITLES[name]


def counted_cells(kind, k):
    """Cells the sweep popcounts per combination, by fc_last_search_kind:
    1 all 3^k (the paper's method), 3 the 2^k with genotypes in {0,1}
    (inclusion-exclusion), 4 the 2 * 3^(k-1) with extension genotype 0/1,
    5 all 3^k from a (k-2)-prefix extended by SNP pairs."""
    if kind == 3:
        return 2 ** k, "IE"
    if kind == 4:
        return 2 * 3 ** (k - 1), "JR"
    if kind == 5:
        return 3 ** k, "PX"
    return 3 ** k, "full"


def executed_popc(ds, k, cells):
    """32-bit POPCs the sweep executes: every counted cell ANDs one 128-bit
    word per class word (padding included) and counts it with three POPCs
    (a carry-save adder folds three of its four 32-bit lanes into two)."""
    words128 = -(-ds.cases // 128) + -(-ds.controls // 128)
    return math.comb(ds.S, k) * cells * words128 * 3


def algorithmic_popc(ds, k):
    """32-bit POPCs per combination of the paper's method (3^k cells x
    32-bit words of both classes), times the number of combinations."""
    words = -(-ds.cases // 32) + -(-ds.controls // 32)
    return math.comb(ds.S, k) * (3 ** k) * words


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # The raw samples go to FC_CLOCKS_DIR (default: the temporary directory);
        # the JSON line carries their summary.
        self.path = os.path.join(os.environ.get("FC_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"fiuncho_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (up to 2 s) for its first
        # sample, so that a short timed region is covered.
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 2.0 and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(kernel_key, source="fc_search.cu"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2201_03331_gb300", "csrc", source)
    try:
        rec = json.load(open(path)).get(kernel_key)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha256") != sha:
        return None
    return rec.get("dram_bytes_per_launch")


def cpu_baseline_sample(ds, k, seconds):
    """Time the oracle on the first P (k-1)-prefixes of the workload, P
    chosen so that the sample takes about ``seconds`` on all host cores."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    # Calibration sample: every thread gets prefixes (fewer when each prefix
    # has many extensions).
    P0 = cores * (16 if k > 2 else 1)
    t0 = time.perf_counter()
    _, _, tested = oracle.search(ds.genotypes, ds.phenotype, k, 10, 0, (0, P0))
    dt = max(time.perf_counter() - t0, 1e-3)
    per_prefix = dt / P0
    npfx = math.comb(ds.S - 1, k - 1)
    P = int(max(8, min(npfx, seconds / per_prefix)))
    t0 = time.perf_counter()
    _, _, tested = oracle.search(ds.genotypes, ds.phenotype, k, 10, 0, (0, P))
    dt = time.perf_counter() - t0
    return {"value": tested / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"(k-1)-prefixes [0, {P}) of {npfx} = {tested} combinations, {dt:.1f} s",
            "seconds": dt}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    from synth import make_config
    oracle.build()
    ds = make_config(args.workload)
    k = ds.k
    cores = os.cpu_count() or 1
    # Size one step at ~ (a few minutes / steps) of CPU time.
    P0 = 16 * cores
    t0 = time.perf_counter()
    oracle.search(ds.genotypes, ds.phenotype, k, ds.top_n, 0, (0, P0))
    per_prefix = max(time.perf_counter() - t0, 1e-3) / P0
    npfx = math.comb(ds.S - 1, k - 1)
    budget = min(8.0, 150.0 / max(1, args.steps + args.warmup))
    P = int(max(8, min(npfx, budget / per_prefix)))
    times, tested = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, _, tested = oracle.search(ds.genotypes, ds.phenotype, k, ds.top_n, 0, (0, P))
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = tested / (ms / 1e3)
    sample = f"(k-1)-prefixes [0, {P}) of {npfx} = {tested} combinations per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_title(args.workload) if not args.snps else
                   f"{args.workload} cut to its first {ds.S} SNPs (profiling case)",
                   "k": k, "snps": ds.S, "samples": ds.M,
                   "top_n": ds.top_n, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    dist = init_group(world)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA path has no CPU fallback)")
    torch.cuda.set_device(local)
    import paper_2201_03331_gb300 as fc
    from paper_2201_03331_gb300 import build as fcbuild
    from synth import make_config, make_dataset
    from synth.genotypes import CONFIGS

    fcbuild.build()
    cfg = dict(CONFIGS[args.workload])
    S = cfg.pop("S")
    if args.snps:
        S = min(S, args.snps)
        cfg["planted"] = tuple(p for p in cfg["planted"] if p < S)
    shard = args.shard and world > 1
    if world > 1 and not shard:
        cfg["seed"] = cfg["seed"] + 1000 * rank      # independent data set per rank
    ds = make_dataset(args.workload, S=S, **cfg) if world > 1 else make_config(args.workload, args.snps)
    k, top_n = ds.k, ds.top_n
    total = math.comb(ds.S, k)
    from paper_2201_03331_gb300.shard import shard_ranges
    part = args.range or {"T4": "63/64", "T5": "63/64", "T6": "63/64"}.get(args.workload)
    if shard:
        # This rank's share of the one search: a contiguous rank range.
        r0, r1 = shard_ranges(total, world)[rank]
    elif part:
        # One range of a search split P ways (what one of P GPUs would run).
        ps, pp = (int(x) for x in part.split("/"))
        r0, r1 = shard_ranges(total, pp)[ps]

    def one_search(handle):
        if shard or part:
            return fc.fc_search_range(handle, k, top_n, r0, r1)
        return fc.fc_search(handle, k, top_n)

    stream = torch.cuda.Stream()
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    fc.fc_set_stream(h, stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # Clock samples from the warm-up (the same searches) through the timed
    # steps, so that a short timed region still gets several.
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(max(3, args.warmup)):
        one_search(h)
    torch.cuda.synchronize()

    fc.fc_timing(h, 1)
    barrier(dist)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with NvtxRange("timed"):
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()                       # L2 flush between timed steps
            ev[i][0].record(stream)
            idx, score = one_search(h)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    sweep_ms, sweeps, launches = fc.fc_timing(h, 0)
    if shard:
        # One search over all ranks: every rank's range ends the step; the
        # merged list (rank 0) is the search's answer.
        from paper_2201_03331_gb300.shard import gather_and_merge
        merged = gather_and_merge(ds.S, k, (idx, score), top_n, dist)
        if rank == 0:
            idx, score = merged
        value, ms_per_step = aggregate(dist, 1, total, args.steps, sum(step_ms))
    elif part:
        value, ms_per_step = aggregate(dist, world, r1 - r0, args.steps, sum(step_ms))
    else:
        value, ms_per_step = aggregate(dist, world, total, args.steps, sum(step_ms))

    # End to end through the public API: pinned host inputs -> fc_load ->
    # fc_search -> host results, every step.
    Gp = torch.from_numpy(ds.genotypes).pin_memory()
    Pp = torch.from_numpy(ds.phenotype).pin_memory()
    Gn, Pn = Gp.numpy(), Pp.numpy()
    e2e_times = []
    for i in range(1 + args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2 = fc.fc_load(Gn, Pn)
        idx2, score2 = one_search(h2)
        fc.fc_free(h2)
        torch.cuda.synchronize()
        if i > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(dist, sum(e2e_times) / len(e2e_times))
    e2e = {"value": world * (r1 - r0 if part and not shard else total) / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(ds.genotypes.nbytes + ds.phenotype.nbytes),
           "d2h_bytes_per_step": int(idx2.nbytes + score2.nbytes + 8 + 4),
           "ms_per_step": 1e3 * e2e_s}

    props = torch.cuda.get_device_properties(local)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", DEFAULT_SM_MAX_MHZ))
    sweep_avg_s = (sweep_ms / max(sweeps, 1)) / 1e3
    kind = fc.fc_last_search_kind(h)
    share = (r1 - r0) / total if (shard or part) and total else 1.0   # this rank's part of the work
    if kind in (2, 6, 7):
        # Tensor-core contraction: contracted cells x M samples x 2 FLOP per
        # combination (orders 2, 3: the 2^k cells with genotypes in {0,1};
        # orders 4-6: all 3^k cells); fp8 peak = measured dense bf16 x 2
        # (nominal ratio).
        cells = {2: 4, 6: 8, 7: 3 ** k}[kind]
        flops = math.comb(ds.S, k) * cells * 2 * (ds.cases + ds.controls) * share
        bf16 = peaks.get("bf16_tflops")
        peak = 2.0 * float(bf16) if bf16 else 2.0 * 1900.0
        achieved = flops / sweep_avg_s / 1e12 if sweeps else None
        tc_name = {2: "k_pairs_tc", 6: "k_triples_tc", 7: f"k_quads_tc<{k}>"}[kind]
        kernel_key = f"{tc_name}<TOPN> {args.workload}"
        roofline = {"bound": "tensor", "kernel": kernel_key, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                    "traffic": traffic_for(kernel_key, {2: "fc_pairs_tc.cu", 6: "fc_triples_tc.cu",
                                                        7: "fc_quads_tc.cu"}[kind]),
                    "peak_basis": ("2 x measured dense bf16 (fp8 e4m3 kind::f8f6f4)" if bf16
                                   else "2 x fallback 1.9 PFLOP/s bf16"),
                    "sweep_ms_per_launch": 1e3 * sweep_avg_s,
                    "algorithmic_flop_per_launch": flops,
                    "paper_method_popc_per_launch": algorithmic_popc(ds, k)}
    else:
        # The sweep is bound by POPC issue (the XU pipe): the POPCs the
        # counting variant executes (executed_popc) against 16 per SM per
        # clock.  The paper's method (3^k cells, one POPC per 32-bit word)
        # is reported beside it as an equivalent rate.
        peak = props.multi_processor_count * POPC_PER_CLK_PER_SM * sm_max * 1e6 / 1e12
        paper_popc = algorithmic_popc(ds, k) * share
        cells, variant = counted_cells(kind, k)
        popc = executed_popc(ds, k, cells) * share
        achieved = popc / sweep_avg_s / 1e12 if sweeps else None
        kernel_key = f"k_search<{k},{variant},TOPN> {args.workload}"
        roofline = {"bound": "alu", "kernel": kernel_key, "achieved": achieved, "peak": peak,
                    "unit": "Tpopc32/s", "frac": (achieved / peak) if achieved else None,
                    "traffic": traffic_for(kernel_key),
                    "peak_basis": f"{props.multi_processor_count} SMs x {POPC_PER_CLK_PER_SM} POPC/clk x {sm_max:.0f} MHz",
                    "sweep_ms_per_launch": 1e3 * sweep_avg_s,
                    "algorithmic_popc_per_launch": popc,
                    "counted_cells_per_combination": cells,
                    "paper_method_popc_per_launch": paper_popc,
                    "paper_method_equivalent_tpopc_s": paper_popc / sweep_avg_s / 1e12 if sweeps else None}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_title(args.workload) if not args.snps else
                   f"{args.workload} cut to its first {ds.S} SNPs (profiling case)",
                   "k": k, "snps": ds.S, "samples": ds.M,
                   "cases": ds.cases, "controls": ds.controls, "top_n": top_n,
                   "l2": "flushed between timed steps (256 MiB write)",
                   "resident": "packed bit table and the data set's tensor-core operands (e4m3 rows and "
                               "inclusion-exclusion tables; orders 4-6: tuple-row slabs), built by fc_load "
                               "and the first search; e2e rebuilds all of them every step",
                   "parallelism": ("one search sharded by rank range over the GPUs" if shard else
                                   "one independent data set per GPU" if world > 1 else "single GPU"),
                   **({"rank_range": f"range {part} of the C(S,k) lexicographic ranks: [{r0}, {r1})",
                       "combinations_per_step": r1 - r0} if part and not shard else {})},
        "sample_combinations_per_s": value * ds.M,
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "top1": [int(x) for x in idx[0]],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(ds, k, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    fc.fc_free(h)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Batched workload: order-3 search of every (data set, replicate) job,
    one graph-captured persistent launch per step, against per-job launches
    (fc_search_job) on the same resident bit tables."""
    import numpy as np
    import torch
    import paper_2201_03331_gb300 as fc
    from paper_2201_03331_gb300 import build as fcbuild
    from synth import make_batch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA path has no CPU fallback)")
    fcbuild.build()
    batch = make_batch(n_datasets=args.c5_datasets, replicates=args.c5_replicates)
    k, top_n = 3, 10
    h = fc.fc_load_batch([ds.genotypes for ds, _ in batch], [ph for _, ph in batch])
    n_jobs = fc.fc_batch_info(h)[2]
    combos = sum(math.comb(ds.S, k) for ds, _ in batch) * args.c5_replicates
    samples = sum(math.comb(ds.S, k) * ds.M for ds, _ in batch) * args.c5_replicates
    stream = torch.cuda.Stream()
    fc.fc_set_stream(h, stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, args.warmup)):
        ref = fc.fc_search_batch(h, k, top_n)
    torch.cuda.synchronize()
    fc.fc_timing(h, 1)
    clocks = ClockSampler(0)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with NvtxRange("timed"):
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[i][0].record(stream)
            out = fc.fc_search_batch(h, k, top_n)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    clk = clocks.stop()
    sweep_ms, sweeps, launches = fc.fc_timing(h, 0)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    identical_replay = bool(np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]))

    # Per-job launches of the same search (one warm-up pass, one timed pass).
    for j in range(n_jobs):
        fc.fc_search_job(h, j, k, top_n)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    same = True
    for j in range(n_jobs):
        idx, s = fc.fc_search_job(h, j, k, top_n)
        same = same and np.array_equal(idx, out[0][j, :len(s)]) and np.array_equal(s, out[1][j, :len(s)])
    e1.record(stream)
    torch.cuda.synchronize()
    per_job_ms = e0.elapsed_time(e1)

    props = torch.cuda.get_device_properties(0)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", DEFAULT_SM_MAX_MHZ))
    # Kernel time per step: the persistent launch plus, for order-3 jobs
    # large enough for the tensor cores, their searches one after another.
    sweep_s = sweep_ms / max(args.steps, 1) / 1e3
    kinds = [fc.fc_batch_job_kind(h, j) for j in range(n_jobs)]
    job_ds = [ds for ds, _ in batch for _ in range(args.c5_replicates)]
    tc_jobs = [j for j in range(n_jobs) if kinds[j] in (6, 8)]
    if tc_jobs:
        # The tensor-core jobs dominate: their contraction (8 cells x M
        # samples x 2 FLOP per combination) over the whole kernel time of the
        # step (which also holds the persistent launch of the small jobs).
        flops = sum(math.comb(job_ds[j].S, k) * 8 * 2 * job_ds[j].M for j in tc_jobs)
        bf16 = peaks.get("bf16_tflops")
        peak = 2.0 * float(bf16) if bf16 else 2.0 * 1900.0
        achieved = flops / sweep_s / 1e12 if sweeps else None
        roof = {"bound": "tensor", "kernel": "k_triples_tc (order-3 jobs >= 384 SNPs) + k_search_batch (the rest)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
                "traffic": None, "kernel_ms_per_step": 1e3 * sweep_s, "tensor_core_jobs": len(tc_jobs),
                "tensor_core_combinations": sum(math.comb(job_ds[j].S, k) for j in tc_jobs),
                "peak_basis": "2 x measured dense bf16 (fp8 e4m3 kind::f8f6f4)"}
    else:
        peak = props.multi_processor_count * POPC_PER_CLK_PER_SM * sm_max * 1e6 / 1e12
        cells, variant = counted_cells(fc.fc_last_search_kind(h), k)
        paper_popc = sum(algorithmic_popc(ds, k) for ds, _ in batch) * args.c5_replicates
        popc = sum(executed_popc(ds, k, cells) for ds, _ in batch) * args.c5_replicates
        achieved = popc / sweep_s / 1e12 if sweeps else None
        roof = {"bound": "alu", "kernel": f"k_search_batch<3,{variant}>", "achieved": achieved,
                "peak": peak, "unit": "Tpopc32/s", "frac": achieved / peak if achieved else None,
                "traffic": None, "kernel_ms_per_step": 1e3 * sweep_s,
                "counted_cells_per_combination": cells, "paper_method_popc_per_launch": paper_popc}
    line = {
        "metric": METRIC, "value": combos / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_title("C5") if args.c5_datasets == 64 and args.c5_replicates == 20 else
                   f"order-3 batched, {args.c5_datasets} data sets x {args.c5_replicates} replicates "
                   "(S ~ U[200,1500], M ~ U[1000,8000], case fraction ~ U[0.3,0.7]), top 10 each",
                   "jobs": n_jobs, "combinations": combos, "l2": "flushed between timed steps (256 MiB write)"},
        "sample_combinations_per_s": samples / (ms / 1e3),
        "roofline": roof,
        "batched_vs_per_job": {"batched_ms": ms, "per_job_ms": per_job_ms, "speedup": per_job_ms / ms,
                               "identical_results": bool(same), "identical_replay": identical_replay},
        "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    fc.fc_free(h)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "C5":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
