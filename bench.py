#!/usr/bin/env python3
"""Benchmark: new configurations per second of the breadth-first exploration.

Workload (default "dense1024"): the seeded 1024-neuron random SNP system
(seed 3; 4 rules per neuron, R = 4096, out-degree 64, c U[1,8], i U[c,8],
j U{0,1,2}, p U[1,8], C0 U[0,16]) explored to depth 4 with the frontier capped
at 2^22 configurations and at most 2^26 candidates examined per depth.  The
line's value is the plain int32 (sparse) transition; the metric's comparison,
the exact tensor-core forms on the same GPU (fp8 on tcgen05, int8 on
mma.sync), is timed after it and reported under "compare", each with its ratio
to the int32 value.  --workload random64 gives the 64-neuron system (depth 8,
cap 2^20, budget 2^24); batch4096 and serving the batch engine and the
serving loop.

One step = one complete snp_explore call (all depths, steps (a)-(d) on the
GPU) with the system already resident.  value = new configurations found over
all timed steps (and all ranks) / the max over ranks of the device time of the
timed region (CUDA events on the exploration's stream).  The working set of a
step (68.7 GB of configurations at dense1024, 2.1 GB at random64) exceeds L2,
so no flush is added.  Each form's handle is freed before the next form runs.

e2e: the same metric through the C ABI with host buffers: every step loads the
system from host arrays, explores, and copies every configuration back to
pinned host memory; wall clock around all of it.  One untimed step first sizes
the pinned result buffer (a caller keeps it between explorations).

With --gpus N > 1 (torchrun), every rank explores its own copy of the system
(replicas: one system's BFS is not sharded); the batch workload gives rank r
its own block of 4096 systems (seeds 1000 + 4096 r ...).  The value aggregates
all ranks.
--impl reference times the CPU oracle on bounded samples instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "new configurations/sec per BFS depth (bit-exact), int8-TC batched vs plain int32"
UNIT = "new configurations/s"

WORKLOADS = {
    "paper": dict(depth=10, cap=0, budget=0,
                  desc="the paper's 3-neuron, 5-rule system generating N - {1} (C0 = (2,1,1), M_Pi of Section 2.2, "
                       "rules a^k -> a read as 'at least k spikes'); BFS to depth 10, no cap, no budget "
                       "(50 configurations)",
                  cpu_sample=dict(depth=10, cap=0, budget=0),
                  ref_sample=dict(depth=10, cap=0, budget=0)),
    "random64": dict(seed=1, depth=8, cap=1 << 20, budget=1 << 24,
                     desc="random SNP system seed 1: m=64, 2-3 rules/neuron, a^i(a^j)* with i U[1,4], j U{0,1,2}, "
                          "c U[1,i], p U{1,2} (15% forgetting), out-degree 4, C0 U[0,6]; BFS depth 8, "
                          "frontier cap 2^20, candidate budget 2^24",
                     # the oracle runs the workload's first two depths, exactly
                     cpu_sample=dict(depth=2, cap=1 << 20, budget=1 << 24),
                     ref_sample=dict(depth=2, cap=1 << 16, budget=1 << 20)),
    "dense1024": dict(seed=3, depth=4, cap=1 << 22, budget=1 << 26,
                      desc="random SNP system seed 3: m=1024, 4 rules/neuron (R=4096), out-degree 64, c U[1,8], "
                           "i U[c,8], j U{0,1,2}, p U[1,8], C0 U[0,16]; BFS depth 4, frontier cap 2^22, candidate "
                           "budget 2^26, passes of up to 2^22 spiking vectors (2^21 in the fp8 tensor-core form, 65536 in the "
                           "int8 one)",
                      cpu_sample=dict(depth=1, cap=1 << 12, budget=1 << 14),
                      ref_sample=dict(depth=1, cap=1 << 11, budget=1 << 13)),
    # rate frozen at 0.8 x the measured batched capacity (125.8 requests/s, --calibrate, 2000 requests)
    "serving": dict(requests=100000, seed=4, cap=1 << 12, budget=1 << 16, rate_per_s=100.0,
                    desc="seeded Poisson stream of requests (seed 4); request k: random SNP system seed 10^7+k with "
                         "m U[8,512], 2-3 rules/neuron, out-degree 4, otherwise as random64, BFS depth U[4,32], "
                         "cap 2^12, budget 2^16; continuous batching on one GPU",
                    cpu_sample=dict(systems=2, depth=6, cap=1 << 12, budget=1 << 16),
                    ref_sample=dict(systems=1, depth=4, cap=1 << 12, budget=1 << 16)),
    "batch4096": dict(n=4096, base_seed=1000, depth=6, cap=1 << 12, budget=1 << 16,
                      desc="4096 independent random SNP systems (system s: seed 1000+s; m U[16,256], 1-4 rules/neuron, "
                           "out-degree U[2,8], otherwise as random64), each explored to depth 6 with cap 2^12 and "
                           "budget 2^16; one launch per depth for all systems (batch engine, CUDA graph)",
                      cpu_sample=dict(systems=2, depth=6, cap=1 << 12, budget=1 << 16),
                      ref_sample=dict(systems=1, depth=4, cap=1 << 12, budget=1 << 16)),
}


# timed steps by default: a timed region of at least 2 s
DEFAULT_STEPS = {"dense1024": 120, "random64": 300, "batch4096": 5, "serving": 1, "paper": 2000}


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate_ranks(ms: float, counts, dist=None, device=None):
    """The job's time and totals: the max over ranks of the timed region (ms)
    and the sums over ranks of `counts` (units processed, launches, ...).
    Without a process group (one rank) the inputs come back unchanged."""
    counts = [float(c) for c in counts]
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, counts
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor(counts, device=device, dtype=torch.float64)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(x) for x in c.tolist()]


def batch_seed_base(w, rank: int) -> int:
    """First seed of the systems rank `rank` explores: ranks take consecutive
    blocks of w["n"] independent systems (a shard of an N x n batch; no data
    is exchanged between ranks)."""
    return w["base_seed"] + rank * w["n"]


def make_system(name, rank: int = 0):
    import snp_synth
    w = WORKLOADS[name]
    if name == "batch4096":
        return snp_synth.batch_systems(w["n"], batch_seed_base(w, rank))
    if name == "paper":
        return snp_synth.paper_example()
    return snp_synth.random_64(w["seed"]) if name == "random64" else snp_synth.dense_1024(w["seed"])


class ClockSampler:
    """nvidia-smi samples of clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def strip_comments(src: str) -> str:
    """C++ source without // and /* */ comments, blank lines and trailing
    blanks (string and character literals are kept as they are)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            while i < n and src[i] != "\n":
                i += 1
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = [ln.rstrip() for ln in "".join(out).split("\n")]
    return "\n".join(ln for ln in lines if ln)


def kernel_source_hash() -> str:
    """Hash of the CUDA/C++ sources' code (comments and blank lines do not
    count), so that a profile summary can be matched to the kernels it was
    taken on."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1104_1824_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        with open(os.path.join(d, name), encoding="utf-8") as f:
            h.update(name.encode() + strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, kernel: str = "expand"):
    """DRAM bytes per candidate of a form's dominant kernel from the committed
    ncu summary (profiles/<kernel>_kernel_<workload>.txt), or None when the
    summary is missing or was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_kernel_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return {"bytes_per_candidate": float(vals["dram_bytes_per_candidate"])}
    except (KeyError, ValueError):
        return None


def run_cpu_baseline(system, sample):
    import oracle
    oracle.build()
    systems = system[: sample["systems"]] if isinstance(system, list) else [system]
    new, dt = 0, 0.0
    for x in systems:
        o = oracle.Oracle(x)
        t0 = time.perf_counter()
        e = o.explore(sample["depth"], cap=sample["cap"], budget=sample["budget"])
        dt += time.perf_counter() - t0
        new += sum(d.new for d in e.depths[1:])
    return new, dt


def transition_code(snp, name: str) -> int:
    return {"sparse": snp.SNP_T_SPARSE_I32, "tc": snp.SNP_T_TC_I8, "f8": snp.SNP_T_TC_F8}[name]


TRANSITION_NAMES = {"sparse": "sparse_i32", "tc": "tc_i8", "f8": "tc_f8"}


def time_form(args, system, w, snp, torch, dist, dev, world, local, transition: str, steps: int, warmup: int,
              packed: bool = False):
    """Times `steps` explorations of the workload in one transition form on a
    side stream (CUDA events around the whole timed region, after `warmup`
    untimed ones); the handle, and its store, is freed afterwards.  packed:
    the store keeps counts in 1 or 2 bytes where the bound allows."""
    s = snp.System(system)
    stream = torch.cuda.Stream(device=dev)
    kw = dict(cap=w["cap"], budget=w["budget"], stream=stream, chunk=w.get("chunk", 0),
              transition=transition_code(snp, transition), packed=packed)
    for _ in range(warmup):
        s.explore(w["depth"], **kw)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    r = dict(total_new=0, expand_bytes=0, expand_ms=0.0, launches=0, candidates=0, chunks=0)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(steps):
            s.explore(w["depth"], kernel_timing=True, **kw)
            st = s.depth_stats()
            r["total_new"] += sum(d.new for d in st[1:])
            r["expand_bytes"] += sum(d.expand_bytes for d in st)
            r["expand_ms"] += sum(d.expand_ms for d in st)
            r["launches"] += sum(d.launches for d in st)
            r["candidates"] += sum(d.examined for d in st[1:])
            r["chunks"] += sum(d.chunks for d in st)
        ev1.record(stream)
    torch.cuda.synchronize()
    r["clocks"] = clocks.stop()
    r["ms"] = ev0.elapsed_time(ev1)
    r["per_depth"] = [{"depth": d, "new": x.new, "examined": x.examined, "chunks": x.chunks, "ms": round(x.ms, 4),
                       "new_per_s": round(x.new / (x.ms * 1e-3)) if x.ms > 0 else None}
                      for d, x in enumerate(st) if d > 0]
    r["row_width"] = s.row_width()
    s.close()
    torch.cuda.synchronize()
    return r


def roofline_of(args, system, snp, transition: str, r, packed: bool = False):
    """Roofline object of the form's dominant kernel: its algorithmic bytes
    (per candidate examined and per configuration kept, as snp_depth_info's
    expand_bytes counts them) or, for the int8 form, its dense operations,
    over the kernel's event time."""
    ms = r["ms"]
    nlaunch = max(1, r["chunks"])
    if transition == "tc":
        # the int8 tensor-core pass: dense 2 * R * m int8 operations per candidate
        peak = snp.snp_tc_peak_tops(20000)
        ops = 2.0 * system.R * system.m * r["candidates"]
        achieved = ops / (r["expand_ms"] * 1e-3) / 1e12 if r["expand_ms"] > 0 else None
        traffic = profiled_traffic(args.workload, "tc_rows")
        return {
            "kernel": "k_tc_digits + k_tc_rows (mma.sync m16n8k32 s8) + k_resolve_rows, per pass",
            "bound": "tensor", "achieved": round(achieved, 2) if achieved else None, "peak": round(peak, 1),
            "peak_kind": "measured mma.sync m16n8k32 s8 rate on this GPU (snp_tc_peak_tops)", "unit": "TOPS",
            "frac": round(achieved / peak, 4) if achieved else None,
            "algorithmic_ops_per_launch": int(ops / nlaunch),
            "avg_launch_ms": round(r["expand_ms"] / nlaunch, 4),
            "traffic": (int(traffic["bytes_per_candidate"] * r["candidates"] / nlaunch) if traffic else None),
            "expand_share_of_step": round(r["expand_ms"] / ms, 4) if ms > 0 else None,
        }
    peak, peak_kind = measured_peaks()
    achieved = r["expand_bytes"] / (r["expand_ms"] * 1e-3) / 1e9 if r["expand_ms"] > 0 else None
    if transition == "f8":
        kernel = "k_tc5_expand (tcgen05 kind::f8f6f4, TMEM, TMA row stores) + k_resolve_rows, per pass"
        traffic = profiled_traffic(args.workload, "tc5")
    else:
        kernel = ("k_expand_wide" if system.m > 128 else "k_expand") + " (decode, C' = C + S.M, hash, probe/compare/claim)"
        if packed:
            kernel += f", rows of {r['row_width']} byte(s) per count"
        traffic = profiled_traffic(args.workload, "expand_packed" if packed else "expand")
    return {
        "kernel": kernel, "bound": "hbm", "achieved": round(achieved, 1) if achieved else None, "peak": peak,
        "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s",
        "frac": round(achieved / peak, 4) if achieved else None,
        "algorithmic_bytes_per_launch": int(r["expand_bytes"] / nlaunch),
        "avg_launch_ms": round(r["expand_ms"] / nlaunch, 4),
        "traffic": (int(traffic["bytes_per_candidate"] * r["candidates"] / nlaunch) if traffic else None),
        "expand_share_of_step": round(r["expand_ms"] / ms, 4) if ms > 0 else None,
    }


def bench_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = rank_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1104_1824_gb300 as snp

    w = WORKLOADS[args.workload]
    if args.workload == "serving":
        return bench_serving(args, w, snp, torch, rank)
    system = make_system(args.workload, rank)
    if args.workload == "batch4096":
        return bench_batch(args, w, system, snp, torch, dist, dev, rank, world, local)
    main_form = args.transition or "sparse"
    r = time_form(args, system, w, snp, torch, dist, dev, world, local, main_form, args.steps, args.warmup,
                  packed=args.packed)
    ms_max, (total_all, launches_all) = aggregate_ranks(r["ms"], [r["total_new"], r["launches"]],
                                                        dist if world > 1 else None, dev)
    total_all, launches_all = int(total_all), int(launches_all)
    value = total_all / (ms_max * 1e-3)
    roofline = roofline_of(args, system, snp, main_form, r, packed=args.packed)

    # the metric's comparison: the tensor-core forms against the plain int32 form on the same GPU
    compare = {}
    if args.transition is None and args.workload == "dense1024" and not args.no_compare:
        for form, steps, warm in (("f8", args.steps, args.warmup), ("tc", 1, 1)):
            rf = time_form(args, system, w, snp, torch, dist, dev, world, local, form, steps, warm)
            msf, (tot_f,) = aggregate_ranks(rf["ms"], [rf["total_new"]], dist if world > 1 else None, dev)
            vf = tot_f / (msf * 1e-3)
            compare[TRANSITION_NAMES[form]] = {
                "value": round(vf, 1), "unit": UNIT, "steps": steps, "warmup": warm,
                "ms_per_step": round(msf / steps, 4), "ratio_to_sparse_i32": round(vf / value, 4),
                "dtype": "fp8 e4m3 operands, fp32 accumulation (exact)" if form == "f8" else "int8, int32 accumulation",
                "new_per_step": rf["total_new"] // steps, "per_depth": rf["per_depth"],
                "roofline": roofline_of(args, system, snp, form, rf), "clocks": rf["clocks"],
                "gpu_launches": rf["launches"],
            }
    # packed configurations: the same sparse form with the store's counts in 1 or 2 bytes
    if args.transition is None and not args.packed and not args.no_compare:
        rp = time_form(args, system, w, snp, torch, dist, dev, world, local, "sparse", args.steps, args.warmup,
                       packed=True)
        msp, (tot_p,) = aggregate_ranks(rp["ms"], [rp["total_new"]], dist if world > 1 else None, dev)
        vp = tot_p / (msp * 1e-3)
        compare["sparse_packed"] = {
            "value": round(vp, 1), "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(msp / args.steps, 4), "ratio_to_sparse_i32": round(vp / value, 4),
            "dtype": {1: "uint8", 2: "uint16", 4: "int32"}[rp["row_width"]] + " store, int32 arithmetic",
            "row_bytes": rp["row_width"] * system.m, "new_per_step": rp["total_new"] // args.steps,
            "per_depth": rp["per_depth"], "roofline": roofline_of(args, system, snp, "sparse", rp, packed=True),
            "clocks": rp["clocks"], "gpu_launches": rp["launches"],
        }

    e2e = None
    if not args.no_e2e:
        e2e = bench_e2e(args, system, w, snp, torch, dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cs = w["cpu_sample"]
        new, dt = run_cpu_baseline(system, cs)
        cpu = {"value": round(new / dt, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the workload's first {cs['depth']} depth(s) with cap {cs['cap']} and budget {cs['budget']}: "
                         f"{new} new configurations in {dt:.2f} s, single-threaded C++ oracle",
               "seconds": round(dt, 2)}
    if rank == 0:
        nps = r["total_new"] // args.steps
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"sparse": "int32", "tc": "int8", "f8": "fp8"}[main_form],
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w['desc']}", "depth": w["depth"], "frontier_cap": w["cap"],
                       "candidate_budget": w["budget"], "transition": TRANSITION_NAMES[main_form],
                       "row_bytes": r["row_width"] * system.m,
                       "new_per_step": nps,
                       "l2": f"inputs larger than L2 ({nps * system.m * r['row_width'] / 1e9:.1f} GB of configurations "
                             "written per step)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "per_depth": r["per_depth"],
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_all,
            "clocks": r["clocks"],
        }
        if compare:
            line["compare"] = compare
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def time_batch(args, w, systems, handles, snp, torch, dist, dev, world, local, form: str, steps: int, warmup: int):
    """Times `steps` batch explorations (one launch per depth for all systems)
    in one transition form; returns the timing, plan and per-step counts."""
    import numpy as np
    hs = [h.h for h in handles]
    stream = torch.cuda.Stream(device=dev)
    o = snp.snp_explore_opts_init()
    o.depth, o.frontier_cap, o.candidate_budget = w["depth"], w["cap"], w["budget"]
    o.stream = stream.cuda_stream
    o.transition = transition_code(snp, form)
    t0 = time.perf_counter()
    chunk, tile, warps = snp.snp_batch_autotune(hs, o) if args.autotune else (2048, 0, 8)
    tune_s = time.perf_counter() - t0
    o.chunk, o.tile, o.warps = chunk, tile, warps
    statuses = np.zeros(len(hs), dtype=np.int32)
    for _ in range(warmup):
        snp.snp_explore_batch(hs, o, statuses)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        snp.snp_explore_batch(hs, o, statuses)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    assert (statuses == 0).all(), statuses[statuses != 0][:8]
    new_step, bytes_step, per_depth = 0, 0, {}
    for h, x in zip(handles, systems):
        st = h.depth_stats()
        row = 4 * x.m
        for d, a in enumerate(st):
            if d == 0:
                continue
            new_step += a.new
            dups = a.examined - a.new
            bytes_step += a.examined * 8 + dups * row + a.new * (row + 8) + a.new * 2 * row + a.parents * row
            per_depth.setdefault(d, 0)
            per_depth[d] += a.new
    return dict(ms=ms, clocks=clk, new_step=new_step, bytes_step=bytes_step, per_depth=per_depth,
                plan={"chunk": chunk, "tile": tile, "warps": warps, "autotuned": bool(args.autotune),
                      "autotune_s": round(tune_s, 2)})


def bench_batch(args, w, systems, snp, torch, dist, dev, rank, world, local):
    """Each rank explores its own block of n independent systems (seeds
    batch_seed_base(w, rank) ...): weak scaling, no exchange between ranks.
    Without --transition the fp8 tensor-core batch is timed after the sparse
    one and reported under "compare"."""
    import numpy as np
    handles = [snp.System(x) for x in systems]
    main_form = args.transition or "sparse"
    r = time_batch(args, w, systems, handles, snp, torch, dist, dev, world, local, main_form, args.steps, args.warmup)
    ms, clk, new_step, bytes_step, per_depth = r["ms"], r["clocks"], r["new_step"], r["bytes_step"], r["per_depth"]
    ms_max, (total_all,) = aggregate_ranks(ms, [new_step * args.steps], dist if world > 1 else None, dev)
    total_all = int(total_all)
    value = total_all / (ms_max * 1e-3)
    peak, peak_kind = measured_peaks()
    achieved = bytes_step * args.steps / (ms * 1e-3) / 1e9
    compare = {}
    if args.transition is None and not args.no_compare:
        rf = time_batch(args, w, systems, handles, snp, torch, dist, dev, world, local, "f8", args.steps, args.warmup)
        msf, (tot_f,) = aggregate_ranks(rf["ms"], [rf["new_step"] * args.steps], dist if world > 1 else None, dev)
        vf = tot_f / (msf * 1e-3)
        compare["tc_f8"] = {
            "value": round(vf, 1), "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(msf / args.steps, 3), "ratio_to_sparse_i32": round(vf / value, 4),
            "dtype": "fp8 e4m3 operands, fp32 accumulation (exact)", "plan": rf["plan"],
            "roofline": {"kernel": "k_batch_depth<tensor-core form> (tcgen05 tiles of 128 candidates per system, "
                                   "one launch per depth)", "bound": "hbm",
                         "achieved": round(rf["bytes_step"] * args.steps / (rf["ms"] * 1e-3) / 1e9, 1),
                         "peak": peak, "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s",
                         "frac": round(rf["bytes_step"] * args.steps / (rf["ms"] * 1e-3) / 1e9 / peak, 4),
                         "traffic": None},
            "clocks": rf["clocks"],
        }
    chunk, tile, warps = r["plan"]["chunk"], r["plan"]["tile"], r["plan"]["warps"]
    tune_s = r["plan"]["autotune_s"]
    o = snp.snp_explore_opts_init()
    o.depth, o.frontier_cap, o.candidate_budget = w["depth"], w["cap"], w["budget"]
    o.chunk, o.tile, o.warps = chunk, tile, warps
    o.transition = transition_code(snp, main_form)
    e2e = None
    if not args.no_e2e:
        arrays = [[np.ascontiguousarray(a, dtype=np.int32) for a in (x.rule_neuron, x.rule_i, x.rule_j, x.M, x.c0)]
                  for x in systems]
        h2d = sum(a.nbytes for arr in arrays for a in arr)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh = [snp.snp_load_system(x.m, *arr) for x, arr in zip(systems, arrays)]
        snp.snp_explore_batch(hh, o)
        d2h, got = 0, 0
        for hnd, x in zip(hh, systems):
            n = snp.snp_reachable_count(hnd)
            out = np.empty((n, x.m), dtype=np.int32)
            snp.snp_reachable(hnd, out, n)
            d2h += out.nbytes
            got += n - 1
        for hnd in hh:
            snp.snp_free(hnd)
        dt = time.perf_counter() - t0
        e2e = {"value": round(got / dt, 1), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": 1, "ms_per_step": round(dt * 1e3, 1)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cs = w["cpu_sample"]
        new, dt = run_cpu_baseline(systems, cs)
        cpu = {"value": round(new / dt, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first {cs['systems']} systems of the batch, full settings: {new} new configurations "
                         f"in {dt:.2f} s, single-threaded C++ oracle", "seconds": round(dt, 2)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"sparse": "int32", "tc": "int8", "f8": "fp8"}[main_form],
            "data": "synthetic",
            "config": {"workload": f"batch4096: {w['desc']}", "systems": len(systems), "depth": w["depth"],
                       "frontier_cap": w["cap"], "candidate_budget": w["budget"],
                       "transition": TRANSITION_NAMES[main_form],
                       "plan": {"chunk": chunk, "tile": tile, "warps": warps, "autotuned": bool(args.autotune),
                                "autotune_s": round(tune_s, 2)},
                       "new_per_step": new_step, "per_depth_new": [per_depth[d] for d in sorted(per_depth)],
                       "l2": "inputs larger than L2 (pools of all systems, tens of GB)",
                       "parallelism": f"dp{world}: rank r explores systems of seeds {w['base_seed']} + {w['n']} r ..."
                       if world > 1 else "single GPU"},
            "roofline": {"kernel": "k_batch_depth (one launch per depth, all systems)", "bound": "hbm",
                         "achieved": round(achieved, 1), "peak": peak, "peak_kind": f"{peak_kind} copy bandwidth",
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "algorithmic_bytes_per_launch": int(bytes_step / w["depth"]),
                         "avg_launch_ms": round(ms / args.steps / w["depth"], 3), "traffic": None},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": (w["depth"] + 2) * args.steps, "clocks": clk,
        }
        if compare:
            line["compare"] = compare
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def bench_serving(args, w, snp, torch, rank):
    """The serving loop on the first --requests arrivals of the seeded stream.
    --calibrate submits them all at once and reports the batched capacity
    (requests/s) whose 0.8 fraction is frozen as the stream's rate."""
    import numpy as np
    import snp_synth
    n = args.requests
    rate = w["rate_per_s"] or 100.0
    reqs = snp_synth.serving_requests(n, rate, seed=w["seed"])
    t0 = time.perf_counter()
    systems = [r.system() for r in reqs]
    gen_s = time.perf_counter() - t0
    handles = [snp.System(x) for x in systems]
    o = [snp.snp_explore_opts_init() for _ in reqs]
    for oo, r in zip(o, reqs):
        oo.depth, oo.frontier_cap, oo.candidate_budget = r.depth, w["cap"], w["budget"]
    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.5, 120 << 30))
    srv = snp.snp_server_create(budget, args.max_active)
    statuses, got = [], [0]
    id_to_k = {}
    stop = [False]

    def consume():
        # the client side: takes finished results and releases their handles
        waiting = []
        while not stop[0] or got[0] < n:
            ids, lat, sts = snp.snp_server_poll(srv)
            for i, st in zip(ids.tolist(), sts.tolist()):
                statuses.append(st)
                waiting.append(i)
            got[0] += len(ids)
            still = []
            for i in waiting:
                k = id_to_k.get(i)
                if k is None:
                    still.append(i)
                else:
                    handles[k].close()
            waiting = still
            if len(ids) == 0:
                time.sleep(0.001)

    import threading
    consumer = threading.Thread(target=consume)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_start = time.perf_counter()
    consumer.start()
    for k, r in enumerate(reqs):
        if not args.calibrate:
            delay = r.arrival_s - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
        rid = snp.snp_server_submit(srv, handles[k].h, o[k])
        id_to_k[rid] = k
    snp.snp_server_wait(srv)
    wall = time.perf_counter() - t_start
    clk = clocks.stop()
    stop[0] = True
    consumer.join()
    info = snp.snp_server_stats(srv)
    snp.snp_server_destroy(srv)
    assert all(x == 0 for x in statuses), [x for x in statuses if x][:5]
    value = info.new_configs / (info.span_ms * 1e-3)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": round(info.span_ms, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"serving: {w['desc']}", "requests": n, "of_stream": w["requests"],
                   "subset": f"the first {n} arrivals of the {w['requests']}-request stream (its whole length would "
                             f"take {w['requests'] / rate / 60:.0f} minutes of arrivals at {rate:g}/s)",
                   "rate_per_s": None if args.calibrate else rate, "calibration": bool(args.calibrate),
                   "max_active": args.max_active, "hbm_budget_gb": round(budget / 2 ** 30, 1),
                   "system_generation_s": round(gen_s, 1)},
        "serving": {"completed": info.completed, "new_configs": info.new_configs, "span_ms": round(info.span_ms, 1),
                    "wall_s": round(wall, 2), "p50_ms": round(info.p50_ms, 2), "p99_ms": round(info.p99_ms, 2),
                    "max_ms": round(info.max_ms, 2), "ticks": info.ticks, "busy_ms": round(info.busy_ms, 1),
                    "capacity_req_per_s": round(info.completed / (info.span_ms * 1e-3), 2)},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def bench_e2e(args, system, w, snp, torch, dev):
    """Host arrays in, every configuration back in pinned host memory, per step."""
    import numpy as np
    arrays = [np.ascontiguousarray(x, dtype=np.int32) for x in (system.rule_neuron, system.rule_i, system.rule_j,
                                                                   system.M, system.c0)]
    h2d = sum(a.nbytes for a in arrays)
    host_out = None
    steps = max(1, min(args.steps, 3))

    def one_step():
        # load from host arrays, explore, read every configuration back
        nonlocal host_out
        h = snp.snp_load_system(system.m, *arrays)
        o = snp.snp_explore_opts_init()
        o.depth, o.frontier_cap, o.candidate_budget = w["depth"], w["cap"], w["budget"]
        o.chunk = w.get("chunk", 0)
        o.transition = transition_code(snp, args.transition or "sparse")
        snp.snp_explore(h, o)
        n = snp.snp_reachable_count(h)
        if host_out is None or host_out.shape[0] < n:
            host_out = torch.empty((n, system.m), dtype=torch.int32, pin_memory=True)
        snp.snp_reachable(h, host_out, n)
        snp.snp_free(h)
        return n

    one_step()  # untimed: sizes the pinned result buffer, which a caller would keep
    total_new, d2h = 0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        n = one_step()
        total_new += n - 1
        d2h = n * system.m * 4
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": round(total_new / dt, 1), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": steps, "ms_per_step": round(dt / steps * 1e3, 3)}


def bench_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    system = make_system(args.workload)
    rs = WORKLOADS[args.workload]["ref_sample"]
    for _ in range(args.warmup):
        run_cpu_baseline(system, rs)
    total_new, total_s = 0, 0.0
    for _ in range(args.steps):
        new, dt = run_cpu_baseline(system, rs)
        total_new += new
        total_s += dt
    value = total_new / total_s
    sample = (f"per step the workload's first {rs['depth']} depth(s) with cap {rs['cap']} and budget {rs['budget']} "
              f"({total_new // args.steps} new configurations), single-threaded C++ oracle")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_s / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]['desc']}", "transition": "oracle"},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: dense1024 80, random64 300 (at least 2 s), batch4096 5, paper 2000)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="dense1024")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--depth", type=int, default=0, help="override the workload's depth (profiling cases)")
    ap.add_argument("--cap", type=int, default=0, help="override the workload's frontier cap (profiling cases)")
    ap.add_argument("--chunk", type=int, default=0, help="override the pass size (profiling cases)")
    ap.add_argument("--autotune", action="store_true", help="batch4096: pick pass size, tile and warps first")
    ap.add_argument("--systems", type=int, default=0, help="batch4096: override the number of systems (profiling cases)")
    ap.add_argument("--requests", type=int, default=2000, help="serving: arrivals of the stream to run")
    ap.add_argument("--max-active", type=int, default=2048, help="serving: requests on the device at once")
    ap.add_argument("--calibrate", action="store_true", help="serving: submit all at once, report the capacity")
    ap.add_argument("--transition", choices=["sparse", "tc", "f8"], default=None,
                    help="step (c): sparse int32 gather, the exact int8 tensor-core product (mma.sync), or the "
                         "exact fp8 product on tcgen05 (default: sparse; on dense1024 the two tensor-core forms are "
                         "also timed and reported under 'compare')")
    ap.add_argument("--no-compare", action="store_true", help="time the line's form only")
    ap.add_argument("--packed", action="store_true",
                    help="the line's form with a packed store (counts in 1 or 2 bytes where the bound allows)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = DEFAULT_STEPS.get(args.workload, 5)
    if args.depth > 0:
        WORKLOADS[args.workload] = dict(WORKLOADS[args.workload], depth=args.depth)
    if args.cap > 0:
        WORKLOADS[args.workload] = dict(WORKLOADS[args.workload], cap=args.cap)
    if args.chunk > 0:
        WORKLOADS[args.workload] = dict(WORKLOADS[args.workload], chunk=args.chunk)
    if args.systems > 0 and args.workload == "batch4096":
        WORKLOADS[args.workload] = dict(WORKLOADS[args.workload], n=args.systems)
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
