#!/usr/bin/env python
"""Benchmark of the concrete-instance race check on GB300.

One step = one full check (expansion, onesweep sort, segmented scan, witness)
of the seeded random affine kernel model: 4096 blocks x 256 threads, 36
statements with loop nests of depth <= 2 and trip counts 1-16, 4 arrays in a
2^30-cell space, 8 barrier intervals, ~1.1e9 access instances (seed 0).  The
model is resident on the device before the timed region; the key buffers
(~9 GB each) are far larger than L2, so no flush is needed between steps.

Printed (rank 0, one JSON line): access instances checked per second (G/s)
over the whole job, the per-kernel HBM roofline of the dominant kernel
(measured live with CUDA events on the check's stream), the end-to-end rate
through the public C-ABI calls from host descriptors, the CPU oracle baseline
on a bounded sample, and the SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun each rank checks its own model (seed + rank): independent
problems, no collective on the data path (weak scaling); the barrier and the
max over ranks of the timed region are the only communication.
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

WORKLOAD = ("seeded random affine kernel model: 4096 blocks x 256 threads, 36 statements, "
            "loop depth <= 2, trips 1-16, 4 arrays in a 2^30-cell space, 8 barrier intervals, "
            "20% floor-div/mod, 30% writes")
METRIC = "access instances checked/sec (G/s)"
UNIT = "G inst/s"
CPU_SAMPLE_BLOCKS = 128       # oracle baseline: same generator and seed, 128 of the 4096 blocks
CPU_SAMPLE_BLOCKS_ALL = 256   # all-cores oracle baseline: 256 of the 4096 blocks
REF_STEP_BLOCKS = 32          # reference arm: per-step sample


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {"onesweep": "sort.cu", "partition": "sort.cu", "partition_a": "bucket.cu",
                  "partition_b": "bucket.cu", "local_sort": "bucket.cu", "histogram_b": "bucket.cu",
                  "scan": "scan.cu", "expand": "jit.cpp", "histogram": "bucket.cu"}


# the part of a source file that holds a kernel and its helpers (first line
# starting with the first marker up to the line starting with the second); a
# kernel without an entry is hashed with its whole file
KERNEL_REGIONS = {"local_sort": ("// Exclusive scan in place of n counters", "// one thread per result: the bucket")}


def kernel_source_hash(kernel="onesweep"):
    """Hash of a kernel's source (its region of its file, else the file): an
    ncu traffic figure is only used while it matches."""
    text = open(os.path.join(ROOT, "paper_2503_08946_gb300", "csrc", KERNEL_SOURCES.get(kernel, "sort.cu")),
                "rb").read()
    if kernel in KERNEL_REGIONS:
        a, b = (m.encode() for m in KERNEL_REGIONS[kernel])
        i = text.index(a)
        text = text[i:text.index(b, i)]
    return hashlib.sha256(text).hexdigest()[:16]


def ncu_traffic_per_key(kernel="onesweep"):
    """DRAM bytes per key of one launch of `kernel` from the committed ncu
    summary (profiles/<kernel>_traffic.json), if it was taken on the current
    kernel source."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_source_hash") != kernel_source_hash(kernel):
        return None
    return float(d["dram_bytes_per_key"])


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons, power = [], [], set(), []
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for name, v in zip(REASONS, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = [p for p in vis.split(",") if p.strip()]
        if local_rank < len(parts) and parts[local_rank].strip().isdigit():
            return int(parts[local_rank])
    return local_rank


# ---------------------------------------------------------------------------
# CPU oracle baseline (test infrastructure, timed as it stands)
# ---------------------------------------------------------------------------
def oracle_rate(seed: int, blocks: int, threads: int = 1):
    """The oracle on a sample of the benchmark model (same generator and seed,
    fewer blocks): one thread, or `threads` workers over cell ranges."""
    import oracle
    import workloads as w
    oracle.build()
    m = w.random_affine(seed, n_blocks=blocks, block=256)
    t0 = time.perf_counter()
    r = oracle.check(m) if threads == 1 else oracle.check_parallel(m, threads)
    dt = time.perf_counter() - t0
    return r.instances, dt, m


def cpu_baselines(seed: int):
    """Single-core and all-core oracle rates on bounded samples (~5-15 s each)."""
    n1, dt1, _ = oracle_rate(seed, CPU_SAMPLE_BLOCKS)
    cores = os.cpu_count() or 1
    nn, dtn, _ = oracle_rate(seed, CPU_SAMPLE_BLOCKS_ALL, cores)
    single = {"value": n1 / dt1 / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"same generator and seed with {CPU_SAMPLE_BLOCKS} of the 4096 blocks "
                        f"({n1} instances, {dt1:.1f} s)"}
    return {"value": nn / dtn / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"same generator and seed with {CPU_SAMPLE_BLOCKS_ALL} of the 4096 blocks ({nn} instances, "
                      f"{dtn:.1f} s): the oracle over {cores} equal cell ranges on std::thread workers "
                      "(each enumerates the whole sample and keeps its own cells)",
            "single_core": single}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    # untimed warm-up steps, then K timed steps, each one oracle check of the sample
    for _ in range(args.warmup):
        oracle_rate(args.seed, REF_STEP_BLOCKS)
    tot_inst, tot_s = 0, 0.0
    for _ in range(args.steps):
        n, dt, _ = oracle_rate(args.seed, REF_STEP_BLOCKS)
        tot_inst += n
        tot_s += dt
    value = tot_inst / tot_s / 1e9
    sample = (f"same generator and seed with {REF_STEP_BLOCKS} of the 4096 blocks "
              f"({tot_inst // max(1, args.steps)} instances per step)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s / max(1, args.steps) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "seed": args.seed, "sample_blocks": REF_STEP_BLOCKS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def run_native(args):
    import torch
    import workloads as w
    import paper_2503_08946_gb300 as rc
    from paper_2503_08946_gb300 import build as b
    from paper_2503_08946_gb300 import distributed as D

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    rc.load()

    seed = args.seed + rank
    model = w.random_affine(seed, n_blocks=args.blocks)
    # the generator's closed form: race-free by construction, or exactly T racy
    # cells when a race is planted (T = threads)
    expect_racy = model.n_model_threads if model.planted else 0
    h = rc.rc_model_create(model)
    lay = rc.rc_model_layout(h)
    opts = {"digit_bits": args.digit_bits, "flags": rc.binding.RC_OPT_STAGE_TIMES}
    ws = rc.workspace(rc.rc_workspace_size(h, opts))
    stream = torch.cuda.current_stream()

    def step(collect):
        t = rc.rc_check(h, opts, ws, stream)
        st = rc.rc_ticket_stage_times(t) if collect else None
        res = rc.rc_report(t)[0]
        if res.status != rc.RC_OK:
            raise RuntimeError(f"check failed: {rc.rc_status_str(res.status)}")
        if res.racy_cells != expect_racy:
            raise RuntimeError(f"check result {res.racy_cells} racy cells, the generator's closed form "
                               f"gives {expect_racy}")
        return res, st

    for _ in range(max(3, args.warmup)):
        res, _ = step(False)
    instances = res.instances

    sampler = ClockSampler(gpu_index(local))
    time.sleep(0.25)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stages = []
    for _ in range(args.steps):
        _, st = step(True)
        stages.append(st)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    # whole job: instances of all ranks over the slowest rank's time
    total_inst, t_max, value = D.weak_scaling_rate(instances * args.steps, elapsed_ms, device="cuda")

    # per-stage means and the roofline of the dominant kernel
    n_keys = stages[0]["n_keys"]
    n_pass = len(stages[0]["sort_ms"])
    mean = lambda xs: sum(xs) / len(xs)
    bucketed = bool(stages[0].get("bucketed"))
    st_mean = {
        "expand_ms": mean([s["expand_ms"] for s in stages]),
        "histogram_ms": mean([s["histogram_ms"] for s in stages]),
        "sort_pass_ms": [mean([s["sort_ms"][k] for s in stages]) for k in range(n_pass)],
        "histogram2_ms": mean([s.get("histogram2_ms", 0.0) for s in stages]),
        "scan_ms": mean([s["scan_ms"] for s in stages]),
        "witness_ms": mean([s["witness_ms"] for s in stages]),
        "check_ms": mean([s["total_ms"] for s in stages]),
    }
    peak, peak_kind = load_peaks()
    # per kernel: (algorithmic bytes per launch, mean launch ms).  Every pass
    # (partition, local sort, radix pass) reads and writes each key once (16 B
    # per key); expansion writes 8 B, histograms and the scan read 8 B.
    if bucketed:
        names = {3: ["partition_a", "partition_b", "local_sort"], 2: ["partition_a", "local_sort"],
                 1: ["local_sort"]}[n_pass]
        kern = {nm: (16.0 * n_keys, st_mean["sort_pass_ms"][i]) for i, nm in enumerate(names)}
        kern["histogram_b"] = (8.0 * n_keys, st_mean["histogram2_ms"])
    else:
        kern = {"onesweep": (16.0 * n_keys, mean(st_mean["sort_pass_ms"][1:] or st_mean["sort_pass_ms"]))}
        if n_pass:
            kern["partition"] = (16.0 * n_keys, st_mean["sort_pass_ms"][0])
    kern["expand"] = (8.0 * n_keys, st_mean["expand_ms"])
    hist_fused = bool(stages[0].get("histogram_fused"))
    if not hist_fused:   # (else the expansion counted it: no pass over the keys)
        kern["histogram"] = (8.0 * n_keys, st_mean["histogram_ms"])
    kern["scan"] = (8.0 * n_keys, st_mean["scan_ms"])
    launches = {"onesweep": max(1, n_pass - 1)} if not bucketed else {}
    dominant = max(kern, key=lambda k: kern[k][1] * launches.get(k, 1))
    alg_bytes, dur_ms = kern[dominant]
    achieved = alg_bytes / (dur_ms / 1e3) / 1e9
    tpk = ncu_traffic_per_key(dominant)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                "alg_bytes_per_launch": alg_bytes, "launch_ms": dur_ms,
                "traffic": (tpk * n_keys) if tpk is not None else None}
    per_kernel = {k: {"ms": v[1], "alg_bytes_per_key": v[0] / n_keys,
                      "frac": v[0] / (v[1] / 1e3) / 1e9 / peak if v[1] > 0 else None} for k, v in kern.items()}
    # the whole check: expansion 8, histograms 8 each (none for a histogram the
    # expansion counts), passes 16 each, scan 8 bytes per key
    pk = 8 + (0 if hist_fused else 8) + 16 * n_pass + 8 + (8 if bucketed and n_pass == 3 else 0)
    pipeline_bytes = pk * n_keys
    pipeline = {"alg_bytes_per_key": pk,
                "gbs": pipeline_bytes / (st_mean["check_ms"] / 1e3) / 1e9,
                "frac": pipeline_bytes / (st_mean["check_ms"] / 1e3) / 1e9 / peak,
                "per_kernel": per_kernel}

    # end to end through the public calls from host descriptors
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 10))
        for _ in range(n_e2e):
            hm = rc.rc_model_create(model)          # host lowering + upload of the program
            t = rc.rc_check(hm, {"digit_bits": args.digit_bits}, ws, stream)
            r = rc.rc_report(t)[0]                  # device-to-host copy of the result record
            if r.status != rc.RC_OK or r.racy_cells != expect_racy:
                raise RuntimeError(f"end-to-end check gave {r}")
            hm.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_val = instances * n_e2e / dt / 1e9
        if dist:
            te = torch.tensor([dt], dtype=torch.float64, device="cuda")
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
            e2e_val = instances * world * n_e2e / float(te.item()) / 1e9
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(lay["program_bytes"]),
               "d2h_bytes_per_step": 256, "steps": n_e2e}

    result = {"racy_cells": res.racy_cells, "verdict": res.verdict, "instances": instances,
              "expected_racy_cells": expect_racy, "checked": "every step against the generator's closed form"}

    # sub-records (not part of the headline): the hash path on the same model,
    # a batch of 10,000 small models against one check per model, a Poisson
    # request stream through the server
    subs = {}
    which = [] if args.no_sub else [x for x in args.sub.split(",") if x]
    if which:
        del ws
        torch.cuda.empty_cache()
    if "hash" in which:
        subs["hash"] = hash_measure(rc, h, model, expect_racy, stream, steps=3)
        torch.cuda.empty_cache()
    if "batch" in which:
        subs["batch"] = batch_measure(args, rc, w, torch, rank, world, dist, steps=5, pm_steps=1, compact=True)
        torch.cuda.empty_cache()
    if "serve" in which:
        subs["serve"] = serve_measure(args, rc, w, torch, rank, world, dist, n_requests=2000, compact=True)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(args.seed)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.blocks == 4096 else WORKLOAD.replace("4096 blocks", f"{args.blocks} blocks"),
                       "seed": args.seed, "instances_per_rank": instances,
                       "keys": n_keys, "sort_bits": lay["sort_hi"] - lay["sort_lo"], "sort_passes": n_pass,
                       "path": "bucket" if bucketed else "lsd sort", "l2": "inputs larger than L2 (key buffers ~9 GB)",
                       "parallelism": f"independent models per rank x{world}"},
            "result": result,
            "roofline": roofline, "pipeline": pipeline, "stages_ms": st_mean,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            # our kernels per check: bucket path 20 with two partition passes (init, expansion,
            # 2 x (histogram, offsets), 2 passes, local sort, tail, scan (3), finish, witness (4);
            # offsets of pass B: 3); LSD path 11 + passes
            "gpu_launches": (({3: 19, 2: 14, 1: 12}[n_pass] - (1 if hist_fused else 0)) if bucketed else (11 + n_pass)) * args.steps,
        }
        line.update(subs)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# a model wider than one key: checked in cell-range chunks
# ---------------------------------------------------------------------------
def run_wide(args):
    import torch
    import workloads as w
    import paper_2503_08946_gb300 as rc
    from paper_2503_08946_gb300 import build as b
    from paper_2503_08946_gb300 import distributed as D

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    rc.load()
    model = w.random_affine(args.seed + rank, n_blocks=args.blocks, row_global=args.wide_row)
    h = rc.rc_model_create(model)
    lay = rc.rc_model_layout(h)
    assert lay["wide"] == 1, "the row length does not make the key wider than 63 bits"
    ws = rc.workspace(rc.rc_workspace_size(h, None))
    stream = torch.cuda.current_stream()

    def step():
        r = rc.rc_report(rc.rc_check(h, None, ws, stream))[0]
        if r.status != rc.RC_OK:
            raise RuntimeError(f"check failed: {rc.rc_status_str(r.status)}")
        return r

    for _ in range(max(3, args.warmup)):
        res = step()
    sampler = ClockSampler(gpu_index(local))
    time.sleep(0.25)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total, t_max, value = D.weak_scaling_rate(res.instances * args.steps, ev0.elapsed_time(ev1), device="cuda")
    if rank == 0:
        line = {
            "metric": METRIC + ", wide keys", "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("4096 blocks", f"{args.blocks} blocks")
                       + f", global rows of {args.wide_row} cells (packed key "
                       f"{lay['cell_shift'] + lay['total_cells'].bit_length()} bits: cell-range chunks)",
                       "seed": args.seed, "instances_per_rank": res.instances, "total_cells": lay["total_cells"],
                       "chunk_cell_bits": lay["cell_bits"], "path": "chunked sort",
                       "l2": "inputs larger than L2", "parallelism": f"independent models per rank x{world}"},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# one model split by cell range, emulated on one GPU
# ---------------------------------------------------------------------------
def run_split(args):
    """k-partition emulation of the one-model split (each rank checks the cells
    of its range): the ranges of k ranks checked one after another on this
    GPU, each timed alone with CUDA events.  The merged partial results must
    equal the whole check; a rank's time is what it would take on its own GPU
    (the k-rank job takes the slowest rank's)."""
    import torch
    import workloads as w
    import paper_2503_08946_gb300 as rc
    from paper_2503_08946_gb300 import build as b
    from paper_2503_08946_gb300 import distributed as D

    b.build()
    rc.load()
    model = w.random_affine(args.seed, n_blocks=args.blocks)
    h = rc.rc_model_create(model)
    total = rc.rc_model_layout(h)["total_cells"]
    stream = torch.cuda.current_stream()
    ws = rc.workspace(rc.rc_workspace_size(h, None))
    whole = rc.rc_report(rc.rc_check(h, {"early_exit": 0}, ws, stream))[0]
    steps = max(1, args.steps)
    out = []
    for by, k in [(by, int(x)) for by in ("range", "hash") for x in args.parts.split(",")]:
        per, parts = [], []
        for rank in range(k):
            o = D.partition_opts(h, rank, k, {"early_exit": 0}, by=by)
            if rc.rc_workspace_size(h, o) > ws.numel():   # (a part's plan needs no more than the whole check's)
                raise RuntimeError("a partial check needs more workspace than the whole check")
            for _ in range(max(3, args.warmup)):
                r = rc.rc_report(rc.rc_check(h, o, ws, stream))[0]
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(steps):
                rc.rc_report(rc.rc_check(h, o, ws, stream))
            ev1.record(stream)
            torch.cuda.synchronize()
            per.append(ev0.elapsed_time(ev1) / steps)
            parts.append(r)
        merged = D.merge_results(parts)
        if (merged.racy_cells, merged.witness) != (whole.racy_cells, whole.witness):
            raise RuntimeError(f"the merged {k}-way split differs from the whole check: {merged} vs {whole}")
        out.append({"by": by, "ranks": k, "rank_ms": [round(x, 3) for x in per], "slowest_rank_ms": round(max(per), 3),
                    "speedup_vs_one": None})
    base = next((o["slowest_rank_ms"] for o in out if o["ranks"] == 1), None)
    for o in out:
        o["speedup_vs_one"] = round(base / o["slowest_rank_ms"], 3) if base else None
    print(json.dumps({"workload": "split", "config": {
        "workload": WORKLOAD.replace("4096 blocks", f"{args.blocks} blocks"), "seed": args.seed,
        "partitions": "range: equal cell ranges of the linear cell space (the read-only array's cells make no keys); "
                      "hash: the check options' hash parts of the cells",
        "emulation": "ranks' ranges checked one after another on one GPU, each timed alone"},
        "racy_cells": whole.racy_cells, "splits": out}), flush=True)
    return 0


# ---------------------------------------------------------------------------
# batched check of many small models vs one check per model
# ---------------------------------------------------------------------------
BATCH_WORKLOAD = ("10,000 seeded random models: threads log-uniform 32..65,536 (multiple of 32, block "
                  "min(T, 256)), 1-8 loop-free access statements, 4 arrays, 8 barrier intervals, 1% planted races")


def batch_closed_form(models, results):
    """Every model's result against the generator's closed form (T racy cells
    when a race is planted, else none); returns the number of racy models."""
    racy = 0
    for m, r in zip(models, results):
        exp = m.n_model_threads if m.planted else 0
        if r.racy_cells != exp:
            raise RuntimeError(f"{m.name}: {r.racy_cells} racy cells, the closed form gives {exp}")
        racy += r.verdict
    return racy


def batch_measure(args, rc, w, torch, rank, world, dist, steps, pm_steps, compact=False):
    """Config 4: 10,000 small models checked as one batch (CUDA graph replay),
    against one check per model on one stream."""
    from paper_2503_08946_gb300 import distributed as D
    models = w.batch_models(args.batch_models, seed0=args.seed * 1000003 + rank * 100003)
    handles = [rc.rc_model_create(m) for m in models]
    opts = {"digit_bits": args.digit_bits, "flags": rc.binding.RC_OPT_GRAPH}   # captured once, replayed
    ws = rc.workspace(rc.rc_batch_workspace_size(handles, opts))
    stream = torch.cuda.current_stream()

    def check_results(res):
        bad = [r for r in res if r.status != rc.RC_OK]
        if bad:
            raise RuntimeError(f"batch check failed: {rc.rc_status_str(bad[0].status)}")
        return res

    def batched():
        return check_results(rc.rc_report(rc.rc_check_batch(handles, opts, ws, stream)))

    def per_model(ws1):
        window, out = [], []
        for h in handles:
            window.append(rc.rc_check(h, opts, ws1, stream))
            if len(window) > 32:
                out.append(rc.rc_report(window.pop(0))[0])
        out += [rc.rc_report(t)[0] for t in window]
        return out

    def timed(fn, n):
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(n):
            r = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = ev0.elapsed_time(ev1)
        if dist:
            t = torch.tensor([ms, wall * 1e3], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms, wall = float(t[0]), float(t[1]) / 1e3
        return r, ms, wall

    for _ in range(max(3, args.warmup)):
        res = batched()
    racy_models = batch_closed_form(models, res)
    inst = sum(r.instances for r in res)
    sampler = ClockSampler(gpu_index(env_rank()[2])) if not compact else None
    if sampler:
        time.sleep(0.25)
    # device throughput: the batches are enqueued back to back (each one graph
    # launch plus its result copy), so the host work of one overlaps the GPU work
    # of the previous; the results are decoded after the timed region
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    tickets = [rc.rc_check_batch(handles, opts, ws, stream) for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    for t in tickets:
        arr = rc.rc_report_array(t)
        if (arr["status"] != rc.RC_OK).any():
            raise RuntimeError("batch check failed: " + rc.rc_status_str(int(arr["status"][arr["status"] != 0][0])))
    wall = time.perf_counter() - t0   # end to end: enqueue, device work, results as one record array
    res = rc.results_of(arr)
    batch_closed_form(models, res)
    clocks = sampler.stop() if sampler else None
    total_i, ms, value = D.weak_scaling_rate(inst * steps, ms, device="cuda")
    total = inst * steps * world

    # one check per model on one stream, same workspace reused (sized for the largest model)
    pm = None
    if not args.no_per_model:
        del ws
        ws1 = rc.workspace(max(rc.rc_workspace_size(h, opts) for h in handles))
        ref = per_model(ws1)
        same = all((a.status, a.instances, a.verdict, a.racy_cells, a.witness) ==
                   (b_.status, b_.instances, b_.verdict, b_.racy_cells, b_.witness) for a, b_ in zip(res, ref))
        _, pm_ms, pm_wall = timed(lambda: per_model(ws1), pm_steps)
        pm_value = inst * pm_steps * world / (pm_ms / 1e3) / 1e9
        pm = {"value": pm_value, "unit": UNIT, "ms_per_step": pm_ms / pm_steps, "steps": pm_steps,
              "results_identical": same}
        # the hash path on the same batch (it checks a batch model by model, full
        # counts without early exit), against the same closed forms
        ho = {"path": rc.RC_PATH_HASH, "early_exit": 0}
        del ws1
        hws = rc.workspace(rc.rc_batch_workspace_size(handles, ho))
        hres = rc.rc_report(rc.rc_check_batch(handles, ho, hws, stream))
        batch_closed_form(models, hres)
        _, h_ms, _ = timed(lambda: check_results(rc.rc_report(rc.rc_check_batch(handles, ho, hws, stream))), 1)
        pm["hash_path"] = {"value": inst * world / (h_ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": h_ms,
                           "results_checked": "every model against the generator's closed form"}
        del hws
    out = {
        "value": value, "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
        "config": {"workload": BATCH_WORKLOAD, "models": len(models), "instances_per_rank": inst,
                   "racy_models": racy_models, "results_checked": "every model against the generator's closed form",
                   "cuda_graph": True, "l2": "key buffers larger than L2",
                   "parallelism": f"independent batches per rank x{world}"},
        "per_model": pm,
        "speedup_vs_per_model": (value / pm["value"]) if pm else None,
        "e2e": {"value": total / wall / 1e9, "unit": UNIT, "h2d_bytes_per_step": 80 * len(models),
                "d2h_bytes_per_step": 136 * len(models)},
    }
    if clocks is not None:
        out["clocks"] = clocks
    for h in handles:
        h.close()
    return out


def run_batch(args):
    import torch
    import workloads as w
    import paper_2503_08946_gb300 as rc
    from paper_2503_08946_gb300 import build as b

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    rc.load()
    m = batch_measure(args, rc, w, torch, rank, world, dist, steps=args.steps, pm_steps=max(1, min(3, args.steps)))
    if rank == 0:
        line = {"metric": METRIC + ", batched", "value": m["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": m["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic"}
        line.update({k: v for k, v in m.items() if k not in line})
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# serving: Poisson arrivals through the continuous-batching request server
# ---------------------------------------------------------------------------
SERVE_WORKLOAD = ("Poisson arrivals at {rate:g} req/s of seeded random models (threads log-uniform 32..65,536, "
                  "1-8 loop-free access statements, 1% planted races), request server with a {mem} GB "
                  "workspace pool and {slots} stream slots")


def serve_measure(args, rc, w, torch, rank, world, dist, n_requests, compact=False):
    """Config 5: a Poisson request stream through the continuous-batching server
    (latency percentiles, sustained rate), then the same requests at once
    (capacity); every result checked against the generator's closed form."""
    import threading
    stream = w.request_stream(n_requests, rate_hz=args.rate, seed=args.seed + rank)
    handles = [rc.rc_model_create(m) for _, m in stream]
    srv = rc.RcServer(memory_bytes=args.pool_gb << 30, slots=args.slots)

    def drain(n, timeout=600.0):
        got, t0 = {}, time.time()
        while len(got) < n:
            for d in srv.poll(cap=4096, wait_ms=20):
                got[d.request] = d
            if time.time() - t0 > timeout:
                raise RuntimeError(f"serving stalled: {len(got)} of {n} finished")
        return got

    # warm-up: the first requests, all at once
    warm = [srv.submit(h) for h in handles[:min(200, len(handles))]]
    drain(len(warm))
    if dist:
        dist.barrier()
    sampler = ClockSampler(gpu_index(env_rank()[2])) if not compact else None
    if sampler:
        time.sleep(0.25)
    ids = [None] * len(handles)

    def submitter():
        t0 = time.perf_counter()
        for i, ((t, _), h) in enumerate(zip(stream, handles)):
            dt = t0 + t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids[i] = srv.submit(h)

    th = threading.Thread(target=submitter)
    th.start()
    got = drain(len(handles))
    th.join()
    clocks = sampler.stop() if sampler else None
    recs = [got[i] for i in ids]
    bad = [r for r in recs if r.result.status != rc.RC_OK]
    if bad:
        raise RuntimeError(f"request failed: {rc.rc_status_str(bad[0].result.status)}")
    batch_closed_form([m for _, m in stream], [r.result for r in recs])
    # capacity: the same requests submitted at once (offered load far above capacity)
    burst_ids = [srv.submit(h) for h in handles]
    burst = drain(len(burst_ids))
    brec = [burst[i] for i in burst_ids]
    b_span = max(r.done_s for r in brec) - min(r.submit_s for r in brec)
    b_inst = sum(r.result.instances for r in brec)
    capacity = {"value": b_inst / b_span / 1e9, "unit": UNIT, "requests_per_s": len(brec) / b_span,
                "batch_size_mean": sum(r.batch_size for r in brec) / len(brec),
                "results_equal_to_poisson_run": all(
                    (a.result.racy_cells, a.result.witness, a.result.instances) ==
                    (b_.result.racy_cells, b_.result.witness, b_.result.instances) for a, b_ in zip(recs, brec))}
    lat = sorted((r.done_s - r.submit_s) * 1e3 for r in recs)
    q = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))]
    t_first = min(r.submit_s for r in recs)
    t_last = max(r.done_s for r in recs)
    inst = sum(r.result.instances for r in recs)
    span = t_last - t_first
    value = inst / span / 1e9
    if dist:
        t = torch.tensor([inst, span], dtype=torch.float64, device="cuda")
        tot = t.clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        value = float(tot[0]) / float(mx[1]) / 1e9
    srv.close()
    for h in handles:
        h.close()
    sizes = [r.batch_size for r in recs]
    out = {
        "value": value, "unit": UNIT, "steps": len(recs), "warmup": len(warm), "ms_per_step": span * 1e3 / len(recs),
        "config": {"workload": SERVE_WORKLOAD.format(rate=args.rate, mem=args.pool_gb, slots=args.slots),
                   "requests": len(recs), "instances": inst,
                   "offered_rate_hz": args.rate, "achieved_rate_hz": len(recs) / span,
                   "results_checked": "every request against the generator's closed form",
                   "l2": "requests are small; pool reused", "parallelism": f"independent streams per rank x{world}"},
        "latency_ms": {"p50": q(0.50), "p90": q(0.90), "p99": q(0.99), "max": lat[-1],
                       "mean": sum(lat) / len(lat)},
        "batch_size": {"mean": sum(sizes) / len(sizes), "max": max(sizes)},
        "capacity": capacity,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 96, "d2h_bytes_per_step": 160},
    }
    if clocks is not None:
        out["clocks"] = clocks
    return out


def run_serve(args):
    import torch
    import workloads as w
    import paper_2503_08946_gb300 as rc
    from paper_2503_08946_gb300 import build as b

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    b.build()
    rc.load()
    m = serve_measure(args, rc, w, torch, rank, world, dist, n_requests=args.requests)
    if rank == 0:
        line = {"metric": METRIC + ", served", "value": m["value"], "unit": UNIT, "n_gpus": world,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                "data": "synthetic"}
        line.update({k: v for k, v in m.items() if k not in line})
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# the hash path (K5) on the benchmark model
# ---------------------------------------------------------------------------
def hash_measure(rc, h, model, expect_racy, stream, steps):
    """The hash path (fused expansion into global group / cell tables) on the
    benchmark model, without early exit (full count); bytes per instance: the
    8-byte key and one 8-byte table word read and written at least once each."""
    import torch
    opts = {"path": rc.RC_PATH_HASH, "early_exit": 0}
    ws = rc.workspace(rc.rc_workspace_size(h, opts))
    r = None
    for _ in range(1):
        r = rc.rc_report(rc.rc_check(h, opts, ws, stream))[0]
    if r.status != rc.RC_OK or r.racy_cells != expect_racy:
        raise RuntimeError(f"hash path gave {r}")
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        r = rc.rc_report(rc.rc_check(h, opts, ws, stream))[0]
        if r.status != rc.RC_OK or r.racy_cells != expect_racy:
            raise RuntimeError(f"hash path gave {r}")
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    del ws
    n = r.instances
    peak, kind = load_peaks()
    return {"value": n / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "racy_cells": r.racy_cells, "early_exit": False,
            "roofline": {"bound": "hbm", "kernel": "hash_expand_kernel", "alg_bytes_per_instance": 16,
                         "achieved": 16.0 * n / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": 16.0 * n / (ms / 1e3) / 1e9 / peak, "peak_source": f"{kind} hbm_gbs"}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--blocks", type=int, default=4096,
                    help="blocks of the model (4096 = the full workload; fewer only for profiling)")
    ap.add_argument("--digit-bits", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sub", default="hash,batch,serve",
                    help="default workload: which sub-records to add (comma-separated of hash, batch, serve)")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload: skip the hash, batch and serve sub-records")
    ap.add_argument("--parts", default="1,2,4,8", help="split: the rank counts to emulate")
    ap.add_argument("--workload", default="affine", choices=["affine", "batch", "serve", "wide", "split"],
                    help="affine: one ~1.1e9-instance model per step (default); batch: 10,000 small models; "
                         "serve: Poisson request stream through the request server")
    ap.add_argument("--batch-models", type=int, default=10000)
    ap.add_argument("--no-per-model", action="store_true", help="batch: skip the one-check-per-model comparison")
    ap.add_argument("--requests", type=int, default=4000)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--pool-gb", type=int, default=8)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--wide-row", type=int, default=1 << 20,
                    help="wide: cells per global-array row (2^20 makes a 66-bit key at 4096 blocks)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "wide":
        return run_wide(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "split":
        return run_split(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
