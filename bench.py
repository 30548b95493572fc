"""Benchmark of the finite-automaton DNA pattern scan on GB300.

Workload (one "step" = the whole hot path over one batch): a 3.2 GB
genome-like synthetic text (GC 0.41, ~50% soft-masked lower case in runs of
mean 300, ~5% N in blocks of mean 50 kb; seed 2) resident in HBM, and five
patterns of lengths 4, 8, 16, 32, 64 (uniform A/C/G/T, seeds 3..7), one
launch per pattern, each producing the exact count and the sorted int64
start positions.  The automata are built once before timing (host setup).

Metric: GB/s of DNA text scanned per pattern (n bytes x patterns / time).
The text (3.2 GB) is far larger than L2 (129 MB), so no flush is needed
between steps.  ``e2e`` repeats the step through the host-buffer entry point
(pinned host text in, host positions out, copies inside the timed region).
``roofline`` reports the find kernel's algorithmic bytes (text + 8 B per
position written) per launch over its CUDA-event duration against the
measured HBM copy bandwidth.  ``cpu_baseline`` times the CPU oracle's
Algorithm 1 scan on the host cores on a bounded sample of the same text.

``workloads`` (N = 1, after the headline, on the same GPU) holds the other
workloads, each with its own roofline: the 16 MiB single-pattern case (m =
8) timed after an L2 flush and as CUDA-graph back-to-back finds; the six
sequences x 256 patterns in one graph launch and the 4096 6-mer census,
each against its one-pattern-per-launch plain form; and serving at the
offered Poisson rate against the plain form.  ``--no-workloads`` skips them.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) each rank scans its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GB/s of DNA text scanned per pattern"
UNIT = "GB/s"
PATTERN_LENGTHS = (4, 8, 16, 32, 64)
PATTERN_SEEDS = (3, 4, 5, 6, 7)
TEXT_BYTES = 3_200_000_000
TEXT_SEED = 2
CLASS_PAIRS, CLASS_SEED = 9, 40          # class-pattern workload: 9 pairs = 18 patterns
WORKLOAD = "genome-scale single-pattern scan"
# one dfa_find per pattern, the two-pass find: pass 1 k_scan_tma (m >= 8:
# the relaxed count kernel, leaving row counts and the stage masks of its
# exact replays; m < 8: the relaxed dense walk recording each row's end
# offsets, then k_tile_offsets scans the tile totals; for m >= 8 the count
# kernel's last CTA does) and pass 3 (k_place copies the recorded offsets;
# k_place_masked walks the masked bytes of the rows with accepts); the
# events time the whole call
DOMINANT_KERNEL = ("dfa_find = k_scan_tma (TMA-staged pass 1) + k_tile_offsets + k_place (m < 8) "
                   "or k_scan_tma (pass 1, tile scan in its last CTA) + k_place_masked (m >= 8)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=TEXT_BYTES)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cfg", default="", help="json launch config (layout/threads/chunk/loader)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: offered queries per second")
    ap.add_argument("--queries", type=int, default=2000, help="serve: queries in the timed trace")
    ap.add_argument("--slots", type=int, default=4, help="serve: CUDA stream slots")
    ap.add_argument("--workload", default="genome", choices=["genome", "batched", "census", "classes", "serve"],
                    help="genome: the single-pattern scan (the headline line); batched: six "
                         "sequences x 256 patterns in one graph launch; census: all 4096 6-mers; "
                         "classes: 18 character-class patterns over the genome text")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="steps of the one-pattern-per-launch comparison (batched/census)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="genome: skip the other workloads (16 MiB single pattern, batched, census, "
                         "serving) reported under 'workloads'")
    ap.add_argument("--serve-queries", type=int, default=600,
                    help="genome: queries of the serving trace reported under 'workloads'")
    ap.add_argument("--shard", action="store_true",
                    help="genome: split ONE text over the ranks (owned starts + m-1 overlap), "
                         "gather counts and positions over the process group (strong scaling); "
                         "the default runs one replica per rank")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def kernels_per_find(m, cfg):
    """Kernels one dfa_find launches on the TMA path: the staged two-pass
    find for the relaxed layouts at any m (count pass, its last CTA scanning
    the tile totals, and placement: two) and for layout 1 up to m = 8 (dense
    pass, tile scan, copy: three; the library's defaults: layout 1 below
    m = 8, layout 4 from there; the workspace bench.py passes always has
    room for it), else the single-pass find kernel."""
    layout = (cfg or {}).get("layout", 0)
    if layout == 0:
        layout = 4 if m >= 8 else 1
    if layout in (3, 4):
        return 2
    return 3 if layout == 1 and m <= 8 else 1


def config_dict(n, world, cfg):
    return {"workload": WORKLOAD, "text_bytes": n, "text": "GC 0.41, 50% soft-masked (runs mean 300),"
            " 5% N (blocks mean 50 kb), seed 2", "patterns": list(PATTERN_LENGTHS),
            "pattern_seeds": list(PATTERN_SEEDS), "outputs": "count + sorted int64 start positions",
            "finds_per_step": len(PATTERN_LENGTHS), "l2": "inputs larger than L2 (no flush)",
            "parallelism": f"replicas x{world}",
            "launch_config": cfg if cfg else "library default"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_smi_id(local):
    """nvidia-smi identifier of the CUDA device `local` (UUID when known)."""
    try:
        import torch
        u = torch.cuda.get_device_properties(local).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        parts = [p for p in vis.split(",") if p.strip()]
        return parts[local] if local < len(parts) else str(local)


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _code_only(src: str) -> str:
    """C/CUDA source without comments and blank lines (a comment edit does
    not change the kernels)."""
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())


def kernel_source_digest():
    """Digest of the single-pattern scan's code (the kernels dfa_find runs),
    comments excluded."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1506_08612_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f in ("scan.cu", "automaton.cpp", "dnadfa_internal.h"):
            with open(os.path.join(csrc, f), encoding="utf-8") as fh:
                h.update(f.encode())
                h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "k_scan_tma_find_genome.txt")
    try:
        kv = {}
        with open(p) as f:
            for ln in f:
                if ":" in ln and not ln.startswith("#"):
                    k, _, v = ln.partition(":")
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_digest") != kernel_source_digest():
            return None
        return float(kv["dram_bytes_per_full_launch"])
    except Exception:
        return None


# ------------------------------------------------------------------ CPU side

def cpu_model() -> str:
    """The host CPU's model as /proc/cpuinfo names it (x86: model name;
    Arm: implementer and part numbers), else the machine type."""
    import platform
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        info = ""
    for key in ("model name", "Model"):
        for line in info.splitlines():
            if line.split(":")[0].strip() == key:
                return line.split(":", 1)[1].strip()
    parts = sorted({line.split(":", 1)[1].strip() for line in info.splitlines()
                    if line.split(":")[0].strip() in ("CPU implementer", "CPU part")})
    return f"{platform.machine()} ({', '.join(parts)})" if parts else platform.machine()


def oracle_timings(text_np, patterns, sample=20_000_000, reps=5):
    """The oracle's single-core forms on a prefix of the text, median of
    ``reps`` runs each: the sequential automaton walk (the paper's
    sequential version, counting) and the brute-force window compare."""
    import statistics

    import oracle
    t = text_np[:sample]
    deltas = [(oracle.dfa_delta(p), len(p)) for p in patterns]

    def med(fn):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)
    seq = med(lambda: [oracle.dfa_scan(t, d, m, cap=0) for d, m in deltas])
    brute = med(lambda: [oracle.count_brute(t, p) for p in patterns])
    work = t.size * len(patterns)
    return {"sample_bytes": int(t.size), "patterns": len(patterns), "reps": reps, "statistic": "median",
            "sequential_dfa_1core_gbs": round(work / seq / 1e9, 4),
            "brute_force_1core_gbs": round(work / brute / 1e9, 4),
            "nproc": os.cpu_count(), "cpu": cpu_model()}


def cpu_baseline(text_np, patterns, budget_s=12.0, scale_n=None):
    """The oracle's Algorithm 1 scan (OpenMP over every host core) on a
    bounded prefix of the same text; GB/s of text per pattern."""
    import oracle
    cores = oracle.num_threads()
    deltas = [(oracle.dfa_delta(p), len(p)) for p in patterns]
    probe = min(text_np.size, 32_000_000)
    t0 = time.perf_counter()
    for d, m in deltas:
        oracle.alg1_scan(text_np[:probe], d, m, p=cores * 8, v=16, nthreads=cores, want_positions=False)
    dt = time.perf_counter() - t0
    rate = probe * len(deltas) / dt
    sample = int(min(text_np.size, max(probe, rate * budget_s / len(deltas))))
    t0 = time.perf_counter()
    for d, m in deltas:
        oracle.alg1_scan(text_np[:sample], d, m, p=cores * 8, v=16, nthreads=cores, want_positions=True)
    dt = time.perf_counter() - t0
    gbs = sample * len(deltas) / dt / 1e9
    return {"value": round(gbs, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {sample} bytes of the {text_np.size}-byte text x {len(deltas)} patterns,"
                      f" Algorithm 1 (p={cores * 8} chunks, v=16 lanes, m-1 overlap), count + positions,"
                      f" {dt:.1f} s",
            "oracle_timings": oracle_timings(text_np, patterns)}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    import synth
    n = args.n
    patterns = [synth.pattern(m, s) for m, s in zip(PATTERN_LENGTHS, PATTERN_SEEDS)]
    import oracle
    cores = oracle.num_threads()
    # each step: a bounded prefix of the workload, sized for ~a few seconds
    sample = min(n, 400_000_000)
    text = synth.genome_text(sample, TEXT_SEED)
    deltas = [(oracle.dfa_delta(p), len(p)) for p in patterns]

    def step():
        for d, m in deltas:
            oracle.alg1_scan(text, d, m, p=cores * 8, v=16, nthreads=cores, want_positions=True)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = sample * len(deltas) * args.steps / dt / 1e9
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "impl": "reference",
            "config": config_dict(n, world, None),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {sample} bytes of the text x {len(deltas)} patterns per step,"
                                       " Algorithm 1 with OpenMP"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU side

def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1506_08612_gb300 as dd
    import synth

    n = args.n
    seed = TEXT_SEED + 1000 * rank         # each rank scans its own replica
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    synth.genome_text(n, seed, out=host.numpy())
    text = host.to(dev, non_blocking=False)
    patterns = [synth.pattern(m, s) for m, s in zip(PATTERN_LENGTHS, PATTERN_SEEDS)]
    tables = [dd.dfa_build(p) for p in patterns]
    stream = torch.cuda.current_stream(dev)
    # launch configuration per pattern: library defaults, one given
    # configuration, or "auto" (the autotuner, timed on dfa_find itself)
    if args.cfg == "auto":
        from paper_1506_08612_gb300 import autotune
        cfgs = [autotune.tune_single(text, t, stream=stream, op="find") for t in tables]
    else:
        cfgs = [json.loads(args.cfg) if args.cfg else None] * len(tables)
    cfg = cfgs[0] if len(set(json.dumps(c, sort_keys=True) for c in cfgs)) == 1 else cfgs

    # exact counts first (sizes the position buffers), untimed
    counts = [dd.count(text, t, cfg=c) for t, c in zip(tables, cfgs)]
    caps = [max(16, c) for c in counts]
    pos = [torch.empty(c, dtype=torch.int64, device=dev) for c in caps]
    cnt = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in tables]
    ws = torch.empty(max(dd.dfa_find_workspace_bytes(n, c) for c in cfgs), dtype=torch.uint8, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in tables]

    def step():
        for i, t in enumerate(tables):
            dd.dfa_find(text, t, pos[i], cnt[i], ws, cfg=cfgs[i], stream=stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    for i in range(len(tables)):
        rc, c = dd.dfa_find_status(ws, cnt[i], caps[i], stream=stream)
        assert rc == dd.DFA_OK and c == counts[i], (i, rc, c, counts[i])

    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(gpu_smi_id(local))
    clocks.start()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step()
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
        torch.distributed.barrier()
    for i in range(len(tables)):
        assert int(cnt[i].item()) == counts[i]
    ms_per_step = total_ms / args.steps
    bytes_per_step = n * len(tables)
    value = bytes_per_step * world / (ms_per_step * 1e-3) / 1e9

    # dominant kernel roofline: every launch is the same kernel; time each one
    # over a separate pass of K launches with events on the launching stream.
    # An untimed step is queued first, so that the events bracket the finds'
    # device time and not the host's submission of the first one.
    k_ms = []
    for _ in range(args.steps):
        step()
        for i, t in enumerate(tables):
            ev[i][0].record(stream)
            dd.dfa_find(text, t, pos[i], cnt[i], ws, cfg=cfgs[i], stream=stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        k_ms.append([ev[i][0].elapsed_time(ev[i][1]) for i in range(len(tables))])
    mean_launch_ms = float(np.mean(k_ms))
    algo_bytes = n + 8 * float(np.mean(counts))
    achieved = algo_bytes / (mean_launch_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": profiled_traffic(),
            "kernel": DOMINANT_KERNEL, "peak_kind": f"{peak_kind} (hbm_gbs copy bandwidth)",
            "per_pattern_ms": [round(float(np.mean([r[i] for r in k_ms])), 4) for i in range(len(tables))],
            "per_pattern_frac": [round((n + 8 * counts[i]) / (float(np.mean([r[i] for r in k_ms])) * 1e-3) / 1e9
                                       / peak, 4) for i in range(len(tables))],
            "algorithmic_bytes_per_launch": "n + 8 * count (text read once, positions written)"}

    e2e = None
    if not args.no_e2e:
        # one call per step: the host text crosses the link once for all five
        # patterns (dfa_find_host_multi), positions come back to host memory
        seg = 256 << 20
        stage = torch.empty(dd.dfa_host_stage_bytes_multi(seg, caps), dtype=torch.uint8, device=dev)
        hpos = [torch.empty(c, dtype=torch.int64, pin_memory=True) for c in caps]
        rc, cs = dd.dfa_find_host_multi(host, tables, hpos, stage, seg, stream=stream)
        assert rc == dd.DFA_OK and cs == counts, (rc, cs, counts)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e2e_steps = min(args.steps, 20)
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(e2e_steps):
            rc, cs = dd.dfa_find_host_multi(host, tables, hpos, stage, seg, stream=stream)
            assert cs == counts
            d2h += sum(8 * c + 8 for c in cs)
        dt = time.perf_counter() - t0
        if world > 1:
            tt = torch.tensor([dt], device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            dt = float(tt.item())
        e2e = {"value": round(bytes_per_step * world * e2e_steps / dt / 1e9, 3), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(min(seg + max(PATTERN_LENGTHS) - 1, n - lo)
                                             for lo in range(0, n, seg))), "d2h_bytes_per_step": int(d2h // e2e_steps),
               "steps": e2e_steps,
               "entry_point": "dfa_find_host_multi (pinned host text copied once per step in 256 MiB"
                              " segments overlapped with the five finds; positions to pinned host)"}

    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        cpu = cpu_baseline(host.numpy(), patterns)

    workloads = None
    if world == 1 and not args.no_workloads:
        del text, pos, ws
        torch.cuda.empty_cache()
        workloads = other_workloads(args, dd, dev, stream, local)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic", "config": config_dict(n, world, cfg), "clocks": clk,
                "e2e": e2e, "gpu_launches": args.steps * sum(kernels_per_find(m, c) for m, c in zip(PATTERN_LENGTHS, cfgs)),
                "roofline": roof,
                "cpu_baseline": cpu, "counts": counts, "workloads": workloads}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------- batched workloads

BATCH_SIZES = (200_000_000, 1_000_000_000, 2_400_000_000, 2_400_000_000, 2_700_000_000,
               3_200_000_000)


def lds_peak_lookups():
    """Shared-memory lookups per second if every warp-wide load were free of
    bank conflicts: SMs x 32 lanes per clock x the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return sms * 32 * mhz * 1e6, sms, mhz


def _brief(line):
    """A workload's line without the keys the headline line already states."""
    drop = ("n_gpus", "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "e2e", "warmup")
    return {k: v for k, v in line.items() if k not in drop}


def other_workloads(args, dd, dev, stream, local):
    """The other workloads, measured after the headline on the same GPU (the
    genome text freed first): the 16 MiB single-pattern case; the batched
    six sequences x 256 patterns and the 6-mer census, each against its
    one-pattern-per-launch plain form; serving on the same six resident
    sequences against the plain form.  Sizes scale with --n."""
    import torch
    out = {"small_16MiB_m8": measure_small(dd, dev, stream)}
    steps = max(3, min(args.steps, 20))
    texts, sizes, pats, exp, wl = make_many("batched", args.n, 0, dev)
    out["batched_6seq_256pat"] = _brief(measure_many("batched", texts, sizes, pats, exp, wl, dev, steps,
                                                     max(args.warmup, 3), 1, local=local))
    ctexts, csizes, cpats, cexp, cwl = make_many("census", args.n, 0, dev)
    out["census_4096_6mers"] = _brief(measure_many("census", ctexts, csizes, cpats, cexp, cwl, dev, steps,
                                                   max(args.warmup, 3), 1, local=local))
    del ctexts
    torch.cuda.empty_cache()
    out["serve_200qps"] = _brief(measure_serve(texts, sizes, args.rate, args.serve_queries, args.slots,
                                               local, search_sustainable=False))
    del texts
    torch.cuda.empty_cache()
    return out


def make_many(kind, n_scale, rank=0, dev=None, texts=None):
    """Inputs of a many-pattern workload: (device texts, sizes, patterns,
    class expansions or None, description).  ``texts`` reuses sequences
    already resident (the batched and serving workloads share theirs)."""
    import itertools

    import torch
    import synth
    expansions = None
    if kind == "classes":
        sizes = [n_scale]
        seeds = [TEXT_SEED + 1000 * rank]
        cp = synth.class_pattern_pairs(CLASS_PAIRS, CLASS_SEED)
        pats = [c for c, _ in cp]
        expansions = [e for _, e in cp]
        workload = ("class patterns: 9 pairs shaped like Table III's class cells (an 8-mer with one "
                    "position widened to the 3 other bases, and its reverse complement) over one "
                    "genome-like text")
    elif kind == "batched":
        sizes = [max(int(s * n_scale / TEXT_BYTES), 4096) for s in BATCH_SIZES]
        seeds = [10 + i + 1000 * rank for i in range(len(sizes))]
        lens = synth.uniform_ints(256, 61, 16) + 4
        pats = [synth.pattern(int(m), 16 * 100_000 + i) for i, m in enumerate(lens)]
        workload = "batched: 6 genome-like sequences x 256 patterns, lengths U[4,64]"
    else:
        sizes = [max(int(1_000_000_000 * n_scale / TEXT_BYTES), 4096)]
        seeds = [20 + 1000 * rank]
        pats = ["".join(x).encode() for x in itertools.product("ACGT", repeat=6)]
        workload = "k-mer census: all 4096 6-mers over one genome-like text"
    if texts is None:
        texts = []
        for n, sd in zip(sizes, seeds):
            h = synth.genome_text(n, sd)
            texts.append(torch.from_numpy(h).to(dev))
            del h
    return texts, sizes, pats, expansions, workload


def measure_many(kind, texts, sizes, pats, expansions, workload, dev, steps, warmup, plain_steps,
                 cfg="auto", world=1, local=0):
    """Many patterns in one persistent graph-captured launch (batched: six
    genome-like sequences x 256 patterns of length U[4, 64]; census: all
    4096 6-mers over 1e9 bytes; classes: 18 character-class patterns shaped
    like Table III's class cells over the 3.2e9-byte genome text), against
    the plain form: one dfa_count launch per (sequence, pattern), for class
    patterns one per plain expansion, summed.  Returns the JSON line."""
    import numpy as np
    import torch

    import paper_1506_08612_gb300 as dd
    classes = kind == "classes"
    total = sum(sizes)
    t0 = time.perf_counter()
    b = dd.BatchedCount(texts, pats, cfg=cfg, classes=classes)
    setup_s = time.perf_counter() - t0
    for _ in range(max(warmup, 0)):
        b.run()
    counts = b.result()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(gpu_smi_id(local))
    clocks.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    for _ in range(steps):
        b.run()
    e1.record(b.stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    assert np.array_equal(b.result(), counts)
    value = len(pats) * total * world / (ms * 1e-3) / 1e9

    # the plain form: one dfa_count launch per (sequence, pattern); a class
    # pattern is the sum of its plain expansions
    flat = [e for exp in expansions for e in exp] if classes else pats
    tables = [dd.dfa_build(p) for p in flat]
    outs = torch.zeros(len(texts) * len(flat), dtype=torch.int64, device=dev)
    st = torch.cuda.current_stream(dev)

    def plain():
        k = 0
        for t in texts:
            for tab in tables:
                dd.dfa_count(t, tab, outs[k:k + 1], stream=st)
                k += 1
    plain()
    torch.cuda.synchronize()
    plain_counts = outs.cpu().numpy().astype(np.uint64).reshape(len(texts), len(flat))
    if classes:
        ends = np.cumsum([len(x) for x in expansions])
        plain_counts = np.stack([plain_counts[:, e - len(x):e].sum(axis=1) for e, x in zip(ends, expansions)],
                                axis=1)
    assert np.array_equal(plain_counts, counts), "batched and plain counts differ"
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(st)
    for _ in range(plain_steps):
        plain()
    p1.record(st)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1) / plain_steps
    plain_value = len(pats) * total * world / (plain_ms * 1e-3) / 1e9
    del tables, outs

    peak_lk, sms, mhz = lds_peak_lookups()
    lookups_per_s = total / (ms * 1e-3)            # one table lookup per text byte
    hbm_peak, hbm_kind = measured_peak_hbm()
    lens = [int(x) for t in b.tables for x in t.lengths]
    metric = ("class patterns x GB/s of DNA text counted (one graph launch)" if classes
              else "patterns x GB/s of DNA text counted (batched, one graph launch)")
    line = {"metric": metric,
            "value": round(value, 1), "unit": "patterns*GB/s", "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "workload": kind,
            "config": {"workload": workload, "sequence_bytes": sizes, "patterns": len(pats),
                       "pattern_lengths": [min(lens), max(lens)],
                       "automaton_states": [t.states() for t in b.tables],
                       "launch_config": b.cfgs, "launches_per_step": b.launches,
                       "graph": b.graph is not None, "l2": "inputs larger than L2 (no flush)",
                       "setup_s": round(setup_s, 3)},
            "text_gbs": round(total * world / (ms * 1e-3) / 1e9, 2),
            "plain_form": {"value": round(plain_value, 1), "unit": "patterns*GB/s",
                           "ms_per_step": round(plain_ms, 3),
                           "launches_per_step": len(texts) * len(flat),
                           "what": ("one dfa_count launch per plain expansion of each class pattern, summed"
                                    if classes else
                                    "one dfa_count launch per (sequence, pattern), library defaults")},
            "speedup_vs_plain": round(plain_ms / ms, 2),
            "roofline": {"bound": "alu", "achieved": round(lookups_per_s / 1e12, 4),
                         "peak": round(peak_lk / 1e12, 4), "unit": "Tlookups/s",
                         "frac": round(lookups_per_s / peak_lk, 4), "traffic": None,
                         "kernel": "k_multi_count (one shared-memory table lookup per text byte)",
                         "peak_kind": f"derived: {sms} SMs x 32 shared-memory lanes/clk x {mhz:.0f} MHz",
                         "hbm_frac": round(total / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                         "hbm_peak": f"{hbm_peak} GB/s ({hbm_kind})"},
            "clocks": clk, "gpu_launches": steps * b.launches, "e2e": None,
            "checksum": int(counts.sum())}
    b.close()
    torch.cuda.empty_cache()
    return line


def run_batched(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    texts, sizes, pats, expansions, workload = make_many(args.workload, args.n, rank, dev)
    cfg = json.loads(args.cfg) if args.cfg else "auto"
    line = measure_many(args.workload, texts, sizes, pats, expansions, workload, dev, args.steps,
                        args.warmup, args.plain_steps, cfg=cfg, world=world, local=local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_serve(seqs, sizes, rate, queries, slots, local=0, search_sustainable=True):
    """Serving: the six batched-workload sequences resident in HBM, a Poisson
    trace of queries (sequence uniform over the six, 1-64 patterns of length
    U[4, 64], count or positions with probability 1/2) replayed open-loop at
    the offered rate; p50/p99 latency from arrival to the answer on the
    host.  The same trace head also runs through the plain form (each query
    alone, one single-pattern launch per pattern).  Returns the JSON line."""
    import torch
    import synth
    from paper_1506_08612_gb300.serve import GpuEngine, Server, latency_summary
    arena = 8 << 30

    def run(rate, k, seed, plain=False):
        eng = GpuEngine(seqs, slots=slots, arena_bytes=arena, plain=plain)
        srv = Server(eng, max_batch_queries=1) if plain else Server(eng)
        srv.replay(synth.query_trace(8, rate, len(seqs), seed + 1))          # warm-up
        trace = synth.query_trace(k, rate, len(seqs), seed)
        clocks = ClockSampler(gpu_smi_id(local))
        clocks.start()
        qs = srv.replay(trace)
        clk = clocks.stop()
        st = latency_summary(qs)
        span = max(q.t_done for q in qs) - min(q.t_arrive for q in qs)
        pbytes = sum(len(q.patterns) * sizes[q.seq] for q in qs)
        st.update({"offered_qps": rate, "queries": k, "trace_s": round(trace[-1]["t"], 3),
                   "span_s": round(span, 3), "patterns_gbs": round(pbytes / span / 1e9, 1),
                   "batches": srv.stats["batches"], "mem_stalls": srv.stats["mem_stalls"],
                   "positions_queries": sum(q.mode == "positions" for q in qs)})
        st["sustained"] = bool(st["qps"] >= 0.95 * rate)
        for key in ("p50_ms", "p99_ms", "max_ms", "mean_ms", "qps"):
            st[key] = round(st[key], 3)
        del eng, srv
        torch.cuda.empty_cache()
        return st, clk

    main, clk = run(rate, queries, 30)
    sustainable = None
    if search_sustainable and not main["sustained"]:
        for r in (0.7, 0.5, 0.35, 0.25, 0.15):
            st, _ = run(rate * r, max(100, queries // 5), 40)
            if st["sustained"]:
                sustainable = st
                break
    plain, _ = run(rate, max(50, queries // 20), 30, plain=True)
    return {"metric": "serving: completed queries per second at the offered Poisson rate",
            "value": main["qps"], "unit": "queries/s", "n_gpus": 1, "steps": queries,
            "warmup": 8, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic", "workload": "serve",
            "config": {"workload": "serving: six resident genome-like sequences, Poisson queries",
                       "sequence_bytes": sizes, "offered_qps": rate, "slots": slots,
                       "position_arena_bytes": arena,
                       "query": "seq U{0..5}, 1-64 patterns of length U[4,64], count or positions p=1/2"},
            "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"], "serving": main,
            "max_sustainable": sustainable, "plain_form": plain,
            "speedup_vs_plain_qps": round(main["qps"] / max(plain["qps"], 1e-9), 2),
            "clocks": clk, "e2e": None}


def run_serve(args):
    import torch

    world, rank, local = dist_env()
    if world > 1 and rank != 0:
        return                                   # one server per box: rank 0 only
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    seqs, sizes, _, _, _ = make_many("batched", args.n, 0, dev)
    line = measure_serve(seqs, sizes, args.rate, args.queries, args.slots, local)
    print(json.dumps(line), flush=True)


C1_BYTES, C1_SEED, C1_M, C1_PSEED = 16 << 20, 0, 8, 1


def measure_small(dd, dev, stream, reps=20, graph_reps=200):
    """The plain single-pattern method on a 16 MiB uniform A/C/G/T text
    (seed 0) and an 8-mer (seed 1): dfa_find (count + sorted positions)
    timed alone after an L2 flush (a 512 MiB write, 4x the L2) before each
    of ``reps`` repetitions (median, p10, p90), and as ``graph_reps`` finds
    back to back in one CUDA graph (the text then stays in L2)."""
    import numpy as np
    import torch
    import synth
    host = synth.uniform_text(C1_BYTES, C1_SEED)
    pat = synth.pattern(C1_M, C1_PSEED)
    text = torch.from_numpy(host).to(dev)
    table = dd.dfa_build(pat)
    want = dd.count(text, table)
    cap = max(16, want)
    pos = torch.empty(cap, dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.empty(dd.dfa_find_workspace_bytes(C1_BYTES), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for _ in range(3):
        dd.dfa_find(text, table, pos, cnt, ws, stream=stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i, (a, b) in enumerate(evs):
            flush.fill_(i & 0xFF)
            a.record(stream)
            dd.dfa_find(text, table, pos, cnt, ws, stream=stream)
            b.record(stream)
    torch.cuda.synchronize()
    rc, c = dd.dfa_find_status(ws, cnt, cap, stream=stream)
    assert rc == dd.DFA_OK and c == want, (rc, c, want)
    us = np.array([a.elapsed_time(b) * 1e3 for a, b in evs])
    # graph: graph_reps finds back to back, one replay
    g_stream = torch.cuda.Stream(dev)
    g_stream.wait_stream(torch.cuda.current_stream(dev))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=g_stream):
        for _ in range(graph_reps):
            dd.dfa_find(text, table, pos, cnt, ws, stream=g_stream)
    with torch.cuda.stream(g_stream):
        g.replay()
    g_stream.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(g_stream):
        g0.record(g_stream)
        g.replay()
        g1.record(g_stream)
    g_stream.synchronize()
    graph_us = g0.elapsed_time(g1) * 1e3 / graph_reps
    assert int(cnt.item()) == want
    peak, kind = measured_peak_hbm()
    med = float(np.median(us))
    algo = C1_BYTES + 8 * want
    del g, flush
    torch.cuda.empty_cache()
    return {"workload": "single pattern, plain method: 16 MiB uniform A/C/G/T (seed 0), m = 8 (seed 1),"
                        " count + sorted int64 positions",
            "count": want,
            "flushed": {"reps": reps, "median_us": round(med, 2),
                        "p10_us": round(float(np.percentile(us, 10)), 2),
                        "p90_us": round(float(np.percentile(us, 90)), 2),
                        "gbs": round(C1_BYTES / (med * 1e-6) / 1e9, 1),
                        "l2": "512 MiB write (4x L2) before each find"},
            "graph_back_to_back": {"finds": graph_reps, "us_per_find": round(graph_us, 2),
                                   "gbs": round(C1_BYTES / (graph_us * 1e-6) / 1e9, 1),
                                   "l2": "text resident in L2 across the finds"},
            "roofline": {"bound": "hbm", "achieved": round(algo / (med * 1e-6) / 1e9, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(algo / (med * 1e-6) / 1e9 / peak, 4),
                         "traffic": None, "peak_kind": f"{kind} (hbm_gbs copy bandwidth)",
                         "note": "16 MiB is a few microseconds of HBM time: launch latency bounds it"},
            "launches_per_find": kernels_per_find(8, None)}


def run_shard(args):
    """One genome split over the ranks, Algorithm 1's chunking one level up:
    rank r finds the occurrences that start in its shard (4 KiB-aligned
    slices, so each keeps the TMA path), reading m - 1 bytes past it; per
    pattern the counts and positions are gathered over the process group
    (NCCL: device tensors, no host copy) and merged in rank order.  A step is
    the five finds plus their exchanges; ``value`` is the whole text x
    patterns over the slowest rank's time.  Rank 0 checks the merged counts
    against one whole-text count on its GPU and the positions' order."""
    import numpy as np
    import torch

    import paper_1506_08612_gb300 as dd
    import synth
    from paper_1506_08612_gb300 import shard

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    align = 4096
    host = synth.genome_text(n, TEXT_SEED)               # every rank: the same text
    patterns = [synth.pattern(m, sd) for m, sd in zip(PATTERN_LENGTHS, PATTERN_SEEDS)]
    tables = [dd.dfa_build(p) for p in patterns]
    s, e = shard.shard_range(n, world, rank, align)
    rs, re = shard.read_range(n, world, rank, max(PATTERN_LENGTHS), align)
    text = torch.from_numpy(np.ascontiguousarray(host[rs:re])).to(dev)
    # pattern i reads [s, min(e + m_i - 1, n)): every occurrence found starts in [s, e)
    lens = [min(e + len(p) - 1, n) - s if e > s else 0 for p in patterns]
    local_counts = [dd.count(text[:k], t) if k else 0 for k, t in zip(lens, tables)]
    caps = [max(16, c) for c in local_counts]
    pos = [torch.empty(c, dtype=torch.int64, device=dev) for c in caps]
    cnt = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in tables]
    ws = torch.empty(dd.dfa_find_workspace_bytes(max(max(lens), 1)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        out = []
        for i, t in enumerate(tables):
            if lens[i]:
                dd.dfa_find(text, t, pos[i], cnt[i], ws, stream=stream, n=lens[i])
        for i in range(len(tables)):
            c = local_counts[i]
            mine = pos[i][:c] + s
            if world > 1:
                out.append(shard.gather_find(c, mine))
            else:
                out.append((c, mine))
        return out

    for _ in range(max(args.warmup, 0)):
        merged = step()
    torch.cuda.synchronize()
    if rank == 0:
        whole = torch.from_numpy(host).to(dev)
        want = [dd.count(whole, t) for t in tables]
        del whole
        torch.cuda.empty_cache()
        for (c, p), w in zip(merged, want):
            assert c == w, (c, w)
            if c > 1:
                assert bool((p[1:] > p[:-1]).all())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([dt], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        dt = float(tt.item())
    value = n * len(tables) * args.steps / dt / 1e9
    if rank == 0:
        cfgd = config_dict(n, world, None)
        cfgd["parallelism"] = f"shard x{world} (4 KiB-aligned shards, m-1 overlap, all-gather of counts + positions)"
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 4),
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u8",
                "data": "synthetic", "config": cfgd, "e2e": None,
                "gpu_launches": args.steps * sum(kernels_per_find(m, None) for m in PATTERN_LENGTHS),
                "counts": [int(c) for c, _ in merged], "shard_bytes": [s, e]}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.shard:
        run_shard(args)
    elif args.workload in ("batched", "census", "classes"):
        run_batched(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
