"""Benchmark: exact HN 1-NN queries/s on one B300 (or N, one process each).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c0|c1|c2|c3|c4] [--prefix f32|bf16|fp8|i8]
                    [--scan auto|stream|dense|dense2] [--clock-log PATH]

Workload (default c2): N = 4,000,000 database entries, a batch of 65,536
queries, D = 128, K = 16, alpha = 1/8, clustered synthetic descriptors
(800,000 centres, entry noise 0.15, query noise 0.10), BF16 major prefix
(--prefix fp8: the FP8-e4m3 form of the same workload; --prefix i8: the int8
fixed-point form, scanned with dp4a on the CUDA cores).  c0 and c1 are the
smaller configurations (FP32 prefix by default); c3 compares the search
seeded by the learned block proposal with the plain search on c2's data;
c4 is uneven batched serving over 16 indexes.

A step is one pass of the hot path over one query batch, all through the C
ABI: HN normalisation of the raw queries, query prefix packing, the prefix
scan, threshold from the best scanned candidates, the bound test, survivor
rescore with binary64 near-ties, argmax.  The dense scan (BF16/FP8 prefix on
the tensor cores) computes the prefix product once per step by default
(--scan dense); --scan dense2 runs Algorithm 1's two passes (Phase 1, then
Phase 2 against the threshold).  The database
index (normalisation and SoA packing of the 4M entries) is built once before
timing; its build time is reported separately.  L2 is flushed (256 MiB
write) before every timed step.

N > 1 (torchrun): every rank holds its own copy of the index and answers its
own 65,536-query batch (weak scaling, no data-path collective); the barrier
serves timing only.

--impl reference times the binary64 CPU oracle on this host's cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import hn_synth  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(hn_synth.CONFIGS) + ["c4"])
    ap.add_argument("--prefix", default=None, choices=["f32", "bf16", "fp8", "i8"])
    ap.add_argument("--scan", default="auto", choices=["auto", "stream", "dense", "dense2"])
    ap.add_argument("--clock-log", default=None,
                    help="file for the nvidia-smi clock samples of the timed region (default: a temporary file)")
    ap.add_argument("--rescore", choices=["filter16", "best_first", "full"], default="filter16",
                    help="Phase-2 rescore of the 1-NN search (same result): certified FP16-row bound before the "
                         "FP32 row (default), the FP32 prefix bound (best first), or every survivor in FP32")
    ap.add_argument("--best-first", action="store_true", help="the same as --rescore best_first")
    ap.add_argument("--train-precision", choices=["bf16", "fp32"], default="bf16",
                    help="c3: the proposal's training GEMMs on the tensor cores (bf16) or the CUDA cores (fp32)")
    ap.add_argument("--no-autotune", action="store_true", help="c4: keep every index's default scan choices")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bruteforce", action="store_true")
    ap.add_argument("--hard", action="store_true",
                    help="stress variant of the workload: entry noise 0.3, query noise 0.2 (many survivors)")
    ap.add_argument("--beta-sweep", action="store_true",
                    help="soft ANN mode: queries/s, survivors and recall@1 for beta = alpha .. 0 (c2 data)")
    return ap.parse_args()


DRAM_PROFILE = os.path.join(ROOT, "profiles", "k_dense_scan_c2_dram.md")
# the scan kernel and the header that fixes its launch configuration (work-unit granularity)
DENSE_SOURCES = [os.path.join(ROOT, "paper_2606_27280_b300", "csrc", f) for f in ("hn_dense.cu", "hn_internal.cuh")]


def measured_traffic(workload: str, prefix: str, scan: int):
    """DRAM bytes (read + write) per launch of the reported dense-scan kernel from the committed
    ncu capture; None unless the capture covers this workload, prefix and scan form and the
    kernel's sources are unchanged since (the sha256 of hn_dense.cu followed by hn_internal.cuh
    is recorded beside the figures)."""
    try:
        with open(DRAM_PROFILE) as f:
            text = f.read()
        h = hashlib.sha256()
        for path in DENSE_SOURCES:
            with open(path, "rb") as f:
                h.update(f.read())
        sha = h.hexdigest()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if line.startswith("- ") and ":" in line:
            key, val = line[2:].split(":", 1)
            vals[key.strip()] = val.strip().strip("`")
    if vals.get("source sha256") != sha or workload != "c2":
        return None
    form = "one-pass" if scan == 2 else "two-pass"
    v = vals.get(f"{prefix} {form} bytes per launch")
    return float(v) if v else None


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return dict(FALLBACK_PEAKS), "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        self.gpu = gpu_index
        self.proc = None
        if path is None:
            import tempfile
            fd, path = tempfile.mkstemp(prefix=f"hn_clocks_gpu{gpu_index}_", suffix=".csv")
            os.close(fd)
        self.path = path

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons, under_load = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    s, m, pw = float(parts[1]), float(parts[2]), float(parts[3])
                except ValueError:
                    continue
                sm.append(s)
                smax.append(m)
                if pw > 200:
                    under_load.append(s)
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        use = under_load or sm
        return {"sm_mhz": statistics.median(use) if use else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_under_load": len(under_load)}


# ---------------------------------------------------------------- oracle (CPU baseline)
def cpu_baseline(wl, c, budget_s: float = 12.0):
    """Time the binary64 oracle on this host on a bounded query sample of the same workload."""
    import oracle
    k, alpha = c["k"], c["alpha"]
    t0 = time.perf_counter()
    db = oracle.normalize(wl.db_raw, k, alpha)
    norm_s = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    probe = min(8, wl.q_raw.shape[0])
    q = oracle.normalize(wl.q_raw[:probe], k, alpha)
    t0 = time.perf_counter()
    oracle.search(db, q)
    dt = time.perf_counter() - t0
    per_q = dt / probe
    m = int(max(probe, min(wl.q_raw.shape[0], budget_s / max(per_q, 1e-9))))
    q = oracle.normalize(wl.q_raw[:m], k, alpha)
    t0 = time.perf_counter()
    oracle.search(db, q)
    dt = time.perf_counter() - t0
    # the same oracle on one core, a few queries (about a quarter of the budget)
    m1 = int(max(1, min(m, 0.25 * budget_s / max(per_q * cores, 1e-9))))
    t1 = time.perf_counter()
    oracle.search(db, q[:m1], nthreads=1)
    dt1 = time.perf_counter() - t1
    return {"value": m / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"first {m} of {wl.q_raw.shape[0]} queries against all {c['n']} entries "
                      f"(binary64 exhaustive search, OpenMP over {cores} threads); "
                      f"database normalisation {norm_s:.1f}s not included",
            "seconds": dt,
            "single_core": {"value": m1 / dt1, "unit": "queries/s", "cores": 1,
                            "sample": f"first {m1} queries, one thread", "seconds": dt1}}


def rank_queries(wl, c: dict, rank: int) -> np.ndarray:
    """The query batch of one rank: the workload's own queries on rank 0, further batches
    drawn the same way from seeded streams of their own on the other ranks (weak scaling:
    every rank answers a full, different batch against its own copy of the index)."""
    if rank == 0:
        return wl.q_raw
    return hn_synth.queries_from(wl.db_raw, c["nq"], seed=c["seed"] * 7919 + rank)[0]


def max_over_ranks(torch, t_local: float, dist, device: str) -> float:
    """The slowest rank's time (seconds); the job's throughput divides all ranks' work by it."""
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def default_prefix(workload: str) -> str:
    return "bf16" if workload == "c2" else "f32"


HARD_NOISE = (0.3, 0.2)  # entry and query noise of the stress variant


def load_workload(workload: str, hard: bool):
    wl, c = hn_synth.config_workload(workload)
    if hard:
        c = dict(c, entry_noise=HARD_NOISE[0], query_noise=HARD_NOISE[1])
        wl = hn_synth.make_workload(c["n"], c["nq"], c["n_centres"], c["seed"], *HARD_NOISE)
    return wl, c


def workload_config(workload: str, c: dict, prefix_name: str, world: int) -> dict:
    """The `config` of a bench line; the reference arm prints the same one."""
    k, alpha, nq = c["k"], c["alpha"], c["nq"]
    hard = (f", hard variant (entry noise {c['entry_noise']}, query noise {c['query_noise']})"
            if "entry_noise" in c else "")
    return {"workload": f"{workload}: N={c['n']} entries, Q={nq} queries per step, D=128, K={k}, "
                        f"alpha={alpha}, {c['n_centres']} centres, {prefix_name} prefix{hard}",
            "n": c["n"], "queries_per_step": nq, "k": k, "alpha": alpha, "prefix": prefix_name,
            "parallelism": f"replicated index, {world} GPU(s), independent query batches",
            "l2": "flushed before every timed step (256 MiB write); index 2 GiB > L2"}


def run_reference(args, rank: int):
    if rank != 0:
        return 0
    workload = args.workload if args.workload in ("c0", "c1", "c2") else "c2"
    wl, c = load_workload(workload, args.hard)
    per_step, total_q = [], 0
    import oracle
    db = oracle.normalize(wl.db_raw, c["k"], c["alpha"])
    # bounded sample per step so that the whole run ends within a few minutes
    m = 64 if c["n"] >= 1_000_000 else min(256, c["nq"])
    for s in range(args.warmup + args.steps):
        lo = (s * m) % max(1, c["nq"] - m)
        t0 = time.perf_counter()
        q = oracle.normalize(wl.q_raw[lo:lo + m], c["k"], c["alpha"])
        oracle.search(db, q)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            per_step.append(dt)
            total_q += m
    t = sum(per_step)
    value = total_q / t
    cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": "exact 1-NN queries/s", "value": value, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(workload, c, args.prefix or default_prefix(workload), args.gpus),
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                             "sample": f"{m} of the {c['nq']} queries per step against all {c['n']} entries "
                                       f"(binary64 exhaustive search incl. query normalisation)"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- ours
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import paper_2606_27280_b300 as hn

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.beta_sweep:
        return run_beta_sweep(args, hn, torch, world, rank)
    if args.workload == "c4":
        return run_serving(args, hn, torch, world, rank, dist, barrier)
    if args.workload == "c3":
        return run_proposal(args, hn, torch, world, rank, dist, barrier)

    wl, c = load_workload(args.workload, args.hard)
    k, alpha = c["k"], c["alpha"]
    prefix_name = args.prefix or default_prefix(args.workload)
    prefix = {"f32": hn.PREFIX_F32, "bf16": hn.PREFIX_BF16, "fp8": hn.PREFIX_FP8, "i8": hn.PREFIX_I8}[prefix_name]
    scan = {"auto": hn.SCAN_AUTO, "stream": hn.SCAN_STREAM, "dense": hn.SCAN_DENSE,
            "dense2": hn.SCAN_DENSE_TWO_PASS}[args.scan]
    stream = torch.cuda.current_stream()
    rescore_name = "best_first" if args.best_first else args.rescore
    rescore_mode = {"filter16": hn.RESCORE_FILTER16, "best_first": hn.RESCORE_BEST_FIRST,
                    "full": hn.RESCORE_FULL}[rescore_name]

    # ---- index (built once, outside the timed region)
    db_raw = torch.from_numpy(wl.db_raw).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    db = hn.normalize(db_raw, k, alpha)
    ix = hn.Index(db, k, alpha, prefix=prefix)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del db_raw, db
    info = ix.info()

    q_host = torch.from_numpy(rank_queries(wl, c, rank)).pin_memory()
    q_raw = q_host.cuda()
    nq = q_raw.shape[0]
    q_norm = torch.empty_like(q_raw)
    out_idx = torch.empty(nq, dtype=torch.int64, device="cuda")
    out_sim = torch.empty(nq, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # the queries are normalised on the search's stream without a host round trip; a row
    # that cannot be normalised is caught by the search itself (HN_ERR_NOT_NORMALIZED)
    def step(timing=False):
        hn.normalize_async(q_raw, k, alpha, out=q_norm)
        return ix.search(q_norm, scan=scan, out_idx=out_idx, out_sim=out_sim, timing=timing,
                         rescore=rescore_mode)

    for _ in range(args.warmup):
        r = step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, events per step, L2 flushed before each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phase = []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local, args.clock_log) as clocks:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            r = step(timing=True)
            ev[i][1].record(stream)
            phase.append(r.stats)
        torch.cuda.synchronize()
    barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_max = max_over_ranks(torch, sum(ms) / 1e3, dist, "cuda")
    value = world * nq * args.steps / t_max

    # ---- end to end through the public API: pinned host raw queries in, results out.  As a
    # serving loop runs it: each step's queries are copied from pinned host memory on a second
    # stream one step ahead (two staging buffers), the main stream waits for that copy,
    # normalises and searches, and copies the step's results back; the timed region spans all
    # steps, every copy inside it.  The inputs (index, code map) are far larger than L2.
    res_idx_host = torch.empty(nq, dtype=torch.int64).pin_memory()
    res_sim_host = torch.empty(nq, dtype=torch.float64).pin_memory()
    q_stage = [torch.empty_like(q_raw), torch.empty_like(q_raw)]
    copy_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_a, e2e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def stage_copy(i):
        buf = i % 2
        with torch.cuda.stream(copy_stream):
            if i >= 2:
                copy_stream.wait_event(free[buf])   # step i - 2 has normalised this buffer
            q_stage[buf].copy_(q_host, non_blocking=True)
            ready[buf].record(copy_stream)

    torch.cuda.synchronize()
    barrier()
    e2e_a.record(stream)
    copy_stream.wait_event(e2e_a)
    stage_copy(0)
    for i in range(args.steps):
        buf = i % 2
        if i + 1 < args.steps:
            stage_copy(i + 1)
        stream.wait_event(ready[buf])
        hn.normalize_async(q_stage[buf], k, alpha, out=q_norm)
        free[buf].record(stream)
        ix.search(q_norm, scan=scan, out_idx=out_idx, out_sim=out_sim, rescore=rescore_mode)
        res_idx_host.copy_(out_idx, non_blocking=True)
        res_sim_host.copy_(out_sim, non_blocking=True)
    e2e_b.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_t = max_over_ranks(torch, e2e_a.elapsed_time(e2e_b) / 1e3, dist, "cuda")
    e2e_value = world * nq * args.steps / e2e_t

    if rank != 0:
        dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel: the prefix scan (2*Q*N*K flop per pass over the batch)
    peaks, peak_src = load_peaks()
    clk = clocks.summary()
    st = phase[-1]
    flops = 2.0 * nq * c["n"] * k
    ms_step = 1e3 * t_max / args.steps
    med = {kk: statistics.median(p[kk] for p in phase) for kk in ("ms_phase1", "ms_threshold", "ms_phase2")}
    smax = (clk.get("sm_max_mhz") or 2032.0)
    if st["scan"] in (hn.SCAN_DENSE, hn.SCAN_DENSE_TWO_PASS):
        # a kernel timed alone against the burst cuBLAS figure when the SM clock held its
        # maximum through the timed steps, else against the sustained one
        at_max = bool(clk.get("sm_mhz")) and clk["sm_mhz"] >= 0.97 * smax
        key = "bf16_tflops" if at_max else "bf16_tflops_sustained"
        peak = peaks.get(key, FALLBACK_PEAKS[key])
        src = f"{peak_src} {'bf16 burst' if at_max else 'bf16 sustained'} (cuBLAS)" + \
              (", SM clock at its maximum in the timed steps" if at_max else ", SM clock below its maximum")
        if prefix_name == "fp8":   # e4m3 operands: the bf16 figure x the nominal fp8/bf16 ratio 4.5/2.25
            peak, src = 2.0 * peak, src + " x 2 (nominal fp8 / bf16 dense ratio)"
        bound, unit = "tensor", "TFLOP/s"
        if st["scan"] == hn.SCAN_DENSE:
            kernel = f"k_dense_scan<{info['k_pad']},4,{int(prefix_name == 'fp8')}> (one-pass tensor-core prefix scan)"
            launches = {"scan (one pass, tensor cores)": med["ms_phase1"]}
            other = {"threshold": med["ms_threshold"], "survivor extraction from the group codes": med["ms_phase2"]}
        else:
            kernel = f"k_dense_scan<{info['k_pad']},1|2,{int(prefix_name == 'fp8')}> (two-pass: Phase 1, Phase 2)"
            launches = {"phase 1 scan": med["ms_phase1"], "phase 2 scan + survivor extraction": med["ms_phase2"]}
            other = {"threshold": med["ms_threshold"]}
    elif prefix_name == "i8":
        # CUDA-core dp4a: a throughput probe measured 64 dp4a issued per clock per SM on B300
        peak = 148 * 64 * 8 * smax * 1e6 / 1e12
        bound, unit = "alu", "TOP/s"
        src = "derived: 148 SMs x 64 dp4a per clock (measured issue rate) x 8 int ops x max SM clock"
        kernel = "k_stream_scan (int8, dp4a)"
        launches = {"phase 1 scan": med["ms_phase1"], "phase 2 scan": med["ms_phase2"]}
        other = {"threshold": med["ms_threshold"]}
    else:
        # CUDA-core FP32 FMA: 148 SMs x 128 lanes x 2 flop x max SM clock
        peak = 148 * 128 * 2 * smax * 1e6 / 1e12
        bound, unit = "alu", "TFLOP/s"
        src = "derived: 148 SMs x 128 FP32 lanes x 2 flop x max SM clock"
        kernel = "k_stream_scan (FP32 FMA)"
        launches = {"phase 1 scan": med["ms_phase1"], "phase 2 scan": med["ms_phase2"]}
        other = {"threshold": med["ms_threshold"]}
    per_launch = {name: {"ms": ms_, "achieved": flops / (ms_ * 1e-3) / 1e12,
                         "frac": flops / (ms_ * 1e-3) / 1e12 / peak} for name, ms_ in launches.items()}
    first = next(iter(per_launch.values()))
    roof = {"bound": bound, "achieved": first["achieved"], "peak": peak, "unit": unit, "frac": first["frac"],
            "traffic": None, "peak_source": src, "kernel": kernel,
            "algorithmic": f"2*Q*N*K = {flops:.3e} {'int ops' if prefix_name == 'i8' else 'flop'} per scan launch "
                           f"(Q={nq}, N={c['n']}, K={k})",
            "avg_launch_ms": first["ms"], "per_launch": per_launch, "other_launches_ms": other,
            "step_frac": flops / (ms_step * 1e-3) / 1e12 / peak,
            "step_frac_note": "one 2*Q*N*K prefix product per step / whole step time / peak"}
    roof["traffic"] = measured_traffic(args.workload, prefix_name, st["scan"]) if bound == "tensor" else None
    roof["traffic_unit"] = "bytes per launch of the kernel above (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
    if bound == "tensor":
        # the epilogue's own floor: one FP32 max per score on 148 SMs x 128 lanes at the maximum clock
        roof["epilogue_alu_floor_ms"] = 1e3 * nq * c["n"] / (148 * 128 * smax * 1e6)

    line = {
        "metric": "exact 1-NN queries/s", "value": value, "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "ms_per_step_median": statistics.median(ms), "ms_per_step_best": min(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prefix_name,
        "data": "synthetic",
        "config": workload_config(args.workload, c, prefix_name, world),
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": nq * 128 * 4,
                "d2h_bytes_per_step": nq * (8 + 8)},
        "gpu_launches": args.steps * (st["kernels"] + 1),
        "clocks": clk,
        "phases_ms": {kk: statistics.median(p[kk] for p in phase) for kk in
                      ("ms_prep", "ms_phase1", "ms_threshold", "ms_phase2", "ms_rescore", "ms_total")},
        "search_stats": {kk: st[kk] for kk in ("survivors", "max_survivors", "fp64_rescored", "reruns", "scan",
                                               "passes", "kernels", "groups_scored", "rescore_skipped")},
        "survivor_frac": st["survivors"] / (nq * c["n"]),
        "rescore": rescore_name,
        "index_build_s": build_s, "index_bytes": info["device_bytes"],
    }

    # ---- GPU brute force (FP32 128-dim) on a query subset, for comparison
    if not args.no_bruteforce:
        sub = min(nq, 2048 if c["n"] >= 1_000_000 else nq)
        qs = q_norm[:sub].contiguous()
        ix.bruteforce(qs)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rb = ix.bruteforce(qs)
        b.record(stream)
        torch.cuda.synchronize()
        bf_s = a.elapsed_time(b) / 1e3
        line["gpu_bruteforce"] = {"value": sub / bf_s, "unit": "queries/s",
                                  "sample": f"{sub} queries x all {c['n']} entries, FP32 128-dim FMA",
                                  "index_mismatch_vs_hn": int((rb.idx != out_idx[:sub]).sum().item())}
        line["vs_gpu_bruteforce"] = value / (sub / bf_s)
        # a library tensor-core brute force on the same sample: cuBLAS BF16 GEMMs (FP32
        # accumulation, BF16 scores) of 256-query chunks against the whole BF16-rounded
        # database, then argmax -- a speed reference, not exact (BF16 operands and scores)
        db_bf = hn.normalize(torch.from_numpy(wl.db_raw).cuda(), k, alpha).to(torch.bfloat16)
        qb = qs.to(torch.bfloat16)
        tc_idx = torch.empty(sub, dtype=torch.int64, device="cuda")

        def tc_bruteforce():
            for i in range(0, sub, 256):
                tc_idx[i:i + 256] = torch.argmax(qb[i:i + 256] @ db_bf.T, dim=1)

        tc_bruteforce()
        torch.cuda.synchronize()
        a.record(stream)
        tc_bruteforce()
        b.record(stream)
        torch.cuda.synchronize()
        tc_s = a.elapsed_time(b) / 1e3
        line["gpu_bruteforce_tensor"] = {
            "value": sub / tc_s, "unit": "queries/s",
            "sample": f"{sub} queries x all {c['n']} entries, cuBLAS BF16 GEMM (FP32 accumulation) + argmax, "
                      "256-query chunks; not exact",
            "index_mismatch_vs_hn": int((tc_idx != out_idx[:sub]).sum().item())}
        line["vs_gpu_bruteforce_tensor"] = value / (sub / tc_s)
        del db_bf

    if not args.no_cpu_baseline and world == 1:   # the oracle is timed at N = 1 only
        line["cpu_baseline"] = cpu_baseline(wl, c)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _timed_steps(torch, stream, steps, fn, flush):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    out = []
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        out.append(fn())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], out


def run_beta_sweep(args, hn, torch, world, rank):
    """Soft ANN mode on the workload's data (threshold relaxation of the paper's closing
    section): the skip test's alpha replaced by beta.  recall@1 is measured against the
    exact search (beta = alpha), which the parity tests hold equal to the oracle."""
    if world > 1:
        raise SystemExit("--beta-sweep runs on one GPU")
    wl, c = hn_synth.config_workload(args.workload)
    k, alpha = c["k"], c["alpha"]
    prefix_name = args.prefix or "bf16"
    prefix = {"f32": hn.PREFIX_F32, "bf16": hn.PREFIX_BF16, "fp8": hn.PREFIX_FP8, "i8": hn.PREFIX_I8}[prefix_name]
    stream = torch.cuda.current_stream()
    db = hn.normalize(torch.from_numpy(wl.db_raw).cuda(), k, alpha)
    ix = hn.Index(db, k, alpha, prefix=prefix)
    del db
    q = hn.normalize(torch.from_numpy(wl.q_raw).cuda(), k, alpha)
    nq = q.shape[0]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    exact = ix.search(q, stats=True)
    rows = []
    for frac in (1.0, 0.5, 0.25, 0.125, 0.0625, 0.0):
        beta = alpha * frac
        for _ in range(args.warmup):
            ix.search(q, beta=beta)
        ms, out = _timed_steps(torch, stream, args.steps, lambda: ix.search(q, beta=beta, stats=True), flush)
        r = out[-1]
        rows.append({"beta": beta, "queries_per_s": nq / (statistics.median(ms) * 1e-3),
                     "ms_per_step": statistics.median(ms),
                     "survivor_frac": r.stats["survivors"] / (nq * c["n"]),
                     "recall_at_1": float((r.idx == exact.idx).float().mean().item()),
                     "max_sim_loss": float((exact.sim - r.sim).max().item())})
    line = {"metric": "soft ANN mode: exact 1-NN recall and queries/s vs beta", "unit": "queries/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": prefix_name, "data": "synthetic",
            "config": {"workload": f"{args.workload}: N={c['n']}, Q={nq}, K={k}, alpha={alpha}, {prefix_name} prefix",
                       "l2": "flushed before every timed step (256 MiB write)"},
            "sweep": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_proposal(args, hn, torch, world, rank, dist, barrier):
    """c3: the learned block proposal seeds the threshold (Phase 1 skipped), versus the plain search."""
    c = dict(hn_synth.CONFIGS["c3"])
    wl = hn_synth.make_workload(c["n"], c["nq"], c["n_centres"], c["seed"])
    k, alpha = c["k"], c["alpha"]
    stream = torch.cuda.current_stream()
    db = hn.normalize(torch.from_numpy(wl.db_raw).cuda(), k, alpha)
    t0 = time.perf_counter()
    ix = hn.Index(db, k, alpha, prefix=hn.PREFIX_BF16, n_blocks=c["n_blocks"])
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    tq_raw, _ = hn_synth.queries_from(wl.db_raw, c["n_train"], seed=c["train_seed"])
    tq = hn.normalize(torch.from_numpy(tq_raw).cuda(), k, alpha)
    del db, tq_raw
    t0 = time.perf_counter()
    prop = hn.Proposal.train(ix, tq, seed=7, precision=0 if args.train_precision == "bf16" else 1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del tq
    q_raw = torch.from_numpy(wl.q_raw).cuda()
    nq = q_raw.shape[0]
    qn = torch.empty_like(q_raw)
    oi = torch.empty(nq, dtype=torch.int64, device="cuda")
    os_ = torch.empty(nq, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    res = {}
    for name, kw in (("seeded", dict(proposal=prop, seed_topk=4)), ("plain", {})):
        def step():
            hn.normalize_async(q_raw, k, alpha, out=qn)
            return ix.search(qn, out_idx=oi, out_sim=os_, timing=True, **kw)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        barrier()
        ms, outs = _timed_steps(torch, stream, args.steps, step, flush)
        st = outs[-1].stats
        res[name] = {"queries_per_s": nq * args.steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / args.steps,
                     "survivor_frac": st["survivors"] / (nq * c["n"]),
                     "phases_ms": {kk: st[kk] for kk in ("ms_prep", "ms_phase1", "ms_threshold", "ms_phase2",
                                                         "ms_rescore")}}
        res[name + "_idx"] = oi.clone()
    same = bool(torch.equal(res.pop("seeded_idx"), res.pop("plain_idx")))
    if rank == 0:
        info = prop.info()
        line = {"metric": "exact 1-NN queries/s (learned block proposal seed)", "value": res["seeded"]["queries_per_s"],
                "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": res["seeded"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": f"c3: N={c['n']}, Q={nq}, K={k}, alpha={alpha}, {c['n_blocks']} blocks, "
                                       f"MLP {k}-256-256-{c['n_blocks']}, {c['n_train']} training pairs, top-4 seed"},
                "seeded": res["seeded"], "plain": res["plain"], "identical_results": same,
                "proposal": {"train_s": train_s, "final_loss": info["last_loss"], "steps": info["steps"],
                             "train_gemms": args.train_precision},
                "index_build_s": build_s}
        print(json.dumps(line), flush=True)
    prop.close()
    ix.close()
    return 0


def run_serving(args, hn, torch, world, rank, dist, barrier):
    """c4: 256 uneven batches over 16 indexes, one graph-replayed hn_search_multi per step."""
    cfg = hn_synth.SERVING
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    indexes, raws = [], []
    for di, n in enumerate(cfg["db_sizes"]):
        w = hn_synth.make_workload(n, 0, max(1, n // 5), seed=di + 1)
        raws.append(w.db_raw)
        raw_dev = torch.from_numpy(w.db_raw).cuda()
        for k in cfg["ks"]:
            for a in cfg["alphas"]:
                x = hn.normalize(raw_dev, k, a)
                indexes.append((hn.Index(x, k, a, prefix=hn.PREFIX_BF16), di, k, a))
                del x
        del raw_dev
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    sizes = hn_synth.log_uniform_sizes(cfg["seed"], cfg["n_batches"], cfg["min_batch"], cfg["max_batch"])
    pick = np.random.default_rng(cfg["seed"]).integers(0, len(indexes), cfg["n_batches"])
    batches, raw_q = [], []
    for b, (nq, g) in enumerate(zip(sizes, pick)):
        ix, di, k, a = indexes[g]
        qr, _ = hn_synth.queries_from(raws[di], int(nq), seed=10_000 + b)
        qd = torch.from_numpy(qr).cuda()
        raw_q.append((qd, k, a))
        batches.append((ix, torch.empty_like(qd), torch.empty(int(nq), dtype=torch.int64, device="cuda"),
                        torch.empty(int(nq), dtype=torch.float64, device="cuda")))
    total_q = int(sizes.sum())
    # the autotuner picks, per index, the dense/stream crossover and the dense work granularity
    # for the batch sizes it will see: a ladder up to its group's concatenated size
    tuned = []
    for g, (ix, di, k, a) in enumerate(indexes if not args.no_autotune else []):
        group_q = int(sizes[pick == g].sum())
        ladder = sorted({min(s_, ix.n) for s_ in (128, 512, 2048, max(group_q, 1))})
        r = ix.autotune(ladder)
        tuned.append({"n": ix.n, "k": k, "alpha": a, "group_queries": group_q, "dense_min_q": r["dense_min_q"],
                      "units_per_cta": r["units_per_cta"]})
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # queries reach a serving system already HN-normalised (HN is the descriptor
    # network's last layer): normalise once, then time the multi-batch search
    for (qd, k, a), (_, qn, _, _) in zip(raw_q, batches):
        hn.normalize(qd, k, a, out=qn)

    def step():
        return hn.search_multi(batches, use_graph=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0")), args.clock_log) as clocks:
        ms, outs = _timed_steps(torch, stream, args.steps, step, flush)
    st = outs[-1]
    if rank == 0:
        line = {"metric": "exact 1-NN queries/s (batched serving, 256 uneven batches, 16 indexes)",
                "value": world * total_q * args.steps / (sum(ms) / 1e3), "unit": "queries/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "data": "synthetic",
                "config": {"workload": "c4: 256 batches, sizes log-uniform 1..4096, databases N=100k/1M/4M/10M x "
                                       "K in {8,16} x alpha in {1/32,1/8}, BF16 prefix",
                           "queries_per_step": total_q, "n_indexes": len(indexes)},
                "graph_replayed": st["graph_replayed"], "groups": st["n_groups"],
                "groups_in_shared_scan": st["joined"],
                "batch_latency_ms": {"p50": st["batch_ms_p50"], "p99": st["batch_ms_p99"], "max": st["batch_ms_max"]},
                "search_multi_ms": st["ms_total"], "survivors": st["survivors"], "autotune": tuned,
                "note": "step = one hn_search_multi over all 256 batches (queries HN-normalised beforehand); "
                        "batch latency is measured from the start of the multi-search graph",
                "clocks": clocks.summary(), "index_build_s": build_s}
        print(json.dumps(line), flush=True)
    for ix, *_ in indexes:
        ix.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
