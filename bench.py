#!/usr/bin/env python3
"""All-pairs IBS benchmark: sample-pair x variant comparisons per second.

Default workload (the headline line): the structured cohort, n = 20,000
samples x m = 500,000 variants (Balding-Nichols five subpopulations, Fst
0.05; 200 parent-offspring pairs and 50 near-duplicates; 1% missing; seed 2),
synthetic, on one GB300.  One step = one ibs_compute call (transpose into
operand planes, the pair-count kernel with its fused epilogue, the split-tile
finalisation) over an input already resident in HBM, timed with CUDA events
on the launching stream; the planes (20 GB) exceed L2 many times over and a
256 MiB L2 flush still runs before every step.

The line carries:
  roofline      the pair kernel (CUDA events inside the library) against the
                tensor peak of its operand type (measured bf16 x nominal ratio);
  e2e           the same calls through the C ABI from pinned host memory,
                input copied in and counts and distances copied back every
                step, pipelined over copy-in, compute and copy-out streams;
  cpu_baseline  the CPU oracle on a bounded block (rows x 2,048 columns x all
                variants) on this machine's cores; the same block spot-checks
                the GPU result (`exact`);
  plain_config2 the plain n = 4,096 x m = 100,000 matrix;
  batched       64 cohort subsets of a 30,000 x 600,000 pool in one batched
                call against the plain path once per subset;
  served        the resident 100,000 x 200,000 panel, Poisson query arrivals,
                engine against one request at a time (p50/p99, throughput).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload structured|plain|batch|serve|ld|cluster|grm] [--no-sub]

With N > 1 (torchrun, one rank per GPU) every rank runs its own copy of the
workload (replicas; weak scaling) and rank 0 prints one JSON line; the
sub-records run at N = 1 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sample-pair×variant comparisons/s; served p50/p99 latency vs plain GPU path"
UNIT = "comparisons/s"
L2_FLUSH_BYTES = 256 << 20


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clk_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) == len(self.FIELDS):
                rows.append(parts)
        os.unlink(self.path)

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        smax = [num(r[1]) for r in rows if num(r[1]) is not None]
        power = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        loaded = [s for s in sm if smax and s > 0.3 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# integer-pipe roofline

def int_pipe_roofline(probe: dict, sm_mhz: float | None) -> dict:
    """Best comparisons per clock per SM over the two exact instruction mixes
    the pair loop can issue, from the measured per-SM pipe rates.

    Per pair and 32-marker word: plain = 3 POPC + 4 LOP3 + 1.5 IADD3;
    carry-save over 3 words = 2 POPC + 6 LOP3 + 2 adds.  LOP3 and the adds
    share the ALU pipe; POPC has its own.  Time per pair-word is the larger of
    the POPC time and the ALU time."""
    r_popc, r_lop, r_add = probe["popc_per_clk_sm"], probe["lop3_per_clk_sm"], probe["iadd3_per_clk_sm"]
    r_alu = min(r_lop, r_add)
    mixes = {"plain": (3.0, 4.0 + 1.5), "csa3": (2.0, 6.0 + 2.0)}
    best = {}
    for name, (popc, alu) in mixes.items():
        t = max(popc / r_popc, alu / r_alu)
        best[name] = 32.0 / t
    comps_clk_sm = max(best.values())
    mhz = sm_mhz or probe["sm_mhz"]
    return {"comps_per_clk_sm": comps_clk_sm, "by_mix": best, "sm_mhz": mhz,
            "peak": comps_clk_sm * probe["sms"] * mhz * 1e6}


def measured_peak(key: str, fallback: float) -> float:
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except Exception:
        return fallback


def hbm_peak_gbs() -> float:
    """Measured copy bandwidth of the GB300s; 6.8 TB/s fallback when absent."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def kernel_dtype(ibs, ctx) -> str:
    """Arithmetic of a context's pair kernel: indicator products in E2M1 or E4M3
    accumulated in FP32 (exact integer counts), or int32 for the integer form."""
    k = ibs.ibs_kernel_info(ctx)
    if k["family"] != "tensor-core":
        return "int32"
    return "e2m1xe2m1->f32" if k["tc_format"] == "e2m1" else "e4m3xe4m3->f32"


def kernel_source_hash(files=("ibs_pairs.cu", "ibs_device.cuh")) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1410_4803_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(name: str, files=("ibs_pairs.cu", "ibs_device.cuh")):
    """DRAM bytes per launch of the pair kernel from the committed ncu summary,
    or None when the summary is missing or the kernel source (`files`) changed
    since."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash(files):
        return None
    return float(m_bytes.group(1))


# ---------------------------------------------------------------------------
# CPU oracle baseline and spot check

def oracle_block_rate(packed, n, m, rows, cols, threads: int = 0):
    """Time the oracle on the block rows x cols of an n x m packed matrix (host
    numpy): unpack only those samples, then the plain per-marker loop.  Returns
    (counts [R][C][4], dist [R][C], comparisons/s, threads used, seconds)."""
    import numpy as np
    import oracle
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    GR = oracle.unpack_subset(packed, n, m, rows, 0, m)
    GC = oracle.unpack_subset(packed, n, m, cols, 0, m)
    used = threads if threads > 0 else (os.cpu_count() or 1)
    t = time.perf_counter()
    counts, dist = oracle.ibs_block(GR, GC, threads=threads)
    dt = time.perf_counter() - t
    return counts, dist, rows.size * cols.size * m / dt, used, dt


def calibrated_rows(packed, n, m, cols, target_s: float, threads: int = 0):
    """Rows (evenly spaced) for an oracle block of about target_s seconds."""
    import numpy as np
    probe = np.linspace(0, n - 1, max(1, min(n, threads if threads > 0 else (os.cpu_count() or 1)))).astype(np.int64)
    _, _, rate, _, _ = oracle_block_rate(packed, n, m, probe, cols[: max(1, min(len(cols), 256))], threads)
    R = int(max(1, min(n, target_s * rate / (len(cols) * m))))
    return np.linspace(0, n - 1, R).astype(np.int64)


def gpu_block(counts_dev, dist_dev, n, rows, cols):
    """Rows x cols of the device triangle (harness: gathered by torch indexing)."""
    import numpy as np
    import torch
    r = np.asarray(rows, dtype=np.int64)[:, None]
    c = np.asarray(cols, dtype=np.int64)[None, :]
    lo, hi = np.minimum(r, c), np.maximum(r, c)
    idx = torch.from_numpy((lo * n - lo * (lo - 1) // 2 + (hi - lo)).reshape(-1)).to(counts_dev.device)
    got_c = counts_dev.index_select(0, idx).cpu().numpy().reshape(r.shape[0], c.shape[1], 4)
    got_d = dist_dev.index_select(0, idx).cpu().numpy().reshape(r.shape[0], c.shape[1]) if dist_dev is not None else None
    return got_c, got_d


def same_block(got_c, got_d, want_c, want_d) -> bool:
    """Counts bit for bit; distances within 1e-12 relative, NaN in the same places."""
    import numpy as np
    if not np.array_equal(got_c, want_c):
        return False
    if got_d is None:
        return True
    nan_g, nan_w = np.isnan(got_d), np.isnan(want_d)
    if not np.array_equal(nan_g, nan_w):
        return False
    ok = ~nan_w
    rel = np.abs(got_d[ok] - want_d[ok]) / np.maximum(np.abs(want_d[ok]), 1e-300)
    return bool(rel.size == 0 or rel.max() <= 1e-12)


# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


WORKLOADS = {
    "plain": "plain n=4096 m=100000 (MAF U(0.01,0.5), 2% missing + 0.5% of variants at 30%), seed 1",
    "structured": "structured n=20000 m=500000 (Balding-Nichols, 5 subpopulations, Fst 0.05, ancestral MAF "
                  "U(0.02,0.5); 200 parent-offspring pairs, 50 duplicates at 0.1% discordance; 1% missing), seed 2",
}


def make_workload(name: str, device=None, samples: int = 0):
    """The named all-pairs workload; packed on `device` (torch) or on the host
    (numpy).  `samples` > 0 keeps the workload's recipe and marker count with
    fewer samples (a smaller case of the same kernel items, for profiling):
    plain takes that many samples; structured keeps its 200 offspring and 50
    duplicates and splits the rest evenly over the five subpopulations."""
    from paper_1410_4803_gb300 import synth
    if name == "plain":
        return synth.plain_config2(n=samples, device=device) if samples > 0 else synth.plain_config2(device=device)
    if name == "structured":
        if samples > 0:
            if samples < 255:
                raise ValueError("structured: --samples must be at least 255 (250 relatives + 5 base)")
            return synth.structured_config3(n_base_per_pop=(samples - 250) // 5, device=device)
        return synth.structured_config3(device=device)
    raise ValueError(name)


def workload_label(name: str, n: int, samples: int) -> str:
    """WORKLOADS[name], with the sample count replaced for a reduced case."""
    if samples <= 0:
        return WORKLOADS[name]
    return re.sub(r"n=\d+", f"n={n}", WORKLOADS[name], count=1) + " (reduced sample count, --samples)"


def run_matrix(args, rank, world, local, name: str, full: bool = True):
    """One all-pairs workload (ibs_compute: transpose + pair kernel + split-tile
    finalisation) over an input resident in HBM, timed per step with CUDA events
    on the launching stream; the pair kernel's own time from the library's
    events gives the roofline.  With `full`: the pipelined e2e through the
    same API from pinned host memory, the integer-pipe kernel on the same input,
    and the CPU oracle on a bounded block, which also spot-checks the GPU
    result (`exact`)."""
    import numpy as np
    import torch
    from paper_1410_4803_gb300 import ibs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    samples = getattr(args, "samples", 0) if full else 0
    w = make_workload(name, device=local, samples=samples)
    gen_s = time.perf_counter() - t0
    n, m = w.n, w.m
    comps = n * (n - 1) // 2 * m
    stream = torch.cuda.Stream(dev)
    packed = w.packed
    P = n * (n + 1) // 2
    counts = torch.empty((P, 4), dtype=torch.int32, device=dev)
    dist_t = torch.empty(P, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    # default: the tensor-core form; IBS_DEFAULT_KERNEL=popc times the bit-plane POPC kernel instead
    use_tc = os.environ.get("IBS_DEFAULT_KERNEL", "tc") != "popc"
    ctx = ibs.ibs_init(local, flags=ibs.IBS_TIMING | (ibs.IBS_KERNEL_TC if use_tc else ibs.IBS_KERNEL_CSA))
    probe = ibs.ibs_probe_int_pipes(ctx)
    kinfo = ibs.ibs_kernel_info(ctx)
    kname = ibs.ibs_compute_kernel(ctx, n, m)
    two_sm = use_tc and kname == "tc-pair"  # cta_group::2 kernel for long items
    mma_probe = ibs.ibs_probe_mma(ctx) if use_tc else None

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            ibs.ibs_compute(ctx, packed, n, m, counts, dist_t, stream)
        ibs.ibs_synchronize(ctx, stream)
        ibs.ibs_kernel_times(ctx)  # drop warm-up records
        launches_per_step = ibs.ibs_last_launch_info(ctx)["launches"]

        clk = ClockSampler(local)
        clk.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            ibs.ibs_compute(ctx, packed, n, m, counts, dist_t, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        wall = time.perf_counter() - t_wall
        clocks = clk.stop()
        ibs.ibs_synchronize(ctx, stream)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        kt = ibs.ibs_kernel_times(ctx)

        # end to end through the same API: pinned host input, results copied
        # back every step, pipelined over a copy-in, a compute and a copy-out
        # stream with two buffer sets, so that step i+1's input and step i-1's
        # results move while step i computes (the copy engines run both
        # directions at once).  The compute calls stay in order on one stream
        # and the L2 flush runs before each of them, inside the timed region.
        h_packed = packed.cpu().pin_memory()
        h_counts = [torch.empty((P, 4), dtype=torch.int32).pin_memory() for _ in range(2)]
        h_dist = [torch.empty(P, dtype=torch.float64).pin_memory() for _ in range(2)]
        d_in = [torch.empty_like(packed) for _ in range(2)]
        d_counts = [torch.empty_like(counts) for _ in range(2)]
        d_dist = [torch.empty_like(dist_t) for _ in range(2)]
        e2e_steps = max(3, args.steps)
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def pipeline(steps):
            """`steps` pipelined e2e steps; ms per step between the first
            copy-in's start and the last copy-out's end."""
            in_ready = [torch.cuda.Event() for _ in range(steps)]
            comp_done = [torch.cuda.Event() for _ in range(steps)]
            out_done = [torch.cuda.Event() for _ in range(steps)]
            t0_ev, t1_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            t0_ev.record(s_in)
            stream.wait_event(t0_ev)
            for i in range(steps):
                b = i % 2
                if i >= 2:
                    s_in.wait_event(comp_done[i - 2])  # compute i-2 has read d_in[b]
                with torch.cuda.stream(s_in):
                    d_in[b].copy_(h_packed, non_blocking=True)
                in_ready[i].record(s_in)
                stream.wait_event(in_ready[i])
                if i >= 2:
                    stream.wait_event(out_done[i - 2])  # results i-2 have left d_counts[b]
                flush.zero_()
                ibs.ibs_compute(ctx, d_in[b], n, m, d_counts[b], d_dist[b], stream)
                comp_done[i].record(stream)
                s_out.wait_event(comp_done[i])
                with torch.cuda.stream(s_out):
                    h_counts[b].copy_(d_counts[b], non_blocking=True)
                    h_dist[b].copy_(d_dist[b], non_blocking=True)
                out_done[i].record(s_out)
            t1_ev.record(s_out)
            torch.cuda.synchronize(dev)
            ibs.ibs_synchronize(ctx, stream)
            return t0_ev.elapsed_time(t1_ev) / steps

        # warm-up steps of the same pipeline, untimed: freshly pinned host
        # buffers were measured slow on their first copies (172.8 against
        # 151.4 ms per step for the same 10 steps run twice)
        pipeline(max(2, min(args.warmup, 3)))
        e2e_ms = pipeline(e2e_steps)
        ibs.ibs_kernel_times(ctx)
        last = (e2e_steps - 1) % 2
        e2e_same = bool(torch.equal(d_counts[last], counts))
        del d_in, d_counts, d_dist, h_counts, h_dist

        # The integer-pipe kernel (bit planes, carry-save LOP3/POPC) on the same
        # input: its fraction of the integer-pipe roofline.
        popc = None
        if use_tc and full:
            ctx_i = ibs.ibs_init(local, flags=ibs.IBS_TIMING | ibs.IBS_KERNEL_CSA)
            k_i = 2 if comps > 1e13 else max(1, min(args.steps, 10))
            tmp_c = torch.empty_like(counts)
            ibs.ibs_compute(ctx_i, packed, n, m, tmp_c, None, stream)
            ibs.ibs_synchronize(ctx_i, stream)
            ibs.ibs_kernel_times(ctx_i)
            for _ in range(k_i):
                flush.zero_()
                ibs.ibs_compute(ctx_i, packed, n, m, tmp_c, None, stream)
            ibs.ibs_synchronize(ctx_i, stream)
            kt_i = ibs.ibs_kernel_times(ctx_i)
            popc_same = bool(torch.equal(tmp_c, counts))
            ibs.ibs_shutdown(ctx_i)
            del tmp_c
            popc = kt_i["pairs_ms"] / max(1, kt_i["calls"])

    total_ms = reduce_max(sum(step_ms), world)
    e2e_total = reduce_max(e2e_ms, world)
    ms_per_step = total_ms / args.steps
    pairs_ms = kt["pairs_ms"] / max(1, kt["calls"])
    planes_ms = kt["planes_ms"] / max(1, kt["calls"])
    finalize_ms = kt["finalize_ms"] / max(1, kt["calls"])
    roof = int_pipe_roofline(probe, clocks.get("sm_mhz"))
    achieved = comps / (pairs_ms * 1e-3)
    fp4 = use_tc and kinfo["tc_format"] == "e2m1"
    if use_tc:
        # tensor peak of the operand type: the measured bf16 burst rate x the nominal
        # dense ratio (FP8 4.5 / bf16 2.25 = 2; FP4 13.5 / 2.25 = 6); 4 MACs = 8 flops
        # per comparison.
        tc_ratio = 6.0 if fp4 else 2.0
        tc_tflops = tc_ratio * measured_peak("bf16_tflops", 1900.0)
    mode = {"0": "plain", "1": "csa3", "2": "csa3-1cta"}.get(os.environ.get("IBS_PAIR_MODE", "1"), "csa3")
    if use_tc:
        mode = "tc-fp4" if fp4 else "tc-fp8"
    # transpose: read the 2-bit input once, write the operand planes (4 planes of one
    # byte (FP8) or half a byte (FP4) per padded genotype)
    k = 64 if fp4 else 32
    transpose_bytes = m * ((n + 3) // 4) + ((n + 127) // 128) * 128 * ((m + k - 1) // k) * k * 4 // (2 if fp4 else 1)
    profile = f"{'tc_pair_kernel' if two_sm else 'tc_kernel_fp4' if fp4 else 'tc_kernel_fp8'}_{name}.md"

    # oracle block: the CPU baseline and the spot check of the last result
    exact = None
    cpu = None
    if rank == 0 and full:
        h = h_packed.numpy()
        cols = np.linspace(0, n - 1, min(n, 2048)).astype(np.int64)
        rows = calibrated_rows(h, n, m, cols, args.cpu_seconds)
        if name == "structured":  # every injected offspring and duplicate among the rows
            rel = np.flatnonzero(w.samples.kind != 0)
            rows = np.unique(np.concatenate([rows, rel[:: max(1, rel.size // 16)]]))
        want_c, want_d, rate, cores, dt = oracle_block_rate(h, n, m, rows, cols)
        got_c, got_d = gpu_block(counts, dist_t, n, rows, cols)
        exact = {"oracle_block": same_block(got_c, got_d, want_c, want_d),
                 "oracle_block_shape": f"{rows.size} rows x {cols.size} columns x all {m} variants",
                 "e2e_equals_resident": e2e_same}
        if popc is not None:
            exact["integer_kernel_equals_tensor_core"] = popc_same
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{rows.size} rows x {cols.size} columns (evenly spaced) x all {m} variants ({dt:.1f} s)"}
        r1 = rows[:: max(1, rows.size // 4)][:4]
        _, _, rate1, _, dt1 = oracle_block_rate(h, n, m, r1, cols[: 1024], threads=1)
        cpu1 = {"value": rate1, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"{r1.size} rows x 1024 columns x all {m} variants ({dt1:.1f} s)"}
    ibs.ibs_shutdown(ctx)
    del counts, dist_t, packed, w
    torch.cuda.empty_cache()

    if rank != 0:
        return None
    line = {
        "metric": METRIC,
        "value": world * comps / (total_ms / args.steps * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        # arithmetic of the pair kernel: E2M1 (or E4M3) indicator products accumulated
        # in FP32, exact integer counts; the integer form computes in int32
        "dtype": ("e2m1xe2m1->f32" if fp4 else "e4m3xe4m3->f32") if use_tc else "int32",
        "data": "synthetic",
        "config": {"workload": workload_label(name, n, samples), "n_samples": n, "n_variants": m,
                   "pairs_incl_diagonal": P,
                   "comparisons_per_step": comps,
                   "l2": "flushed between steps (256 MiB write, outside the step events); the operand planes "
                         f"({tc_planes_gb(n, m, fp4):.1f} GB) exceed L2 many times over",
                   "parallelism": f"replicas x{world}", "kernel_mode": mode, "pair_kernel": kname,
                   "input_generation_s": gen_s},
        "roofline": ({"bound": "alu", "achieved": achieved, "peak": roof["peak"], "unit": UNIT,
                      "frac": achieved / roof["peak"],
                      "traffic": profiled_traffic(f"popc_tri_kernel_{name}.md"),
                      "kernel": "tri_kernel (pair counts)", "kernel_ms": pairs_ms,
                      "peak_basis": f"{roof['comps_per_clk_sm']:.1f} comparisons/clk/SM x {probe['sms']} SMs x "
                                    f"{roof['sm_mhz']:.0f} MHz (median SM clock in the timed region); pipe rates "
                                    f"measured live: POPC {probe['popc_per_clk_sm']:.2f}, LOP3 "
                                    f"{probe['lop3_per_clk_sm']:.2f}, IADD3 {probe['iadd3_per_clk_sm']:.2f} /clk/SM"}
                     if not use_tc else
                     {"bound": "tensor", "achieved": 8.0 * achieved / 1e12, "peak": tc_tflops, "unit": "TFLOP/s",
                      "frac": 8.0 * achieved / 1e12 / tc_tflops,
                      "traffic": profiled_traffic(profile, ("ibs_tc.cu", "ibs_device.cuh", "ibs_tc_common.cuh")),
                      "kernel": ("tc_pair_kernel (tcgen05 cta_group::2, M = 256 over two SMs, E2M1 kind::mxf4 "
                                 "indicator GEMMs)" if two_sm else
                                 f"tc_persistent_kernel (tcgen05 {'E2M1 kind::mxf4' if fp4 else 'E4M3 kind::f8f6f4'} "
                                 f"indicator GEMMs)"), "kernel_ms": pairs_ms,
                      "peak_basis": f"measured bf16 burst TFLOP/s (MEASURED_PEAKS.json) x {tc_ratio:.0f}, the nominal "
                                    f"{'FP4' if fp4 else 'FP8'}/bf16 dense ratio (of measured); algorithmic flops = 8 "
                                    "per comparison (4 MACs: VV^T, UU^T, QR^T, RQ^T); achieved = that work / the pair "
                                    "kernel's CUDA-event time per call",
                      "mma_probe": {"unit": "TFLOP/s",
                                    "measured": mma_probe["e2m1_tflops" if fp4 else "e4m3_tflops"],
                                    "frac": 8.0 * achieved / 1e12 / mma_probe["e2m1_tflops" if fp4 else "e4m3_tflops"],
                                    "basis": "ibs_probe_mma: back-to-back 128x128 MMAs of this kind from "
                                             "shared-memory tiles on all SMs, measured live"}}),
        "integer_kernel": None if popc is None else {
            "kernel": "tri_kernel, carry-save LOP3/POPC over bit planes (IBS_KERNEL_CSA)",
            "kernel_ms": popc, "value": comps / (popc * 1e-3), "unit": UNIT,
            "roofline_peak": roof["peak"], "frac": comps / (popc * 1e-3) / roof["peak"],
            "peak_basis": "integer-pipe roofline (measured pipe rates x SMs x clock)"},
        "transpose": {"kernel_ms": planes_ms, "bytes": transpose_bytes,
                      "achieved_gbs": transpose_bytes / (planes_ms * 1e-3) / 1e9,
                      "peak_gbs": hbm_peak_gbs(), "frac": transpose_bytes / (planes_ms * 1e-3) / 1e9 / hbm_peak_gbs()},
        "finalize_ms": finalize_ms,
        "e2e": {"value": world * comps / (e2e_total * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(n // 4 * m if n % 4 == 0 else (n + 3) // 4 * m),
                "d2h_bytes_per_step": int(P * 16 + P * 8), "steps": e2e_steps,
                "pipelined": "copy-in, compute and copy-out streams, two buffer sets; the fill and drain of the "
                             "pipeline are inside the timed region"},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    if exact is not None:
        line["exact"] = exact
    if cpu is not None:
        line["cpu_baseline"] = cpu
        line["cpu_baseline_1core"] = cpu1
    return line


def tc_planes_gb(n, m, fp4=True):
    k = 64 if fp4 else 32
    return ((n + 127) // 128) * 128 * ((m + k - 1) // k) * k * 4 / (2 if fp4 else 1) / 1e9


def run_reference(args, rank, world, local):
    """The oracle arm: the CPU oracle as it stands, on this machine's host cores,
    each step a bounded block of the same workload (rows x evenly spaced
    columns x all variants; only those samples are generated and unpacked)."""
    if rank != 0:
        return None
    import numpy as np
    from paper_1410_4803_gb300 import synth
    name = args.workload if args.workload in WORKLOADS else "structured"
    if name == "plain":
        model = synth.plain_model(100_000, 1, maf=(0.01, 0.5), miss=0.02, hi_miss_frac=0.005, hi_miss_rate=0.3)
        smp = synth.Samples.base(4096)
    else:
        model = synth.balding_nichols_model(500_000, 2, n_pop=5, fst=0.05, anc=(0.02, 0.5), miss=0.01)
        smp = synth.structured_samples(3950 * 5, 5, 200, 50, 2)
    n, m = smp.n, model.m
    cols = np.linspace(0, n - 1, min(n, 2048)).astype(np.int64)
    cores = os.cpu_count() or 1
    # size a step at about args.ref_step_seconds from a calibration block
    probe_rows = np.linspace(0, n - 1, min(n, cores)).astype(np.int64)
    sel = np.unique(np.concatenate([cols, probe_rows]))
    packed = synth.generate(model, smp.take(sel))  # only the sampled samples
    pos = {int(v): i for i, v in enumerate(sel)}
    cidx = np.array([pos[int(v)] for v in cols])
    pidx = np.array([pos[int(v)] for v in probe_rows])
    _, _, rate, _, _ = oracle_block_rate(packed, sel.size, m, pidx, cidx[:256])
    R = int(max(1, min(n, args.ref_step_seconds * rate / (cols.size * m))))
    rows = np.linspace(0, n - 1, R).astype(np.int64)
    sel = np.unique(np.concatenate([cols, rows]))
    packed = synth.generate(model, smp.take(sel))
    pos = {int(v): i for i, v in enumerate(sel)}
    cidx = np.array([pos[int(v)] for v in cols])
    ridx = np.array([pos[int(v)] for v in rows])
    for _ in range(args.warmup):
        oracle_block_rate(packed, sel.size, m, ridx[: max(1, R // 4)], cidx)
    times = []
    for _ in range(args.steps):
        _, _, _, _, dt = oracle_block_rate(packed, sel.size, m, ridx, cidx)
        times.append(dt)
    comps = R * cols.size * m
    value = comps / statistics.mean(times)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOADS[name], "n_samples": n, "n_variants": m,
                   "sample_per_step": f"{R} rows x {cols.size} columns (evenly spaced) x all {m} variants"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{R} rows x {cols.size} columns x all {m} variants per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def subset_packed_device(pool_dev, idx_dev, vb: int, vl: int):
    """Harness input preparation: the packed .bed matrix of one subset
    (samples idx, markers [vb, vb+vl)) gathered from the pool on the device."""
    import torch
    rows = pool_dev[vb:vb + vl]
    byte = rows.index_select(1, idx_dev // 4)
    shift = (2 * (idx_dev % 4)).to(torch.uint8)
    code = (byte >> shift) & 3
    pad = (-idx_dev.numel()) % 4
    if pad:
        code = torch.nn.functional.pad(code, (0, pad))
    code = code.view(vl, -1, 4)
    return (code[..., 0] | (code[..., 1] << 2) | (code[..., 2] << 4) | (code[..., 3] << 6)).contiguous()


def run_batch(args, rank, world, local):
    """64 cohort subsets of a 30,000 x 600,000 pool: one batched call (gather
    transpose from the pool and persistent pair launches in stages, graph-captured,
    autotuned) against the plain path run once per subset."""
    import numpy as np
    import torch
    import oracle
    from paper_1410_4803_gb300 import ibs, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    w = synth.batch_pool(device=local)
    subs = synth.batch_subsets()
    gen_s = time.perf_counter() - t0
    pool = w.packed
    comps = sum(s.comparisons for s in subs)
    stream = torch.cuda.Stream(dev)
    args_b, plain_in, outs_b, outs_p = [], [], [], []
    for s in subs:
        idx = torch.from_numpy(s.sample_idx).to(dev)
        P = s.n * (s.n + 1) // 2
        cb = torch.empty((P, 4), dtype=torch.int32, device=dev)
        db = torch.empty(P, dtype=torch.float64, device=dev)
        args_b.append((idx, s.var_begin, s.var_len, cb, db))
        outs_b.append((cb, db))
        plain_in.append(subset_packed_device(pool, idx, s.var_begin, s.var_len))
        outs_p.append((torch.empty((P, 4), dtype=torch.int32, device=dev),
                       torch.empty(P, dtype=torch.float64, device=dev)))
    torch.cuda.synchronize(dev)
    tune_path = os.path.join(tempfile.gettempdir(), f"ibs_tune_{os.getpid()}.jsonl")
    ctx_b = ibs.ibs_init(local, autotune_cache_path=tune_path)
    ctx_p = ibs.ibs_init(local, flags=ibs.IBS_TIMING)
    with torch.cuda.stream(stream):
        t = time.perf_counter()
        ibs.ibs_compute_batch(ctx_b, pool, w.n, w.m, args_b, stream)  # plan, autotune, graph capture
        ibs.ibs_synchronize(ctx_b, stream)
        first_call_s = time.perf_counter() - t
        plan = ibs.ibs_batch_plan_info(ctx_b)

        def timed(fn, k):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
            for i in range(k):
                ev[i][0].record(stream)
                fn()
                ev[i][1].record(stream)
            torch.cuda.synchronize(dev)
            return [a.elapsed_time(b) for a, b in ev]

        def batched():
            ibs.ibs_compute_batch(ctx_b, pool, w.n, w.m, args_b, stream)

        def plain_loop():
            for s, pk, (c, d) in zip(subs, plain_in, outs_p):
                ibs.ibs_compute(ctx_p, pk, s.n, s.var_len, c, d, stream)

        for _ in range(args.warmup):
            batched()
            plain_loop()
        torch.cuda.synchronize(dev)
        batched()
        launches_b = ibs.ibs_last_launch_info(ctx_b)["launches"]
        launches_p = 0
        for s, pk, (c, d) in zip(subs, plain_in, outs_p):
            ibs.ibs_compute(ctx_p, pk, s.n, s.var_len, c, d, stream)
            launches_p += ibs.ibs_last_launch_info(ctx_p)["launches"]
        torch.cuda.synchronize(dev)
        ibs.ibs_kernel_times(ctx_p)  # drop warm-up records
        clk = ClockSampler(local)
        clk.start()
        ms_b = timed(batched, args.steps)
        ms_p = timed(plain_loop, args.steps)
        kt_p = ibs.ibs_kernel_times(ctx_p)  # the plain loop's kernels only
        clocks = clk.stop()
        ibs.ibs_synchronize(ctx_b, stream)
        ibs.ibs_synchronize(ctx_p, stream)
    # exactness: every subset, batched vs plain, bit for bit; sampled pairs vs the oracle
    same = all(torch.equal(a[0], b[0]) and torch.equal(torch.nan_to_num(a[1], nan=-1.0),
                                                        torch.nan_to_num(b[1], nan=-1.0))
               for a, b in zip(outs_b, outs_p))
    rng = np.random.default_rng(0)
    oracle_ok = True
    pool_host = pool.cpu().numpy()
    for k in rng.choice(len(subs), 4, replace=False):
        s = subs[k]
        rows = np.sort(rng.choice(s.n, min(s.n, 24), replace=False))
        G = oracle.unpack_subset(pool_host, w.n, w.m, s.sample_idx[rows], s.var_begin, s.var_len)
        oc, _ = oracle.ibs_block(G, G)
        got = outs_b[k][0].cpu().numpy()
        for a in range(rows.size):
            for b in range(a, rows.size):
                if (got[oracle.tri_index(rows[a], rows[b], s.n)] != oc[a, b]).any():
                    oracle_ok = False
    dtype_b = kernel_dtype(ibs, ctx_b)
    ibs.ibs_shutdown(ctx_b)
    ibs.ibs_shutdown(ctx_p)
    mb, mp = statistics.mean(ms_b), statistics.mean(ms_p)
    return {
        "metric": METRIC, "value": comps / (mb * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mb, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_b, "data": "synthetic",
        "config": {"workload": f"batched: {len(subs)} subsets of pool n={w.n} m={w.m} "
                               f"(n ~ U[200, 8000], windows ~ U[10k, 200k]), seed 3",
                   "comparisons_per_step": comps, "plan": plan, "first_call_s_incl_autotune": first_call_s,
                   "generation_s": gen_s},
        "plain_loop": {"value": comps / (mp * 1e-3), "ms_per_step": mp, "launches_per_step": launches_p,
                       "transpose_ms_per_step": kt_p["planes_ms"] / args.steps,
                       "pair_kernel_ms_per_step": kt_p["pairs_ms"] / args.steps,
                       "finalize_ms_per_step": kt_p["finalize_ms"] / args.steps},
        "speedup_vs_plain_loop": mp / mb,
        "exact": {"batched_equals_plain_all_subsets": bool(same), "oracle_sampled_pairs": bool(oracle_ok)},
        "gpu_launches": int(args.steps * launches_b),
        "clocks": clocks,
    }


def run_serve(args, rank, world, local):
    """Resident 100,000 x 200,000 panel; Poisson arrivals of 1-512-sample
    query requests.  The engine (continuous batching) against the plain path
    (one request at a time through ibs_query_sync), same arrivals."""
    import threading
    import numpy as np
    import torch
    from paper_1410_4803_gb300 import ibs, synth

    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    samples = getattr(args, "samples", 0)
    if samples > 0:
        # a smaller panel for profiling captures: the same recipe and markers,
        # its 1,000 offspring and 250 duplicates, fewer base samples
        if samples < 1255:
            raise ValueError("serve: --samples must be at least 1,255 (1,250 relatives + 5 base)")
        panel = synth.serving_panel(n_base_per_pop=(samples - 1250) // 5, device=local)
    else:
        panel = synth.serving_panel(device=local)
    gen_s = time.perf_counter() - t0
    n_payload = 48
    sizes = synth.serving_query_sizes(n_payload)
    payloads = [synth.serving_queries(panel, int(q), request_id=i)[0] for i, q in enumerate(sizes)]
    k = 16
    bufs = [(torch.empty((int(q), panel.n, 4), dtype=torch.int32).pin_memory(),
             torch.empty((int(q), k), dtype=torch.int32).pin_memory(),
             torch.empty((int(q), k), dtype=torch.float64).pin_memory()) for q in sizes]
    # every request buffer copied into once before any timing (freshly pinned
    # host memory was measured slow on its first copies)
    with torch.no_grad():
        warm = torch.zeros(max(b[0].numel() for b in bufs), dtype=torch.int32, device=local)
        for b in bufs:
            for x in b:
                flat = x.view(-1)
                flat.copy_(warm[:flat.numel()].view(flat.dtype) if flat.dtype == torch.int32 else
                           warm[:flat.numel()].to(flat.dtype))
        torch.cuda.synchronize(local)
        del warm
    ctx = ibs.ibs_init(local)
    t = time.perf_counter()
    ibs.ibs_panel_load(ctx, panel.packed, panel.n, panel.m)
    load_s = time.perf_counter() - t
    # oracle spot check later: two query rows against 4,096 evenly spaced panel samples
    check_cols = np.linspace(0, panel.n - 1, 4096).astype(np.int64)
    # the oracle check's panel samples only (a 4,096-sample .bed matrix, 205 MB), taken on the device
    check_packed = subset_packed_device(panel.packed, torch.from_numpy(check_cols).to(panel.packed.device), 0,
                                        panel.m).cpu().numpy()
    panel.packed = None  # the library holds its own planes of the panel
    torch.cuda.empty_cache()

    def comps_of(i):
        return int(sizes[i]) * panel.n * panel.m

    def run_engine(arrivals):
        ids = [None] * len(arrivals)
        done = [0.0] * len(arrivals)
        start = time.perf_counter()

        def waiter():
            for i in range(len(arrivals)):
                while ids[i] is None:
                    time.sleep(0.0002)
                ibs.ibs_wait(ctx, ids[i], timeout_ms=600000)
                done[i] = time.perf_counter() - start
        th = threading.Thread(target=waiter)
        th.start()
        for i, ta in enumerate(arrivals):
            now = time.perf_counter() - start
            if ta > now:
                time.sleep(ta - now)
            p = i % n_payload
            ids[i] = ibs.ibs_query(ctx, payloads[p], int(sizes[p]), k, *bufs[p])
        th.join()
        return done

    def run_plain(arrivals):
        done = [0.0] * len(arrivals)
        start = time.perf_counter()
        for i, ta in enumerate(arrivals):
            now = time.perf_counter() - start
            if ta > now:
                time.sleep(ta - now)
            p = i % n_payload
            ibs.ibs_query_sync(ctx, payloads[p], int(sizes[p]), k, *bufs[p])
            done[i] = time.perf_counter() - start
        return done

    def summarize(arrivals, done):
        lat = np.array(done) - np.array(arrivals)
        total = sum(comps_of(i % n_payload) for i in range(len(arrivals)))
        span = max(done) - min(arrivals)
        return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "throughput": total / span, "requests": len(arrivals)}

    # warm-up both paths (the exactness checks run after the timed runs, so
    # that the CPU oracle does not run just before them)
    run_engine([0.0] * 4)
    run_plain([0.0] * 2)
    rng = np.random.default_rng(4)
    results = []
    clk = ClockSampler(local)
    clk.start()
    for lam in args.rates:
        n_req = args.requests
        if lam > 0:
            arrivals = list(np.cumsum(rng.exponential(1.0 / lam, n_req)))
        else:
            arrivals = [0.0] * n_req  # saturation: everything arrives at once
        eng = summarize(arrivals, run_engine(arrivals))
        pln = summarize(arrivals, run_plain(arrivals))
        results.append({"lambda_per_s": lam if lam > 0 else "saturation", "engine": eng, "plain": pln})
    clocks = clk.stop()
    # Context for the saturation figures, which depend on the host: the
    # device -> host rate into these pinned request buffers (it varied between
    # processes on the same kind of box), and the engine at saturation with
    # device-resident outputs (no host copies at all).
    host_flat = bufs[0][0].view(-1)
    probe = torch.empty(host_flat.numel(), dtype=torch.int32, device=local)
    for _ in range(2):
        host_flat.copy_(probe)
    torch.cuda.synchronize(local)
    t = time.perf_counter()
    for _ in range(3):
        host_flat.copy_(probe)
    torch.cuda.synchronize(local)
    host_gbs = 3 * probe.numel() * 4 / (time.perf_counter() - t) / 1e9
    del probe
    dev_bufs = [(torch.empty((int(q), panel.n, 4), dtype=torch.int32, device=local),
                 torch.empty((int(q), k), dtype=torch.int32, device=local),
                 torch.empty((int(q), k), dtype=torch.float64, device=local)) for q in sizes]
    host_bufs, bufs = bufs, dev_bufs
    run_engine([0.0] * n_payload)  # first use of the device buffers
    dev_sat = summarize([0.0] * n_payload, run_engine([0.0] * n_payload))
    bufs = host_bufs
    del dev_bufs
    # exactness: a few requests, engine vs plain, bit for bit; the first
    # request's first and last rows against the oracle on 4,096 panel samples
    exact = True
    oracle_ok = False
    for p in range(3):
        q = int(sizes[p])
        a = [torch.empty((q, panel.n, 4), dtype=torch.int32).pin_memory(),
             torch.empty((q, k), dtype=torch.int32).pin_memory(),
             torch.empty((q, k), dtype=torch.float64).pin_memory()]
        b = [torch.empty_like(x).pin_memory() for x in a]
        rid = ibs.ibs_query(ctx, payloads[p], q, k, *a)
        ibs.ibs_wait(ctx, rid, timeout_ms=600000)
        ibs.ibs_query_sync(ctx, payloads[p], q, k, *b)
        exact &= all(torch.equal(x, y) for x, y in zip(a[:2], b[:2]))
        exact &= torch.equal(torch.nan_to_num(a[2], nan=-1.0), torch.nan_to_num(b[2], nan=-1.0))
        if p == 0:
            import oracle
            qrows = np.array([0, q - 1], dtype=np.int64)
            GQ = oracle.unpack_subset(payloads[0], q, panel.m, qrows, 0, panel.m)
            GP = oracle.unpack(check_packed, check_cols.size, panel.m)
            want_c, _ = oracle.ibs_block(GQ, GP)
            oracle_ok = bool(np.array_equal(a[0].numpy()[qrows][:, check_cols], want_c))
    del check_packed
    stats = ibs.ibs_serve_stats_get(ctx)
    dtype_s = kernel_dtype(ibs, ctx)
    ibs.ibs_shutdown(ctx)
    sat = [r for r in results if r["lambda_per_s"] == "saturation"]
    head = sat[0] if sat else results[-1]
    return {
        "metric": METRIC, "value": head["engine"]["throughput"], "unit": UNIT, "n_gpus": 1,
        "steps": len(results), "warmup": 1, "ms_per_step": head["engine"]["mean_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_s, "data": "synthetic",
        "config": {"workload": f"serving: panel n={panel.n} m={panel.m} resident; requests of q = "
                               f"floor(exp(U(0, ln 512))) + 1 samples, Poisson arrivals; counts [q][n][4] and "
                               f"top-{k} to pinned host buffers", "distinct_payloads": n_payload,
                   "mean_q": float(np.mean(sizes)), "panel_generation_s": gen_s, "panel_load_s": load_s},
        "serving": results, "engine_stats": stats,
        "host_context": {"d2h_gbs_into_request_buffers": host_gbs,
                         "engine_saturation_device_outputs": dev_sat},
        "exact": {"engine_equals_plain": bool(exact),
                  "oracle_two_query_rows_x_4096_panel_samples": oracle_ok},
        "clocks": clocks,
    }


def run_ld(args, rank, world, local):
    """LD correlation r of every marker pair within a window (paper, "Bitwise
    parallelism", r with missing calls) on the plain workload's genotypes:
    n = 4,096 samples, m = 100,000 markers.  Unit: marker pair x sample."""
    import numpy as np
    import torch
    import oracle
    from paper_1410_4803_gb300 import ibs

    torch.cuda.set_device(local)
    w = make_workload("plain")
    n, m, W = w.n, w.m, args.window
    pairs = m * W - W * (W + 1) // 2 if W < m else m * (m - 1) // 2
    comps = pairs * n
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    packed = torch.from_numpy(w.packed).to(dev)
    r = torch.empty((m, W), dtype=torch.float64, device=dev)
    cnt = torch.empty((m, W), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ctx = ibs.ibs_init(local)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ibs.ibs_ld_r(ctx, packed, n, m, W, r, cnt, stream)
        ibs.ibs_synchronize(ctx, stream)
        launches = ibs.ibs_last_launch_info(ctx)["launches"]
        clk = ClockSampler(local)
        clk.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            ibs.ibs_ld_r(ctx, packed, n, m, W, r, cnt, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        clocks = clk.stop()
        ibs.ibs_synchronize(ctx, stream)
        ms = [a.elapsed_time(b) for a, b in ev]
        # end to end: pinned host input, r and N copied back each step
        h_in = torch.from_numpy(w.packed).pin_memory()
        h_r = torch.empty((m, W), dtype=torch.float64).pin_memory()
        h_n = torch.empty((m, W), dtype=torch.int32).pin_memory()
        d_in = torch.empty_like(packed)
        e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            e2e_ev[i][0].record(stream)
            d_in.copy_(h_in, non_blocking=True)
            ibs.ibs_ld_r(ctx, d_in, n, m, W, r, cnt, stream)
            h_r.copy_(r, non_blocking=True)
            h_n.copy_(cnt, non_blocking=True)
            e2e_ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = [a.elapsed_time(b) for a, b in e2e_ev]
    # spot check against the oracle on a marker range
    G = oracle.unpack(w.packed, n, m)
    lo, hi = 50_000, 50_000 + 64
    want_r, want_n = oracle.ld_r(np.ascontiguousarray(G[:, lo:hi + W]), W)
    got_r, got_n = r[lo:hi].cpu().numpy(), cnt[lo:hi].cpu().numpy()
    ok = bool((got_n == want_n[:hi - lo]).all()) and bool(
        np.allclose(got_r, want_r[:hi - lo], rtol=1e-12, atol=0, equal_nan=True))
    ibs.ibs_shutdown(ctx)
    mean_ms = statistics.mean(ms)
    line = {
        "metric": "marker-pair x sample comparisons/s (LD r within a window)", "value": comps / (mean_ms * 1e-3),
        "unit": "comparisons/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "e2m1xe2m1->f32",
        "data": "synthetic",
        "config": {"workload": f"LD r, plain workload genotypes n={n} m={m}, window {W}", "pairs": pairs,
                   "l2": "flushed between steps (256 MiB write, outside the step events)"},
        "e2e": {"value": comps / (statistics.mean(e2e_ms) * 1e-3), "unit": "comparisons/s",
                "h2d_bytes_per_step": int(w.packed.nbytes), "d2h_bytes_per_step": int(m * W * 12)},
        "exact": {"oracle_markers_50000_50063": ok},
        "gpu_launches": int(launches * args.steps),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        t = time.perf_counter()
        Gs = np.ascontiguousarray(G[:, :10_000 + W])
        oracle.ld_r(Gs, W)
        dt = time.perf_counter() - t
        sample_pairs = sum(min(W, Gs.shape[1] - 1 - a) for a in range(Gs.shape[1]))
        line["cpu_baseline"] = {"value": sample_pairs * n / dt, "unit": "comparisons/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": f"markers 0..{Gs.shape[1] - 1} (all their pairs within the "
                                                            f"window) x {n} samples ({dt:.1f} s)"}
    return line


def run_grm(args, rank, world, local):
    """GCTA genomic relationship matrix (paper, "Partial sum lookup") of the
    plain workload's genotypes, n = 4,096 samples x m = 100,000 markers, on the
    tensor cores (FP16 hi/lo operands, FP32 segments, float-float sums).
    Unit: sample pair (with the diagonal) x marker."""
    import numpy as np
    import torch
    import oracle
    from paper_1410_4803_gb300 import ibs

    torch.cuda.set_device(local)
    from paper_1410_4803_gb300 import synth
    w = synth.plain_config2(m=args.markers)
    n, m = w.n, w.m
    P = n * (n + 1) // 2
    comps = P * m
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    packed = torch.from_numpy(w.packed).to(dev)
    out = torch.empty(P, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ctx = ibs.ibs_init(local)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ibs.ibs_grm(ctx, packed, n, m, out, stream)
        ibs.ibs_synchronize(ctx, stream)
        launches = ibs.ibs_last_launch_info(ctx)["launches"]
        clk = ClockSampler(local)
        clk.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            ibs.ibs_grm(ctx, packed, n, m, out, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        clocks = clk.stop()
        ibs.ibs_synchronize(ctx, stream)
        ms = [a.elapsed_time(b) for a, b in ev]
        # end to end: pinned host input, the matrix copied back each step,
        # pipelined as in the plain workload (copy-in, compute and copy-out
        # streams, two buffer sets; the compute calls in order on one stream)
        h_in = torch.from_numpy(w.packed).pin_memory()
        h_out = [torch.empty(P, dtype=torch.float64).pin_memory() for _ in range(2)]
        d_in = [torch.empty_like(packed) for _ in range(2)]
        d_out = [out, torch.empty_like(out)]
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        in_ready = [torch.cuda.Event() for _ in range(args.steps)]
        comp_done = [torch.cuda.Event() for _ in range(args.steps)]
        out_done = [torch.cuda.Event() for _ in range(args.steps)]
        t0_ev, t1_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t0_ev.record(s_in)
        stream.wait_event(t0_ev)
        for i in range(args.steps):
            b = i % 2
            if i >= 2:
                s_in.wait_event(comp_done[i - 2])
            with torch.cuda.stream(s_in):
                d_in[b].copy_(h_in, non_blocking=True)
            in_ready[i].record(s_in)
            stream.wait_event(in_ready[i])
            if i >= 2:
                stream.wait_event(out_done[i - 2])
            flush.zero_()
            ibs.ibs_grm(ctx, d_in[b], n, m, d_out[b], stream)
            comp_done[i].record(stream)
            s_out.wait_event(comp_done[i])
            with torch.cuda.stream(s_out):
                h_out[b].copy_(d_out[b], non_blocking=True)
            out_done[i].record(s_out)
        t1_ev.record(s_out)
        torch.cuda.synchronize(dev)
        e2e_ms = [t0_ev.elapsed_time(t1_ev) / args.steps] * args.steps
        h_out = h_out[(args.steps - 1) % 2]
    got = h_out.numpy()
    # spot check: sampled rows against the oracle's row sampler
    G = oracle.unpack(w.packed, n, m)
    rows = np.array([0, 2047, 4095])
    want = oracle.grm_rows(G, rows)
    k = np.arange(n)
    got_rows = np.stack([got[oracle.tri_index(np.minimum(j, k), np.maximum(j, k), n)] for j in rows])
    err = float(np.nanmax(np.abs(got_rows - want)))
    ibs.ibs_shutdown(ctx)
    mean_ms = statistics.mean(ms)
    tflops = 8.0 * comps / (mean_ms * 1e-3) / 1e12
    peak = measured_peak("bf16_tflops", 1900.0)
    line = {
        "metric": "sample-pair x marker terms/s (GCTA relationship matrix)", "value": comps / (mean_ms * 1e-3),
        "unit": "terms/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16xf16->f32 (hi/lo split)",
        "data": "synthetic",
        "config": {"workload": f"GCTA relationship matrix, plain workload genotypes n={n} m={m}",
                   "pairs_incl_diagonal": P,
                   "l2": "flushed between steps (256 MiB write, outside the step events)"},
        "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                     "traffic": profiled_traffic("tc_grm_kernel_plain.md",
                                                 ("ibs_grm.cu", "ibs_tc_common.cuh", "ibs_device.cuh")),
                     "kernel": "whole ibs_grm call (frequency and operand kernels included)",
                     "kernel_ms": mean_ms,
                     "peak_basis": "measured bf16 burst TFLOP/s (MEASURED_PEAKS.json; FP16 runs at the bf16 rate); "
                                   "algorithmic flops = 8 per term (4 MACs: hi hi, hi lo, lo hi, V'V')"},
        "e2e": {"value": comps / (statistics.mean(e2e_ms) * 1e-3), "unit": "terms/s",
                "h2d_bytes_per_step": int(w.packed.nbytes), "d2h_bytes_per_step": int(P * 8),
                "pipelined": "copy-in, compute and copy-out streams, two buffer sets"},
        "accuracy": {"max_abs_err_rows_0_2047_4095": err},
        "gpu_launches": int(launches * args.steps),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        R = 32
        t = time.perf_counter()
        oracle.grm_rows(G, np.linspace(0, n - 1, R).astype(np.int64))
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": R * n * m / dt, "unit": "terms/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": f"{R} rows x all {n} columns x {m} markers ({dt:.1f} s)"}
    return line


def run_cluster(args, rank, world, local):
    """Complete-linkage clustering (paper, "Identity-by-state matrices, complete
    linkage clustering") of the plain workload's 4,096 samples under their IBS
    distances: ibs_compute once, then ibs_cluster_complete timed per step."""
    import numpy as np
    import torch
    import oracle
    from paper_1410_4803_gb300 import ibs

    torch.cuda.set_device(local)
    w = make_workload("plain")
    n, m = w.n, w.m
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    ctx = ibs.ibs_init(local)
    z = torch.empty((n - 1, 4), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        _, dist = ibs.compute(ctx, torch.from_numpy(w.packed).to(dev), n, m, stream=stream)
        for _ in range(args.warmup):
            ibs.ibs_cluster_complete(ctx, dist, n, z, stream)
        ibs.ibs_synchronize(ctx, stream)
        launches = ibs.ibs_last_launch_info(ctx)["launches"]
        clk = ClockSampler(local)
        clk.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            ev[i][0].record(stream)
            ibs.ibs_cluster_complete(ctx, dist, n, z, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        clocks = clk.stop()
        ibs.ibs_synchronize(ctx, stream)
        ms = [a.elapsed_time(b) for a, b in ev]
        # end to end: the distance triangle from pinned host memory, the linkage back
        h_d = dist.cpu().pin_memory()
        h_z = torch.empty((n - 1, 4), dtype=torch.float64).pin_memory()
        d_in = torch.empty_like(dist)
        e2e = []
        for i in range(max(1, args.steps // 2)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d_in.copy_(h_d, non_blocking=True)
            ibs.ibs_cluster_complete(ctx, d_in, n, z, stream)
            h_z.copy_(z, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            e2e.append(e0.elapsed_time(e1))
    tri = h_d.numpy()
    t_or = time.perf_counter()
    want = oracle.complete_linkage(tri, n)
    dt_or = time.perf_counter() - t_or
    exact = bool(np.array_equal(h_z.numpy(), want))
    ibs.ibs_shutdown(ctx)
    mean_ms = statistics.mean(ms)
    line = {
        "metric": "complete-linkage merges/s (IBS distance matrix)", "value": (n - 1) / (mean_ms * 1e-3),
        "unit": "merges/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"complete linkage of the plain workload's n={n} samples (IBS distances, m={m})"},
        "e2e": {"value": (n - 1) / (statistics.mean(e2e) * 1e-3), "unit": "merges/s",
                "h2d_bytes_per_step": int(tri.nbytes), "d2h_bytes_per_step": int((n - 1) * 32)},
        "exact": {"linkage_equals_oracle": exact},
        "gpu_launches": int(launches * args.steps),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        # the whole workload (the exactness check above): the oracle's O(n^3)
        # greedy takes about 12 s at n = 4,096
        dt = dt_or
        line["cpu_baseline"] = {"value": (n - 1) / dt, "unit": "merges/s", "cores": 1, "kind": "oracle",
                                "sample": f"all {n} samples' distances, O(n^3) greedy ({dt:.1f} s)"}
    return line


def sub_record(line: dict, keys) -> dict:
    return {k: line[k] for k in keys if k in line}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="structured",
                    choices=["plain", "structured", "batch", "serve", "ld", "cluster", "grm"])
    ap.add_argument("--no-sub", action="store_true",
                    help="structured: skip the plain, batched and served sub-records")
    ap.add_argument("--window", type=int, default=1000, help="ld: marker window")
    ap.add_argument("--markers", type=int, default=100_000,
                    help="grm: markers of the plain genotypes (100,000 is the benchmarked size)")
    ap.add_argument("--rates", type=float, nargs="*", default=None,
                    help="serving: Poisson arrival rates per second (0 = all at once)")
    ap.add_argument("--requests", type=int, default=None, help="serving: requests per rate")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--samples", type=int, default=0,
                    help="plain/structured/serve: a smaller case with this many samples (profiling captures)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=3.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    rank, world, local = dist_env()
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.impl == "reference":
        line = run_reference(args, rank, world, local)
    elif args.workload == "batch":
        line = run_batch(args, rank, world, local)
    elif args.workload == "serve":
        if args.rates is None:
            args.rates = [4.0, 12.0, 24.0, 0.0]
        if args.requests is None:
            args.requests = 60
        line = run_serve(args, rank, world, local)
    elif args.workload == "ld":
        line = run_ld(args, rank, world, local)
    elif args.workload == "cluster":
        line = run_cluster(args, rank, world, local)
    elif args.workload == "grm":
        line = run_grm(args, rank, world, local)
    else:
        if args.no_cpu_baseline:
            args.cpu_seconds = 1.0  # the spot check still runs, on a small block
        line = run_matrix(args, rank, world, local, args.workload, full=True)
        if args.workload == "structured" and not args.no_sub and world == 1:
            import torch
            torch.cuda.empty_cache()
            # the plain workload, the batched cohorts and the served panel on the same
            # GPU and in the same run, each with its own timing and exactness checks
            p = run_matrix(args, rank, world, local, "plain", full=False)
            line["plain_config2"] = sub_record(p, ["value", "unit", "ms_per_step", "dtype", "config", "roofline",
                                                   "transpose", "finalize_ms", "e2e", "gpu_launches", "clocks"])
            torch.cuda.empty_cache()
            b = run_batch(args, rank, world, local)
            line["batched"] = sub_record(b, ["value", "unit", "ms_per_step", "dtype", "config", "plain_loop",
                                             "speedup_vs_plain_loop", "exact", "gpu_launches", "clocks"])
            torch.cuda.empty_cache()
            if args.rates is None:
                args.rates = [6.0, 24.0, 0.0]
            if args.requests is None:
                args.requests = 48
            sv = run_serve(args, rank, world, local)
            line["served"] = sub_record(sv, ["value", "unit", "dtype", "config", "serving", "engine_stats",
                                             "host_context", "exact", "clocks"])
    if line is not None:
        print(json.dumps(line))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
