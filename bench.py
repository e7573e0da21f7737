#!/usr/bin/env python
"""Throughput of the in-silico PCR path (scan, site compaction, pairing, FP64 Tm, trimming and
barcodes) on GB300, as Gbp/s, with the scan kernel's roofline fraction.

Default workload (N=1): 2,000 synthetic genomes, lognormal lengths (median 3.5 Mbp, sigma 0.4,
~7.6 Gbp), per-genome GC ~ U(0.30, 0.70), 0.5 % N in runs of 1-50, 1-15 planted 16S-like
templates per genome; one degenerate pair (19 nt with 2 codes, 20 nt with 3), k=3, clamp 3,
window 50-2000, all four orientations, primer trimming and 16-nt barcodes.

`value` times one step over the packed genomes already resident in HBM.  `e2e` times the same
step through the C ABI from pinned host ASCII: host->device copy and packing, the step, and the
device->host copy of sites, amplicons and sequences.  `--impl reference` times the oracle (plain
C on the host cores) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gbp/s scanned (k=2, 4 orientations), % of HBM roofline; p99 request latency"
# ALU-pipe peak from unit counts and clocks: 152 SMs x 4 sub-partitions x 16 lanes of LOP3/SHF per
# clock x 2.07 GHz maximum SM clock (LOP3 and SHF share this pipe; integer adds run beside it).
SM_COUNT, ALU_LANES_PER_SM_CLK, SM_MAX_GHZ = 152, 64, 2.07
ALU_PEAK_TOPS = SM_COUNT * ALU_LANES_PER_SM_CLK * SM_MAX_GHZ / 1e3   # T lane-ops/s


TM_KERNELS = {"generated": 0, "builtin": 1}


def engine_for(args, device):
    """An engine on `device` with the degenerate-site Tm kernel the command line asks for."""
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Engine

    eng = Engine(device)
    ah.ah_ctx_set_tm_kernel(eng.ctx, TM_KERNELS[getattr(args, "tm_kernel", "generated")])
    if getattr(args, "tm_split", 0):
        ah.ah_ctx_set_tm_split(eng.ctx, args.tm_split)
    fixed = getattr(args, "scan_fixed", "")
    if fixed:
        t, g, mode, mb, w, queue = ([int(x) for x in fixed.split(",")] + [0])[:6]   # queue defaults to 0
        ah.ah_ctx_set_scan_config(eng.ctx, t, g, 256, mode)
        ah.ah_ctx_set_scan_circuit(eng.ctx, mb, w, queue)
    return eng


def autotune(args):
    """Plans choose their scan kernel by timing candidates unless --scan-fixed names one."""
    return not getattr(args, "scan_fixed", "")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def alg_ops_per_base(fwd, rev, clamp):
    """Algorithmic lane-ops per base of the bit-sliced scan: per oriented pattern of length L, one
    lane-op per position for the IUPAC test, two for carry-save counting of each non-clamp
    position, one to fold each clamp position into the failure word; one lane-op covers 32
    positions."""
    total = 0
    for p in list(fwd) + list(rev):
        L = len(p)
        total += 2 * (3 * (L - clamp) + 2 * clamp)   # both strands
    return total / 32.0


# DRAM bytes per base of scan kernels captured with ncu on a smaller case of the same kernel
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch, larger than L2), scaled to a launch by
# its bases (the traffic is one pass over the planes), keyed by what identifies the kernel: LOP3/SHF
# per 32 positions of its circuit, threads, groups per thread, shift mode, persistent.  A kernel not
# in this table reports traffic null.
SCAN_TRAFFIC = {
    # the bench pair: plain_scale's first 200 genomes, 756,529,120 bases, 189 MB of planes
    (186, 256, 8, 0, 0): ((189_561_088 + 1_595_904) / 756_529_120,
                          "plain_scale's first 200 genomes (profiles/ah_scan_jit_alu_pipe.md)"),
    # the batched set: its first 2,000 genomes, 3,487,157,421 bases, 872 MB of planes (the kernel the
    # autotuner keeps, registers bounded for 4 blocks per SM)
    (996, 128, 8, 0, 0): ((873_291_008 + 743_168) / 3_487_157_421,
                          "the batched set's first 2,000 genomes (profiles/ah_scan_jit_alu_pipe.md)"),
}


# ALU-pipe work the scan kernel actually executes, from ncu on a smaller case of the same circuit
# (smsp__inst_executed_pipe_alu.sum x 32 lanes / bases scanned, and sm__pipe_alu_cycles_active as a
# fraction of peak), keyed by the circuit's LOP3/SHF per 32 positions, then by the register bound
# (blocks per SM, 0 for none) where it changes the code.  profiles/ holds the captures.
SCAN_PIPE = {
    # the bench pair (19/20 nt, k=3, clamp 3): plain_scale's first 200 genomes (756.5 Mbp), autotuned
    # 256 threads x 8 groups, shift mode 0; 109,810,167 ALU-pipe warp instructions per launch
    186: {"alu_lane_ops_per_base": 109_810_167 * 32 / 756_529_120, "alu_pipe_busy": 0.966,
          "source": "ncu smsp__inst_executed_pipe_alu.sum x 32 / bases of one launch, plain_scale 200 genomes "
                    "(profiles/ah_scan_jit_alu_pipe.md)"},
    # the batched set (8 pairs = 32 patterns, k = i mod 4): its first 2,000 genomes (3.49 Gbp), the
    # kernel the autotuner keeps: 128 threads x 8 groups, shift mode 0, registers bounded for 4 blocks
    # per SM, phase split drawn for 4,096 windows per vote (996 LOP3/SHF per 32 positions);
    # 2,178,723,827 ALU-pipe warp instructions per launch
    (996, 4): {"alu_lane_ops_per_base": 2_178_723_827 * 32 / 3_487_157_421, "alu_pipe_busy": 0.876,
               "source": "ncu smsp__inst_executed_pipe_alu.sum x 32 / bases of one launch, batched 2,000 genomes, "
                         "register bound 4 blocks/SM, split for 4,096 windows (profiles/ah_scan_jit_alu_pipe.md)"},
    # the circuit split for 1,024 windows per vote (1,030 LOP3/SHF per 32 positions), without and with
    # the register bound: 2,215,146,059 and 2,205,943,674 ALU-pipe warp instructions per launch
    1030: {"alu_lane_ops_per_base": 2_215_146_059 * 32 / 3_487_157_421, "alu_pipe_busy": 0.783,
           "source": "ncu smsp__inst_executed_pipe_alu.sum x 32 / bases of one launch, batched 2,000 genomes "
                     "(profiles/ah_scan_jit_alu_pipe.md)"},
    (1030, 4): {"alu_lane_ops_per_base": 2_205_943_674 * 32 / 3_487_157_421, "alu_pipe_busy": 0.863,
                "source": "ncu smsp__inst_executed_pipe_alu.sum x 32 / bases of one launch, batched 2,000 genomes, "
                          "register bound 4 blocks/SM (profiles/ah_scan_jit_alu_pipe.md)"},
}


def scan_roofline(ops_per_group, fwd, rev, clamp, bases, ms, shape=None, sm_mhz=None, min_blocks=0):
    """ALU roofline of one scan launch.  `achieved` is algorithmic: the per-base lane-op count of the
    bit-sliced method (3 per non-clamp and 2 per clamp position of every oriented pattern, 32
    positions per lane-op) times the bases of the launch, over its CUDA-event time.  The generated
    circuit needs fewer instructions than that count (it shares plane derivations and shifts across
    patterns, reads two-base IUPAC sets straight from the code planes and folds the counter tree),
    and a warp skips a pattern's second phase when every one of its windows already failed the
    first, so the algorithmic fraction can exceed 1.  `circuit` gives the generator's instruction
    count with every phase run (an upper bound on what executes).  `shape` = (threads, groups per
    thread, shift mode, persistent) of the launch."""
    ops = ops_per_group / 32.0
    rec = SCAN_TRAFFIC.get((ops_per_group,) + tuple(shape)) if shape is not None else None
    traffic = rec[0] * bases if rec is not None else None
    norm = alg_ops_per_base(fwd, rev, clamp)
    achieved = norm * bases / (ms * 1e-3) / 1e12
    circuit = ops * bases / (ms * 1e-3) / 1e12
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm = 0.25 * bases / (ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TOPS, "unit": "Tlane-op/s",
            "frac": achieved / ALU_PEAK_TOPS, "traffic": traffic,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel (same circuit and "
                               f"shape) on {rec[1]}, scaled to the bases of this launch")
                              if rec is not None else None,
            "kernel": "ah_scan_jit (bit-sliced scan)", "kernel_ms": ms,
            "ops_per_base": norm, "ops_source": "algorithmic: sum over oriented patterns of (3 (L - c) + 2 c) / 32",
            "peak_source": "derived: 152 SMs x 64 ALU lanes/clk x 2.07 GHz",
            "circuit": {"ops_per_base": ops, "achieved": circuit, "frac": circuit / ALU_PEAK_TOPS,
                        "source": "LOP3 + funnel shifts of the generated circuit with every phase run "
                                  "(warps skip phase two when all their windows failed phase one)"},
            "hbm": {"achieved_gbs": hbm, "peak_gbs": hbm_peak,
                    "peak_source": "measured" if "hbm_gbs" in peaks else "fallback", "frac": hbm / hbm_peak,
                    "algorithmic_bytes_per_base": 0.25},
            "executed": _executed(ops_per_group, bases, ms, sm_mhz, min_blocks)}


def _executed(ops_per_group, bases, ms, sm_mhz, min_blocks=0):
    """The scan's executed ALU-pipe lane-ops per second against the pipe's peak at the clock the run
    saw (152 SMs x 64 lanes x sampled SM clock): a fraction of at most 1 that says how busy the pipe
    the kernel is bound by is kept."""
    rec = SCAN_PIPE.get((ops_per_group, min_blocks)) if min_blocks else SCAN_PIPE.get(ops_per_group)
    if rec is None:
        return None
    mhz = sm_mhz or SM_MAX_GHZ * 1e3
    peak = SM_COUNT * ALU_LANES_PER_SM_CLK * mhz / 1e6   # T lane-ops/s
    achieved = rec["alu_lane_ops_per_base"] * bases / (ms * 1e-3) / 1e12
    return {"ops_per_base": rec["alu_lane_ops_per_base"], "achieved": achieved, "peak": peak, "unit": "Tlane-op/s",
            "frac": achieved / peak, "alu_pipe_busy_ncu": rec["alu_pipe_busy"],
            "peak_source": f"derived: 152 SMs x 64 ALU lanes/clk x {mhz:.0f} MHz (median SM clock sampled in the run)",
            "ops_source": rec["source"]}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_workload(args):
    import synth

    if args.workload == "plain_scale":
        return synth.plain_scale(n_genomes=args.genomes or 2000)
    if args.workload == "plain_small":
        return synth.plain_small(n_genomes=args.genomes or 16)
    if args.workload == "batched":
        return synth.batched(n_genomes=args.genomes or 2000)
    if args.workload == "dense":
        # 5,000 genomes (17.5 Gbp) drawn on the device, byte-identical to the host drawer
        import synth.gpu

        return synth.gpu.dense(n_genomes=args.genomes or 5000)
    raise SystemExit(f"unknown workload {args.workload}")


L2_FLUSH_BELOW = 256 << 20   # packed bytes below which timed steps are separated by an L2 flush


def describe(wl):
    return {"workload": f"{wl.name}: {wl.n_records} synthetic genomes, {wl.total_bp / 1e9:.3f} Gbp, "
                        f"{len(wl.fwd)} degenerate primer pair(s), k={wl.k}, clamp {wl.clamp}, "
                        f"window {wl.min_len}-{wl.max_len}, orientations mask {wl.orient_mask}, "
                        f"trim={wl.trim}, barcodes {wl.fb_len}/{wl.rb_len}, "
                        f"Tm filter {wl.tm.min_tm}",
            "genomes": wl.n_records, "bases": wl.total_bp, "pairs": len(wl.fwd),
            "l2": ("inputs larger than L2 (packed genomes %.2f GB >> 129 MB)" % (wl.total_bp / 4e9)
                   if wl.total_bp / 4 > L2_FLUSH_BELOW else
                   "inputs smaller than L2 (packed genomes %.1f MB): a 512 MB buffer is written between timed "
                   "steps, outside the timed intervals" % (wl.total_bp / 4e6))}


# ------------------------------------------------------------------------------------------ oracle arm
def oracle_sample_seconds(wl, n_genomes):
    import oracle

    sub = wl.subset(range(n_genomes))
    t = time.perf_counter()
    oracle.run(sub, threads=os.cpu_count() or 1)
    return time.perf_counter() - t, sub.total_bp


def pick_sample(wl, target_s):
    """Number of leading genomes whose oracle run takes about target_s on the host cores."""
    # the oracle runs records in parallel, so calibrate on one record per host core
    t1, bp1 = oracle_sample_seconds(wl, min(os.cpu_count() or 1, wl.n_records))
    rate = bp1 / max(t1, 1e-3)
    want = rate * target_s
    n, acc = 0, 0
    lens = wl.lengths()
    while n < wl.n_records and acc < want:
        acc += int(lens[n])
        n += 1
    return max(1, n)


def cpu_baseline(wl, target_s=15.0):
    n = pick_sample(wl, target_s)
    t, bp = oracle_sample_seconds(wl, n)
    return {"value": bp / t / 1e9, "unit": "Gbp/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"first {n} of {wl.n_records} genomes ({bp / 1e6:.1f} Mbp), whole path "
                      f"(scan, pair, Tm, extract), {os.cpu_count()} threads, {t:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_workload(args)
    n = pick_sample(wl, 2.0)
    import oracle

    sub = wl.subset(range(n))
    for _ in range(args.warmup):
        oracle.run(sub, threads=os.cpu_count() or 1)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(sub, threads=os.cpu_count() or 1)
    dt = (time.perf_counter() - t) / args.steps
    v = sub.total_bp / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gbp/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+f64", "data": "synthetic",
            "config": describe(wl),
            "cpu_baseline": {"value": v, "unit": "Gbp/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: first {n} genomes ({sub.total_bp / 1e6:.1f} Mbp), whole path"},
            "e2e": {"value": v, "unit": "Gbp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------ engine arm
def job_time_and_value(ms_local, bases_per_rank, world):
    """Replicas (one process per GPU, each scanning its own copy of the workload): the job's step time
    is the slowest rank's, and the job's throughput counts every rank's bases.  Needs an initialised
    process group when world > 1."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * bases_per_rank / (ms * 1e-3) / 1e9


def fasta_into(dst, seq, offsets, width=80):
    """Write the records as FASTA (">genome_<r> synthetic" headers, `width`-column lines) into the
    uint8 array dst; returns the length.  With dst None, only the length."""
    import numpy as np

    pos = 0
    for r in range(len(offsets) - 1):
        head = b">genome_%d synthetic\n" % r
        L = int(offsets[r + 1] - offsets[r])
        rows = (L + width - 1) // width
        n = len(head) + L + rows
        if dst is not None:
            dst[pos:pos + len(head)] = np.frombuffer(head, dtype=np.uint8)
            body = dst[pos + len(head):pos + n]
            s = seq[int(offsets[r]):int(offsets[r + 1])]
            full = (L // width) * (width + 1)
            if full:
                grid = body[:full].reshape(-1, width + 1)
                grid[:, :width] = s[:(L // width) * width].reshape(-1, width)
                grid[:, width] = 10
            tail = L - (L // width) * width
            if tail:
                body[full:full + tail] = s[L - tail:]
                body[full + tail] = 10
        pos += n
    return pos


def e2e_from_fasta(ah, eng, wl, batch, plan, bufs, on_device, steps):
    """End to end from FASTA text in pinned host memory: ah_plan_launch_fasta (the text parsed on the
    device in chunks as it lands, the completed records packed and their tiles scanned at once, the
    rest of the step after the last chunk) -> results into pinned host buffers; and beside it the
    form that parses and packs all of the text before the step."""
    import numpy as np
    import torch

    seq = wl.d_seq.cpu().numpy() if on_device else wl.seq
    n = fasta_into(None, seq, wl.offsets)
    t_text = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    fasta_into(t_text.numpy(), seq, wl.offsets)
    del seq

    def timed(overlap):
        times = []
        for it in range(1 + steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            if overlap:
                ah.ah_plan_launch_fasta(plan, t_text.data_ptr(), n, eng.ctx)
            else:
                ah.ah_fasta_pack_into(eng.ctx, t_text.data_ptr(), batch, n_bytes=n)
                ah.ah_plan_launch(plan, eng.ctx)
            ah.ah_plan_copy_results(plan, eng.ctx, *bufs)
            dt = time.perf_counter() - t
            if it > 0:
                times.append(dt)
        return statistics.median(times)

    t_overlap, t_serial = timed(True), timed(False)
    del t_text
    return {"value": wl.total_bp / t_overlap / 1e9, "unit": "Gbp/s", "h2d_bytes_per_step": n,
            "ms_per_step": t_overlap * 1e3,
            "path": "pinned FASTA text (80-column lines) -> ah_plan_launch_fasta (parsed on the device in 256 MiB "
                    "chunks as they land, completed records packed and their tiles scanned at once) -> "
                    "ah_plan_copy_results into pinned host buffers",
            "parse_then_step": {"value": wl.total_bp / t_serial / 1e9, "unit": "Gbp/s", "ms_per_step": t_serial * 1e3,
                                "path": "ah_fasta_pack_into -> ah_plan_launch -> ah_plan_copy_results"}}


def run_engine(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)

    wl = make_workload(args)
    base = None
    if rank == 0 and not args.no_cpu_baseline:
        base = cpu_baseline(wl, args.cpu_seconds)   # host cores only; before the engine's GPU work

    import __graft_entry__

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Engine, Params

    eng = engine_for(args, local)
    stream = torch.cuda.ExternalStream(ah.ah_ctx_stream(eng.ctx))
    params = Params.from_workload(wl)
    on_device = hasattr(wl, "d_seq")   # drawn on the device
    d_seq = wl.d_seq if on_device else torch.from_numpy(wl.seq).to(f"cuda:{local}")
    torch.cuda.synchronize()
    batch = eng.pack_device(d_seq.data_ptr(), wl.offsets.astype(np.uint64), wl.genome_ids)
    ah.ah_ctx_synchronize(eng.ctx)
    if not on_device:
        del d_seq
        torch.cuda.empty_cache()

    # the whole step as one autotuned, graph-captured plan (sized by one exact run of the step)
    with_seqs = getattr(wl, "extract", True)
    plan = eng.plan(batch, params, with_seqs=with_seqs, autotune=autotune(args), persistent=-1)
    info = ah.ah_plan_info_get(plan)

    def one_step():
        ah.ah_plan_launch(plan)

    for _ in range(max(3, args.warmup)):
        one_step()
    ah.ah_ctx_synchronize(eng.ctx)
    ah.ah_plan_check(plan, eng.ctx)

    def barrier():
        if world > 1:
            dist.barrier()

    ah.ah_ctx_stats_reset(eng.ctx)
    ah.ah_ctx_set_timing(eng.ctx, True)
    flush = wl.total_bp / 4 <= L2_FLUSH_BELOW   # inputs that fit in L2: flush it between timed steps
    scratch = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{local}") if flush else None
    marks = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps if flush else 1)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        if flush:
            for a, z in marks:
                with torch.cuda.stream(stream):
                    scratch.fill_(1)
                a.record(stream)
                one_step()
                z.record(stream)
        else:
            marks[0][0].record(stream)
            for _ in range(args.steps):
                one_step()
            marks[0][1].record(stream)
        torch.cuda.synchronize()
    barrier()
    ah.ah_ctx_set_timing(eng.ctx, False)
    ah.ah_plan_check(plan, eng.ctx)   # every replay fitted its buffers (raises on overflow)
    ms = sum(a.elapsed_time(z) for a, z in marks) / args.steps
    del scratch
    stats = ah.ah_ctx_stats_get(eng.ctx)
    ms, value = job_time_and_value(ms, wl.total_bp, world)

    # roofline of the dominant kernel (the bit-sliced scan), from its own CUDA-event times
    scan_ms = stats["scan_ms"] / max(1, stats["scan_launches"])
    bases_per_launch = stats["scan_bases"] / max(1, stats["scan_launches"])
    roofline = scan_roofline(stats["scan_ops_per_group"], wl.fwd, wl.rev, wl.clamp, bases_per_launch, scan_ms,
                             (info["threads"], info["groups_per_thread"], info["shift_mode"], info["persistent"]),
                             clk.summary().get("sm_mhz"), info["min_blocks"])
    roofline["step_gbps_frac_of_alu_bound"] = value / world / (ALU_PEAK_TOPS * 1e3 / roofline["circuit"]["ops_per_base"])

    # end to end through the C ABI from pinned host memory: every step packs the records from host
    # ASCII into the plan's batch (copy engines in 256 Mi-base chunks, packed from HBM as they land),
    # replays the plan and copies sites, amplicons and sequences into pinned host buffers
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(wl.total_bp, dtype=torch.uint8, pin_memory=True)
        if on_device:
            pinned.copy_(wl.d_seq)
        else:
            pinned.numpy()[:] = wl.seq
        offs = np.ascontiguousarray(wl.offsets, dtype=np.uint64)

        def pinned_array(n, dtype):   # page-locked result buffer with room for a quarter more
            n = int(n * 1.25) + 1024
            t = torch.empty(n * np.dtype(dtype).itemsize, dtype=torch.uint8, pin_memory=True)
            return t, t.numpy().view(dtype)

        keep = [pinned_array(info["n_hits"], ah.HIT_DTYPE), pinned_array(info["n_kept"], ah.AMP_DTYPE)]
        if with_seqs:
            keep += [pinned_array(info["arena_bytes"], np.uint8), pinned_array(5 * info["n_kept"] + 1, np.uint64)]
        bufs = [k[1] for k in keep] + [None] * (4 - len(keep))
        h2d = d2h = 0
        times = []
        for it in range(1 + args.e2e_steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            ah.ah_plan_launch_host(plan, pinned.data_ptr(), offs, eng.ctx)
            ah.ah_plan_copy_results(plan, eng.ctx, *bufs)
            dt = time.perf_counter() - t
            if it > 0:
                times.append(dt)
            i2 = ah.ah_plan_info_get(plan)
            h2d = wl.total_bp
            d2h = i2["n_hits"] * ah.HIT_DTYPE.itemsize + i2["n_kept"] * ah.AMP_DTYPE.itemsize + (
                i2["arena_bytes"] + 8 * (5 * i2["n_kept"] + 1) if with_seqs else 0)
        e2e = {"value": wl.total_bp / statistics.median(times) / 1e9, "unit": "Gbp/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": len(times), "ms_per_step": statistics.median(times) * 1e3,
               "path": "pinned host ASCII -> ah_plan_launch_host (chunked copies, packed as they land, each range of "
                       "scan tiles scanned once its bases are in, the rest of the step after the last chunk) -> "
                       "ah_plan_copy_results (sites, amplicons, sequences) into pinned host buffers"}
        # the same with the scan after the whole upload (pack, then the plan's replay)
        times = []
        for it in range(1 + args.e2e_steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            ah.ah_batch_pack_range(eng.ctx, batch, 0, pinned.data_ptr(), offs)
            ah.ah_plan_launch(plan, eng.ctx)
            ah.ah_plan_copy_results(plan, eng.ctx, *bufs)
            dt = time.perf_counter() - t
            if it > 0:
                times.append(dt)
        e2e["scan_after_upload"] = {"value": wl.total_bp / statistics.median(times) / 1e9, "unit": "Gbp/s",
                                    "ms_per_step": statistics.median(times) * 1e3,
                                    "path": "ah_batch_pack_range -> ah_plan_launch -> ah_plan_copy_results"}
        del pinned
        # the same from stored 2-bit batches (the paper streams its 2-bit batch files): exported
        # planes and sparse invalid words in pinned memory, imported every step
        v = ah.ah_batch_view_get(batch)
        pl_t = torch.empty(v["n_groups"] * 8, dtype=torch.uint8, pin_memory=True)
        planes = pl_t.numpy().view(np.uint32).reshape(-1, 2)
        _, groups0, words0 = ah.ah_batch_export(batch, planes)
        g_t = torch.empty(max(1, len(groups0)) * 8, dtype=torch.uint8, pin_memory=True)
        w_t = torch.empty(max(1, len(words0)) * 4, dtype=torch.uint8, pin_memory=True)
        groups = g_t.numpy().view(np.uint64)[:len(groups0)]
        words = w_t.numpy().view(np.uint32)[:len(words0)]
        groups[:] = groups0
        words[:] = words0
        def packed_steps(overlap):
            times = []
            for it in range(1 + args.e2e_steps):
                torch.cuda.synchronize()
                t = time.perf_counter()
                if overlap:
                    ah.ah_plan_launch_packed(plan, planes, groups, words, eng.ctx)
                else:
                    ah.ah_batch_import(eng.ctx, batch, planes, groups, words)
                    ah.ah_plan_launch(plan, eng.ctx)
                ah.ah_plan_copy_results(plan, eng.ctx, *bufs)
                dt = time.perf_counter() - t
                if it > 0:
                    times.append(dt)
            return statistics.median(times)

        t_overlap, t_serial = packed_steps(True), packed_steps(False)
        e2e["from_packed_batches"] = {
            "value": wl.total_bp / t_overlap / 1e9, "unit": "Gbp/s",
            "h2d_bytes_per_step": planes.nbytes + groups.nbytes + words.nbytes, "d2h_bytes_per_step": d2h,
            "ms_per_step": t_overlap * 1e3,
            "path": "pinned 2-bit planes + sparse invalid words -> ah_plan_launch_packed (invalid words first, "
                    "planes in 256 Mi-base chunks, each range of scan tiles scanned as its planes land) -> "
                    "ah_plan_copy_results into pinned host buffers",
            "import_then_step": {"value": wl.total_bp / t_serial / 1e9, "unit": "Gbp/s", "ms_per_step": t_serial * 1e3,
                                 "path": "ah_batch_import -> ah_plan_launch -> ah_plan_copy_results"}}
        del pl_t, g_t, w_t
        if args.e2e_fasta:
            e2e["from_fasta"] = e2e_from_fasta(ah, eng, wl, batch, plan, bufs, on_device, args.e2e_steps)

    ah.ah_plan_free(plan)
    ah.ah_batch_free(batch)
    eng.close()
    if on_device:
        wl.d_seq = None
    torch.cuda.empty_cache()
    # the other measured rows of the path at one GPU (batched plan against the plain per-record
    # form, the dense-hit stress, serving latency), each with its own clock record
    extras = {}
    if world == 1 and not args.no_extras and args.workload == "plain_scale":
        extras["batched"] = batched_record(args, min(args.steps, 5), 3)
        extras["dense"] = dense_record(args, min(args.steps, 10), 3)
        stable, loaded = serving_record(args, [(args.serve_requests, args.serve_rate), (args.serve_burst, 200.0)])
        extras["serving"] = {"stable_rate": stable, "offered_200_per_s": loaded}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gbp/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32+f64", "data": "synthetic",
                "config": dict(describe(wl), launch=f"one CUDA-graph replay of the whole step per step; autotuned scan "
                               f"{info['threads']} threads x {info['groups_per_thread']} groups, shift mode "
                               f"{info['shift_mode']}, persistent {info['persistent']}, register bound "
                               f"{info['min_blocks']} blocks/SM (0: none), phase split drawn for {info['vote_windows']} windows "
                               f"per warp vote, candidate queue {info['emit_queue']}"),
                "clocks": clk.summary(), "e2e": e2e, "gpu_launches": stats["kernel_launches"],
                "gpu_launches_per_step": stats["kernel_launches"] / args.steps, "roofline": roofline,
                "cpu_baseline": base}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------ dense arm
def dense_record(args, steps, warmup):
    """The dense-hit workload (tandem repeats, highly degenerate primers, about one site per kb) as one
    graph-captured plan: scan, compaction, pairing and the FP64 Tm of every paired site."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth.gpu as sg

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Engine, Params

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    wl = sg.dense(n_genomes=5000)
    eng = engine_for(args, 0)
    batch = eng.pack_device(wl.d_seq.data_ptr(), wl.offsets.astype(np.uint64), wl.genome_ids)
    ah.ah_ctx_synchronize(eng.ctx)
    gen_s = time.perf_counter() - t0
    wl.d_seq = None
    torch.cuda.empty_cache()
    params = Params.from_workload(wl)
    stream = torch.cuda.ExternalStream(ah.ah_ctx_stream(eng.ctx))
    plan = eng.plan(batch, params, with_seqs=getattr(wl, "extract", True), autotune=autotune(args), persistent=-1)
    for _ in range(max(3, warmup)):
        ah.ah_plan_launch(plan, eng.ctx)
    ah.ah_ctx_synchronize(eng.ctx)
    ah.ah_plan_check(plan, eng.ctx)
    ah.ah_ctx_stats_reset(eng.ctx)
    ah.ah_ctx_set_timing(eng.ctx, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(steps):
            ah.ah_plan_launch(plan, eng.ctx)
        e1.record(stream)
        torch.cuda.synchronize()
    ah.ah_ctx_set_timing(eng.ctx, False)
    ah.ah_plan_check(plan, eng.ctx)
    ms = e0.elapsed_time(e1) / steps
    st = ah.ah_ctx_stats_get(eng.ctx)
    info = ah.ah_plan_info_get(plan)
    scan_ms = st["scan_ms"] / max(1, st["scan_launches"])
    line = {"workload": "dense", "value": wl.total_bp / (ms * 1e-3) / 1e9, "unit": "Gbp/s", "steps": steps,
            "warmup": max(3, warmup), "ms_per_step": ms,
            "config": {"workload": f"dense: {wl.n_records} genomes, {wl.total_bp / 1e9:.2f} Gbp, 30 % with tandem "
                                   f"repeats; {len(wl.fwd)} pair of {len(wl.fwd[0])}/{len(wl.rev[0])} nt with "
                                   f"degenerate codes, k={wl.k}, window {wl.min_len}-{wl.max_len}, all orientations, "
                                   "Tm of every paired site (no sequences)",
                       "bases": wl.total_bp, "l2": "inputs larger than L2"},
            "sites": info["n_hits"], "amplicons": info["n_amps"],
            "sites_per_kb": info["n_hits"] / (wl.total_bp / 1e3),
            "scan_kernel_ms": scan_ms, "rest_of_step_ms": ms - scan_ms,
            "gpu_launches_per_step": st["kernel_launches"] / steps, "generate_and_pack_s": gen_s,
            "clocks": clk.summary()}
    ah.ah_plan_free(plan)
    ah.ah_batch_free(batch)
    eng.close()
    torch.cuda.empty_cache()
    return line


# ------------------------------------------------------------------------------------------ batched arm
def run_batched(args):
    print(json.dumps(batched_record(args, args.steps, args.warmup)), flush=True)


def batched_record(args, steps, warmup):
    """The batched workload (many genomes x 8 pairs) as one graph-captured plan, against the plain
    form (one scan launch per genome per pair) and the one-launch scan on the same GPU."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth.gpu as sg

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Engine, Params

    torch.cuda.set_device(0)
    t_gen = time.perf_counter()
    wl = sg.batched(n_genomes=args.genomes or 50_000)
    eng = engine_for(args, 0)
    batch = eng.pack_device(wl.d_seq.data_ptr(), wl.offsets.astype(np.uint64), wl.genome_ids)
    ah.ah_ctx_synchronize(eng.ctx)
    gen_s = time.perf_counter() - t_gen
    del wl.d_seq
    torch.cuda.empty_cache()
    p = Params(wl.fwd, wl.rev, wl.k, wl.clamp, wl.min_len, wl.max_len, wl.orient_mask)
    stream = torch.cuda.ExternalStream(ah.ah_ctx_stream(eng.ctx))
    t0 = time.perf_counter()
    plan = eng.plan(batch, p, with_seqs=True, autotune=autotune(args), persistent=-1)
    plan_s = time.perf_counter() - t0
    info = ah.ah_plan_info_get(plan)
    for _ in range(max(3, warmup)):
        ah.ah_plan_run(plan, eng.ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ah.ah_ctx_stats_reset(eng.ctx)
    ah.ah_ctx_set_timing(eng.ctx, True)   # each replay's scan node between its own CUDA events
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(steps):
            ah.ah_plan_launch(plan, eng.ctx)
        e1.record(stream)
        torch.cuda.synchronize()
    ah.ah_ctx_set_timing(eng.ctx, False)
    ms = e0.elapsed_time(e1) / steps
    ah.ah_plan_check(plan, eng.ctx)
    info = ah.ah_plan_info_get(plan)
    st = ah.ah_ctx_stats_get(eng.ctx)
    launches_per_step = st["kernel_launches"] / steps
    scan_ms = st["scan_ms"] / st["scan_launches"]
    roof = scan_roofline(st["scan_ops_per_group"], wl.fwd, wl.rev, wl.clamp, wl.total_bp, scan_ms,
                         (info["threads"], info["groups_per_thread"], info["shift_mode"], info["persistent"]),
                         clk.summary().get("sm_mhz"), info["min_blocks"])
    pr = eng.primers(p)
    # the plain form: one launch per genome per pair
    ah.ah_ctx_stats_reset(eng.ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = ah.ah_scan_primers_per_record(eng.ctx, batch, pr)
    per_record_s = time.perf_counter() - t0
    n_pr = ah.ah_hits_count(h)
    ah.ah_hits_free(h)
    st2 = ah.ah_ctx_stats_get(eng.ctx)
    ah.ah_ctx_set_timing(eng.ctx, False)
    line = {"metric": METRIC, "workload": "batched", "value": wl.total_bp / (ms * 1e-3) / 1e9, "unit": "Gbp/s",
            "n_gpus": 1, "steps": steps, "warmup": max(3, warmup), "ms_per_step": ms,
            "higher_is_better": True, "dtype": "u32+f64", "data": "synthetic",
            "config": {"workload": f"batched: {wl.n_records} genomes log-uniform 10 kbp-12 Mbp, "
                                   f"{wl.total_bp / 1e9:.2f} Gbp, {len(wl.fwd)} pairs of 17-26 nt, k=i mod 4, "
                                   "graph-captured plan (scan, compaction, pairing, Tm, extraction)",
                       "bases": wl.total_bp, "patterns": 4 * len(wl.fwd)},
            "plan": {k: info[k] for k in ("threads", "groups_per_thread", "shift_mode", "persistent", "min_blocks",
                                          "vote_windows", "emit_queue", "grid", "n_hits", "n_amps", "arena_bytes")},
            "plan_create_s": plan_s, "autotune_ms": info["autotune_ms"], "generate_and_pack_s": gen_s,
            "scan_kernel_ms": scan_ms, "gpu_launches_per_step": launches_per_step,
            "roofline": roof,
            "plain_per_record": {"launches": st2["scan_launches"], "seconds": per_record_s,
                                 "gbps": wl.total_bp / per_record_s / 1e9, "hits": n_pr,
                                 "note": "scan stage only, one launch per genome per pair, wall clock"},
            "plan_speedup_vs_plain_scan": per_record_s / (ms * 1e-3),
            "clocks": clk.summary()}
    ah.ah_plan_free(plan)
    ah.ah_batch_free(batch)
    eng.close()
    torch.cuda.empty_cache()
    return line


# ------------------------------------------------------------------------------------------ serving arm
def run_serving(args):
    print(json.dumps(serving_record(args, [(args.requests, args.rate)])[0]), flush=True)


def serving_record(args, runs):
    """Poisson request streams against one device-resident database, continuous batching: one line
    per (requests, rate) in runs, each a fixed seeded trace."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth
    import synth.gpu as sg

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Engine

    torch.cuda.set_device(0)
    n_db = args.genomes or 40_000
    lengths, _ = sg.serving_layout(n_genomes=n_db)
    eng = engine_for(args, 0)
    t0 = time.perf_counter()
    db = ah.ah_batch_create(eng.ctx, np.asarray(lengths, dtype=np.uint64))
    for first, d, offs in sg.serving_db_chunks(n_genomes=n_db):
        ah.ah_batch_pack_range(eng.ctx, db, first, d.data_ptr(), offs.astype(np.uint64))
        del d
        torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t0
    db_bp = int(sum(lengths))
    lines = []
    for n_req, rate in runs:
        lines.append(_serve_trace(args, ah, db, n_db, db_bp, gen_s, n_req, rate))
    ah.ah_batch_free(db)
    eng.close()
    torch.cuda.empty_cache()
    return lines


def _serve_trace(args, ah, db, n_db, db_bp, gen_s, n_requests, rate):
    import numpy as np

    import synth

    trace = synth.serving_trace(synth.SEED, n_requests, rate, n_db)
    srv = ah.ah_server_create(db, n_slots=args.slots)
    ah.ah_server_set_scan_mode(srv, args.scan_mode)
    keys = ("fwd", "rev", "k", "clamp", "first_record", "n_records", "min_len", "max_len", "orient_mask")
    t_start = time.perf_counter()
    tickets = []
    with ClockSampler(0) as clk:
        for r in trace:
            delay = t_start + r["arrival"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(ah.ah_server_submit(srv, **{k: r[k] for k in keys}))
        res = [ah.ah_server_wait(srv, t) for t in tickets]
    ah.ah_server_destroy(srv)
    lat = np.array([x["t_done"] - x["t_submit"] for x in res])
    wait = np.array([x["t_admit"] - x["t_submit"] for x in res])
    span = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
    bases = sum(x["bases"] for x in res)
    pattern_bases = sum(x["bases"] * 4 * len(r["fwd"]) for x, r in zip(res, trace))
    line = {"metric": METRIC, "workload": "serving", "value": bases / span / 1e9, "unit": "Gbp/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"serving: {n_db} genomes ({db_bp / 1e9:.1f} Gbp, "
                                   f"{db_bp / 4e9:.1f} GB packed) resident; Poisson {rate} req/s, "
                                   f"{n_requests} requests of 1-32 pairs (17-26 nt, k 0-3) over contiguous "
                                   "subsets of 1-100 % of the database", "slots": args.slots,
                       "scan_mode": {0: "generated kernels (compiled per primer set)", 1: "generic kernel (no compile)",
                                     2: "generic kernel while the generated kernels compile"}[args.scan_mode]},
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "max": float(lat.max())},
            "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
            "completed": len(res), "makespan_s": span, "offered_rate": rate,
            "served_rate": len(res) / span, "pattern_gbp_per_s": pattern_bases / span / 1e9,
            "db_build_s": gen_s, "clocks": clk.summary()}
    if args.dump_requests:
        with open(args.dump_requests, "w") as f:
            json.dump([{"submit": x["t_submit"], "admit": x["t_admit"], "done": x["t_done"], "stages": x["t_stage"],
                        "bases": x["bases"],
                        "pairs": len(r["fwd"]), "hits": len(x["hits"]), "amps": len(x["amps"])}
                       for x, r in zip(res, trace)], f)
    return line


# ------------------------------------------------------------------------------------------ FASTQ reads arm
def run_reads(args):
    """Amplicon-sequencing reads end to end from FASTQ text in pinned host memory: ah_fastq_pack
    (copy, parse and pack on the device, qualities kept there), the whole step, the amplicons'
    qualities, and sites, amplicons, sequences and qualities copied to the host, every step."""
    import numpy as np
    import torch

    import __graft_entry__
    import synth

    __graft_entry__.build()
    from paper_2511_00170_gb300 import ah
    from paper_2511_00170_gb300.pipeline import Engine, Params

    torch.cuda.set_device(0)
    n_reads = args.genomes or 2_000_000
    text_np, wl = synth.amplicon_reads(n_reads=n_reads)
    text = torch.empty(text_np.nbytes, dtype=torch.uint8, pin_memory=True)
    text.numpy()[:] = text_np
    del text_np
    eng = engine_for(args, 0)
    p = Params.from_workload(wl)
    L = ah.load()
    pinned = {}

    def pinned_buf(name, nbytes):   # page-locked result buffers, grown when a step needs more
        if name not in pinned or pinned[name].numel() < nbytes:
            pinned[name] = torch.empty(int(nbytes * 1.25) + 4096, dtype=torch.uint8, pin_memory=True)
        return pinned[name]

    stages = {"fastq_ms": [], "step_ms": [], "qual_ms": [], "copy_ms": []}
    totals, counts = [], None
    with ClockSampler(0) as clk:
        for it in range(max(3, args.warmup) + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch, q, _ = ah.ah_fastq_pack(eng.ctx, text.data_ptr(), n_bytes=text.numel(), names=False)
            t1 = time.perf_counter()
            hits, amps = eng.step(batch, p, with_seqs=True, copy_out=False)
            ah.ah_ctx_synchronize(eng.ctx)
            t2 = time.perf_counter()
            ah.ah_extract_qualities(eng.ctx, q, batch, eng.primers(p), hits, amps)
            ah.ah_ctx_synchronize(eng.ctx)
            t3 = time.perf_counter()
            # sites, amplicons, sequences and qualities into page-locked host buffers
            nh, na, nb = ah.ah_hits_count(hits), ah.ah_amplicons_count(amps), ah.ah_amplicons_arena_size(amps)
            bh, ba = pinned_buf("hits", nh * 12 + 1), pinned_buf("amps", na * 32 + 1)
            bs, bo, bq = pinned_buf("seq", nb + 1), pinned_buf("off", (5 * na + 1) * 8), pinned_buf("qual", nb + 1)
            for st in (L.ah_hits_copy(hits, bh.data_ptr(), nh), L.ah_amplicons_copy(amps, ba.data_ptr(), na),
                       L.ah_amplicons_seq_copy(amps, bs.data_ptr(), nb, bo.data_ptr(), 5 * na + 1),
                       L.ah_amplicons_qual_copy(amps, bq.data_ptr(), nb)):
                if st:
                    raise RuntimeError(f"copy failed: {st}")
            t4 = time.perf_counter()
            ah.ah_hits_free(hits), ah.ah_amplicons_free(amps), ah.ah_quals_free(q), ah.ah_batch_free(batch)
            if it >= max(3, args.warmup):
                for k, v in zip(stages, (t1 - t0, t2 - t1, t3 - t2, t4 - t3)):
                    stages[k].append(v * 1e3)
                totals.append(t4 - t0)
                counts = (nh, na, 2 * nb)
    eng.close()
    ms = statistics.median(totals) * 1e3
    line = {"metric": METRIC, "workload": "amplicon_reads", "value": wl.total_bp / (ms * 1e-3) / 1e9, "unit": "Gbp/s",
            "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "data": "synthetic", "dtype": "u32+f64",
            "config": {"workload": f"amplicon_reads: {n_reads} FASTQ reads of 300 bp ({wl.total_bp / 1e9:.2f} Gbp, "
                                   f"{text.numel() / 1e9:.2f} GB of text), the plain primer pair, k=2, trim, "
                                   "qualities propagated", "reads": n_reads},
            "e2e": {"value": wl.total_bp / (ms * 1e-3) / 1e9, "unit": "Gbp/s", "h2d_bytes_per_step": int(text.numel()),
                    "d2h_bytes_per_step": counts[0] * 12 + counts[1] * 32 + counts[2] if counts else 0,
                    "path": "pinned FASTQ text -> ah_fastq_pack -> scan, pairing, Tm, extraction -> "
                            "ah_extract_qualities -> sites, amplicons, sequences and qualities into pinned host buffers"},
            "stages_ms": {k: statistics.median(v) for k, v in stages.items()},
            "sites": counts[0] if counts else 0, "amplicons": counts[1] if counts else 0, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--workload", default="plain_scale")
    ap.add_argument("--genomes", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-fasta", action="store_true",
                    help="also time end to end from FASTA text (80-column lines) parsed and packed on the device")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--dump-requests", default="", help="serving: write per-request times to this JSON file")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the batched, dense and serving sub-records")
    ap.add_argument("--serve-requests", type=int, default=40, help="sub-record: requests of the stable-rate trace")
    ap.add_argument("--serve-rate", type=float, default=3.0, help="sub-record: arrival rate of the stable trace")
    ap.add_argument("--serve-burst", type=int, default=100, help="sub-record: requests offered at 200 req/s")
    ap.add_argument("--tm-kernel", default="generated", choices=sorted(TM_KERNELS),
                    help="degenerate-site Tm: the kernel generated per primer set, or the built-in one")
    ap.add_argument("--tm-split", type=int, default=0,
                    help="site count from which the generated Tm kernel runs once per group of primers "
                         "(0: the library's default)")
    ap.add_argument("--scan-fixed", default="",
                    help="threads,groups,shift_mode,min_blocks,vote_windows,emit_queue: plans take this scan kernel "
                         "instead of autotuning (for profiling one kernel)")
    ap.add_argument("--scan-mode", type=int, default=2,
                    help="serving: 0 generated scan kernels, 1 generic kernel, 2 generic while compiling")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "amplicon_reads":
        run_reads(args)
    elif args.workload == "dense_step":
        print(json.dumps(dense_record(args, args.steps, args.warmup)), flush=True)
    else:
        run_engine(args)


if __name__ == "__main__":
    main()
