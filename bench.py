"""Benchmark of the px hot path: hash exchange -> per-partition hash join ->
Partial/Final hash aggregation, on the at-scale workload (60M-row fact with
Zipf(1.1) keys over a 2M-row dimension, 64 partitions, group-by on a 10k-valued
attribute), one step = one full pass of the pipeline over the batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl px|reference]

Prints ONE JSON line (rank 0). `value` is whole-job fact rows per second with the
inputs resident in HBM; `e2e` is the same metric through the same public calls
with host inputs copied in (pinned memory) and the final groups copied out every
step. `operators` breaks the step down per C-ABI call (rows/s and fraction of the
measured HBM copy bandwidth on algorithmic bytes). `roofline` is the dominant
call, the fact-side exchange (px_partition: histogram + scan + scatter kernels).
`cpu_baseline` is the CPU oracle timed on this host on a bounded sample.

`--impl reference` times the CPU oracle (the only reference implementation of
this path) on the same workload and metric, on bounded samples per step.

With N > 1 (torchrun, one process per GPU) every rank runs an independent replica
on its own seeded shard of fact rows (weak scaling, no data-path collective);
ranks meet only at the timing barriers and the max-over-ranks reduction.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pxdata  # noqa: E402

METRIC = "rows/s & % HBM peak per operator; served QPS + p50/p99 vs one-at-a-time"
WORKLOAD = ("plain at scale: 60M-row fact (fk Zipf s=1.1 over 2M pks, amount int64, date int32) x 2M-row dim "
            "(pk int64, attr int32 over 10k values); exchange both sides into 64 partitions, per-partition "
            "join build+probe, Partial group-by attr per partition, Final merge")
NFACT, NDIM, NATTR, NPARTS = 60_000_000, 2_000_000, 10_000, 64

# Algorithmic bytes per unit of each call:
#   partition: read every column + write every column       (fact 20+20 B/row, dim 12+12 B/row)
#   build:     read the key + write the 2 table slots per row (8 + 32 B/dim row)
#   probe:     read fk + amount, write amount + attr          (16 + 12 B/fact row)
#   partial:   read amount + attr                             (12 B/joined row)
#   final:     read attr + 2 partial aggregates                (20 B/partial group)


def alg_bytes(nf, nd, npartial):
    return {
        "px_partition(dim)": 24 * nd,
        "px_partition(fact)": 40 * nf,
        "px_join_build": 40 * nd,
        "px_join_probe": 28 * nf,
        "px_groupby_agg(partial)": 12 * nf,
        "px_groupby_agg(final)": 20 * npartial,
    }


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_seed(rank: int) -> int:
    """Seed of a rank's fact shard: rank 0 draws the single-GPU workload itself."""
    return 3 + 1000 * rank


def reduce_max(value: float, group=None) -> float:
    """Max over ranks of a host float (timing only; no data-path collective)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def whole_job_rate(rows_per_rank: int, world: int, seconds_max: float) -> float:
    """Units all ranks processed / the slowest rank's time."""
    return rows_per_rank * world / seconds_max


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def ncu_traffic(kernel_src: str):
    """DRAM bytes per launch of the dominant call from the committed ncu summary, or
    None once the kernel source has changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as f:
        d = json.load(f)
    src = os.path.join(ROOT, kernel_src)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if d.get("source_sha256_16") != h:
        return None, d.get("source_sha256_16")
    return d.get("traffic_bytes_per_launch"), h


# ---------------------------------------------------------------- oracle ----

def oracle_rate(d: dict, nsample: int) -> tuple[float, str]:
    """The CPU oracle (single-threaded, as it stands) on the first `nsample` fact rows
    with the whole dimension: returns (fact rows/s, description)."""
    import oracle
    s = {"pk": d["pk"], "attr": d["attr"], "fk": d["fk"][:nsample], "amount": d["amount"][:nsample],
         "date": d["date"][:nsample]}
    t0 = time.perf_counter()
    oracle.pipeline_at_scale(s, NPARTS)
    dt = time.perf_counter() - t0
    return nsample / dt, f"first {nsample} fact rows x full {d['pk'].size}-row dim, {dt:.1f} s"


def host_cpu() -> dict:
    """This host's logical core count and CPU model (stated beside every CPU timing)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"host_cores": os.cpu_count(), "cpu_model": model or platform.machine()}


def merge_final(parts: list) -> tuple:
    """Final groups of per-chunk at-scale answers merged by key (sums mod 2^64)."""
    keys = np.concatenate([p["final"]["keys"][0] for p in parts])
    aggs = [np.concatenate([p["final"]["aggs"][a] for p in parts]).view(np.uint64) for a in range(2)]
    order = np.argsort(keys, kind="stable")
    keys = keys[order]
    starts = np.flatnonzero(np.r_[True, keys[1:] != keys[:-1]])
    return keys[starts], [np.add.reduceat(a[order], starts).view(np.int64) for a in aggs]


def oracle_rate_all_cores(d: dict, nsample: int, threads: int) -> tuple[float, str]:
    """The CPU oracle on all host cores: the first `nsample` fact rows split into one
    chunk per thread, each chunk through the whole at-scale pipeline with the full
    dimension (the oracle's C calls release the interpreter lock), then the chunks'
    Final groups merged by key. A labelled extra beside the single-threaded
    oracle, which stays the correctness reference."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    bounds = np.linspace(0, nsample, threads + 1).astype(np.int64)
    chunks = [{"pk": d["pk"], "attr": d["attr"], "fk": d["fk"][a:b], "amount": d["amount"][a:b],
               "date": d["date"][a:b]} for a, b in zip(bounds[:-1], bounds[1:])]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda c: oracle.pipeline_at_scale(c, NPARTS), chunks))
    merge_final(parts)
    dt = time.perf_counter() - t0
    return nsample / dt, f"first {nsample} fact rows in {threads} chunks x full {d['pk'].size}-row dim, {dt:.1f} s"


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    oracle.build()
    d = pxdata.plain_at_scale(NDIM, NFACT, NATTR, seed=shard_seed(0))
    # size each step's sample so the whole run stays within ~2 minutes
    probe_rate, _ = oracle_rate(d, 200_000)
    per_step_s = min(10.0, 120.0 / max(1, args.steps + args.warmup))
    nsample = int(min(NFACT, max(100_000, probe_rate * per_step_s * 0.8)))
    for _ in range(args.warmup):
        oracle_rate(d, nsample)
    rates, desc = [], ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, desc = oracle_rate(d, nsample)
        rates.append(r)
    total = time.perf_counter() - t0
    value = nsample * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded numpy PCG64; TPC-H-like shapes, no TPC-H data)",
            "config": {"workload": WORKLOAD, "fact_rows": NFACT, "dim_rows": NDIM, "nparts": NPARTS,
                       "reference": "CPU oracle (plain single-threaded C++: stable-sort partition, sorted-build "
                                    "join, ordered-map group-by), bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "kind": "oracle",
                             "sample": f"per step: {desc.split(',')[0]}", **host_cpu()},
            "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


# -------------------------------------------------------------------- px ----

def same_final(host_out: dict, fin: dict) -> bool:
    """The end-to-end run's final groups (copied to pinned host buffers) equal the
    resident run's: same count, and the same (key, SUM, COUNT) rows in key order."""
    n = int(host_out["n"].item())
    if n != int(fin["ngroups"].item()):
        return False
    k1 = host_out["keys"][:n].numpy().astype(np.int64)
    k2 = fin["keys"][0][:n].cpu().numpy().astype(np.int64)
    o1, o2 = np.argsort(k1, kind="stable"), np.argsort(k2, kind="stable")
    return (np.array_equal(k1[o1], k2[o2]) and
            np.array_equal(host_out["sum"][:n].numpy()[o1], fin["aggs"][0][:n].cpu().numpy()[o2]) and
            np.array_equal(host_out["cnt"][:n].numpy()[o1], fin["aggs"][1][:n].cpu().numpy()[o2]))


def run_px(args):
    import torch
    import torch.distributed as dist

    import paper_2606_24647_gb300 as px
    from paper_2606_24647_gb300.pipelines import AtScalePipeline

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    px.load()
    dev = torch.device("cuda", torch.cuda.current_device())

    d = pxdata.plain_at_scale(NDIM, NFACT, NATTR, seed=shard_seed(rank))
    host = {k: torch.from_numpy(v).pin_memory() for k, v in d.items()}
    dd = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
    torch.cuda.synchronize()
    # exchange launch shapes for this GPU and these inputs (cached per GPU)
    from paper_2606_24647_gb300 import autotune
    tag = f"{NFACT}x{NDIM}p{NPARTS}"
    fcfg = autotune.tune_partition([dd["fk"], dd["amount"], dd["date"]], 0, NPARTS, f"fact{tag}")
    dcfg = autotune.tune_partition([dd["pk"], dd["attr"]], 0, NPARTS, f"dim{tag}")
    pipe = AtScalePipeline(dd, nparts=NPARTS, nattr_bound=NATTR, fact_config=fcfg, dim_config=dcfg)
    stream = torch.cuda.current_stream()

    ops = list(alg_bytes(1, 1, 1).keys())
    assert ops == AtScalePipeline.CALLS

    def step(ev=None):
        """One pass of the pipeline; ev: list of 7 events recorded between the calls."""
        r = pipe.run(stream, mark=(lambda i: ev[i].record(stream)) if ev else None)
        return r["partial"], r["final"]

    # correctness gate on this exact configuration before timing
    part, fin = step()
    st = pipe.ws.status(stream)
    if st != px.PX_OK:
        raise RuntimeError(f"device status {st} in the benchmarked pipeline")
    npartial = int(part["ngroups"].item())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, per-call events, inputs (1.2 GB) larger than L2 ----
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.15)
    launches0 = px.kernel_launches()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = px.kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    if pipe.ws.status(stream) != px.PX_OK:
        raise RuntimeError("device status set during the timed region")

    per_op_ms = {op: 0.0 for op in ops}
    for k in range(args.steps):
        for i, op in enumerate(ops):
            per_op_ms[op] += evs[k][i].elapsed_time(evs[k][i + 1])
    for op in ops:
        per_op_ms[op] /= args.steps
    max_total_s = reduce_max(total_ms / 1000.0)
    ms_per_step = 1000 * max_total_s / args.steps
    value = whole_job_rate(NFACT * args.steps, world, max_total_s)

    peak, peak_kind = measured_peaks()
    ab = alg_bytes(NFACT, NDIM, npartial)
    rows = {"px_partition(dim)": NDIM, "px_partition(fact)": NFACT, "px_join_build": NDIM, "px_join_probe": NFACT,
            "px_groupby_agg(partial)": NFACT, "px_groupby_agg(final)": npartial}
    operators = {}
    for op in ops:
        s = per_op_ms[op] / 1000
        gbs = ab[op] / s / 1e9
        operators[op] = {"ms": round(per_op_ms[op], 4), "rows_per_s": rows[op] / s, "alg_bytes": ab[op],
                         "GBps": round(gbs, 1), "hbm_frac": round(gbs / peak, 4)}
    # The dominant kernel of the step is part_scatter_kernel (the largest share of
    # the ncu launch list); it runs inside the fact-side px_partition call, which is
    # timed as a whole (hist + scan + scatter).
    dom = "px_partition(fact)"
    traffic, _ = ncu_traffic("paper_2606_24647_gb300/csrc/px_partition.cu")
    dom_gbs = ab[dom] / (per_op_ms[dom] / 1000) / 1e9
    roofline = {"bound": "hbm", "achieved": round(dom_gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(dom_gbs / peak, 4), "traffic": traffic,
                "kernel": "px_partition on the 60M-row fact (hist + scan + scatter kernels, one C-ABI call); "
                          "part_scatter_kernel is the step's largest kernel",
                "alg_bytes_per_launch": ab[dom], "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)"}

    # ---- the same pipeline with the probe and Partial aggregation fused ----
    fpipe = AtScalePipeline(dd, nparts=NPARTS, nattr_bound=NATTR, fused=True, fact_config=fcfg, dim_config=dcfg)
    fr = fpipe.run(stream)
    torch.cuda.synchronize()
    if fpipe.ws.status() != px.PX_OK:
        raise RuntimeError("device status set in the fused pipeline")
    nfin = int(fr["final"]["ngroups"].item())
    if nfin != int(fin["ngroups"].item()) or not all(
            torch.equal(torch.sort(x[:nfin])[0], torch.sort(y[:nfin])[0])
            for x, y in zip(fr["final"]["aggs"] + fr["final"]["keys"], fin["aggs"] + fin["keys"])):
        raise RuntimeError("fused and unfused pipelines disagree")
    for _ in range(args.warmup):
        fpipe.run(stream)
    fcalls = AtScalePipeline.CALLS_FUSED
    fev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fcalls) + 1)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        fpipe.run(stream, mark=lambda i, k=k: fev[k][i].record(stream))
    torch.cuda.synchronize()
    f_ms = sum(fev[k][0].elapsed_time(fev[k][-1]) for k in range(args.steps)) / args.steps
    f_max_s = reduce_max(f_ms / 1000.0)
    fused = {"value": whole_job_rate(NFACT, world, f_max_s), "unit": "rows/s", "ms_per_step": round(f_ms, 4),
             "operators_ms": {c: round(sum(fev[k][i].elapsed_time(fev[k][i + 1]) for k in range(args.steps)) /
                                       args.steps, 4) for i, c in enumerate(fcalls)},
             "note": "px_join_probe + px_groupby_agg(partial) replaced by px_join_probe_agg (join output never "
                     "written); same final groups (checked)"}

    # ---- end to end through the same public calls, host buffers in and out ----
    # Every step copies its five input columns from pinned host memory and reads
    # its final groups back. Two device input sets and a copy stream let step k+1's
    # upload run while step k computes (the copies, ~210 GB/s host-to-device, take
    # longer than the compute), so a step costs max(copy, compute), not the sum.
    e2e_steps = max(3, min(20, args.steps // 10))
    dd2 = {k: torch.empty_like(v) for k, v in dd.items()}
    pipes = [pipe, AtScalePipeline(dd2, nparts=NPARTS, nattr_bound=NATTR, fact_config=fcfg, dim_config=dcfg)]
    dsets = [dd, dd2]
    outs = [{"keys": torch.empty(pipe.max_final, dtype=torch.int32).pin_memory(),
             "sum": torch.empty(pipe.max_final, dtype=torch.int64).pin_memory(),
             "cnt": torch.empty(pipe.max_final, dtype=torch.int64).pin_memory(),
             "n": torch.empty(1, dtype=torch.int64).pin_memory()} for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in outs[0].values())
    cstream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    computed = [torch.cuda.Event() for _ in range(2)]

    def upload(k):
        b = k % 2
        if k >= 2:
            cstream.wait_event(computed[b])  # step k-2 is done with this input set
        with torch.cuda.stream(cstream):
            for name, v in host.items():
                dsets[b][name].copy_(v, non_blocking=True)
        copied[b].record(cstream)

    def e2e_run(nsteps):
        upload(0)
        for k in range(nsteps):
            if k + 1 < nsteps:
                upload(k + 1)
            b = k % 2
            stream.wait_event(copied[b])
            f = pipes[b].run(stream)["final"]
            o = outs[b]
            o["keys"].copy_(f["keys"][0], non_blocking=True)
            o["sum"].copy_(f["aggs"][0], non_blocking=True)
            o["cnt"].copy_(f["aggs"][1], non_blocking=True)
            o["n"].copy_(f["ngroups"], non_blocking=True)
            computed[b].record(stream)

    e2e_run(2)
    torch.cuda.synchronize()
    runs = []
    for _ in range(3):  # three timed runs of e2e_steps steps; the median is reported
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_run(e2e_steps)
        torch.cuda.synchronize()
        runs.append(reduce_max(time.perf_counter() - t0))
    e2e_s = statistics.median(runs)
    e2e_value = whole_job_rate(NFACT * e2e_steps, world, e2e_s)
    if pipe.ws.status(stream) != px.PX_OK or pipes[1].ws.status(stream) != px.PX_OK:
        raise RuntimeError("device status set during the end-to-end run")
    if not same_final(outs[0], fin):
        raise RuntimeError("end-to-end result differs")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        hc = host_cpu()
        rate, desc = oracle_rate(d, min(NFACT, args.cpu_sample))
        cpu = {"value": rate, "unit": "rows/s", "cores": 1, "kind": "oracle", "sample": desc, **hc}
        if hc["host_cores"] and hc["host_cores"] > 1:
            arate, adesc = oracle_rate_all_cores(d, min(NFACT, args.cpu_sample), hc["host_cores"])
            cpu["all_cores"] = {"value": arate, "unit": "rows/s", "cores": hc["host_cores"],
                                "kind": "oracle, per-thread chunks + merge of the Final groups", "sample": adesc}

    line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded numpy PCG64; TPC-H-like shapes, no TPC-H data)",
            "config": {"workload": WORKLOAD, "fact_rows": NFACT, "dim_rows": NDIM, "nparts": NPARTS,
                       "attr_values": NATTR, "zipf_s": 1.1, "per_gpu_fact_rows": NFACT,
                       "l2": "inputs larger than L2 (1.22 GB of fact+dim columns per step vs 129 MB L2)",
                       "parallelism": f"replicas x{world} (independent seeded shards)",
                       "tuned_partition": {"fact": dict(zip(("items", "blocks_per_sm"), fcfg)),
                                           "dim": dict(zip(("items", "blocks_per_sm"), dcfg))}},
            "operators": operators, "roofline": roofline, "fused_probe_partial": fused, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "rows/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "runs_s": [round(x, 5) for x in runs],
                    "clock": "host wall clock around each synchronised run; median of three",
                    "overlap": "step k+1's host-to-device upload runs on a copy stream during step k's compute"},
            "gpu_launches": launches, "clocks": clk}
    if world > 1:
        dist.destroy_process_group()
    return line if rank == 0 else None


# ------------------------------------------------ batched fragments workload ----
FRAG_N = 512
FRAG_WORKLOAD = ("512 batched fragments: fact rows log-uniform [1e4, 4e6] (sum ~341M), build rows log-uniform "
                 "[1e3, 1e6], group domain log-uniform [4, 1e5]; per fragment filter date in [895, 1662) -> join "
                 "key = pk (~5% of keys miss) -> group by dim.attr: SUM(price), SUM(price*qty), COUNT(*)")


def build_fragments(nfrags: int, scale: float):
    from paper_2606_24647_gb300.pipelines import FragmentSet
    sz = pxdata.fragment_sizes(nfrags, seed=4, scale=scale)
    datas = [pxdata.fragment(int(sz["nfact"][i]), int(sz["nbuild"][i]), int(sz["ngroups"][i]), seed=10_000 + i)
             for i in range(nfrags)]
    fs = FragmentSet(datas, [int(g) for g in sz["ngroups"]], pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI)
    return fs, datas


def _time_steps(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1000.0 / steps


def run_fragments(args):
    """Config 4: the fused batch (one persistent kernel + emit) against the same
    fragments one at a time through the unfused calls."""
    import torch
    import paper_2606_24647_gb300 as px
    from paper_2606_24647_gb300 import autotune
    from paper_2606_24647_gb300.pipelines import OneAtATime

    torch.cuda.set_device(0)
    px.load()
    stream = torch.cuda.current_stream()
    fs, _ = build_fragments(args.fragments, args.frag_scale)
    torch.cuda.synchronize()
    batch = fs.batch()
    workload = f"fragments{args.fragments}x{args.frag_scale:g}"
    cfg = autotune.tune_fragments(batch, workload)
    batch.cfg = px.px_fragments_config(*cfg)
    one = OneAtATime(fs)
    # consistency: the fused batch equals the one-at-a-time calls on every fragment
    res = batch.run(stream)
    ref = one.run(stream)
    torch.cuda.synchronize()
    if batch.ws.status() != px.PX_OK or one.ws.status() != px.PX_OK:
        raise RuntimeError("device status set in the fragments workload")
    for r, q in zip(res, ref):
        n = int(r["ngroups"].item())
        if n != int(q["ngroups"].item()):
            raise RuntimeError("fused and one-at-a-time group counts differ")
        o1 = torch.argsort(r["keys"][:n].long())
        o2 = torch.argsort(q["keys"][0][:n].long())
        if not (torch.equal(r["keys"][:n].long()[o1], q["keys"][0][:n].long()[o2]) and
                all(torch.equal(x[:n][o1], y[:n][o2]) for x, y in zip(r["aggs"], q["aggs"]))):
            raise RuntimeError("fused and one-at-a-time results differ")
    launches0 = px.kernel_launches()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.15)
    t_fused = _time_steps(lambda: batch.run(stream), args.steps, args.warmup, stream)
    clk = clocks.stop()
    fused_launches = (px.kernel_launches() - launches0) // (args.steps + args.warmup)
    launches0 = px.kernel_launches()
    ones = max(3, args.steps // 10)
    t_one = _time_steps(lambda: one.run(stream), ones, 3, stream)
    one_launches = (px.kernel_launches() - launches0) // (ones + 3)
    peak, peak_kind = measured_peaks()
    # algorithmic bytes per fact row: date 4 + key 8 + price 8 + qty 8 read once
    alg = 28 * fs.rows
    line = {"metric": "fact rows/s over a batch of fused filter->probe->aggregate fragments",
            "value": fs.rows / t_fused, "unit": "rows/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * t_fused, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded numpy PCG64; TPC-H-like shapes, no TPC-H data)",
            "config": {"workload": FRAG_WORKLOAD if args.frag_scale == 1 else
                       f"REDUCED x{args.frag_scale:g}: " + FRAG_WORKLOAD,
                       "fragments": args.fragments, "fact_rows": fs.rows,
                       "tuned_launch": dict(zip(("threads", "items", "chunk_rows", "blocks_per_sm"), cfg)),
                       "l2": f"inputs larger than L2 ({alg / 1e9:.1f} GB of fact columns per step)"},
            "one_at_a_time": {"value": fs.rows / t_one, "unit": "rows/s", "ms_per_step": round(1000 * t_one, 4),
                              "kernel_launches_per_step": one_launches, "steps": ones},
            "speedup_vs_one_at_a_time": t_one / t_fused,
            "roofline": {"bound": "hbm", "achieved": round(alg / t_fused / 1e9, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(alg / t_fused / 1e9 / peak, 4), "traffic": None,
                         "kernel": "frag_kernel (fused) + frag_emit_kernel, one px_fragments_run",
                         "alg_bytes_per_launch": alg, "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)"},
            "gpu_launches": fused_launches * args.steps, "clocks": clk,
            "check": "fused batch == one-at-a-time calls on every fragment (keys and aggregates)"}
    del batch, one, fs
    return line


# ------------------------------------------- plain and plain-join workloads ----
L2_BYTES = 129 * 1024 * 1024
SMALL_WORKLOADS = {
    "plain": ("plain: 1M rows (key int64 U[0,2^20), price int64, qty int64, date int32 U[0,2557), flag int8, "
              "status int8); filter date < 2506 (98.0 %) -> exchange on key into 8 partitions -> group by "
              "(flag, status): SUM(price), SUM(price*qty), SUM(qty), COUNT(*)"),
    "plain-join": ("plain join: 6M-row fact (fk U[1,200000], amount int64, date int32) x 200k-row dim (pk "
                   "permutation, attr int32 U[0,25)); filter date in [895, 1662) (30.0 %) -> build on pk -> probe "
                   "fk (carry amount, gather attr) -> group by attr: SUM(amount), COUNT(*)"),
}


def _small_pipeline(which: str, d: dict):
    from paper_2606_24647_gb300.pipelines import JoinPipeline, PlainPipeline
    if which == "plain":
        return PlainPipeline(d, pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, nparts=pxdata.CFG1_PARTS)
    return JoinPipeline(d, pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI)


def _small_alg_bytes(which: str, n: dict) -> dict:
    """Algorithmic bytes per call: every input column read once and every output written
    once (a second read of the exchange key is not counted)."""
    if which == "plain":
        return {"px_filter": 4 * n["rows"] + 4 * n["sel"],
                "px_partition": (4 + 30 + 30) * n["sel"],      # sel, 30-byte row read and written
                "px_groupby_agg": 18 * n["sel"]}               # flag 1 + status 1 + price 8 + qty 8
    return {"px_filter": 4 * n["rows"] + 4 * n["sel"],
            "px_join_build": 40 * n["dim"],                    # pk 8 + attr 4 read, 28 B of table per row
            "px_join_probe": 20 * n["rows"] + 12 * n["out"],   # sel 4 + fk 8 + amount 8 (every sector), 12 B out
            "px_groupby_agg": 12 * n["out"]}                   # attr 4 + amount 8


def _small_counts(which: str, p, res) -> dict:
    if which == "plain":
        return {"rows": int(p.d["key"].numel()), "sel": int(res["nsel"].item())}
    return {"rows": int(p.d["fk"].numel()), "dim": int(p.d["pk"].numel()), "sel": int(res["nsel"].item()),
            "out": int(res["join"]["nout"].item())}


def oracle_check_small(which: str, host: dict, res: dict) -> str:
    """The small pipeline's result against the CPU oracle on the same input: the
    selection count, the exchange offsets (plain) or the join count (plain join),
    and every group (keys and aggregates, in key order)."""
    import oracle
    if which == "plain":
        w = oracle.pipeline_plain(host, pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, pxdata.CFG1_PARTS)
        ok = int(res["nsel"].item()) == w["sel"].size and np.array_equal(res["offsets"].cpu().numpy(), w["offsets"])
    else:
        w = oracle.pipeline_join(host, pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI)
        ok = int(res["nsel"].item()) == w["sel"].size and int(res["join"]["nout"].item()) == w["probe_rows"].size
    g = res["groups"]
    n = int(g["ngroups"].item())
    keys = [t[:n].cpu().numpy().astype(np.int64) for t in g["keys"]]
    order = np.lexsort(tuple(reversed(keys)))
    ok = ok and n == w["groups"]["ngroups"]
    ok = ok and all(np.array_equal(k[order], wk) for k, wk in zip(keys, w["groups"]["keys"]))
    ok = ok and all(np.array_equal(a[:n].cpu().numpy()[order], wa) for a, wa in zip(g["aggs"], w["groups"]["aggs"]))
    if not ok:
        raise RuntimeError(f"{which}: GPU pipeline differs from the CPU oracle")
    return "equal to the CPU oracle (selection count, " + ("exchange offsets" if which == "plain" else "join count") + \
           ", every group's keys and aggregates)"


def _same_groups(a: dict, b: dict) -> bool:
    """Equal group sets (group order is not part of the result)."""
    def rows(g):
        n = int(g["ngroups"].item())
        return sorted(zip(*[t[:n].tolist() for t in list(g["keys"]) + list(g["aggs"])]))
    return rows(a) == rows(b)


def run_small(args):
    """Configs 1 and 2 (the 1M-row plain and 6M-row plain-join pipelines, whose inputs
    fit in L2): per call, the cold protocol (a buffer of 2.5x L2 written before every
    timed call, median over the reps); for the whole pipeline, back-to-back steps on
    distinct input copies (more than 4x L2 in total) replayed from one captured CUDA
    graph, so neither launch gaps nor L2 hits decide the number."""
    import torch
    import paper_2606_24647_gb300 as px

    which = args.workload
    torch.cuda.set_device(0)
    px.load()
    dev = torch.device("cuda", 0)
    host = pxdata.plain(1_000_000, seed=0) if which == "plain" else pxdata.plain_join(seed=2)
    d = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    stream = torch.cuda.current_stream()
    p = _small_pipeline(which, d)
    ref = p.run(stream)
    torch.cuda.synchronize()
    if p.ws.status() != px.PX_OK:
        raise RuntimeError("device status set in the pipeline")
    counts = _small_counts(which, p, ref)
    alg = _small_alg_bytes(which, counts)
    in_bytes = sum(t.numel() * t.element_size() for t in d.values())

    # cold protocol, per call
    flush = torch.empty(int(2.5 * L2_BYTES), dtype=torch.uint8, device=dev)
    reps = max(20, min(args.steps, 200))
    steps = p.steps(stream)
    times = {name: [] for name, _ in steps}
    evs = []
    for r in range(reps + 3):
        for name, f in steps:
            flush.fill_(r & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f()
            b.record(stream)
            if r >= 3:
                evs.append((name, a, b))
    torch.cuda.synchronize()
    for name, a, b in evs:
        times[name].append(a.elapsed_time(b) / 1000.0)
    peak, peak_kind = measured_peaks()
    ops = {}
    for name, _ in steps:
        t = statistics.median(times[name])
        ops[name] = {"ms_median_cold": round(1000 * t, 4), "rows_per_s": counts["rows"] / t,
                     "alg_bytes": alg[name], "GBps": round(alg[name] / t / 1e9, 1),
                     "hbm_frac": round(alg[name] / t / 1e9 / peak, 4)}
    cold_ms = sum(v["ms_median_cold"] for v in ops.values())

    # back-to-back steps over distinct copies, one CUDA graph
    copies = int(np.ceil(4 * L2_BYTES / in_bytes)) + 1
    pipes = [p] + [_small_pipeline(which, {k: v.clone() for k, v in d.items()}) for _ in range(copies - 1)]
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for q in pipes:
            q.run(side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    launches0 = px.kernel_launches()
    with torch.cuda.graph(graph):
        outs = [q.run() for q in pipes]
    per_replay = px.kernel_launches() - launches0
    gs = torch.cuda.current_stream()
    graph.replay()
    torch.cuda.synchronize()
    if any(q.ws.status() != px.PX_OK for q in pipes) or not all(_same_groups(o["groups"], ref["groups"])
                                                                 for o in outs):
        raise RuntimeError("graph replay results differ from the eager pipeline")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(gs)
    for _ in range(args.warmup):
        graph.replay()
    b.record(gs)
    torch.cuda.synchronize()
    t_replay = a.elapsed_time(b) / 1000.0 / args.warmup
    # enough replays for the clock samples (every 50 ms) to fall inside the timed region
    nrep = max(5, args.steps // copies, int(np.ceil(0.4 / t_replay)))
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.15)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(gs)
    for _ in range(nrep):
        graph.replay()
    b.record(gs)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_graph = a.elapsed_time(b) / 1000.0 / nrep / copies          # seconds per pipeline step
    top = max(ops, key=lambda k: ops[k]["ms_median_cold"])

    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        if which == "plain":
            oracle.pipeline_plain(host, pxdata.CFG1_DATE_LO, pxdata.CFG1_DATE_HI, pxdata.CFG1_PARTS)
        else:
            oracle.pipeline_join(host, pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI)
        dt = time.perf_counter() - t0
        cpu = {"value": counts["rows"] / dt, "unit": "rows/s", "cores": 1, "kind": "oracle",
               "sample": f"the whole {counts['rows']}-row input, one pipeline pass, {dt:.2f} s", **host_cpu()}
    line = {"metric": "rows/s & % HBM peak per operator", "value": counts["rows"] / t_graph, "unit": "rows/s",
            "n_gpus": 1, "steps": nrep * copies, "warmup": args.warmup, "ms_per_step": round(1000 * t_graph, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded numpy PCG64; TPC-H-like shapes, no TPC-H data)",
            "config": {"workload": SMALL_WORKLOADS[which], "rows": counts["rows"], "input_bytes": in_bytes,
                       "l2": f"graph stream over {copies} distinct input copies ({copies * in_bytes / 1e6:.0f} MB, "
                             f"> 4x the 129 MB L2); per-call times under a 2.5x-L2 flush before every call"},
            "operators_cold": ops, "pipeline_cold_ms": round(cold_ms, 4),
            "graph_stream": {"copies": copies, "replays": nrep, "ms_per_step": round(1000 * t_graph, 4),
                             "rows_per_s": counts["rows"] / t_graph, "kernels_per_step": per_replay / copies},
            "roofline": {"bound": "hbm", "achieved": ops[top]["GBps"], "peak": peak, "unit": "GB/s",
                         "frac": ops[top]["hbm_frac"], "traffic": None,
                         "kernel": f"{top} (the pipeline's longest call, cold protocol)",
                         "alg_bytes_per_launch": alg[top], "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)"},
            "gpu_launches": per_replay * nrep, "clocks": clk}
    if cpu:
        line["cpu_baseline"] = cpu
    line["check"] = oracle_check_small(which, host, ref)
    return line


# ------------------------------------------------ late materialization ----
LATE_WORKLOAD = ("selective join over a wide fact: 60M-row fact (fk Zipf s=1.1 over 2M pks, amount, price, qty "
                 "int64, date int32) x the 2M-row dim's rows with attr < 1000 (about 10 %); exchange both into 64 "
                 "partitions, per-partition join, Partial group-by attr: SUM(amount), SUM(price*qty), COUNT, Final")


def run_late_mat(args):
    """NEXT 4: the same selective join eagerly (exchange fk + amount + price + qty)
    and late-materialized (exchange fk + row id, gather the payload after the join)."""
    import torch
    import paper_2606_24647_gb300 as px
    from paper_2606_24647_gb300.pipelines import WideJoinPipeline

    torch.cuda.set_device(0)
    px.load()
    stream = torch.cuda.current_stream()
    nf = args.fact_rows or NFACT
    d = pxdata.wide_at_scale(NDIM, nf, NATTR, build_attr_below=1_000)
    dd = {k: torch.from_numpy(v).cuda() for k, v in d.items()}
    torch.cuda.synchronize()
    out = {}
    finals = {}
    for name, late in (("eager", False), ("late", True)):
        p = WideJoinPipeline(dd, late=late, nparts=NPARTS, nattr_bound=1_000)
        calls = WideJoinPipeline.CALLS_LATE if late else WideJoinPipeline.CALLS_EAGER
        r = p.run(stream)
        torch.cuda.synchronize()
        if p.ws.status() != px.PX_OK:
            raise RuntimeError(f"device status in the {name} plan")
        n = int(r["final"]["ngroups"].item())
        k = r["final"]["keys"][0][:n].long()
        o = torch.argsort(k)
        finals[name] = [k[o]] + [a[:n][o] for a in r["final"]["aggs"]]
        for _ in range(args.warmup):
            p.run(stream)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)] for _ in range(args.steps)]
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for s in range(args.steps):
            p.run(stream, mark=lambda i, s=s: evs[s][i].record(stream))
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / args.steps
        ops = {c: round(sum(evs[s][i].elapsed_time(evs[s][i + 1]) for s in range(args.steps)) / args.steps, 4)
               for i, c in enumerate(calls)}
        nj = int(r["join"]["nout"].item())
        out[name] = {"ms_per_step": round(t, 4), "fact_rows_per_s": nf / (t / 1000), "operators_ms": ops,
                     "joined_rows": nj}
    if not all(torch.equal(x, y) for x, y in zip(finals["eager"], finals["late"])):
        raise RuntimeError("eager and late-materialized plans disagree")
    line = {"metric": "fact rows/s, selective wide join: late materialization vs eager exchange",
            "value": out["late"]["fact_rows_per_s"], "unit": "rows/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out["late"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded numpy PCG64; TPC-H-like shapes, no TPC-H data)",
            "config": {"workload": LATE_WORKLOAD, "fact_rows": nf, "dim_rows": NDIM,
                       "build_rows": int(d["pk_b"].size), "nparts": NPARTS},
            "late": out["late"], "eager": out["eager"],
            "speedup_late_vs_eager": out["eager"]["ms_per_step"] / out["late"]["ms_per_step"]}
    return line


# -------------------------------------------------------- serving workload ----
SERVE_WORKLOAD = ("served fragment queries: 32 resident dimension tables (1K..2M rows, log-spaced; group domains "
                  "log-uniform [4, 1e5]); Poisson arrivals of fragment queries (fact rows log-uniform [1e4, 4e6]) "
                  "and at-scale queries (60M-row Zipf s=1.1 fact over the 2M dimension) at 20:1; filter date in "
                  "[895, 1662) -> join -> group by attr: SUM(price), SUM(price*qty), COUNT; 120 GB admission budget")


def build_serving(npool: int, big: int, scale: float, seed: int = 5):
    import torch
    from paper_2606_24647_gb300 import serving
    g = np.random.Generator(np.random.PCG64(seed))
    sizes = np.unique(np.logspace(3, np.log10(2e6 * scale if scale < 1 else 2e6), 32).astype(np.int64))
    ngroups = np.floor(np.exp(g.uniform(np.log(4), np.log(1e5), size=sizes.size))).astype(np.int64)
    dims, dim_np = [], []
    for i, (nb, ng) in enumerate(zip(sizes, ngroups)):
        d = pxdata.fragment(0, int(nb), int(ng), seed=20_000 + i)
        dims.append(serving.ResidentDim(torch.from_numpy(d["pk"]).cuda(), torch.from_numpy(d["attr"]).cuda(), int(ng)))
        dim_np.append(d)
    pool = []  # (dim index, device columns, kind)
    nf = np.floor(np.exp(g.uniform(np.log(1e4 * scale), np.log(4e6 * scale), size=npool))).astype(np.int64)
    for i in range(npool):
        k = int(g.integers(0, len(dims)))
        d = pxdata.fragment(int(nf[i]), int(sizes[k]), int(ngroups[k]), seed=30_000 + i)
        pool.append((k, {c: torch.from_numpy(d[c]).cuda() for c in ("key", "price", "qty", "date")}, "fragment"))
    kb = len(dims) - 1  # the largest (2M-row) dimension
    for j in range(big):
        n = int(60_000_000 * scale)
        gg = np.random.Generator(np.random.PCG64(40_000 + j))
        pk_of_rank = gg.permutation(dim_np[kb]["pk"])
        key = pk_of_rank[pxdata.zipf_ranks(gg, pk_of_rank.size, n, 1.1) - 1]
        d = pxdata.fragment(n, 1, 1, seed=41_000 + j)
        cols = {"key": torch.from_numpy(key).cuda()}
        cols.update({c: torch.from_numpy(d[c]).cuda() for c in ("price", "qty", "date")})
        pool.append((kb, cols, "at-scale"))
    return dims, pool


def make_trace(dims, pool, n, seed):
    from paper_2606_24647_gb300 import serving
    g = np.random.Generator(np.random.PCG64(seed))
    frag_idx = [i for i, p in enumerate(pool) if p[2] == "fragment"]
    big_idx = [i for i, p in enumerate(pool) if p[2] == "at-scale"]
    qs = []
    for q in range(n):
        i = int(g.choice(big_idx)) if big_idx and g.random() < 1 / 21 else int(g.choice(frag_idx))
        k, cols, _ = pool[i]
        qs.append(serving.Query(q, dims[k], cols, pxdata.CFG2_DATE_LO, pxdata.CFG2_DATE_HI))
        qs[-1].prepare()  # the request's result buffer and batch descriptor, before it arrives
    return qs


def same_query_result(a, b) -> bool:
    """Equal (key, aggregates) group sets of two served queries (order-free)."""
    na, nb = int(a.out[2].item()), int(b.out[2].item())
    if na != nb:
        return False
    ka = a.out[0][:na].cpu().numpy().astype(np.int64)
    kb = b.out[0][:nb].cpu().numpy().astype(np.int64)
    oa, ob = np.argsort(ka, kind="stable"), np.argsort(kb, kind="stable")
    return np.array_equal(ka[oa], kb[ob]) and all(
        np.array_equal(x[:na].cpu().numpy()[oa], y[:nb].cpu().numpy()[ob]) for x, y in zip(a.out[1], b.out[1]))


def run_serve(args):
    """Config 5: continuous batching against one-at-a-time service of the same
    Poisson arrivals, at 0.5x, 0.8x and 1.0x of the batched server's saturation QPS."""
    import torch
    import paper_2606_24647_gb300 as px
    from paper_2606_24647_gb300 import serving

    torch.cuda.set_device(0)
    px.load()
    dims, pool = build_serving(args.serve_pool, args.serve_big, args.frag_scale)
    torch.cuda.synchronize()
    budget = 120 * 10**9
    n = args.serve_queries

    def fresh(seed):
        return make_trace(dims, pool, n, seed)

    # warm-up, then saturation: everything arrives at once
    serving.Server(budget, max_batch=512).serve(fresh(1)[:64], np.zeros(64))
    sat = serving.Server(budget, max_batch=512).serve(fresh(2), np.zeros(n))
    one_sat = serving.OneAtATimeServer().serve(fresh(2), np.zeros(n))
    levels = []
    mismatches = 0
    for f in (0.5, 0.8, 1.0):
        rate = f * sat["qps"]
        arr = serving.poisson_arrivals(rate, n, seed=int(100 * f))
        qb, qo = fresh(3), fresh(3)
        b = serving.Server(budget, max_batch=512).serve(qb, arr)
        o = serving.OneAtATimeServer().serve(qo, arr)
        levels.append({"offered_load": f, "offered_qps": rate, "batched": b, "one_at_a_time": o})
        if f == 1.0:  # every query served in the mix equals the same query served alone
            torch.cuda.synchronize()
            mismatches = sum(0 if same_query_result(x, y) else 1 for x, y in zip(qb, qo))
    if mismatches:
        raise RuntimeError(f"served: {mismatches} queries differ between batched and one-at-a-time service")
    nbig = sum(1 for q in qb if q.cols["key"].numel() >= 10_000_000)
    check = (f"at 1.0x load all {n} queries ({nbig} at-scale) equal between continuous batching and "
             "one-at-a-time service (keys and aggregates)")
    line = {"metric": "served QPS + p50/p99 latency vs one-at-a-time", "value": sat["qps"], "unit": "queries/s",
            "n_gpus": 1, "steps": n, "warmup": 64, "ms_per_step": round(1000 / sat["qps"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic (seeded numpy PCG64; TPC-H-like shapes, no TPC-H data)",
            "config": {"workload": SERVE_WORKLOAD if args.frag_scale == 1 else
                       f"REDUCED x{args.frag_scale:g}: " + SERVE_WORKLOAD,
                       "queries_per_level": n, "pool": len(pool), "resident_dims": len(dims)},
            "saturation": {"batched": sat, "one_at_a_time": one_sat}, "levels": levels,
            "check": check}
    return line


def emit(line) -> None:
    if line is not None:
        print(json.dumps(line), flush=True)


def run_extras(args) -> dict:
    """The other workloads of the headline metric, measured in the default run and
    nested in its line: the 1M-row plain and 6M-row plain-join pipelines (cold
    protocol per call, CUDA-graph stream per step, checked against the oracle),
    the 512-fragment fused batch against one-at-a-time launches (checked equal),
    and the served mix against one-at-a-time service (checked equal per query).
    A sub-workload that fails reports its error here instead of hiding the rest."""
    import copy
    import gc
    import torch
    out = {}
    for key, wl in (("plain", "plain"), ("plain_join", "plain-join"), ("fragments", "fragments"), ("served", "serve")):
        a = copy.copy(args)
        a.workload = wl
        if wl == "fragments":
            a.steps = min(args.steps, 50)
        t0 = time.perf_counter()
        try:
            r = {"plain": run_small, "plain-join": run_small, "fragments": run_fragments, "serve": run_serve}[wl](a)
            for k in ("n_gpus", "scaling", "vs_baseline", "dtype", "data"):
                r.pop(k, None)
        except Exception as e:  # noqa: BLE001 - reported in the line
            r = {"error": f"{type(e).__name__}: {e}"}
        r["wall_s"] = round(time.perf_counter() - t0, 1)
        out[key] = r
        gc.collect()
        torch.cuda.empty_cache()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="px", choices=["px", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=30_000_000,
                    help="fact rows of the oracle's CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the at-scale pipeline (skip the plain, plain-join, fragments and served sub-records)")
    ap.add_argument("--fact-rows", type=int, default=None,
                    help="smaller fact side for profiling captures (the reported workload is then reduced)")
    ap.add_argument("--dim-rows", type=int, default=None)
    ap.add_argument("--serve-queries", type=int, default=1000)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-big", type=int, default=2)
    ap.add_argument("--workload", default="at-scale",
                    choices=["at-scale", "fragments", "serve", "late-mat", "plain", "plain-join"],
                    help="at-scale: the exchange-join-aggregate pipeline (default); fragments: the batched fused "
                         "fragments against one-at-a-time calls")
    ap.add_argument("--fragments", type=int, default=FRAG_N)
    ap.add_argument("--frag-scale", type=float, default=1.0, help="scale of the fragment sizes (tests use < 1)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    global NFACT, NDIM, WORKLOAD
    if args.fact_rows or args.dim_rows:
        NFACT = args.fact_rows or NFACT
        NDIM = args.dim_rows or NDIM
        WORKLOAD = f"REDUCED for profiling: {NFACT}-row fact x {NDIM}-row dim; otherwise " + WORKLOAD
    others = {"plain": (run_small, "the plain and plain-join lines carry the oracle as cpu_baseline"),
              "plain-join": (run_small, "the plain and plain-join lines carry the oracle as cpu_baseline"),
              "late-mat": (run_late_mat, "the late-materialization plan is compared with the eager plan"),
              "serve": (run_serve, "the serving workload is compared with one-at-a-time GPU service"),
              "fragments": (run_fragments, "the fragments workload is compared with one-at-a-time GPU calls")}
    if args.workload in others:
        fn, why = others[args.workload]
        if args.impl == "reference":
            emit({"impl": "reference", "unavailable": "the oracle reference arm covers the at-scale workload; " + why})
            return 0
        emit(fn(args))
        return 0
    if args.impl == "reference":
        emit(run_reference(args))
        return 0
    line = run_px(args)
    if line is not None and line["n_gpus"] == 1 and not args.headline_only and args.fact_rows is None:
        line.update(run_extras(args))
    emit(line)
    return 0


if __name__ == "__main__":
    sys.exit(main())
