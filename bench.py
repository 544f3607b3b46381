"""Benchmark of the batched GF(256) encode (Eq. 2) on one GB300, plus the
region multiply-accumulate against HBM bandwidth, the plain
one-region-op-per-launch form, and the CPU oracle as the reference arm.

Default workload: 4096 generations x N = 64 source packets x 1500 B,
K = 64 coded packets each, coding matrices uniform over GF(256) minus 0
(393 MB of source, larger than the 129 MB L2, so no flush is needed between
steps).  A step encodes the whole batch in one persistent launch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gf|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own
GPU (generations are independent; no collective on the data path) and rank 0
prints one JSON line with the whole-job throughput (max time over ranks).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GF(256) batched encode GB/s (coded output)"
WORKLOAD = "uniform batched encode: 4096 generations x N=64 x 1500 B, K=64, GF(256)"
N_GENS, N_SRC, N_CODED, LEN = 4096, 64, 64, 1500


def _traffic(kernel_src: str, summary: str):
    """DRAM bytes per launch recorded in profiles/ for a kernel, or None when
    the kernel source no longer matches the hash the counters were taken on."""
    import hashlib
    try:
        fields = {}
        for line in open(os.path.join(ROOT, "profiles", summary)):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()
        if sha.startswith(fields["source_sha256_prefix"]):
            return float(fields["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        sm_max = max(r[1] for r in rows)
        loaded = [r[0] for r in rows if r[0] > 0.5 * sm_max] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": sm_max, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# whole-job aggregation over ranks (one replica per GPU, no data-path collective)
# ---------------------------------------------------------------------------
def max_over_ranks(x: float, device) -> float:
    """The largest `x` over all ranks (the job's time is its slowest rank's);
    `x` itself without an initialised process group of more than one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, steps: int, total_ms: float) -> float:
    """Units all ranks processed per second over the max-over-ranks time."""
    return world * units_per_rank * steps / (total_ms / 1e3)


def rank_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


# ---------------------------------------------------------------------------
# reference arm / cpu baseline: the oracle on the host cores
# ---------------------------------------------------------------------------
def host_info() -> dict:
    """Host CPU model (lscpu) and core count, recorded beside every CPU figure."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "model": model}


def oracle_encode_round(batch, first: int, threads: int):
    """Encodes generations first .. first+threads-1 (mod the batch) with the
    C oracle, one generation per host thread (the oracle's C call releases
    the GIL); returns the seconds taken."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    n = batch.src.shape[0]
    idx = [(first + t) % n for t in range(threads)]
    t0 = time.perf_counter()
    if threads == 1:
        oracle.encode(batch.field, batch.src[idx[0]], batch.coef[idx[0]])
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda i: oracle.encode(batch.field, batch.src[i], batch.coef[i]), idx))
    return time.perf_counter() - t0


def oracle_encode_rate(batch, threads: int, budget_s: float, max_gens: int):
    """Rounds of `threads` generations until `budget_s` seconds have passed or
    `max_gens` generations are done, whichever comes first; returns
    (coded-output GB/s, generations done, seconds)."""
    import oracle
    oracle.build()
    K, L = batch.coef.shape[1], batch.src.shape[2]
    done, el = 0, 0.0
    while done < max_gens and el < budget_s:
        el += oracle_encode_round(batch, done, threads)
        done += threads
    return done * K * L / el / 1e9, done, el


def run_reference(args, rank, world):
    """The reference arm: the C oracle on the host cores, on the GPU arm's
    batch (4096 x 64 x 1500 B, GF(256), K = 64).  A step encodes one round of
    generations, one per host thread; `ms_per_step` is that round's measured
    time and the whole batch's time is extrapolated under its own key."""
    if rank != 0:
        return
    import oracle
    from paper_1909_02871_gb300 import synth
    oracle.build()
    threads = os.cpu_count() or 1
    batch = synth.uniform_batch(n_gens=N_GENS, index=0)
    for w in range(args.warmup):
        oracle_encode_round(batch, w * threads, threads)
    times = [oracle_encode_round(batch, (args.warmup + s) * threads, threads) for s in range(args.steps)]
    total = sum(times)
    value = args.steps * threads * N_CODED * LEN / total / 1e9
    ms = total / args.steps * 1e3
    sample = (f"each step: {threads} generations (64 x 64 x 1500 B, K = 64) of the batch encoded by the C oracle, "
              f"one generation per host thread, {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gens": N_GENS, "n_src": N_SRC, "n_coded": N_CODED, "len": LEN,
                       "field": "GF(256)", "sample": sample},
            "generations_per_step": threads,
            "extrapolated_ms_per_batch": ms * N_GENS / threads,
            "host": host_info(),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gf(args, rank, world, local_rank):
    import torch

    from paper_1909_02871_gb300 import gf, synth
    from paper_1909_02871_gb300 import build as gbuild

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gbuild.build()
    gf.load()
    hbm_peak, bf16_peak, peak_kind = _peaks()

    batch = synth.uniform_batch(n_gens=N_GENS, index=0)
    src_h = torch.from_numpy(batch.src).pin_memory()
    coef_h = torch.from_numpy(batch.coef).pin_memory()
    src = src_h.to(dev)
    coef = coef_h.to(dev)
    out = torch.empty((N_GENS, N_CODED, LEN), dtype=torch.uint8, device=dev)
    gens = [(8, N_SRC, N_CODED, LEN, src[i], coef[i], out[i]) for i in range(N_GENS)]
    path = {"auto": gf.PATH_AUTO, "table": gf.PATH_TABLE, "bitsliced": gf.PATH_BITSLICED}[args.path]
    plan = gf.Plan.encode(gens, path=path)
    chosen = gf.gf_autotune_query(8, N_SRC, N_CODED, LEN) if path == gf.PATH_AUTO else (path, 0)
    stream = torch.cuda.Stream(device=dev)
    launches_per_step = plan.kernel_count

    # warm-up
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.launch(stream)
    stream.synchronize()

    # timed region: per-step events on the launching stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    rank_barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for s in range(args.steps):
                plan.launch(stream)
                ev[s + 1].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    rank_barrier()
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dev)
    out_bytes = N_GENS * N_CODED * LEN
    value = whole_job_rate(out_bytes, world, args.steps, total_ms) / 1e9
    ms_per_step = total_ms / args.steps
    clocks = clk.summary()

    # roofline of the dominant kernel (the step is one launch of it)
    avg_ms = statistics.mean(step_ms)
    if chosen[0] == gf.PATH_BITSLICED:
        flops = 2.0 * (8 * N_CODED) * (8 * N_SRC) * LEN * N_GENS
        # E2M1 (fp4) operands: dense fp4 = 6 x bf16 (nominal 13.5 / 2.25 PFLOP/s)
        peak = bf16_peak * 6.0
        achieved = flops / (avg_ms / 1e3) / 1e12
        # the K = 64 kind::mxf4 MMA itself: one 128x256x64 MMA per 128 SM clocks per SM
        sm_mhz = clocks.get("sm_mhz") or 2070.0
        mma_ceiling = 2.0 * 128 * 256 * 64 / 128.0 * 152 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "kernel": "encode_bitsliced_kernel", "peak_kind": f"{peak_kind} bf16 x 6 (fp4 nominal ratio)",
                "mma_k64_ceiling": mma_ceiling, "frac_of_mma_k64_ceiling": achieved / mma_ceiling}
    else:
        # 5 integer instructions (2 prmt + 3 lop3) per 4-byte word and coefficient
        ops = 5.0 * (LEN / 4.0) * N_SRC * N_CODED * N_GENS
        sm_mhz = clocks.get("sm_mhz") or 2070.0
        peak = 152 * 128 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": ops / (avg_ms / 1e3) / 1e12, "peak": peak, "unit": "Tops/s",
                "kernel": "encode_table_kernel",
                "peak_kind": "derived: 152 SMs x 128 int32 lanes x median SM clock"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if args.traffic is not None:
        roof["traffic"] = args.traffic
    elif chosen[0] == gf.PATH_BITSLICED:
        roof["traffic"] = _traffic("paper_1909_02871_gb300/csrc/gf_encode_tc.cu", "encode_bitsliced_traffic.txt")
    else:
        roof["traffic"] = None

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_gens": N_GENS, "n_src": N_SRC, "n_coded": N_CODED, "len": LEN,
                       "field": "GF(256)", "path": {0: "auto", 1: "table", 2: "bitsliced"}[chosen[0]],
                       "l2": "inputs larger than L2 (393 MB source per step)",
                       "parallelism": f"replicas x{world}"},
            "p50_step_ms": statistics.median(step_ms),
            "p99_step_ms": float(np.percentile(step_ms, 99)),
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks, "roofline": roof}

    if rank == 0 and not args.quick:
        line["source_GBps"] = value * N_SRC / N_CODED
        line["region_madd"] = bench_region(gf, torch, dev, stream, hbm_peak, peak_kind)
        line["plain"] = bench_plain(gf, torch, dev, stream, src, coef, out, value)
        line["e2e"] = bench_e2e(gf, torch, dev, stream, src_h, coef_h, args, plan, src, coef, out)
    plan.close()
    if rank == 0 and not args.quick:
        del src, coef, out
        torch.cuda.empty_cache()
        line["serving"] = serve_leg(torch, dev, args.serve_requests, (0.5,))
        host = host_info()
        v, done, el = oracle_encode_rate(batch, 1, args.cpu_seconds, 400)
        line["cpu_baseline"] = {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle", "host": host,
                                "sample": f"{done} generations of the same batch (64 x 64 x 1500 B, K = 64) encoded "
                                          f"by the C oracle in {el:.1f} s, one thread"}
        nt = host["nproc"] or 1
        v, done, el = oracle_encode_rate(batch, nt, args.cpu_seconds, 64 * nt)
        line["cpu_baseline_all_cores"] = {
            "value": v, "unit": "GB/s", "cores": nt, "kind": "oracle", "host": host,
            "sample": f"{done} generations of the same batch encoded by the C oracle in {el:.1f} s, one generation "
                      f"per thread, {nt} threads"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def bench_region(gf, torch, dev, stream, hbm_peak, peak_kind):
    """gf_region_madd / gf_region_mul on a 1 GiB region (larger than L2) in
    every field, against the measured HBM copy bandwidth: 3 bytes moved per
    region byte for madd, 2 for mul."""
    n = 1 << 30
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    a = torch.randint(0, 256, (n,), dtype=torch.uint8, device=dev, generator=g)
    b = torch.randint(0, 256, (n,), dtype=torch.uint8, device=dev, generator=g)
    points = []
    coefs = {1: 1, 2: 0x2, 4: 0xB, 8: 0x8E}
    with torch.cuda.stream(stream):
        for field in (1, 2, 4, 8):
            for name, fn, bytes_per in (("madd", gf.gf_region_madd, 3), ("mul", gf.gf_region_mul, 2)):
                c = coefs[field]
                for _ in range(3):
                    fn(field, b, a, c, stream=stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 10
                e0.record(stream)
                for _ in range(reps):
                    fn(field, b, a, c, stream=stream)
                e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1) / reps
                gbs = bytes_per * n / (ms / 1e3) / 1e9
                points.append({"field": field, "op": name, "coef": c, "GBps_hbm": gbs, "frac": gbs / hbm_peak,
                               "ms": ms, "len": n})
    del a, b
    torch.cuda.empty_cache()
    res = {"points": points, "peak": hbm_peak, "peak_kind": peak_kind,
           "min_frac": min(p["frac"] for p in points), "launches": len(points) * 13}
    # the GF(256) points under their old keys
    for p in points:
        if p["field"] == 8:
            res[p["op"]] = {k: p[k] for k in ("GBps_hbm", "frac", "ms", "len")}
    return res


def bench_plain(gf, torch, dev, stream, src, coef, out, batched_value):
    """The plain form: one region op per launch (K zero fills + K*N madds per
    generation), timed on 4 generations and extrapolated to the batch."""
    coef_h = coef[:4].cpu().numpy()
    G = 4
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for gi in range(G):
            for k in range(N_CODED):
                dst = out[gi, k]
                gf.gf_region_mul(8, dst, dst, 0, stream=stream)
                for i in range(N_SRC):
                    gf.gf_region_madd(8, dst, src[gi, i], int(coef_h[gi, k, i]), stream=stream)
        e1.record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
    ms = max(e0.elapsed_time(e1), wall * 1e3)
    value = G * N_CODED * LEN / (ms / 1e3) / 1e9
    return {"value": value, "unit": "GB/s", "launches": G * N_CODED * (N_SRC + 1),
            "sample": f"{G} generations, extrapolated (rate is per generation)",
            "batched_over_plain": batched_value / value}


def bench_e2e(gf, torch, dev, stream, src_h, coef_h, args, plan, src, coef, out):
    """Same metric through the public API with host buffers: every step uploads
    the sources and coding matrices from pinned host memory, encodes and
    downloads the coded packets (pipeline.HostEncoder: the batch in chunks on
    three streams, so uploads, encodes and downloads of different chunks
    overlap).  Timed with CUDA events from the first upload to the last
    download."""
    from paper_1909_02871_gb300 import pipeline
    out_h = torch.empty(out.shape, dtype=torch.uint8).pin_memory()
    steps = max(3, min(args.steps, 5))
    enc = pipeline.HostEncoder(8, src_h, coef_h, out_h, src, coef, out, chunks=8)
    for _ in range(2):
        enc.step()
    torch.cuda.synchronize()
    # the steps' first upload to their last download: start and end events on
    # every copy stream, the earliest start and the latest end taken
    starts = [torch.cuda.Event(enable_timing=True) for _ in enc.ups]
    ends = [torch.cuda.Event(enable_timing=True) for _ in enc.downs]
    for e, st in zip(starts, enc.ups):
        e.record(st)
    for _ in range(steps):
        enc.step()
    for e, st in zip(ends, enc.downs):
        e.record(st)
    torch.cuda.synchronize()
    ms = max(s.elapsed_time(e) for s in starts for e in ends) / steps
    res = {"value": N_GENS * N_CODED * LEN / (ms / 1e3) / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": int(src_h.numel() + coef_h.numel()), "d2h_bytes_per_step": int(out_h.numel()),
           "ms_per_step": ms, "chunks": len(enc.ranges), "gpu_launches_per_step": enc.kernel_count}
    enc.close()
    # the host link's own bound: the same bytes copied with no encode, the
    # uploads and downloads on two streams at once
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record(up)
    down.wait_event(e0)
    for _ in range(steps):
        with torch.cuda.stream(up):
            src.copy_(src_h, non_blocking=True)
            coef.copy_(coef_h, non_blocking=True)
        with torch.cuda.stream(down):
            out_h.copy_(out, non_blocking=True)
    e1.record(up)
    e2.record(down)
    torch.cuda.synchronize()
    link_ms = max(e0.elapsed_time(e1), e0.elapsed_time(e2)) / steps
    res["copies_only_ms_per_step"] = link_ms
    res["frac_of_copies_only"] = link_ms / ms
    return res


# ---------------------------------------------------------------------------
# other workloads (python bench.py --workload uneven|serve)
# ---------------------------------------------------------------------------
def run_uneven(args, rank, world, local_rank):
    """Uneven batched encode + decode over a lossy channel: 2048 generations,
    N ~ U{8..255}, len log-uniform in [64, 9000] B, field ~ U{GF(2), GF(4),
    GF(16), GF(256)}, 10 % erasures; one step = one CUDA-graph replay of the
    encode launch and the decode launches."""
    import torch

    from paper_1909_02871_gb300 import gf, pipeline, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gf.load()
    batch = synth.uneven_batch(n_gens=args.gens, index=0)
    work = pipeline.build(batch, dev)
    step = pipeline.UnevenStep(work)
    stream = torch.cuda.Stream(device=dev)
    step.capture(stream)
    for _ in range(args.warmup):
        step.replay()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    rank_barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for i in range(args.steps):
                step.replay()
                ev[i + 1].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    rank_barrier()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dev)
    bad = [i for i in (0, 1, len(batch.gens) // 2, len(batch.gens) - 1)
           if not np.array_equal(pipeline.decoded(work, i), batch.gens[i].src)]
    # plain form on a subset, extrapolated by source bytes
    sub = list(range(0, len(batch.gens), max(1, len(batch.gens) // 64)))
    sub_bytes = sum(batch.gens[i].src.size for i in sub)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        pipeline.plain_step(work, sub, stream=stream)
    stream.synchronize()
    plain_s = time.perf_counter() - t0
    value = whole_job_rate(work.bytes_src, world, args.steps, total_ms) / 1e9
    # the two plans of a step timed on their own (outside the graph)
    part_ms = {}
    for name, plan in (("encode", step.enc), ("decode", step.dec)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            plan.launch(stream)
            e0.record(stream)
            for _ in range(3):
                plan.launch(stream)
            e1.record(stream)
        stream.synchronize()
        part_ms[name] = e0.elapsed_time(e1) / 3
    # algorithmic work in the bit-sliced count of the scope table: 2 * 8K * 8N * len FLOP per
    # generation for the sender's K packets, 2 * 8N * 8R * len for the payload phase of the
    # decode (N sources from R received packets); the coefficient phase's byte multiply-adds
    # (about N^2 (N + R) per generation) on the integer ALU are counted apart
    enc_flop = sum(2.0 * 64 * g.n_src * k * g.length for g, k in zip(batch.gens, work.k_sent))
    dec_flop = sum(2.0 * 64 * g.n_src * rr.size * g.length for g, rr in zip(batch.gens, work.recv_rows))
    coef_madds = sum(float(g.n_src) ** 2 * (g.n_src + rr.size) for g, rr in zip(batch.gens, work.recv_rows))
    _, bf16_peak, peak_kind = _peaks()
    peak = 6.0 * bf16_peak
    step_avg = statistics.mean(step_ms)
    roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": peak,
            "peak_kind": f"{peak_kind} bf16 x 6 (fp4 nominal ratio)",
            "kernel": "whole step: sender encode + decode payload phase in the bit-sliced FLOP count",
            "achieved": (enc_flop + dec_flop) / (step_avg / 1e3) / 1e12,
            "encode": {"flop": enc_flop, "ms": part_ms["encode"],
                       "achieved": enc_flop / (part_ms["encode"] / 1e3) / 1e12},
            "decode": {"payload_flop": dec_flop, "coef_phase_byte_madds": coef_madds, "ms": part_ms["decode"]},
            "traffic": None}
    roof["frac"] = roof["achieved"] / peak
    roof["encode"]["frac"] = roof["encode"]["achieved"] / peak
    line = {"metric": "uneven encode+decode GB/s (source bytes per step)", "value": value, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"uneven encode+decode: {len(batch.gens)} generations, N~U{{8..255}}, "
                                   "len log-uniform 64-9000 B, field ~U{GF2,GF4,GF16,GF256}, 10% erasures",
                       "source_bytes": work.bytes_src, "coded_bytes": work.bytes_coded,
                       "packets_sent": int(sum(work.k_sent))},
            "p50_step_ms": statistics.median(step_ms), "p99_step_ms": float(np.percentile(step_ms, 99)),
            "gpu_launches": step.kernel_count * args.steps, "clocks": clk.summary(), "roofline": roof,
            "round_trip_ok": not bad,
            "plain": {"value": sub_bytes / plain_s / 1e9, "unit": "GB/s",
                      "sample": f"{len(sub)} generations, one encode + one decode call each, host wall time"}}
    step.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_leg(torch, dev, n: int, fractions, budget: int = 4 << 30, systematic: bool = False, loss: float = 0.1,
              redundancy: float = 0.0, rate_base: float | None = None) -> dict:
    """Serving: n requests (half encode, half decode) with the uneven
    workload's shapes; saturation throughput (every request arriving at once)
    and, for each fraction f, Poisson arrivals at f x rate_base (default: this
    run's saturation) with decode packets arriving 20 us apart: p50/p99
    request latency.  An encode request makes N + ceil(redundancy N) packets;
    a decode request receives a stream with i.i.d. losses `loss`.  With
    `systematic` the senders send the N sources uncoded first.  Every result is
    checked: decoded sources against the sources, encode results against a
    batched encode of the same packets."""
    from paper_1909_02871_gb300 import gf, serve, synth
    batch = synth.uneven_batch(n_gens=n, index=7, loss=loss)
    # coded packets of the decode requests, produced by the library (untimed)
    coded, rows = {}, {}
    items, keep = [], []
    for i, ge in enumerate(batch.gens):
        if i % 2 == 1:
            if systematic:
                stream = synth.systematic_stream(ge.coef_stream)
                c = np.ascontiguousarray(stream[~synth.erasures(stream.shape[0], loss, 7, i)])
            else:
                c = np.ascontiguousarray(ge.coef_stream[~ge.erased])
            s_d = torch.from_numpy(ge.src).to(dev)
            c_d = torch.from_numpy(c).to(dev)
            o_d = torch.empty((c.shape[0], ge.length), dtype=torch.uint8, device=dev)
            keep.append((s_d, c_d, o_d))
            items.append((ge.field, ge.n_src, c.shape[0], ge.length, s_d, c_d, o_d))
            coded[i] = (c, o_d)
        else:
            extra = int(np.ceil(redundancy * ge.n_src))
            rows[i] = np.ascontiguousarray(ge.coef_stream[:extra if systematic else ge.n_src + extra])
    gf.gf_encode_batched(items)
    torch.cuda.synchronize()
    coded = {i: (c, o.cpu().numpy()) for i, (c, o) in coded.items()}
    del keep

    def requests(times, gap):
        out = []
        for i, (ge, t) in enumerate(zip(batch.gens, times)):
            if i % 2 == 0:
                out.append(serve.EncodeRequest(i, float(t), ge.field, ge.src, rows[i], systematic=systematic))
            else:
                c, p = coded[i]
                out.append(serve.DecodeRequest(i, float(t), ge.field, ge.n_src, ge.length, c, p,
                                               float(t) + gap * np.arange(1, c.shape[0] + 1)))
        return out

    def ok(reqs):
        return all(np.array_equal(r.result, batch.gens[r.rid].src) for r in reqs
                   if isinstance(r, serve.DecodeRequest))

    serve.Server(mem_budget=budget).run(requests(np.zeros(n), 0.0)[:32])  # warm-up
    reqs = requests(np.zeros(n), 0.0)
    srv = serve.Server(mem_budget=budget)
    wall = srv.run(reqs)
    sat = n / wall
    good = ok(reqs)
    # encode results: the same packets from one batched encode (a systematic request's first N
    # packets are its sources)
    enc = [r for r in reqs if isinstance(r, serve.EncodeRequest) and r.coef.shape[0]]
    outs = [torch.empty((r.coef.shape[0], r.src.shape[1]), dtype=torch.uint8, device=dev) for r in enc]
    srcs = [(torch.from_numpy(r.src).to(dev), torch.from_numpy(r.coef).to(dev)) for r in enc]
    gf.gf_encode_batched([(r.field, r.src.shape[0], r.coef.shape[0], r.src.shape[1], s_, c_, o)
                          for r, (s_, c_), o in zip(enc, srcs, outs)])
    torch.cuda.synchronize()
    for r, o in zip(enc, outs):
        want = o.cpu().numpy()
        good = good and np.array_equal(r.result[r.src.shape[0]:] if systematic else r.result, want)
        if systematic:
            good = good and np.array_equal(r.result[:r.src.shape[0]], r.src)
    launches = srv.launches
    rates = {}
    for f in fractions:
        rate = f * (rate_base or sat)
        r2 = requests(synth.arrivals(rate, n, index=int(f * 100)), 20e-6)
        s2 = serve.Server(mem_budget=budget)
        w2 = s2.run(r2)
        good = good and ok(r2)
        st = serve.latency_stats(r2)
        st.update({"rate_req_per_s": rate, "throughput_req_per_s": n / w2, "batches": s2.batches})
        rates[f"{f:.2f}x"] = st
        launches += s2.launches
    return {"requests": n, "saturation_req_per_s": sat, "saturation_wall_s": wall,
            "source_bytes": int(sum(ge.src.size for ge in batch.gens)), "rates": rates, "round_trip_ok": good,
            "gpu_launches": launches, "device_memory_budget": budget, "systematic": systematic, "loss": loss,
            "redundancy": redundancy,
            "workload": f"{n} requests, half encode and half decode, uneven shapes (N ~ U{{8..255}}, len "
                        f"log-uniform 64-9000 B, four fields), {'systematic' if systematic else 'random linear'} "
                        f"coding, {int(loss * 100)}% losses, decode packets 20 us apart"}


def run_serve(args, rank, world, local_rank):
    """Serving: Poisson arrivals of encode and decode requests (shapes of the
    uneven workload), admitted by device memory, decode packets arriving one
    by one; throughput and p50/p99 latency at several arrival rates."""
    import torch

    from paper_1909_02871_gb300 import gf, serve, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gf.load()
    n = args.requests
    rank_barrier()
    with Clocks(local_rank) as clk:
        leg = serve_leg(torch, dev, n, (0.25, 0.5, 0.9))
    sat = whole_job_rate(n, world, 1, max_over_ranks(leg["saturation_wall_s"], dev) * 1e3)
    # the plain form: one request at a time
    batch = synth.uneven_batch(n_gens=64, index=7)
    plain_reqs = [serve.EncodeRequest(i, 0.0, ge.field, ge.src, np.ascontiguousarray(ge.coef_stream[:ge.n_src]))
                  for i, ge in enumerate(batch.gens)]
    plain_wall = serve.Server(max_active=1).run(plain_reqs)
    # systematic against random linear coding, 0 % and 10 % losses, at one arrival rate per loss
    # (half the random-linear saturation); encode requests add 15 % coded packets either way
    compare = {}
    for loss in (0.0, 0.1):
        base = None
        for sysm in (False, True):
            leg2 = serve_leg(torch, dev, n, (0.5,), systematic=sysm, loss=loss, redundancy=0.15, rate_base=base)
            base = base or leg2["saturation_req_per_s"]
            key = f"{'systematic' if sysm else 'random'}_loss{int(loss * 100)}"
            compare[key] = {"saturation_req_per_s": leg2["saturation_req_per_s"], "at_rate": leg2["rates"]["0.50x"],
                            "round_trip_ok": leg2["round_trip_ok"]}
            leg["gpu_launches"] += leg2["gpu_launches"]
            leg["round_trip_ok"] = leg["round_trip_ok"] and leg2["round_trip_ok"]
    line = {"metric": "serving throughput req/s and p99 ms", "value": sat, "unit": "req/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": leg["saturation_wall_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "serving: " + leg["workload"] + ", Poisson arrivals",
                       "device_memory_budget": leg["device_memory_budget"], "source_bytes": leg["source_bytes"]},
            "saturation_GBps_source": leg["source_bytes"] / leg["saturation_wall_s"] / 1e9, "rates": leg["rates"],
            "plain_encode_req_per_s": len(plain_reqs) / plain_wall, "round_trip_ok": leg["round_trip_ok"],
            "systematic_vs_random": compare,
            "clocks": clk.summary(), "gpu_launches": leg["gpu_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_recode(args, rank, world, local_rank):
    """Recoding at relays: 4096 generations, each node holding 64 coded
    packets of 1500 B (GF(256)) and making 64 new ones with fresh
    coefficients: recoded payloads and their composed coding vectors in one
    gf_recode_batched call per step."""
    import torch

    import oracle
    from paper_1909_02871_gb300 import gf, synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gf.load()
    b = synth.uniform_batch(n_gens=N_GENS, index=5)  # src stands in for held coded payloads, coef for their vectors
    g = synth.choice(95)
    mix = synth.coefficients(g, 8, (N_GENS, N_CODED, N_CODED), nonzero=True)
    ci, pi, mx = (torch.from_numpy(x).to(dev) for x in (b.coef, b.src, mix))
    co = torch.empty((N_GENS, N_CODED, N_SRC), dtype=torch.uint8, device=dev)
    po = torch.empty((N_GENS, N_CODED, LEN), dtype=torch.uint8, device=dev)
    items = [(8, N_SRC, N_CODED, N_CODED, LEN, ci[i], pi[i], mx[i], co[i], po[i]) for i in range(N_GENS)]
    stream = torch.cuda.Stream(device=dev)
    plan = gf.Plan.recode(items)  # descriptors uploaded once, like the uniform encode's plan
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.launch(stream)
    stream.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    rank_barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for i in range(args.steps):
                plan.launch(stream)
                ev[i + 1].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    rank_barrier()
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dev)
    out_bytes = N_GENS * N_CODED * (LEN + N_SRC)
    ok = True
    for i in (0, N_GENS - 1):
        wc, wp = oracle.recode(8, b.coef[i], b.src[i], mix[i])
        ok = ok and np.array_equal(co[i].cpu().numpy(), wc) and np.array_equal(po[i].cpu().numpy(), wp)
    line = {"metric": "GF(256) batched recode GB/s (recoded output)",
            "value": whole_job_rate(out_bytes, world, args.steps, total_ms) / 1e9, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "recode: 4096 generations, 64 coded packets of 1500 B held, 64 recoded packets "
                                   "and their coding vectors made per generation, GF(256)",
                       "l2": "inputs larger than L2"},
            "clocks": clk.summary(), "round_trip_ok": ok, "gpu_launches": plan.kernel_count * args.steps}
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fig1(args, rank, world, local_rank):
    """The paper's Fig. 1 workload on the GPU: generations of N = 16 packets,
    K = 16 random combinations, packet size 128 B .. 64 KiB, each field.  One
    batched encode per step over enough generations to fill the GPU (about
    256 MB of coded output, at least 1024 generations); GB/s of coded output
    (the paper's throughput) and the same per SM."""
    import torch

    from paper_1909_02871_gb300 import gf, synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gf.load()
    stream = torch.cuda.Stream(device=dev)
    import oracle
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    points, launches, bit_exact = [], 0, True
    rank_barrier()
    with Clocks(local_rank) as clk:
        for field in (1, 2, 4, 8):
            for e in range(7, 17):
                P = 1 << e
                G = int(min(65536, max(1024, (256 << 20) // (16 * P))))
                g = synth.choice(96, field, P)
                src = torch.randint(0, 256, (G, 16, P), dtype=torch.uint8, device=dev)
                coef = torch.from_numpy(synth.coefficients(g, field, (G, 16, 16), nonzero=True)).to(dev)
                out = torch.empty((G, 16, P), dtype=torch.uint8, device=dev)
                # the autotuner times the table tile shapes and the tensor-core path for this shape bucket
                path, variant = gf.gf_autotune_encode(field, 16, 16, P, min(G, 2048), stream=stream)
                plan = gf.Plan.encode([(field, 16, 16, P, src[i], coef[i], out[i]) for i in range(G)])
                with torch.cuda.stream(stream):
                    for _ in range(3):
                        plan.launch(stream)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(args.steps):
                        plan.launch(stream)
                    e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                gbs = G * 16 * P / (ms / 1e3) / 1e9
                # the first and last generations of the point against the oracle
                ok = all(np.array_equal(out[i].cpu().numpy(),
                                        oracle.encode(field, src[i].cpu().numpy(), coef[i].cpu().numpy()))
                         for i in (0, G - 1))
                bit_exact = bit_exact and ok
                points.append({"field": field, "packet_bytes": P, "generations": G, "ms": ms, "GBps_coded": gbs,
                               "GBps_coded_per_SM": gbs / n_sm, "bit_exact_sampled": ok,
                               "path": {1: "table", 2: "bitsliced"}.get(path, path), "table_variant": variant})
                launches += plan.kernel_count * args.steps
                plan.close()
                del src, coef, out
    torch.cuda.empty_cache()
    line = {"metric": "N=16 encode GB/s of coded output vs packet size (Fig. 1 workload)",
            "value": statistics.median(p["GBps_coded"] for p in points), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": 3, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "generations of N=16, K=16 random combinations, packet 128 B..64 KiB, GF(2), "
                                   "GF(4), GF(16), GF(256); >= 1024 generations per point (about 256 MB out)",
                       "value_is": "median over the 40 points"},
            "points": points, "clocks": clk.summary(), "gpu_launches": launches,
            "round_trip_ok": bit_exact}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_region_sweep(args, rank, world, local_rank):
    """Region madd / mul over 2^10 .. 2^30 bytes in GF(2), GF(4), GF(16),
    GF(256): HBM GB/s (3 bytes moved per region byte for madd, 2 for mul)
    against the measured copy bandwidth.  Regions that fit in L2 are timed
    one call at a time with L2 flushed (a 256 MB write) before each call."""
    import torch

    from paper_1909_02871_gb300 import gf
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gf.load()
    hbm_peak, _, peak_kind = _peaks()
    stream = torch.cuda.Stream(device=dev)
    n_max = 1 << 30
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    a = torch.randint(0, 256, (n_max,), dtype=torch.uint8, device=dev, generator=g)
    b = torch.randint(0, 256, (n_max,), dtype=torch.uint8, device=dev, generator=g)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    l2_bytes = 128 << 20
    points = []
    launches = 0  # timed region-op launches (one kernel each)
    crng = np.random.default_rng(1909)
    rank_barrier()
    with Clocks(local_rank) as clk, torch.cuda.stream(stream):
        for field in args.region_fields:
            for op, fn, per in (("madd", gf.gf_region_madd, 3), ("mul", gf.gf_region_mul, 2)):
                for e in range(args.region_min_log, 31):
                    n = 1 << e
                    c = int(crng.integers(1, 1 << field)) if field > 1 else 1
                    for _ in range(3):
                        fn(field, b, a, c, length=n, stream=stream)
                    cold = per * n <= 2 * l2_bytes
                    reps = 5 if cold else max(3, min(50, (1 << 33) // (per * n)))
                    times = []
                    for _ in range(reps):
                        if cold:
                            flush.fill_(1)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        fn(field, b, a, c, length=n, stream=stream)
                        e1.record(stream)
                        e1.synchronize()
                        times.append(e0.elapsed_time(e1))
                    ms = statistics.median(times)
                    gbs = per * n / (ms / 1e3) / 1e9
                    points.append({"field": field, "op": op, "len": n, "coef": c, "us": ms * 1e3,
                                   "GBps_hbm": gbs, "frac": gbs / hbm_peak, "l2_flushed": cold})
                    launches += reps
    stream.synchronize()
    big = [p for p in points if p["len"] == n_max]
    line = {"metric": "region madd/mul HBM GB/s (sweep)", "value": min(p["GBps_hbm"] for p in big), "unit": "GB/s",
            "n_gpus": world, "steps": len(points), "warmup": 3, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "region madd/mul, len 2^10..2^30 B, GF(2), GF(4), GF(16), GF(256), random "
                                   "nonzero coefficient per point; regions up to 2 x L2 timed with L2 flushed",
                       "value_is": "the lowest of the eight 1 GiB points"},
            "peak": hbm_peak, "peak_kind": peak_kind, "clocks": clk.summary(), "points": points,
            "gpu_launches": launches}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_single(args, rank, world, local_rank):
    """One generation (N = 16 sources of 1500 B, K = 16 coded packets) per
    call in each field: device time and host-call time of one encode and of
    one decode of the 16 packets, each checked against the oracle."""
    import torch

    import oracle
    from paper_1909_02871_gb300 import gf, synth
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gf.load()
    stream = torch.cuda.Stream(device=dev)
    res = {}
    ok = True
    reps = 200
    rank_barrier()
    with Clocks(local_rank) as clk:
        for field in (1, 2, 4, 8):
            gen = synth.generation(field)
            coef_np = np.ascontiguousarray(gen.coef_stream[:gen.n_coded])
            N, K, L = gen.n_src, coef_np.shape[0], gen.length
            src = torch.from_numpy(gen.src).to(dev)
            coef = torch.from_numpy(coef_np).to(dev)
            out = torch.empty((K, L), dtype=torch.uint8, device=dev)
            dec_out = torch.empty((N, L), dtype=torch.uint8, device=dev)
            rnk = torch.zeros(1, dtype=torch.int32, device=dev)
            enc = [(field, N, K, L, src, coef, out)]
            decs = [(field, N, K, L, coef, out, dec_out, rnk, None, None)]
            timings = {}
            for name, call in (("encode", lambda: gf.gf_encode_batched(enc, stream=stream)),
                               ("decode", lambda: gf.gf_decode_batched(decs, stream=stream))):
                for _ in range(5):
                    call()
                stream.synchronize()
                dev_us, host_us = [], []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    t0 = time.perf_counter()
                    e0.record(stream)
                    call()
                    e1.record(stream)
                    e1.synchronize()
                    host_us.append((time.perf_counter() - t0) * 1e6)
                    dev_us.append(e0.elapsed_time(e1) * 1e3)
                timings[name] = {"device_us_p50": statistics.median(dev_us),
                                 "device_us_p99": float(np.percentile(dev_us, 99)),
                                 "call_us_p50": statistics.median(host_us)}
            coded = out.cpu().numpy()
            good = np.array_equal(coded, oracle.encode(field, gen.src, coef_np))
            rank_ok = int(rnk.item())
            if rank_ok == N:
                good = good and np.array_equal(dec_out.cpu().numpy(), gen.src)
            ok = ok and good
            timings["rank"] = rank_ok
            timings["bit_exact"] = bool(good)
            res[f"GF(2^{field})"] = timings
    enc_us = res["GF(2^8)"]["encode"]["device_us_p50"]
    line = {"metric": "single generation encode/decode latency (us)", "value": enc_us, "unit": "us",
            "n_gpus": world, "steps": reps, "warmup": 5, "ms_per_step": enc_us / 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "one generation: N=16 x 1500 B, K=16, four fields, one call per encode and "
                                   "per decode", "value_is": "GF(256) encode, device time, median"},
            "fields": res, "round_trip_ok": ok, "clocks": clk.summary(),
            "gpu_launches": 4 * reps * 3}  # per field and rep: one encode kernel, two decode kernels
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gf", "reference"], default="gf")
    ap.add_argument("--workload", choices=["uniform", "uneven", "serve", "region", "single", "recode", "fig1"], default="uniform")
    ap.add_argument("--gens", type=int, default=2048, help="generations of the uneven workload")
    ap.add_argument("--requests", type=int, default=600, help="requests of the serving workload")
    ap.add_argument("--path", choices=["auto", "table", "bitsliced"], default="auto")
    ap.add_argument("--quick", action="store_true", help="skip the side measurements")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-requests", type=int, default=300, help="requests of the default line's serving leg")
    ap.add_argument("--region-min-log", type=int, default=10, help="region sweep: smallest size 2^k bytes")
    ap.add_argument("--region-fields", type=int, nargs="+", default=[1, 2, 4, 8], help="region sweep: fields")
    ap.add_argument("--uniform-gens", type=int, default=None,
                    help="generations of the uniform workload (smaller cases for profiler captures; "
                         "the reported workload is the 4096-generation batch only without it)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture")
    args = ap.parse_args()
    if args.uniform_gens is not None:
        global N_GENS, WORKLOAD
        N_GENS = args.uniform_gens
        WORKLOAD = WORKLOAD.replace("4096 generations", f"{N_GENS} generations")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "gf":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "uneven":
        run_uneven(args, rank, world, local_rank)
    elif args.workload == "serve":
        run_serve(args, rank, world, local_rank)
    elif args.workload == "region":
        run_region_sweep(args, rank, world, local_rank)
    elif args.workload == "single":
        run_single(args, rank, world, local_rank)
    elif args.workload == "recode":
        run_recode(args, rank, world, local_rank)
    elif args.workload == "fig1":
        run_fig1(args, rank, world, local_rank)
    else:
        run_gf(args, rank, world, local_rank)
    if world > 1 and args.impl == "gf":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
