#!/usr/bin/env python3
"""Benchmark of the GB300 two-pass parallel gzip decompression (libpgz).

Default workload (one GPU): 512 independent synthetic gzip members (seed 3)
with log-uniform uncompressed sizes 64 KiB .. 64 MiB, half FASTQ (150 bp
reads) and half order-2 Markov text, gzip levels 1/6/9 (host zlib); about
2.9 GB compressed and 4.5 GB decompressed.  One step decompresses all of them
(block-start search, pass 1, window chain, translation, CRC-32/ISIZE check)
with inputs and outputs resident in device memory, in two forms:

  batched (the reported value): every member in one run of the pass kernels,
      parts taken from a device work queue, captured once in a CUDA graph
      (pgz_batch_prepare / pgz_batch_run); part size, pass-1 CTA shape and
      execution form chosen by the library's autotuner (pgz_autotune) on the
      same members unless --chunk-bytes fixes them;
  plain: one pgz_decompress call per member (the library's default parts).

e2e times the same members through pgz_decompress_batch_host: pinned host
input and output, the copies inside the call.  Extra keys of the same line:
the two 256 MiB FASTQ files at gzip -1 and -9 (batched and plain, per-level
block-start and placeholder statistics) and the served request loop (p50 and
p99 latency at offered loads of 1, 4 and 16 GB/s, a reduced request count).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pgz|reference]
                  [--workload batch512|fastq256|fastq1m|fastq4g|served|stream]
                  [--chunk-bytes B] [--served-requests R] [--profile-case SPEC]

Prints one JSON line.  --impl reference times the CPU oracle (the plain
bit-at-a-time RFC 1951 inflater under oracle/), member-parallel on the host's
cores, on the same members.  Under torchrun every rank decodes its own copy of
the workload (independent members, no collective: weak scaling) and rank 0
prints the whole-job throughput.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 126 * (1 << 20)
CHUNK_BYTES = 64 << 10        # compressed bytes per part when the autotuner is not run
TUNE_CHUNKS = [32 << 10, 64 << 10, 128 << 10, 256 << 10, 512 << 10]   # the autotuner's part sizes (and 1-2 waves) ...
TUNE_WPB = [2, 4, 8]                                                # ... and pass-1 CTA shapes (warps)
PLAIN_PARTS = 1024            # parts per file of the plain one-file-at-a-time form
METRIC = "decompressed GB/s on 1 GB300 (batched vs plain), %HBM roofline; served p50/p99 ms"
HEADLINE_DESC = ("512 synthetic gzip members, log-uniform 64 KiB-64 MiB (seed 3), FASTQ 150 bp / order-2 Markov "
                 "text, gzip -1/-6/-9")
TUNE_CHUNKS_BATCH = [128 << 10, 256 << 10, 512 << 10]   # the autotuner's part sizes on the 512 members
                                                        # (and the sizes of 1-4 whole waves of pass-1 warps)
TUNE_WPB_BATCH = [2, 4]
SERVED_REQUESTS = 240         # requests per offered load in the default run (the full served run uses 2000)
# DRAM bytes (read + write) of pass 1 (k_sync + k_inflate) per decompressed byte, from one-pass ncu captures
# of the current kernels.  The two 256 MiB FASTQ files as one batch, by (part size, warps per block, pipelined
# execution) (profiles/pass1_traffic_fastq256.md) ...
PASS1_TRAFFIC_PER_OUT_BYTE = {
    (88162, 2, 0): (0.852781568e9 + 0.524115712e9 + 3.037636864e9 + 1.317603072e9) / 536870912,
    (88162, 4, 0): (0.854030592e9 + 0.524192512e9 + 3.039483648e9 + 1.317075712e9) / 536870912,
}
# ... and the 512-member batch, by (part size, warps per block, pipelined execution, determined tail)
# (profiles/pass1_traffic_batch512.md).  Other configurations report null.
PASS1_TRAFFIC_PER_OUT_BYTE_BATCH512 = {
    (499078, 4, 0, 0): (0.964350464e9 + 0.952157696e9 + 39.964783360e9 + 23.372040960e9) / 4467581835,
    (499078, 2, 0, 0): (0.966032640e9 + 0.953315840e9 + 39.960246528e9 + 23.372556288e9) / 4467581835,
}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def _compress_job(args):
    from paper_1905_07224_gb300 import synth
    kind, n, level, seed, read_len, p_n = args
    raw = synth.fastq(n, read_len, p_n, seed) if kind == "fastq" else synth.markov(n, seed)
    return raw, synth.gzip_compress(raw, level)


def make_workload(name: str):
    """List of (label, raw, gz) and a description."""
    import multiprocessing as mp
    if name == "fastq256":
        jobs = [("fastq", 256 << 20, 1, 1, 150, 0.001), ("fastq", 256 << 20, 9, 1, 150, 0.001)]
        desc = "2 x 256 MiB synthetic FASTQ (150 bp, seed 1), gzip -1 and -9"
    elif name == "fastq1m":
        jobs = [("fastq", 1 << 20, 6, 0, 100, 0.001)]
        desc = "1 MiB synthetic FASTQ (100 bp, seed 0), gzip -6"
    else:
        raise ValueError(name)
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_compress_job, jobs)
    files = [(f"{j[0]}-L{j[2]}", raw, gz) for j, (raw, gz) in zip(jobs, res)]
    return files, desc


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# replicas: every rank decodes its own copy of the workload (independent members, no data exchange)
# ---------------------------------------------------------------------------
def max_over_ranks(values, device):
    """The slowest rank's times (all ranks take part; the process group is initialised)."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_gbs(bytes_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank's bytes over the slowest rank's time per step."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def run_pgz(args, rank, world):
    """Both files of the workload, batched (headline) and plain (one file at a time, fixed part count)."""
    import numpy as np
    import torch
    from paper_1905_07224_gb300 import build, pgz

    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    files, desc = make_workload(args.workload)
    stream = torch.cuda.current_stream()
    gz_dev = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).cuda() for _, _, g in files]
    outs = [torch.empty(len(r) + 4096, dtype=torch.uint8, device="cuda") for _, r, _ in files]
    total_out = sum(len(r) for _, r, _ in files)
    total_in = sum(len(g) for _, _, g in files)
    jobs = [(gz_dev[k].data_ptr(), len(g), outs[k].data_ptr(), outs[k].numel()) for k, (_, _, g) in enumerate(files)]
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def check(what):
        torch.cuda.synchronize()
        for k, (_, raw, _) in enumerate(files):
            if outs[k][:len(raw)].cpu().numpy().tobytes() != raw:
                raise RuntimeError(f"output mismatch ({what}, file {k})")
        for o in outs:
            o.fill_(0)

    def timed(step, ctx):
        """W untimed steps, then K steps between barriers, CUDA events on the launching stream."""
        for _ in range(args.warmup):
            step()
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()
        l0 = pgz.pgz_kernel_launches(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        return e0.elapsed_time(e1) / args.steps, pgz.pgz_kernel_launches(ctx) - l0

    # ---- batched: every file of the step in one graph-captured run of the pass kernels, with the part size
    # and pass-1 CTA shape chosen by the library's autotuner on these files (unless --chunk-bytes fixes them)
    ctx_b = pgz.pgz_create(pgz.pgz_config_init(device=dev, cuda_stream=stream.cuda_stream, n_chunks=0,
                                               chunk_bytes=args.chunk_bytes or CHUNK_BYTES,
                                               warps_per_block=args.warps_per_block,
                                               exec_pipelined=args.exec_pipelined))
    tune = None
    if not args.chunk_bytes:
        tune = autotune(pgz, ctx_b, jobs, TUNE_CHUNKS, TUNE_WPB)
    chunk_bytes = tune["best"][0] if tune else args.chunk_bytes
    wpb = tune["best"][1] if tune else args.warps_per_block
    xp = tune["best"][2] if tune else args.exec_pipelined
    batch = pgz.Batch(ctx_b, jobs)

    def step_batched():
        r, res, _ = batch.run()
        if r != 0 or any(st != 0 or n != len(files[k][1]) for k, (st, n) in enumerate(res)):
            raise RuntimeError(f"pgz_batch_run failed: {pgz.pgz_strerror(r)}")

    step_batched()
    check("batched")
    with Clocks(dev) as clk:
        ms, launches = timed(step_batched, ctx_b)
    clocks = clk.summary()
    # per-stage times of the same batch (the library's CUDA events on the same stream, graph-free run)
    stage = {k: 0.0 for k in ("ms_sync", "ms_inflate", "ms_chain", "ms_translate", "ms_crc", "ms_total")}
    nst = 3
    for _ in range(nst):
        r, _, s = pgz.pgz_decompress_batch(ctx_b, jobs, stats=True)
        if r != 0:
            raise RuntimeError(f"pgz_decompress_batch failed: {pgz.pgz_strerror(r)}")
        for k in stage:
            stage[k] += s[k] / nst
    batch_parts = s["chunks"]
    # the translation reads the 32 KiB window of every part that holds a placeholder
    _, _, nph_parts = pgz.pgz_inspect_parts(ctx_b)
    window_bytes = int((nph_parts > 0).sum()) * 32768

    # ---- plain: one file at a time through pgz_decompress, PLAIN_PARTS equal parts per file, with the
    # batched form's CTA shape and execution form
    ctx_p = pgz.pgz_create(pgz.pgz_config_init(device=dev, cuda_stream=stream.cuda_stream, n_chunks=PLAIN_PARTS,
                                               warps_per_block=wpb, exec_pipelined=xp))

    def step_plain(stats=False):
        res = []
        for k, (_, raw, g) in enumerate(files):
            st, n, s = pgz.pgz_decompress(ctx_p, jobs[k][0], jobs[k][1], jobs[k][2], jobs[k][3], stats)
            if st != 0 or n != len(raw):
                raise RuntimeError(f"pgz_decompress failed: {pgz.pgz_strerror(st)}")
            res.append(s)
        return res

    step_plain()
    check("plain")
    ms_plain, _ = timed(step_plain, ctx_p)
    per_level = {}
    for (label, raw, g), s in zip(files, step_plain(stats=True)):
        per_level[label] = {"parts": s["chunks"], "empty_parts": s["empty_chunks"], "false_syncs": s["false_syncs"],
                            "retries": s["retries"], "placeholder_fraction": round(s["placeholders"] / max(1, s["symbols"]), 4),
                            "in_bytes": len(g), "ms": round(s["ms_total"], 3)}
    pgz.pgz_destroy(ctx_p)

    # ---- end to end: pinned host input -> device, the batched run, device -> pinned host output
    pin_in = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).pin_memory() for _, _, g in files]
    pin_out = [torch.empty(len(r) + 4096, dtype=torch.uint8).pin_memory() for _, r, _ in files]

    def e2e_step():
        for k in range(len(files)):
            gz_dev[k].copy_(pin_in[k], non_blocking=True)
        step_batched()
        for k, (_, raw, _) in enumerate(files):
            pin_out[k][:len(raw)].copy_(outs[k][:len(raw)], non_blocking=True)
        torch.cuda.synchronize()

    # ---- end to end, pipelined through the library's request loop (pgz_server_*): each file runs in its own
    # slot (stream), so the second file's upload overlaps the first file's decode and each download overlaps
    # what is still decoding; the slots' runs share the GPU as the batch does
    srv = pgz.Server(pgz.pgz_config_init(device=dev, chunk_bytes=chunk_bytes, warps_per_block=wpb,
                                         exec_pipelined=xp), slots=len(files))
    ids = [srv.add_file(gz_dev[k].data_ptr(), len(g)) for k, (_, _, g) in enumerate(files)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()

    def e2e_pipelined():
        evs = []
        for k in range(len(files)):
            with torch.cuda.stream(up):
                gz_dev[k].copy_(pin_in[k], non_blocking=True)
                e = torch.cuda.Event()
                e.record(up)
                evs.append(e)
        reqs, copied, nxt = [None] * len(files), [False] * len(files), 0
        while not all(copied):
            if nxt < len(files) and evs[nxt].query():        # the member is on the device: submit it
                reqs[nxt] = srv.submit(ids[nxt], outs[nxt].data_ptr(), outs[nxt].numel())
                nxt += 1
            srv.poll()
            for k, q in enumerate(reqs):
                if q is not None and not copied[k] and q.status >= 0:
                    if q.status != 0 or q.out_len != len(files[k][1]):
                        raise RuntimeError(f"served request failed: {pgz.pgz_strerror(q.status)}")
                    with torch.cuda.stream(down):
                        pin_out[k][:q.out_len].copy_(outs[k][:q.out_len], non_blocking=True)
                    copied[k] = True
        down.synchronize()

    def timed_host(step):
        """Each step timed on the host clock (it includes the copies and the host side of the calls); the
        median step is reported so that one host stall does not stand for the whole run."""
        step()
        for k, (_, raw, _) in enumerate(files):
            if pin_out[k][:len(raw)].numpy().tobytes() != raw:
                raise RuntimeError("e2e output mismatch")
            pin_out[k].zero_()
        steps = []
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step()
            steps.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(steps), sum(steps) / len(steps)

    e2e_serial_ms, _ = timed_host(e2e_step)
    e2e_ms, e2e_mean = timed_host(e2e_pipelined)
    srv.close()
    batch.free()
    pgz.pgz_destroy(ctx_b)
    if dist:
        ms, e2e_ms, ms_plain, e2e_serial_ms = max_over_ranks([ms, e2e_ms, ms_plain, e2e_serial_ms], "cuda")

    gbs = whole_job_gbs(total_out, world, ms)
    pk = _peaks()
    hbm = pk.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    pass1_ms = stage["ms_sync"] + stage["ms_inflate"]
    alg1 = total_in + 2 * total_out                  # compressed bytes read + u16 symbols written
    ach1 = alg1 / (pass1_ms * 1e-3) / 1e9
    alg4 = 3 * total_out + window_bytes              # u16 symbols and windows read, bytes written
    ach4 = alg4 / (stage["ms_translate"] * 1e-3) / 1e9 if stage["ms_translate"] > 0 else None
    alg5 = total_out                                 # bytes read by the CRC
    ach5 = alg5 / (stage["ms_crc"] * 1e-3) / 1e9 if stage["ms_crc"] > 0 else None
    tpb = PASS1_TRAFFIC_PER_OUT_BYTE.get((chunk_bytes, wpb, xp))
    traffic1 = tpb * total_out if tpb else None
    line = {
        "metric": METRIC,
        "value": round(gbs, 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": desc, "form": "batched (all files of the step in one graph-captured run)",
                   "files": len(files), "out_bytes_per_step": total_out, "in_bytes_per_step": total_in,
                   "chunk_bytes": chunk_bytes, "warps_per_block": wpb, "exec_pipelined": xp, "parts": batch_parts,
                   "l2": "inputs (%.0f MB) and outputs (%.0f MB) larger than L2" % (total_in / 1e6, total_out / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "compressed_MBps": round(world * total_in / (ms * 1e-3) / 1e6, 1),
        "plain": {"value": round(world * total_out / (ms_plain * 1e-3) / 1e9, 3), "unit": "GB/s",
                  "ms_per_step": round(ms_plain, 3), "parts_per_file": PLAIN_PARTS,
                  "form": "one file at a time through pgz_decompress", "per_level": per_level},
        "stages_ms": {k: round(v, 3) for k, v in stage.items()},
        "roofline": {"bound": "hbm", "kernel": "pass 1 (k_sync + k_inflate)", "achieved": round(ach1, 2),
                     "peak": hbm, "unit": "GB/s", "frac": round(ach1 / hbm, 5),
                     "traffic": round(traffic1) if traffic1 else None, "peak_source": peak_src},
        "roofline_translate": {"bound": "hbm", "kernel": "k_translate", "achieved": round(ach4, 1) if ach4 else None,
                               "peak": hbm, "unit": "GB/s", "frac": round(ach4 / hbm, 4) if ach4 else None,
                               "bytes": alg4, "window_bytes": window_bytes},
        "roofline_crc": {"bound": "hbm", "kernel": "k_crc", "achieved": round(ach5, 1) if ach5 else None,
                         "peak": hbm, "unit": "GB/s", "frac": round(ach5 / hbm, 4) if ach5 else None},
        "e2e": {"value": round(world * total_out / (e2e_ms * 1e-3) / 1e9, 3), "unit": "GB/s",
                "h2d_bytes_per_step": total_in, "d2h_bytes_per_step": total_out,
                "ms_per_step_median": round(e2e_ms, 3), "ms_per_step_mean": round(e2e_mean, 3),
                "path": "pinned host -> device copy per file, pgz_server_submit/poll (one slot per file), "
                        "device -> pinned host copy per file as it completes; copies overlap decoding",
                "serial": {"value": round(world * total_out / (e2e_serial_ms * 1e-3) / 1e9, 3),
                           "path": "both uploads, pgz_batch_run, both downloads, one after another"}},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "autotune": tune,
    }
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(files)
        line["zlib_context"] = zlib_context(files)
    return line


def timed_steps(step, steps: int, warmup: int, stream, dist: bool = False, mark=None):
    """W untimed steps, then K steps between barriers and synchronisations, timed by CUDA events on the
    launching stream: one event before the first step and one after each step.  Returns the mean ms per step
    over the K steps and the list of per-step times.  mark(0) / mark(1), if given, run just before and just
    after the timed steps."""
    import torch
    for _ in range(warmup):
        step()
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    if mark:
        mark(0)
    ev[0].record(stream)
    for k in range(steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if mark:
        mark(1)
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return ev[0].elapsed_time(ev[steps]) / steps, per


def stage_means(pgz, ctx, jobs, reps: int = 3):
    """Per-stage CUDA-event times of one run of the pass kernels over `jobs` (pgz_decompress_batch, the same
    launches as the captured graph), mean of reps runs, and the run's part count."""
    stage = {k: 0.0 for k in ("ms_sync", "ms_inflate", "ms_chain", "ms_translate", "ms_crc", "ms_total")}
    s = None
    for _ in range(reps):
        r, _, s = pgz.pgz_decompress_batch(ctx, jobs, stats=True)
        if r != 0:
            raise RuntimeError(f"pgz_decompress_batch failed: {pgz.pgz_strerror(r)}")
        for k in stage:
            stage[k] += s[k] / reps
    return stage, s["chunks"]


def rooflines(stage, total_in, total_out, window_bytes, hbm, traffic_per_out_byte=None, determined=0):
    """The pass-1 pair against HBM (its algorithmic bytes: compressed input read + symbols written, 2 bytes each
    or 1 in a determined tail), and the two HBM-bound stages: translation (symbols and windows read, bytes
    written) and CRC (bytes read)."""
    pass1_ms = stage["ms_sync"] + stage["ms_inflate"]
    alg1 = total_in + 2 * total_out - determined
    ach1 = alg1 / (pass1_ms * 1e-3) / 1e9
    alg4 = 3 * total_out - determined + window_bytes
    ach4 = alg4 / (stage["ms_translate"] * 1e-3) / 1e9 if stage["ms_translate"] > 0 else None
    ach5 = total_out / (stage["ms_crc"] * 1e-3) / 1e9 if stage["ms_crc"] > 0 else None
    traffic = round(traffic_per_out_byte * total_out) if traffic_per_out_byte else None
    return ({"bound": "hbm", "kernel": "pass 1 (k_sync + k_inflate)", "achieved": round(ach1, 2), "peak": hbm,
             "unit": "GB/s", "frac": round(ach1 / hbm, 5), "traffic": traffic, "algorithmic_bytes": alg1,
             "ms": round(pass1_ms, 3)},
            {"bound": "hbm", "kernel": "k_translate", "achieved": round(ach4, 1) if ach4 else None, "peak": hbm,
             "unit": "GB/s", "frac": round(ach4 / hbm, 4) if ach4 else None, "bytes": alg4,
             "window_bytes": window_bytes},
            {"bound": "hbm", "kernel": "k_crc", "achieved": round(ach5, 1) if ach5 else None, "peak": hbm,
             "unit": "GB/s", "frac": round(ach5 / hbm, 4) if ach5 else None, "bytes": total_out})


def config2_legs(pgz, files, dev, stream, steps: int, warmup: int, hbm: float):
    """The two 256 MiB FASTQ files (150 bp, seed 1) at gzip -1 and -9: batched (autotuned, graph) and plain
    (one pgz_decompress per file, 1024 equal parts), per-level block-start and placeholder statistics."""
    import numpy as np
    import torch
    labels = ["fastq-L1", "fastq-L9"]
    gz_dev = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).cuda() for _, g in files]
    outs = [torch.empty(len(r) + 4096, dtype=torch.uint8, device="cuda") for r, _ in files]
    refs = [torch.from_numpy(np.frombuffer(r, dtype=np.uint8).copy()).cuda() for r, _ in files]
    jobs = [(gz_dev[k].data_ptr(), len(g), outs[k].data_ptr(), outs[k].numel()) for k, (_, g) in enumerate(files)]
    total_out = sum(len(r) for r, _ in files)
    total_in = sum(len(g) for _, g in files)

    def check(what):
        torch.cuda.synchronize()
        for k, (r, _) in enumerate(files):
            if not torch.equal(outs[k][:len(r)], refs[k]):
                raise RuntimeError(f"output mismatch ({what}, {labels[k]})")
            outs[k].zero_()

    ctx = pgz.pgz_create(pgz.pgz_config_init(device=dev, cuda_stream=stream.cuda_stream))
    tune = autotune(pgz, ctx, jobs, sorted(set(TUNE_CHUNKS) | set(wave_sizes(pgz, ctx, jobs, [4, 8], [1, 2]))),
                    TUNE_WPB)
    chunk, wpb, xp = tune["best"]
    batch = pgz.Batch(ctx, jobs)

    def step_batched():
        r, res, _ = batch.run()
        if r != 0:
            raise RuntimeError(f"pgz_batch_run failed: {pgz.pgz_strerror(r)}")

    step_batched()
    check("batched")
    ms_b, per_b = timed_steps(step_batched, steps, warmup, stream)
    stage, parts = stage_means(pgz, ctx, jobs)
    _, _, nph_parts = pgz.pgz_inspect_parts(ctx)
    window_bytes = int((nph_parts > 0).sum()) * 32768
    batch.free()
    pgz.pgz_destroy(ctx)
    ctx_p = pgz.pgz_create(pgz.pgz_config_init(device=dev, cuda_stream=stream.cuda_stream, n_chunks=PLAIN_PARTS,
                                               warps_per_block=wpb, exec_pipelined=xp))

    def step_plain(stats=False):
        res = []
        for k, (r, _) in enumerate(files):
            st, n, s = pgz.pgz_decompress(ctx_p, *jobs[k], stats)
            if st != 0 or n != len(r):
                raise RuntimeError(f"pgz_decompress failed: {pgz.pgz_strerror(st)}")
            res.append(s)
        return res

    step_plain()
    check("plain")
    ms_p, _ = timed_steps(step_plain, steps, warmup, stream)
    per_level = {}
    for label, (r, g), s in zip(labels, files, step_plain(stats=True)):
        per_level[label] = {"parts": s["chunks"], "empty_parts": s["empty_chunks"], "false_syncs": s["false_syncs"],
                            "retries": s["retries"],
                            "placeholder_fraction": round(s["placeholders"] / max(1, s["symbols"]), 4),
                            "in_bytes": len(g), "ms": round(s["ms_total"], 3)}
    pgz.pgz_destroy(ctx_p)
    r1, r4, r5 = rooflines(stage, total_in, total_out, window_bytes, hbm,
                           PASS1_TRAFFIC_PER_OUT_BYTE.get((chunk, wpb, xp)))
    return {"workload": "2 x 256 MiB synthetic FASTQ (150 bp, seed 1), gzip -1 and -9",
            "out_bytes_per_step": total_out, "in_bytes_per_step": total_in,
            "batched": {"value": round(total_out / (ms_b * 1e-3) / 1e9, 3), "unit": "GB/s", "ms_per_step": round(ms_b, 3),
                        "step_ms": {"median": round(statistics.median(per_b), 3), "min": round(min(per_b), 3),
                                    "max": round(max(per_b), 3)},
                        "chunk_bytes": chunk, "warps_per_block": wpb, "exec_pipelined": xp, "parts": parts},
            "plain": {"value": round(total_out / (ms_p * 1e-3) / 1e9, 3), "unit": "GB/s", "ms_per_step": round(ms_p, 3),
                      "parts_per_file": PLAIN_PARTS, "form": "one file at a time through pgz_decompress",
                      "per_level": per_level},
            "stages_ms": {k: round(v, 3) for k, v in stage.items()},
            "roofline_pass1": r1, "roofline_translate": r4, "roofline_crc": r5, "autotune": tune}


def _stage_line(stage, total_in, total_out, window_bytes, hbm):
    stage = {k: v for k, v in stage.items() if k.startswith("ms_")}
    t = stage["ms_translate"] * 1e-3
    c = stage["ms_crc"] * 1e-3
    return {"stages_ms": {k: round(v, 3) for k, v in stage.items()},
            "roofline_translate": {"achieved": round((3 * total_out + window_bytes) / t / 1e9, 1) if t else None,
                                   "frac": round((3 * total_out + window_bytes) / t / 1e9 / hbm, 4) if t else None},
            "roofline_crc": {"achieved": round(total_out / c / 1e9, 1) if c else None,
                             "frac": round(total_out / c / 1e9 / hbm, 4) if c else None}}


def wave_sizes(pgz, ctx, jobs, wpbs, waves):
    """Part sizes that give whole waves of the resident pass-1 warps over these jobs (pgz_wave_chunk_bytes),
    for each CTA shape and wave count."""
    out = set()
    for w in wpbs:
        for k in waves:
            st, cb, _ = pgz.pgz_wave_chunk_bytes(ctx, jobs, w, k)
            if st == 0:
                out.add(cb)
    return sorted(out)


def autotune(pgz, ctx, jobs, chunks, wpbs):
    """The library's autotuner over part size x pass-1 CTA shape x pass-1 execution form on these jobs; the
    context keeps the fastest configuration.  Returns {"best": [chunk, wpb, pipelined], "ms": {...}}."""
    st, entries, best = pgz.pgz_autotune(ctx, jobs, chunks, wpbs, 2, sweep_exec=True)
    if st != 0:
        raise RuntimeError(f"pgz_autotune failed: {pgz.pgz_strerror(st)}")
    return {"best": [best["chunk_bytes"], best["warps_per_block"], best["exec_pipelined"]],
            "ms": {f"{e['chunk_bytes'] >> 10}K/{e['warps_per_block']}w/{'p' if e['exec_pipelined'] else 's'}":
                   round(e["ms"], 2) for e in entries}}


def run_tune4g(args):
    """4 GiB FASTQ (150 bp, 1 % N, seed 2) at gzip -6, ISIZE = 0: the autotuner's sweep of part size x pass-1
    CTA shape, then the chosen pair timed."""
    import numpy as np
    import torch
    from paper_1905_07224_gb300 import build, pgz, synth
    build.build()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    raw = synth.fastq_large(4 << 30, 150, 0.01, 2)
    gz = synth.gzip_compress_parallel(raw, 6)
    t_make = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    ctx = pgz.pgz_create(pgz.pgz_config_init(device=0, cuda_stream=stream.cuda_stream))
    d_in = torch.from_numpy(np.frombuffer(gz, dtype=np.uint8).copy()).cuda()
    d_out = torch.empty(len(raw) + 4096, dtype=torch.uint8, device="cuda")
    chunks = [32 << 10, 64 << 10, 128 << 10, 256 << 10, 512 << 10, 1 << 20, 2 << 20, 4 << 20]
    tune = autotune(pgz, ctx, [(d_in.data_ptr(), len(gz), d_out.data_ptr(), d_out.numel())], chunks, [2, 4, 8])
    ref = torch.from_numpy(np.frombuffer(raw, dtype=np.uint8).copy()).cuda()
    if not torch.equal(d_out[:len(raw)], ref):
        raise RuntimeError("output mismatch")
    for _ in range(args.warmup):
        pgz.pgz_decompress(ctx, d_in.data_ptr(), len(gz), d_out.data_ptr(), d_out.numel())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st, n, _ = pgz.pgz_decompress(ctx, d_in.data_ptr(), len(gz), d_out.data_ptr(), d_out.numel())
        if st != 0 or n != len(raw):
            raise RuntimeError(f"pgz_decompress failed: {pgz.pgz_strerror(st)}")
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    st, n, s = pgz.pgz_decompress(ctx, d_in.data_ptr(), len(gz), d_out.data_ptr(), d_out.numel(), True)
    _, _, nph = pgz.pgz_inspect_parts(ctx)
    pgz.pgz_destroy(ctx)
    hbm = _peaks().get("hbm_gbs") or 6800.0
    line = {"workload": "4 GiB synthetic FASTQ (150 bp, 1 % N, seed 2), gzip -6 (parallel pieces, one member), "
                        "ISIZE 0", "in_bytes": len(gz), "out_bytes": len(raw), "isize": int.from_bytes(gz[-4:], "little"),
            "make_s": round(t_make, 1), "tune": tune["ms"], "best": tune["best"], "parts": s["chunks"],
            "value": round(len(raw) / (ms * 1e-3) / 1e9, 3), "unit": "GB/s", "ms_per_call": round(ms, 3),
            "placeholder_fraction": round(s["placeholders"] / max(1, s["symbols"]), 4),
            "false_syncs": s["false_syncs"], "retries": s["retries"], "empty_parts": s["empty_chunks"]}
    line.update(_stage_line(s, len(gz), len(raw), int((nph > 0).sum()) * 32768, hbm))
    return line


def run_headline(args, rank, world):
    """The 512 members: batched (autotuned, one graph-captured run) against plain (one pgz_decompress per
    member); e2e through pgz_decompress_batch_host; on rank 0 also the config-2 files, the served loop and the
    oracle on the host's cores."""
    import numpy as np
    import torch
    from paper_1905_07224_gb300 import build, pgz, synth
    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = world > 1
    extras = rank == 0 and not args.headline_only
    t0 = time.perf_counter()
    man4 = synth.batch_manifest(512, 3)
    man2 = [("fastq", 256 << 20, 1, 1), ("fastq", 256 << 20, 9, 1)] if extras else []
    man5, rng5 = served_manifest() if extras and args.served_requests > 0 else ([], None)
    allf = synth.make_files(man4 + man2 + man5)
    files, files2, files5 = allf[:512], allf[512:512 + len(man2)], allf[512 + len(man2):]
    t_make = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    total_out = sum(len(r) for r, _ in files)
    total_in = sum(len(g) for _, g in files)
    d_in = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).cuda() for _, g in files]
    d_out = [torch.empty(len(r) + 4096, dtype=torch.uint8, device="cuda") for r, _ in files]
    refs = [torch.from_numpy(np.frombuffer(r, dtype=np.uint8).copy()).cuda() for r, _ in files]
    jobs = [(d_in[k].data_ptr(), len(g), d_out[k].data_ptr(), d_out[k].numel()) for k, (_, g) in enumerate(files)]

    def check(what):
        torch.cuda.synchronize()
        for k, (r, _) in enumerate(files):
            if not torch.equal(d_out[k][:len(r)], refs[k]):
                raise RuntimeError(f"output mismatch ({what}, member {k})")
            d_out[k].zero_()

    # ---- batched: every member in one graph-captured run, the configuration chosen by the autotuner
    ctx = pgz.pgz_create(pgz.pgz_config_init(device=dev, cuda_stream=stream.cuda_stream,
                                             chunk_bytes=args.chunk_bytes or (256 << 10),
                                             warps_per_block=args.warps_per_block,
                                             exec_pipelined=args.exec_pipelined))
    tune = None if args.chunk_bytes else autotune(
        pgz, ctx, jobs, sorted(set(TUNE_CHUNKS_BATCH) | set(wave_sizes(pgz, ctx, jobs, [4], [1, 2, 3, 4]))),
        TUNE_WPB_BATCH)
    chunk, wpb, xp = tune["best"] if tune else (args.chunk_bytes, args.warps_per_block, args.exec_pipelined)
    batch = pgz.Batch(ctx, jobs)

    def step_batched():
        r, res, _ = batch.run()
        if r != 0:
            raise RuntimeError(f"pgz_batch_run failed: {pgz.pgz_strerror(r)}")

    step_batched()
    check("batched")
    count = [0, 0]

    def mark(k):
        count[k] = pgz.pgz_kernel_launches(ctx)

    with Clocks(dev) as clk:
        ms, per = timed_steps(step_batched, args.steps, args.warmup, stream, dist, mark)
    clocks = clk.summary()
    launches = count[1] - count[0]
    # the same steps with no clock sampler running (a check that sampling does not disturb the timed region)
    ms_quiet, per_quiet = timed_steps(step_batched, args.steps, 1, stream, dist)
    stage, parts = stage_means(pgz, ctx, jobs)
    _, _, nph_parts = pgz.pgz_inspect_parts(ctx)
    window_bytes = int((nph_parts > 0).sum()) * 32768
    batch.free()
    # the same configuration with the determined tail (pass 1 stores a part's symbols as bytes once its last
    # 32 KiB hold no placeholder): timed the same way, reported beside; the faster of the two is the value
    ctx_t = pgz.pgz_create(pgz.pgz_config_init(device=dev, cuda_stream=stream.cuda_stream, chunk_bytes=chunk,
                                               warps_per_block=wpb, exec_pipelined=xp, determined_tail=1))
    batch_t = pgz.Batch(ctx_t, jobs)

    def step_tail():
        r, res, _ = batch_t.run()
        if r != 0:
            raise RuntimeError(f"pgz_batch_run (determined tail) failed: {pgz.pgz_strerror(r)}")

    step_tail()
    check("batched, determined tail")
    count_t = [0, 0]

    def mark_t(k):
        count_t[k] = pgz.pgz_kernel_launches(ctx_t)

    with Clocks(dev) as clk_t:
        ms_t, per_t = timed_steps(step_tail, args.steps, args.warmup, stream, dist, mark_t)
    clocks_t = clk_t.summary()
    stage_t, _ = stage_means(pgz, ctx_t, jobs)
    _, _, s_t = pgz.pgz_decompress_batch(ctx_t, jobs, stats=True)
    determined = s_t["determined"]
    batch_t.free()
    pgz.pgz_destroy(ctx_t)
    tail_leg = {"ms_per_step": round(ms_t, 3), "value": round(whole_job_gbs(total_out, world, ms_t), 3),
                "determined_fraction": round(determined / total_out, 4),
                "stages_ms": {k: round(v, 3) for k, v in stage_t.items()}}
    use_tail = ms_t < ms
    if use_tail:
        ms, per, clocks, stage, launches = ms_t, per_t, clocks_t, stage_t, count_t[1] - count_t[0]

    # ---- plain: one pgz_decompress per member, the library's default part size
    ctx_p = pgz.pgz_create(pgz.pgz_config_init(device=dev, cuda_stream=stream.cuda_stream, chunk_bytes=CHUNK_BYTES))

    def step_plain():
        for gp, gl, op, oc in jobs:
            st, n, _ = pgz.pgz_decompress(ctx_p, gp, gl, op, oc)
            if st != 0:
                raise RuntimeError(f"pgz_decompress failed: {pgz.pgz_strerror(st)}")

    step_plain()
    check("plain")
    steps_plain = max(1, min(args.steps, 3))
    ms_plain, _ = timed_steps(step_plain, steps_plain, 1, stream, dist)
    pgz.pgz_destroy(ctx_p)

    # ---- end to end: pinned host memory in and out, through the C ABI's host-buffer batch call
    pin_in = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).pin_memory() for _, g in files]
    pin_out = [torch.zeros(len(r) + 4096, dtype=torch.uint8).pin_memory() for r, _ in files]
    hjobs = [(pin_in[k].data_ptr(), len(g), pin_out[k].data_ptr(), pin_out[k].numel()) for k, (_, g) in enumerate(files)]

    def e2e_step():
        r, res, _ = pgz.pgz_decompress_batch_host(ctx, hjobs)
        if r != 0:
            raise RuntimeError(f"pgz_decompress_batch_host failed: {pgz.pgz_strerror(r)}")

    e2e_step()
    for k, (r, _) in enumerate(files):
        if pin_out[k][:len(r)].numpy().tobytes() != r:
            raise RuntimeError(f"e2e output mismatch (member {k})")
    e2e = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        e2e_step()
        if k >= args.warmup:
            e2e.append((time.perf_counter() - t) * 1e3)
    e2e_ms = statistics.median(e2e)
    pgz.pgz_destroy(ctx)
    del pin_in, pin_out
    if dist:
        ms, ms_plain, e2e_ms = max_over_ranks([ms, ms_plain, e2e_ms], "cuda")

    pk = _peaks()
    hbm = pk.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    r1, r4, r5 = rooflines(stage, total_in, total_out, window_bytes, hbm,
                           PASS1_TRAFFIC_PER_OUT_BYTE_BATCH512.get((chunk, wpb, xp, int(use_tail))),
                           determined if use_tail else 0)
    r1["peak_source"] = peak_src
    gbs = whole_job_gbs(total_out, world, ms)
    plain_gbs = whole_job_gbs(total_out, world, ms_plain)
    line = {
        "metric": METRIC,
        "value": round(gbs, 3),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "gpu_launches": int(launches),
        "config": {"workload": HEADLINE_DESC, "members": len(files),
                   "form": "batched: every member in one graph-captured run of the pass kernels",
                   "out_bytes_per_step": total_out, "in_bytes_per_step": total_in, "chunk_bytes": chunk,
                   "warps_per_block": wpb, "exec_pipelined": xp, "determined_tail": int(use_tail), "parts": parts,
                   "l2": "inputs (%.1f GB) and outputs (%.1f GB) larger than L2" % (total_in / 1e9, total_out / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "compressed_MBps": round(world * total_in / (ms * 1e-3) / 1e6, 1),
        "step_ms": {"median": round(statistics.median(per), 3), "min": round(min(per), 3), "max": round(max(per), 3),
                    "without_clock_sampler": round(ms_quiet, 3)},
        "plain": {"value": round(plain_gbs, 3), "unit": "GB/s", "ms_per_step": round(ms_plain, 3),
                  "steps": steps_plain, "form": "one pgz_decompress per member", "chunk_bytes": CHUNK_BYTES},
        "batched_over_plain": round(gbs / plain_gbs, 2),
        "determined_tail": tail_leg,
        "stages_ms": {k: round(v, 3) for k, v in stage.items()},
        "roofline": r1, "roofline_translate": r4, "roofline_crc": r5,
        "e2e": {"value": round(whole_job_gbs(total_out, world, e2e_ms), 3), "unit": "GB/s",
                "h2d_bytes_per_step": total_in, "d2h_bytes_per_step": total_out,
                "ms_per_step_median": round(e2e_ms, 3), "ms_per_step_min": round(min(e2e), 3),
                "path": "pgz_decompress_batch_host (C ABI): pinned host input and output, the host-device copies "
                        "inside the call, overlapped with decoding group by group; host clock around each call"},
        "clocks": clocks,
        "autotune": tune,
        "make_s": round(t_make, 1),
    }
    if extras:
        if files2:
            line["fastq256"] = config2_legs(pgz, files2, dev, stream, args.steps, args.warmup, hbm)
        if files5:
            line["served"] = served_legs(pgz, files5, rng5, args.served_requests, CHUNK_BYTES, dev)
        cpu, zl = cpu_baseline_parallel(files)
        line["cpu_baseline"] = cpu
        line["zlib_context"] = zl
    return line


def run_stream(args):
    """Memory-bounded streaming: the 4 GiB FASTQ member (150 bp, 1 % N, seed 2, gzip -6, ISIZE 0) held in host
    memory, decoded by pgz_decompress_stream in 256 MiB segments of compressed data, output handed to a sink
    that copies it into a host array (and, second, to a sink that drops it).  Host clock around each call
    (the call is synchronous); median of the steps.  Beside it: the device memory the streaming context holds
    and the memory the whole-member host path (pgz_decompress_host) holds for the same member."""
    import numpy as np
    import torch
    from paper_1905_07224_gb300 import build, pgz, synth
    build.build()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    raw = synth.fastq_large(4 << 30, 150, 0.01, 2)
    gz = np.frombuffer(synth.gzip_compress_parallel(raw, 6), dtype=np.uint8)
    ref = np.frombuffer(raw, dtype=np.uint8)
    t_make = time.perf_counter() - t0
    seg = 256 << 20
    dst = np.empty(len(raw), dtype=np.uint8)
    pos = [0]

    def copy_sink(v):
        a = np.frombuffer(v, dtype=np.uint8)
        dst[pos[0]:pos[0] + a.size] = a
        pos[0] += a.size
        return 0

    nseg = [0]

    def count_sink(v):
        nseg[0] += 1
        return 0

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx = pgz.pgz_create(pgz.pgz_config_init(device=0))
    st, n, s, _ = pgz.pgz_decompress_stream(ctx, gz, seg, sink=copy_sink, stats=True)
    if st != 0 or n != len(raw) or not np.array_equal(dst, ref):
        raise RuntimeError(f"pgz_decompress_stream failed: {pgz.pgz_strerror(st)}")
    held_stream = free0 - torch.cuda.mem_get_info()[0]
    pgz.pgz_decompress_stream(ctx, gz, seg, sink=count_sink)
    segments = nseg[0]

    def timed(sink):
        ts = []
        for k in range(args.warmup + args.steps):
            pos[0] = 0
            t = time.perf_counter()
            r, m, _, _ = pgz.pgz_decompress_stream(ctx, gz, seg, sink=sink)
            dt = time.perf_counter() - t
            if r != 0 or m != len(raw):
                raise RuntimeError(f"pgz_decompress_stream failed: {pgz.pgz_strerror(r)}")
            if k >= args.warmup:
                ts.append(dt)
        return float(np.median(ts))

    t_copy = timed(copy_sink)
    t_noop = timed(lambda v: 0)
    pgz.pgz_destroy(ctx)
    # the whole member at once through the host entry point, for the memory it needs
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    ctx = pgz.pgz_create(pgz.pgz_config_init(device=0))
    out = np.empty(len(raw) + 4096, dtype=np.uint8)
    ts = []
    for k in range(1 + args.steps):
        t = time.perf_counter()
        r, m, _ = pgz.pgz_decompress_host(ctx, gz, out)
        ts.append(time.perf_counter() - t)
        if r != 0 or m != len(raw):
            raise RuntimeError(f"pgz_decompress_host failed: {pgz.pgz_strerror(r)}")
    held_whole = free1 - torch.cuda.mem_get_info()[0]
    t_whole = float(np.median(ts[1:]))
    pgz.pgz_destroy(ctx)
    D = len(raw)
    return {"workload": "4 GiB synthetic FASTQ (150 bp, 1 % N, seed 2), gzip -6, one member, ISIZE 0, in host memory",
            "in_bytes": int(gz.size), "out_bytes": D, "make_s": round(t_make, 1), "segment_bytes": seg,
            "segments": segments, "unit": "GB/s",
            "value": round(D / t_copy / 1e9, 3),
            "form": "pgz_decompress_stream, host in, sink copies each segment into a host array",
            "value_sink_drops": round(D / t_noop / 1e9, 3),
            "whole_member_host": {"value": round(D / t_whole / 1e9, 3),
                                  "form": "pgz_decompress_host (whole member on the device, copies in the call)"},
            "device_bytes_held": {"stream": int(held_stream), "whole_member": int(held_whole)},
            "stages_ms_summed": {k: round(v, 3) for k, v in s.items() if k.startswith("ms_")},
            "timing": "host clock around each synchronous call, median of the steps after the warm-up"}


def served_manifest():
    """The served pool: 256 members, log-uniform 4 KiB .. 256 MiB (seed 4), half FASTQ and half Markov text,
    levels 1/6/9.  Returns the manifest and the generator, which goes on to draw the requests."""
    import numpy as np
    from paper_1905_07224_gb300 import synth
    rng = np.random.default_rng(4)
    sizes = synth.log_uniform_sizes(256, 4 << 10, 256 << 20, rng)
    levels = rng.choice(np.array([1, 6, 9]), size=256)
    entries = [("fastq" if k % 2 == 0 else "markov", int(sizes[k]), int(levels[k]), 400003 + k) for k in range(256)]
    return entries, rng


def served_legs(pgz, files, rng, n_req: int, chunk_bytes: int, dev: int = 0):
    """Poisson arrivals at offered loads of 1, 4 and 16 GB/s decompressed (rate = load / mean member size);
    70 % whole members and 30 % byte ranges (offset uniform, length log-uniform 4 KiB .. 1 MiB, clipped);
    n_req requests per load, 4 slots, a 64 GiB device-memory budget.  Latency runs from the scheduled arrival
    to the completion seen by the host; 40 results per load are checked byte for byte."""
    import numpy as np
    import torch
    mean_d = float(np.mean([len(r) for r, _ in files]))
    srv = pgz.Server(pgz.pgz_config_init(device=dev, chunk_bytes=chunk_bytes), slots=4, mem_budget=64 << 30)
    d_in = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).cuda() for _, g in files]
    ids = [srv.add_file(d.data_ptr(), len(g)) for d, (_, g) in zip(d_in, files)]
    results = []
    for load in (1e9, 4e9, 16e9):
        lam = load / mean_d
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
        reqs = []
        for _ in range(n_req):
            f = int(rng.integers(len(files)))
            D = len(files[f][0])
            if rng.random() < 0.7:
                reqs.append((f, None, None, D))
            else:
                off = int(rng.integers(D))
                ln = int(min(D - off, np.exp(rng.uniform(np.log(4 << 10), np.log(1 << 20)))))
                reqs.append((f, off, ln, ln))
        outs = [torch.empty(r[3] + 64, dtype=torch.uint8, device="cuda") for r in reqs]
        torch.cuda.synchronize()
        qs = []
        start = time.monotonic()
        for k, (f, off, ln, _) in enumerate(reqs):
            while time.monotonic() - start < arrivals[k]:
                srv.poll()
            qs.append(srv.submit(ids[f], outs[k].data_ptr(), outs[k].numel(), offset=off or 0, length=ln))
        while srv.pending():
            srv.poll()
        end = max(q.t_done for q in qs)
        lat = np.array([q.t_done - (start + arrivals[k]) for k, q in enumerate(qs)]) * 1e3
        bad = sum(q.status != 0 for q in qs)
        for k in rng.choice(n_req, size=min(40, n_req), replace=False):      # exact bytes, sampled
            f, off, ln, _ = reqs[k]
            raw = files[f][0] if off is None else files[f][0][off:off + ln]
            if outs[k][:len(raw)].cpu().numpy().tobytes() != raw:
                raise RuntimeError(f"served request {k}: output mismatch")
        served = sum(r[3] for r in reqs)
        results.append({"offered_GBps": load / 1e9, "requests": n_req, "failed": int(bad),
                        "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                        "achieved_GBps": round(served / (end - start) / 1e9, 3),
                        "span_s": round(end - start, 3)})
        del outs
    srv.close()
    return {"workload": "served: 256 synthetic members, log-uniform 4 KiB-256 MiB (seed 4), FASTQ/Markov, "
                        "gzip -1/-6/-9; Poisson arrivals, 70 % whole / 30 % ranges, 64 GiB budget, 4 slots",
            "mean_member_bytes": round(mean_d), "chunk_bytes": chunk_bytes,
            "latency": "scheduled arrival to completion seen by the host", "loads": results}


def run_served(args):
    """Served requests at the full request count (2000 per load unless PGZ_SERVED_REQUESTS says otherwise)."""
    import torch
    from paper_1905_07224_gb300 import build, pgz, synth
    build.build()
    torch.cuda.set_device(0)
    entries, rng = served_manifest()
    t0 = time.perf_counter()
    files = synth.make_files(entries)
    t_make = time.perf_counter() - t0
    n_req = int(os.environ.get("PGZ_SERVED_REQUESTS", "2000"))
    out = served_legs(pgz, files, rng, n_req, args.chunk_bytes or CHUNK_BYTES)
    out["make_s"] = round(t_make, 1)
    return out


def cpu_baseline(files, budget_s: float = 20.0):
    """The oracle (plain bit-at-a-time inflater, one thread) on the same files."""
    import oracle
    oracle.build()
    done_out, t_used, sample = 0, 0.0, []
    for label, raw, gz in files:
        if t_used > budget_s:
            break
        t0 = time.perf_counter()
        e, out, _, _ = oracle.gunzip(gz, cap=len(raw) + 1024)
        dt = time.perf_counter() - t0
        if e != 0 or len(out) != len(raw):
            raise RuntimeError("oracle failed")
        t_used += dt
        done_out += len(raw)
        sample.append(label)
    return {"value": round(done_out / t_used / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle.gunzip (one thread) over {', '.join(sample)} ({done_out >> 20} MiB out, {t_used:.1f} s)"}


def zlib_context(files):
    """Host zlib inflate, one thread, on the same files: context beside the oracle, not a target."""
    import zlib
    t0 = time.perf_counter()
    done = 0
    for _, raw, gz in files:
        if len(zlib.decompress(gz, 31)) != len(raw):
            raise RuntimeError("zlib failed")
        done += len(raw)
    dt = time.perf_counter() - t0
    return {"value": round(done / dt / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "host zlib (context)",
            "sample": f"zlib.decompress (one thread) over the step's files ({done >> 20} MiB out, {dt:.1f} s)"}


def cpu_baseline_parallel(members, target_s: float = 10.0):
    """The oracle file-parallel on all host cores over a bounded sample of the members (list of (raw, gz)),
    and host zlib on one core over the same sample as context.  The sample is the first members, in order,
    up to about target_s seconds of the oracle's work per core (at 60 MB/s per core)."""
    import zlib
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    want = target_s * 60e6 * cores
    sample, out = [], 0
    for raw, gz in members:
        if out >= want:
            break
        sample.append((raw, gz))
        out += len(raw)

    def one(m):
        raw, gz = m
        e, o, _, _ = oracle.gunzip(gz, cap=len(raw) + 1024)    # the C oracle releases the GIL
        if e != 0 or len(o) != len(raw):
            raise RuntimeError("oracle failed")
        return len(raw)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        done = sum(ex.map(one, sample))
    t_or = time.perf_counter() - t0
    t0 = time.perf_counter()
    for raw, gz in sample:
        if len(zlib.decompress(gz, 31)) != len(raw):
            raise RuntimeError("zlib failed")
    t_z = time.perf_counter() - t0
    desc = f"the first {len(sample)} members ({done >> 20} MiB out)"
    return ({"value": round(done / t_or / 1e9, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
             "sample": f"oracle.gunzip, one member per thread on {cores} threads, over {desc}, {t_or:.1f} s"},
            {"value": round(done / t_z / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "host zlib (context)",
             "sample": f"zlib.decompress, one thread, over {desc}, {t_z:.1f} s"})


def run_reference_batch512(args, budget_s: float = 150.0, oracle_gbs_per_core: float = 0.06):
    """--impl reference on the 512 members: the CPU oracle, as it stands (oracle.gunzip, trailer checked), one
    member per thread on every host core.  A step decodes the first members of the manifest up to about
    budget_s / (W + K) seconds of the oracle's work at oracle_gbs_per_core GB/s per core (all 512 when they
    fit), so the whole run ends within a few minutes."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    from paper_1905_07224_gb300 import synth
    oracle.build()
    t0 = time.perf_counter()
    files = synth.make_files(synth.batch_manifest(512, 3))
    t_make = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    want = budget_s / (args.warmup + args.steps) * oracle_gbs_per_core * 1e9 * cores
    sample, out = [], 0
    for raw, gz in files:
        if sample and out + len(raw) > want:
            break
        sample.append((raw, gz))
        out += len(raw)

    def one(m):
        raw, gz = m
        e, o, _, _ = oracle.gunzip(gz, cap=len(raw) + 1024)    # the C oracle releases the GIL
        if e != 0 or len(o) != len(raw):
            raise RuntimeError("oracle failed")
        return len(raw)

    with ThreadPoolExecutor(max_workers=cores) as ex:
        def step():
            return sum(ex.map(one, sorted(sample, key=lambda m: -len(m[0]))))
        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        done = sum(step() for _ in range(args.steps))
        dt = time.perf_counter() - t0
    v = done / dt / 1e9
    what = "all 512 members" if len(sample) == len(files) else f"the first {len(sample)} of the 512 members"
    desc = f"oracle.gunzip, one member per thread on {cores} threads, {what} ({out >> 20} MiB out) per step"
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": HEADLINE_DESC, "members": len(files),
                       "out_bytes_per_step": out, "sample_members": len(sample)},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "make_s": round(t_make, 1)}


def run_reference(args, budget_s: float = 150.0, oracle_gbs: float = 0.06):
    """--impl reference: the CPU oracle, as it stands, on the same workload.  A step decodes every file of
    the workload -- whole (oracle.gunzip, trailer checked) when the whole run fits in about budget_s seconds
    at the oracle's speed of about oracle_gbs GB/s, else the same prefix of each file, up to the first block
    boundary past that fraction of its compressed data (oracle.inflate_from from the first block, whole
    blocks, empty context)."""
    import oracle
    oracle.build()
    files, desc = make_workload(args.workload)
    total = sum(len(r) for _, r, _ in files)
    frac = min(1.0, budget_s / (args.warmup + args.steps) / (total / (oracle_gbs * 1e9)))

    def step():
        done = 0
        for _, raw, gz in files:
            if frac >= 1.0:
                e, out, _, _ = oracle.gunzip(gz, cap=len(raw) + 1024)
                if e != 0 or len(out) != len(raw):
                    raise RuntimeError("oracle failed")
                done += len(out)
            else:
                s0 = oracle.gzip_header(gz)
                end_bit = (len(gz) - 8) * 8
                stop = s0 * 8 + int(frac * (end_bit - s0 * 8))
                r = oracle.inflate_from(gz, end_bit, s0 * 8, stop_bit=stop, known=True, cap=len(raw) + 1024)
                if r["status"] != 0:
                    raise RuntimeError("oracle failed")
                done += r["n"]
        return done

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    done = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    ms = dt * 1e3 / args.steps
    v = done / dt / 1e9
    sample = ("the whole workload per step (oracle.gunzip)" if frac >= 1.0 else
              f"the first {100 * frac:.0f} % of each file's compressed data per step, to a block boundary "
              f"(oracle.inflate_from), {done // args.steps >> 20} MiB out per step")
    return {"impl": "reference", "metric": METRIC,
            "value": round(v, 4), "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic", "config": {"workload": desc, "out_bytes_per_step": total},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"one thread; {sample}"},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(spec: str, chunk_bytes: int, wpb: int = 4, xp: int = 0):
    """--profile-case MIB:LEVEL:CALLS -- a small fixed case for ncu captures: one synthetic FASTQ file
    (150 bp, seed 1) of MIB MiB at gzip LEVEL, decompressed CALLS times through pgz_decompress on device
    buffers; the output of the last call is checked byte for byte and its stage times printed."""
    import numpy as np
    import torch
    from paper_1905_07224_gb300 import build, pgz, synth
    if spec.startswith("batch:"):
        return run_profile_batch(int(spec.split(":")[1]), chunk_bytes, wpb, xp)
    if spec.startswith("batchsweep:"):
        return run_profile_sweep(spec.split(":", 1)[1])
    if spec.startswith("members:"):
        _, nm, calls = spec.split(":")
        return run_profile_members(int(nm), int(calls), chunk_bytes, wpb, xp)
    mib, level, calls = (int(x) for x in spec.split(":"))
    build.build()
    raw = synth.fastq(mib << 20, 150, 0.001, 1)
    gz = synth.gzip_compress(raw, level)
    stream = torch.cuda.current_stream()
    ctx = pgz.pgz_create(pgz.pgz_config_init(device=0, cuda_stream=stream.cuda_stream, n_chunks=0,
                                             chunk_bytes=chunk_bytes, warps_per_block=wpb, exec_pipelined=xp))
    d_in = torch.from_numpy(np.frombuffer(gz, dtype=np.uint8).copy()).cuda()
    d_out = torch.empty(len(raw) + 4096, dtype=torch.uint8, device="cuda")
    for _ in range(calls):
        st, n, s = pgz.pgz_decompress(ctx, d_in.data_ptr(), len(gz), d_out.data_ptr(), d_out.numel(), True)
        if st != 0 or n != len(raw):
            raise RuntimeError(f"pgz_decompress failed: {pgz.pgz_strerror(st)}")
    torch.cuda.synchronize()
    if d_out[:len(raw)].cpu().numpy().tobytes() != raw:
        raise RuntimeError("output mismatch")
    pgz.pgz_destroy(ctx)
    return {"case": f"{mib} MiB FASTQ gzip -{level}", "in_bytes": len(gz), "out_bytes": len(raw),
            **{k: (round(v, 3) if isinstance(v, float) else v) for k, v in s.items()}}


def run_profile_members(n_members: int, calls: int, chunk_bytes: int, wpb: int, xp: int = 0):
    """--profile-case members:N:CALLS -- the first N members of the 512-member manifest decoded together by
    pgz_decompress_batch, CALLS times (a prefix small enough for an ncu capture); outputs checked."""
    import numpy as np
    import torch
    from paper_1905_07224_gb300 import build, pgz, synth
    build.build()
    files = synth.make_files(synth.batch_manifest(512, 3)[:n_members])
    stream = torch.cuda.current_stream()
    ctx = pgz.pgz_create(pgz.pgz_config_init(device=0, cuda_stream=stream.cuda_stream, n_chunks=0,
                                             chunk_bytes=chunk_bytes, warps_per_block=wpb, exec_pipelined=xp))
    d_in = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).cuda() for _, g in files]
    d_out = [torch.empty(len(r) + 4096, dtype=torch.uint8, device="cuda") for r, _ in files]
    jobs = [(d_in[k].data_ptr(), len(g), d_out[k].data_ptr(), d_out[k].numel()) for k, (_, g) in enumerate(files)]
    s = None
    for _ in range(calls):
        r, res, s = pgz.pgz_decompress_batch(ctx, jobs, stats=True)
        if r != 0:
            raise RuntimeError(f"pgz_decompress_batch failed: {pgz.pgz_strerror(r)}")
    torch.cuda.synchronize()
    for k, (raw, _) in enumerate(files):
        if d_out[k][:len(raw)].cpu().numpy().tobytes() != raw:
            raise RuntimeError("output mismatch")
    pgz.pgz_destroy(ctx)
    return {"case": f"the first {n_members} members of the 512-member manifest (batched)", "chunk_bytes": chunk_bytes,
            "warps_per_block": wpb, "exec_pipelined": xp,
            **{k: (round(v, 3) if isinstance(v, float) else v) for k, v in s.items()}}


def run_profile_batch(calls: int, chunk_bytes: int, wpb: int, xp: int = 0):
    """--profile-case batch:CALLS -- the benchmark's two files decoded together by pgz_decompress_batch (the
    batched form without the graph), CALLS times; outputs checked."""
    import numpy as np
    import torch
    from paper_1905_07224_gb300 import build, pgz
    build.build()
    files, desc = make_workload("fastq256")
    stream = torch.cuda.current_stream()
    ctx = pgz.pgz_create(pgz.pgz_config_init(device=0, cuda_stream=stream.cuda_stream, n_chunks=0,
                                             chunk_bytes=chunk_bytes, warps_per_block=wpb, exec_pipelined=xp))
    d_in = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).cuda() for _, _, g in files]
    d_out = [torch.empty(len(r) + 4096, dtype=torch.uint8, device="cuda") for _, r, _ in files]
    jobs = [(d_in[k].data_ptr(), len(g), d_out[k].data_ptr(), d_out[k].numel()) for k, (_, _, g) in enumerate(files)]
    for _ in range(calls):
        r, res, s = pgz.pgz_decompress_batch(ctx, jobs, stats=True)
        if r != 0:
            raise RuntimeError(f"pgz_decompress_batch failed: {pgz.pgz_strerror(r)}")
    torch.cuda.synchronize()
    for k, (_, raw, _) in enumerate(files):
        if d_out[k][:len(raw)].cpu().numpy().tobytes() != raw:
            raise RuntimeError("output mismatch")
    pgz.pgz_destroy(ctx)
    return {"case": desc + " (batched)", "chunk_bytes": chunk_bytes, "warps_per_block": wpb, "exec_pipelined": xp,
            **{k: (round(v, 3) if isinstance(v, float) else v) for k, v in s.items()}}


def run_profile_sweep(spec: str):
    """--profile-case batchsweep:CHUNK/WPB/PIPE,... -- the benchmark's two files decoded together by one
    pgz_decompress_batch call per configuration (part size, warps per block, pipelined execution), in the order
    given, on one context each; outputs checked.  An ncu capture of k_sync / k_inflate then gives each
    configuration's pass-1 traffic in launch order."""
    import numpy as np
    import torch
    from paper_1905_07224_gb300 import build, pgz
    build.build()
    files, desc = make_workload("fastq256")
    stream = torch.cuda.current_stream()
    d_in = [torch.from_numpy(np.frombuffer(g, dtype=np.uint8).copy()).cuda() for _, _, g in files]
    d_out = [torch.empty(len(r) + 4096, dtype=torch.uint8, device="cuda") for _, r, _ in files]
    jobs = [(d_in[k].data_ptr(), len(g), d_out[k].data_ptr(), d_out[k].numel()) for k, (_, _, g) in enumerate(files)]
    refs = [torch.from_numpy(np.frombuffer(r, dtype=np.uint8).copy()).cuda() for _, r, _ in files]
    rows = []
    for item in spec.split(","):
        cb, w, x = (int(v) for v in item.split("/"))
        ctx = pgz.pgz_create(pgz.pgz_config_init(device=0, cuda_stream=stream.cuda_stream, n_chunks=0,
                                                 chunk_bytes=cb, warps_per_block=w, exec_pipelined=x))
        r, res, s = pgz.pgz_decompress_batch(ctx, jobs, stats=True)
        torch.cuda.synchronize()
        if r != 0:
            raise RuntimeError(f"pgz_decompress_batch failed: {pgz.pgz_strerror(r)}")
        for k, (_, raw, _) in enumerate(files):
            if not torch.equal(d_out[k][:len(raw)], refs[k]):
                raise RuntimeError("output mismatch")
            d_out[k].zero_()
        pgz.pgz_destroy(ctx)
        rows.append({"chunk_bytes": cb, "warps_per_block": w, "exec_pipelined": x, "parts": s["chunks"],
                     "ms_sync": round(s["ms_sync"], 3), "ms_inflate": round(s["ms_inflate"], 3)})
    return {"case": desc + " (batched, one call per configuration)", "out_bytes": sum(len(r) for _, r, _ in files),
            "configs": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pgz", choices=["pgz", "reference"])
    ap.add_argument("--workload", default="batch512",
                    choices=["batch512", "fastq256", "fastq1m", "fastq4g", "served", "stream"],
                    help="batch512: the benchmark (512 members, batched vs plain, with the fastq256 files and the "
                         "served loop as extra keys); fastq256: the two 256 MiB FASTQ files alone; fastq4g: "
                         "autotuner sweep on 4 GiB; served: the request loop at the full request count; stream: "
                         "the 4 GiB member streamed from host memory in 256 MiB segments")
    ap.add_argument("--chunk-bytes", type=int, default=0, help="fixed part size (default: autotuned)")
    ap.add_argument("--warps-per-block", type=int, default=4, choices=[2, 4, 8],
                    help="pass-1 CTA shape with a fixed --chunk-bytes or --profile-case")
    ap.add_argument("--exec-pipelined", type=int, default=0, choices=[0, 1],
                    help="pass-1 execution form with a fixed --chunk-bytes (default: autotuned)")
    ap.add_argument("--served-requests", type=int, default=SERVED_REQUESTS,
                    help="requests per offered load of the served extra (0: leave it out)")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the 512-member legs (no fastq256 files, served loop or CPU baseline)")
    ap.add_argument("--profile-case", default=None, metavar="MIB:LEVEL:CALLS|batch:CALLS|batchsweep:C/W/P,...",
                    help="run one checked case for an ncu capture and print its stage times: one FASTQ file, or "
                         "the benchmark's two files as one batch")
    args = ap.parse_args()
    if args.profile_case:
        print(json.dumps(run_profile_case(args.profile_case, args.chunk_bytes or CHUNK_BYTES, args.warps_per_block,
                                          args.exec_pipelined)), flush=True)
        return
    args.warmup = max(3, args.warmup)
    if args.workload in ("fastq4g", "served", "stream") and args.impl == "pgz":
        run = {"fastq4g": run_tune4g, "served": run_served, "stream": run_stream}[args.workload]
        print(json.dumps(run(args)), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            ref = run_reference_batch512(args) if args.workload == "batch512" else run_reference(args)
            print(json.dumps(ref), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
    line = run_headline(args, rank, world) if args.workload == "batch512" else run_pgz(args, rank, world)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
