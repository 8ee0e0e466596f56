#!/usr/bin/env python
"""Throughput of 3DES-EDE ECB on GB300 (one JSON line on rank 0).

Workload ("plain single-buffer throughput"): one 4 GiB device-resident buffer
(2^29 64-bit blocks of seeded SplitMix64 bytes) and one parity-adjusted 3-key
triple.  One step = 3DES encryption of the whole buffer in place followed by
3DES decryption in place (paper Sec. II.A: E-D-E, and its reverse), so every
step processes 8 GiB and leaves the buffer as it found it.  The buffer is 32x
the 129 MB L2, so no flush is needed between steps.

Fields beyond the base contract:
  roofline      the dominant kernel against its binding pipe (the integer ALU
                pipe for the bitsliced kernel), with the peak measured in the
                same run by des3_pipe_probe before the timed region
  pipe_probe    that probe: LOP3, IMAD, mixed and shared-load lanes per SM
                per clock
  cpu_baseline  the CPU oracle (OpenMP over all host cores) on a sample
  e2e           the same steps through des3_ecb_host on pinned host memory,
                every byte of the round trip checked, beside the same copies
                with no kernel between them
  size_sweep    64 KiB .. 4 GiB x {3-key, 2-key} x {encrypt, decrypt} x
                {tuned default, bitsliced, SP-table}
  batched       4096 buffers with their own keys in one graph-replayed launch
  serving       the request server under Poisson load from 0.1x to 1.25x
  clocks        nvidia-smi SM clock and throttle reasons during the timed region

--impl reference times the CPU oracle itself on the same metric.
--gpus N under torchrun runs N independent replicas (one buffer per GPU, no
communication: ECB blocks are independent) and reports their sum.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GIB = 1 << 30
WORKLOAD_BYTES = 4 * GIB
CONFIG_ID = 2  # data seed 0xDE5C0DE0 + 2, key seed 0x3DE5 + 2
METRIC = "3DES-ECB GB/s on 1 GB300, % of INT/HBM roofline; batched p50/p99 latency"
# Sizes of the size and keying sweep (64 KiB .. 4 GiB); the larger ones only
# when the buffer holds them.
SWEEP_SIZES = (64 << 10, 1 << 20, 16 << 20, 256 << 20, 4 << 30)
# Headline serving point: the highest offered load whose p99 latency stays
# within this bound.
SERVE_P99_BOUND_MS = 5.0
# DRAM bytes (read + written) per block of the dominant kernel, from an ncu
# --set full capture of one 256 MiB launch (268.49 MB read + 206.99 MB
# written for 2^25 blocks).  Only valid for the kernel sources it was taken
# with, identified by a digest of the files below; otherwise null.
KERNEL_SOURCES = ["common.cuh", "bs_generated.cuh", "kernels.cu", "tile_io.cuh", "internal.h"]
PROFILED_TRAFFIC = {"kernel": "bitslice", "sources_sha256": "b385f69969198d99",
                    "bytes_per_block": (268.485120e6 + 206.987264e6) / 2 ** 25}


def kernel_sources_digest():
    """First 16 hex digits of SHA-256 over the bitsliced kernel's sources."""
    import hashlib
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1305_4376_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "bitslice", "sptable"])
    ap.add_argument("--bytes", type=int, default=WORKLOAD_BYTES, help="buffer size (default 4 GiB)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-modes", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=40000)
    ap.add_argument("--no-probe", action="store_true", help="skip the in-run pipe probe (peak from nominal figures)")
    ap.add_argument("--batched-max-bytes", type=int, default=16 << 20,
                    help="largest buffer of the batched workload (smaller only for profiling)")
    ap.add_argument("--batched-kernel", default="auto", choices=["auto", "bitslice", "sptable"],
                    help="batched kernel of the batched line (auto: the library's choice; others for profiling)")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers

class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_oracle_rate(target_s: float = 12.0):
    """The CPU oracle (as it stands, OpenMP over all cores) on a bounded prefix
    of the workload: encrypt then decrypt, like one step.  Returns (GB/s,
    cores, sample description)."""
    import oracle
    from paper_1305_4376_gb300 import inputs

    key = inputs.key_triple(inputs.key_seed(CONFIG_ID))
    probe = 1 << 20
    data = inputs.data_bytes(inputs.data_seed(CONFIG_ID), probe)
    t = time.perf_counter()
    ct = oracle.tdes_ecb(key, data)
    oracle.tdes_ecb(key, ct, decrypt=True)
    dt = time.perf_counter() - t
    nbytes = int(min(512 << 20, max(probe, (target_s / max(dt, 1e-6)) * probe))) // (1 << 20) * (1 << 20)
    data = inputs.data_bytes(inputs.data_seed(CONFIG_ID), nbytes)
    t = time.perf_counter()
    ct = oracle.tdes_ecb(key, data)
    back = oracle.tdes_ecb(key, ct, decrypt=True)
    dt = time.perf_counter() - t
    assert (back == data).all()
    rate = 2 * nbytes / dt / 1e9
    return rate, oracle.max_threads(), "first %d MiB of the 4 GiB workload, encrypt + decrypt (%.1f s)" % (
        nbytes >> 20, dt)


def arena(torch, inputs, sizes, seed, dev, align=256):
    """Device arena with every buffer at an `align`-aligned offset, seeded bytes."""
    offs, pos = inputs.arena_offsets(sizes, align)
    words = inputs.splitmix64_torch(seed, 0, pos // 8 + 32, dev)
    return words.view(torch.uint8), offs


def run_batched(torch, des3, inputs, dev, stream, steps, plain_gbs, max_bytes=16 << 20, kernel="auto"):
    """Batched workload: 4096 buffers, log-uniform 512 B .. max_bytes (16 MiB
    by default), a 3-key triple each, mixed directions, one graph-captured
    persistent launch of the library's batched kernel (or `kernel`)."""
    sizes, dec = inputs.batch_recipe(inputs.data_seed(4), hi=max_bytes)
    keys = inputs.key_triples(inputs.key_seed(4), len(sizes))
    karr = des3.make_keys([des3.des3_key_schedule(k) for k in keys])
    src, offs = arena(torch, inputs, sizes, inputs.data_seed(4), dev)
    out = torch.empty_like(src)
    jobs = des3.make_jobs([(src[o:o + int(n)], out[o:o + int(n)], int(n), i, bool(dec[i]))
                           for i, (n, o) in enumerate(zip(sizes, offs))])
    plan = des3.BatchPlan(karr, jobs, kernel=kernel)
    total, tiles = plan.info()
    kid, threads, ctas = plan.kernel()
    for _ in range(3):
        plan.launch(stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        plan.launch(stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    plan.close()
    gbs = total / (ms * 1e-3) / 1e9
    return {"value": gbs, "unit": "GB/s", "jobs": len(sizes), "total_bytes": int(total), "tiles": int(tiles),
            "ms_per_launch": ms, "steps": steps, "vs_plain": gbs / plain_gbs,
            "kernel": {des3.DES3_KERNEL_BITSLICE: "bitslice", des3.DES3_KERNEL_SPTABLE: "sptable"}[kid],
            "threads": threads, "ctas_per_sm": ctas,
            "workload": "4096 buffers, sizes log-uniform 512 B..%d KiB, own 3-key triple each, "
                        "mixed encrypt/decrypt, one persistent launch replayed from a CUDA graph" % (max_bytes >> 10)}


def run_serving(torch, des3, inputs, dev, plain_gbs, nreq):
    """Serving workload: Poisson arrivals of encrypt/decrypt requests, sizes
    log-normal (median 256 KiB, sigma 1.5, clamped to 4 KiB..64 MiB), keys
    from 10000 cached triples, 16 GiB admission budget.  The offered rate is
    swept from 0.1x to 1.25x of the plain kernel's request rate (1.0x offers
    the plain kernel's own rate, at or above what the server can sustain, so
    p99 there grows with the run's length).  Headline:
    the highest offered load whose p99 stays within SERVE_P99_BOUND_MS; the
    load at which the server stops keeping up (achieved below 95 % of
    offered, so the queue and p99 grow without bound) is reported as the
    point where p99 diverges."""
    import numpy as np
    sizes, kidx, dec, gaps = inputs.serve_recipe(inputs.data_seed(5), nreq)
    nkeys = 10000
    keys = inputs.key_triples(inputs.key_seed(5), nkeys)
    srv = des3.Server(budget_bytes=16 << 30, max_inflight=1 << 16, max_queue=1 << 20, nstreams=4,
                      max_batch_requests=8192, max_batch_bytes=2 << 30, key_capacity=nkeys)
    first = srv.add_keys([des3.des3_key_schedule(k) for k in keys])
    in_bytes = 4 << 30
    src = inputs.splitmix64_torch(inputs.data_seed(5), 0, in_bytes // 8, dev).view(torch.uint8)
    ring = 16 << 30
    out = torch.empty(ring + (64 << 20), dtype=torch.uint8, device=dev)
    r = inputs.splitmix64(inputs.data_seed(5) + 99, 0, nreq)
    reqs = (des3.des3_request_t * nreq)()
    pos = 0
    for i in range(nreq):
        n = int(sizes[i])
        o = int(r[i] % np.uint64((in_bytes - n) // 256)) * 256
        if pos + n > ring:
            pos = 0
        reqs[i] = des3.Server.request(src.data_ptr() + o, out.data_ptr() + pos, n, first + int(kidx[i]),
                                      bool(dec[i]), i)
        pos += (n + 255) // 256 * 256
    total = int(sizes.sum())
    mean = total / nreq
    sat = plain_gbs * 1e9 / mean
    sweep = []
    for f in (0.1, 0.25, 0.5, 0.8, 0.9, 0.95, 1.0, 1.1, 1.25):
        arrival = np.cumsum(gaps) / (f * sat)
        arrival -= arrival[0]
        rc, lat = srv.replay(reqs, arrival, 600000)
        if rc != 0:
            raise RuntimeError("serving replay failed: %d" % rc)
        span = float((arrival + lat).max())
        gbs = total / span / 1e9
        sweep.append({"offered_x_saturation": f, "offered_rps": f * sat, "offered_GB/s": f * plain_gbs,
                      "GB/s": gbs, "kept_up": gbs >= 0.95 * f * plain_gbs,
                      "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                      "max_ms": 1e3 * float(lat.max())})
    st = srv.stats()
    srv.close()
    head, div, peak = serving_points(sweep)
    return {"value": head["GB/s"], "unit": "GB/s", "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
            "at_offered_x_saturation": head["offered_x_saturation"], "vs_plain": head["GB/s"] / plain_gbs,
            "headline_rule": "highest offered load with p99 <= %.1f ms" % SERVE_P99_BOUND_MS,
            "peak_GB/s": peak["GB/s"], "peak_at_offered_x_saturation": peak["offered_x_saturation"],
            "peak_vs_plain": peak["GB/s"] / plain_gbs,
            "lambda_at_divergence": None if div is None else {
                "offered_x_saturation": div["offered_x_saturation"], "offered_rps": div["offered_rps"],
                "rule": "lowest offered load whose achieved GB/s is below 95 % of offered"},
            "saturation_rps": sat, "requests_per_point": nreq, "mean_request_bytes": mean,
            "launches": st["launches"], "table_kernel_launches": st["table_launches"], "sweep": sweep,
            "workload": "Poisson arrivals, sizes log-normal median 256 KiB sigma 1.5 in [4 KiB, 64 MiB], "
                        "10000 cached key triples, 16 GiB admission budget, 4 streams, continuous batching"}


def serving_points(sweep, bound_ms=SERVE_P99_BOUND_MS):
    """From a load sweep (dicts with offered_x_saturation, GB/s, p99_ms,
    kept_up): the headline point, the highest offered load whose p99 is within
    bound_ms (the lowest-p99 point if none is); the point where p99 diverges,
    the lowest offered load that did not keep up (None if all did); and the
    highest-throughput point."""
    bounded = [x for x in sweep if x["p99_ms"] <= bound_ms]
    head = max(bounded, key=lambda x: x["offered_x_saturation"]) if bounded else min(sweep, key=lambda x: x["p99_ms"])
    diverged = [x for x in sweep if not x["kept_up"]]
    div = min(diverged, key=lambda x: x["offered_x_saturation"]) if diverged else None
    peak = max(sweep, key=lambda x: x["GB/s"])
    return head, div, peak


def pipe_peaks(torch, des3, dev, stream):
    """The in-run pipe probe (des3_pipe_probe): lane-instructions per SM per
    clock of the LOP3 (integer ALU), IMAD (FMA), mixed and shared-load pipes,
    at the SM clock the probe itself measured (its cycle counter against the
    global nanosecond timer).  Best of three timed launches after one
    warm-up, CUDA events on the launching stream."""
    sink = torch.zeros(4, dtype=torch.int64, device=dev)
    out = {}
    for name, iters in (("lop3", 3000), ("imad", 3000), ("lop3+imad", 3000), ("lds", 1500)):
        best = None
        for rep in range(4):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ins, sms = des3.des3_pipe_probe(name, iters, sink, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            cyc, ns = int(sink[1].item()), int(sink[2].item())
            mhz = cyc / ns * 1e3 if ns else None
            rate = ins / (ms * 1e-3)
            if rep and mhz and (best is None or rate > best["rate_per_s"]):
                best = {"lanes_per_sm_clk": rate / sms / (mhz * 1e6), "rate_per_s": rate, "probe_sm_mhz": mhz,
                        "ms": ms, "sms": sms}
        out[name] = best
    return out


def pipeline_copies_gbs(torch, h_in, h_out, work, nbytes, stream, chunk=64 << 20, passes=2):
    """GB/s each way of the host pipeline's copies with no kernel: the same
    pinned buffers and three 64 MiB device slots, every copy in on one stream
    and every copy out on another, so that exactly one copy runs in each
    direction at a time.  A chunk's copy out waits for its copy in, and a copy
    into a slot waits for that slot's previous copy out, as in des3_ecb_host:
    the schedule the pipeline reaches when its kernel is faster than the
    copies.  On a quiet host this and three streams each copying a chunk in
    and straight back out both gave 164-166 GB/s; the host link is shared,
    and under load either reading falls (113-134 GB/s were seen)."""
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    slots = [work[i * chunk:(i + 1) * chunk] for i in range(3)]
    copied_in = [torch.cuda.Event() for _ in range(3)]
    copied_out = [torch.cuda.Event() for _ in range(3)]
    used = [False] * 3
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    up.wait_stream(stream)
    down.wait_stream(stream)
    i = 0
    for _ in range(passes):
        for off in range(0, nbytes, chunk):
            n = min(chunk, nbytes - off)
            k = i % 3
            with torch.cuda.stream(up):
                if used[k]:
                    up.wait_event(copied_out[k])
                slots[k][:n].copy_(h_in[off:off + n], non_blocking=True)
                copied_in[k].record(up)
            with torch.cuda.stream(down):
                down.wait_event(copied_in[k])
                h_out[off:off + n].copy_(slots[k][:n], non_blocking=True)
                copied_out[k].record(down)
            used[k] = True
            i += 1
    stream.wait_stream(up)
    stream.wait_stream(down)
    b.record(stream)
    torch.cuda.synchronize()
    return passes * nbytes / (a.elapsed_time(b) * 1e-3) / 1e9


def run_sweep(torch, des3, inputs, autotune, lib, buf, nbytes, stream, probe, sm_mhz):
    """The size and keying sweep: single buffers of SWEEP_SIZES (prefixes of
    the plain workload's buffer, in place), 3-key and 2-key triples from the
    sweep's key seed, encryption and decryption, the tuned default and each
    kernel forced.  Each cell is CUDA-event time over repeated calls on one
    stream; up to 16 MiB also as 20 calls captured in a CUDA graph (device
    time without the host's per-call cost).  A cell's encryptions are
    followed by as many decryptions, so the buffer ends as it began.  Each
    cell also gives the fraction of its binding pipe's measured peak: the
    integer ALU pipe for the bitsliced kernel, the shared-memory pipe for the
    table kernel."""
    import ctypes
    s = stream.cuda_stream
    ptr = buf.data_ptr()
    info = {k: des3.des3_kernel_info(k) for k in ("bitslice", "sptable")}
    peak = {}
    for k, pname, field in (("bitslice", "lop3", "alu_ops_per_block"), ("sptable", "lds", "smem_loads_per_block")):
        if probe and probe.get(pname):
            peak[k] = (field, probe[pname]["lanes_per_sm_clk"] * probe[pname]["sms"] * sm_mhz * 1e6, pname)
    cells = []
    for size in SWEEP_SIZES:
        if size > nbytes:
            continue
        for keying in ("3key", "2key"):
            ks = des3.des3_key_schedule(inputs.key_triple(inputs.key_seed(3), keying))
            ksp = ctypes.byref(ks)
            for kname in ("auto", "bitslice", "sptable"):
                kid = des3.KERNELS[kname]
                used = kname
                if kname == "auto":
                    e = autotune.get_entry(des3.DES3_TUNE_SINGLE, size.bit_length() - 1)
                    used = "sptable" if e[1] == des3.DES3_KERNEL_SPTABLE else "bitslice"
                est = max(12e-6, size / (400e9 if used == "bitslice" else 150e9))
                reps = int(min(2000, max(3, 0.03 / est)))
                for d in (0, 1):
                    if lib.des3_ecb_crypt_ex(ksp, ptr, ptr, size, d, kid, s):
                        raise RuntimeError("size sweep warm-up failed")
                torch.cuda.synchronize()
                for d in (0, 1):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    for _ in range(reps):
                        if lib.des3_ecb_crypt_ex(ksp, ptr, ptr, size, d, kid, s):
                            raise RuntimeError("size sweep launch failed")
                    b.record(stream)
                    torch.cuda.synchronize()
                    t = a.elapsed_time(b) / reps * 1e-3
                    cell = {"bytes": size, "keying": keying, "direction": "decrypt" if d else "encrypt",
                            "kernel": kname, "kernel_used": used, "GB/s": size / t / 1e9, "us_per_call": t * 1e6,
                            "calls": reps}
                    if used in peak:
                        field, pk, pname = peak[used]
                        cell["pipe"] = pname
                        cell["pipe_frac"] = info[used][field] * (size // 8) / t / pk
                    if size <= (16 << 20):
                        ncap = 20
                        g = torch.cuda.CUDAGraph()
                        with torch.cuda.graph(g):
                            cs = torch.cuda.current_stream().cuda_stream
                            for _ in range(ncap):
                                if lib.des3_ecb_crypt_ex(ksp, ptr, ptr, size, d, kid, cs):
                                    raise RuntimeError("size sweep capture failed")
                        g.replay()
                        torch.cuda.synchronize()
                        a.record(stream)
                        for _ in range(5):
                            g.replay()
                        b.record(stream)
                        torch.cuda.synchronize()
                        tg = a.elapsed_time(b) / (5 * ncap) * 1e-3
                        cell["graph_GB/s"] = size / tg / 1e9
                        cell["graph_us_per_call"] = tg * 1e6
                        cell["graph_calls"] = 6 * ncap
                        del g
                    cells.append(cell)
    # graph replays: each direction ran 6 x 20 times, so the buffer is back too
    best = {}
    for c in cells:
        if c["kernel"] == "auto":
            continue
        key = (c["bytes"], c["keying"], c["direction"])
        if key not in best or c["GB/s"] > best[key]["GB/s"]:
            best[key] = c
    fastest = [{"bytes": k[0], "keying": k[1], "direction": k[2], "fastest": v["kernel"], "GB/s": v["GB/s"]}
               for k, v in sorted(best.items())]
    return {"cells": cells, "fastest_kernel": fastest,
            "data": "prefixes of the plain workload's buffer, in place; keys from the sweep's seed 0x3DE8",
            "note": "pipe_frac: kernel_info's per-block instructions on the binding pipe x blocks / time, "
                    "over the in-run probe's peak at the timed region's median SM clock"}


def emit(obj):
    print(json.dumps(obj), flush=True)


# ---------------------------------------------------------- reference arm

def workload_name(nbytes):
    """The plain workload's description, the same in both arms."""
    return ("plain single-buffer: 3-key 3DES-EDE ECB encrypt + decrypt in place, "
            "%d MiB device-resident buffer (%d blocks), one key triple" % (nbytes >> 20, nbytes // 8))


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1305_4376_gb300 import inputs

    key = inputs.key_triple(inputs.key_seed(CONFIG_ID))
    sample = 4 << 20
    data = inputs.data_bytes(inputs.data_seed(CONFIG_ID), sample)
    warmup = max(3, args.warmup)
    for _ in range(warmup):
        oracle.tdes_ecb(key, oracle.tdes_ecb(key, data), decrypt=True)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.tdes_ecb(key, oracle.tdes_ecb(key, data), decrypt=True)
    dt = time.perf_counter() - t
    value = 2 * sample * args.steps / dt / 1e9
    cores = oracle.max_threads()
    desc = "4 MiB prefix of the 4 GiB workload per step, encrypt + decrypt"
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
          "n_gpus": world, "steps": args.steps, "warmup": warmup,
          "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u32", "data": "synthetic (SplitMix64 bytes, seeded)",
          "config": {"workload": workload_name(args.bytes), "sample_per_step_bytes": sample,
                     "sample": "the oracle runs on the workload's first %d MiB each step" % (sample >> 20)},
          "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
          "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import ctypes

    import torch

    from paper_1305_4376_gb300 import autotune, build, des3, inputs, replicas

    build.build()
    torch.cuda.set_device(local_rank)
    tuned = autotune.load_tuning()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream

    key = inputs.key_triple(inputs.key_seed(CONFIG_ID))
    ks = des3.des3_key_schedule(key)
    nbytes = args.bytes
    nblocks = nbytes // 8
    words = inputs.splitmix64_torch(inputs.data_seed(CONFIG_ID), 0, nblocks, dev)
    buf = words.view(torch.uint8)
    check_idx = torch.arange(0, nblocks, max(1, nblocks // 4096), device=dev)
    before = words[check_idx].clone()

    lib = des3.lib()
    ksp = ctypes.byref(ks)
    kernel = des3.KERNELS[args.kernel]
    ptr = buf.data_ptr()

    # the roofline denominators, measured on this device in this run
    probe = None if args.no_probe else pipe_peaks(torch, des3, dev, stream)

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        rc = lib.des3_ecb_crypt_ex(ksp, ptr, ptr, nbytes, 0, kernel, s)
        if evs is not None:
            evs[1].record(stream)
        rc |= lib.des3_ecb_crypt_ex(ksp, ptr, ptr, nbytes, 1, kernel, s)
        if evs is not None:
            evs[2].record(stream)
        if rc:
            raise RuntimeError("launch failed: %d" % rc)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local_rank) if rank == 0 else None
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    replicas.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    replicas.barrier()
    clocks = sampler.stop() if sampler else None
    ms = t0.elapsed_time(t1)
    launch_ms = []
    for e in evs:
        launch_ms.append(e[0].elapsed_time(e[1]))
        launch_ms.append(e[1].elapsed_time(e[2]))
    # the buffer must be back to its plaintext after every step
    assert torch.equal(words[check_idx], before), "encrypt + decrypt did not restore the buffer"

    ms = replicas.max_over_ranks(ms, device=dev)
    sm_mhz = (clocks or {}).get("sm_mhz") or ((probe or {}).get("lop3") or {}).get("probe_sm_mhz")

    # ---- end to end through the host-memory entry point ----
    e2e = None
    if not args.no_e2e:
        work_bytes = 3 * (64 << 20)
        work = torch.empty(work_bytes, dtype=torch.uint8, device=dev)
        h_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        h_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        h_in.copy_(buf)
        wp = work.data_ptr()

        def host_call(src, dst, d):
            rc = lib.des3_ecb_host(ksp, src.data_ptr(), dst.data_ptr(), nbytes, d, wp, work_bytes, s)
            if rc:
                raise RuntimeError("des3_ecb_host failed: %d" % rc)

        def e2e_step():
            host_call(h_in, h_out, 0)
            host_call(h_out, h_out, 1)

        e2e_step()
        torch.cuda.synchronize()
        link_before = pipeline_copies_gbs(torch, h_in, h_out, work, nbytes, stream)
        # leave h_out encrypted, so that only timed steps that really run
        # turn it back into h_in; every check runs after the timed region
        host_call(h_in, h_out, 0)
        torch.cuda.synchronize()
        replicas.barrier()
        # events between the steps too (des3_ecb_host joins the caller's
        # stream at both ends), to show how steady the host link was
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps + 1)]
        marks[0].record(stream)
        for i in range(args.e2e_steps):
            e2e_step()
            marks[i + 1].record(stream)
        torch.cuda.synchronize()
        e_ms = marks[0].elapsed_time(marks[-1])
        step_gbs = [2 * nbytes / (marks[i].elapsed_time(marks[i + 1]) * 1e-3) / 1e9 for i in range(args.e2e_steps)]
        e_ms = replicas.max_over_ranks(e_ms, device=dev)
        assert torch.equal(h_out, h_in), "host-memory round trip did not restore every byte of the input"
        link_after = pipeline_copies_gbs(torch, h_in, h_out, work, nbytes, stream)
        # one host-memory encryption, compared in full with the device
        # kernel's encryption of the same buffer
        host_call(h_in, h_out, 0)
        torch.cuda.synchronize()
        d_ct = buf.clone()
        lib.des3_ecb_crypt_ex(ksp, d_ct.data_ptr(), d_ct.data_ptr(), nbytes, 0, 0, s)
        torch.cuda.synchronize()
        assert torch.equal(h_out, d_ct.cpu()), "host-memory encryption differs from the device kernel's"
        del d_ct
        value_e2e = 2 * nbytes * args.e2e_steps * world / (e_ms * 1e-3) / 1e9
        link = max(link_before, link_after)
        e2e = {"value": value_e2e, "unit": "GB/s",
               "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": 2 * nbytes,
               "api": "des3_ecb_host (pinned host buffers, 3 x 64 MiB device slots)", "steps": args.e2e_steps,
               "checked": "after the timed steps: every byte of the round trip compared with the input, and "
                          "one more encryption compared in full with the device kernel's",
               "step_gbs": step_gbs,
               "copies_alone_each_way_gbs": {"before": link_before, "after": link_after},
               "vs_copies_alone": value_e2e / (link * world),
               "note": "copies alone: the same pinned buffers, slots, streams and chunk size as des3_ecb_host "
                       "with no kernel between copy in and copy out, measured just before and just after the "
                       "timed steps; the shared host's load varies between runs"}
        del work, h_in, h_out

    # the two other parallel modes on the same buffer (one launch each, timed alone)
    modes = {}
    if not args.no_modes:
        iv = bytes(range(8))
        for name, fn in (("ctr", lib.des3_ctr_crypt), ("cbc_decrypt", lib.des3_cbc_decrypt)):
            out = torch.empty_like(buf) if name == "cbc_decrypt" else buf
            fn(ksp, iv, ptr, out.data_ptr(), nbytes, s)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            reps = 3
            for _ in range(reps):
                if fn(ksp, iv, ptr, out.data_ptr(), nbytes, s):
                    raise RuntimeError("%s failed" % name)
            b.record(stream)
            torch.cuda.synchronize()
            modes[name] = {"value": nbytes * reps / (a.elapsed_time(b) * 1e-3) / 1e9, "unit": "GB/s"}
            del out
        torch.cuda.empty_cache()
        # CTR ran an even number of times in place (4): the buffer is restored
        # single DES (16 rounds) on the same buffer: encrypt then decrypt in place
        ks1 = des3.des3_key_schedule_des(key[:8])
        ks1p = ctypes.byref(ks1)
        for d in (0, 1):
            lib.des3_ecb_crypt_ex(ks1p, ptr, ptr, nbytes, d, 0, s)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        reps = 4
        for i in range(reps):
            if lib.des3_ecb_crypt_ex(ks1p, ptr, ptr, nbytes, i & 1, 0, s):
                raise RuntimeError("single DES failed")
        b.record(stream)
        torch.cuda.synchronize()
        t_ms = a.elapsed_time(b) / reps
        modes["single_des_ecb"] = {"value": nbytes / (t_ms * 1e-3) / 1e9, "unit": "GB/s",
                                   "hbm_gbs": 2 * nbytes / (t_ms * 1e-3) / 1e9}
        assert torch.equal(words[check_idx], before), "single DES round trip did not restore the buffer"

    sweep = None
    if not args.no_sweep:
        sweep = run_sweep(torch, des3, inputs, autotune, lib, buf, nbytes, stream, probe, sm_mhz)
        assert torch.equal(words[check_idx], before), "size sweep did not restore the buffer"
    batched = serving = None
    value = replicas.aggregate_gbs(2 * nbytes * args.steps, ms, world)
    plain_gbs = value / world
    if not (args.no_batched and args.no_serving):
        del words, buf, before
        torch.cuda.empty_cache()
    if not args.no_batched:
        batched = run_batched(torch, des3, inputs, dev, stream, max(3, args.steps // 3), plain_gbs,
                              args.batched_max_bytes, args.batched_kernel)
        torch.cuda.empty_cache()
    if not args.no_serving:
        serving = run_serving(torch, des3, inputs, dev, plain_gbs, args.serve_requests)
        torch.cuda.empty_cache()

    if rank != 0:
        return

    if args.kernel != "auto":
        kname = args.kernel
    else:
        c = max(0, nbytes.bit_length() - 1)
        kname = "sptable" if autotune.get_entry(des3.DES3_TUNE_SINGLE, min(c, 39))[1] == des3.DES3_KERNEL_SPTABLE \
            else "bitslice"
    info = des3.des3_kernel_info(kname)
    avg_launch_ms = statistics.mean(launch_ms)
    traffic = None
    src_digest = kernel_sources_digest()
    pt = PROFILED_TRAFFIC
    if kname == pt["kernel"] and src_digest == pt["sources_sha256"]:
        traffic = pt["bytes_per_block"] * nblocks
    # the binding pipe: the integer ALU pipe for the bitsliced kernel, the
    # shared-memory pipe for the table kernel
    pipe, field = ("lop3", "alu_ops_per_block") if kname == "bitslice" else ("lds", "smem_loads_per_block")
    achieved = info[field] * nblocks / (avg_launch_ms * 1e-3) / 1e12
    if probe and probe.get(pipe) and sm_mhz:
        lanes = probe[pipe]["lanes_per_sm_clk"]
        sms = probe[pipe]["sms"]
        peak = lanes * sms * sm_mhz * 1e6 / 1e12
        peak_source = ("measured in this run: %s probe %.2f lanes/SM/clk at %.0f MHz (des3_pipe_probe) x %d SMs "
                       "x %.0f MHz median SM clock of the timed region" % (
                           pipe, lanes, probe[pipe]["probe_sm_mhz"], sms, sm_mhz))
    else:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        lanes = 64 if pipe == "lop3" else 32
        peak = lanes * sms * 2070e6 / 1e12
        peak_source = "nominal: %d lanes/SM/clk x %d SMs x 2070 MHz (probe skipped)" % (lanes, sms)
    launch_gbs = sorted(nbytes / (t * 1e-3) / 1e9 for t in launch_ms)
    hbm_peak = measured_hbm_gbs()
    cpu = None
    if world == 1 and not args.no_cpu:
        rate, cores, desc = cpu_oracle_rate()
        cpu = {"value": rate, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc}
    emit({
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (SplitMix64 bytes generated on the device, seeded)",
        "config": {"workload": workload_name(nbytes),
                   "kernel": kname, "l2": ("inputs %d MiB > 129 MB L2; no flush" % (nbytes >> 20)) if nbytes > (129 << 20)
                   else "inputs fit in L2; no flush (not a valid bench size)",
                   "tuning": "autotuned table for this GPU" if tuned else "built-in defaults",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu" if pipe == "lop3" else "lsu", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": "ncu capture of a 256 MiB launch, scaled by blocks" if traffic
                     else "no ncu capture of these kernel sources", "kernel_sources_sha256": src_digest,
                     "kernel": kname, "ops_per_block": info[field],
                     "alu_ops_per_block": info["alu_ops_per_block"],
                     "fma_ops_per_block": info["fma_ops_per_block"],
                     "smem_loads_per_block": info["smem_loads_per_block"],
                     "sbox_gates": info["sbox_gates"], "avg_launch_ms": avg_launch_ms,
                     "peak_source": peak_source,
                     "hbm_gbs": 2 * nbytes / (avg_launch_ms * 1e-3) / 1e9,
                     "hbm_frac": (2 * nbytes / (avg_launch_ms * 1e-3) / 1e9 / hbm_peak) if hbm_peak else None},
        "pipe_probe": probe,
        "launch_gbs": {"median": statistics.median(launch_gbs), "p10": quantile(launch_gbs, 0.1),
                       "p90": quantile(launch_gbs, 0.9), "launches": len(launch_gbs),
                       "note": "per-launch GB/s from CUDA events around each encrypt and decrypt launch"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "modes": modes or None,
        "size_sweep": sweep,
        "batched": batched,
        "serving": serving,
        "clocks": clocks,
        "gpu_launches": 2 * args.steps,
    })


def quantile(sorted_vals, q):
    """Linear-interpolated quantile of an ascending list."""
    if not sorted_vals:
        return None
    x = q * (len(sorted_vals) - 1)
    i = int(x)
    j = min(i + 1, len(sorted_vals) - 1)
    return sorted_vals[i] + (sorted_vals[j] - sorted_vals[i]) * (x - i)


def measured_hbm_gbs():
    """The machine's measured copy bandwidth (GB/s) when the peaks file is present."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
