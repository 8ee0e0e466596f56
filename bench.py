#!/usr/bin/env python
"""Throughput of 3DES-EDE ECB on GB300 (one JSON line on rank 0).

Workload ("plain single-buffer throughput"): one 4 GiB device-resident buffer
(2^29 64-bit blocks of seeded SplitMix64 bytes) and one parity-adjusted 3-key
triple.  One step = 3DES encryption of the whole buffer in place followed by
3DES decryption in place (paper Sec. II.A: E-D-E, and its reverse), so every
step processes 8 GiB and leaves the buffer as it found it.  The buffer is 32x
the 129 MB L2, so no flush is needed between steps.

Fields beyond the base contract:
  roofline      the dominant kernel against the integer (LOP3) pipe peak
  cpu_baseline  the CPU oracle (OpenMP over all host cores) on a sample
  e2e           the same steps through des3_ecb_host on pinned host memory
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
# LOP3 (integer ALU pipe) instructions per SM per clock on GB300, measured
# by the throughput probe python -m paper_1305_4376_gb300.alu_peak (63.9 at 2067 MHz).
ALU_LANES_PER_SM_CLK = 64
SM_COUNT = 152
SM_MAX_MHZ = 2070
# DRAM bytes (read + written) per block of the dominant kernel, from an ncu
# --set full capture of one 256 MiB launch (268.48 MB read + 207.15 MB
# written for 2^25 blocks).  Only valid for the kernel sources it was taken
# with, identified by a digest of the files below; otherwise null.
KERNEL_SOURCES = ["common.cuh", "bs_generated.cuh", "kernels.cu", "tile_io.cuh", "internal.h"]
PROFILED_TRAFFIC = {"kernel": "bitslice", "sources_sha256": "460abf37b2760bdb",
                    "bytes_per_block": (268.481536e6 + 207.151872e6) / 2 ** 25}


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
    ap.add_argument("--batched-max-bytes", type=int, default=16 << 20,
                    help="largest buffer of the batched workload (smaller only for profiling)")
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
    offs, pos = [], 0
    for n in sizes:
        offs.append(pos)
        pos += (int(n) + align - 1) // align * align
    words = inputs.splitmix64_torch(seed, 0, pos // 8 + 32, dev)
    return words.view(torch.uint8), offs


def run_batched(torch, des3, inputs, dev, stream, steps, plain_gbs, max_bytes=16 << 20):
    """Batched workload: 4096 buffers, log-uniform 512 B .. max_bytes (16 MiB
    by default), a 3-key triple each, mixed directions, one graph-captured
    persistent launch."""
    sizes, dec = inputs.batch_recipe(inputs.data_seed(4), hi=max_bytes)
    keys = inputs.key_triples(inputs.key_seed(4), len(sizes))
    karr = des3.make_keys([des3.des3_key_schedule(k) for k in keys])
    src, offs = arena(torch, inputs, sizes, inputs.data_seed(4), dev)
    out = torch.empty_like(src)
    jobs = des3.make_jobs([(src[o:o + int(n)], out[o:o + int(n)], int(n), i, bool(dec[i]))
                           for i, (n, o) in enumerate(zip(sizes, offs))])
    plan = des3.BatchPlan(karr, jobs)
    total, tiles = plan.info()
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
            "workload": "4096 buffers, sizes log-uniform 512 B..%d KiB, own 3-key triple each, "
                        "mixed encrypt/decrypt, one persistent launch replayed from a CUDA graph" % (max_bytes >> 10)}


def run_serving(torch, des3, inputs, dev, plain_gbs, nreq):
    """Serving workload: Poisson arrivals of encrypt/decrypt requests, sizes
    log-normal (median 256 KiB, sigma 1.5, clamped to 4 KiB..64 MiB), keys
    from 10000 cached triples, 16 GiB admission budget; the offered rate is
    swept from 0.25x to 1.25x of the plain kernel's request rate."""
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
    for f in (0.25, 0.5, 0.8, 1.0, 1.25):
        arrival = np.cumsum(gaps) / (f * sat)
        arrival -= arrival[0]
        rc, lat = srv.replay(reqs, arrival, 600000)
        if rc != 0:
            raise RuntimeError("serving replay failed: %d" % rc)
        span = float((arrival + lat).max())
        sweep.append({"offered_x_saturation": f, "offered_rps": f * sat, "GB/s": total / span / 1e9,
                      "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                      "max_ms": 1e3 * float(lat.max())})
    st = srv.stats()
    srv.close()
    best = max(sweep, key=lambda x: x["GB/s"])
    return {"value": best["GB/s"], "unit": "GB/s", "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"],
            "at_offered_x_saturation": best["offered_x_saturation"], "vs_plain": best["GB/s"] / plain_gbs,
            "requests_per_point": nreq, "mean_request_bytes": mean, "launches": st["launches"],
            "sweep": sweep,
            "workload": "Poisson arrivals, sizes log-normal median 256 KiB sigma 1.5 in [4 KiB, 64 MiB], "
                        "10000 cached key triples, 16 GiB admission budget, 4 streams, continuous batching"}


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
    import torch

    from paper_1305_4376_gb300 import build, des3, inputs

    build.build()
    torch.cuda.set_device(local_rank)
    from paper_1305_4376_gb300 import autotune
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
    import ctypes
    ksp = ctypes.byref(ks)
    kernel = des3.KERNELS[args.kernel]
    ptr = buf.data_ptr()

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

    from paper_1305_4376_gb300 import replicas

    def barrier():
        replicas.barrier()

    sampler = ClockSampler(local_rank) if rank == 0 else None
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
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
    barrier()
    clocks = sampler.stop() if sampler else None
    ms = t0.elapsed_time(t1)
    launch_ms = []
    for e in evs:
        launch_ms.append(e[0].elapsed_time(e[1]))
        launch_ms.append(e[1].elapsed_time(e[2]))
    # the buffer must be back to its plaintext after every step
    assert torch.equal(words[check_idx], before), "encrypt + decrypt did not restore the buffer"

    ms = replicas.max_over_ranks(ms, device=dev)

    # ---- end to end through the host-memory entry point ----
    e2e = None
    if not args.no_e2e:
        work_bytes = 3 * (64 << 20)
        work = torch.empty(work_bytes, dtype=torch.uint8, device=dev)
        h_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        h_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        h_in.copy_(buf)
        wp = work.data_ptr()

        def e2e_step():
            rc = lib.des3_ecb_host(ksp, h_in.data_ptr(), h_out.data_ptr(), nbytes, 0, wp, work_bytes, s)
            rc |= lib.des3_ecb_host(ksp, h_out.data_ptr(), h_out.data_ptr(), nbytes, 1, wp, work_bytes, s)
            if rc:
                raise RuntimeError("des3_ecb_host failed: %d" % rc)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = a.elapsed_time(b)
        e_ms = replicas.max_over_ranks(e_ms, device=dev)
        ok = torch.equal(h_out[:1 << 20], h_in[:1 << 20]) and torch.equal(h_out[-(1 << 20):], h_in[-(1 << 20):])
        assert ok, "host-memory round trip did not restore the input"
        e2e = {"value": 2 * nbytes * args.e2e_steps * world / (e_ms * 1e-3) / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": 2 * nbytes,
               "api": "des3_ecb_host (pinned host buffers, 3 x 64 MiB device slots)", "steps": args.e2e_steps,
               "link_each_way_gbs": host_link_gbs(torch, h_in, h_out, buf, stream),
               "note": "the link figure is plain concurrent copies in and out on the same buffers and "
                       "run: the ceiling of this number on this machine at this time"}
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

    # the tuned single-buffer call at the smaller sizes of the size sweep
    # (prefixes of the same buffer, in place, alternating encrypt and decrypt
    # so the buffer ends as it began); below the 129 MB L2 the data stays in
    # L2 and the small sizes are bound by launch latency
    sweep = None
    if not args.no_sweep:
        sweep = []
        for size in (64 << 10, 1 << 20, 16 << 20, 256 << 20):
            if size > nbytes:
                break
            reps = max(20, min(2000, (8 << 30) // size)) & ~1
            for i in range(4):
                lib.des3_ecb_crypt_ex(ksp, ptr, ptr, size, i & 1, 0, s)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for i in range(reps):
                if lib.des3_ecb_crypt_ex(ksp, ptr, ptr, size, i & 1, 0, s):
                    raise RuntimeError("size sweep launch failed")
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / reps
            # the same calls captured in a CUDA graph: device time without the
            # host's per-call cost (ctypes and the launch API)
            ncap = 20
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                cs = torch.cuda.current_stream().cuda_stream
                for i in range(ncap):
                    if lib.des3_ecb_crypt_ex(ksp, ptr, ptr, size, i & 1, 0, cs):
                        raise RuntimeError("size sweep capture failed")
            g.replay()
            torch.cuda.synchronize()
            a.record()
            for _ in range(10):
                g.replay()
            b.record()
            torch.cuda.synchronize()
            tg = a.elapsed_time(b) / (10 * ncap)
            del g
            entry = autotune.get_entry(des3.DES3_TUNE_SINGLE, size.bit_length() - 1)
            sweep.append({"bytes": size, "GB/s": size / (t * 1e-3) / 1e9, "us_per_call": t * 1e3,
                          "graph_GB/s": size / (tg * 1e-3) / 1e9, "graph_us_per_call": tg * 1e3,
                          "kernel": "sptable" if entry[1] == des3.DES3_KERNEL_SPTABLE else "bitslice",
                          "threads": entry[2], "ctas_per_sm": entry[3], "calls": reps})
        assert torch.equal(words[check_idx], before), "size sweep did not restore the buffer"
    batched = serving = None
    value = replicas.aggregate_gbs(2 * nbytes * args.steps, ms, world)
    plain_gbs = value / world
    if not (args.no_batched and args.no_serving):
        del words, buf, before
        torch.cuda.empty_cache()
    if not args.no_batched:
        batched = run_batched(torch, des3, inputs, dev, stream, max(3, args.steps // 3), plain_gbs,
                              args.batched_max_bytes)
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
    ops = info["alu_ops_per_block"] * nblocks
    pt = PROFILED_TRAFFIC
    traffic = None
    src_digest = kernel_sources_digest()
    if kname == pt["kernel"] and src_digest == pt["sources_sha256"]:
        traffic = pt["bytes_per_block"] * nblocks
    achieved = ops / (avg_launch_ms * 1e-3) / 1e12
    peak = SM_COUNT * SM_MAX_MHZ * 1e6 * ALU_LANES_PER_SM_CLK / 1e12
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
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": "ncu capture of a 256 MiB launch, scaled by blocks" if traffic
                     else "no ncu capture of these kernel sources", "kernel_sources_sha256": src_digest,
                     "kernel": kname, "ops_per_block": info["alu_ops_per_block"],
                     "fma_ops_per_block": info["fma_ops_per_block"],
                     "sbox_gates": info["sbox_gates"], "avg_launch_ms": avg_launch_ms,
                     "peak_source": "%d SMs x %d MHz x %d LOP3/SM/clk" % (SM_COUNT, SM_MAX_MHZ,
                                                                          ALU_LANES_PER_SM_CLK),
                     "hbm_gbs": 2 * nbytes / (avg_launch_ms * 1e-3) / 1e9,
                     "hbm_frac": (2 * nbytes / (avg_launch_ms * 1e-3) / 1e9 / hbm_peak) if hbm_peak else None},
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


def host_link_gbs(torch, h_in, h_out, dbuf, stream):
    """GB/s each way of plain pinned-host <-> device copies running at the same
    time in both directions (1 GiB each, three times): the link the
    end-to-end number shares."""
    n = min(1 << 30, h_in.numel() // 2, dbuf.numel() // 2)
    s1 = torch.cuda.Stream()
    s2 = torch.cuda.Stream()
    d_in = dbuf[:n]
    d_out = dbuf[n:2 * n]
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s1.wait_stream(stream)
    s2.wait_stream(stream)
    for _ in range(3):
        with torch.cuda.stream(s1):
            d_in.copy_(h_in[:n], non_blocking=True)
        with torch.cuda.stream(s2):
            h_out[:n].copy_(d_out, non_blocking=True)
    stream.wait_stream(s1)
    stream.wait_stream(s2)
    b.record(stream)
    torch.cuda.synchronize()
    return 3 * n / (a.elapsed_time(b) * 1e-3) / 1e9


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
