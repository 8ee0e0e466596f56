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
# LOP3 (integer ALU pipe) instructions per SM per clock on GB300, measured
# by a throughput micro-benchmark ("ALU roofline").
ALU_LANES_PER_SM_CLK = 64
SM_COUNT = 152
SM_MAX_MHZ = 2070


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "bitslice", "sptable"])
    ap.add_argument("--bytes", type=int, default=WORKLOAD_BYTES, help="buffer size (default 4 GiB)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
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


def emit(obj):
    print(json.dumps(obj), flush=True)


# ---------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1305_4376_gb300 import inputs

    key = inputs.key_triple(inputs.key_seed(CONFIG_ID))
    sample = 4 << 20
    data = inputs.data_bytes(inputs.data_seed(CONFIG_ID), sample)
    for _ in range(args.warmup):
        oracle.tdes_ecb(key, oracle.tdes_ecb(key, data), decrypt=True)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.tdes_ecb(key, oracle.tdes_ecb(key, data), decrypt=True)
    dt = time.perf_counter() - t
    value = 2 * sample * args.steps / dt / 1e9
    cores = oracle.max_threads()
    desc = "4 MiB prefix of the 4 GiB workload per step, encrypt + decrypt"
    emit({"impl": "reference", "metric": "3DES-ECB GB/s", "value": value, "unit": "GB/s",
          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "u64", "data": "synthetic (SplitMix64 bytes, seeded)",
          "config": {"workload": "3-key 3DES-EDE ECB encrypt + decrypt, 4 GiB buffer (2^29 blocks), one key triple",
                     "sample_per_step_bytes": sample},
          "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
          "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1305_4376_gb300 import build, des3, inputs

    build.build()
    torch.cuda.set_device(local_rank)
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

    def barrier():
        if world > 1:
            dist.barrier()

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

    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

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
        if world > 1:
            t = torch.tensor([e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        ok = torch.equal(h_out[:1 << 20], h_in[:1 << 20]) and torch.equal(h_out[-(1 << 20):], h_in[-(1 << 20):])
        assert ok, "host-memory round trip did not restore the input"
        e2e = {"value": 2 * nbytes * args.e2e_steps * world / (e_ms * 1e-3) / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": 2 * nbytes,
               "api": "des3_ecb_host (pinned host buffers, 3 x 64 MiB device slots)", "steps": args.e2e_steps}
        del work, h_in, h_out

    if rank != 0:
        return

    kname = args.kernel if args.kernel != "auto" else ("bitslice" if nblocks >= 8192 else "sptable")
    info = des3.des3_kernel_info(kname)
    avg_launch_ms = statistics.mean(launch_ms)
    ops = info["alu_ops_per_block"] * nblocks
    achieved = ops / (avg_launch_ms * 1e-3) / 1e12
    peak = SM_COUNT * SM_MAX_MHZ * 1e6 * ALU_LANES_PER_SM_CLK / 1e12
    value = 2 * nbytes * args.steps * world / (ms * 1e-3) / 1e9
    cpu = None
    if world == 1 and not args.no_cpu:
        rate, cores, desc = cpu_oracle_rate()
        cpu = {"value": rate, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc}
    emit({
        "metric": "3DES-ECB GB/s", "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (SplitMix64 bytes generated on the device, seeded)",
        "config": {"workload": "plain single-buffer: 3-key 3DES-EDE ECB encrypt + decrypt in place, "
                               "%d MiB device-resident buffer (%d blocks), one key triple" % (nbytes >> 20, nblocks),
                   "kernel": kname, "l2": "inputs 4 GiB >> 129 MB L2; no flush",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": kname, "ops_per_block": info["alu_ops_per_block"],
                     "sbox_gates": info["sbox_gates"], "avg_launch_ms": avg_launch_ms,
                     "peak_source": "%d SMs x %d MHz x %d LOP3/SM/clk" % (SM_COUNT, SM_MAX_MHZ,
                                                                          ALU_LANES_PER_SM_CLK),
                     "hbm_gbs": 2 * nbytes / (avg_launch_ms * 1e-3) / 1e9},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": 2 * args.steps,
    })


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
