"""Autotuner for the launch tables (des3_tune_set).

For every size class it times each candidate on the GPU and keeps the
fastest:

* single-buffer table: the bitsliced kernel and the SP-table kernel, each
  with CTA sizes 64 to 384 and the CTAs per SM their registers and shared
  memory allow, on one buffer of 2^c bytes (c = 12 .. 32);
* batch table: the batched bitsliced kernel and the batched table kernel,
  each with its CTA sizes and CTAs per SM, on batches of log-uniform buffers
  totalling 2^c bytes (c = 16 .. 32).

Timing: CUDA events around repeated launches on one stream, after warm-up,
on seeded data; each candidate's figure is the median of 5 repetitions.
The result is written as JSON keyed by GPU name and applied with
load_tuning(); classes between measured ones take the nearest measured
choice.

    python -m paper_1305_4376_gb300.autotune [--out FILE] [--max-class 32]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics

from paper_1305_4376_gb300 import des3, inputs

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")

SINGLE_CANDIDATES = [(des3.DES3_KERNEL_BITSLICE, 384, 1), (des3.DES3_KERNEL_BITSLICE, 128, 3),
                     (des3.DES3_KERNEL_BITSLICE, 256, 1), (des3.DES3_KERNEL_BITSLICE, 128, 2),
                     (des3.DES3_KERNEL_BITSLICE, 128, 1), (des3.DES3_KERNEL_BITSLICE, 64, 4),
                     (des3.DES3_KERNEL_SPTABLE, 384, 3), (des3.DES3_KERNEL_SPTABLE, 256, 3),
                     (des3.DES3_KERNEL_SPTABLE, 128, 3), (des3.DES3_KERNEL_SPTABLE, 384, 2),
                     (des3.DES3_KERNEL_SPTABLE, 256, 2), (des3.DES3_KERNEL_SPTABLE, 128, 2),
                     (des3.DES3_KERNEL_SPTABLE, 64, 3)]
BATCH_CANDIDATES = [(des3.DES3_KERNEL_BITSLICE, 384, 1), (des3.DES3_KERNEL_BITSLICE, 128, 3),
                    (des3.DES3_KERNEL_BITSLICE, 256, 1), (des3.DES3_KERNEL_BITSLICE, 128, 2),
                    (des3.DES3_KERNEL_BITSLICE, 64, 4), (des3.DES3_KERNEL_BITSLICE, 128, 1),
                    (des3.DES3_KERNEL_SPTABLE, 384, 3), (des3.DES3_KERNEL_SPTABLE, 256, 3),
                    (des3.DES3_KERNEL_SPTABLE, 128, 3)]


class des3_tune_entry_t(ctypes.Structure):
    _fields_ = [("size_class", ctypes.c_uint32), ("kernel", ctypes.c_int32), ("threads", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32)]


def _lib():
    lib = des3.lib()
    lib.des3_tune_set.argtypes = [ctypes.c_int, ctypes.POINTER(des3_tune_entry_t), ctypes.c_uint32]
    lib.des3_tune_set.restype = ctypes.c_int
    lib.des3_tune_get.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(des3_tune_entry_t)]
    lib.des3_tune_get.restype = ctypes.c_int
    lib.des3_tune_reset.argtypes = []
    lib.des3_tune_reset.restype = ctypes.c_int
    return lib


def set_entries(table: int, entries) -> None:
    arr = (des3_tune_entry_t * len(entries))()
    for i, (c, k, t, n) in enumerate(entries):
        arr[i] = des3_tune_entry_t(c, k, t, n)
    rc = _lib().des3_tune_set(table, arr, len(entries))
    if rc != des3.DES3_OK:
        raise des3.Des3Error(rc, "des3_tune_set")


def get_entry(table: int, c: int):
    e = des3_tune_entry_t()
    rc = _lib().des3_tune_get(table, c, ctypes.byref(e))
    if rc != des3.DES3_OK:
        raise des3.Des3Error(rc, "des3_tune_get")
    return (e.size_class, e.kernel, e.threads, e.ctas_per_sm)


def reset() -> None:
    _lib().des3_tune_reset()


def fill_classes(measured: dict) -> list:
    """Entries for all 40 classes: each takes the nearest measured class's choice."""
    keys = sorted(measured)
    out = []
    for c in range(40):
        near = min(keys, key=lambda m: (abs(m - c), m))
        k, t, n = measured[near]
        out.append((c, k, t, n))
    return out


def tuning_path(gpu_name: str) -> str:
    return os.path.join(TUNING_DIR, gpu_name.replace(" ", "_") + ".json")


def load_tuning(path: str | None = None) -> bool:
    """Installs a saved table (default: the one for the current GPU).  Returns
    False when no file exists."""
    if path is None:
        import torch
        path = tuning_path(torch.cuda.get_device_name())
    if not os.path.exists(path):
        return False
    doc = json.load(open(path))
    for name, table in (("single", des3.DES3_TUNE_SINGLE), ("batch", des3.DES3_TUNE_BATCH)):
        meas = {int(c): tuple(v) for c, v in doc[name].items()}
        set_entries(table, fill_classes(meas))
    return True


def _time(fn, stream, reps=5, inner=1):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(inner):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / inner)
    return statistics.median(ts)


def tune_single(max_class=32, min_class=12):
    import torch
    lib = _lib()
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    ks = des3.des3_key_schedule(inputs.key_triple(0xA77))
    big = inputs.splitmix64_torch(0xA78, 0, (1 << max_class) // 8, "cuda").view(torch.uint8)
    results = {}
    for c in range(min_class, max_class + 1, 2):
        n = 1 << c
        buf = big[:n]
        inner = max(1, min(200, (1 << 26) // n))
        best = None
        rows = []
        for (k, t, ctas) in SINGLE_CANDIDATES:
            reset()
            set_entries(des3.DES3_TUNE_SINGLE, [(c, k, t, ctas)])

            def run():
                rc = lib.des3_ecb_crypt_ex(ctypes.byref(ks), buf.data_ptr(), buf.data_ptr(), n, 0, 0, s)
                if rc:
                    raise des3.Des3Error(rc, "des3_ecb_crypt_ex")

            ms = _time(run, stream, inner=inner)
            rows.append({"kernel": k, "threads": t, "ctas_per_sm": ctas, "ms": ms, "GB/s": n / ms / 1e6})
            if best is None or ms < best[0]:
                best = (ms, (k, t, ctas))
        results[c] = {"choice": best[1], "candidates": rows}
    reset()
    return results


def tune_batch(max_class=32, min_class=16):
    import torch
    stream = torch.cuda.current_stream()
    results = {}
    keys = des3.make_keys([des3.des3_key_schedule(k) for k in inputs.key_triples(0xB00, 64)])
    for c in range(min_class, max_class + 1, 2):
        total_target = 1 << c
        sizes, dec = inputs.batch_recipe(0xB01 + c, njobs=256, lo=512, hi=max(1024, total_target // 16))
        scale = total_target / float(sizes.sum())
        sizes = [max(8, int(x * scale) // 8 * 8) for x in sizes]
        offs, pos = [], 0
        for n in sizes:
            offs.append(pos)
            pos += (n + 255) // 256 * 256
        buf = inputs.splitmix64_torch(0xB02, 0, pos // 8 + 32, "cuda").view(torch.uint8)
        jobs = des3.make_jobs([(buf[o:o + n], buf[o:o + n], n, i % 64, bool(dec[i]))
                               for i, (n, o) in enumerate(zip(sizes, offs))])
        best = None
        rows = []
        for (k, t, ctas) in BATCH_CANDIDATES:
            reset()
            set_entries(des3.DES3_TUNE_BATCH, [(cc, k, t, ctas) for cc in range(40)])
            plan = des3.BatchPlan(keys, jobs)
            inner = max(1, min(100, (1 << 27) // total_target))
            ms = _time(lambda: plan.launch(stream), stream, inner=inner)
            plan.close()
            rows.append({"kernel": k, "threads": t, "ctas_per_sm": ctas, "ms": ms, "GB/s": sum(sizes) / ms / 1e6})
            if best is None or ms < best[0]:
                best = (ms, (k, t, ctas))
        results[c] = {"choice": best[1], "candidates": rows}
        del buf
    reset()
    return results


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--max-class", type=int, default=32)
    args = ap.parse_args()
    from paper_1305_4376_gb300 import build
    build.build()
    name = torch.cuda.get_device_name()
    single = tune_single(args.max_class)
    batch = tune_batch(args.max_class)
    doc = {"gpu": name, "sms": torch.cuda.get_device_properties(0).multi_processor_count,
           "method": "median of 5 CUDA-event timings per candidate, in-place encryption of seeded data",
           "single": {str(c): list(v["choice"]) for c, v in single.items()},
           "batch": {str(c): list(v["choice"]) for c, v in batch.items()},
           "measurements": {"single": {str(c): v["candidates"] for c, v in single.items()},
                            "batch": {str(c): v["candidates"] for c, v in batch.items()}}}
    out = args.out or tuning_path(name)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    with open(out, "w") as f:
        json.dump(doc, f, indent=1)
    for c in sorted(single):
        print("single 2^%d: %s" % (c, single[c]["choice"]))
    for c in sorted(batch):
        print("batch  2^%d: %s" % (c, batch[c]["choice"]))
    print("wrote", out)


if __name__ == "__main__":
    main()
