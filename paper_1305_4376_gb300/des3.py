"""Thin Python binding of libdes3gpu.so (include/des3.h), through ctypes.

Only argument marshalling happens here: every step of the cipher runs in the
library's CUDA kernels.  PyTorch is used for device memory and streams only
(``tensor.data_ptr()`` and ``torch.cuda.current_stream().cuda_stream``).

The functions keep the C names.  They raise ``Des3Error`` (carrying the
DES3_E* code) instead of returning error codes; ``lib()`` gives the raw
ctypes handle for callers that want the codes.  There is no fallback: if the
shared library has not been built, or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdes3gpu.so")

DES3_OK = 0
DES3_EINVAL = -1
DES3_EKEY = -2
DES3_ECUDA = -3
DES3_ETIMEOUT = -4
DES3_ENOMEM = -5
DES3_ENODEV = -6
DES3_EBUSY = -7

DES3_KERNEL_AUTO = 0
DES3_KERNEL_BITSLICE = 1
DES3_KERNEL_SPTABLE = 2
KERNELS = {"auto": DES3_KERNEL_AUTO, "bitslice": DES3_KERNEL_BITSLICE, "sptable": DES3_KERNEL_SPTABLE}

DES3_JOB_DECRYPT = 1
DES3_FAULT_AT_LAUNCH = 0
DES3_FAULT_AT_COMPLETION = 1
DES3_TUNE_SINGLE = 0
DES3_TUNE_BATCH = 1
DES3_KS_MAGIC = 0x4B533344
DES3_KS_SINGLE_DES = 1


class des3_ks_t(ctypes.Structure):
    """Key schedule: rk[0] = the 48 encryption round keys in application order,
    rk[1] = the same reversed (decryption)."""
    _fields_ = [("magic", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("rk", (ctypes.c_uint64 * 48) * 2)]


class des3_job_t(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("nbytes", ctypes.c_uint64),
                ("key_index", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class des3_kernel_info_t(ctypes.Structure):
    _fields_ = [("alu_ops_per_block", ctypes.c_double), ("fma_ops_per_block", ctypes.c_double),
                ("smem_loads_per_block", ctypes.c_double), ("sbox_gates", ctypes.c_int),
                ("blocks_per_thread", ctypes.c_int)]


class des3_server_config_t(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_queue", ctypes.c_uint32), ("nstreams", ctypes.c_uint32),
                ("max_batch_requests", ctypes.c_uint32), ("max_batch_bytes", ctypes.c_uint64),
                ("key_capacity", ctypes.c_uint32), ("fault_every", ctypes.c_uint32),
                ("fault_stage", ctypes.c_uint32)]


class des3_request_t(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("nbytes", ctypes.c_uint64),
                ("key_id", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("tag", ctypes.c_uint64)]


class des3_completion_t(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int),
                ("batch_size", ctypes.c_uint32), ("latency_s", ctypes.c_double)]


class des3_server_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "launches", "bytes_completed",
                                               "inflight_bytes", "inflight_requests", "queued_requests",
                                               "table_launches")]


class Des3Error(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = "%s failed: %s (%d)" % (what, strerror(code) if _lib is not None else "error", code)
        if code == DES3_ECUDA and _lib is not None:
            msg += ", CUDA error %d" % _lib.des3_last_cuda_error()
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def _declare(lib):
    vp, sz, i, u32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
    ks_p = ctypes.POINTER(des3_ks_t)
    job_p = ctypes.POINTER(des3_job_t)
    sigs = {
        "des3_key_schedule": ([ctypes.c_char_p, ks_p], i),
        "des3_key_schedule_des": ([ctypes.c_char_p, ks_p], i),
        "des3_ecb_encrypt": ([ks_p, vp, vp, sz, vp], i),
        "des3_ecb_decrypt": ([ks_p, vp, vp, sz, vp], i),
        "des3_ecb_crypt_ex": ([ks_p, vp, vp, sz, i, i, vp], i),
        "des3_ecb_host": ([ks_p, vp, vp, sz, i, vp, sz, vp], i),
        "des3_ecb_host_multi": ([ks_p, vp, vp, sz, i, u32, ctypes.POINTER(i), ctypes.POINTER(vp),
                                 ctypes.POINTER(sz)], i),
        "des3_range_split": ([u64, u32, u64, ctypes.POINTER(u64)], i),
        "des3_ctr_crypt": ([ks_p, ctypes.c_char_p, vp, vp, sz, vp], i),
        "des3_cbc_decrypt": ([ks_p, ctypes.c_char_p, vp, vp, sz, vp], i),
        "des3_ecb_batch": ([ks_p, u32, job_p, u32, vp], i),
        "des3_ecb_batch_noalloc": ([ks_p, u32, job_p, u32, vp], i),
        "des3_batch_plan_create": ([ks_p, u32, job_p, u32, i, ctypes.POINTER(vp)], i),
        "des3_batch_plan_launch": ([vp, vp], i),
        "des3_batch_plan_destroy": ([vp], i),
        "des3_batch_plan_info": ([vp, ctypes.POINTER(u64), ctypes.POINTER(u64)], i),
        "des3_batch_plan_kernel": ([vp, ctypes.POINTER(i), ctypes.POINTER(u32), ctypes.POINTER(u32)], i),
        "des3_batch_choose": ([job_p, u32, u32, ctypes.POINTER(i), ctypes.POINTER(u32), ctypes.POINTER(u32)], i),
        "des3_strerror": ([i], ctypes.c_char_p),
        "des3_last_cuda_error": ([], i),
        "des3_self_test": ([], i),
        "des3_server_create": ([ctypes.POINTER(des3_server_config_t), ctypes.POINTER(vp)], i),
        "des3_server_add_keys": ([vp, ks_p, u32, ctypes.POINTER(u32)], i),
        "des3_server_submit": ([vp, ctypes.POINTER(des3_request_t), ctypes.POINTER(u64)], i),
        "des3_server_poll": ([vp, ctypes.POINTER(des3_completion_t), u32, ctypes.POINTER(u32)], i),
        "des3_server_drain": ([vp, i], i),
        "des3_server_stats": ([vp, ctypes.POINTER(des3_server_stats_t)], i),
        "des3_server_replay": ([vp, ctypes.POINTER(des3_request_t), ctypes.POINTER(ctypes.c_double), u32,
                                ctypes.POINTER(ctypes.c_double), i], i),
        "des3_server_destroy": ([vp], i),
        "des3_kernel_info": ([i, ctypes.POINTER(des3_kernel_info_t)], i),
        "des3_pipe_probe": ([i, u32, vp, ctypes.POINTER(u64), ctypes.POINTER(u32), vp], i),
        "des3_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.argtypes = args
        fn.restype = res


def lib():
    """The loaded shared library (raises if it is missing)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError("libdes3gpu.so is not built (%s); run paper_1305_4376_gb300.build.build()"
                                       % LIB_PATH)
                handle = ctypes.CDLL(LIB_PATH)
                _declare(handle)
                _lib = handle
    return _lib


def strerror(code: int) -> str:
    return lib().des3_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != DES3_OK:
        raise Des3Error(rc, what)


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x) -> int:
    return x if isinstance(x, int) else x.data_ptr()


def _nbytes(x) -> int:
    return x.numel() * x.element_size()


# ---- the C calls, same names ---------------------------------------------

def des3_key_schedule(key24: bytes) -> des3_ks_t:
    if len(key24) != 24:
        raise ValueError("a 3DES key is 24 bytes K1||K2||K3")
    ks = des3_ks_t()
    _check(lib().des3_key_schedule(bytes(key24), ctypes.byref(ks)), "des3_key_schedule")
    return ks


def des3_key_schedule_des(key8: bytes) -> des3_ks_t:
    """Single-DES schedule (flags = DES3_KS_SINGLE_DES); usable with every call."""
    if len(key8) != 8:
        raise ValueError("a DES key is 8 bytes")
    ks = des3_ks_t()
    _check(lib().des3_key_schedule_des(bytes(key8), ctypes.byref(ks)), "des3_key_schedule_des")
    return ks


def des3_ecb_encrypt(ks: des3_ks_t, d_in, d_out, nbytes: int | None = None, stream=None) -> None:
    n = _nbytes(d_in) if nbytes is None else nbytes
    _check(lib().des3_ecb_encrypt(ctypes.byref(ks), _ptr(d_in), _ptr(d_out), n, _stream(stream)),
           "des3_ecb_encrypt")


def des3_ecb_decrypt(ks: des3_ks_t, d_in, d_out, nbytes: int | None = None, stream=None) -> None:
    n = _nbytes(d_in) if nbytes is None else nbytes
    _check(lib().des3_ecb_decrypt(ctypes.byref(ks), _ptr(d_in), _ptr(d_out), n, _stream(stream)),
           "des3_ecb_decrypt")


def des3_ecb_crypt_ex(ks: des3_ks_t, d_in, d_out, nbytes: int | None = None, decrypt: bool = False,
                      kernel="auto", stream=None) -> None:
    n = _nbytes(d_in) if nbytes is None else nbytes
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    _check(lib().des3_ecb_crypt_ex(ctypes.byref(ks), _ptr(d_in), _ptr(d_out), n, int(bool(decrypt)), k,
                                   _stream(stream)), "des3_ecb_crypt_ex")


def des3_ecb_host(ks: des3_ks_t, h_in: int, h_out: int, nbytes: int, decrypt: bool, d_work: int,
                  work_bytes: int, stream=None) -> None:
    _check(lib().des3_ecb_host(ctypes.byref(ks), h_in, h_out, nbytes, int(bool(decrypt)), d_work,
                               work_bytes, _stream(stream)), "des3_ecb_host")


def des3_ecb_host_multi(ks: des3_ks_t, h_in: int, h_out: int, nbytes: int, decrypt: bool, devices,
                        d_work, work_bytes) -> None:
    """Host buffer split into contiguous block ranges, range i through
    devices[i] with workspace d_work[i] (device pointers or tensors) of
    work_bytes[i] bytes; returns when every range is done."""
    n = len(devices)
    if len(d_work) != n or len(work_bytes) != n:
        raise ValueError("one workspace and size per device")
    devs = (ctypes.c_int * n)(*devices)
    works = (ctypes.c_void_p * n)(*[_ptr(w) if w is not None else None for w in d_work])
    sizes = (ctypes.c_size_t * n)(*work_bytes)
    _check(lib().des3_ecb_host_multi(ctypes.byref(ks), h_in, h_out, nbytes, int(bool(decrypt)), n, devs, works,
                                     sizes), "des3_ecb_host_multi")


def des3_range_split(nblocks: int, nparts: int, granule: int = 1024) -> list[int]:
    """Boundaries first[0..nparts] of the contiguous split des3_ecb_host_multi uses."""
    out = (ctypes.c_uint64 * (nparts + 1))()
    _check(lib().des3_range_split(nblocks, nparts, granule, out), "des3_range_split")
    return list(out)


def des3_ctr_crypt(ks: des3_ks_t, counter8: bytes, d_in, d_out, nbytes: int | None = None, stream=None) -> None:
    """CTR mode (encrypts and decrypts): out_i = in_i ^ E(counter + i)."""
    if len(counter8) != 8:
        raise ValueError("the counter block is 8 bytes")
    n = _nbytes(d_in) if nbytes is None else nbytes
    _check(lib().des3_ctr_crypt(ctypes.byref(ks), bytes(counter8), _ptr(d_in), _ptr(d_out), n, _stream(stream)),
           "des3_ctr_crypt")


def des3_cbc_decrypt(ks: des3_ks_t, iv8: bytes, d_in, d_out, nbytes: int | None = None, stream=None) -> None:
    """CBC decryption (out of place): out_i = D(in_i) ^ in_{i-1}."""
    if len(iv8) != 8:
        raise ValueError("the IV is 8 bytes")
    n = _nbytes(d_in) if nbytes is None else nbytes
    _check(lib().des3_cbc_decrypt(ctypes.byref(ks), bytes(iv8), _ptr(d_in), _ptr(d_out), n, _stream(stream)),
           "des3_cbc_decrypt")


def make_keys(schedules) -> ctypes.Array:
    arr = (des3_ks_t * len(schedules))()
    for i, ks in enumerate(schedules):
        arr[i] = ks
    return arr


def make_jobs(jobs) -> ctypes.Array:
    """jobs: iterable of (d_in, d_out, nbytes, key_index, decrypt)."""
    jobs = list(jobs)
    arr = (des3_job_t * len(jobs))()
    for i, (src, dst, n, kidx, dec) in enumerate(jobs):
        arr[i].d_in = _ptr(src)
        arr[i].d_out = _ptr(dst)
        arr[i].nbytes = n
        arr[i].key_index = kidx
        arr[i].flags = DES3_JOB_DECRYPT if dec else 0
    return arr


def des3_ecb_batch(keys: ctypes.Array, jobs: ctypes.Array, stream=None) -> None:
    _check(lib().des3_ecb_batch(keys, len(keys), jobs, len(jobs), _stream(stream)), "des3_ecb_batch")


def des3_batch_choose(jobs: ctypes.Array, sms: int):
    """(kernel, threads, ctas_per_sm) a batched call would choose for these jobs
    on a device with `sms` SMs, under the current tuning table; host only."""
    k, t, c = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().des3_batch_choose(jobs, len(jobs), sms, ctypes.byref(k), ctypes.byref(t), ctypes.byref(c)),
           "des3_batch_choose")
    return k.value, t.value, c.value


class BatchPlan:
    """des3_batch_plan_create / _launch / _destroy as a Python object."""

    def __init__(self, keys: ctypes.Array, jobs: ctypes.Array, kernel="auto"):
        self._h = ctypes.c_void_p()
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        _check(lib().des3_batch_plan_create(keys, len(keys), jobs, len(jobs), k, ctypes.byref(self._h)),
               "des3_batch_plan_create")

    def launch(self, stream=None) -> None:
        _check(lib().des3_batch_plan_launch(self._h, _stream(stream)), "des3_batch_plan_launch")

    def info(self):
        tb, tl = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().des3_batch_plan_info(self._h, ctypes.byref(tb), ctypes.byref(tl)), "des3_batch_plan_info")
        return tb.value, tl.value

    def kernel(self):
        """(kernel, threads, ctas_per_sm) of the launch the plan replays."""
        k, t, c = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().des3_batch_plan_kernel(self._h, ctypes.byref(k), ctypes.byref(t), ctypes.byref(c)),
               "des3_batch_plan_kernel")
        return k.value, t.value, c.value

    def close(self) -> None:
        if self._h:
            _check(lib().des3_batch_plan_destroy(self._h), "des3_batch_plan_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """des3_server_*: continuous batching of requests on device buffers."""

    def __init__(self, budget_bytes=16 << 30, max_inflight=8192, max_queue=1 << 20, nstreams=4,
                 max_batch_requests=2048, max_batch_bytes=1 << 30, key_capacity=10000, fault_every=0,
                 fault_stage=0):
        cfg = des3_server_config_t(budget_bytes, max_inflight, max_queue, nstreams, max_batch_requests,
                                   max_batch_bytes, key_capacity, fault_every, fault_stage)
        self._h = ctypes.c_void_p()
        _check(lib().des3_server_create(ctypes.byref(cfg), ctypes.byref(self._h)), "des3_server_create")

    def add_keys(self, schedules) -> int:
        arr = make_keys(list(schedules))
        first = ctypes.c_uint32()
        _check(lib().des3_server_add_keys(self._h, arr, len(arr), ctypes.byref(first)), "des3_server_add_keys")
        return first.value

    @staticmethod
    def request(d_in, d_out, nbytes, key_id, decrypt=False, tag=0) -> des3_request_t:
        return des3_request_t(_ptr(d_in), _ptr(d_out), nbytes, key_id, DES3_JOB_DECRYPT if decrypt else 0, tag)

    def submit(self, d_in, d_out, nbytes, key_id, decrypt=False, tag=0) -> int:
        req = self.request(d_in, d_out, nbytes, key_id, decrypt, tag)
        t = ctypes.c_uint64()
        _check(lib().des3_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "des3_server_submit")
        return t.value

    def poll(self, max_n=4096) -> list:
        buf = (des3_completion_t * max_n)()
        n = ctypes.c_uint32()
        _check(lib().des3_server_poll(self._h, buf, max_n, ctypes.byref(n)), "des3_server_poll")
        return [dict(ticket=c.ticket, tag=c.tag, status=c.status, batch_size=c.batch_size, latency_s=c.latency_s)
                for c in buf[:n.value]]

    def drain(self, timeout_ms=60000) -> None:
        _check(lib().des3_server_drain(self._h, timeout_ms), "des3_server_drain")

    def stats(self) -> dict:
        st = des3_server_stats_t()
        _check(lib().des3_server_stats(self._h, ctypes.byref(st)), "des3_server_stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def replay(self, requests, arrival_s, timeout_ms=600000):
        """requests: ctypes array of des3_request_t; arrival_s: float64 numpy array."""
        import numpy as np
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.empty(len(arr), dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        rc = lib().des3_server_replay(self._h, requests, arr.ctypes.data_as(dp), len(arr), lat.ctypes.data_as(dp),
                                      timeout_ms)
        return rc, lat

    def close(self) -> None:
        if self._h:
            _check(lib().des3_server_destroy(self._h), "des3_server_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def des3_self_test() -> None:
    _check(lib().des3_self_test(), "des3_self_test")


def des3_kernel_info(kernel="bitslice") -> dict:
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    info = des3_kernel_info_t()
    _check(lib().des3_kernel_info(k, ctypes.byref(info)), "des3_kernel_info")
    return {f: getattr(info, f) for f, _ in info._fields_}


PROBE_KINDS = {"lop3": 0, "imad": 1, "lop3+imad": 2, "lds": 3}


def des3_pipe_probe(kind, iters: int, d_sink, stream=None):
    """Launches the pipe-throughput probe (kind: a PROBE_KINDS name or number)
    on ``stream``; d_sink: a device tensor of at least 24 bytes.  Returns
    (lane-instructions of the launch, SM count)."""
    k = PROBE_KINDS[kind] if isinstance(kind, str) else int(kind)
    ins, sms = ctypes.c_uint64(), ctypes.c_uint32()
    _check(lib().des3_pipe_probe(k, iters, _ptr(d_sink), ctypes.byref(ins), ctypes.byref(sms), _stream(stream)),
           "des3_pipe_probe")
    return ins.value, sms.value


def des3_version() -> str:
    return lib().des3_version().decode()


def exported_symbols() -> list[str]:
    """Names declared in include/des3.h (for the export test)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "des3.h")
    src = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(des3_[a-z_0-9]+)\s*\(", src, re.M)))
