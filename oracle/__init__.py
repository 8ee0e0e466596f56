"""Plain CPU oracle for 3DES-EDE in ECB mode (DES per FIPS 46-3).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package.  The GPU library never
imports, links or calls it, and it shares no code or table with the library.

The arithmetic lives in ``des_oracle.c`` (per-bit loops over the standard's
tables, OpenMP over blocks).  This module compiles it with gcc on first use
and exposes it through ctypes with numpy buffers.

Functions (citations are to the paper "3DES ECB Optimized for Massively
Parallel CUDA GPU Architecture"):

* ``tdes_ecb(key24, data, decrypt)``: Sec. II.A, 3DES-EDE over independent
  64-bit blocks (ECB, abstract and Fig. 2).
* ``des_ecb(key8, data, decrypt)``: the DES standard the paper builds on.
* ``des_key_schedule(key8)``: the 16 round keys of FIPS 46-3.
* ``tdes_cbc``, ``tdes_ctr``: CBC and CTR modes of NIST SP 800-38A on the same
  block function; the paper uses ECB only, these back the library's mode
  extension.
* ``table(name)``: the standard's tables, for the structural pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "des_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.oracle_tdes_ecb.argtypes = [u8p, u8p, u8p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
            lib.oracle_tdes_ecb.restype = ctypes.c_int
            lib.oracle_tdes_cbc.argtypes = [u8p, u8p, u8p, u8p, ctypes.c_uint64, ctypes.c_int]
            lib.oracle_tdes_cbc.restype = ctypes.c_int
            lib.oracle_tdes_ctr.argtypes = [u8p, u8p, u8p, u8p, ctypes.c_uint64, ctypes.c_int]
            lib.oracle_tdes_ctr.restype = ctypes.c_int
            lib.oracle_des_ecb.argtypes = [u8p, u8p, u8p, ctypes.c_uint64, ctypes.c_int]
            lib.oracle_des_ecb.restype = ctypes.c_int
            lib.oracle_des_key_schedule.argtypes = [u8p, ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_des_key_schedule.restype = None
            lib.oracle_table.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.POINTER(ctypes.c_int))]
            lib.oracle_table.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _as_bytes(data) -> np.ndarray:
    a = np.ascontiguousarray(np.frombuffer(bytes(data), dtype=np.uint8) if isinstance(data, (bytes, bytearray)) else data)
    if a.dtype != np.uint8:
        a = a.view(np.uint8)
    return np.ascontiguousarray(a.reshape(-1))


def tdes_ecb(key24, data, decrypt: bool = False, nthreads: int = 0) -> np.ndarray:
    """3DES-EDE ECB of ``data`` (bytes or uint8 array, length a multiple of 8)."""
    key = _as_bytes(key24)
    if key.size != 24:
        raise ValueError("3DES key must be 24 bytes (K1||K2||K3)")
    src = _as_bytes(data)
    if src.size % 8:
        raise ValueError("length must be a multiple of 8 bytes")
    out = np.empty_like(src)
    rc = _load().oracle_tdes_ecb(_u8(key), _u8(src), _u8(out), src.size, int(bool(decrypt)), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_tdes_ecb failed: %d" % rc)
    return out


def tdes_cbc(key24, iv8, data, decrypt: bool = False) -> np.ndarray:
    """3DES-EDE in CBC mode (NIST SP 800-38A): not in the paper, an extension."""
    key, iv, src = _as_bytes(key24), _as_bytes(iv8), _as_bytes(data)
    if key.size != 24 or iv.size != 8:
        raise ValueError("need a 24-byte key and an 8-byte IV")
    if src.size % 8:
        raise ValueError("length must be a multiple of 8 bytes")
    out = np.empty_like(src)
    if _load().oracle_tdes_cbc(_u8(key), _u8(iv), _u8(src), _u8(out), src.size, int(bool(decrypt))) != 0:
        raise RuntimeError("oracle_tdes_cbc failed")
    return out


def tdes_ctr(key24, counter8, data, nthreads: int = 0) -> np.ndarray:
    """3DES-EDE in CTR mode: counter block i = counter + i mod 2^64 (big-endian)."""
    key, ctr, src = _as_bytes(key24), _as_bytes(counter8), _as_bytes(data)
    if key.size != 24 or ctr.size != 8:
        raise ValueError("need a 24-byte key and an 8-byte counter block")
    if src.size % 8:
        raise ValueError("length must be a multiple of 8 bytes")
    out = np.empty_like(src)
    if _load().oracle_tdes_ctr(_u8(key), _u8(ctr), _u8(src), _u8(out), src.size, int(nthreads)) != 0:
        raise RuntimeError("oracle_tdes_ctr failed")
    return out


def des_ecb(key8, data, decrypt: bool = False) -> np.ndarray:
    """Single DES ECB with an 8-byte key."""
    key = _as_bytes(key8)
    if key.size != 8:
        raise ValueError("DES key must be 8 bytes")
    src = _as_bytes(data)
    if src.size % 8:
        raise ValueError("length must be a multiple of 8 bytes")
    out = np.empty_like(src)
    rc = _load().oracle_des_ecb(_u8(key), _u8(src), _u8(out), src.size, int(bool(decrypt)))
    if rc != 0:
        raise RuntimeError("oracle_des_ecb failed: %d" % rc)
    return out


def des_key_schedule(key8) -> list[int]:
    """The 16 round keys K_1..K_16 as 48-bit integers (bit 1 = MSB)."""
    key = _as_bytes(key8)
    if key.size != 8:
        raise ValueError("DES key must be 8 bytes")
    out = (ctypes.c_uint64 * 16)()
    _load().oracle_des_key_schedule(_u8(key), out)
    return [int(v) for v in out]


def table(name: str) -> list[int]:
    """A FIPS 46-3 table by name: IP, FP, E, P, PC1, PC2, SHIFT, SBOX (8x4x16 flat)."""
    ptr = ctypes.POINTER(ctypes.c_int)()
    n = _load().oracle_table(name.encode(), ctypes.byref(ptr))
    if n == 0:
        raise KeyError(name)
    return [int(ptr[i]) for i in range(n)]


def max_threads() -> int:
    """Threads the OpenMP oracle uses by default."""
    return int(_load().oracle_max_threads())
