"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no cipher arithmetic.  It only draws data and keys.

Every random value comes from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014).  It is counter
based: word ``i`` of a stream seeded with ``s`` is the (i+1)-th output of the
sequential generator started from state ``s``, i.e.
``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``.  This lets any block of a 4 GiB
input be recomputed on the host without generating the whole stream, and lets
the device generate the stream in place.

The paper encrypts an unnamed ~512 MB file (Sec. III); no public dataset is
involved.  Uniform random bytes stand in for it: ECB treats every block the
same way, so the cost does not depend on the data.

Keys are "parity-adjusted": uniform bytes whose low bit is then set so that
each byte has odd parity (the DES convention; the cipher ignores these bits).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# Seeds of the five workloads: data seed 0xDE5C0DE0 + id, key seed 0x3DE5 + id.
DATA_SEED_BASE = 0xDE5C0DE0
KEY_SEED_BASE = 0x3DE5


def data_seed(config_id: int) -> int:
    return DATA_SEED_BASE + config_id


def key_seed(config_id: int) -> int:
    return KEY_SEED_BASE + config_id


def splitmix64_scalar(seed: int, index: int) -> int:
    """Word ``index`` of the SplitMix64 stream seeded with ``seed`` (pure Python)."""
    z = (seed + (index + 1) * GOLDEN) & MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Words ``start .. start+count-1`` of the stream, as a numpy uint64 array."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + idx * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))


def splitmix64_at(seed: int, indices: np.ndarray) -> np.ndarray:
    """Words at arbitrary indices of the stream (numpy uint64)."""
    with np.errstate(over="ignore"):
        idx = np.asarray(indices, dtype=np.uint64) + np.uint64(1)
        z = np.uint64(seed & MASK64) + idx * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))


def data_bytes(seed: int, nbytes: int, start_block: int = 0) -> np.ndarray:
    """``nbytes`` (a multiple of 8) of data: word i stored little-endian."""
    assert nbytes % 8 == 0
    words = splitmix64(seed, start_block, nbytes // 8)
    return words.astype("<u8").view(np.uint8)


def _signed(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >> 63 else v


def splitmix64_torch(seed: int, start: int, count: int, device, chunk: int = 1 << 26):
    """The same stream generated with torch int64 ops on ``device`` (wrapping
    multiplies, logical shifts by masking).  Returns an int64 tensor whose
    bytes equal ``splitmix64(seed, start, count)``."""
    import torch

    out = torch.empty(count, dtype=torch.int64, device=device)
    g = _signed(GOLDEN)
    m1 = _signed(M1)
    m2 = _signed(M2)
    base = _signed(seed)

    def lsr(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)

    for off in range(0, count, chunk):
        n = min(chunk, count - off)
        idx = torch.arange(start + off + 1, start + off + n + 1, dtype=torch.int64, device=device)
        z = idx * g + base
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        out[off:off + n] = z ^ lsr(z, 31)
    return out


def odd_parity(b: int) -> int:
    """Set the low bit of byte ``b`` so that it has odd parity."""
    b &= 0xFE
    return b | (1 - (bin(b).count("1") & 1))


def key_triple(seed: int, keying: str = "3key") -> bytes:
    """A parity-adjusted 24-byte key K1||K2||K3 drawn from the seed's stream.

    ``keying="2key"`` gives K1||K2||K1 (keying option 2); ``"1key"`` gives
    K1||K1||K1, which reduces 3DES-EDE to single DES."""
    w = splitmix64(seed, 0, 3)
    raw = w.astype("<u8").view(np.uint8)
    k = bytes(odd_parity(int(x)) for x in raw)
    if keying == "2key":
        k = k[:16] + k[:8]
    elif keying == "1key":
        k = k[:8] * 3
    elif keying != "3key":
        raise ValueError(keying)
    return k


def key_triples(seed: int, count: int) -> list[bytes]:
    """``count`` independent parity-adjusted 3-key triples (3 words each)."""
    w = splitmix64(seed, 0, 3 * count).astype("<u8").view(np.uint8)
    par = np.array([odd_parity(i) for i in range(256)], dtype=np.uint8)
    adj = par[w].reshape(count, 24)
    return [bytes(row) for row in adj]


def uniforms(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of each word."""
    w = splitmix64(seed, start, count)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def batch_recipe(seed: int, njobs: int = 4096, lo: int = 512, hi: int = 16 << 20):
    """Batched workload: ``njobs`` buffer sizes log-uniform on [lo, hi] bytes,
    rounded down to a multiple of 8, and direction flags Bernoulli(0.5).
    Returns (sizes: int64 array, decrypt: bool array)."""
    u = uniforms(seed, 2 * njobs)
    sizes = np.exp(np.log(lo) + u[:njobs] * (np.log(hi) - np.log(lo)))
    sizes = (np.floor(sizes / 8.0) * 8).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    decrypt = u[njobs:] < 0.5
    return sizes, decrypt


def arena_offsets(sizes, align: int = 256):
    """Byte offsets of buffers laid out back to back in one arena, each
    starting at a multiple of ``align``: buffer i starts where buffer i-1
    ends, rounded up.  Returns (offsets, arena bytes).  The arena's bytes are
    word ``offset // 8 + j`` of the data stream, so buffer i holds
    ``data_bytes(seed, sizes[i], start_block=offsets[i] // 8)``."""
    offs, pos = [], 0
    for n in sizes:
        offs.append(pos)
        pos += (int(n) + align - 1) // align * align
    return offs, pos


def serve_recipe(seed: int, nreq: int, nkeys: int = 10000, median: int = 256 << 10,
                 sigma: float = 1.5, lo: int = 4 << 10, hi: int = 64 << 20):
    """Serving workload: sizes log-normal (median, sigma) clamped to [lo, hi]
    and rounded down to 8 bytes; key index uniform over ``nkeys``; direction
    Bernoulli(0.5); unit-rate exponential inter-arrival gaps (scale by 1/rate).
    Normal deviates use the Box-Muller transform on pairs of uniforms."""
    u = uniforms(seed, 5 * nreq)
    u1 = np.maximum(u[:nreq], 1e-300)
    u2 = u[nreq:2 * nreq]
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    sizes = np.exp(np.log(median) + sigma * z)
    sizes = np.clip(sizes, lo, hi)
    sizes = (np.floor(sizes / 8.0) * 8).astype(np.int64)
    key_idx = np.minimum((u[2 * nreq:3 * nreq] * nkeys).astype(np.int64), nkeys - 1)
    decrypt = u[3 * nreq:4 * nreq] < 0.5
    gaps = -np.log(np.maximum(1.0 - u[4 * nreq:5 * nreq], 1e-300))
    return sizes, key_idx, decrypt, gaps
