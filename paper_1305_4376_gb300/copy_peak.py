"""Host<->device copy bandwidth on this machine (the ceiling of des3_ecb_host).

Pinned 1 GiB buffers; H2D, D2H, both at once on two streams, and H2D in
64 MiB chunks.  The end-to-end benchmark copies every byte in and out, so
its throughput cannot exceed the bidirectional figure.

    python -m paper_1305_4376_gb300.copy_peak
"""
import torch, time
n = 1 << 30
h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
h2 = torch.empty(n, dtype=torch.uint8, pin_memory=True)
d = torch.empty(n, dtype=torch.uint8, device="cuda")
d2 = torch.empty(n, dtype=torch.uint8, device="cuda")
s1 = torch.cuda.Stream(); s2 = torch.cuda.Stream()
for name, fn in [("h2d", lambda: d.copy_(h, non_blocking=True)), ("d2h", lambda: h.copy_(d, non_blocking=True))]:
    fn(); torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(5): fn()
    torch.cuda.synchronize(); dt = time.perf_counter() - t
    print(name, "%.1f GB/s" % (5 * n / dt / 1e9))
# bidirectional on two streams
torch.cuda.synchronize(); t = time.perf_counter()
for _ in range(5):
    with torch.cuda.stream(s1): d.copy_(h, non_blocking=True)
    with torch.cuda.stream(s2): h2.copy_(d2, non_blocking=True)
torch.cuda.synchronize(); dt = time.perf_counter() - t
print("bidir each way %.1f GB/s" % (5 * n / dt / 1e9))
# chunked 64 MiB
c = 64 << 20
torch.cuda.synchronize(); t = time.perf_counter()
for off in range(0, n, c):
    d[off:off+c].copy_(h[off:off+c], non_blocking=True)
torch.cuda.synchronize(); dt = time.perf_counter() - t
print("h2d 64MiB chunks %.1f GB/s" % (n / dt / 1e9))
