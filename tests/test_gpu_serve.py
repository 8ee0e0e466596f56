"""The continuous-batching server: every request's bytes equal the
single-buffer call's (alone vs in the mix), the admission budget holds,
failures injected on the host complete with an error status and leave the
server usable, and the native arrival driver returns sane latencies."""
import numpy as np
import pytest

import oracle
from paper_1305_4376_gb300 import des3, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_4376_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    des3.lib()


def _workload(seed, n, max_bytes, nkeys):
    w = inputs.splitmix64(seed, 0, 4 * n)
    sizes = [8 * int(1 + w[i] % (max_bytes // 8)) for i in range(n)]
    offs, pos = [], 0
    for sz in sizes:
        offs.append(pos)
        pos += (sz + 255) // 256 * 256
    src = inputs.splitmix64_torch(seed + 1, 0, pos // 8 + 32, "cuda").view(torch.uint8)
    keys = inputs.key_triples(seed + 2, nkeys)
    kidx = [int(w[n + i] % nkeys) for i in range(n)]
    dec = [bool(w[2 * n + i] & 1) for i in range(n)]
    return src, offs, sizes, keys, kidx, dec


def _expected(src, offs, sizes, kss, kidx, dec):
    ref = torch.zeros_like(src)
    for o, n, k, d in zip(offs, sizes, kidx, dec):
        des3.des3_ecb_crypt_ex(kss[k], src[o:o + n], ref[o:o + n], n, d, "auto")
    torch.cuda.synchronize()
    return ref


def test_requests_in_the_mix_equal_alone():
    src, offs, sizes, keys, kidx, dec = _workload(7001, 300, 1 << 20, 9)
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=64 << 20, nstreams=4, max_batch_requests=64, key_capacity=16)
    first = srv.add_keys(kss)
    out = torch.zeros_like(src)
    tickets = {}
    for i, (o, n, k, d) in enumerate(zip(offs, sizes, kidx, dec)):
        tickets[srv.submit(src[o:o + n], out[o:o + n], n, first + k, d, tag=i)] = i
    srv.drain(60000)
    done = srv.poll(1000)
    assert len(done) == len(sizes)
    assert all(c["status"] == des3.DES3_OK for c in done)
    assert {c["ticket"] for c in done} == set(tickets)
    assert all(c["tag"] == tickets[c["ticket"]] for c in done)
    assert max(c["batch_size"] for c in done) >= 1
    ref = _expected(src, offs, sizes, kss, kidx, dec)
    assert torch.equal(out, ref)
    i = 17
    o, n = offs[i], sizes[i]
    assert np.array_equal(out[o:o + n].cpu().numpy(), oracle.tdes_ecb(keys[kidx[i]], src[o:o + n].cpu().numpy(), dec[i]))
    st = srv.stats()
    assert st["completed"] == len(sizes) and st["failed"] == 0 and st["inflight_requests"] == 0
    assert st["bytes_completed"] == sum(sizes)
    srv.close()


def test_admission_budget_and_limits():
    src, offs, sizes, keys, kidx, dec = _workload(7101, 40, 1 << 19, 2)
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=1 << 20, max_inflight=3, nstreams=2, max_batch_requests=8, key_capacity=2)
    first = srv.add_keys(kss)
    out = torch.zeros_like(src)
    with pytest.raises(des3.Des3Error) as e:
        srv.submit(src[:2 << 20], out[:2 << 20], 2 << 20, first, False)  # larger than the budget
    assert e.value.code == des3.DES3_EINVAL
    with pytest.raises(des3.Des3Error):
        srv.submit(src[:8], out[:8], 8, first + 5, False)  # unknown key
    for o, n, k, d in zip(offs, sizes, kidx, dec):
        srv.submit(src[o:o + n], out[o:o + n], n, first + k, d)
    srv.drain(60000)
    done = srv.poll(100)
    assert len(done) == len(sizes) and all(c["status"] == 0 for c in done)
    assert max(c["batch_size"] for c in done) <= 3
    assert torch.equal(out, _expected(src, offs, sizes, kss, kidx, dec))
    assert srv.stats()["inflight_bytes"] == 0
    with pytest.raises(des3.Des3Error):
        des3.Server(key_capacity=1).add_keys(kss)  # cache full
    srv.close()


def test_failure_injected_on_the_host_completes_with_error_and_recovers():
    src, offs, sizes, keys, kidx, dec = _workload(7201, 30, 1 << 16, 3)
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=1 << 30, nstreams=1, max_batch_requests=1, key_capacity=4, fault_every=3)
    first = srv.add_keys(kss)
    out = torch.zeros_like(src)
    for i, (o, n, k, d) in enumerate(zip(offs, sizes, kidx, dec)):
        srv.submit(src[o:o + n], out[o:o + n], n, first + k, d, tag=i)
    srv.drain(60000)
    done = srv.poll(100)
    assert len(done) == len(sizes)
    failed = [c for c in done if c["status"] != des3.DES3_OK]
    assert len(failed) == len(sizes) // 3
    assert all(c["status"] == des3.DES3_ECUDA for c in failed)
    st = srv.stats()
    assert st["failed"] == len(failed) and st["inflight_bytes"] == 0 and st["inflight_requests"] == 0
    ref = _expected(src, offs, sizes, kss, kidx, dec)
    bad = {c["tag"] for c in failed}
    for i, (o, n) in enumerate(zip(offs, sizes)):
        if i not in bad:
            assert torch.equal(out[o:o + n], ref[o:o + n])
    srv.close()


def test_failure_at_completion_is_reported_per_request_and_recovers():
    """The completion-stage hook lets every third batch's kernel run and then
    reports the batch failed, the path an error raised on the device takes:
    each of its requests completes with DES3_ECUDA, the budget is released,
    and the server goes on serving correct results afterwards."""
    src, offs, sizes, keys, kidx, dec = _workload(7251, 30, 1 << 16, 3)
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=1 << 30, nstreams=1, max_batch_requests=1, key_capacity=4, fault_every=3,
                      fault_stage=des3.DES3_FAULT_AT_COMPLETION)
    first = srv.add_keys(kss)
    out = torch.zeros_like(src)
    for i, (o, n, k, d) in enumerate(zip(offs, sizes, kidx, dec)):
        srv.submit(src[o:o + n], out[o:o + n], n, first + k, d, tag=i)
    srv.drain(60000)
    done = srv.poll(100)
    assert len(done) == len(sizes)
    failed = [c for c in done if c["status"] != des3.DES3_OK]
    assert len(failed) == len(sizes) // 3
    assert all(c["status"] == des3.DES3_ECUDA and c["batch_size"] == 1 for c in failed)
    st = srv.stats()
    assert st["failed"] == len(failed) and st["inflight_bytes"] == 0 and st["inflight_requests"] == 0
    ref = _expected(src, offs, sizes, kss, kidx, dec)
    # the kernels of the failed batches ran too: every request's bytes are right
    assert torch.equal(out, ref)
    # still serving: a second round, failures again exactly every third batch
    out.zero_()
    for i, (o, n, k, d) in enumerate(zip(offs, sizes, kidx, dec)):
        srv.submit(src[o:o + n], out[o:o + n], n, first + k, d, tag=100 + i)
    srv.drain(60000)
    done2 = srv.poll(100)
    assert len(done2) == len(sizes)
    assert sum(c["status"] != des3.DES3_OK for c in done2) == len(sizes) // 3
    assert all(c["latency_s"] > 0 for c in done + done2)
    assert torch.equal(out, ref)
    srv.close()


def test_replay_driver_latencies():
    src, offs, sizes, keys, kidx, dec = _workload(7301, 500, 1 << 18, 5)
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=256 << 20, nstreams=4, key_capacity=8)
    first = srv.add_keys(kss)
    out = torch.zeros_like(src)
    reqs = (des3.des3_request_t * len(sizes))()
    for i, (o, n, k, d) in enumerate(zip(offs, sizes, kidx, dec)):
        reqs[i] = des3.Server.request(src[o:o + n], out[o:o + n], n, first + k, d, i)
    gaps = inputs.serve_recipe(7302, len(sizes))[3]
    arrival = np.cumsum(gaps) / 20000.0  # 20k requests/s
    rc, lat = srv.replay(reqs, arrival, 120000)
    assert rc == des3.DES3_OK
    assert (lat > 0).all() and (lat < 10).all()
    assert torch.equal(out, _expected(src, offs, sizes, kss, kidx, dec))
    srv.close()


def test_serving_workload_sample_alone_equals_in_the_mix():
    """The serving workload's distributions at full key-cache size: 10000
    cached key triples, log-normal sizes (median 256 KiB, sigma 1.5, clamped
    to 4 KiB..64 MiB), mixed directions, Poisson arrivals replayed at about
    twice the rate the GPU can serve (so batches grow large).  2000 requests
    with their own output buffers: every output equals the single-buffer
    call on the same input, and every output byte, hashed in request order,
    equals the oracle's (tests/golden/oracle_serve_digests.json, written by
    make_serve_digests.py from oracle/ alone)."""
    n = 2000
    sizes, kidx, dec, gaps = inputs.serve_recipe(inputs.data_seed(5), n)
    keys = inputs.key_triples(inputs.key_seed(5), 10000)
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=16 << 30, nstreams=4, max_batch_requests=4096, key_capacity=10000)
    first = srv.add_keys(kss)
    offs, pos = [], 0
    for sz in sizes:
        offs.append(pos)
        pos += (int(sz) + 255) // 256 * 256
    src = inputs.splitmix64_torch(inputs.data_seed(5) + 7, 0, pos // 8 + 32, "cuda").view(torch.uint8)
    out = torch.zeros_like(src)
    reqs = (des3.des3_request_t * n)()
    for i, (o, sz) in enumerate(zip(offs, sizes)):
        sz = int(sz)
        reqs[i] = des3.Server.request(src[o:o + sz], out[o:o + sz], sz, first + int(kidx[i]), bool(dec[i]), i)
    rate = 2 * 400e9 / float(sizes.mean())  # about twice the plain kernel's request rate
    rc, lat = srv.replay(reqs, np.cumsum(gaps) / rate, 300000)
    assert rc == des3.DES3_OK and (lat > 0).all()
    st = srv.stats()
    assert st["launches"] < n  # requests were batched together
    srv.close()
    ref = torch.zeros_like(src)
    for i, (o, sz) in enumerate(zip(offs, sizes)):
        sz = int(sz)
        des3.des3_ecb_crypt_ex(kss[int(kidx[i])], src[o:o + sz], ref[o:o + sz], sz, bool(dec[i]), "auto")
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    i = int(np.argmax(sizes))
    o, sz = offs[i], int(sizes[i])
    blocks = np.array([0, sz // 8 - 1], dtype=np.int64)
    t = torch.from_numpy(blocks + o // 8).cuda()
    plain = src.view(torch.int64)[t].cpu().numpy().view(np.uint8)
    got = out.view(torch.int64)[t].cpu().numpy().view(np.uint8)
    assert np.array_equal(got, oracle.tdes_ecb(keys[int(kidx[i])], plain, bool(dec[i])))
    # every byte against the oracle's digests of the same sample
    import hashlib
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_serve_digests.json")))
    assert gold["nreq"] == n and gold["total_bytes"] == int(sizes.sum()) and gold["arena_bytes"] >= pos
    host_in, host_out = src.cpu().numpy(), out.cpu().numpy()
    h_in, h_out, g = hashlib.sha256(), hashlib.sha256(), hashlib.sha256()
    groups = []
    for i, (o, sz) in enumerate(zip(offs, sizes)):
        sz = int(sz)
        h_in.update(host_in[o:o + sz])
        h_out.update(host_out[o:o + sz])
        g.update(host_out[o:o + sz])
        if (i + 1) % gold["group_requests"] == 0 or i + 1 == n:
            groups.append(g.hexdigest())
            g = hashlib.sha256()
    assert h_in.hexdigest() == gold["sha256_in"]
    bad = [k for k, (a, b) in enumerate(zip(groups, gold["sha256_out_groups"])) if a != b]
    assert not bad, "request groups differing from the oracle: %s" % bad
    assert h_out.hexdigest() == gold["sha256_out"]


def test_concurrent_add_keys_get_disjoint_ids_and_keep_the_device():
    """Key uploads from several threads at once: every call gets its own id
    range and each id encrypts with its own key."""
    import threading
    keys = [inputs.key_triple(7401 + i) for i in range(64)]
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=64 << 20, nstreams=2, key_capacity=64)
    firsts = [None] * 8
    dev_before = torch.cuda.current_device()

    def add(t):
        firsts[t] = srv.add_keys(kss[8 * t:8 * t + 8])

    th = [threading.Thread(target=add, args=(t,)) for t in range(8)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert sorted(firsts) == list(range(0, 64, 8))
    assert torch.cuda.current_device() == dev_before
    data = inputs.data_bytes(7450, 8 * 1000)
    src = torch.from_numpy(data).cuda()
    outs = []
    for t in range(8):
        for j in (0, 7):
            out = torch.zeros_like(src)
            srv.submit(src, out, src.numel(), firsts[t] + j, False, tag=8 * t + j)
            outs.append((8 * t + j, out))
    srv.drain(60000)
    assert all(c["status"] == des3.DES3_OK for c in srv.poll())
    for k, out in outs:
        assert np.array_equal(out.cpu().numpy(), oracle.tdes_ecb(keys[k], data))
    srv.close()


def test_replay_leaves_other_completions_for_poll():
    src, offs, sizes, keys, kidx, dec = _workload(7501, 20, 1 << 16, 2)
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=64 << 20, nstreams=2, key_capacity=4)
    first = srv.add_keys(kss)
    out = torch.zeros_like(src)
    t0 = srv.submit(src[offs[0]:offs[0] + sizes[0]], out[offs[0]:offs[0] + sizes[0]], sizes[0],
                    first + kidx[0], dec[0], tag=999)
    reqs = (des3.des3_request_t * (len(sizes) - 1))()
    for i in range(1, len(sizes)):
        o, n = offs[i], sizes[i]
        reqs[i - 1] = des3.Server.request(src[o:o + n], out[o:o + n], n, first + kidx[i], dec[i], i)
    rc, lat = srv.replay(reqs, np.linspace(0, 1e-3, len(sizes) - 1), 60000)
    assert rc == des3.DES3_OK and (lat > 0).all()
    srv.drain(60000)
    left = srv.poll()
    assert [c["ticket"] for c in left] == [t0] and left[0]["tag"] == 999 and left[0]["status"] == des3.DES3_OK
    assert torch.equal(out, _expected(src, offs, sizes, kss, kidx, dec))
    srv.close()


def test_small_batches_run_on_the_table_kernel_and_equal_single_calls():
    """With the built-in (GB300) tuning tables, a batch of up to 1 MiB runs on
    the batched table kernel: requests of up to 16 KiB, each drained before
    the next, all go to the table kernel (the server's table_launches counts
    every launch); alone, requests of 8 and 6 MiB run bitsliced and requests
    of 512 and 64 KiB on the table kernel.  Every output equals the
    single-buffer call's."""
    from paper_1305_4376_gb300 import autotune
    autotune.reset()
    src, offs, sizes, keys, kidx, dec = _workload(7601, 60, 16 << 10, 5)
    kss = [des3.des3_key_schedule(k) for k in keys]
    srv = des3.Server(budget_bytes=256 << 20, nstreams=2, max_batch_requests=64, key_capacity=8)
    first = srv.add_keys(kss)
    out = torch.zeros_like(src)
    for o, n, k, d in zip(offs, sizes, kidx, dec):
        srv.submit(src[o:o + n], out[o:o + n], n, first + k, d)
        srv.drain(10000)
    done = srv.poll(1000)
    assert len(done) == len(sizes) and all(c["status"] == des3.DES3_OK for c in done)
    st = srv.stats()
    assert st["launches"] == len(sizes) and st["table_launches"] == st["launches"], st
    assert torch.equal(out, _expected(src, offs, sizes, kss, kidx, dec))
    i = 3
    o, n = offs[i], sizes[i]
    assert np.array_equal(out[o:o + n].cpu().numpy(), oracle.tdes_ecb(keys[kidx[i]], src[o:o + n].cpu().numpy(), dec[i]))

    # alone, 8 MiB and 6 MiB run bitsliced and 512 KiB and 64 KiB on the table kernel
    sizes2 = [8 << 20, 512 << 10, 6 << 20, 64 << 10]
    offs2 = [0, 8 << 20, (8 << 20) + (512 << 10), (14 << 20) + (512 << 10)]
    src2 = inputs.splitmix64_torch(7603, 0, (15 << 20) // 8, "cuda").view(torch.uint8)
    out2 = torch.zeros_like(src2)
    base = srv.stats()
    for j, (o, n) in enumerate(zip(offs2, sizes2)):
        srv.submit(src2[o:o + n], out2[o:o + n], n, first + j % 5, j % 2 == 1)
        srv.drain(30000)
    assert len(srv.poll(1000)) == len(sizes2)
    st = srv.stats()
    assert st["launches"] - base["launches"] == 4 and st["table_launches"] - base["table_launches"] == 2, (st, base)
    ref2 = torch.zeros_like(src2)
    for j, (o, n) in enumerate(zip(offs2, sizes2)):
        des3.des3_ecb_crypt_ex(kss[j % 5], src2[o:o + n], ref2[o:o + n], n, j % 2 == 1, "bitslice")
    torch.cuda.synchronize()
    assert torch.equal(out2, ref2)
    srv.close()
