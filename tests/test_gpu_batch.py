"""The batched path (many buffers, a key triple each, mixed directions, one
persistent launch or a CUDA-graph plan) against the oracle and against the
single-buffer calls: every job's bytes are identical alone and in the mix."""
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


def _arena(sizes, seed, align=256, offset=0):
    """One device arena holding every job's input at `align`-aligned offsets
    (+ `offset` bytes), filled with seeded bytes."""
    offs = []
    pos = 0
    for n in sizes:
        pos = (pos + align - 1) // align * align
        offs.append(pos + offset)
        pos += n + offset
    total = (pos + 4095) // 4096 * 4096 + 4096
    words = inputs.splitmix64_torch(seed, 0, total // 8, "cuda")
    return words.view(torch.uint8), offs


def _single(ks, src, dst, decrypt, kernel="auto"):
    des3.des3_ecb_crypt_ex(ks, src, dst, src.numel(), decrypt, kernel)


def test_mixed_small_batch_matches_oracle_and_single_calls():
    rng_sizes = inputs.splitmix64(31, 0, 60)
    sizes = [int(8 * (v % 12000)) for v in rng_sizes]
    sizes[3] = 0
    sizes[7] = 8
    sizes[11] = 8 * 1024
    sizes[12] = 8 * 1025
    keys = inputs.key_triples(32, 7)
    kss = [des3.des3_key_schedule(k) for k in keys]
    karr = des3.make_keys(kss)
    src, offs = _arena(sizes, 33)
    out = torch.zeros_like(src)
    alone = torch.zeros_like(src)
    spec = []
    for i, (n, o) in enumerate(zip(sizes, offs)):
        k = i % 7
        dec = bool(i % 3 == 1)
        inplace = i % 5 == 4
        s = src[o:o + n]
        d = s if inplace else out[o:o + n]
        if inplace:
            # keep a copy of the input for the checks; the in-place job overwrites src
            pass
        spec.append((s, d, n, k, dec, inplace))
    src_copy = src.clone()
    jobs = des3.make_jobs([(s, d, n, k, dec) for (s, d, n, k, dec, _) in spec])
    des3.des3_ecb_batch(karr, jobs)
    for (s, d, n, k, dec, inplace), o in zip(spec, offs):
        if n:
            _single(kss[k], src_copy[o:o + n], alone[o:o + n], dec)
    torch.cuda.synchronize()
    for (s, d, n, k, dec, inplace), o in zip(spec, offs):
        got = d.cpu().numpy()
        want = oracle.tdes_ecb(keys[k], src_copy[o:o + n].cpu().numpy(), dec)
        assert np.array_equal(got, want), (n, k, dec, inplace)
        assert torch.equal(d, alone[o:o + n])


def test_plan_graph_replay_matches_one_shot():
    sizes = [8 * 1024 * 7 + 8 * 13, 512, 8 * 333, 1 << 20]
    keys = inputs.key_triples(40, 3)
    karr = des3.make_keys([des3.des3_key_schedule(k) for k in keys])
    src, offs = _arena(sizes, 41)
    a = torch.zeros_like(src)
    b = torch.zeros_like(src)
    ja = des3.make_jobs([(src[o:o + n], a[o:o + n], n, i % 3, i % 2 == 0) for i, (n, o) in enumerate(zip(sizes, offs))])
    jb = des3.make_jobs([(src[o:o + n], b[o:o + n], n, i % 3, i % 2 == 0) for i, (n, o) in enumerate(zip(sizes, offs))])
    des3.des3_ecb_batch(karr, ja)
    plan = des3.BatchPlan(karr, jb)
    total, tiles = plan.info()
    assert total == sum(sizes)
    assert tiles == sum((n // 8 + 1023) // 1024 for n in sizes)
    plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    b.zero_()
    plan.launch()
    plan.launch()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    plan.close()


def test_unaligned_jobs():
    sizes = [8 * 5000, 8 * 1024, 8 * 77]
    keys = inputs.key_triples(50, 2)
    kss = [des3.des3_key_schedule(k) for k in keys]
    src, offs = _arena(sizes, 51, offset=8)
    out = torch.zeros_like(src)
    jobs = des3.make_jobs([(src[o:o + n], out[o + 8:o + 8 + n] if i == 1 else out[o:o + n], n, i % 2, i == 2)
                           for i, (n, o) in enumerate(zip(sizes, offs))])
    des3.des3_ecb_batch(des3.make_keys(kss), jobs)
    torch.cuda.synchronize()
    for i, (n, o) in enumerate(zip(sizes, offs)):
        d = out[o + 8:o + 8 + n] if i == 1 else out[o:o + n]
        want = oracle.tdes_ecb(keys[i % 2], src[o:o + n].cpu().numpy(), i == 2)
        assert np.array_equal(d.cpu().numpy(), want)


def test_batched_workload_4096_buffers():
    """4096 buffers, sizes log-uniform 512 B .. 16 MiB (~6 GiB), a 3-key
    triple each, mixed directions, as one graph-captured persistent launch.
    Every byte must equal the single-buffer calls' output; the oracle checks
    the first, last and 30 seeded blocks of every job."""
    sizes, dec = inputs.batch_recipe(inputs.data_seed(4))
    sizes = [int(x) for x in sizes]
    keys = inputs.key_triples(inputs.key_seed(4), len(sizes))
    kss = [des3.des3_key_schedule(k) for k in keys]
    karr = des3.make_keys(kss)
    src, offs = _arena(sizes, inputs.data_seed(4))
    out = torch.zeros_like(src)
    jobs = des3.make_jobs([(src[o:o + n], out[o:o + n], n, i, bool(dec[i])) for i, (n, o) in enumerate(zip(sizes, offs))])
    plan = des3.BatchPlan(karr, jobs)
    plan.launch()
    torch.cuda.synchronize()
    alone = torch.zeros_like(src)
    for i, (n, o) in enumerate(zip(sizes, offs)):
        _single(kss[i], src[o:o + n], alone[o:o + n], bool(dec[i]))
    torch.cuda.synchronize()
    assert torch.equal(out, alone)
    # oracle on sampled blocks of every job
    src64 = src.view(torch.int64)
    out64 = out.view(torch.int64)
    picks = inputs.splitmix64(77, 0, 30 * len(sizes))
    for i, (n, o) in enumerate(zip(sizes, offs)):
        nb = n // 8
        idx = sorted(set([0, nb - 1] + [int(v % nb) for v in picks[30 * i:30 * i + 30]]))
        t = torch.tensor([o // 8 + j for j in idx], device="cuda")
        plain = src64[t].cpu().numpy().view(np.uint8)
        got = out64[t].cpu().numpy().view(np.uint8)
        assert np.array_equal(got, oracle.tdes_ecb(keys[i], plain, bool(dec[i]))), i
    plan.close()


def _batch_shapes():
    from paper_1305_4376_gb300 import autotune
    return autotune.BATCH_CANDIDATES


@pytest.mark.parametrize("kernel,threads,ctas", _batch_shapes())
def test_every_tunable_batch_shape_is_bit_exact(kernel, threads, ctas):
    from paper_1305_4376_gb300 import autotune
    sizes = [8 * 1024 * 5 + 8 * 3, 4096, 8 * 77, 1 << 20]
    keys = inputs.key_triples(60, 2)
    kss = [des3.des3_key_schedule(k) for k in keys]
    src, offs = _arena(sizes, 61)
    ref = torch.zeros_like(src)
    out = torch.zeros_like(src)
    spec = [(i % 2, i == 1) for i in range(len(sizes))]
    for (o, n), (k, d) in zip(zip(offs, sizes), spec):
        _single(kss[k], src[o:o + n], ref[o:o + n], d)
    try:
        autotune.set_entries(des3.DES3_TUNE_BATCH, [(c, kernel, threads, ctas) for c in range(40)])
        des3.des3_ecb_batch(des3.make_keys(kss), des3.make_jobs(
            [(src[o:o + n], out[o:o + n], n, k, d) for (o, n), (k, d) in zip(zip(offs, sizes), spec)]))
        torch.cuda.synchronize()
    finally:
        autotune.reset()
    assert torch.equal(out, ref)


def test_batched_workload_whole_output_equals_the_oracle():
    """The batched workload exactly as the benchmark runs it (4096 buffers in
    one arena, the graph-captured plan): every output byte, hashed in job
    order, against the oracle's digest of the whole workload
    (tests/golden/oracle_batch_digests.json, written by
    make_batch_digests.py from oracle/ alone)."""
    import hashlib
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oracle_batch_digests.json")))
    seed = inputs.data_seed(4)
    sizes, dec = inputs.batch_recipe(seed)
    assert gold["data_seed"] == seed and gold["njobs"] == len(sizes) and gold["total_bytes"] == int(sizes.sum())
    keys = inputs.key_triples(inputs.key_seed(4), len(sizes))
    karr = des3.make_keys([des3.des3_key_schedule(k) for k in keys])
    offs, arena_bytes = inputs.arena_offsets(sizes)
    assert arena_bytes == gold["arena_bytes"]
    src = inputs.splitmix64_torch(seed, 0, arena_bytes // 8 + 32, "cuda").view(torch.uint8)
    out = torch.zeros_like(src)
    jobs = des3.make_jobs([(src[o:o + int(n)], out[o:o + int(n)], int(n), i, bool(dec[i]))
                           for i, (n, o) in enumerate(zip(sizes, offs))])
    plan = des3.BatchPlan(karr, jobs)
    plan.launch()
    torch.cuda.synchronize()
    host_in = src.cpu().numpy()
    host_out = out.cpu().numpy()
    h_in, h_out = hashlib.sha256(), hashlib.sha256()
    groups = []
    g = hashlib.sha256()
    for i, (n, o) in enumerate(zip(sizes, offs)):
        h_in.update(host_in[o:o + int(n)])
        h_out.update(host_out[o:o + int(n)])
        g.update(host_out[o:o + int(n)])
        if (i + 1) % gold["group_jobs"] == 0 or i + 1 == len(sizes):
            groups.append(g.hexdigest())
            g = hashlib.sha256()
    assert h_in.hexdigest() == gold["sha256_in"]
    bad = [k for k, (a, b) in enumerate(zip(groups, gold["sha256_out_groups"])) if a != b]
    assert not bad, "job groups differing from the oracle: %s" % bad
    assert h_out.hexdigest() == gold["sha256_out"]
    plan.close()


@pytest.mark.parametrize("threads,ctas", [(384, 3), (64, 1)])
def test_table_kernel_batch_ragged_tiny_zero_and_in_place_jobs(threads, ctas):
    """The batched table kernel on jobs around its 64-block segment (63, 64,
    65 blocks), single blocks, zero-size jobs, multi-segment and multi-tile
    jobs, unaligned and in-place jobs, mixed keys and directions: every job
    equals the single-buffer call and the oracle, through the one-shot call
    and a graph plan replayed twice."""
    from paper_1305_4376_gb300 import autotune
    sizes = [8 * 63, 8 * 64, 8 * 65, 8, 0, 8 * 1000, 0, 8 * 4097, 8 * 127, 8 * 129, 8 * 3, 8 * 20000]
    keys = inputs.key_triples(70, 5)
    kss = [des3.des3_key_schedule(k) for k in keys]
    src, offs = _arena(sizes, 71, offset=8)
    spec = [(i % 5, i % 3 == 1, i % 4 == 2) for i in range(len(sizes))]  # key, decrypt, in place
    ref = src.clone()
    for (o, n), (k, d, inpl) in zip(zip(offs, sizes), spec):
        if n:
            _single(kss[k], src[o:o + n], ref[o:o + n], d, "bitslice")
    torch.cuda.synchronize()
    try:
        autotune.set_entries(des3.DES3_TUNE_BATCH, [(c, des3.DES3_KERNEL_SPTABLE, threads, ctas) for c in range(40)])
        for use_plan in (False, True):
            a = src.clone()
            b = src.clone()
            jobs = des3.make_jobs([(a[o:o + n], (a if inpl else b)[o:o + n], n, k, d)
                                   for (o, n), (k, d, inpl) in zip(zip(offs, sizes), spec)])
            if use_plan:
                plan = des3.BatchPlan(des3.make_keys(kss), jobs)
                plan.launch()
                torch.cuda.synchronize()
                # a replay of an in-place plan transforms those jobs again: compare after one launch
                plan.close()
            else:
                des3.des3_ecb_batch(des3.make_keys(kss), jobs)
            torch.cuda.synchronize()
            for (o, n), (k, d, inpl) in zip(zip(offs, sizes), spec):
                got = (a if inpl else b)[o:o + n]
                assert torch.equal(got, ref[o:o + n]), (n, k, d, inpl, use_plan)
                if n:
                    want = oracle.tdes_ecb(keys[k], src[o:o + n].cpu().numpy(), d)
                    assert np.array_equal(got.cpu().numpy(), want), (n, k, d, inpl, use_plan)
    finally:
        autotune.reset()


def test_table_kernel_batch_of_many_tiny_jobs_and_explicit_plan_kernel():
    """2000 jobs of 8 to 1024 bytes with 64 keys: the batched table kernel
    (chosen explicitly for the plan) equals the bitsliced batch on every
    byte, and the plan replays."""
    w = inputs.splitmix64(81, 0, 4000)
    sizes = [8 * int(1 + v % 128) for v in w[:2000]]
    keys = inputs.key_triples(82, 64)
    karr = des3.make_keys([des3.des3_key_schedule(k) for k in keys])
    src, offs = _arena(sizes, 83)
    a = torch.zeros_like(src)
    b = torch.zeros_like(src)
    spec = [(int(w[2000 + i] % 64), bool(w[2000 + i] & 64)) for i in range(len(sizes))]
    ja = des3.make_jobs([(src[o:o + n], a[o:o + n], n, k, d) for (o, n), (k, d) in zip(zip(offs, sizes), spec)])
    jb = des3.make_jobs([(src[o:o + n], b[o:o + n], n, k, d) for (o, n), (k, d) in zip(zip(offs, sizes), spec)])
    pa = des3.BatchPlan(karr, ja, kernel="bitslice")
    pb = des3.BatchPlan(karr, jb, kernel="sptable")
    pa.launch()
    pb.launch()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    b.zero_()
    pb.launch()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    i = 17
    o, n = offs[i], sizes[i]
    k, d = spec[i]
    assert np.array_equal(b[o:o + n].cpu().numpy(), oracle.tdes_ecb(keys[k], src[o:o + n].cpu().numpy(), d))
    pa.close()
    pb.close()


@pytest.mark.parametrize("kernel", [des3.DES3_KERNEL_BITSLICE, des3.DES3_KERNEL_SPTABLE])
def test_one_shot_batch_over_a_large_key_table_uses_the_named_keys(kernel):
    """The one-shot call expands only the keys its jobs name and renumbers
    them: with 3000 keys of which jobs name a scattered, repeated few (the
    first and last index among them, zero-size jobs naming keys no other job
    uses), every job equals the single-buffer call under its own key, in
    both kernels, and the oracle checks two jobs."""
    from paper_1305_4376_gb300 import autotune
    keys = inputs.key_triples(90, 3000)
    kss = [des3.des3_key_schedule(k) for k in keys]
    karr = des3.make_keys(kss)
    names = [2999, 0, 1234, 2999, 7, 1234, 0, 2500, 7, 2999, 42, 1500]
    sizes = [8 * (97 * i + 5) for i in range(len(names))] + [0, 0]
    names += [11, 2222]  # zero-size jobs
    src, offs = _arena(sizes, 91)
    out = torch.zeros_like(src)
    ref = torch.zeros_like(src)
    for i, (o, n) in enumerate(zip(offs, sizes)):
        if n:
            _single(kss[names[i]], src[o:o + n], ref[o:o + n], i % 2 == 1, "bitslice")
    jobs = des3.make_jobs([(src[o:o + n], out[o:o + n], n, names[i], i % 2 == 1)
                           for i, (o, n) in enumerate(zip(offs, sizes))])
    try:
        autotune.set_entries(des3.DES3_TUNE_BATCH, [(c, kernel, 384, 3 if kernel == des3.DES3_KERNEL_SPTABLE else 1)
                                                    for c in range(40)])
        des3.des3_ecb_batch(karr, jobs)
        torch.cuda.synchronize()
    finally:
        autotune.reset()
    assert torch.equal(out, ref)
    for i in (0, 10):
        o, n = offs[i], sizes[i]
        want = oracle.tdes_ecb(keys[names[i]], src[o:o + n].cpu().numpy(), i % 2 == 1)
        assert np.array_equal(out[o:o + n].cpu().numpy(), want)


def test_auto_choice_takes_the_table_kernel_for_sparse_tiles():
    """With every batch size class set to the bitsliced kernel, a plan in
    AUTO still takes the table kernel (default shape 384 x 3) for 4096 jobs
    of 64 blocks, which fill one sixteenth of their tiles, and keeps the
    bitsliced kernel for 4096 jobs of one full tile each and for 100 small
    jobs (below one tile per warp of the bitsliced grid, where the table
    decides).  The one-shot call makes the same choice, and every output
    equals the single-buffer calls."""
    from paper_1305_4376_gb300 import autotune
    keys = inputs.key_triples(95, 16)
    kss = [des3.des3_key_schedule(k) for k in keys]
    karr = des3.make_keys(kss)
    cases = [(4096, 512, des3.DES3_KERNEL_SPTABLE, 384, 3), (4096, 8192, des3.DES3_KERNEL_BITSLICE, 384, 1),
             (100, 512, des3.DES3_KERNEL_BITSLICE, 384, 1)]
    try:
        autotune.set_entries(des3.DES3_TUNE_BATCH, [(c, des3.DES3_KERNEL_BITSLICE, 384, 1) for c in range(40)])
        for njobs, size, want_kernel, want_threads, want_ctas in cases:
            sizes = [size] * njobs
            src, offs = _arena(sizes, 96 + njobs + size)
            ref = torch.zeros_like(src)
            for i, o in enumerate(offs):
                _single(kss[i % 16], src[o:o + size], ref[o:o + size], i % 3 == 0, "bitslice")
            for use_plan in (True, False):
                out = torch.zeros_like(src)
                jobs = des3.make_jobs([(src[o:o + size], out[o:o + size], size, i % 16, i % 3 == 0)
                                       for i, o in enumerate(offs)])
                if use_plan:
                    plan = des3.BatchPlan(karr, jobs)
                    assert plan.kernel() == (want_kernel, want_threads, want_ctas), (njobs, size)
                    plan.launch()
                    torch.cuda.synchronize()
                    plan.close()
                else:
                    des3.des3_ecb_batch(karr, jobs)
                    torch.cuda.synchronize()
                assert torch.equal(out, ref), (njobs, size, use_plan)
            o = offs[5]
            want = oracle.tdes_ecb(keys[5], src[o:o + size].cpu().numpy(), False)
            assert np.array_equal(ref[o:o + size].cpu().numpy(), want)
    finally:
        autotune.reset()


def test_plan_reports_an_explicit_kernel_and_the_tables_shape():
    """An explicit kernel keeps the tuning table's shape when the table names
    it, else takes that kernel's default shape."""
    from paper_1305_4376_gb300 import autotune
    karr = des3.make_keys([des3.des3_key_schedule(k) for k in inputs.key_triples(97, 2)])
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    jobs = des3.make_jobs([(buf[:4096], buf[:4096], 4096, 0, False), (buf[8192:16384], buf[8192:16384], 8192, 1, True)])
    try:
        autotune.set_entries(des3.DES3_TUNE_BATCH, [(c, des3.DES3_KERNEL_SPTABLE, 128, 3) for c in range(40)])
        for kernel, want in (("auto", (des3.DES3_KERNEL_SPTABLE, 128, 3)), ("sptable", (des3.DES3_KERNEL_SPTABLE, 128, 3)),
                             ("bitslice", (des3.DES3_KERNEL_BITSLICE, 384, 1))):
            plan = des3.BatchPlan(karr, jobs, kernel=kernel)
            assert plan.kernel() == want, kernel
            plan.close()
        autotune.set_entries(des3.DES3_TUNE_BATCH, [(c, des3.DES3_KERNEL_BITSLICE, 128, 2) for c in range(40)])
        for kernel, want in (("auto", (des3.DES3_KERNEL_BITSLICE, 128, 2)), ("sptable", (des3.DES3_KERNEL_SPTABLE, 384, 3))):
            plan = des3.BatchPlan(karr, jobs, kernel=kernel)
            assert plan.kernel() == want, kernel
            plan.close()
    finally:
        autotune.reset()


def test_host_choice_query_matches_the_plans_choice():
    """des3_batch_choose (host only, given the SM count) names the same kernel
    and shape that a plan in AUTO captures, on job lists on both sides of the
    tuning table's classes and of the wave model's crossover."""
    from paper_1305_4376_gb300 import autotune
    autotune.reset()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    karr = des3.make_keys([des3.des3_key_schedule(k) for k in inputs.key_triples(98, 4)])
    buf = torch.zeros(64 << 20, dtype=torch.uint8, device="cuda")
    w = inputs.splitmix64(99, 0, 64)
    cases = [(1, 256 << 10), (16, 64 << 10), (4096, 512), (4096, 4096), (2000, 8192), (100, 1 << 16),
             (3000, 8 * int(1 + w[0] % 900))]
    for njobs, size in cases:
        pitch = (size + 255) // 256 * 256
        assert njobs * pitch <= buf.numel()
        jobs = des3.make_jobs([(buf[i * pitch:i * pitch + size], buf[i * pitch:i * pitch + size], size, i % 4,
                                bool(i & 1)) for i in range(njobs)])
        plan = des3.BatchPlan(karr, jobs)
        assert des3.des3_batch_choose(jobs, sms) == plan.kernel(), (njobs, size)
        plan.close()
