"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every symbol include/des3.h declares, passes its self test, computes
the same key schedule as the oracle, and rejects bad arguments before it
touches the device."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1305_4376_gb300 import des3, inputs


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_4376_gb300 import build
    build.build()


def test_exports_every_declared_symbol():
    names = des3.exported_symbols()
    assert "des3_ecb_encrypt" in names and "des3_key_schedule" in names
    lib = des3.lib()
    for n in names:
        assert hasattr(lib, n), n


def test_self_test_passes():
    """S-box circuits (all 64 inputs), SP tables, IP/FP networks, and the
    bitsliced and table pipelines run on the host against each other."""
    des3.des3_self_test()


@pytest.mark.parametrize("keying", ["3key", "2key", "1key"])
def test_key_schedule_matches_oracle(keying):
    key = inputs.key_triple(4242, keying)
    ks = des3.des3_key_schedule(key)
    assert ks.magic == des3.DES3_KS_MAGIC
    k1, k2, k3 = (oracle.des_key_schedule(key[8 * i:8 * i + 8]) for i in range(3))
    enc = k1 + k2[::-1] + k3  # E_K1, D_K2, E_K3 (Sec. II.A)
    assert [ks.rk[0][r] for r in range(48)] == enc
    assert [ks.rk[1][r] for r in range(48)] == enc[::-1]


def test_key_schedule_ignores_parity():
    key = inputs.key_triple(17)
    a = des3.des3_key_schedule(key)
    b = des3.des3_key_schedule(bytes(x ^ 1 for x in key))
    assert bytes(a) == bytes(b)


def test_argument_errors_without_device():
    lib = des3.lib()
    ks = des3.des3_key_schedule(inputs.key_triple(3))
    bad = des3.des3_ks_t()
    fake = 1 << 40  # never dereferenced: validation fails first
    assert lib.des3_key_schedule(None, ctypes.byref(ks)) == des3.DES3_EINVAL
    assert lib.des3_ecb_crypt_ex(None, fake, fake, 64, 0, 0, None) == des3.DES3_EINVAL
    assert lib.des3_ecb_crypt_ex(ctypes.byref(bad), fake, fake, 64, 0, 0, None) == des3.DES3_EKEY
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), fake, fake, 12, 0, 0, None) == des3.DES3_EINVAL
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), fake + 4, fake + 4, 16, 0, 0, None) == des3.DES3_EINVAL
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), fake, fake + 8, 64, 0, 0, None) == des3.DES3_EINVAL
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), fake, fake, 64, 3, 0, None) == des3.DES3_EINVAL
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), fake, fake, 64, 0, 7, None) == des3.DES3_EINVAL
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), fake, fake, 0, 0, 0, None) == des3.DES3_OK
    assert lib.des3_ecb_host(ctypes.byref(ks), fake, fake, 64, 0, fake, 1024, None) == des3.DES3_EINVAL
    assert lib.des3_ecb_host(ctypes.byref(ks), fake, fake + 8, 64, 0, fake, 4 << 20, None) == des3.DES3_EINVAL
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -99):
        assert isinstance(des3.strerror(code), str)


def test_batch_validation_without_device():
    lib = des3.lib()
    keys = des3.make_keys([des3.des3_key_schedule(inputs.key_triple(i)) for i in range(2)])
    fake = 1 << 40
    ok = des3.make_jobs([(fake, fake + (1 << 20), 4096, 1, False)])
    bad_key = des3.make_jobs([(fake, fake + (1 << 20), 4096, 2, False)])
    bad_size = des3.make_jobs([(fake, fake + (1 << 20), 4090, 0, False)])
    overlap = des3.make_jobs([(fake, fake + 8, 4096, 0, True)])
    for jobs in (bad_key, bad_size, overlap):
        assert lib.des3_ecb_batch(keys, 2, jobs, 1, None) == des3.DES3_EINVAL
    badks = des3.make_keys([des3.des3_ks_t()])
    assert lib.des3_ecb_batch(badks, 1, des3.make_jobs([(fake, fake, 8, 0, False)]), 1, None) == des3.DES3_EKEY
    empty = des3.make_jobs([(fake, fake, 0, 0, False)])
    assert lib.des3_ecb_batch(keys, 2, empty, 1, None) == des3.DES3_OK
    assert ok[0].nbytes == 4096


def test_server_rejects_bad_config_without_device():
    lib = des3.lib()
    h = ctypes.c_void_p()
    good = dict(budget_bytes=1 << 20, max_inflight=4, max_queue=4, nstreams=2, max_batch_requests=4,
                max_batch_bytes=1 << 20, key_capacity=4, fault_every=0, fault_stage=0)
    for field, bad in (("budget_bytes", 0), ("max_inflight", 0), ("max_queue", 0), ("nstreams", 0),
                       ("nstreams", 17), ("max_batch_requests", 0), ("max_batch_bytes", 0), ("key_capacity", 0),
                       ("fault_stage", 2)):
        cfg = des3.des3_server_config_t(**dict(good, **{field: bad}))
        assert lib.des3_server_create(ctypes.byref(cfg), ctypes.byref(h)) == des3.DES3_EINVAL, field
    assert lib.des3_server_create(None, ctypes.byref(h)) == des3.DES3_EINVAL
    assert lib.des3_server_destroy(None) == des3.DES3_OK
    assert lib.des3_server_drain(None, 0) == des3.DES3_EINVAL


def test_tuning_table_set_get_reset_and_validation():
    from paper_1305_4376_gb300 import autotune
    autotune.reset()
    assert autotune.get_entry(des3.DES3_TUNE_SINGLE, 30)[1] == des3.DES3_KERNEL_BITSLICE
    assert autotune.get_entry(des3.DES3_TUNE_SINGLE, 12)[1] == des3.DES3_KERNEL_SPTABLE
    autotune.set_entries(des3.DES3_TUNE_SINGLE, [(30, des3.DES3_KERNEL_SPTABLE, 128, 3)])
    assert autotune.get_entry(des3.DES3_TUNE_SINGLE, 30) == (30, des3.DES3_KERNEL_SPTABLE, 128, 3)
    autotune.set_entries(des3.DES3_TUNE_SINGLE, [(29, des3.DES3_KERNEL_SPTABLE, 384, 3)])
    assert autotune.get_entry(des3.DES3_TUNE_SINGLE, 29) == (29, des3.DES3_KERNEL_SPTABLE, 384, 3)
    bad = [(30, des3.DES3_KERNEL_SPTABLE, 256, 4),       # 4 x 64.4 KiB of tables do not fit
           (30, des3.DES3_KERNEL_BITSLICE, 256, 2),      # 512 threads of a 168-register kernel
           (30, des3.DES3_KERNEL_SPTABLE, 512, 1),       # the table kernel is built for 384 threads at most
           (30, des3.DES3_KERNEL_BITSLICE, 96, 2),       # CTA size
           (40, des3.DES3_KERNEL_BITSLICE, 256, 2),      # class out of range
           (30, 7, 256, 2)]
    for e in bad:
        with pytest.raises(des3.Des3Error):
            autotune.set_entries(des3.DES3_TUNE_SINGLE, [e])
    autotune.set_entries(des3.DES3_TUNE_BATCH, [(20, des3.DES3_KERNEL_SPTABLE, 384, 3)])  # the batched table kernel
    assert autotune.get_entry(des3.DES3_TUNE_BATCH, 20) == (20, des3.DES3_KERNEL_SPTABLE, 384, 3)
    with pytest.raises(des3.Des3Error):
        autotune.set_entries(des3.DES3_TUNE_BATCH, [(20, des3.DES3_KERNEL_SPTABLE, 256, 4)])  # 4 x 68 KiB
    with pytest.raises(des3.Des3Error):
        autotune.set_entries(des3.DES3_TUNE_BATCH, [(20, des3.DES3_KERNEL_BITSLICE, 384, 2)])  # 768 bitsliced threads
    autotune.reset()
    assert autotune.get_entry(des3.DES3_TUNE_SINGLE, 30)[1] == des3.DES3_KERNEL_BITSLICE
    filled = autotune.fill_classes({12: (2, 256, 3), 20: (1, 256, 2)})
    assert len(filled) == 40 and filled[0][1] == 2 and filled[39][1] == 1 and filled[16][1] == 2


def test_built_in_tuning_tables_equal_the_committed_gb300_file():
    """The library's built-in tables (used until a tuning file is loaded) are
    the committed GB300 measurements, every class taking the nearest measured
    class's entry, in both tables."""
    import json
    from paper_1305_4376_gb300 import autotune
    doc = json.load(open(autotune.tuning_path("NVIDIA GB300")))
    autotune.reset()
    for name, table in (("single", des3.DES3_TUNE_SINGLE), ("batch", des3.DES3_TUNE_BATCH)):
        want = autotune.fill_classes({int(c): tuple(v) for c, v in doc[name].items()})
        got = [autotune.get_entry(table, c) for c in range(40)]
        assert got == want, name


def test_batch_choice_follows_the_measured_crossover_without_a_device():
    """des3_batch_choose on the host, built-in GB300 tables, 152 SMs: the
    choices the graph-replayed sweep of equal jobs measured as fastest."""
    from paper_1305_4376_gb300 import autotune
    autotune.reset()
    fake = 1 << 40
    bs, sp = des3.DES3_KERNEL_BITSLICE, des3.DES3_KERNEL_SPTABLE
    cases = [  # (jobs, bytes each, expected (kernel, threads, ctas_per_sm))
        (4096, 512, (sp, 256, 3)),        # 2 MiB: the tuning table (24.7 vs 127 us measured)
        (4096, 4096, (sp, 384, 3)),       # 16 MiB, fill 1/2: the wave model (114.9 vs 128.3 us)
        (4096, 8192, (bs, 256, 1)),       # 32 MiB, full tiles: the table (108.7 vs 224.1 us)
        (32768, 3584, (bs, 384, 1)),      # 112 MiB, fill 7/16: the model keeps it (750.5 vs 770.7 us)
        (32768, 512, (sp, 384, 3)),       # 16 MiB, fill 1/16: the model (118.6 vs 735.2 us)
        (1000, 8192, (bs, 384, 1)),       # below one bitsliced wave: the table decides
        (1, 256 << 10, (sp, 256, 3)),     # one 256 KiB job: the table
    ]
    for njobs, n, want in cases:
        jobs = des3.make_jobs([(fake, fake, n, 0, False)] * njobs)
        assert des3.des3_batch_choose(jobs, 152) == want, (njobs, n)
    # an explicit table without the table kernel is still overruled for sparse tiles
    autotune.set_entries(des3.DES3_TUNE_BATCH, [(c, bs, 384, 1) for c in range(40)])
    try:
        assert des3.des3_batch_choose(des3.make_jobs([(fake, fake, 512, 0, False)] * 4096), 152) == (sp, 384, 3)
        assert des3.des3_batch_choose(des3.make_jobs([(fake, fake, 512, 0, False)] * 100), 152) == (bs, 384, 1)
    finally:
        autotune.reset()
    lib = des3.lib()
    k = ctypes.c_int()
    bad = des3.make_jobs([(fake, fake, 12, 0, False)])
    assert lib.des3_batch_choose(bad, 1, 152, ctypes.byref(k), None, None) == des3.DES3_EINVAL
    assert lib.des3_batch_choose(des3.make_jobs([(fake, fake, 8, 0, False)]), 1, 0, ctypes.byref(k), None, None) \
        == des3.DES3_EINVAL
    assert lib.des3_batch_choose(None, 0, 152, ctypes.byref(k), None, None) == des3.DES3_OK


def test_single_des_key_schedule_matches_oracle():
    key = inputs.key_triple(4343)[:8]
    ks = des3.des3_key_schedule_des(key)
    assert ks.flags == des3.DES3_KS_SINGLE_DES and ks.magic == des3.DES3_KS_MAGIC
    sub = oracle.des_key_schedule(key)
    assert [ks.rk[0][r] for r in range(16)] == sub
    assert [ks.rk[1][r] for r in range(16)] == sub[::-1]
    assert all(ks.rk[0][r] == 0 for r in range(16, 48))


def test_plain_c_consumer(tmp_path):
    """include/des3.h is plain C: a C99 program includes it, links against
    libdes3gpu.so and calls the host-only entry points."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not installed")
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "consumer.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "des3.h"
int main(void) {
    uint8_t key[24];
    for (int i = 0; i < 24; i++) key[i] = (uint8_t)(i * 37 + 1);
    des3_ks_t ks;
    if (des3_key_schedule(key, &ks) != DES3_OK || ks.magic != DES3_KS_MAGIC) return 1;
    if (ks.rk[1][0] != ks.rk[0][47]) return 2;
    if (des3_self_test() != DES3_OK) return 3;
    if (des3_ecb_crypt_ex(&ks, NULL, NULL, 16, 0, DES3_KERNEL_AUTO, NULL) != DES3_EINVAL) return 4;
    des3_kernel_info_t info;
    if (des3_kernel_info(DES3_KERNEL_BITSLICE, &info) != DES3_OK || info.sbox_gates <= 0) return 5;
    printf("%s %s\n", des3_version(), des3_strerror(DES3_EKEY));
    return 0;
}
''')
    libdir = os.path.join(root, "paper_1305_4376_gb300")
    exe = tmp_path / "consumer"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src),
                    "-L", libdir, "-ldes3gpu", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, (res.returncode, res.stderr)
    assert "key schedule" in res.stdout


def test_batch_plan_rejects_an_unknown_kernel_without_device():
    lib = des3.lib()
    keys = des3.make_keys([des3.des3_key_schedule(inputs.key_triple(9))])
    fake = 1 << 40
    jobs = des3.make_jobs([(fake, fake, 64, 0, False)])
    h = ctypes.c_void_p()
    assert lib.des3_batch_plan_create(keys, 1, jobs, 1, 7, ctypes.byref(h)) == des3.DES3_EINVAL
    assert lib.des3_batch_plan_create(keys, 1, jobs, 1, -1, ctypes.byref(h)) == des3.DES3_EINVAL
    k = ctypes.c_int()
    assert lib.des3_batch_plan_kernel(None, ctypes.byref(k), None, None) == des3.DES3_EINVAL


def test_range_split_arithmetic():
    """The contiguous split des3_ecb_host_multi uses: covers every block once,
    boundaries on the granule, granule counts within one of each other and
    larger ranges first, empty ranges past the end."""
    cases = [(0, 1), (0, 3), (1, 1), (1, 4), (1023, 2), (1024, 2), (1025, 2), (5 * 1024 + 77, 3), (3 * 1024, 3),
             (3 * 1024, 8), ((1 << 29), 7), ((1 << 30) + 1, 5), (10 ** 12 + 3, 64)]
    for nblocks, nparts in cases:
        first = des3.des3_range_split(nblocks, nparts)
        assert len(first) == nparts + 1 and first[0] == 0 and first[-1] == nblocks
        assert all(a <= b for a, b in zip(first, first[1:]))
        assert all(b % 1024 == 0 or b == nblocks for b in first)
        units = [(b - a + 1023) // 1024 for a, b in zip(first, first[1:])]
        assert max(units) - min(units) <= 1
        assert units == sorted(units, reverse=True)
        assert sum(units) == (nblocks + 1023) // 1024
    assert des3.des3_range_split(10, 2, granule=4) == [0, 8, 10]
    lib = des3.lib()
    out = (ctypes.c_uint64 * 3)()
    assert lib.des3_range_split(10, 0, 1024, out) == des3.DES3_EINVAL
    assert lib.des3_range_split(10, 2, 0, out) == des3.DES3_EINVAL
    assert lib.des3_range_split(10, 2, 1024, None) == des3.DES3_EINVAL


def test_host_multi_argument_errors_without_device():
    lib = des3.lib()
    ks = des3.des3_key_schedule(bytes(range(24)))
    buf = (ctypes.c_uint8 * 64)()
    p = ctypes.addressof(buf)
    devs = (ctypes.c_int * 1)(0)
    work = (ctypes.c_void_p * 1)(None)
    sizes = (ctypes.c_size_t * 1)(0)
    kp = ctypes.byref(ks)
    assert lib.des3_ecb_host_multi(kp, p, p, 64, 0, 0, devs, work, sizes) == des3.DES3_EINVAL  # no device
    assert lib.des3_ecb_host_multi(kp, p, p, 64, 0, 65, devs, work, sizes) == des3.DES3_EINVAL  # too many
    assert lib.des3_ecb_host_multi(kp, p, p, 60, 0, 1, devs, work, sizes) == des3.DES3_EINVAL  # ragged size
    assert lib.des3_ecb_host_multi(kp, p, p, 64, 2, 1, devs, work, sizes) == des3.DES3_EINVAL  # direction
    assert lib.des3_ecb_host_multi(kp, p, p, 64, 0, 1, None, work, sizes) == des3.DES3_EINVAL
    assert lib.des3_ecb_host_multi(kp, p, p + 8, 48, 0, 1, devs, work, sizes) == des3.DES3_EINVAL  # overlap
    assert lib.des3_ecb_host_multi(kp, p, p, 0, 0, 1, devs, work, sizes) == des3.DES3_OK
    bad = des3.des3_ks_t()
    assert lib.des3_ecb_host_multi(ctypes.byref(bad), p, p, 64, 0, 1, devs, work, sizes) == des3.DES3_EKEY


def test_committed_tuning_tables_are_launchable():
    """Every committed launch table installs (each entry passes the library's
    resource checks for its kernel) and names a choice for all 40 size
    classes."""
    import glob
    import os
    from paper_1305_4376_gb300 import autotune
    files = glob.glob(os.path.join(autotune.TUNING_DIR, "*.json"))
    assert files
    try:
        for path in files:
            assert autotune.load_tuning(path)
            for table in (des3.DES3_TUNE_SINGLE, des3.DES3_TUNE_BATCH):
                for c in range(40):
                    e = autotune.get_entry(table, c)
                    assert e[0] == c and e[1] in (des3.DES3_KERNEL_BITSLICE, des3.DES3_KERNEL_SPTABLE)
    finally:
        autotune.reset()
